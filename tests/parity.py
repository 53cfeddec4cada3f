"""Frame-by-frame comparison of the CUDA path's candidate record with the FP64 oracle.

Integer decisions (selected triplets, tracks as hit quadruplets, energy-test
combinations, vertex pass, frame reason) must be identical, except where the
oracle's cut variable for the candidate lies inside the boundary band of its
threshold; a frame whose differences are all such candidates counts as
"boundary".  Floating-point results of matched candidates must agree within the
tolerances below.

Bands and tolerances:
  BAND_REL   1e-5 relative to the threshold for every cut variable (selection
             cuts, chi2 < 32, energy window, vertex cuts);
  KAPPA_REL, THETA_REL  1e-5 relative for the global curvature and theta01;
  the energy, vertex and 4th-hit quantities are computed from the fitted
  curvatures, so their bands add the propagation of KAPPA_REL (see DERIVED).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from oracle import oracle as O

BAND_REL = 1e-5
KAPPA_REL = 1e-5
THETA_REL = 1e-5
# derived quantities: relative tolerance of values computed from the fitted tracks
DERIVED_REL = 2e-3
DERIVED_ABS = 2e-3


@dataclass
class FrameResult:
    frame: int
    status: str = "match"          # match | boundary | fail
    fails: list = field(default_factory=list)
    bounds: list = field(default_factory=list)


def _near(v, thr, rel=BAND_REL, extra=0.0):
    return abs(abs(v) - thr) <= rel * abs(thr) + extra


def _trip_boundary(c, hits_f, idx):
    hs = [O.decode(c, int(hits_f[i])) for i in idx]
    v = O.cut_vars(c, *[[h.x, h.y, h.z] for h in hs])
    cos01, cos12 = math.cos(c.phi01_max), math.cos(c.phi12_max)
    tests = [(abs(v[0]), c.dlambda_max), (v[1], cos01), (v[2], cos12), (abs(v[3]), c.rtc_min), (abs(v[3]), c.rtc_max)]
    return any(_near(a, b) for a, b in tests), v


def _close(a, b, rel, abs_=0.0):
    return abs(a - b) <= rel * max(abs(a), abs(b)) + abs_


def compare_frame(c, hits_f, g: dict, f: int) -> FrameResult:
    """c: oracle config; hits_f: the frame's addresses; g: the GPU record of this frame
    (reason, n_trip, trip[n,4], trk_status[n], trk_val[n,4], n_combo, combo[m,4], combo_val[m,4])."""
    R = FrameResult(f)
    o = O.select_frame(c, hits_f, records=True, caps=(1100, 1100, 1100, 1100))
    # ---------------- triplets
    no, ng = o["n_triplets"], int(g["n_trip"])
    over_o, over_g = no > c.max_triplets, ng > c.max_triplets
    o_trip = {tuple(t.i): k for k, t in enumerate(o["trips"])}
    g_trip = {}
    if not over_g:
        for k in range(min(ng, g["trip"].shape[0])):
            g_trip[tuple(int(x) for x in g["trip"][k, :3])] = k
    if over_o or over_g:
        if over_o != over_g:
            # one side overflows: the count difference must come from boundary triplets
            nb = sum(_trip_boundary(c, hits_f, t)[0] for t in o_trip)
            (R.bounds if nb >= abs(no - ng) else R.fails).append(("triplet-overflow", no, ng, nb))
        if int(g["reason"]) != o["reason"] and not R.bounds:
            R.fails.append(("reason", o["reason"], int(g["reason"])))
        return _finish(R)
    if ng != len(g_trip):
        R.fails.append(("duplicate-triplet", ng, len(g_trip)))
    for t in set(o_trip) ^ set(g_trip):
        b, v = _trip_boundary(c, hits_f, t)
        (R.bounds if b else R.fails).append(("triplet", t, "oracle" if t in o_trip else "gpu", v.tolist()))
    # ---------------- tracks of the common triplets
    bad_trk = set()
    addr = lambda i: int(hits_f[i]) if i >= 0 else -1  # noqa: E731
    for t in set(o_trip) & set(g_trip):
        ot = o["tracks"][o_trip[t]]
        gs = int(g["trk_status"][g_trip[t]])
        # the 4th hit is compared by pixel address: among duplicated addresses (distinct
        # hits, identical positions) either choice gives the same track
        gi3 = int(g["trip"][g_trip[t], 3])
        gi3 = next((j for j in range(len(hits_f)) if addr(j) == addr(gi3)), gi3) if gi3 >= 0 else gi3
        oi3 = next((j for j in range(len(hits_f)) if addr(j) == addr(ot.i[3])), -1) if ot.i[3] >= 0 else -1
        kb, th, chi2, mb = (float(x) for x in g["trk_val"][g_trip[t]])
        tie = (ot.m_second - ot.m_best) <= DERIVED_REL * (1.0 + ot.m_best)
        if ot.status != gs or (ot.status >= 3 and oi3 != gi3):
            why = []
            if oi3 != gi3 and tie:
                why.append("4th-hit tie")
            if {ot.status, gs} == {4, 5} and _near(ot.chi2, c.chi2_track_max, DERIVED_REL):
                why.append("chi2 at cut")
            (R.bounds if why else R.fails).append(("track", t, ot.status, gs, oi3, gi3, why, ot.chi2, chi2))
            bad_trk.add(t)
            continue
        if gs == 5:  # a kept track: its fitted values (rejected fits only carry the chi2 decision)
            if not _close(ot.kappa_bar, kb, KAPPA_REL):
                R.fails.append(("kappa", t, ot.kappa_bar, kb))
            if not _close(ot.theta01, th, THETA_REL):
                R.fails.append(("theta01", t, ot.theta01, th))
            if not _close(ot.chi2, chi2, DERIVED_REL, DERIVED_ABS):
                R.fails.append(("chi2", t, ot.chi2, chi2))
    # ---------------- track overflow
    nko, nkg = o["n_tracks"], sum(1 for t, k in g_trip.items() if int(g["trk_status"][k]) == 5)
    if nko > c.max_tracks or nkg > c.max_tracks or o["reason"] == O.TRACK_OVERFLOW:
        if (nko > c.max_tracks) != (nkg > c.max_tracks) and not R.bounds:
            R.fails.append(("track-overflow", nko, nkg))
        if int(g["reason"]) != o["reason"] and not R.bounds:
            R.fails.append(("reason", o["reason"], int(g["reason"])))
        return _finish(R)
    # ---------------- combinations
    first = {}
    for j in range(len(hits_f)):
        first.setdefault(int(hits_f[j]), j)
    canon = lambda i: first[int(hits_f[i])] if i >= 0 else -1  # noqa: E731
    o_trkkey = [tuple(o["tracks"][ti].i[:3]) + (canon(o["tracks"][ti].i[3]),) for ti in o["kept"]]
    def okey(cb):
        a, b, e = (o_trkkey[k] for k in cb.t)
        return (tuple(sorted([a, b])), e)
    g_tripkey = {k: tuple(int(x) for x in g["trip"][k, :3]) + (canon(int(g["trip"][k, 3])),) for k in g_trip.values()}
    def gkey(row):
        a, b, e = (g_tripkey.get(int(k), ("?",)) for k in row[:3])
        return (tuple(sorted([a, b])), e)
    o_cb = {okey(cb): cb for cb in o["combos"]}
    nco, ncg = o["n_combos"], int(g["n_combo"])
    over_o, over_g = nco > c.max_combos, ncg > c.max_combos
    g_cb = {}
    if not over_g:
        for k in range(min(ncg, g["combo"].shape[0])):
            g_cb[gkey(g["combo"][k])] = k
    bad_keys = {tuple(t) for t in bad_trk}
    def involves_bad(key):
        (a, b), e = key
        return any(tuple(q[:3]) in bad_keys for q in (a, b, e))
    if over_o or over_g:
        if over_o != over_g and not R.bounds:
            R.fails.append(("combo-overflow", nco, ncg))
        if int(g["reason"]) != o["reason"] and not R.bounds:
            R.fails.append(("reason", o["reason"], int(g["reason"])))
        return _finish(R)
    for key in set(o_cb) ^ set(g_cb):
        if involves_bad(key):
            R.bounds.append(("combo-of-boundary-track", key))
            continue
        de = o_cb[key].de if key in o_cb else float(g["combo_val"][g_cb[key], 0])
        band = DERIVED_REL * c.e_window
        (R.bounds if _near(de, c.e_window, 0.0, band) else R.fails).append(("combo", key, de))
    for key in set(o_cb) & set(g_cb):
        ob = o_cb[key]
        row = g["combo"][g_cb[key]]
        gst, gpass = int(row[3]) & 255, int(row[3]) >> 8
        gv = [float(x) for x in g["combo_val"][g_cb[key]]]
        soft = (ob.disc_min <= DERIVED_REL or ob.filt_margin <= DERIVED_ABS * 10
                or (ob.chi2_second - ob.chi2) <= DERIVED_REL * (1.0 + ob.chi2))
        if gst != ob.status:
            (R.bounds if soft else R.fails).append(("vertex-status", key, ob.status, gst, ob.disc_min, ob.filt_margin))
            continue
        if gst == 2:
            near = (_near(ob.chi2, c.vtx_chi2_max, DERIVED_REL) or _near(ob.tdist, c.target_dist_max, DERIVED_REL)
                    or _near(ob.ptot, c.ptot_max, DERIVED_REL))
            if gpass != ob.pass_:
                (R.bounds if (near or soft) else R.fails).append(("vertex-pass", key, ob.pass_, gpass,
                                                                  ob.chi2, ob.tdist, ob.ptot, gv))
            elif not soft:
                for name, a, b in (("vtx-chi2", ob.chi2, gv[1]), ("tdist", ob.tdist, gv[2]), ("ptot", ob.ptot, gv[3])):
                    if not _close(a, b, DERIVED_REL, DERIVED_ABS):
                        R.fails.append((name, key, a, b))
    if int(g["reason"]) != o["reason"] and not R.bounds:
        R.fails.append(("reason", o["reason"], int(g["reason"])))
    return _finish(R)


def _finish(R: FrameResult) -> FrameResult:
    R.status = "fail" if R.fails else ("boundary" if R.bounds else "match")
    return R


def record_of_frame(rec: dict, f: int) -> dict:
    """Slice one frame out of a numpy copy of the debug record."""
    return {k: (v[f] if k not in ("cap",) else v) for k, v in rec.items()}


def compare_batch(c, hits, off, rec: dict, frames=None):
    """rec: numpy arrays from Context.select_frames_debug.  Returns list of FrameResult."""
    out = []
    frames = range(len(off) - 1) if frames is None else frames
    for f in frames:
        g = record_of_frame(rec, f)
        out.append(compare_frame(c, hits[off[f]:off[f + 1]], g, f))
    return out


def summary(results) -> dict:
    s = {"match": 0, "boundary": 0, "fail": 0}
    for r in results:
        s[r.status] += 1
    return s
