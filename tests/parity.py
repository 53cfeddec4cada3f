"""Frame-by-frame comparison of the CUDA path's candidate record with the FP64 oracle.

Integer decisions (selected triplets, tracks as hit quadruplets with their status,
energy-test combinations with vertex status and pass, frame reason) must be
identical, except where the oracle's value of the variable that takes the decision
lies inside that variable's boundary band.  A frame whose differences all lie
inside bands counts as "boundary"; each such difference is counted under the name
of its band (band_counts).  Values of matched candidates must agree within the
tolerances below.

Bands.  The selection cuts (Sec. "Selection Cuts") act on FP32 hit positions that
are the oracle's FP64 pixel centres rounded once: their band is 1e-5 relative to
the threshold.  Every later variable is computed in FP32 from the fitted tracks.
Its band was set from the largest difference between the CUDA path and the oracle
on matched candidates (matched_errors below): all 1,000 frames of the parity
workload in every form, 2,000 frames each of the throughput and uneven workloads
in the fused and plain forms, and 20,000 frames each of those two in the staged
form.  The band is four times that difference, rounded up to one significant
digit.  The differences are heavy-tailed (near-tangent circle pairs, long arcs):
the largest one grew with the sample, which is why the margin is wide.

  band          scale                                   measured max   band
  selection     threshold (Delta lambda, cos Phi, r_tc)  --             1e-5
  chi2_track    chi2 cut (32)                            4.5e-5         2e-4
  fourth_hit    mm, on sqrt(m_second) - sqrt(m_best)     2 x 7.1e-3     6e-2
  energy        energy window                            3.1e-5         2e-4
  vtx_chi2      vertex chi2 cut                          3.0e-4         2e-3
  tdist         target-distance cut                      5.2e-3         3e-2
  ptot          |sum p| cut                              4.5e-5         2e-4
  disc          |h^2| / (r_a r_b) of a circle pair       1.6e-3         7e-3
  filter        mm, | |point| - filter radius |          6.7e-3         3e-2
  choice        1 + chi2, on chi2_second - chi2          3.5e-3         2e-2

Values of matched candidates: the fitted curvature and polar angle within 1e-5
relative (largest differences 2.6e-6 and 7.2e-7); the chi2 of a kept track within
the chi2_track band; vertex values within band x threshold + VAL_REL x value
(far from the threshold, largest relative differences 1.7e-3, 7.6e-4 and 6.9e-5
for the vertex chi2, the target distance and |sum p|).

The 4th-hit metric m is a squared distance (mm^2) from the estimated layer-3 point;
the difference of sqrt(m) between the two sides is at most the displacement of
that point, so two hits swap places only when their sqrt(m) differ by less than
twice it.
"""
from __future__ import annotations

import math
from collections import Counter
from dataclasses import dataclass, field

from oracle import oracle as O

# boundary bands (see the table above)
BAND = dict(selection=1e-5, chi2_track=2e-4, fourth_hit=6e-2, energy=2e-4, vtx_chi2=2e-3, tdist=3e-2, ptot=2e-4,
            disc=7e-3, filter=3e-2, choice=2e-2)
# values of matched candidates: fitted curvature and polar angle, relative
KAPPA_REL = 1e-5
THETA_REL = 1e-5
# vertex values of matched combinations: |gpu - oracle| <= band * threshold + VAL_REL * |oracle|
# (far from the thresholds the vertex values are large and their error grows with them)
VAL_REL = dict(vtx_chi2=7e-3, tdist=4e-3, ptot=3e-4)


@dataclass
class FrameResult:
    frame: int
    status: str = "match"          # match | boundary | fail
    fails: list = field(default_factory=list)
    bounds: list = field(default_factory=list)  # (band name, details...)


def _near(v, thr, band):
    """v within band (relative to the threshold) of the threshold."""
    return abs(abs(v) - thr) <= band * abs(thr)


def _trip_boundary(c, hits_f, idx):
    hs = [O.decode(c, int(hits_f[i])) for i in idx]
    v = O.cut_vars(c, *[[h.x, h.y, h.z] for h in hs])
    cos01, cos12 = math.cos(c.phi01_max), math.cos(c.phi12_max)
    tests = [(abs(v[0]), c.dlambda_max), (v[1], cos01), (v[2], cos12), (abs(v[3]), c.rtc_min), (abs(v[3]), c.rtc_max)]
    return any(_near(a, b, BAND["selection"]) for a, b in tests), v


def _close(a, b, rel, abs_=0.0):
    return abs(a - b) <= rel * max(abs(a), abs(b)) + abs_


def compare_frame(c, hits_f, g: dict, f: int) -> FrameResult:
    """c: oracle config; hits_f: the frame's addresses; g: the GPU record of this frame
    (reason, n_trip, trip[n,4], trk_status[n], trk_val[n,4], n_combo, combo[m,4],
    combo_val[m,4], combo_aux[m,4])."""
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
            (R.bounds if nb >= abs(no - ng) else R.fails).append(("selection", "triplet-overflow", no, ng, nb))
        if int(g["reason"]) != o["reason"] and not R.bounds:
            R.fails.append(("reason", o["reason"], int(g["reason"])))
        return _finish(R)
    if ng != len(g_trip):
        R.fails.append(("duplicate-triplet", ng, len(g_trip)))
    for t in set(o_trip) ^ set(g_trip):
        b, v = _trip_boundary(c, hits_f, t)
        (R.bounds if b else R.fails).append(("selection", "triplet", t, "oracle" if t in o_trip else "gpu",
                                             v.tolist()))
    # ---------------- tracks of the common triplets
    bad_trk = set()
    addr = lambda i: int(hits_f[i]) if i >= 0 else -1  # noqa: E731
    chi2_abs = BAND["chi2_track"] * c.chi2_track_max
    for t in set(o_trip) & set(g_trip):
        ot = o["tracks"][o_trip[t]]
        gs = int(g["trk_status"][g_trip[t]])
        # the 4th hit is compared by pixel address: among duplicated addresses (distinct
        # hits, identical positions) either choice gives the same track
        gi3 = int(g["trip"][g_trip[t], 3])
        gi3 = next((j for j in range(len(hits_f)) if addr(j) == addr(gi3)), gi3) if gi3 >= 0 else gi3
        oi3 = next((j for j in range(len(hits_f)) if addr(j) == addr(ot.i[3])), -1) if ot.i[3] >= 0 else -1
        kb, th, chi2, mb = (float(x) for x in g["trk_val"][g_trip[t]])
        tie = (math.isfinite(ot.m_second) and
               math.sqrt(max(ot.m_second, 0.0)) - math.sqrt(max(ot.m_best, 0.0)) <= BAND["fourth_hit"])
        if ot.status != gs or (ot.status >= 3 and oi3 != gi3):
            why = None
            if oi3 != gi3 and tie:
                why = "fourth_hit"
            elif {ot.status, gs} == {4, 5} and _near(ot.chi2, c.chi2_track_max, BAND["chi2_track"]):
                why = "chi2_track"
            if why:
                R.bounds.append((why, "track", t, ot.status, gs, oi3, gi3, ot.chi2, chi2))
            else:
                R.fails.append(("track", t, ot.status, gs, oi3, gi3, ot.chi2, chi2))
            bad_trk.add(t)
            continue
        if gs == 5:  # a kept track: its fitted values (rejected fits only carry the chi2 decision)
            if not _close(ot.kappa_bar, kb, KAPPA_REL):
                R.fails.append(("kappa", t, ot.kappa_bar, kb))
            if not _close(ot.theta01, th, THETA_REL):
                R.fails.append(("theta01", t, ot.theta01, th))
            if abs(ot.chi2 - chi2) > chi2_abs:
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
            R.bounds.append(("track", "combo-of-boundary-track", key))
            continue
        de = o_cb[key].de if key in o_cb else float(g["combo_val"][g_cb[key], 0])
        (R.bounds if _near(de, c.e_window, BAND["energy"]) else R.fails).append(("energy", "combo", key, de))
    for key in set(o_cb) & set(g_cb):
        ob = o_cb[key]
        row = g["combo"][g_cb[key]]
        gst, gpass = int(row[3]) & 255, int(row[3]) >> 8
        gv = [float(x) for x in g["combo_val"][g_cb[key]]]
        # the geometric steps: how close a pair is to not meeting, a point to the filter
        # radius, two intersection choices to each other's chi2
        soft = []
        if ob.disc_min <= BAND["disc"]:
            soft.append("disc")
        if ob.filt_margin <= BAND["filter"]:
            soft.append("filter")
        if (ob.chi2_second - ob.chi2) <= BAND["choice"] * (1.0 + ob.chi2):
            soft.append("choice")
        if gst != ob.status:
            geo = [s for s in soft if s != "choice"]
            if geo:
                R.bounds.append((geo[0], "vertex-status", key, ob.status, gst, ob.disc_min, ob.filt_margin))
            else:
                R.fails.append(("vertex-status", key, ob.status, gst, ob.disc_min, ob.filt_margin))
            continue
        if gst == 2:
            near = [n for n, v, thr in (("vtx_chi2", ob.chi2, c.vtx_chi2_max), ("tdist", ob.tdist, c.target_dist_max),
                                        ("ptot", ob.ptot, c.ptot_max)) if _near(v, thr, BAND[n])]
            if gpass != ob.pass_:
                why = (near + soft)[:1]
                if why:
                    R.bounds.append((why[0], "vertex-pass", key, ob.pass_, gpass, ob.chi2, ob.tdist, ob.ptot, gv))
                else:
                    R.fails.append(("vertex-pass", key, ob.pass_, gpass, ob.chi2, ob.tdist, ob.ptot, gv))
            elif "choice" not in soft:
                for name, a, b, thr in (("vtx_chi2", ob.chi2, gv[1], c.vtx_chi2_max),
                                        ("tdist", ob.tdist, gv[2], c.target_dist_max),
                                        ("ptot", ob.ptot, gv[3], c.ptot_max)):
                    if abs(a - b) > BAND[name] * thr + VAL_REL[name] * abs(a):
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


def band_counts(results) -> dict:
    """Differences inside a boundary band, counted per band (frames without a failure)."""
    cnt = Counter()
    for r in results:
        if r.status == "boundary":
            for b in r.bounds:
                cnt[b[0]] += 1
    return {k: cnt.get(k, 0) for k in list(BAND) + ["track"]}


# Scale of each measured difference (matched_errors), as the band table states.
_FAR = 2.0  # vertex values farther than this factor from their threshold go to the *_value entries


def matched_errors(c, hits, off, rec: dict, frames=None) -> dict:
    """Largest difference between the CUDA path and the oracle over the candidates
    both sides agree on, per variable, on the scale of its band: the measurement the
    bands above were set from.  Entries: name -> [largest difference, candidates]."""
    out = {k: [0.0, 0] for k in ("kappa", "theta", "chi2_track", "fourth_hit", "energy", "vtx_chi2", "tdist", "ptot",
                                 "disc", "filter", "choice", "vtx_chi2_value", "tdist_value", "ptot_value")}

    def put(k, v):
        out[k][0] = max(out[k][0], float(v))
        out[k][1] += 1
    frames = range(len(off) - 1) if frames is None else frames
    for f in frames:
        hf = hits[off[f]:off[f + 1]]
        g = record_of_frame(rec, f)
        o = O.select_frame(c, hf, records=True, caps=(1100, 1100, 1100, 1100))
        ng = int(g["n_trip"])
        if o["n_triplets"] > c.max_triplets or ng > c.max_triplets:
            continue
        g_trip = {tuple(int(x) for x in g["trip"][k, :3]): k for k in range(min(ng, g["trip"].shape[0]))}
        o_trip = {tuple(t.i): k for k, t in enumerate(o["trips"])}
        for t in set(o_trip) & set(g_trip):
            ot = o["tracks"][o_trip[t]]
            k = g_trip[t]
            gi3 = int(g["trip"][k, 3])
            if int(g["trk_status"][k]) != ot.status or ot.status < 3 or int(hf[gi3]) != int(hf[ot.i[3]]):
                continue
            kb, th, chi2, mb = (float(x) for x in g["trk_val"][k])
            put("fourth_hit", abs(math.sqrt(max(mb, 0.0)) - math.sqrt(ot.m_best)))
            if ot.status == 5:
                put("kappa", abs(kb - ot.kappa_bar) / abs(ot.kappa_bar))
                put("theta", abs(th - ot.theta01) / abs(ot.theta01))
            if ot.status >= 4 and abs(ot.chi2 - c.chi2_track_max) <= 0.5 * c.chi2_track_max:
                put("chi2_track", abs(chi2 - ot.chi2) / c.chi2_track_max)
        if o["n_tracks"] > c.max_tracks or o["n_combos"] > c.max_combos or int(g["n_combo"]) > c.max_combos:
            continue
        first = {}
        for j in range(len(hf)):
            first.setdefault(int(hf[j]), j)
        canon = lambda i: first[int(hf[i])] if i >= 0 else -1  # noqa: E731
        okeys = [tuple(o["tracks"][ti].i[:3]) + (canon(o["tracks"][ti].i[3]),) for ti in o["kept"]]
        o_cb = {}
        for cb in o["combos"]:
            a, b, e = (okeys[k] for k in cb.t)
            o_cb[(tuple(sorted([a, b])), e)] = cb
        gk = {k: tuple(int(x) for x in g["trip"][k, :3]) + (canon(int(g["trip"][k, 3])),) for k in g_trip.values()}
        for k in range(min(int(g["n_combo"]), g["combo"].shape[0])):
            row = g["combo"][k]
            a, b, e = (gk.get(int(x), ("?",)) for x in row[:3])
            ob = o_cb.get((tuple(sorted([a, b])), e))
            if ob is None:
                continue
            gv = [float(x) for x in g["combo_val"][k]]
            ga = [float(x) for x in g["combo_aux"][k]]
            put("energy", abs(gv[0] - ob.de) / c.e_window)
            if math.isfinite(ob.disc_min) and ob.disc_min < 0.05 and ga[0] < 1e30:
                put("disc", abs(ga[0] - ob.disc_min))
            if math.isfinite(ob.filt_margin) and ob.filt_margin < 1.0 and ga[1] < 1e30:
                put("filter", abs(ga[1] - ob.filt_margin))
            if int(row[3]) & 255 != 2 or ob.status != 2:
                continue
            gap = ob.chi2_second - ob.chi2
            if math.isfinite(ob.chi2_second) and ga[2] < 1e30 and gap < 0.1 * (1.0 + ob.chi2):
                put("choice", abs((ga[2] - gv[1]) - gap) / (1.0 + ob.chi2))
            if gap <= BAND["choice"] * (1.0 + ob.chi2):
                continue  # the two sides may take different intersection choices
            for name, ov, gvv, thr in (("vtx_chi2", ob.chi2, gv[1], c.vtx_chi2_max),
                                       ("tdist", ob.tdist, gv[2], c.target_dist_max),
                                       ("ptot", ob.ptot, gv[3], c.ptot_max)):
                if thr / _FAR <= ov <= _FAR * thr:
                    put(name, abs(gvv - ov) / thr)
                elif ov > _FAR * thr:
                    put(name + "_value", abs(gvv - ov) / ov)
    return out
