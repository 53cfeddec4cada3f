"""Calibrate the cut values the paper does not print and freeze them in the JSON
parameter file (``paper_2206_11535_gb300/configs/default.json``).

TEST INFRASTRUCTURE: this script calls only the FP64 oracle and the seeded input
generator.  Run:  ``python oracle/calibrate.py [--write]``.

Readings (the paper gives the cut quantities but not their values):
  * Selection cuts (Sec. "Selection Cuts"): each window keeps a fraction Q_SEL of
    the truth triplets (three hits of one track on layers 0, 1, 2) of a calibration
    sample; |r_tc| is a two-sided window.  The paper's aggregates are then checked:
    > 95 % of all combinations removed, > 98.5 % of true triplets kept, the first
    cut alone removing > 80 %.
  * Vertex cuts (Sec. "Vertex Fit", Algorithm 4): on frames that carry a
    reconstructable signal decay (all three tracks with four hits and all three
    reconstructed), each of energy window, vertex chi2, target distance and total
    momentum is set, in that order, to keep Q_VTX of the frames still passing.
The calibration sample uses seed 1001, distinct from every test and bench seed.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path = [q for q in sys.path if os.path.abspath(q or ".") != HERE]
sys.path.insert(0, os.path.dirname(HERE))

from oracle import oracle as O  # noqa: E402
from paper_2206_11535_gb300 import gen  # noqa: E402

Q_SEL = 0.997
Q_VTX = 0.99
SEED = 1001


def _positions(c, addrs):
    out = np.zeros((len(addrs), 3))
    for i, a in enumerate(addrs):
        h = O.decode(c, int(a))
        out[i] = (h.x, h.y, h.z)
    return out


def truth_triplet_vars(c, d):
    """Cut variables of every truth triplet (hits of one track on layers 0,1,2)."""
    ht, lay = d["hit_track"], d["hit_layer"]
    sel = ht >= 0
    idx = np.nonzero(sel)[0]
    order = idx[np.lexsort((lay[idx], ht[idx]))]
    vs = []
    i = 0
    while i < order.size:
        t = ht[order[i]]
        j = i
        while j < order.size and ht[order[j]] == t:
            j += 1
        group = order[i:j]
        ls = lay[group]
        if all((ls == L).sum() == 1 for L in (0, 1, 2)):
            g3 = [group[ls == L][0] for L in (0, 1, 2)]
            p = _positions(c, d["hits"][g3])
            vs.append(O.cut_vars(c, p[0], p[1], p[2]))
        i = j
    return np.array(vs)


def all_triplet_vars(c, d, n_frames):
    """Cut variables of every layer-0/1/2 combination of the first frames (fills the
    lattice of values that digitised hits can produce)."""
    out = []
    for f in range(n_frames):
        a, b = d["off"][f], d["off"][f + 1]
        lay = d["hit_layer"][a:b]
        pos = _positions(c, d["hits"][a:b])
        for i0 in np.nonzero(lay == 0)[0]:
            for i1 in np.nonzero(lay == 1)[0]:
                for i2 in np.nonzero(lay == 2)[0]:
                    out.append(O.cut_vars(c, pos[i0], pos[i1], pos[i2]))
    return np.array(out)


def off_lattice(thr, values, upward):
    """Digitised hits make the cut variables take discrete values (Delta lambda lives
    on a lattice of step pitch / (r2 - r1)), and a quantile lands on one of them.  Move
    the threshold halfway to the next distinct value beyond it, so that no achievable
    value sits on the threshold and the decision never hangs on rounding."""
    u = np.unique(np.round(values, 9))  # one entry per lattice point despite rounding
    t = round(float(thr), 9)
    nxt = u[u > t] if upward else u[u < t][::-1]
    return float(0.5 * (thr + nxt[0])) if nxt.size else float(thr)


def calibrate_selection(cfg):
    c = O.make_config(cfg)
    d = gen.generate(4000, 10.0, 0.5, 10, seed=SEED)
    v = truth_triplet_vars(c, d)
    w = all_triplet_vars(c, d, 200)
    q = Q_SEL
    cuts = cfg["cuts"]
    cuts["dlambda_max"] = off_lattice(np.quantile(np.abs(v[:, 0]), q), np.abs(np.r_[v[:, 0], w[:, 0]]), True)
    ph01 = np.arccos(np.clip(np.r_[v[:, 1], w[:, 1]], -1, 1))
    ph12 = np.arccos(np.clip(np.r_[v[:, 2], w[:, 2]], -1, 1))
    cuts["phi01_max"] = off_lattice(np.quantile(np.arccos(np.clip(v[:, 1], -1, 1)), q), ph01, True)
    cuts["phi12_max"] = off_lattice(np.quantile(np.arccos(np.clip(v[:, 2], -1, 1)), q), ph12, True)
    r = np.abs(v[:, 3])
    rall = np.abs(np.r_[v[:, 3], w[:, 3]])
    rall = rall[np.isfinite(rall)]
    cuts["rtc_min"] = off_lattice(np.quantile(r, (1 - q) / 2), rall, False)
    cuts["rtc_max"] = off_lattice(np.quantile(r, 1 - (1 - q) / 2), rall, True)
    return cfg


def selection_report(cfg, n_frames=1000, seed=SEED + 1):
    c = O.make_config(cfg)
    d = gen.generate(n_frames, 10.0, 0.5, 10, seed=seed)
    v = truth_triplet_vars(c, d)
    cu = cfg["cuts"]
    ok = ((np.abs(v[:, 0]) <= cu["dlambda_max"]) & (v[:, 1] >= math.cos(cu["phi01_max"]))
          & (v[:, 2] >= math.cos(cu["phi12_max"])) & (np.abs(v[:, 3]) >= cu["rtc_min"])
          & (np.abs(v[:, 3]) <= cu["rtc_max"]))
    tested = 0
    passed = np.zeros(4)
    for f in range(n_frames):
        o = O.select_frame(c, d["hits"][d["off"][f]:d["off"][f + 1]], records=False)
        tested += o["n_tested"]
        passed += np.array(o["n_pass"])
    return dict(true_kept=float(ok.mean()), removed_total=float(1 - passed[3] / tested),
                removed_cut1=float(1 - passed[0] / tested), kept_after_each=(passed / tested).tolist())


def _truth_tracks_of_frame(d, f):
    a, b = d["off"][f], d["off"][f + 1]
    return d["hit_track"][a:b]


def signal_quantities(cfg, n_frames=3000, seed=SEED):
    """For frames with a reconstructable signal decay, the energy deviation, vertex chi2,
    target distance and total momentum of the combination of the three truth tracks,
    computed by the oracle with the vertex cuts open."""
    open_cfg = json.loads(json.dumps(cfg))
    for k in ("e_window", "vtx_chi2_max", "target_dist_max", "ptot_max"):
        open_cfg["cuts"][k] = 1e30
    c = O.make_config(open_cfg)
    d = gen.generate(n_frames, 10.0, 0.5, 1, seed=seed)
    out = []
    n_recon = 0
    for f in range(n_frames):
        a, b = d["off"][f], d["off"][f + 1]
        ht = d["hit_track"][a:b]
        sig_tracks = [t for t in np.unique(ht[ht >= 0]) if d["trk_signal"][t]]
        if len(sig_tracks) != 3 or any(d["trk_n_hits"][t] != 4 for t in sig_tracks):
            continue
        n_recon += 1
        o = O.select_frame(c, d["hits"][a:b], records=True)
        if o["reason"] not in (O.DROP, O.VERTEX):
            continue
        # kept tracks whose four hits are all of one signal track
        kt = {}
        for ki, ti in enumerate(o["kept"]):
            tr = o["tracks"][ti]
            owners = {int(ht[i]) for i in tr.i}
            if len(owners) == 1 and owners.pop() in sig_tracks:
                kt[ki] = int(ht[tr.i[0]])
        if len(set(kt.values())) != 3:
            continue
        for cb in o["combos"]:
            if all(t in kt for t in cb.t) and len({kt[t] for t in cb.t}) == 3:
                out.append((abs(cb.de), cb.chi2, cb.tdist, cb.ptot, cb.status))
                break
    return np.array(out), n_recon


def calibrate_vertex(cfg):
    q, n_recon = signal_quantities(cfg)
    good = q[q[:, 4] == 2]
    cu = cfg["cuts"]
    e = np.quantile(q[:, 0], Q_VTX)
    cu["e_window"] = float(e)
    s = good[good[:, 0] <= e]
    cu["vtx_chi2_max"] = float(np.quantile(s[:, 1], Q_VTX))
    s = s[s[:, 1] <= cu["vtx_chi2_max"]]
    cu["target_dist_max"] = float(np.quantile(s[:, 2], Q_VTX))
    s = s[s[:, 2] <= cu["target_dist_max"]]
    cu["ptot_max"] = float(np.quantile(s[:, 3], Q_VTX))
    return cfg, dict(n_recon_frames=n_recon, n_truth_combos=len(q), n_vertexed=len(good))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--write", action="store_true")
    args = ap.parse_args()
    cfg = gen.load_config()
    cfg = calibrate_selection(cfg)
    print("selection cuts:", {k: cfg["cuts"][k] for k in ("dlambda_max", "phi01_max", "phi12_max", "rtc_min",
                                                          "rtc_max")})
    print("selection report:", selection_report(cfg))
    cfg, info = calibrate_vertex(cfg)
    print("vertex calibration:", info)
    print("vertex cuts:", {k: cfg["cuts"][k] for k in ("e_window", "vtx_chi2_max", "target_dist_max", "ptot_max")})
    if args.write:
        for k, v in cfg["cuts"].items():
            if isinstance(v, float):
                cfg["cuts"][k] = float("%.9g" % v)
        with open(gen.config_path(), "w") as f:
            json.dump(cfg, f, indent=2)
            f.write("\n")
        print("wrote", gen.config_path())


if __name__ == "__main__":
    main()
