"""The momentum bound the decision-only GPU runs apply before the vertex (a
combination whose longitudinal momentum sum alone fails the |sum p| cut is not
fitted), checked on the FP64 oracle's combination records (Sec. "Vertex Fit"):

- its premise: |sum p| >= |P_z|, with P_z independent of the vertex position;
- its FP32 form (p cos(theta) per track rounded, the pair sum first, the square
  against the squared cut widened by a relative 1e-4) never removes a combination
  that passes the vertex cuts, here on frames that each carry a signal decay;
- it removes most of the combinations the vertex fits on the background workload."""
import numpy as np

from oracle import oracle as O
from paper_2206_11535_gb300 import gen


def _combos(c, d, nf):
    out = []
    for f in range(nf):
        o = O.select_frame(c, d["hits"][d["off"][f]:d["off"][f + 1]], records=True)
        for cb in o["combos"]:
            if cb.status == 2:
                pv = np.array([[cb.pvec[i][j] for j in range(3)] for i in range(3)])
                out.append((cb.pass_, cb.ptot, pv))
    return out


def _bound_fails(pz3, ptot_max):
    f = np.float32
    pz = (f(pz3[0]) + f(pz3[1])) + f(pz3[2])  # FP32, pair first, as the kernels add
    return f(pz) * f(pz) > f(ptot_max) * f(ptot_max) * f(1.0001)


def test_bound_premise_and_no_passing_combination_removed(ocfg):
    cfg = gen.load_config()
    ptot_max = cfg["cuts"]["ptot_max"]
    d = gen.generate(150, 10.0, 0.5, 1, seed=81)  # a signal decay in every frame
    combos = _combos(ocfg, d, 150)
    passing = [x for x in combos if x[0]]
    assert len(passing) > 50
    for _, ptot, pv in combos:
        assert ptot >= abs(pv[:, 2].sum()) * (1 - 1e-12)
    for _, _, pv in passing:
        assert not _bound_fails(pv[:, 2], ptot_max)


def test_bound_removes_most_fitted_background_combinations(ocfg):
    cfg = gen.load_config()
    d = gen.workload("c2", n_frames=120)
    combos = _combos(ocfg, d, 120)
    assert len(combos) > 500
    removed = np.mean([_bound_fails(pv[:, 2], cfg["cuts"]["ptot_max"]) for _, _, pv in combos])
    assert removed > 0.7, removed
