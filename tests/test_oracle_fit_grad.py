"""Pins of the oracle's track-fit chi2 under layer alignment and field scale, and of
its central-difference gradient (the reference for the gradient kernel).

The chi2 of a track (Sec. "Track Reconstruction", global chi2 at the mean
curvature) depends on the hit positions only through chords, axial distances and
the transverse circle: it is exactly invariant under a common translation of all
layers and a common rotation about the field axis.  The field scale enters only
through the multiple-scattering width sigma_MS ~ 1/p, and the inverse-variance
weights of the two triplets scale alike, so chi2 is exactly quadratic in it.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2206_11535_gb300 import gen


def _kept_candidates(c, d, max_frames=None, min_status=5):
    """Quadruplets (global hit indices) of the oracle's tracks with status >= min_status."""
    cand, chi2 = [], []
    off = d["off"]
    nf = off.size - 1 if max_frames is None else min(max_frames, off.size - 1)
    for f in range(nf):
        o = O.select_frame(c, d["hits"][off[f]:off[f + 1]], records=True)
        for t in o["tracks"]:
            if t.status >= min_status:
                cand.append([off[f] + i for i in t.i])
                chi2.append(t.chi2)
    return np.array(cand, np.int32).reshape(-1, 4), np.array(chi2)


@pytest.fixture(scope="module")
def c1_cands(ocfg):
    d = gen.workload("c1", n_frames=300)
    cand, chi2 = _kept_candidates(ocfg, d)
    assert cand.shape[0] > 500
    return d, cand, chi2


def _random_params(seed, scale_t=0.05, scale_r=5e-4):
    rng = np.random.default_rng(seed)
    p = O.nominal_params()
    for L in range(4):
        p[6 * L:6 * L + 3] = rng.normal(0, scale_t, 3)
        p[6 * L + 3:6 * L + 6] = rng.normal(0, scale_r, 3)
    return p


def test_rotation_convention():
    """R = Rz(wz) Ry(wy) Rx(wx): x is rotated first; hand cases that tell the order apart."""
    q = math.pi / 2
    np.testing.assert_allclose(O.align_point([0, 0, 0, q, 0, q], [0, 0, 1]), [1, 0, 0], atol=1e-15)
    np.testing.assert_allclose(O.align_point([0, 0, 0, q, 0, q], [1, 0, 0]), [0, 1, 0], atol=1e-15)
    np.testing.assert_allclose(O.align_point([0, 0, 0, 0, q, 0], [1, 0, 0]), [0, 0, -1], atol=1e-15)
    np.testing.assert_allclose(O.align_point([1, 2, 3, 0, 0, 0], [4, 5, 6]), [5, 7, 9], atol=1e-15)
    # rigid: lengths and angles kept, orthonormal columns
    w = [0.3, -0.2, 0.7]
    cols = np.array([O.align_point([0, 0, 0, *w], e) for e in np.eye(3)]).T
    np.testing.assert_allclose(cols.T @ cols, np.eye(3), atol=1e-14)
    assert abs(np.linalg.det(cols) - 1) < 1e-14
    # small angles: R ~ I + [w]x
    w = np.array([1e-7, -2e-7, 3e-7])
    x = np.array([25.0, 3.0, -40.0])
    # first order in w: the rest is bounded by |w|^2 |x|
    np.testing.assert_allclose(O.align_point([0, 0, 0, *w], x) - x, np.cross(w, x), rtol=0,
                               atol=float(w @ w) * np.linalg.norm(x))


def test_nominal_alignment_reproduces_the_selection_chi2(ocfg, c1_cands):
    d, cand, chi2 = c1_cands
    got = O.fit_chi2(ocfg, d["hits"], cand, O.nominal_params(), 4)
    np.testing.assert_allclose(got, chi2, rtol=1e-12, atol=1e-12)
    # a hit on the wrong layer, an index out of range: no chi2
    bad = cand[:2].copy()
    bad[0, [0, 1]] = bad[0, [1, 0]]
    bad[1, 3] = d["hits"].size
    assert np.isnan(O.fit_chi2(ocfg, d["hits"], bad, O.nominal_params())).all()


def test_common_translation_and_z_rotation_leave_chi2(ocfg, c1_cands):
    d, cand, _ = c1_cands
    p = _random_params(3)
    base = O.fit_chi2(ocfg, d["hits"], cand, p, 4)
    t = np.array([0.7, -1.3, 2.1])
    pt = p.copy()
    for L in range(4):
        pt[6 * L:6 * L + 3] += t
    np.testing.assert_allclose(O.fit_chi2(ocfg, d["hits"], cand, pt, 4), base, rtol=1e-8, atol=1e-9)
    # rotating every layer by delta about z: wz += delta and d -> Rz(delta) d
    delta = 0.37
    cz, sz = math.cos(delta), math.sin(delta)
    pr = p.copy()
    for L in range(4):
        dx, dy = p[6 * L], p[6 * L + 1]
        pr[6 * L], pr[6 * L + 1] = cz * dx - sz * dy, sz * dx + cz * dy
        pr[6 * L + 5] += delta
    np.testing.assert_allclose(O.fit_chi2(ocfg, d["hits"], cand, pr, 4), base, rtol=1e-8, atol=1e-9)
    # a rotation about x is not a symmetry (the field is along z)
    px = p.copy()
    for L in range(4):
        px[6 * L + 3] += 0.01
    assert not np.allclose(O.fit_chi2(ocfg, d["hits"], cand, px, 4), base, rtol=1e-3)


def test_chi2_is_quadratic_in_the_field_scale(ocfg, c1_cands):
    d, cand, _ = c1_cands
    p = _random_params(5)
    base = O.fit_chi2(ocfg, d["hits"], cand, p, 4)
    for s in (0.5, 1.001, 3.0):
        ps = p.copy()
        ps[24] = s
        np.testing.assert_allclose(O.fit_chi2(ocfg, d["hits"], cand, ps, 4), s * s * base, rtol=1e-10)


def test_fd_gradient_obeys_the_symmetries(ocfg, c1_cands):
    """The central-difference gradient: zero along the common translations and the
    common z-rotation (whose tangent moves wz_L by 1 and d_L by (-d_y, d_x, 0)),
    and 2 chi2 / s along the field scale."""
    d, cand, _ = c1_cands
    p = _random_params(7)
    tot, g, ok = O.fit_grad_fd(ocfg, d["hits"], cand, p, 4)
    assert ok.all()
    gn = np.abs(g[:24]).max()
    assert gn > 1.0
    for k in range(3):
        assert abs(sum(g[6 * L + k] for L in range(4))) < 1e-6 * gn
    rot = sum(g[6 * L + 5] - g[6 * L] * p[6 * L + 1] + g[6 * L + 1] * p[6 * L] for L in range(4))
    assert abs(rot) < 1e-6 * gn
    assert g[24] == pytest.approx(2.0 * tot / p[24], rel=1e-7)
    # directional derivative = finite difference of the sum along a random direction
    rng = np.random.default_rng(11)
    v = rng.normal(size=25) * np.array(O.FD_STEPS) * 100
    h = 1e-2
    fp = np.nansum(O.fit_chi2(ocfg, d["hits"], cand, p + h * v, 4))
    fm = np.nansum(O.fit_chi2(ocfg, d["hits"], cand, p - h * v, 4))
    assert (fp - fm) / (2 * h) == pytest.approx(float(g @ v), rel=1e-5)


def test_injected_misalignment_is_the_better_fit(ocfg):
    """Frames from a displaced detector (c4 truth): the true alignment fits better
    than the nominal one, and the gradient at nominal points towards the truth."""
    d = gen.workload("c4", n_frames=300)
    cand, _ = _kept_candidates(ocfg, d, min_status=4)
    # truth-matched tracks only (all four hits from one generated track): fake
    # combinations have chi2 of any size and carry no alignment information
    trk = d["hit_track"][cand]
    cand = cand[(trk[:, 0] >= 0) & (trk == trk[:, :1]).all(1)]
    assert cand.shape[0] > 1000
    truth = O.nominal_params()
    truth[:24] = d["truth_align"].reshape(-1)
    truth[24] = d["truth_b_scale"]
    nominal = O.nominal_params()
    s_nom = np.nansum(O.fit_chi2(ocfg, d["hits"], cand, nominal, 4))
    s_true = np.nansum(O.fit_chi2(ocfg, d["hits"], cand, truth, 4))
    assert s_true < 0.9 * s_nom
    _, g, _ = O.fit_grad_fd(ocfg, d["hits"], cand, nominal, 4)
    step = truth - nominal
    step[24] = 0.0  # the field scale is not identifiable from the chi2 sum (quadratic)
    assert float(g @ step) < 0.0
