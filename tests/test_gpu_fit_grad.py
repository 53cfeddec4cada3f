"""Gradient of the summed track chi2 (m3e_fit_grad) on the GPU against the FP64
oracle: chi2 per candidate, the sum and its central-difference gradient, the
exact symmetries, the autograd wrapper, determinism and edge cases."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2206_11535_gb300 import gen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# Tolerances.  chi2 of one candidate: FP32 fit vs FP64, relative to the value plus
# the track-chi2 band of the selection's parity check (2e-4 of the cut, 32), which
# also covers the displaced geometries.  Gradient: every component within 1e-3 of
# itself, plus a noise floor GRAD_FLOOR times the largest component: a component
# is a sum over thousands of candidates of FP32 terms of both signs, so one that
# cancels to almost nothing keeps the rounding of the terms, not of itself.
CHI2_REL, CHI2_ABS = 1e-4, 6.4e-3
GRAD_REL = 1e-3
GRAD_FLOOR = 5e-5


@pytest.fixture(scope="module")
def m3e():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_11535_gb300 import m3e as mod
    return mod


@pytest.fixture(scope="module")
def c4(m3e, cfg):
    """c4 frames (displaced layers), the tracks the GPU selection kept at nominal
    geometry, restricted to truth-matched ones for the gradient checks."""
    d = gen.workload("c4", n_frames=1500)
    with m3e.Context(cfg, 0) as ctx:
        hits, off = torch.from_numpy(d["hits"]).cuda(), torch.from_numpy(d["off"]).cuda()
        rec = {k: v.cpu().numpy() for k, v in ctx.select_frames_debug(hits, off).items()}
    cand = m3e.kept_candidates(rec, d["off"])
    trk = d["hit_track"][cand]
    truth_matched = (trk[:, 0] >= 0) & (trk == trk[:, :1]).all(1)
    truth = O.nominal_params()
    truth[:24] = d["truth_align"].reshape(-1)
    truth[24] = d["truth_b_scale"]
    return dict(d=d, rec=rec, cand=cand, tm=np.ascontiguousarray(cand[truth_matched]), truth=truth)


def _dev(d, cand, params):
    return (torch.from_numpy(d["hits"]).cuda(), torch.from_numpy(d["off"]).cuda(),
            torch.from_numpy(np.ascontiguousarray(cand, np.int32)).cuda(),
            torch.tensor(np.asarray(params), dtype=torch.float32, device="cuda"))


def test_nominal_chi2_equals_the_selection(m3e, cfg, c4):
    """At nominal alignment the fit of each kept track gives the selection's chi2.
    Both kernels inline the same FP32 fit (Sec. "Single Triplet Fit") into different
    code, where the compiler may fuse different multiply-adds: they agree to a few
    roundings of its ~100 operations (2e-5 relative; the chi2 band against the
    FP64 oracle is wider)."""
    d, rec, cand = c4["d"], c4["rec"], c4["cand"]
    with m3e.Context(cfg, 0) as ctx:
        chi2 = ctx.fit_chi2(*_dev(d, cand, O.nominal_params())).cpu().numpy()
        assert ctx.fit_valid_count() == cand.shape[0]
    st = rec["trk_status"]
    f_idx, t_idx = np.nonzero((np.arange(st.shape[1])[None, :] < np.minimum(rec["n_trip"], st.shape[1])[:, None])
                              & (st >= 5))
    np.testing.assert_allclose(chi2, rec["trk_val"][f_idx, t_idx, 2], rtol=2e-5, atol=1e-6)


def test_chi2_and_gradient_match_the_oracle(m3e, cfg, ocfg, c4):
    d, cand, truth = c4["d"], c4["tm"], c4["truth"]
    assert cand.shape[0] > 3000
    rng = np.random.default_rng(5)
    # nominal, the injected truth, and a point off the truth at the scale of the
    # misalignment (20 um, 0.2 mrad, 1e-3 in field)
    off_truth = truth + np.r_[np.concatenate([rng.normal(0, 0.02, (4, 3)), rng.normal(0, 2e-4, (4, 3))], 1).ravel(),
                              1e-3]
    for params in (O.nominal_params(), truth, off_truth):
        with m3e.Context(cfg, 0) as ctx:
            args = _dev(d, cand, params)
            each = ctx.fit_chi2(*args).cpu().numpy()
            s, g = ctx.fit_grad(*args)
            s, g = float(s.item()), g.cpu().numpy()
            n_ok = ctx.fit_valid_count()
        p32 = np.asarray(params, np.float32).astype(np.float64)  # the GPU sees the FP32 parameters
        ref = O.fit_chi2(ocfg, d["hits"], cand, p32, 8)
        ok = np.isfinite(ref)
        assert (np.isfinite(each) == ok).all() and n_ok == ok.sum()
        np.testing.assert_allclose(each[ok], ref[ok], rtol=CHI2_REL, atol=CHI2_ABS)
        tot, gfd, _ = O.fit_grad_fd(ocfg, d["hits"], cand[ok], p32, 8)
        assert s == pytest.approx(tot, rel=1e-4)
        err = np.abs(g - gfd)
        scale = np.abs(gfd[:24]).max()
        rel = err[:24] / np.abs(gfd[:24])
        print("gradient: largest component", scale, "per-component relative error", np.array2string(rel, precision=2),
              "error / largest", np.array2string(err[:24] / scale, precision=2))
        bad = err[:24] > GRAD_REL * np.abs(gfd[:24]) + GRAD_FLOOR * scale
        assert not bad.any(), (np.nonzero(bad)[0], rel[bad], err[:24][bad] / scale)
        assert g[24] == pytest.approx(gfd[24], rel=1e-4)


def test_fitted_curvature_matches_the_oracle(m3e, cfg, ocfg, c4):
    """m3e_fit_kappa: the weighted mean curvature of each candidate's fit at a
    displaced alignment equals the oracle's fit of the moved FP64 hit positions
    within 1e-5, and the field scale does not enter it (both triplet weights scale
    alike; up to rounding)."""
    d, cand, truth = c4["d"], c4["tm"][:400], c4["truth"]
    p32 = np.asarray(truth, np.float32).astype(np.float64)
    with m3e.Context(cfg, 0) as ctx:
        hits, off, cq, p = _dev(d, cand, truth)
        k1 = ctx.fit_kappa(hits, off, cq, p).cpu().numpy()
        p2 = p.clone()
        p2[24] *= 1.01
        k2 = ctx.fit_kappa(hits, off, cq, p2).cpu().numpy()
    assert (np.isnan(k1) == np.isnan(k2)).all()
    np.testing.assert_allclose(k2[~np.isnan(k1)], k1[~np.isnan(k1)], rtol=1e-6)
    ref = np.full(cand.shape[0], np.nan)
    for k, q in enumerate(cand):
        pos = []
        for L, h in enumerate(q):
            hd = O.decode(ocfg, int(d["hits"][h]))
            pos.append(O.align_point(p32[6 * L:6 * L + 6], [hd.x, hd.y, hd.z]))
        r = O.fit_track_positions(ocfg, np.array(pos))
        if r is not None:
            ref[k] = r[0]
    ok = np.isfinite(ref)
    assert ok.mean() > 0.99 and (np.isfinite(k1) == ok).all()
    np.testing.assert_allclose(k1[ok], ref[ok], rtol=1e-5)


def test_gradient_symmetries(m3e, cfg, c4):
    """No component along a common translation or a common rotation about z;
    d chi2 / d scale = 2 chi2 / scale."""
    d, cand, truth = c4["d"], c4["tm"], c4["truth"]
    with m3e.Context(cfg, 0) as ctx:
        s, g = ctx.fit_grad(*_dev(d, cand, truth))
    s, g = float(s.item()), g.cpu().numpy().astype(np.float64)
    p = np.asarray(truth, np.float32).astype(np.float64)
    gn = np.abs(g[:24]).max()
    for k in range(3):
        assert abs(sum(g[6 * L + k] for L in range(4))) < GRAD_REL * gn
    rot = sum(g[6 * L + 5] - g[6 * L] * p[6 * L + 1] + g[6 * L + 1] * p[6 * L] for L in range(4))
    assert abs(rot) < GRAD_REL * gn
    assert g[24] == pytest.approx(2 * s / p[24], rel=1e-4)


def test_autograd_function_and_determinism(m3e, cfg, c4):
    d, cand, truth = c4["d"], c4["tm"], c4["truth"]
    with m3e.Context(cfg, 0) as ctx:
        hits, off, cq, p = _dev(d, cand, truth)
        s1, g1 = ctx.fit_grad(hits, off, cq, p)
        s2, g2 = ctx.fit_grad(hits, off, cq, p)
        assert torch.equal(s1, s2) and torch.equal(g1, g2)
        s0, g0 = ctx.fit_grad(hits, off, cq, p, grad=False)
        assert torch.equal(s0, s1) and g0 is None
        x = p.clone().requires_grad_(True)
        loss = 0.5 * m3e.fit_chi2_sum(x, ctx, hits, off, cq)
        loss.backward()
        assert loss.item() == pytest.approx(0.5 * s1.item(), rel=1e-7)
        assert torch.allclose(x.grad, 0.5 * g1, rtol=1e-6, atol=0)


def test_edge_cases(m3e, cfg, c4):
    d, cand = c4["d"], c4["tm"]
    with m3e.Context(cfg, 0) as ctx:
        hits, off, cq, p = _dev(d, cand[:10], O.nominal_params())
        # no candidates
        s, g = ctx.fit_grad(hits, off, cq[:0], p)
        assert s.item() == 0.0 and torch.count_nonzero(g).item() == 0
        # a hit on the wrong layer and an index past the last hit are left out
        bad = cq.clone()
        bad[0, [0, 1]] = bad[0, [1, 0]]
        bad[1, 3] = int(d["off"][-1])
        each = ctx.fit_chi2(hits, off, bad, p).cpu().numpy()
        assert np.isnan(each[:2]).all() and np.isfinite(each[2:]).all()
        assert ctx.fit_valid_count() == 8
        # misaligned candidate rows are refused
        raw = torch.zeros(41, dtype=torch.int32, device="cuda")
        with pytest.raises(m3e.M3EError) as e:
            ctx.fit_grad(hits, off, raw[1:].view(10, 4), p)
        assert e.value.code == m3e.EINVAL
