"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, on the GPU."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2206_11535_gb300 import gen

from . import parity as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def m3e():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_11535_gb300 import m3e as mod
    return mod


@pytest.fixture(scope="module")
def ctx(m3e, cfg):
    c = m3e.Context(cfg, 0)
    yield c
    c.close()


def _dev(d):
    return torch.from_numpy(d["hits"]).cuda(), torch.from_numpy(d["off"]).cuda()


def _np(rec):
    return {k: v.cpu().numpy() for k, v in rec.items()}


def _check_results(res, max_boundary_frac=0.01):
    s = P.summary(res)
    print("boundary differences per band", {k: v for k, v in P.band_counts(res).items() if v})
    fails = [r for r in res if r.status == "fail"]
    msg = "\n".join(f"frame {r.frame}: {r.fails[:4]}" for r in fails[:10])
    assert s["fail"] == 0, f"{s}\n{msg}"
    assert s["boundary"] <= max_boundary_frac * len(res) + 1, s
    return s


FORMS = {"staged": 0, "fused": 1, "plain": 2}


@pytest.mark.parametrize("form", list(FORMS))
def test_c1_parity_all_frames(ctx, ocfg, form):
    """1,000 frames of the parity workload, every candidate list and decision, for
    each form of the selection."""
    d = gen.workload("c1")
    hits, off = _dev(d)
    rec = _np(ctx.select_frames_debug(hits, off, cap_trip=1024, cap_combo=1024, form=FORMS[form]))
    s = _check_results(P.compare_batch(ocfg, d["hits"], d["off"], rec))
    print("c1 parity", form, s)
    entry = {"staged": ctx.select_frames, "fused": ctx.select_frames_fused, "plain": ctx.select_frames_plain}[form]
    keep, reason = entry(hits, off)
    assert (reason.cpu().numpy() == rec["reason"]).all()
    assert (keep.cpu().numpy() == rec["keep"]).all()
    ctx.check()


@pytest.mark.parametrize("form", ["staged", "fused"])
def test_c2_sample_parity(ctx, ocfg, form):
    """2,000 frames of the throughput workload's generator (seed 2)."""
    d = gen.workload("c2", n_frames=2000)
    hits, off = _dev(d)
    rec = _np(ctx.select_frames_debug(hits, off, cap_trip=1024, cap_combo=1024, form=FORMS[form]))
    s = _check_results(P.compare_batch(ocfg, d["hits"], d["off"], rec))
    print("c2 sample parity", form, s)


def test_c2_full_size_sampled(ctx, ocfg):
    """The full 1,000,000-frame throughput batch, in the launch configuration the
    benchmark times; 400 sampled frames checked against the oracle one by one,
    plus invariants over all frames."""
    d = gen.workload("c2")
    hits, off = _dev(d)
    keep, reason = ctx.select_frames(hits, off)
    ctx.check()
    r = reason.cpu().numpy()
    # the other forms decide every frame identically
    for entry in (ctx.select_frames_fused, ctx.select_frames_plain):
        assert (entry(hits, off)[1].cpu().numpy() == r).all()
    k = keep.cpu().numpy()
    assert ((k == 1) == (r != 0)).all()
    assert r.max() <= 6
    rng = np.random.default_rng(123)
    sample = np.sort(rng.choice(d["off"].size - 1, 400, replace=False))
    diff = []
    for f in sample:
        o = O.select_frame(ocfg, d["hits"][d["off"][f]:d["off"][f + 1]], records=False)
        if o["reason"] != r[f]:
            diff.append(int(f))
    # any disagreement must be a boundary frame of the candidate-level comparison
    for f in diff:
        sub = gen_subbatch(d, [f])
        rec = _np(ctx.select_frames_debug(*_dev(sub), cap_trip=1024, cap_combo=1024))
        res = P.compare_frame(ocfg, sub["hits"], P.record_of_frame(rec, 0), f)
        assert res.status == "boundary", (f, res.fails)
    assert len(diff) <= 4


def gen_subbatch(d, frames):
    parts = [d["hits"][d["off"][f]:d["off"][f + 1]] for f in frames]
    off = np.zeros(len(frames) + 1, np.int64)
    off[1:] = np.cumsum([p.size for p in parts])
    return dict(hits=np.concatenate(parts) if parts else np.zeros(0, np.int32), off=off)


def test_derived_errors_leave_margin(ctx, ocfg):
    """The bands of the derived variables hold at least twice the largest difference
    measured here between the CUDA path and the oracle on matched candidates (all
    parity frames and 2,000 throughput frames, every form)."""
    worst = {}
    for wl, n in (("c1", None), ("c2", 2000)):
        d = gen.workload(wl) if n is None else gen.workload(wl, n_frames=n)
        for form in FORMS.values():
            rec = _np(ctx.select_frames_debug(*_dev(d), cap_trip=1024, cap_combo=1024, form=form))
            for k, (m, cnt) in P.matched_errors(ocfg, d["hits"], d["off"], rec).items():
                worst[k] = max(worst.get(k, 0.0), m)
    print("largest differences", {k: f"{v:.2e}" for k, v in worst.items()})
    assert worst["kappa"] <= P.KAPPA_REL / 2 and worst["theta"] <= P.THETA_REL / 2
    assert 2 * worst["fourth_hit"] <= P.BAND["fourth_hit"] / 2
    for k in ("chi2_track", "energy", "vtx_chi2", "tdist", "ptot", "disc", "filter", "choice"):
        assert worst[k] <= P.BAND[k] / 2, (k, worst[k], P.BAND[k])
    for k in ("vtx_chi2", "tdist", "ptot"):
        assert worst[k + "_value"] <= P.VAL_REL[k] / 2, (k, worst[k + "_value"])


def test_permutation_invariance(ctx):
    d = gen.workload("c1", n_frames=300, seed=9)
    rng = np.random.default_rng(1)
    hp = d["hits"].copy()
    for f in range(300):
        a, b = d["off"][f], d["off"][f + 1]
        hp[a:b] = hp[a:b][rng.permutation(b - a)]
    r1 = _np(ctx.select_frames_debug(*_dev(d)))
    r2 = _np(ctx.select_frames_debug(torch.from_numpy(hp).cuda(), torch.from_numpy(d["off"]).cuda()))
    assert (r1["reason"] == r2["reason"]).all()
    assert (r1["n_trip"] == r2["n_trip"]).all() and (r1["n_combo"] == r2["n_combo"]).all()
    for f in range(0, 300, 7):
        a = d["off"][f]
        n = min(r1["n_trip"][f], 768)
        s1 = sorted(tuple(d["hits"][a + r1["trip"][f, t, :3]]) for t in range(n))
        s2 = sorted(tuple(hp[a + r2["trip"][f, t, :3]]) for t in range(n))
        assert s1 == s2


def test_edge_cases(ctx, m3e, cfg, ocfg):
    g = cfg["geometry"]
    frames = []
    frames.append(np.zeros(0, np.int32))                                               # empty frame
    frames.append(gen.encode([0, 1, 2], [0, 0, 0], [1, 1, 1], [5, 5, 5]))              # no layer 3
    frames.append(gen.encode([0, 1, 0, 1], [0, 0, 1, 1], [3, 3, 5, 5], [100, 100, 200, 200]))  # two layers
    base = gen.generate(3, 10.0, 0.5, None, seed=5)
    f0 = base["hits"][base["off"][0]:base["off"][1]]
    frames.append(np.concatenate([f0, f0]))                                            # duplicated hits
    heavy = gen.generate(2, 80.0, 5.0, None, seed=6)                                   # deferred to the CTA stage
    frames.append(heavy["hits"][heavy["off"][0]:heavy["off"][1]])
    frames.append(heavy["hits"][heavy["off"][1]:heavy["off"][2]])
    big = gen.generate(1, 1500.0, 0.0, None, seed=7)                                   # more than max_hits
    frames.append(big["hits"])
    frames.append(f0)                                                                  # ordinary frame last
    off = np.zeros(len(frames) + 1, np.int64)
    off[1:] = np.cumsum([f.size for f in frames])
    hits = np.concatenate(frames).astype(np.int32)
    d = dict(hits=hits, off=off)
    assert frames[4].size > 160 and big["hits"].size > cfg["caps"]["max_hits"]
    for form in FORMS.values():
        rec = _np(ctx.select_frames_debug(*_dev(d), cap_trip=1024, cap_combo=1024, form=form))
        res = P.compare_batch(ocfg, hits, off, rec)
        _check_results(res, max_boundary_frac=0.5)
        assert rec["reason"][0] == 0 and rec["reason"][1] == 0 and rec["reason"][2] == 0
        assert rec["reason"][6] == m3e.HIT_OVERFLOW
        keep, reason = ctx.select_frames(*_dev(d))
        assert (reason.cpu().numpy() == rec["reason"]).all()
    ctx.check()
    # an invalid address: frame kept with ERR_BADHIT, EBADHIT latched until checked
    bad = np.concatenate([f0, gen.encode([2], [g["n_ladders"][2]], [0], [0])]).astype(np.int32)
    d2 = gen_subbatch(dict(hits=np.concatenate([f0, bad]), off=np.array([0, f0.size, f0.size + bad.size])), [0, 1])
    keep, reason = ctx.select_frames(*_dev(d2))
    assert reason.cpu().tolist()[1] == m3e.ERR_BADHIT and keep.cpu().tolist()[1] == 1
    with pytest.raises(m3e.M3EError) as e:
        ctx.check()
    assert e.value.code == m3e.EBADHIT
    ctx.check()  # cleared
    # zero frames
    z = dict(hits=np.zeros(0, np.int32), off=np.zeros(1, np.int64))
    keep, reason = ctx.select_frames(*_dev(z))
    assert keep.numel() == 0


def test_small_caps_overflow_parity(m3e, cfg):
    """Caps lowered so that every overflow path triggers: decisions equal the
    oracle's under the same caps."""
    over = dict(max_triplets=12, max_tracks=6, max_combos=4)
    import copy
    c2 = copy.deepcopy(cfg)
    c2["caps"].update(over)
    oc = O.make_config(c2)
    d = gen.workload("c1", n_frames=400, seed=19)
    with m3e.Context(c2, 0) as ctx:
        for form in FORMS.values():
            rec = _np(ctx.select_frames_debug(*_dev(d), cap_trip=64, cap_combo=64, form=form))
            res = P.compare_batch(oc, d["hits"], d["off"], rec)
            _check_results(res)
            counts = np.bincount(rec["reason"], minlength=7)
            assert counts[2] > 0 and counts[3] > 0 and counts[4] > 0, counts


def test_host_entry_matches_device(ctx, m3e):
    """The host entry point (the selection running while the chunks of the batch
    arrive; 16 chunks at this size) decides as the device entry point, from
    page-locked and from ordinary host memory, call after call, and for a batch
    that fits one chunk."""
    d = gen.workload("c1", n_frames=850_000, seed=12)
    keep, reason = ctx.select_frames(*_dev(d))
    reason, keep = reason.cpu().numpy(), keep.cpu().numpy()
    hh = torch.from_numpy(d["hits"]).pin_memory()
    ho = torch.from_numpy(d["off"]).pin_memory()
    hk = torch.empty(d["off"].size - 1, dtype=torch.uint8).pin_memory()
    hr = torch.empty(d["off"].size - 1, dtype=torch.uint8).pin_memory()
    s = torch.cuda.current_stream()
    for _ in range(3):
        hr.fill_(9)
        ctx.select_frames_host(hh, ho, hk, hr, stream=s)
        s.synchronize()
        assert (hr.numpy() == reason).all()
        assert (hk.numpy() == keep).all()
    ctx.check()
    k2, r2 = ctx.select_frames_host(d["hits"], d["off"], stream=s)
    s.synchronize()
    assert (r2 == reason).all() and (k2 == keep).all()
    n = 20_000  # one chunk
    k3, r3 = ctx.select_frames_host(d["hits"][:d["off"][n]], d["off"][:n + 1], stream=s)
    s.synchronize()
    assert (r3 == reason[:n]).all()
    ctx.check()


def test_host_entry_edge_cases(ctx, m3e, cfg):
    """The host entry point on ragged batches: runs of empty frames across chunk
    boundaries, a batch without a single hit, one frame, an invalid address (kept,
    EBADHIT latched), and the edge frames of the device test."""
    g = cfg["geometry"]
    s = torch.cuda.current_stream()
    d = gen.workload("c1", n_frames=120_000, seed=15)
    sizes = np.diff(d["off"])
    sizes[40_000:70_000] = 0  # empty frames, across the boundaries of 50,000-frame chunks
    hits = np.concatenate([d["hits"][d["off"][f]:d["off"][f + 1]] for f in range(sizes.size) if sizes[f]])
    off = np.zeros(sizes.size + 1, np.int64)
    off[1:] = np.cumsum(sizes)
    assert off[-1] == hits.size
    dd = dict(hits=hits.astype(np.int32), off=off)
    ref = ctx.select_frames(*_dev(dd))[1].cpu().numpy()
    ctx.set_host_pipeline(max_chunks=3)
    try:
        _, r = ctx.select_frames_host(dd["hits"], dd["off"], stream=s)
        s.synchronize()
        assert (r == ref).all()
        ctx.check()
    finally:
        ctx.set_host_pipeline()
    # no hits at all, and a single frame
    z = dict(hits=np.zeros(0, np.int32), off=np.zeros(7, np.int64))
    _, r = ctx.select_frames_host(z["hits"], z["off"], stream=s)
    s.synchronize()
    assert (r == ctx.select_frames(*_dev(z))[1].cpu().numpy()).all()
    one = dict(hits=d["hits"][:d["off"][1]].copy(), off=d["off"][:2].copy())
    _, r = ctx.select_frames_host(one["hits"], one["off"], stream=s)
    s.synchronize()
    assert r[0] == ref[0]
    # an invalid address in the second frame
    f0 = d["hits"][:d["off"][1]]
    bad = np.concatenate([f0, gen.encode([2], [g["n_ladders"][2]], [0], [0])]).astype(np.int32)
    hb = np.concatenate([f0, bad]).astype(np.int32)
    ob = np.array([0, f0.size, f0.size + bad.size], np.int64)
    k, r = ctx.select_frames_host(hb, ob, stream=s)
    s.synchronize()
    assert r[1] == m3e.ERR_BADHIT and k[1] == 1 and r[0] == ref[0]
    with pytest.raises(m3e.M3EError) as e:
        ctx.check(stream=s)
    assert e.value.code == m3e.EBADHIT
    ctx.check(stream=s)


def test_host_entry_chunk_wait_is_bounded(cfg, m3e):
    """A chunk whose arrival flag is never set: stage 1 gives up after the wait
    limit, the call latches ETIMEOUT, and the context stays usable."""
    d = gen.workload("c1", n_frames=300_000, seed=14)
    with m3e.Context(cfg, 0) as c:
        ref = c.select_frames(*_dev(d))[1].cpu().numpy()
        s = torch.cuda.current_stream()
        c.set_host_pipeline(max_chunks=6, wait_ms=50, drop_chunk=3)
        c.select_frames_host(d["hits"], d["off"], stream=s)
        with pytest.raises(m3e.M3EError) as e:
            c.check(stream=s)
        assert e.value.code == m3e.ETIMEOUT
        c.set_host_pipeline()
        _, r = c.select_frames_host(d["hits"], d["off"], stream=s)
        s.synchronize()
        assert (r == ref).all()
        c.check(stream=s)
        with pytest.raises(m3e.M3EError):
            c.set_host_pipeline(max_chunks=0)


@pytest.mark.parametrize("form", ["staged", "fused"])
def test_stats_counters(ctx, m3e, ocfg, form):
    d = gen.workload("c1", n_frames=500, seed=13)
    st = m3e.new_stats()
    entry = ctx.select_frames if form == "staged" else ctx.select_frames_fused
    keep, reason = entry(*_dev(d), stats=st)
    torch.cuda.synchronize()
    s = m3e.stats_dict(st)
    assert sum(s["reasons"]) == 500
    assert s["frames"] == 500 - s["reasons"][5] - s["reasons"][6]
    assert s["hits"] <= d["hits"].size
    _, _, cnt = O.select_frames(ocfg, d["hits"], d["off"], 4, counts=True)
    assert abs(s["triplets"] - cnt[:, 3].sum()) <= 5
    assert abs(s["tracks"] - cnt[:, 4].sum()) <= 5
    # binned work counts: the warp stage (every lane's share) and the CTA-per-frame
    # form count the same phi windows and candidate triplets; the binned pairs are
    # a subset of the oracle's brute-force pairs, and every selected triplet was a candidate
    stp = m3e.new_stats()
    ctx.select_frames_plain(*_dev(d), stats=stp)
    torch.cuda.synchronize()
    sp = m3e.stats_dict(stp)
    for k in ("pair_tests", "triplet_tests", "triplets", "tracks", "energy_tests", "combos", "pz_open"):
        assert s[k] == sp[k], (k, s[k], sp[k])
    assert 0 < s["pz_open"] < s["combos"] and s["vertexed_pz_open"] <= s["vertexed"]
    assert 0 < s["pair_tests"] <= cnt[:, 1].sum()
    # candidate triplets = sum over layer-1 hits of (Phi01 partners x Phi12 partners),
    # the oracle's count in FP64 (equal up to hits on a Phi-cut boundary)
    assert abs(s["triplet_tests"] - cnt[:, 2].sum()) <= 1e-3 * cnt[:, 2].sum() + 5
    assert s["triplets"] <= s["triplet_tests"]


def test_c3_uneven_frames_sample(ctx, ocfg):
    """Frames of the uneven workload (lognormal track counts, some at 100x noise):
    the staged form with its CTA tier for large frames, checked candidate by
    candidate, and the plain form deciding identically."""
    d = gen.workload("c3", n_frames=400, seed=33)
    assert (np.diff(d["off"]) > 160).sum() > 20  # the CTA tier of stage 1 is exercised
    hits, off = _dev(d)
    rec = _np(ctx.select_frames_debug(hits, off, cap_trip=1024, cap_combo=1024, form=FORMS["staged"]))
    s = _check_results(P.compare_batch(ocfg, d["hits"], d["off"], rec), max_boundary_frac=0.02)
    print("c3 sample parity", s)
    keep_p, reason_p = ctx.select_frames_plain(hits, off)
    assert (reason_p.cpu().numpy() == rec["reason"]).all()


def test_graph_and_autotune_keep_decisions(m3e, cfg):
    """The persistent batched form: autotuned launch parameters and a captured CUDA
    graph (staged and fused) give the decisions of a direct call."""
    d = gen.workload("c3", n_frames=3000, seed=34)
    hits, off = _dev(d)
    nf = d["off"].size - 1
    with m3e.Context(cfg, 0) as ctx:
        ref = ctx.select_frames(hits, off)[1].cpu().numpy()
        t = ctx.autotune(hits, off)
        assert t["configs_tried"] > 10 and t["ms_best"] <= t["ms_default"] * 1.05
        assert (ctx.select_frames(hits, off)[1].cpu().numpy() == ref).all()
        ctx.prepare(nf)
        for form in (m3e.STAGED, m3e.FUSED):
            keep = torch.empty(nf, dtype=torch.uint8, device="cuda")
            reason = torch.empty(nf, dtype=torch.uint8, device="cuda")
            g = ctx.graph(hits, off, keep, reason, form=form)
            for _ in range(2):
                reason.fill_(9)
                g.launch()
                torch.cuda.synchronize()
                assert (reason.cpu().numpy() == ref).all()
            g.close()
        ctx.check()


def test_graph_decisions_match_the_oracle(m3e, cfg, ocfg):
    """The persistent batched form (autotuned, the batch captured as one CUDA graph)
    against the FP64 oracle directly, on uneven frames: every frame's decision, and
    for any frame that differs, a candidate-level check that the difference lies
    inside a boundary band."""
    d = gen.workload("c3", n_frames=3000, seed=33)
    hits, off = _dev(d)
    nf = d["off"].size - 1
    _, o_reason = O.select_frames(ocfg, d["hits"], d["off"], 4)
    with m3e.Context(cfg, 0) as ctx:
        ctx.autotune(hits, off)
        ctx.prepare(nf)
        keep = torch.empty(nf, dtype=torch.uint8, device="cuda")
        reason = torch.empty(nf, dtype=torch.uint8, device="cuda")
        g = ctx.graph(hits, off, keep, reason, form=m3e.STAGED)
        reason.fill_(9)
        g.launch()
        torch.cuda.synchronize()
        r = reason.cpu().numpy()
        g.close()
        diff = np.nonzero(r != o_reason)[0]
        for f in diff:
            sub = gen_subbatch(d, [int(f)])
            rec = _np(ctx.select_frames_debug(*_dev(sub), cap_trip=1024, cap_combo=1024))
            res = P.compare_frame(ocfg, sub["hits"], P.record_of_frame(rec, 0), int(f))
            assert res.status == "boundary", (int(f), res.fails[:3])
        assert diff.size <= 0.01 * nf + 1
        ctx.check()


def test_high_rate_sample(ctx, ocfg):
    """Frames at 1e9 muons/s (Poisson(64) tracks): dense frames, CTA tiers and
    triplet overflows, candidate by candidate."""
    d = gen.generate(120, 64.0, 0.5, 1000, seed=63)
    hits, off = _dev(d)
    rec = _np(ctx.select_frames_debug(hits, off, cap_trip=1024, cap_combo=1024, form=FORMS["staged"]))
    s = _check_results(P.compare_batch(ocfg, d["hits"], d["off"], rec), max_boundary_frac=0.05)
    print("1e9 muons/s sample parity", s)
    for form in ("fused", "plain"):
        rf = _np(ctx.select_frames_debug(hits, off, cap_trip=1024, cap_combo=1024, form=FORMS[form]))
        assert (rf["reason"] == rec["reason"]).all()


@pytest.mark.parametrize("workload", ["c1", "c2", "signal"])
def test_momentum_bound_keeps_the_decisions(ctx, m3e, cfg, workload):
    """Decision-only runs skip the vertex of combinations whose longitudinal
    momentum alone fails the |sum p| cut; runs with statistics or debug records fit
    every combination.  All of them decide every frame alike, in every form."""
    if workload == "signal":
        d = gen.generate(3000, 10.0, 0.5, 1, seed=71)  # a signal decay in every frame
    else:
        d = gen.workload(workload, n_frames=3000, seed=71)
    hits, off = _dev(d)
    ref = ctx.select_frames(hits, off, stats=m3e.new_stats())[1].cpu().numpy()
    assert (ref == m3e.VERTEX).sum() > (1000 if workload == "signal" else 0)
    for form, entry in (("staged", ctx.select_frames), ("fused", ctx.select_frames_fused),
                        ("plain", ctx.select_frames_plain)):
        assert (entry(hits, off)[1].cpu().numpy() == ref).all(), form
    rec = _np(ctx.select_frames_debug(hits, off, form=FORMS["staged"]))
    assert (rec["reason"] == ref).all()
    # the bound is active: most fitted combinations fail the momentum cut
    st = rec["combo"][..., 3]
    fitted = (st & 255) == 2
    assert (rec["combo_val"][..., 3][fitted] > cfg["cuts"]["ptot_max"]).mean() > 0.5
