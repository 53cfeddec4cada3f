"""The selection entry point that allocates nothing (m3e_select_frames_noalloc).

Callers that must not allocate device memory once running (a filter loop at a
fixed frame rate, a process under a fixed memory budget) use this entry point;
its scratch is a fixed static device array.  This file runs last, and passes both
alone in a fresh process and after the other tests (the array keeps the previous
call's contents, so each call must clear what it needs)."""
import numpy as np
import pytest

from paper_2206_11535_gb300 import gen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def m3e():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_11535_gb300 import m3e as mod
    return mod


def _batch():
    """c1 frames plus heavy frames that the warp stage defers to the CTA kernel."""
    d = gen.workload("c1", n_frames=3000, seed=61)
    heavy = gen.generate(40, 60.0, 5.0, 4, seed=62)
    hits = np.concatenate([d["hits"], heavy["hits"]]).astype(np.int32)
    off = np.concatenate([d["off"], d["off"][-1] + heavy["off"][1:]]).astype(np.int64)
    return hits, off


def test_noalloc_matches_allocating_entry_points_twice(m3e, cfg):
    hits, off = _batch()
    assert (np.diff(off) > 160).any()  # some frames take the deferred path
    h = torch.from_numpy(hits).cuda()
    o = torch.from_numpy(off).cuda()
    nf = off.size - 1
    with m3e.Context(cfg, 0) as ctx:
        keep_ref, reason_ref = ctx.select_frames(h, o)
        keep_f, reason_f = ctx.select_frames_fused(h, o)
        ref = reason_ref.cpu().numpy()
        assert (reason_f.cpu().numpy() == ref).all()
        for _ in range(2):  # two calls in a row: the static scratch is reused and re-cleared
            keep = torch.full((nf,), 7, dtype=torch.uint8, device="cuda")
            reason = torch.full((nf,), 7, dtype=torch.uint8, device="cuda")
            ctx.select_frames_noalloc(h, o, keep, reason)
            torch.cuda.synchronize()
            assert (reason.cpu().numpy() == ref).all()
            assert (keep.cpu().numpy() == keep_ref.cpu().numpy()).all()
        ctx.check()


def test_noalloc_rejects_oversize_batches(m3e, cfg):
    with m3e.Context(cfg, 0) as ctx:
        n = (1 << 18) + 1
        o = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
        k = torch.empty(n, dtype=torch.uint8, device="cuda")
        h = torch.zeros(1, dtype=torch.int32, device="cuda")
        with pytest.raises(m3e.M3EError) as e:
            ctx.select_frames_noalloc(h, o, k, k.clone())
        assert e.value.code == m3e.EINVAL and "262144" in str(e.value)
