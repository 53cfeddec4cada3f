"""Streaming selection (m3e_stream_*) on the GPU: every frame's decision equals the
batch selection's, alone and among others; the bounded device waits end in a
reported error, not a hang; admission refuses what does not fit."""
import ctypes as C
import time

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


def _csr(frames):
    off = np.zeros(len(frames) + 1, np.int64)
    off[1:] = np.cumsum([f.size for f in frames])
    return np.concatenate(frames).astype(np.int32) if frames else np.zeros(0, np.int32), off


def _mixed_batch(cfg, n=3000):
    """c5 frames with the special cases mixed in: empty, more hits than the warp
    stage holds, more than max_hits, and an invalid address."""
    d = gen.workload("c5", n_frames=n)
    frames = [d["hits"][d["off"][f]:d["off"][f + 1]] for f in range(n)]
    heavy = gen.generate(3, 80.0, 5.0, None, seed=6)
    big = gen.generate(1, 1500.0, 0.0, None, seed=7)["hits"]
    g = cfg["geometry"]
    bad = np.concatenate([frames[1], gen.encode([2], [g["n_ladders"][2]], [0], [0])])
    special = {5: np.zeros(0, np.int32), 17: heavy["hits"][heavy["off"][0]:heavy["off"][1]],
               18: heavy["hits"][heavy["off"][1]:heavy["off"][2]], 400: big, 401: bad,
               402: heavy["hits"][heavy["off"][2]:heavy["off"][3]]}
    for k, v in special.items():
        if k < n:
            frames[k] = v.astype(np.int32)
    assert special[17].size > 160 and big.size > cfg["caps"]["max_hits"]
    return _csr(frames)


def _batch_reference(m3e, ctx, hits, off):
    keep, reason = ctx.select_frames_fused(torch.from_numpy(hits).cuda(), torch.from_numpy(off).cuda())
    try:
        ctx.check()
    except m3e.M3EError as e:  # the invalid-address frame latches EBADHIT
        assert e.code == m3e.EBADHIT
    return keep.cpu().numpy(), reason.cpu().numpy()


def _submit_all(m3e, ctx, hits, off, order=None):
    nf = off.size - 1
    res = (m3e.Result * nf)()
    for f in (range(nf) if order is None else order):
        while ctx.stream_submit(hits[off[f]:off[f + 1]], 1000 + f, res[f]) == m3e.EBUSY:
            time.sleep(1e-4)
    assert ctx.stream_drain(30000) == m3e.OK
    return res


def test_stream_matches_batch(m3e, cfg):
    hits, off = _mixed_batch(cfg)
    nf = off.size - 1
    with m3e.Context(cfg, 0) as ctx:
        keep, reason = _batch_reference(m3e, ctx, hits, off)
        ctx.stream_open()
        res = _submit_all(m3e, ctx, hits, off)
        got_keep = np.array([r.keep for r in res], np.uint8)
        got_reason = np.array([r.reason for r in res], np.uint8)
        assert all(r.done == 1 for r in res)
        assert [r.tag for r in res] == [1000 + f for f in range(nf)]
        assert all(r.t_done_ns >= r.t_submit_ns > 0 for r in res)
        np.testing.assert_array_equal(got_reason, reason)
        np.testing.assert_array_equal(got_keep, keep)
        assert res[401].err == m3e.EBADHIT and res[401].reason == m3e.ERR_BADHIT
        assert res[400].reason == m3e.HIT_OVERFLOW and res[5].reason == m3e.DROP
        assert all(res[f].err == m3e.OK for f in range(nf) if f != 401)
        st = ctx.stream_poll()
        assert st["submitted"] == st["completed"] == nf and st["failed"] == 0
        assert st["heavy_frames"] >= 4 and st["kernel_launches"] >= 1
        assert ctx.stream_close() == m3e.OK


def test_stream_alone_and_in_the_mix(m3e, cfg):
    """A frame's result does not depend on what else is in flight: each of a few
    frames submitted alone (drained in between) equals its result in a Poisson
    replay of the whole batch and in reverse-order submission."""
    hits, off = _mixed_batch(cfg, n=2000)
    nf = off.size - 1
    with m3e.Context(cfg, 0) as ctx:
        ctx.stream_open()
        picks = [0, 5, 17, 33, 400, 401, 402, 999, nf - 1]
        alone = {}
        for f in picks:
            r = m3e.Result()
            assert ctx.stream_submit(hits[off[f]:off[f + 1]], f, r) == m3e.OK
            assert ctx.stream_drain(10000) == m3e.OK
            alone[f] = (r.keep, r.reason)
        rep = ctx.stream_replay(hits, off, rate_hz=2.0e6, seed=11)
        rev = _submit_all(m3e, ctx, hits, off, order=range(nf - 1, -1, -1))
        keep, reason = _batch_reference(m3e, ctx, hits, off)
        np.testing.assert_array_equal(rep["reason"], reason)
        np.testing.assert_array_equal(np.array([r.reason for r in rev], np.uint8), reason)
        for f, (k, rs) in alone.items():
            assert (k, rs) == (rep["keep"][f], rep["reason"][f]) == (keep[f], reason[f]), f
        assert (rep["lat_submit_ns"] > 0).all() and (rep["lat_arrival_ns"] >= rep["lat_submit_ns"] - 1000).all()


def _oracle_agrees(m3e, ctx, ocfg, hits, off, reason, form):
    """Every frame's decision equals the FP64 oracle's, except frames whose differences
    all lie inside a boundary band (candidate by candidate, with the record of `form`)."""
    _, o_reason = O.select_frames(ocfg, hits, off, 4)
    diff = np.nonzero(o_reason != reason)[0]
    for f in diff:
        sub = np.ascontiguousarray(hits[off[f]:off[f + 1]])
        so = np.array([0, sub.size], np.int64)
        rec = ctx.select_frames_debug(torch.from_numpy(sub).cuda(), torch.from_numpy(so).cuda(), cap_trip=1024,
                                      cap_combo=1024, form=form)
        rec = {k: v.cpu().numpy() for k, v in rec.items()}
        try:
            ctx.check()
        except m3e.M3EError:
            pass
        res = P.compare_frame(ocfg, sub, P.record_of_frame(rec, 0), int(f))
        assert res.status == "boundary", (int(f), res.fails[:3])
    assert diff.size <= 0.01 * reason.size + 1, diff.size
    return diff.size


def test_stream_decisions_match_the_oracle(m3e, cfg, ocfg):
    """The streaming kernel's decisions against the FP64 oracle directly (not against
    the library's batch path): 2,000 frames of the streaming mix with its special
    frames (empty, heavy frames for the CTA kernel, more than max_hits, an invalid
    address), replayed as Poisson arrivals."""
    hits, off = _mixed_batch(cfg, n=2000)
    with m3e.Context(cfg, 0) as ctx:
        ctx.stream_open()
        rep = ctx.stream_replay(hits, off, rate_hz=2.0e6, seed=17)
        assert ctx.stream_close() == m3e.OK
        nb = _oracle_agrees(m3e, ctx, ocfg, hits, off, rep["reason"], m3e.FUSED)
        print("stream vs oracle: boundary frames", nb)
        assert (rep["keep"] == (rep["reason"] != 0)).all()


def test_stream_idle_exit_and_relaunch(m3e, cfg):
    """The resident kernel leaves the GPU after idle_us without frames and the
    library thread relaunches it for the next submission."""
    hits, off = _mixed_batch(cfg, n=50)
    with m3e.Context(cfg, 0) as ctx:
        ctx.stream_open(idle_us=2000)
        r = m3e.Result()
        assert ctx.stream_submit(hits[off[0]:off[1]], 1, r) == m3e.OK
        assert ctx.stream_drain(10000) == m3e.OK
        deadline = time.time() + 5.0
        while ctx.stream_poll()["kernel_running"] and time.time() < deadline:
            time.sleep(0.005)
        st = ctx.stream_poll()
        assert st["kernel_running"] == 0 and st["kernel_launches"] == 1
        r2 = m3e.Result()
        assert ctx.stream_submit(hits[off[1]:off[2]], 2, r2) == m3e.OK
        assert ctx.stream_drain(10000) == m3e.OK
        assert ctx.stream_poll()["kernel_launches"] == 2
        keep, reason = _batch_reference(m3e, ctx, hits, off)
        assert (r.reason, r2.reason) == (reason[0], reason[1])


def test_stream_wait_limit_expires_and_reports(m3e, cfg):
    """Nothing publishes frames to the workers (test mode): their bounded waits run
    out, the kernel returns, the frame is failed with M3E_ETIMEOUT, the stream
    reports the failure, and the context still selects batches afterwards."""
    hits, off = _mixed_batch(cfg, n=20)
    with m3e.Context(cfg, 0) as ctx:
        ctx.stream_open(no_feeder=1, wait_limit_ms=50, lifetime_ms=200, idle_us=1000)
        r = m3e.Result()
        assert ctx.stream_submit(hits[off[0]:off[1]], 7, r) == m3e.OK
        t = time.time()
        assert ctx.stream_drain(10000) == m3e.ETIMEOUT
        assert time.time() - t < 5.0
        assert r.done == 1 and r.err == m3e.ETIMEOUT and r.tag == 7
        st = ctx.stream_poll()
        assert st["failed"] == 1 and st["kernel_running"] == 0
        r2 = m3e.Result()
        with pytest.raises(m3e.M3EError) as e:
            ctx.stream_submit(hits[off[1]:off[2]], 8, r2)
        assert e.value.code == m3e.ETIMEOUT
        ctx.stream_close()
        keep, reason = _batch_reference(m3e, ctx, hits, off)
        assert reason.size == 20
        # a new stream on the same context works
        ctx.stream_open()
        res = _submit_all(m3e, ctx, hits, off)
        np.testing.assert_array_equal(np.array([x.reason for x in res], np.uint8), reason)


def test_stream_admission(m3e, cfg):
    """Small rings: a packet larger than the ring is refused (EINVAL); a fast
    replay through 8 slots and a 16 KiB ring is admitted piecewise (EBUSY
    retries) with unchanged decisions."""
    hits, off = _mixed_batch(cfg, n=2000)
    with m3e.Context(cfg, 0) as ctx:
        ctx.stream_open(slots=8, ring_bytes=16384)
        r = m3e.Result()
        big = hits[off[400]:off[401]]
        assert big.size * 4 > 16384
        with pytest.raises(m3e.M3EError) as e:
            ctx.stream_submit(big, 0, r)
        assert e.value.code == m3e.EINVAL
        keep, reason = _batch_reference(m3e, ctx, hits, off)
        keep_idx = np.array([f for f in range(off.size - 1) if off[f + 1] - off[f] <= 4096])
        frames = [hits[off[f]:off[f + 1]] for f in keep_idx]
        h2, o2 = _csr(frames)
        rep = ctx.stream_replay(h2, o2, rate_hz=1.0e7, seed=3)
        np.testing.assert_array_equal(rep["reason"], reason[keep_idx])
        assert rep["busy_retries"] > 0


def test_stream_submit_many(m3e, cfg):
    """Batched submission: chunks of a CSR batch admitted in order (a prefix when the
    slots run out), tags and decisions as for single submissions."""
    hits, off = _mixed_batch(cfg, n=3000)
    nf = off.size - 1
    with m3e.Context(cfg, 0) as ctx:
        keep, reason = _batch_reference(m3e, ctx, hits, off)
        ctx.stream_open(slots=1024)
        res = (m3e.Result * nf)()
        tags = np.arange(nf, dtype=np.uint64) * 3 + 7
        f = 0
        partial = 0
        while f < nf:
            e = min(nf, f + 700)
            sub_off = off[f:e + 1] - off[f]
            slot0 = m3e.Result.from_buffer(res, f * C.sizeof(m3e.Result))
            k = ctx.stream_submit_many(hits[off[f]:off[e]], sub_off, slot0, tags[f:e])
            assert 0 <= k <= e - f
            partial += k < e - f
            f += k
            if k == 0:
                time.sleep(1e-4)
        assert ctx.stream_drain(30000) == m3e.OK
        np.testing.assert_array_equal(np.array([r.reason for r in res], np.uint8), reason)
        np.testing.assert_array_equal(np.array([r.keep for r in res], np.uint8), keep)
        assert [r.tag for r in res] == [int(t) for t in tags]
        # a full slot ring admits a prefix only
        ctx.stream_close()
        ctx.stream_open(slots=8)
        res2 = (m3e.Result * 64)()
        k = ctx.stream_submit_many(hits[:off[64]], off[:65], res2)
        assert 1 <= k <= 8
        assert ctx.stream_drain(10000) == m3e.OK
        assert all(res2[i].done == 1 and res2[i].tag == i and res2[i].reason == reason[i] for i in range(k))
