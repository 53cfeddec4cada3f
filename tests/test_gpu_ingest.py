"""Hit ingest (m3e_ingest) through the C ABI against the FP64 oracle's decode
(Sec. "Memory Layout"): every coordinate must be the oracle's FP64 value rounded
once to FP32, bit for bit."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2206_11535_gb300 import gen

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


def _oracle_f32(ocfg, addrs):
    """The oracle's decode of each address, rounded once to FP32 (NaN where invalid)."""
    out = np.full((len(addrs), 4), np.nan, np.float32)
    for k, a in enumerate(addrs):
        h = O.decode(ocfg, int(a))
        if h is not None:
            out[k] = np.array([h.x, h.y, h.z, h.phi], np.float64).astype(np.float32)
    return out


def _same_bits(got, want):
    g = np.ascontiguousarray(got, np.float32).view(np.uint32)
    w = np.ascontiguousarray(want, np.float32).view(np.uint32)
    return np.array_equal(g, w)


def _run(ctx, hits_np, with_phi=True, offset=0):
    """Ingest with the device arrays starting `offset` elements into their allocation
    (offset 1 misaligns every array: the scalar path)."""
    n = hits_np.size
    hbuf = torch.zeros(n + offset, dtype=torch.int32, device="cuda")
    hbuf[offset:] = torch.from_numpy(hits_np).cuda()
    outs = [torch.full((n + offset,), -7.0, dtype=torch.float32, device="cuda") for _ in range(4)]
    h = hbuf[offset:]
    x, y, z, p = (o[offset:] for o in outs)
    ctx.ingest(h, x, y, z, p if with_phi else None, with_phi=with_phi)
    torch.cuda.synchronize()
    res = np.stack([t.cpu().numpy() for t in (x, y, z, p)], axis=1)
    return res


def test_c1_every_hit_bit_exact(ctx, ocfg):
    d = gen.workload("c1")
    got = _run(ctx, d["hits"])
    ctx.check()
    want = _oracle_f32(ocfg, d["hits"])
    assert _same_bits(got, want)


def test_every_column_and_every_row_bit_exact(ctx, ocfg, cfg):
    """One hit on every pixel column (all layers, ladders, columns) and one on every
    row: the computed azimuth and the table coordinates reproduce the oracle's FP64
    values rounded once, everywhere on the detector."""
    g = cfg["geometry"]
    parts = []
    for L in range(4):
        lad, col = np.meshgrid(np.arange(g["n_ladders"][L]), np.arange(g["n_cols"][L]), indexing="ij")
        parts.append(gen.encode(np.full(lad.size, L), lad.ravel(), col.ravel(), np.full(lad.size, 7)))
        rows = np.arange(g["n_rows"][L])
        parts.append(gen.encode(np.full(rows.size, L), np.zeros(rows.size, int), np.full(rows.size, 3), rows))
    a = np.concatenate(parts).astype(np.int32)
    got = _run(ctx, a)
    ctx.check()
    assert _same_bits(got, _oracle_f32(ocfg, a))


@pytest.mark.parametrize("n,offset", [(1, 0), (3, 0), (5, 0), (4099, 0), (4099, 1), (33, 3)])
def test_ragged_sizes_and_misaligned_arrays(ctx, ocfg, n, offset):
    d = gen.workload("c2", n_frames=200)
    a = d["hits"][:n]
    got = _run(ctx, a, offset=offset)
    assert _same_bits(got, _oracle_f32(ocfg, a))


def test_without_phi_leaves_phi_untouched(ctx, ocfg):
    d = gen.workload("c1", n_frames=50)
    got = _run(ctx, d["hits"], with_phi=False)
    want = _oracle_f32(ocfg, d["hits"])
    assert _same_bits(got[:, :3], want[:, :3])
    assert (got[:, 3] == -7.0).all()


def test_empty_batch(ctx):
    h = torch.zeros(0, dtype=torch.int32, device="cuda")
    x, y, z, p = ctx.ingest(h)
    ctx.check()
    assert x.numel() == 0 and p.numel() == 0


def test_invalid_address_gives_nan_and_latches(ctx, m3e, cfg, ocfg):
    g = cfg["geometry"]
    good = gen.encode([0, 1, 2, 3], [1, 2, 3, 4], [5, 6, 7, 8], [9, 10, 11, 12])
    bad = np.array([int(gen.encode(2, g["n_ladders"][2], 0, 0)), 1 << 28, -1], np.int64).astype(np.int32)
    a = np.concatenate([good, bad, good]).astype(np.int32)
    got = _run(ctx, a)
    with pytest.raises(m3e.M3EError) as e:
        ctx.check()
    assert e.value.code == m3e.EBADHIT
    ctx.check()  # the flag was consumed
    assert np.isnan(got[4:7]).all()
    assert _same_bits(got, _oracle_f32(ocfg, a))


def test_full_size_batch_sampled(ctx, ocfg, cfg):
    """The full 1,000,000-frame throughput batch (85 M hits), in the launch the benchmark
    times: 20,000 sampled hits bit for bit, and at every hit the point lies on its
    layer's cylinder and inside its length."""
    d = gen.workload("c2")
    hits = torch.from_numpy(d["hits"]).cuda()
    x, y, z, p = ctx.ingest(hits)
    ctx.check()
    rng = np.random.default_rng(7)
    idx = np.sort(rng.choice(d["hits"].size, 20000, replace=False))
    got = np.stack([t[torch.from_numpy(idx).cuda()].cpu().numpy() for t in (x, y, z, p)], axis=1)
    assert _same_bits(got, _oracle_f32(ocfg, d["hits"][idx]))
    g = cfg["geometry"]
    layer = torch.from_numpy(((d["hits"] >> 26) & 3).astype(np.int64)).cuda()
    r = torch.tensor(g["r_mm"], dtype=torch.float64, device="cuda")[layer]
    hl = torch.tensor(g["half_len_mm"], dtype=torch.float64, device="cuda")[layer]
    rr = torch.sqrt(x.double() ** 2 + y.double() ** 2)
    assert float(((rr - r).abs() / r).max()) < 2e-7
    assert bool((z.double().abs() < hl).all())
    assert bool(((p >= 0) & (p < 2 * np.pi)).all())
    # the azimuth and the point agree
    dphi = torch.remainder(torch.atan2(y.double(), x.double()) - p.double() + np.pi, 2 * np.pi) - np.pi
    assert float(dphi.abs().max()) < 1e-6
