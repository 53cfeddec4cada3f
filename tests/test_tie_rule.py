"""The tie rule of the closest layer-3 hit (Sec. "Triplets Fit", Algorithm 3; the
reading: the smallest (r3 dphi)^2 + dz^2, ties to the smaller address) on the GPU,
for two distinct pixels.

The frame holds one track at a polar angle of exactly 90 degrees: its three first
hits sit on the row of z = +0.04 mm of their layers, so the second segment's z / Phi
is exactly zero and the estimated layer-3 point has the z of the layer-2 hit.  Two
layer-3 hits sit in one pixel column (the same azimuth) on the rows of z = -0.04 and
z = +0.12 mm.  Their FP32 coordinates are symmetric about +0.04 to the last bit
(0.12f - 0.04f = 0.04f - (-0.04f) = 0.08f), so their FP32 metrics are equal: the GPU
must take the one with the smaller address (the lower row), whatever their order in
the input.  The FP64 oracle, where the two distances differ in the 15th digit, takes
the same hit, which the test checks as well.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2206_11535_gb300 import gen

torch = pytest.importorskip("torch")

FORMS = {"staged": 0, "fused": 1, "plain": 2}


@pytest.fixture(scope="module")
def ctx(cfg):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_11535_gb300 import m3e
    c = m3e.Context(cfg, 0)
    yield c
    c.close()


def _tie_frame(cfg):
    g = cfg["geometry"]
    pitch = g["pitch_mm"]
    R, phic = 100.0, 1.0  # transverse radius and centre direction of the track circle

    def column(L, phi):
        ntot = g["n_ladders"][L] * g["n_cols"][L]
        gg = int(math.floor((phi % (2 * math.pi)) * ntot / (2 * math.pi)))
        return gg // g["n_cols"][L], gg % g["n_cols"][L]

    row0 = [round(g["half_len_mm"][L] / pitch) for L in range(4)]  # the row of z = +pitch/2
    hits = []
    for L in range(3):
        lad, col = column(L, phic - math.acos(g["r_mm"][L] / (2 * R)))
        hits.append(int(gen.encode(L, lad, col, row0[L])))
    lad3, col3 = column(3, phic - math.acos(g["r_mm"][3] / (2 * R)))
    low = int(gen.encode(3, lad3, col3, row0[3] - 1))   # z = -0.04 mm, the smaller address
    high = int(gen.encode(3, lad3, col3, row0[3] + 1))  # z = +0.12 mm
    return hits, low, high


def test_coordinates_make_an_exact_fp32_tie(cfg, ocfg):
    """(CPU) the frame's FP32 coordinates tie exactly, and the lower row has the smaller address."""
    hits, low, high = _tie_frame(cfg)
    z = [np.float32(O.decode(ocfg, a).z) for a in hits + [low, high]]
    assert z[0] == z[1] == z[2] == np.float32(0.04)
    assert np.float32(z[4] - z[2]) == np.float32(z[2] - z[3])
    assert low < high


@pytest.mark.gpu
@pytest.mark.parametrize("form", sorted(FORMS))
@pytest.mark.parametrize("low_first", [True, False])
def test_equal_metrics_go_to_the_smaller_address(ctx, cfg, ocfg, form, low_first):
    hits, low, high = _tie_frame(cfg)
    addrs = np.array(hits + ([low, high] if low_first else [high, low]), np.int32)
    want = 3 if low_first else 4  # input index of the lower-row hit
    o = O.select_frame(ocfg, addrs)
    assert o["n_triplets"] == 1 and list(o["tracks"][0].i) == [0, 1, 2, want]
    h = torch.from_numpy(addrs).cuda()
    off = torch.tensor([0, addrs.size], dtype=torch.int64, device="cuda")
    rec = {k: v.cpu().numpy() for k, v in ctx.select_frames_debug(h, off, form=FORMS[form]).items()}
    assert int(rec["n_trip"][0]) == 1
    assert sorted(rec["trip"][0, 0, :3].tolist()) == [0, 1, 2]
    assert int(rec["trip"][0, 0, 3]) == want
