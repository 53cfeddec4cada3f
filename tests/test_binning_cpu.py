"""The phi bin of a pixel column, floor(g * NB / ntot), as the kernels compute it:
one FP32 addition and one FP32 multiplication by 1/ntot (rounded once), with no
integer division.  Checked against the integer division for every column of every
layer size the configuration admits (1..32 ladders x 1..256 columns)."""
import numpy as np

NB = 32  # phi bins per layer, as in the kernels


def test_float_bin_equals_the_integer_division():
    sizes = np.unique(np.outer(np.arange(1, 33), np.arange(1, 257)).ravel())
    for n in sizes:
        g = np.arange(n, dtype=np.int64)
        m = g * NB
        inv = np.float32(1.0 / float(n))
        b = ((m.astype(np.float32) + np.float32(0.5)) * inv).astype(np.int32)
        assert (b == m // n).all(), n
