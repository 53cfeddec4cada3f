"""The rewritten forms of three steps of the track stage (Sec. "Triplets Fit",
Algorithm 3: the estimated layer-3 point and the closest layer-3 hit) return what the
plain forms return.  The forms are restated here in numpy FP32 with their arguments:

- the first circle crossing reached from h2 in the turning sense, chosen by half
  planes and a 2D cross product instead of comparing two atan2 turning angles;
- the azimuth difference of two hits wrapped to [-pi, pi] by one fused multiply-add
  with rint(d / 2 pi) instead of conditional subtractions of 2 pi;
- the straight scan of the layer-3 hits that reads no addresses (it flags an equal
  metric and only then repeats the scan with the address rule) against the scan with
  the rule (ties to the smaller address).
"""
import numpy as np

F = np.float32
TWO_PI_F = F(6.28318530717958647692)
PI_F = F(3.14159265358979323846)


def _fma32(a, b, c):
    """a * b + c rounded once to FP32 (the FP64 product of two FP32 values is exact)."""
    return (np.float64(a) * np.float64(b) + np.float64(c)).astype(F)


def _wrap_2pi(a):
    a = a.copy()
    a = np.where(a < 0, (a + TWO_PI_F).astype(F), a)
    a = np.where(a >= TWO_PI_F, (a - TWO_PI_F).astype(F), a)
    return a


def _wrap_pi(a):
    a = np.where(a > PI_F, (a - TWO_PI_F).astype(F), a)
    a = np.where(a < -PI_F, (a + TWO_PI_F).astype(F), a)
    return a


def test_first_crossing_by_half_planes():
    rng = np.random.default_rng(11)
    n = 200_000
    # w: from the circle centre to h2; v0, v1: to the two crossings; eps: turning sense
    w = rng.normal(size=(n, 2)).astype(F)
    v0 = rng.normal(size=(n, 2)).astype(F)
    v1 = rng.normal(size=(n, 2)).astype(F)
    eps = np.where(rng.random(n) < 0.5, F(1), F(-1))
    cr0 = (w[:, 0] * v0[:, 1] - w[:, 1] * v0[:, 0]).astype(F)
    dt0 = (w[:, 0] * v0[:, 0] + w[:, 1] * v0[:, 1]).astype(F)
    cr1 = (w[:, 0] * v1[:, 1] - w[:, 1] * v1[:, 0]).astype(F)
    dt1 = (w[:, 0] * v1[:, 0] + w[:, 1] * v1[:, 1]).astype(F)
    # plain form: the two turning angles in [0, 2 pi), the smaller wins (ties to crossing 0)
    al0 = _wrap_2pi((-eps * np.arctan2(cr0, dt0)).astype(F))
    al1 = _wrap_2pi((-eps * np.arctan2(cr1, dt1)).astype(F))
    plain = al1 < al0
    # rewritten form
    t0, t1 = (-eps * cr0).astype(F), (-eps * cr1).astype(F)
    lo0, lo1 = ~(t0 < 0), ~(t1 < 0)
    cross = (np.float64(dt0) * t1 - np.float64(t0) * dt1)
    fast = (lo1 & ~lo0) | ((lo1 == lo0) & (cross < 0))
    differ = plain != fast
    # they may differ only where the two turns are equal to rounding
    assert differ.sum() <= 5
    assert np.all(np.abs(al0[differ] - al1[differ]) < 1e-5)
    # and the chosen turn equals the smaller of the two
    chosen = np.where(fast, al1, al0)
    assert np.all(chosen[~differ] == np.minimum(al0, al1)[~differ])


def test_azimuth_difference_wrap_by_rint():
    rng = np.random.default_rng(12)
    a = rng.uniform(0, float(TWO_PI_F), 1_000_000).astype(F)
    b = rng.uniform(0, float(TWO_PI_F), 1_000_000).astype(F)
    # special values: equal azimuths, the ends of [0, 2 pi), differences near +-pi
    a = np.concatenate([a, np.array([0, 0, TWO_PI_F * F(0.999999), PI_F, PI_F], F)])
    b = np.concatenate([b, np.array([0, TWO_PI_F * F(0.999999), 0, 0, F(0)], F)])
    d = (a - b).astype(F)
    plain = _wrap_pi(d)
    k = np.rint((d * F(1.0 / 6.28318530717958647692)).astype(F)).astype(F)
    fast = _fma32(-TWO_PI_F, k, d)
    same = plain == fast
    # elsewhere only at |d| = pi to rounding, where the two choices have equal size
    assert np.all(np.abs(np.abs(d[~same]) - PI_F) < 1e-6)
    assert np.all(np.abs(np.abs(plain[~same]) - np.abs(fast[~same])) < 1e-6)
    assert np.all(np.abs(fast) <= PI_F + 1e-6)


def _scan_with_rule(m, addr):
    best, mb, ab = -1, np.float32(np.finfo(np.float32).max), 0
    for j in range(len(m)):
        if best < 0 or m[j] < mb or (m[j] == mb and addr[j] < ab):
            best, mb, ab = j, m[j], addr[j]
    return best


def _scan_with_flag(m, addr):
    if len(m) == 0:
        return -1
    best, mb, tie = 0, m[0], False
    for j in range(1, len(m)):
        if m[j] < mb:
            best, mb, tie = j, m[j], False
        elif m[j] == mb:
            tie = True
    return _scan_with_rule(m, addr) if tie else best


def test_address_free_scan_returns_the_rule_hit():
    rng = np.random.default_rng(13)
    for trial in range(20_000):
        n = int(rng.integers(0, 40))
        # metrics from a small set, so that equal metrics are frequent, and a few NaN
        m = rng.choice(np.array([0.5, 1.0, 2.0, 3.0, np.nan], F), size=n, p=[0.3, 0.3, 0.2, 0.15, 0.05])
        addr = rng.permutation(1000)[:n].astype(np.uint32)
        assert _scan_with_flag(m, addr) == _scan_with_rule(m, addr), (m, addr)
