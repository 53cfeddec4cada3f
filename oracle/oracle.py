"""ctypes loader of the FP64 CPU oracle (``oracle/m3e_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, the smoke check and the CPU
baseline leg of ``bench.py``.  It shares no code with the CUDA library; it reads
the same JSON parameter file and fills its own struct.
"""
from __future__ import annotations

import ctypes as C
import json
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "m3e_oracle.c")
LIB = os.path.join(HERE, "liborc.so")

DROP, VERTEX, TRIPLET_OVERFLOW, TRACK_OVERFLOW, COMBO_OVERFLOW, HIT_OVERFLOW, ERR_BADHIT = range(7)


def build(force: bool = False) -> str:
    """Compile the oracle with plain -O2 (no intrinsics, no -march)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "m3e_oracle.h"))):
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", LIB, SRC, "-lm", "-lpthread"])
    return LIB


class Config(C.Structure):
    _fields_ = [("r", C.c_double * 4), ("H", C.c_double * 4),
                ("nlad", C.c_int32 * 4), ("ncol", C.c_int32 * 4), ("nrow", C.c_int32 * 4),
                ("pitch", C.c_double),
                ("B", C.c_double), ("field_scale", C.c_double), ("x_over_X0", C.c_double * 4),
                ("k", C.c_double), ("m_mu", C.c_double), ("m_e", C.c_double),
                ("target_r", C.c_double), ("target_half_len", C.c_double),
                ("dlambda_max", C.c_double), ("phi01_max", C.c_double), ("phi12_max", C.c_double),
                ("rtc_min", C.c_double), ("rtc_max", C.c_double), ("chi2_track_max", C.c_double),
                ("e_window", C.c_double), ("isect_margin", C.c_double), ("vtx_chi2_max", C.c_double),
                ("target_dist_max", C.c_double), ("ptot_max", C.c_double),
                ("max_hits", C.c_int32), ("max_triplets", C.c_int32), ("max_tracks", C.c_int32),
                ("max_combos", C.c_int32)]


class Hit(C.Structure):
    _fields_ = [("x", C.c_double), ("y", C.c_double), ("z", C.c_double),
                ("layer", C.c_int32), ("ladder", C.c_int32), ("col", C.c_int32), ("row", C.c_int32),
                ("addr", C.c_uint32), ("in_idx", C.c_int32), ("phi", C.c_double)]


class TFit(C.Structure):
    _fields_ = [("valid", C.c_int32), ("rtc", C.c_double), ("Rct", C.c_double), ("eps", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double),
                ("d", C.c_double * 2), ("zs", C.c_double * 2), ("phiC", C.c_double * 2), ("RC", C.c_double * 2),
                ("thetaC", C.c_double * 2), ("dphi", C.c_double * 2), ("dtheta", C.c_double * 2),
                ("alpha", C.c_double), ("a0", C.c_double), ("beta", C.c_double), ("b0", C.c_double),
                ("s", C.c_double), ("Rstar", C.c_double), ("sigmaR", C.c_double), ("kappa", C.c_double),
                ("sigma_kappa", C.c_double), ("chi2min", C.c_double), ("sigma_ms", C.c_double)]


class TripRec(C.Structure):
    _fields_ = [("i", C.c_int32 * 3), ("dlambda", C.c_double), ("cos01", C.c_double), ("cos12", C.c_double),
                ("rtc", C.c_double)]


class TrackRec(C.Structure):
    _fields_ = [("i", C.c_int32 * 4), ("status", C.c_int32), ("m_best", C.c_double), ("m_second", C.c_double),
                ("kappa1", C.c_double), ("kappa2", C.c_double), ("sk1", C.c_double), ("sk2", C.c_double),
                ("kappa_bar", C.c_double), ("R_bar", C.c_double), ("theta01", C.c_double), ("chi2", C.c_double)]


class ComboRec(C.Structure):
    _fields_ = [("t", C.c_int32 * 3), ("de", C.c_double), ("status", C.c_int32), ("pass_", C.c_int32),
                ("chi2", C.c_double), ("tdist", C.c_double), ("ptot", C.c_double), ("chi2_second", C.c_double),
                ("disc_min", C.c_double), ("filt_margin", C.c_double), ("mu", C.c_double * 3),
                ("pvec", (C.c_double * 3) * 3)]


class FrameOut(C.Structure):
    _fields_ = [("reason", C.c_int32), ("keep", C.c_int32), ("n_hits", C.c_int32), ("n_layer", C.c_int32 * 4),
                ("n_tested", C.c_int64), ("n_pass", C.c_int64 * 4),
                ("n_triplets", C.c_int32), ("n_tracks", C.c_int32), ("n_combos", C.c_int32),
                ("n_vertexed", C.c_int32),
                ("trips", C.POINTER(TripRec)), ("trips_cap", C.c_int32), ("trips_n", C.c_int32),
                ("trks", C.POINTER(TrackRec)), ("trks_cap", C.c_int32), ("trks_n", C.c_int32),
                ("kept_trk", C.POINTER(C.c_int32)), ("kept_cap", C.c_int32), ("kept_n", C.c_int32),
                ("combos", C.POINTER(ComboRec)), ("combos_cap", C.c_int32), ("combos_n", C.c_int32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.POINTER
        _lib.orc_decode.argtypes = [P(Config), C.c_uint32, P(Hit)]
        _lib.orc_cut_vars.argtypes = [P(Config), P(C.c_double), P(C.c_double), P(C.c_double), P(C.c_double)]
        _lib.orc_fit_triplet.argtypes = [P(Config), P(C.c_double), P(C.c_double), P(C.c_double), C.c_int,
                                         P(TFit)]
        _lib.orc_highland.argtypes = [P(Config), C.c_double, C.c_int]
        _lib.orc_highland.restype = C.c_double
        _lib.orc_select_frame.argtypes = [P(Config), P(C.c_int32), C.c_int32, P(FrameOut)]
        _lib.orc_select_frame_hits.argtypes = [P(Config), P(Hit), C.c_int32, P(FrameOut)]
        _lib.orc_select_frames.argtypes = [P(Config), P(C.c_int32), P(C.c_int64), C.c_int64, P(C.c_uint8),
                                           P(C.c_uint8), C.c_int32, P(C.c_int64)]
        _lib.orc_fit_track_positions.argtypes = [P(Config), P(C.c_double), P(C.c_double)]
        _lib.orc_align_point.argtypes = [P(C.c_double), P(C.c_double), P(C.c_double)]
        _lib.orc_fit_chi2.argtypes = [P(Config), P(C.c_int32), C.c_int64, P(C.c_int32), C.c_int64, P(C.c_double),
                                      P(C.c_double), C.c_int32]
        _lib.orc_fit_chi2.restype = C.c_int64
        _lib.orc_fit_triplet_exact.argtypes = [P(Config), P(C.c_double), P(C.c_double), P(C.c_double), C.c_int,
                                               C.c_double, C.c_double, P(C.c_double)]
    return _lib


def make_config(cfg: dict, **override) -> Config:
    """Fill the oracle's parameter struct from the JSON dictionary."""
    g, cu, ca = cfg["geometry"], cfg["cuts"], cfg["caps"]
    c = Config()
    c.r[:] = g["r_mm"]; c.H[:] = g["half_len_mm"]
    c.nlad[:] = g["n_ladders"]; c.ncol[:] = g["n_cols"]; c.nrow[:] = g["n_rows"]
    c.pitch = g["pitch_mm"]
    c.B = cfg["field"]["B_T"]; c.field_scale = cfg["field"]["field_scale"]
    c.x_over_X0[:] = cfg["material"]["x_over_X0"]
    k = cfg["constants"]
    c.k = k["k_MeV_per_T_mm"]; c.m_mu = k["m_mu_MeV"]; c.m_e = k["m_e_MeV"]
    c.target_r = cfg["target"]["r_mm"]; c.target_half_len = cfg["target"]["half_len_mm"]
    for name in ("dlambda_max", "phi01_max", "phi12_max", "rtc_min", "rtc_max", "chi2_track_max", "e_window",
                 "isect_margin", "vtx_chi2_max", "target_dist_max", "ptot_max"):
        setattr(c, name, float(cu[name]))
    for name in ("max_hits", "max_triplets", "max_tracks", "max_combos"):
        setattr(c, name, int(ca[name]))
    for kk, v in override.items():
        setattr(c, kk, v)
    return c


def load_config_json(path: str | None = None) -> dict:
    path = path or os.path.join(os.path.dirname(HERE), "paper_2206_11535_gb300", "configs", "default.json")
    with open(path) as f:
        return json.load(f)


def _dp(a):
    a = np.ascontiguousarray(a, np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def decode(c: Config, addr: int):
    h = Hit()
    rc = lib().orc_decode(C.byref(c), C.c_uint32(int(addr) & 0xffffffff), C.byref(h))
    return None if rc else h


def cut_vars(c: Config, h0, h1, h2) -> np.ndarray:
    a, pa = _dp(h0); b, pb = _dp(h1); d, pd = _dp(h2)
    v, pv = _dp(np.zeros(4))
    lib().orc_cut_vars(C.byref(c), pa, pb, pd, pv)
    return v


def fit_triplet(c: Config, ha, hb, hc, mid_layer: int) -> TFit:
    a, pa = _dp(ha); b, pb = _dp(hb); d, pd = _dp(hc)
    f = TFit()
    lib().orc_fit_triplet(C.byref(c), pa, pb, pd, mid_layer, C.byref(f))
    return f


def fit_triplet_exact(c: Config, ha, hb, hc, mid_layer: int, r_lo: float, r_hi: float):
    a, pa = _dp(ha); b, pb = _dp(hb); d, pd = _dp(hc)
    out = C.c_double()
    rc = lib().orc_fit_triplet_exact(C.byref(c), pa, pb, pd, mid_layer, r_lo, r_hi, C.byref(out))
    return None if rc else out.value


def highland(c: Config, p: float, layer: int) -> float:
    return lib().orc_highland(C.byref(c), p, layer)


def fit_track_positions(c: Config, h4) -> np.ndarray | None:
    a, pa = _dp(np.asarray(h4, float).reshape(12))
    o, po = _dp(np.zeros(4))
    rc = lib().orc_fit_track_positions(C.byref(c), pa, po)
    return None if rc else o


def select_frame(c: Config, addrs, records: bool = True, caps=(1024, 1024, 1024, 2048), positions=None) -> dict:
    """One frame; returns reason/keep/stats and (records=True) the kept triplets,
    the track reconstruction of each kept triplet, the kept-track list and the
    energy-test combinations with their vertex results (indices are input indices).
    With ``positions`` (n x 3, FP64), ``addrs`` holds the layer of each hit instead
    and no pixel decoding takes place."""
    o = FrameOut()
    bufs = []
    if records:
        tr = (TripRec * caps[0])(); tk = (TrackRec * caps[1])(); kt = (C.c_int32 * caps[2])()
        cb = (ComboRec * caps[3])()
        bufs = [tr, tk, kt, cb]
        o.trips = C.cast(tr, C.POINTER(TripRec)); o.trips_cap = caps[0]
        o.trks = C.cast(tk, C.POINTER(TrackRec)); o.trks_cap = caps[1]
        o.kept_trk = C.cast(kt, C.POINTER(C.c_int32)); o.kept_cap = caps[2]
        o.combos = C.cast(cb, C.POINTER(ComboRec)); o.combos_cap = caps[3]
    if positions is None:
        a = np.ascontiguousarray(addrs, np.int32)
        rc = lib().orc_select_frame(C.byref(c), a.ctypes.data_as(C.POINTER(C.c_int32)), a.size, C.byref(o))
    else:
        lay = np.asarray(addrs, np.int64)  # layers when positions are given
        hs = (Hit * max(len(lay), 1))()
        for i in range(len(lay)):
            hs[i].x, hs[i].y, hs[i].z = (float(v) for v in positions[i])
            hs[i].layer = int(lay[i])
            hs[i].addr = (int(lay[i]) << 26) | i
        rc = lib().orc_select_frame_hits(C.byref(c), hs, len(lay), C.byref(o))
    if rc:
        raise RuntimeError("oracle failed")
    out = dict(reason=o.reason, keep=o.keep, n_hits=o.n_hits, n_layer=list(o.n_layer), n_tested=o.n_tested,
               n_pass=list(o.n_pass), n_triplets=o.n_triplets, n_tracks=o.n_tracks, n_combos=o.n_combos,
               n_vertexed=o.n_vertexed)
    if records:
        tr, tk, kt, cb = bufs
        out["trips"] = [tr[i] for i in range(o.trips_n)]
        out["tracks"] = [tk[i] for i in range(o.trks_n)]
        out["kept"] = [kt[i] for i in range(o.kept_n)]
        out["combos"] = [cb[i] for i in range(o.combos_n)]
    return out


def select_frames(c: Config, hits, off, n_threads: int = 1, counts: bool = False):
    """Batch of frames (threads over disjoint frame ranges).  Returns keep, reason and,
    with counts=True, an (F, 8) int64 array of per-frame work counts."""
    h = np.ascontiguousarray(hits, np.int32)
    o = np.ascontiguousarray(off, np.int64)
    nf = o.size - 1
    keep = np.zeros(max(nf, 1), np.uint8); reason = np.zeros(max(nf, 1), np.uint8)
    cnt = np.zeros((max(nf, 1), 8), np.int64) if counts else None
    rc = lib().orc_select_frames(C.byref(c), h.ctypes.data_as(C.POINTER(C.c_int32)),
                                 o.ctypes.data_as(C.POINTER(C.c_int64)), nf,
                                 keep.ctypes.data_as(C.POINTER(C.c_uint8)),
                                 reason.ctypes.data_as(C.POINTER(C.c_uint8)), n_threads,
                                 cnt.ctypes.data_as(C.POINTER(C.c_int64)) if counts else None)
    if rc:
        raise RuntimeError("oracle batch failed")
    if counts:
        return keep[:nf], reason[:nf], cnt[:nf]
    return keep[:nf], reason[:nf]


# ---------------------------------------------------------------- alignment and the fit gradient

N_PARAMS = 25  # 4 layers x (dx, dy, dz [mm], wx, wy, wz [rad]) and the field scale


def nominal_params() -> np.ndarray:
    p = np.zeros(N_PARAMS)
    p[24] = 1.0
    return p


def align_point(p6, x_nom) -> np.ndarray:
    """R(w) x_nom + d for one layer's params (dx, dy, dz, wx, wy, wz), R = Rz Ry Rx."""
    (_, pa), (_, pb), o = _dp(p6), _dp(x_nom), np.zeros(3)
    lib().orc_align_point(pa, pb, o.ctypes.data_as(C.POINTER(C.c_double)))
    return o


def fit_chi2(c: Config, hits, cand, params, n_threads: int = 1) -> np.ndarray:
    """chi2 of each frozen candidate (rows of 4 global hit indices, layers 0..3) at the
    given alignment and field scale; NaN where a fit is invalid."""
    h = np.ascontiguousarray(hits, np.int32)
    q = np.ascontiguousarray(cand, np.int32).reshape(-1, 4)
    _, pr = _dp(params)
    out = np.empty(max(q.shape[0], 1))
    lib().orc_fit_chi2(C.byref(c), h.ctypes.data_as(C.POINTER(C.c_int32)), h.size,
                       q.ctypes.data_as(C.POINTER(C.c_int32)), q.shape[0], pr,
                       out.ctypes.data_as(C.POINTER(C.c_double)), n_threads)
    return out[:q.shape[0]]


FD_STEPS = ([1e-4] * 3 + [1e-6] * 3) * 4 + [1e-6]  # central-difference steps: mm, rad, scale


def fit_grad_fd(c: Config, hits, cand, params, n_threads: int = 1, steps=None):
    """Sum of chi2 over the candidates valid at ``params`` and its gradient by central
    differences in FP64 (the definition of the derivative, error O(h^2)): the
    reference for the gradient kernel.  Returns (sum, grad[25], valid mask)."""
    p0 = np.array(params, np.float64)
    base = fit_chi2(c, hits, cand, p0, n_threads)
    ok = np.isfinite(base)
    sel = np.ascontiguousarray(np.asarray(cand, np.int32).reshape(-1, 4)[ok])
    g = np.zeros(N_PARAMS)
    for i, h in enumerate(steps or FD_STEPS):
        pp, pm = p0.copy(), p0.copy()
        pp[i] += h
        pm[i] -= h
        fp = fit_chi2(c, hits, sel, pp, n_threads)
        fm = fit_chi2(c, hits, sel, pm, n_threads)
        if not (np.isfinite(fp).all() and np.isfinite(fm).all()):
            raise RuntimeError(f"a candidate's fit fails under the step of parameter {i}")
        g[i] = (fp.sum() - fm.sum()) / (2.0 * h)
    return float(base[ok].sum()), g, ok
