"""Python binding of libm3e (``include/m3e.h``): argument marshalling only.

Every computation runs in the library's CUDA kernels; this module converts torch
tensors (device memory, streams) and numpy arrays (host memory) into the plain
pointers and sizes of the C ABI.  Importing it loads ``libm3e.so`` and raises if
the library has not been built (``paper_2206_11535_gb300.build.build()``):
there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libm3e.so")

OK, EINVAL, ENOMEM, EBADHIT, ECUDA, EBUSY, ETIMEOUT, ESTATE = 0, -1, -2, -3, -4, -5, -6, -7
STAGED, FUSED, PLAIN = 0, 1, 2  # forms of the selection (m3e_select_frames_debug)
DROP, VERTEX, TRIPLET_OVERFLOW, TRACK_OVERFLOW, COMBO_OVERFLOW, HIT_OVERFLOW, ERR_BADHIT = range(7)
REASONS = ("DROP", "VERTEX", "TRIPLET_OVERFLOW", "TRACK_OVERFLOW", "COMBO_OVERFLOW", "HIT_OVERFLOW", "ERR_BADHIT")


class M3EError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"m3e error {code}: {msg}")
        self.code = code


class Config(C.Structure):
    _fields_ = [("size", C.c_uint32),
                ("r_mm", C.c_double * 4), ("half_len_mm", C.c_double * 4),
                ("n_ladders", C.c_int32 * 4), ("n_cols", C.c_int32 * 4), ("n_rows", C.c_int32 * 4),
                ("pitch_mm", C.c_double), ("B_T", C.c_double), ("field_scale", C.c_double),
                ("x_over_X0", C.c_double * 4),
                ("k_MeV_per_T_mm", C.c_double), ("m_mu_MeV", C.c_double), ("m_e_MeV", C.c_double),
                ("target_r_mm", C.c_double), ("target_half_len_mm", C.c_double),
                ("dlambda_max", C.c_double), ("phi01_max", C.c_double), ("phi12_max", C.c_double),
                ("rtc_min", C.c_double), ("rtc_max", C.c_double), ("chi2_track_max", C.c_double),
                ("e_window", C.c_double), ("isect_margin", C.c_double), ("vtx_chi2_max", C.c_double),
                ("target_dist_max", C.c_double), ("ptot_max", C.c_double),
                ("max_hits", C.c_int32), ("max_triplets", C.c_int32), ("max_tracks", C.c_int32),
                ("max_combos", C.c_int32)]


STATS_FIELDS = ("frames", "hits", "pair_tests", "triplet_tests", "triplets", "tracks", "energy_tests", "combos",
                "vertexed", "deferred", "pz_open", "vertexed_pz_open")
N_STATS = len(STATS_FIELDS) + 8


class Dump(C.Structure):
    _fields_ = [("cap_trip", C.c_int32), ("cap_combo", C.c_int32),
                ("n_trip", C.c_void_p), ("trip", C.c_void_p), ("trk_status", C.c_void_p), ("trk_val", C.c_void_p),
                ("n_combo", C.c_void_p), ("combo", C.c_void_p), ("combo_val", C.c_void_p),
                ("combo_aux", C.c_void_p)]


class Tuning(C.Structure):
    _fields_ = [("frames_per_grab", C.c_int32), ("defer_hits", C.c_int32), ("s1_ctas_per_sm", C.c_int32),
                ("configs_tried", C.c_int32), ("ms_default", C.c_float), ("ms_best", C.c_float),
                ("mid_cta_threads", C.c_int32), ("s2_ctas_per_sm", C.c_int32), ("ms_worst", C.c_float)]


class Result(C.Structure):
    """``m3e_result``: one submitted frame's result slot (written by the library)."""
    _fields_ = [("done", C.c_uint32), ("keep", C.c_uint8), ("reason", C.c_uint8), ("reserved", C.c_uint16),
                ("err", C.c_int32), ("tag", C.c_uint64), ("t_submit_ns", C.c_uint64), ("t_done_ns", C.c_uint64)]


class StreamParams(C.Structure):
    _fields_ = [("size", C.c_uint32), ("slots", C.c_int32), ("ring_bytes", C.c_int64), ("ctas_per_sm", C.c_int32),
                ("idle_us", C.c_int32), ("lifetime_ms", C.c_int32), ("wait_limit_ms", C.c_int32),
                ("no_feeder", C.c_int32)]


class StreamStatus(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("busy_refusals", C.c_uint64),
                ("kernel_launches", C.c_uint64), ("heavy_frames", C.c_uint64), ("delivery_passes", C.c_uint64),
                ("tail_publications", C.c_uint64), ("kernel_running", C.c_int32),
                ("failed", C.c_int32)]


class ReplayStats(C.Structure):
    _fields_ = [("offered_hz", C.c_double), ("sustained_hz", C.c_double), ("submit_hz", C.c_double),
                ("busy_retries", C.c_uint64), ("kernel_launches", C.c_uint64), ("duration_ns", C.c_int64)]


def _load(path: str = LIB_PATH):
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2206_11535_gb300.build.build() "
                           "(the selection has no CPU path)")
    lib = C.CDLL(path)
    vp, i64 = C.c_void_p, C.c_int64
    lib.m3e_create.argtypes = [C.POINTER(Config), C.c_int, C.POINTER(vp)]
    lib.m3e_destroy.argtypes = [vp]
    for name in ("m3e_select_frames", "m3e_select_frames_fused", "m3e_select_frames_plain"):
        getattr(lib, name).argtypes = [vp, vp, vp, i64, vp, vp, vp, vp]
    lib.m3e_select_frames_debug.argtypes = [vp, C.c_int, vp, vp, i64, vp, vp, C.POINTER(Dump), vp]
    lib.m3e_stage_times.argtypes = [vp, C.POINTER(C.c_float), C.c_int]
    lib.m3e_prepare.argtypes = [vp, i64]
    lib.m3e_graph_create.argtypes = [vp, C.c_int, vp, vp, i64, vp, vp, C.POINTER(vp)]
    lib.m3e_graph_launch.argtypes = [vp, vp]
    lib.m3e_graph_destroy.argtypes = [vp]
    lib.m3e_autotune.argtypes = [vp, vp, vp, i64, vp, vp, C.POINTER(Tuning)]
    lib.m3e_select_frames_host.argtypes = [vp, vp, vp, i64, vp, vp, vp]
    lib.m3e_select_frames_noalloc.argtypes = [vp, vp, vp, i64, vp, vp, vp]
    lib.m3e_ingest.argtypes = [vp, vp, i64, vp, vp, vp, vp, vp]
    lib.m3e_check.argtypes = [vp, vp]
    lib.m3e_set_launch.argtypes = [vp, C.c_int, C.c_int]
    lib.m3e_set_host_pipeline.argtypes = [vp, C.c_int, C.c_int, C.c_int]
    lib.m3e_last_launch_count.argtypes = [vp]
    lib.m3e_last_error_string.restype = C.c_char_p
    lib.m3e_set_profiling.argtypes = [vp, C.c_int]
    lib.m3e_fit_grad.argtypes = [vp, vp, vp, i64, vp, i64, vp, vp, vp, vp]
    lib.m3e_fit_chi2.argtypes = [vp, vp, vp, i64, vp, i64, vp, vp, vp]
    lib.m3e_fit_kappa.argtypes = [vp, vp, vp, i64, vp, i64, vp, vp, vp]
    lib.m3e_fit_valid_count.argtypes = [vp, vp, C.POINTER(C.c_int64)]
    lib.m3e_stream_open.argtypes = [vp, C.POINTER(StreamParams)]
    lib.m3e_stream_submit.argtypes = [vp, vp, C.c_int32, C.c_uint64, vp]
    lib.m3e_stream_submit_many.argtypes = [vp, vp, vp, i64, vp, vp, C.POINTER(C.c_int64)]
    lib.m3e_stream_poll.argtypes = [vp, C.POINTER(StreamStatus)]
    lib.m3e_stream_drain.argtypes = [vp, i64]
    lib.m3e_stream_close.argtypes = [vp]
    lib.m3e_stream_replay.argtypes = [vp, vp, vp, i64, C.c_double, C.c_uint64, vp, vp, vp, vp,
                                      C.POINTER(ReplayStats)]
    lib.m3e_kernel_times.argtypes = [vp, C.POINTER(C.c_float), C.POINTER(C.c_float)]
    return lib


lib = _load()


def version() -> int:
    return lib.m3e_version()


def _check(rc: int):
    if rc != OK:
        raise M3EError(rc, lib.m3e_last_error_string().decode())


def config_from_json(cfg: dict, **override) -> Config:
    """Fill the library's parameter struct from the JSON parameter dictionary."""
    g, cu, ca = cfg["geometry"], cfg["cuts"], cfg["caps"]
    c = Config()
    c.size = C.sizeof(Config)
    c.r_mm[:] = g["r_mm"]; c.half_len_mm[:] = g["half_len_mm"]
    c.n_ladders[:] = g["n_ladders"]; c.n_cols[:] = g["n_cols"]; c.n_rows[:] = g["n_rows"]
    c.pitch_mm = g["pitch_mm"]
    c.B_T = cfg["field"]["B_T"]; c.field_scale = cfg["field"]["field_scale"]
    c.x_over_X0[:] = cfg["material"]["x_over_X0"]
    k = cfg["constants"]
    c.k_MeV_per_T_mm = k["k_MeV_per_T_mm"]; c.m_mu_MeV = k["m_mu_MeV"]; c.m_e_MeV = k["m_e_MeV"]
    c.target_r_mm = cfg["target"]["r_mm"]; c.target_half_len_mm = cfg["target"]["half_len_mm"]
    for name in ("dlambda_max", "phi01_max", "phi12_max", "rtc_min", "rtc_max", "chi2_track_max", "e_window",
                 "isect_margin", "vtx_chi2_max", "target_dist_max", "ptot_max"):
        setattr(c, name, float(cu[name]))
    for name in ("max_hits", "max_triplets", "max_tracks", "max_combos"):
        setattr(c, name, int(ca[name]))
    for kk, v in override.items():
        setattr(c, kk, v)
    return c


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


class Context:
    """An m3e context on one CUDA device (``m3e_create`` / ``m3e_destroy``)."""

    def __init__(self, cfg: dict | Config | None = None, device: int = 0):
        if cfg is None:
            from . import gen
            cfg = gen.load_config()
        self.config = cfg if isinstance(cfg, Config) else config_from_json(cfg)
        self.device = device
        h = C.c_void_p()
        _check(lib.m3e_create(C.byref(self.config), device, C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _check(lib.m3e_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- entry points (device tensors) -------------------------------------------------------
    def _outs(self, hits, off, keep, reason):
        import torch
        nf = off.numel() - 1
        dev = off.device
        if keep is None:
            keep = torch.empty(nf, dtype=torch.uint8, device=dev)
        if reason is None:
            reason = torch.empty(nf, dtype=torch.uint8, device=dev)
        return nf, keep, reason

    def select_frames(self, hits, off, keep=None, reason=None, stats=None, stream=None):
        """``m3e_select_frames`` on int32 ``hits`` and int64 ``off`` (CUDA tensors).
        Returns (keep, reason) uint8 tensors."""
        nf, keep, reason = self._outs(hits, off, keep, reason)
        _check(lib.m3e_select_frames(self._h, _ptr(hits), _ptr(off), nf, _ptr(keep), _ptr(reason), _ptr(stats),
                                     _stream(stream)))
        return keep, reason

    def select_frames_fused(self, hits, off, keep=None, reason=None, stats=None, stream=None):
        """``m3e_select_frames_fused``: one persistent kernel, a warp per frame."""
        nf, keep, reason = self._outs(hits, off, keep, reason)
        _check(lib.m3e_select_frames_fused(self._h, _ptr(hits), _ptr(off), nf, _ptr(keep), _ptr(reason),
                                           _ptr(stats), _stream(stream)))
        return keep, reason

    def select_frames_plain(self, hits, off, keep=None, reason=None, stats=None, stream=None):
        """``m3e_select_frames_plain``: one CTA per frame, one launch per batch."""
        nf, keep, reason = self._outs(hits, off, keep, reason)
        _check(lib.m3e_select_frames_plain(self._h, _ptr(hits), _ptr(off), nf, _ptr(keep), _ptr(reason),
                                           _ptr(stats), _stream(stream)))
        return keep, reason

    def select_frames_debug(self, hits, off, cap_trip=768, cap_combo=1024, stream=None, form=STAGED):
        """``m3e_select_frames_debug`` through ``form`` (STAGED, FUSED or PLAIN):
        returns keep, reason and the candidate record (torch tensors on the device,
        frame-major)."""
        import torch
        nf, keep, reason = self._outs(hits, off, None, None)
        dev = off.device
        rec = dict(n_trip=torch.zeros(nf, dtype=torch.int32, device=dev),
                   trip=torch.full((nf, cap_trip, 4), -2, dtype=torch.int32, device=dev),
                   trk_status=torch.full((nf, cap_trip), -1, dtype=torch.int32, device=dev),
                   trk_val=torch.zeros((nf, cap_trip, 4), dtype=torch.float32, device=dev),
                   n_combo=torch.zeros(nf, dtype=torch.int32, device=dev),
                   combo=torch.full((nf, cap_combo, 4), -2, dtype=torch.int32, device=dev),
                   combo_val=torch.zeros((nf, cap_combo, 4), dtype=torch.float32, device=dev),
                   combo_aux=torch.zeros((nf, cap_combo, 4), dtype=torch.float32, device=dev))
        d = Dump(cap_trip, cap_combo, *[_ptr(rec[k]) for k in ("n_trip", "trip", "trk_status", "trk_val", "n_combo",
                                                                  "combo", "combo_val", "combo_aux")])
        _check(lib.m3e_select_frames_debug(self._h, form, _ptr(hits), _ptr(off), nf, _ptr(keep), _ptr(reason),
                                           C.byref(d), _stream(stream)))
        rec["keep"], rec["reason"] = keep, reason
        return rec

    def select_frames_noalloc(self, hits, off, keep, reason, stream=None):
        """``m3e_select_frames_noalloc``: the selection without any device allocation in
        the call, for callers that must not allocate while running (fixed-rate
        loops, fixed memory budgets).  ``keep`` and ``reason`` must be allocated by
        the caller beforehand; at most 262,144 frames per call."""
        nf = off.numel() - 1
        _check(lib.m3e_select_frames_noalloc(self._h, _ptr(hits), _ptr(off), nf, _ptr(keep), _ptr(reason),
                                             _stream(stream)))
        return keep, reason

    def ingest(self, hits, x=None, y=None, z=None, phi=None, with_phi: bool = True, stream=None):
        """``m3e_ingest``: FP32 x, y, z (and phi) of every hit of the int32 device tensor
        ``hits``, as four float32 device tensors (phi is None when not requested)."""
        import torch
        n = hits.numel()
        mk = lambda t: torch.empty(n, dtype=torch.float32, device=hits.device) if t is None else t  # noqa: E731
        x, y, z = mk(x), mk(y), mk(z)
        phi = mk(phi) if with_phi else None
        _check(lib.m3e_ingest(self._h, _ptr(hits), n, _ptr(x), _ptr(y), _ptr(z), _ptr(phi), _stream(stream)))
        return x, y, z, phi

    def set_host_pipeline(self, max_chunks: int = 16, wait_ms: int = 2000, drop_chunk: int = -1):
        """``m3e_set_host_pipeline``: chunking and the bounded chunk wait of
        select_frames_host (drop_chunk >= 0 leaves that chunk's arrival flag unset:
        a test of the wait)."""
        _check(lib.m3e_set_host_pipeline(self._h, max_chunks, wait_ms, drop_chunk))

    def select_frames_host(self, hits: np.ndarray, off: np.ndarray, keep=None, reason=None, stream=None):
        """``m3e_select_frames_host`` on host arrays (numpy or pinned torch CPU tensors).
        Synchronise ``stream`` before reading keep/reason."""
        nf = (off.numel() if hasattr(off, "numel") else off.size) - 1
        if keep is None:
            keep = np.empty(nf, np.uint8)
        if reason is None:
            reason = np.empty(nf, np.uint8)
        _check(lib.m3e_select_frames_host(self._h, _ptr(hits), _ptr(off), nf, _ptr(keep), _ptr(reason),
                                          _stream(stream)))
        return keep, reason

    def check(self, stream=None) -> int:
        """``m3e_check``: synchronise the stream; raises M3EError(EBADHIT) when a frame
        held an invalid address since the last check."""
        _check(lib.m3e_check(self._h, _stream(stream)))
        return OK

    def prepare(self, max_frames: int):
        """``m3e_prepare``: size the scratch for batches of up to max_frames frames."""
        _check(lib.m3e_prepare(self._h, max_frames))

    def graph(self, hits, off, keep, reason, form=STAGED) -> "Graph":
        """``m3e_graph_create``: one batch captured as a CUDA graph."""
        return Graph(self, hits, off, keep, reason, form)

    def autotune(self, hits, off, keep=None, reason=None) -> dict:
        """``m3e_autotune`` on a calibration batch; returns the chosen parameters."""
        nf, keep, reason = self._outs(hits, off, keep, reason)
        t = Tuning()
        _check(lib.m3e_autotune(self._h, _ptr(hits), _ptr(off), nf, _ptr(keep), _ptr(reason), C.byref(t)))
        return {k: getattr(t, k) for k, _ in Tuning._fields_}

    def set_launch(self, frames_per_grab: int, ctas_per_sm: int = 0):
        _check(lib.m3e_set_launch(self._h, frames_per_grab, ctas_per_sm))

    def last_launch_count(self) -> int:
        return lib.m3e_last_launch_count(self._h)

    def set_profiling(self, on: bool = True):
        _check(lib.m3e_set_profiling(self._h, int(on)))

    def stage_times(self) -> list[float]:
        """ms of stage 1 (warp, middle and top tiers), stages 2-5 and the deferred-frame
        kernel of the last timed staged call."""
        a = (C.c_float * 8)()
        _check(lib.m3e_stage_times(self._h, a, 8))
        return list(a)

    def kernel_times(self) -> tuple[float, float]:
        """(main kernel ms, deferred-frame kernel ms) of the last timed select call."""
        a, b = C.c_float(), C.c_float()
        _check(lib.m3e_kernel_times(self._h, C.byref(a), C.byref(b)))
        return a.value, b.value


    # ---------------------------------------------------------------- fit gradient

    def fit_grad(self, hits, off, cand, params, grad: bool = True, stream=None):
        """``m3e_fit_grad``: (chi2 sum, gradient[25] or None) as float32 device tensors.
        cand: int32 device tensor (n, 4) of global hit indices; params: float32 (25,)."""
        import torch
        dev = hits.device
        s = torch.empty(1, dtype=torch.float32, device=dev)
        g = torch.empty(25, dtype=torch.float32, device=dev) if grad else None
        c = cand.contiguous()
        _check(lib.m3e_fit_grad(self._h, _ptr(hits), _ptr(off), off.numel() - 1, _ptr(c), c.shape[0],
                                _ptr(params.contiguous()), _ptr(s), _ptr(g), _stream(stream)))
        return s, g

    def fit_chi2(self, hits, off, cand, params, stream=None):
        """``m3e_fit_chi2``: chi2 of each candidate (NaN where left out)."""
        import torch
        c = cand.contiguous()
        out = torch.empty(c.shape[0], dtype=torch.float32, device=hits.device)
        _check(lib.m3e_fit_chi2(self._h, _ptr(hits), _ptr(off), off.numel() - 1, _ptr(c), c.shape[0],
                                _ptr(params.contiguous()), _ptr(out), _stream(stream)))
        return out

    def fit_kappa(self, hits, off, cand, params, stream=None):
        """``m3e_fit_kappa``: the weighted mean curvature of each candidate's fit (NaN where left out)."""
        import torch
        c = cand.contiguous()
        out = torch.empty(c.shape[0], dtype=torch.float32, device=hits.device)
        _check(lib.m3e_fit_kappa(self._h, _ptr(hits), _ptr(off), off.numel() - 1, _ptr(c), c.shape[0],
                                 _ptr(params.contiguous()), _ptr(out), _stream(stream)))
        return out

    def fit_valid_count(self, stream=None) -> int:
        n = C.c_int64()
        _check(lib.m3e_fit_valid_count(self._h, _stream(stream), C.byref(n)))
        return n.value

    # ---------------------------------------------------------------- streaming

    def stream_open(self, **params):
        """``m3e_stream_open``; keyword arguments are fields of ``m3e_stream_params``."""
        p = StreamParams()
        p.size = C.sizeof(StreamParams)
        for k, v in params.items():
            setattr(p, k, v)
        _check(lib.m3e_stream_open(self._h, C.byref(p)))

    def stream_submit(self, packet: np.ndarray, tag: int, slot: Result) -> int:
        """``m3e_stream_submit`` of one frame (int32 addresses); returns OK or EBUSY, raises otherwise."""
        pk = np.ascontiguousarray(packet, dtype=np.int32)
        rc = lib.m3e_stream_submit(self._h, pk.ctypes.data if pk.size else None, pk.size, tag, C.addressof(slot))
        if rc not in (OK, EBUSY):
            _check(rc)
        return rc

    def stream_submit_many(self, hits: np.ndarray, off: np.ndarray, slots, tags: np.ndarray | None = None) -> int:
        """``m3e_stream_submit_many`` of a host CSR batch into ``slots`` (a ctypes array of
        Result with one slot per frame); returns the number admitted."""
        h = np.ascontiguousarray(hits, dtype=np.int32)
        o = np.ascontiguousarray(off, dtype=np.int64)
        t = None if tags is None else np.ascontiguousarray(tags, dtype=np.uint64)
        n = C.c_int64()
        rc = lib.m3e_stream_submit_many(self._h, h.ctypes.data if h.size else None, o.ctypes.data, o.size - 1,
                                        None if t is None else t.ctypes.data, C.addressof(slots), C.byref(n))
        if rc not in (OK, EBUSY):
            _check(rc)
        return n.value

    def stream_poll(self) -> dict:
        st = StreamStatus()
        _check(lib.m3e_stream_poll(self._h, C.byref(st)))
        return {k: getattr(st, k) for k, _ in StreamStatus._fields_}

    def stream_drain(self, timeout_ms: int = 10000) -> int:
        """``m3e_stream_drain``; returns OK or ETIMEOUT."""
        rc = lib.m3e_stream_drain(self._h, timeout_ms)
        if rc not in (OK, ETIMEOUT):
            _check(rc)
        return rc

    def stream_close(self) -> int:
        return lib.m3e_stream_close(self._h)

    def stream_replay(self, hits: np.ndarray, off: np.ndarray, rate_hz: float, seed: int = 5) -> dict:
        """``m3e_stream_replay``: open-loop Poisson arrivals of a host CSR batch; per-frame decisions
        and latencies (ns) plus the run's rates."""
        h = np.ascontiguousarray(hits, dtype=np.int32)
        o = np.ascontiguousarray(off, dtype=np.int64)
        nf = o.size - 1
        keep = np.zeros(max(nf, 1), np.uint8)
        reason = np.zeros(max(nf, 1), np.uint8)
        ls = np.zeros(max(nf, 1), np.int64)
        la = np.zeros(max(nf, 1), np.int64)
        st = ReplayStats()
        _check(lib.m3e_stream_replay(self._h, h.ctypes.data, o.ctypes.data, nf, float(rate_hz), seed,
                                     keep.ctypes.data, reason.ctypes.data, ls.ctypes.data, la.ctypes.data,
                                     C.byref(st)))
        out = {k: getattr(st, k) for k, _ in ReplayStats._fields_}
        out.update(keep=keep[:nf], reason=reason[:nf], lat_submit_ns=ls[:nf], lat_arrival_ns=la[:nf])
        return out


class Graph:
    """A batch captured as a CUDA graph (``m3e_graph_*``); keeps its buffers alive."""

    def __init__(self, ctx: Context, hits, off, keep, reason, form=STAGED):
        self._bufs = (hits, off, keep, reason)
        self.ctx = ctx
        h = C.c_void_p()
        _check(lib.m3e_graph_create(ctx._h, form, _ptr(hits), _ptr(off), off.numel() - 1, _ptr(keep), _ptr(reason),
                                    C.byref(h)))
        self._h = h

    def launch(self, stream=None):
        _check(lib.m3e_graph_launch(self._h, _stream(stream)))

    def close(self):
        if getattr(self, "_h", None):
            lib.m3e_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def stats_dict(t) -> dict:
    """Decode an ``m3e_stats`` buffer (int64 tensor of N_STATS entries)."""
    v = [int(x) for x in t.cpu().tolist()]
    d = dict(zip(STATS_FIELDS, v[:len(STATS_FIELDS)]))
    d["reasons"] = v[len(STATS_FIELDS):len(STATS_FIELDS) + 8]
    return d


def new_stats(device="cuda"):
    import torch
    return torch.zeros(N_STATS, dtype=torch.int64, device=device)


def kept_candidates(rec: dict, off, min_status: int = 5):
    """Quadruplets (global hit indices, int32 (n, 4)) of the tracks a debug selection
    record holds with track status >= min_status (5: kept by the chi2 cut)."""
    import numpy as _np
    n_trip = _np.asarray(rec["n_trip"])
    trip = _np.asarray(rec["trip"])
    st = _np.asarray(rec["trk_status"])
    cap = trip.shape[1]
    f_idx, t_idx = _np.nonzero((_np.arange(cap)[None, :] < _np.minimum(n_trip, cap)[:, None]) & (st >= min_status))
    q = trip[f_idx, t_idx, :4].astype(_np.int64) + _np.asarray(off)[f_idx][:, None]
    return _np.ascontiguousarray(q.astype(_np.int32))


def _fit_chi2_function():
    import torch

    class FitChi2(torch.autograd.Function):
        """Sum of the track chi2 of frozen candidates as a function of the 25 alignment
        and field-scale parameters.  Forward runs m3e_fit_grad without the gradient;
        backward runs it again with the gradient (the fit is recomputed, nothing per
        candidate is kept between the two)."""

        @staticmethod
        def forward(fctx, params, m3e_ctx, hits, off, cand):
            p = params.detach().to(torch.float32).contiguous()
            s, _ = m3e_ctx.fit_grad(hits, off, cand, p, grad=False)
            fctx.save_for_backward(p)
            fctx.m3e = (m3e_ctx, hits, off, cand)
            return s[0].to(params.dtype)

        @staticmethod
        def backward(fctx, g_out):
            (p,) = fctx.saved_tensors
            m3e_ctx, hits, off, cand = fctx.m3e
            _, g = m3e_ctx.fit_grad(hits, off, cand, p, grad=True)
            return (g_out * g).to(p.dtype), None, None, None, None

    return FitChi2


_FIT = None


def fit_chi2_sum(params, ctx: "Context", hits, off, cand):
    """Differentiable sum of the track chi2 (torch.autograd.Function over m3e_fit_grad)."""
    global _FIT
    if _FIT is None:
        _FIT = _fit_chi2_function()
    return _FIT.apply(params, ctx, hits, off, cand)
