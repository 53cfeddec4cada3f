#!/usr/bin/env python
"""Throughput benchmark of the Mu3e online event selection on GB300.

Workload (one step): the full-rate batch of 1,000,000 synthetic frames per GPU
(Poisson(20) tracks per frame, 2 noise hits per layer, a signal decay in 0.1 % of
the frames, seed 2 on rank 0), int32 pixel addresses resident in HBM (343 MB,
larger than L2, so no flush is needed between steps).  A step is one
m3e_select_frames call over the whole batch: every stage of the method runs in
the library's kernels.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

The reference arm (--impl reference) times the FP64 CPU oracle on the host
cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "frames/s and hits/s per GB300 vs plain per-frame form; % issue roofline; p99 latency"
WORKLOAD = ("full-rate throughput: 1,000,000 frames per GPU, Poisson(20) tracks/frame (p 15-53 MeV, "
            "|cos theta| < 0.8, double-cone target), 2 noise hits/layer, signal decay in 0.1% of frames, "
            "4 layers r=25/31/73/85 mm, B=1 T, 80 um pixels, int32 addresses")
# Arithmetic operations per work item of the method's formulas (FMA = 2, each
# transcendental, division or square root = 1), grouped by the stage kernel that
# does the work: a Phi pair test is a dot product and a compare (4); a candidate
# triplet the Delta lambda difference and compare (6); a selected triplet two
# triplet fits (~190 each), the layer-3 extrapolation and search and the global
# fit (~460); an energy test three additions and a compare (7); a combination
# passing it the longitudinal momentum bound (3); a combination whose P_z leaves
# the momentum cut open the vertex prefilter (75) and, if vertexed, the
# intersections, closest points, chi2 and cuts (565).  The work items are counted
# by the library's statistics (a timed run evaluates no other vertex).
STAGE_OPS = {  # name: (indices into m3e_stage_times, ops per counted item)
    "stage1 decode+sort+cuts (warp and CTA tiers)": ((0, 1, 2), {"pair_tests": 4, "triplet_tests": 6}),
    "stage2 track fits": ((3,), {"triplets": 460}),
    "stage3 energy test": ((4,), {"energy_tests": 7, "combos": 3}),
    "stage4 vertex": ((5,), {"pz_open": 75, "vertexed_pz_open": 565}),
    "stage5 decision": ((6,), {}),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--frames", type=int, default=1_000_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-c3", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="keep the default launch parameters (no autotuner)")
    ap.add_argument("--arms", default="main,forms,e2e,c3,c4,c5,rates",
                    help="comma list of measurements: main (staged, always), forms (fused and plain), e2e, c3, "
                         "c4 (alignment gradient), c5 (streaming latency), rates (muon-rate sweep)")
    ap.add_argument("--c5-frames", type=int, default=1_000_000)
    return ap.parse_args()


def shard_seed(rank: int) -> int:
    """Weak scaling: rank r selects its own batch (seed 2 on rank 0)."""
    return 2 + 7919 * rank


def max_over_ranks(ms: float, device, world: int) -> float:
    """The job's time is the slowest rank's: max-reduce one float over the process group."""
    if world == 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_batch(n_frames: int, rank: int):
    from paper_2206_11535_gb300 import gen
    return gen.generate(n_frames, 20.0, 2.0, 1000, seed=shard_seed(rank))


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during a timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        self.rows = []
        if self.p is None:
            return
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 8:
                self.rows.append(f)

    def summary(self):
        if not getattr(self, "rows", None):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = np.array([float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()])
        mx = max(float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[4 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm.size else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(self.rows)}


def kernel_source_hash(unit: str = "m3e_staged.cu") -> str:
    """Hash of the sources a unit's kernels compile from: the unit, the shared device
    code and the parameter structs of the internal header (not its host declarations)."""
    h = hashlib.sha256()
    src = os.path.join(ROOT, "paper_2206_11535_gb300", "csrc")
    for f in (unit, "m3e_device.cuh"):
        h.update(open(os.path.join(src, f), "rb").read())
    txt = open(os.path.join(src, "m3e_internal.cuh"), "rb").read()
    h.update(txt[txt.index(b"constexpr int NB"):txt.index(b"// Host-side launchers")])
    return h.hexdigest()[:16]


PROFILE_OF = {"ingest": ("ingest_c2_traffic.txt", "m3e_ingest.cu")}


def _recorded(key: str):
    """A counter of a committed ncu summary (the stage kernels', or the ingest kernel's
    for keys ending in .ingest), or None when the summary was taken on other kernel
    sources (or lacks the key)."""
    fname, unit = PROFILE_OF.get(key.rsplit(".", 1)[-1], ("staged_c2_traffic.txt", "m3e_staged.cu"))
    p = os.path.join(ROOT, "profiles", fname)
    if not os.path.exists(p):
        return None
    kv = {}
    for line in open(p):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("kernel_source_sha256_16") != kernel_source_hash(unit):
        return None
    try:
        return float(kv[key])
    except (KeyError, ValueError):
        return None


def recorded_traffic(n_frames: int, stage: str):
    """DRAM bytes (read + write) of one batch's launches of the given stage, from the committed
    ncu summary (bytes per frame of a smaller batch of the same workload, scaled to n_frames);
    None when the summary was taken on other kernel sources."""
    v = _recorded("dram_bytes_per_frame." + stage)
    return None if v is None else v * n_frames


def cpu_baseline(d, seconds_target=12.0):
    """The FP64 oracle as it stands, on the host cores, on a bounded prefix of the batch."""
    from oracle import oracle as O
    from paper_2206_11535_gb300 import gen
    c = O.make_config(gen.load_config())
    cores = os.cpu_count() or 1
    nf = d["off"].size - 1
    # calibrate the sample size on a small prefix, then time a prefix worth ~seconds_target
    n0 = min(2000, nf)
    t = time.perf_counter()
    O.select_frames(c, d["hits"], d["off"][:n0 + 1], cores)
    rate0 = n0 / max(time.perf_counter() - t, 1e-6)
    n = int(min(nf, max(n0, rate0 * seconds_target)))
    t = time.perf_counter()
    O.select_frames(c, d["hits"], d["off"][:n + 1], cores)
    dt = time.perf_counter() - t
    return {"value": n / dt, "unit": "frames/s", "cores": cores, "kind": "oracle",
            "sample": f"first {n} frames of the rank-0 batch, FP64 C oracle (-O2), {cores} threads over "
                      f"disjoint frame ranges, brute force over every hit triplet ({dt:.1f} s)"}


def measured_hbm_peak():
    """(GB/s, source) of the machine's measured copy bandwidth, else the stated fallback."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(p))["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s"


def ingest_roofline(ctx, hits, dev, stream, steps=20) -> dict:
    """m3e_ingest over the whole batch's hits (int32 addresses -> x, y, z, phi as FP32
    structure of arrays): 4 bytes read and 16 written per hit, against HBM."""
    import torch
    n = hits.numel()
    outs = [torch.empty(n, dtype=torch.float32, device=dev) for _ in range(4)]
    for _ in range(3):
        ctx.ingest(hits, *outs, stream=stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        ctx.ingest(hits, *outs, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    ctx.check()
    peak, src = measured_hbm_peak()
    alg = 20 * n
    tr = _recorded("dram_bytes_per_hit.ingest")
    del outs
    return {"kernel": "k_ingest (m3e_ingest)", "bound": "hbm", "achieved": alg / (ms / 1e3) / 1e9, "peak": peak,
            "unit": "GB/s", "frac": alg / (ms / 1e3) / 1e9 / peak, "peak_source": src, "kernel_ms": ms,
            "algorithmic_bytes": alg, "hits": n, "traffic": None if tr is None else tr * n}


def compaction_roofline(nf: int, stage1_ms: float) -> dict | None:
    """The stream-compaction writes of stage 1 (the sorted hits and the ballot-compacted
    triplets of every frame it emits): DRAM bytes written per frame from the committed
    ncu summary of the stage kernels, over this run's stage-1 time."""
    wb = _recorded("dram_write_bytes_per_frame.stage1")
    if wb is None or stage1_ms <= 0:
        return None
    peak, src = measured_hbm_peak()
    gbs = wb * nf / (stage1_ms / 1e3) / 1e9
    return {"kernel": "k_stage1 (emit of sorted hits and compacted triplets)", "bound": "alu (reported against hbm)",
            "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak, "peak_source": src,
            "dram_write_bytes_per_frame": wb}


def parity_sample(ctx, d, dev, n_frames=2000):
    """Part of the CPU-baseline leg: the first n_frames frames of the batch through the
    staged form with its candidate record, compared candidate by candidate with the
    oracle; frames that match, differ only inside a boundary band (counted per band),
    or fail."""
    import torch
    from oracle import oracle as O
    from paper_2206_11535_gb300 import gen
    from tests import parity
    nf = min(n_frames, d["off"].size - 1)
    hits = d["hits"][:d["off"][nf]]
    off = d["off"][:nf + 1]
    rec = ctx.select_frames_debug(torch.from_numpy(hits).to(dev), torch.from_numpy(off).to(dev),
                                  cap_trip=1024, cap_combo=1024)
    rec = {k: v.cpu().numpy() for k, v in rec.items()}
    res = parity.compare_batch(O.make_config(gen.load_config()), hits, off, rec)
    return {"frames": nf, "form": "staged", **parity.summary(res),
            "boundary_differences_per_band": parity.band_counts(res),
            "bands": dict(parity.BAND), "oracle": "FP64 C oracle, candidate by candidate"}


def run_reference(args, rank, world):
    """Reference arm: the FP64 oracle on the host cores, bounded sample per step."""
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_2206_11535_gb300 import gen
    O.build()
    c = O.make_config(gen.load_config())
    cores = os.cpu_count() or 1
    n = min(args.frames, 20000)
    d = make_batch(n, 0)
    for _ in range(args.warmup):
        O.select_frames(c, d["hits"], d["off"], cores)
    t = time.perf_counter()
    for _ in range(args.steps):
        O.select_frames(c, d["hits"], d["off"], cores)
    dt = time.perf_counter() - t
    v = n * args.steps / dt
    sample = (f"{n} frames of the rank-0 batch per step (bounded sample of the 1,000,000-frame workload), "
              f"FP64 C oracle, {cores} threads")
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": "frames/s", "n_gpus": world,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                      "data": "synthetic", "config": {"workload": WORKLOAD, "frames_per_step": n},
                      "cpu_baseline": {"value": v, "unit": "frames/s", "cores": cores, "kind": "oracle",
                                       "sample": sample},
                      "e2e": {"value": v, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
          flush=True)


ALIGN_SCALE = np.array(([0.05] * 3 + [5e-4] * 3) * 4 + [1.0])  # mm, rad, field scale: the c4 truth's widths


def _euler_zyx(R):
    """(wx, wy, wz) of R = Rz(wz) Ry(wy) Rx(wx)."""
    return np.array([np.arctan2(R[2, 1], R[2, 2]), -np.arcsin(np.clip(R[2, 0], -1, 1)), np.arctan2(R[1, 0], R[0, 0])])


def _relative_to_layer0(p, gen):
    """Each layer's displacement relative to layer 0 (the common translation and
    rotation of all layers leave every chi2 unchanged)."""
    p = np.asarray(p, float)
    R0, d0 = gen.rotation(p[3:6]), p[0:3]
    out = np.zeros((4, 6))
    for L in range(4):
        RL, dL = gen.rotation(p[6 * L + 3:6 * L + 6]), p[6 * L:6 * L + 3]
        out[L, :3] = R0.T @ (dL - d0)
        out[L, 3:] = _euler_zyx(R0.T @ RL)
    return out


def align_arm(ctx, gen, m3e, n_frames: int, dev, steps: int = 200) -> dict:
    """c4: frames from a displaced detector, the selection's kept tracks (at nominal
    geometry, frozen), the gradient kernel's throughput, and 200 Adam steps on the
    alignment of layers 1-3 (layer 0 fixed: common translation and z-rotation are
    exact null modes; the field scale fixed: the chi2 sum is quadratic in it)."""
    import torch
    d = gen.workload("c4", n_frames=n_frames)
    truth = np.r_[d["truth_align"].reshape(-1), d["truth_b_scale"]]
    hits, off = torch.from_numpy(d["hits"]).to(dev), torch.from_numpy(d["off"]).to(dev)
    rec = {k: v.cpu().numpy() for k, v in ctx.select_frames_debug(hits, off).items()}
    cand = m3e.kept_candidates(rec, d["off"])
    cq = torch.from_numpy(cand).to(dev)
    nominal = torch.tensor(np.r_[np.zeros(24), 1.0], dtype=torch.float32, device=dev)

    def time_calls(grad):
        for _ in range(3):
            ctx.fit_grad(hits, off, cq, nominal, grad=grad)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(20):
            ctx.fit_grad(hits, off, cq, nominal, grad=grad)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 20

    ms_grad, ms_fwd = time_calls(True), time_calls(False)
    scale = torch.tensor(ALIGN_SCALE, dtype=torch.float32, device=dev)
    free = torch.zeros(25, device=dev)
    free[6:24] = 1.0
    x = torch.zeros(25, device=dev, requires_grad=True)
    opt = torch.optim.Adam([x], lr=0.1)
    hist = []
    for _ in range(steps):
        opt.zero_grad()
        loss = m3e.fit_chi2_sum(x * scale * free + nominal, ctx, hits, off, cq)
        loss.backward()
        opt.step()
        hist.append(loss.item())
    est = (x * scale * free + nominal).detach().cpu().numpy().astype(np.float64)
    s_end = float(ctx.fit_grad(hits, off, cq, torch.tensor(est, dtype=torch.float32, device=dev), grad=False)[0])
    s_truth = float(ctx.fit_grad(hits, off, cq, torch.tensor(truth, dtype=torch.float32, device=dev), grad=False)[0])
    # modes: Hessian of the chi2 sum in the 18 free parameters (units of the injected
    # widths), by central differences of the gradient kernel
    fi = np.arange(6, 24)
    H = np.zeros((18, 18))
    for a, i in enumerate(fi):
        h = 0.02 * ALIGN_SCALE[i]
        gp = ctx.fit_grad(hits, off, cq, torch.tensor(est + h * (np.arange(25) == i), dtype=torch.float32,
                                                       device=dev))[1].cpu().numpy()
        gm = ctx.fit_grad(hits, off, cq, torch.tensor(est - h * (np.arange(25) == i), dtype=torch.float32,
                                                       device=dev))[1].cpu().numpy()
        H[:, a] = (gp[fi] - gm[fi]) / (2 * h) * ALIGN_SCALE[fi] * ALIGN_SCALE[i]
    ev, V = np.linalg.eigh(0.5 * (H + H.T))
    rel_truth = _relative_to_layer0(truth, gen)[1:].reshape(-1) / ALIGN_SCALE[fi]
    rel_est = _relative_to_layer0(est, gen)[1:].reshape(-1) / ALIGN_SCALE[fi]
    res_m, tru_m = V.T @ (rel_est - rel_truth), V.T @ rel_truth
    names = [f"L{1 + j // 6}{['dx', 'dy', 'dz', 'wx', 'wy', 'wz'][j % 6]}" for j in range(18)]
    modes = [{"eigenvalue": float(ev[k]), "injected": float(tru_m[k]), "residual": float(res_m[k]),
              "main_params": [names[j] for j in np.argsort(-np.abs(V[:, k]))[:3]]} for k in range(18)]
    stiff = ev >= 1e-2 * ev.max()
    trk = d["hit_track"][cand]
    return {"workload": f"c4: {n_frames:,} frames of the c1 mix from a detector with layers displaced by "
                        "N(0, 50 um) and N(0, 0.5 mrad) per axis and the field off by N(0, 1e-3), seed 4",
            "candidates": int(cand.shape[0]),
            "truth_matched_fraction": float(((trk[:, 0] >= 0) & (trk == trk[:, :1]).all(1)).mean()),
            "fit_grad_ms": ms_grad, "fit_chi2_only_ms": ms_fwd,
            "candidates_per_s_gradient": cand.shape[0] / (ms_grad / 1e3),
            "steps": steps, "optimizer": "Adam lr 0.1 in units of the injected widths; layer 0 and field scale fixed",
            "chi2_start": hist[0], "chi2_end": s_end, "chi2_at_truth": s_truth,
            "stiff_modes": int(stiff.sum()),
            "stiff_residual_over_injected": float(np.linalg.norm(res_m[stiff]) / np.linalg.norm(tru_m[stiff])),
            "weak_residual_over_injected": float(np.linalg.norm(res_m[~stiff]) / max(np.linalg.norm(tru_m[~stiff]),
                                                                                        1e-30)),
            "modes": modes,
            "field_scale": field_scale_fit(ctx, d, cand, hits, off, est, truth, dev)}


def _signal_decays(d, cand):
    """Rows of `cand` (kept quadruplets) for the signal decays whose three tracks were all
    kept, each track by one truth-matched candidate: an (n, 3) index array."""
    trk = d["hit_track"][cand]
    tm = (trk[:, 0] >= 0) & (trk == trk[:, :1]).all(1)
    first = {}
    for k in np.nonzero(tm)[0]:
        first.setdefault(int(trk[k, 0]), k)
    groups = {}
    for t in np.nonzero(d["trk_signal"])[0]:
        groups.setdefault(int(d["trk_frame"][t]), []).append(int(t))
    return np.array([[first[t] for t in g] for g in groups.values() if len(g) == 3 and all(t in first for t in g)],
                    np.int64).reshape(-1, 3)


def _energy_scale(ctx, hits, off, cand, decays, params, dev):
    """The field scale s minimising sum_decays (sum_i sqrt((k B s / |kappa_i|)^2 + m_e^2)
    - m_mu)^2 (Newton steps in FP64), with the curvatures from m3e_fit_kappa at `params`;
    returns (s, decays used, its statistical error, rms of the energy sums at s)."""
    import torch
    from paper_2206_11535_gb300 import gen as G
    cfg = G.load_config()
    kB = cfg["constants"]["k_MeV_per_T_mm"] * cfg["field"]["B_T"]
    me, mmu = cfg["constants"]["m_e_MeV"], cfg["constants"]["m_mu_MeV"]
    sub = torch.from_numpy(np.ascontiguousarray(cand[decays.reshape(-1)])).to(dev)
    k = ctx.fit_kappa(hits, off, sub, torch.tensor(params, dtype=torch.float32, device=dev)).cpu().numpy()
    p1 = (kB / np.abs(k.astype(np.float64))).reshape(-1, 3)
    p1 = p1[np.isfinite(p1).all(1)]
    s = 1.0
    for _ in range(20):
        E = np.sqrt((s * p1) ** 2 + me ** 2)
        r = E.sum(1) - mmu
        dr = (s * p1 ** 2 / E).sum(1)
        s -= (r * dr).sum() / (dr * dr).sum()
    E = np.sqrt((s * p1) ** 2 + me ** 2)
    r = E.sum(1) - mmu
    dr = (s * p1 ** 2 / E).sum(1)
    err = float(np.sqrt((r ** 2).mean() / (dr * dr).sum()))
    return float(s), int(p1.shape[0]), err, float(np.sqrt((r ** 2).mean()))


def field_scale_fit(ctx, d, cand, hits, off, est, truth, dev) -> dict:
    """The field scale, which the chi2 sum cannot fix (it grows as the square of the
    scale), from the energy sum of the signal decays (Sec. "Vertex Fit": the three
    tracks of mu+ -> e+ e- e+ at rest carry E = m_mu): the decays whose three tracks
    the selection kept, their curvatures from m3e_fit_kappa at the fitted alignment,
    and the scale that brings their energy sums to m_mu.  The momentum from a fitted
    curvature, k B s / |kappa|, is biased upward by the curvature's spread, so the raw
    scale is divided by the raw scale of a calibration sample of the same generator at
    the nominal field and geometry (seed 1004): the usual simulation-calibrated energy
    scale."""
    import torch
    from paper_2206_11535_gb300 import gen as G
    decays = _signal_decays(d, cand)
    if decays.shape[0] == 0:
        return {"signal_decays": 0}
    s_fit, n, err, rms = _energy_scale(ctx, hits, off, cand, decays, est, dev)
    s_true_align = _energy_scale(ctx, hits, off, cand, decays, truth, dev)[0]
    # calibration sample: nominal detector and field, the same frame mix
    dc = G.generate(d["off"].size - 1, 10.0, 0.5, 10, seed=1004)
    hc, oc = torch.from_numpy(dc["hits"]).to(dev), torch.from_numpy(dc["off"]).to(dev)
    rec = {k: v.cpu().numpy() for k, v in ctx.select_frames_debug(hc, oc).items()}
    from paper_2206_11535_gb300 import m3e as M
    cc = M.kept_candidates(rec, dc["off"])
    s_cal, n_cal, err_cal, _ = _energy_scale(ctx, hc, oc, cc, _signal_decays(dc, cc), np.r_[np.zeros(24), 1.0], dev)
    rec_scale = s_fit / s_cal
    return {"signal_decays": n, "injected": float(truth[24]), "recovered": rec_scale,
            "residual": rec_scale - float(truth[24]),
            "statistical_error": float(np.hypot(err / s_cal, err_cal * s_fit / s_cal ** 2)),
            "recovered_at_true_alignment": s_true_align / s_cal, "raw_scale": s_fit,
            "calibration_raw_scale": s_cal, "calibration_decays": n_cal, "energy_sum_rms_MeV": rms,
            "method": "energy sum of the signal decays whose three tracks were kept (curvatures from m3e_fit_kappa "
                      "at the fitted alignment), least squares in the scale, divided by the same on a nominal "
                      "calibration sample (seed 1004)"}


MU_RATES = (1e8, 2e8, 5e8, 1e9)


def rate_arm(ctx, gen, m3e, n_frames: int, dev, steps: int = 5) -> dict:
    """Muon-rate sweep: 64 ns frames hold Poisson(6.4 x rate / 1e8) decay tracks
    (6.4 at the paper's 1e8 muons/s), 0.5 noise hits per layer, a signal decay in
    every 1000th frame.  Staged-form frames/s and the kept fraction by reason."""
    import torch
    out = []
    for k, rate in enumerate(MU_RATES):
        d = gen.generate(n_frames, 6.4 * rate / 1e8, 0.5, 1000, seed=60 + k)
        hits, off = torch.from_numpy(d["hits"]).to(dev), torch.from_numpy(d["off"]).to(dev)
        nf = n_frames
        keep = torch.empty(nf, dtype=torch.uint8, device=dev)
        reason = torch.empty(nf, dtype=torch.uint8, device=dev)
        for _ in range(2):
            ctx.select_frames(hits, off, keep, reason)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            ctx.select_frames(hits, off, keep, reason)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        r = reason.cpu().numpy()
        out.append({"muons_per_s": rate, "mean_tracks_per_frame": 6.4 * rate / 1e8,
                    "hits_per_frame": float(d["off"][-1]) / nf, "frames_per_s": nf / (ms / 1e3),
                    "ms_per_batch": ms, "kept_fraction": float((r != 0).mean()),
                    "kept_by_reason": {m3e.REASONS[i]: float((r == i).mean()) for i in range(1, 7)}})
        del hits, off, keep, reason
    return {"workload": f"{n_frames:,} frames per rate, tracks Poisson(6.4 x rate / 1e8), 0.5 noise/layer, "
                        "signal every 1000th frame, seeds 60-63", "rates": out}


C5_RATES = (15.625e6 / 12, 15.625e6 / 4, 15.625e6)


def stream_arm(ctx, gen, n_frames: int, dev) -> dict:
    """Latency of the streaming path on the c5 frame mix at three arrival rates."""
    import torch
    d = gen.workload("c5", n_frames=n_frames)
    keep, reason = ctx.select_frames_fused(torch.from_numpy(d["hits"]).to(dev), torch.from_numpy(d["off"]).to(dev))
    ref = reason.cpu().numpy()
    ctx.stream_open()
    ctx.stream_replay(d["hits"], d["off"][:20001], rate_hz=1e6, seed=99)  # warm-up
    rates = []
    for k, rate in enumerate(C5_RATES):
        r = ctx.stream_replay(d["hits"], d["off"], rate_hz=rate, seed=5 + k)
        q = lambda a, p: float(np.percentile(a, p)) / 1e3  # noqa: E731  (microseconds)
        rates.append({"offered_frames_per_s": rate, "sustained_frames_per_s": r["sustained_hz"],
                      "submitted_frames_per_s": r["submit_hz"], "busy_retries": int(r["busy_retries"]),
                      "kernel_launches": int(r["kernel_launches"]),
                      "latency_submit_us": {"p50": q(r["lat_submit_ns"], 50), "p99": q(r["lat_submit_ns"], 99),
                                            "p99.9": q(r["lat_submit_ns"], 99.9)},
                      "latency_arrival_us": {"p50": q(r["lat_arrival_ns"], 50), "p99": q(r["lat_arrival_ns"], 99),
                                             "p99.9": q(r["lat_arrival_ns"], 99.9)},
                      "kept_fraction": float(r["keep"].mean()),
                      "identical_to_batch": bool((r["reason"] == ref).all())})
    st = ctx.stream_poll()
    ctx.stream_close()
    return {"workload": f"c5: {n_frames:,} frames of the c1 mix (Poisson(10) tracks, 0.5 noise/layer, "
                        "signal every 10th frame), seed 5; Poisson arrivals, one submitting host thread",
            "latency": "submit: m3e_stream_submit to result delivered into the caller's slot; arrival: "
                       "scheduled arrival to result (includes waiting for admission)",
            "rates": rates, "heavy_frames": int(st["heavy_frames"])}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    import __graft_entry__
    __graft_entry__.build()
    from paper_2206_11535_gb300 import gen, m3e
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    cfg = gen.load_config()
    d = make_batch(args.frames, rank)
    nf = d["off"].size - 1
    nh = int(d["off"][-1])
    dev = torch.device("cuda", local)
    hits = torch.from_numpy(d["hits"]).to(dev)
    off = torch.from_numpy(d["off"]).to(dev)
    keep = torch.empty(nf, dtype=torch.uint8, device=dev)
    reason = torch.empty(nf, dtype=torch.uint8, device=dev)
    ctx = m3e.Context(cfg, local)
    stream = torch.cuda.current_stream(dev)

    # launch parameters from the library's autotuner on a calibration slice (the first 250,000 frames)
    arms = set(args.arms.split(","))
    ncal = min(nf, 250000)
    tuning = None if args.no_tune else ctx.autotune(hits, off[:ncal + 1])
    # work counts of this batch (untimed) for the algorithmic operation count
    st = m3e.new_stats(dev)
    ctx.select_frames(hits, off, keep, reason, stats=st)
    torch.cuda.synchronize()
    stats = m3e.stats_dict(st)
    ctx.check()

    def timed(fn, steps, warm, profile=False):
        for _ in range(warm):
            fn()
        barrier()
        ks = []
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
            if profile:
                ks.append(ctx.stage_times())
        e1.record(stream)
        barrier()
        return max_over_ranks(e0.elapsed_time(e1), dev, world), ks

    # main arm: the staged form, back to back, SM clocks sampled during the timed region
    with Clocks(local) as clk:
        ms, _ = timed(lambda: ctx.select_frames(hits, off, keep, reason, stream=stream), args.steps, args.warmup)
    launches = ctx.last_launch_count() * args.steps
    # kernel durations, from CUDA events recorded by the library on the launching stream
    ctx.set_profiling(True)
    _, ks = timed(lambda: ctx.select_frames(hits, off, keep, reason, stream=stream), max(3, args.steps // 4), 1,
                  profile=True)
    ctx.set_profiling(False)
    # the fused (one persistent kernel, warp per frame) and plain (CTA per frame) forms
    alt_steps = max(2, args.steps // 2)
    forms = None
    if "forms" in arms:
        ms_fused, _ = timed(lambda: ctx.select_frames_fused(hits, off, keep, reason, stream=stream), alt_steps, 1)
        ms_plain, _ = timed(lambda: ctx.select_frames_plain(hits, off, keep, reason, stream=stream), alt_steps, 1)
        forms = {"fused_form": {"value": world * nf * alt_steps / (ms_fused / 1e3), "unit": "frames/s",
                                "ms_per_step": ms_fused / alt_steps},
                 "plain_per_frame": {"value": world * nf * alt_steps / (ms_plain / 1e3), "unit": "frames/s",
                                     "ms_per_step": ms_plain / alt_steps,
                                     "speedup_of_staged": (ms_plain / alt_steps) / (ms / args.steps)}}
    # end to end from pinned host memory through the C ABI host entry point
    e2e = None
    if not args.no_e2e and "e2e" in arms:
        hh = torch.from_numpy(d["hits"]).pin_memory()
        ho = torch.from_numpy(d["off"]).pin_memory()
        hk = torch.empty(nf, dtype=torch.uint8).pin_memory()
        hr = torch.empty(nf, dtype=torch.uint8).pin_memory()
        ms_e2e, _ = timed(lambda: ctx.select_frames_host(hh, ho, hk, hr, stream=stream), args.steps, args.warmup)
        e2e = {"value": world * nf * args.steps / (ms_e2e / 1e3), "unit": "frames/s",
               "h2d_bytes_per_step": int(hh.numel() * 4 + ho.numel() * 8), "d2h_bytes_per_step": int(2 * nf),
               "ms_per_step": ms_e2e / args.steps}
    # uneven frames (lognormal track counts, 1 % of frames at 100x noise): staged vs plain
    c3 = None
    if not args.no_c3 and "c3" in arms:
        dc = gen.workload("c3", seed=3 + 7919 * rank)
        h3 = torch.from_numpy(dc["hits"]).to(dev)
        o3 = torch.from_numpy(dc["off"]).to(dev)
        n3 = dc["off"].size - 1
        k3 = torch.empty(n3, dtype=torch.uint8, device=dev)
        r3 = torch.empty(n3, dtype=torch.uint8, device=dev)
        # the persistent batched form: autotuned on a calibration slice, the batch captured as one graph
        tune3 = None if args.no_tune else ctx.autotune(h3, o3[:min(n3, 50000) + 1])
        ctx.set_profiling(True)
        _, k3s = timed(lambda: ctx.select_frames(h3, o3, k3, r3, stream=stream), 3, 1, profile=True)
        ctx.set_profiling(False)
        ctx.prepare(n3)
        graph3 = ctx.graph(h3, o3, k3, r3)
        ms3, _ = timed(lambda: graph3.launch(stream), args.steps, args.warmup)
        rs = r3.clone()
        ms3p, _ = timed(lambda: ctx.select_frames_plain(h3, o3, k3, r3, stream=stream), alt_steps, 1)
        c3 = {"workload": "200,000 frames, tracks min(400, lognormal(median 15, sigma 1)), 0.5 noise/layer, "
                          "1% of frames at 100x noise, seed 3",
              "staged_frames_per_s": world * n3 * args.steps / (ms3 / 1e3),
              "plain_frames_per_s": world * n3 * alt_steps / (ms3p / 1e3),
              "speedup_of_staged": (ms3p / alt_steps) / (ms3 / args.steps),
              "identical_decisions": bool(torch.equal(rs, r3)),
              "stage_ms": [round(float(x), 3) for x in np.mean(np.array(k3s), axis=0)],
              "form": "staged, captured as one CUDA graph, launch parameters from the autotuner",
              "tuning": tune3,
              "frames_over_160_hits": int((np.diff(dc["off"]) > 160).sum())}
        graph3.close()
        del h3, o3
        if tuning is not None:
            ctx.autotune(hits, off[:ncal + 1])  # back to the main batch's parameters
    # the main arm's decisions are those of the last timed staged call
    ctx.select_frames(hits, off, keep, reason, stream=stream)
    ctx.check()

    value = world * nf * args.steps / (ms / 1e3)
    st_ms = np.mean(np.array(ks), axis=0) if ks else np.full(8, np.nan)
    props = torch.cuda.get_device_properties(dev)
    cl = clk.summary()
    f_mhz = cl["sm_mhz"] or 1455.0
    peak = props.multi_processor_count * 128 * 2 * f_mhz * 1e6 / 1e12
    stages = []
    for name, (idx, per) in STAGE_OPS.items():
        ops = sum(stats[k] * v for k, v in per.items())
        t = float(sum(st_ms[i] for i in idx))
        stages.append({"kernel": name, "ms": t, "ops": ops, "tflops": ops / (t / 1e3) / 1e12 if t > 0 else 0.0,
                       "frac_of_peak": ops / (t / 1e3) / 1e12 / peak if t > 0 else 0.0})
    stages.append({"kernel": "deferred frames (CTA per frame)", "ms": float(st_ms[7])})
    stages[0]["ms_tiers"] = [float(st_ms[0]), float(st_ms[1]), float(st_ms[2])]
    dom = max(stages[:5], key=lambda x: x["ms"])
    tr = recorded_traffic(nf, dom["kernel"].split()[0])
    roof = {"bound": "alu", "kernel": dom["kernel"], "achieved": dom["tflops"], "peak": peak, "unit": "TFLOP/s",
            "frac": dom["frac_of_peak"], "traffic": tr, "kernel_ms": dom["ms"],
            "peak_source": f"FP32 lanes x 2 x SM clock: {props.multi_processor_count} SMs x 128 x 2 x "
                           f"{f_mhz:.0f} MHz (median sampled under load)",
            "stages": stages,
            "algorithmic_hbm_bytes": nh * 4 + (nf + 1) * 8 + 2 * nf}
    # the same kernel's use of its issue slots: warp instructions per frame from the ncu
    # capture, over this run's kernel time, against 4 schedulers x SMs x clock
    roof["ingest"] = ingest_roofline(ctx, hits, dev, stream)
    roof["compaction"] = compaction_roofline(nf, float(sum(st_ms[i] for i in (0, 1, 2))))
    wi = _recorded("warp_inst_per_frame." + dom["kernel"].split()[0])
    ia = _recorded("issue_active_pct." + dom["kernel"].split()[0])
    if wi is not None and dom["ms"] > 0:
        ipk = 4 * props.multi_processor_count * f_mhz * 1e6
        ach = wi * nf / (dom["ms"] / 1e3)
        roof["issue"] = {"achieved": ach, "peak": ipk, "unit": "warp instructions/s", "frac": ach / ipk,
                         "warp_instructions_per_frame": wi, "ncu_issue_active_pct": ia}
    # muon-rate sweep
    rates = None
    if "rates" in arms and world == 1:
        rates = rate_arm(ctx, gen, m3e, 200_000, dev)
    # alignment gradient (c4)
    c4 = None
    if "c4" in arms and world == 1:
        c4 = align_arm(ctx, gen, m3e, 100_000, dev)
    # streaming (c5): open-loop Poisson arrivals at the frame rates of 1e8 muons/s
    # (64 ns frames) divided by 12, 4 and 1, frame by frame through m3e_stream_submit
    c5 = None
    if "c5" in arms and world == 1:
        c5 = stream_arm(ctx, gen, args.c5_frames, dev)
    out = {"metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": WORKLOAD, "frames_per_gpu": nf, "hits_per_gpu": nh,
                      "l2": "inputs larger than L2 (no flush)",
                      "form": "staged: 5 persistent kernels regrouping the batch by candidate",
                      "parallelism": f"{world} independent GPU shard(s), no collective on the data path"},
           "hits_per_s": world * nh * args.steps / (ms / 1e3),
           **(forms or {}),
           "work_per_frame": {k: stats[k] / nf for k in m3e.STATS_FIELDS if k not in ("frames",)},
           "kept_fraction": float(keep.float().mean().item()),
           "reasons": dict(zip(m3e.REASONS, stats["reasons"][:7])),
           "tuning": tuning,
           "uneven_frames_c3": c3,
           "rate_sweep": rates,
           "alignment_c4": c4,
           "streaming_c5": c5,
           "roofline": roof, "e2e": e2e, "clocks": cl, "gpu_launches": launches}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(d)
        out["parity"] = parity_sample(ctx, d, dev)
    if rank == 0:
        print(json.dumps(out), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
