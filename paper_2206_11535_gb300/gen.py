"""Seeded synthetic Mu3e frames: a stand-in for the Geant4 Monte Carlo of the paper.

The paper evaluates on Geant4 simulation of the full detector (Sec. "Online Event
Selection" and Sec. "Benchmarks"); that data is not available, so this module draws
frames with the same structure: background electron/positron tracks from the
hollow double-cone target, the three-track signal decay mu+ -> e+ e- e+ at rest,
Highland multiple scattering at each of the four central pixel layers, pixel
digitisation and uniform noise hits.  Output is a CSR batch of packed int32 pixel
addresses (``hits[off[f]:off[f+1]]`` is frame ``f``) plus truth arrays that are
never passed to the selection.

This module is the input generator shared by the CUDA path's tests and by the
oracle's tests; it contains none of the selection arithmetic (cuts, fits,
vertexing).  Pixel address layout (32-bit, little end = row):
``[31:28]`` zero, ``[27:26]`` layer, ``[25:21]`` ladder, ``[20:13]`` column,
``[12:0]`` row.  Global column ``g = ladder*n_cols + col`` counts around the
cylinder from phi = 0.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

TWO_PI = 2.0 * math.pi
CHUNK_FRAMES = 65536  # frames per independently seeded chunk (fixed: keeps output seed-stable)


def config_path() -> str:
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "configs", "default.json")


def load_config(path: str | None = None) -> dict:
    with open(path or config_path()) as f:
        return json.load(f)


def encode(layer, ladder, col, row) -> np.ndarray:
    layer = np.asarray(layer, np.int64)
    return ((layer << 26) | (np.asarray(ladder, np.int64) << 21)
            | (np.asarray(col, np.int64) << 13) | np.asarray(row, np.int64)).astype(np.int32)


def highland(p_mev, x_over_x0):
    """Highland width of the projected scattering angle (beta = 1), radians."""
    return (13.6 / p_mev) * math.sqrt(x_over_x0) * (1.0 + 0.038 * math.log(x_over_x0))


class Geometry:
    def __init__(self, cfg: dict):
        g = cfg["geometry"]
        self.r = np.array(g["r_mm"], float)
        self.H = np.array(g["half_len_mm"], float)
        self.nlad = np.array(g["n_ladders"], np.int64)
        self.ncol = np.array(g["n_cols"], np.int64)
        self.nrow = np.array(g["n_rows"], np.int64)
        self.pitch = float(g["pitch_mm"])
        self.ntot = self.nlad * self.ncol
        self.B = float(cfg["field"]["B_T"])
        self.x0 = np.array(cfg["material"]["x_over_X0"], float)
        self.k = float(cfg["constants"]["k_MeV_per_T_mm"])
        self.m_mu = float(cfg["constants"]["m_mu_MeV"])
        self.m_e = float(cfg["constants"]["m_e_MeV"])
        self.target_r = float(cfg["target"]["r_mm"])
        self.target_half = float(cfg["target"]["half_len_mm"])


# --------------------------------------------------------------------------- tracks

def _target_points(rng, n, geo: Geometry):
    """Uniform-by-area points on the hollow double cone (radius 19 mm at z = 0,
    apex at |z| = 50 mm): |z| has density proportional to 1 - |z|/50."""
    u = rng.random(n)
    az = geo.target_half * (1.0 - np.sqrt(1.0 - u))
    z = np.where(rng.random(n) < 0.5, -az, az)
    rho = geo.target_r * (1.0 - az / geo.target_half)
    ph = rng.random(n) * TWO_PI
    return rho * np.cos(ph), rho * np.sin(ph), z


def rotation(w) -> np.ndarray:
    """R = Rz(wz) Ry(wy) Rx(wx): the rotation of a displaced layer (detector model)."""
    cx, sx, cy, sy, cz, sz = (math.cos(w[0]), math.sin(w[0]), math.cos(w[1]), math.sin(w[1]),
                              math.cos(w[2]), math.sin(w[2]))
    Rx = np.array([[1, 0, 0], [0, cx, -sx], [0, sx, cx]])
    Ry = np.array([[cy, 0, sy], [0, 1, 0], [-sy, 0, cy]])
    Rz = np.array([[cz, -sz, 0], [sz, cz, 0], [0, 0, 1]])
    return Rz @ Ry @ Rx


def _propagate(geo: Geometry, x, y, z, p, theta, psi, q, rng, ms: bool, align=None):
    """Exact helix propagation (B along +z, positive charge turns clockwise) through
    the four cylinders in layer order, outward crossings only.  A track stops at the
    first layer it misses (curls back before reaching it, or leaves |z| <= H).
    With ``align`` (4 x 6: dx, dy, dz, wx, wy, wz per layer) layer L is the nominal
    cylinder moved to R(w) x + d: the crossing is found by Newton steps from the
    nominal one and the hit is reported in the layer's own (nominal) frame.
    Returns a list over layers of (ok, x, y, z, xl, yl, zl) arrays: the global and
    the layer-frame crossing points."""
    n = p.shape[0]
    alive = np.ones(n, bool)
    x = x.copy(); y = y.copy(); z = z.copy(); theta = theta.copy(); psi = psi.copy()
    out = []
    for L in range(4):
        st, ct = np.sin(theta), np.cos(theta)
        Rt = p * st / (geo.k * geo.B)
        cx = x + q * Rt * np.sin(psi)
        cy = y - q * Rt * np.cos(psi)
        D = np.hypot(cx, cy)
        rL = geo.r[L]
        reach = alive & (D + Rt >= rL) & (D > 0.0)
        Ds = np.where(D > 0.0, D, 1.0)
        a = (rL * rL - Rt * Rt + Ds * Ds) / (2.0 * Ds)
        h = np.sqrt(np.maximum(rL * rL - a * a, 0.0))
        ux, uy = cx / Ds, cy / Ds
        p1x, p1y = a * ux - h * uy, a * uy + h * ux
        p2x, p2y = a * ux + h * uy, a * uy - h * ux
        a0 = np.arctan2(y - cy, x - cx)
        al1 = np.mod(q * (a0 - np.arctan2(p1y - cy, p1x - cx)), TWO_PI)
        al2 = np.mod(q * (a0 - np.arctan2(p2y - cy, p2x - cx)), TWO_PI)
        first1 = al1 <= al2
        alpha = np.where(first1, al1, al2)
        nx = np.where(first1, p1x, p2x)
        ny = np.where(first1, p1y, p2y)
        nz = z + Rt * alpha * ct / np.where(st != 0.0, st, 1.0)
        cot = ct / np.where(st != 0.0, st, 1.0)
        lx, ly, lz = nx, ny, nz
        if align is not None:
            Rm, dv = rotation(align[L][3:]), np.asarray(align[L][:3], float)
            ang0 = np.arctan2(y - cy, x - cx)
            for _ in range(4):  # Newton on |(R^T (h(alpha) - d))_xy|^2 = r^2
                ang = ang0 - q * alpha
                h = np.stack([cx + Rt * np.cos(ang), cy + Rt * np.sin(ang), z + Rt * alpha * cot], 1) - dv
                dh = np.stack([Rt * q * np.sin(ang), -Rt * q * np.cos(ang), Rt * cot], 1)
                loc, dloc = h @ Rm, dh @ Rm  # rows: R^T h
                f = loc[:, 0] ** 2 + loc[:, 1] ** 2 - rL * rL
                df = 2.0 * (loc[:, 0] * dloc[:, 0] + loc[:, 1] * dloc[:, 1])
                alpha = alpha - np.where(reach & (df != 0.0), f / np.where(df != 0.0, df, 1.0), 0.0)
            ang = ang0 - q * alpha
            nx, ny, nz = cx + Rt * np.cos(ang), cy + Rt * np.sin(ang), z + Rt * alpha * cot
            loc = (np.stack([nx, ny, nz], 1) - dv) @ Rm
            lx, ly, lz = loc[:, 0], loc[:, 1], loc[:, 2]
        ok = reach & (np.abs(lz) <= geo.H[L])
        if align is not None:
            ok &= alpha > 0.0  # Newton stays on the forward branch
        psi_n = psi - q * alpha
        if ms:
            sig = highland(1.0, geo.x0[L]) / p
            t1 = rng.normal(0.0, 1.0, n) * sig
            t2 = rng.normal(0.0, 1.0, n) * sig
            cps, sps = np.cos(psi_n), np.sin(psi_n)
            dx = st * cps - t1 * sps - t2 * ct * cps
            dy = st * sps + t1 * cps - t2 * ct * sps
            dz = ct + t2 * st
            nrm = np.sqrt(dx * dx + dy * dy + dz * dz)
            theta = np.where(ok, np.arccos(np.clip(dz / nrm, -1.0, 1.0)), theta)
            psi_n = np.arctan2(dy, dx)
        x, y, z, psi = nx, ny, nz, psi_n
        alive = ok
        out.append((ok, nx, ny, nz, lx, ly, lz))
    return out


def _decay_momenta(rng, n, geo: Geometry):
    """Uniform three-body phase space of mu+ -> e+ e- e+ at rest (Dalitz-plot
    rejection with massive electrons), isotropically oriented.  Returns
    momenta (n, 3, 3) for particles (e+, e-, e+)."""
    M, m = geo.m_mu, geo.m_e
    lo, hi = (2 * m) ** 2, (M - m) ** 2
    m12 = np.empty(0); m23 = np.empty(0)
    while m12.size < n:
        k = 2 * (n - m12.size) + 64
        a = lo + (hi - lo) * rng.random(k)
        b = lo + (hi - lo) * rng.random(k)
        ma = np.sqrt(a)
        e2s = (a - m * m + m * m) / (2 * ma)
        e3s = (M * M - a - m * m) / (2 * ma)
        pa = np.sqrt(np.maximum(e2s ** 2 - m * m, 0.0))
        pb = np.sqrt(np.maximum(e3s ** 2 - m * m, 0.0))
        bmin = (e2s + e3s) ** 2 - (pa + pb) ** 2
        bmax = (e2s + e3s) ** 2 - (pa - pb) ** 2
        acc = (b >= bmin) & (b <= bmax)
        m12 = np.concatenate([m12, a[acc]]); m23 = np.concatenate([m23, b[acc]])
    m12, m23 = m12[:n], m23[:n]
    E3 = (M * M + m * m - m12) / (2 * M)
    E1 = (M * M + m * m - m23) / (2 * M)
    E2 = M - E1 - E3
    P1 = np.sqrt(np.maximum(E1 ** 2 - m * m, 0.0))
    P2 = np.sqrt(np.maximum(E2 ** 2 - m * m, 0.0))
    P3 = np.sqrt(np.maximum(E3 ** 2 - m * m, 0.0))
    c13 = np.clip((P2 ** 2 - P1 ** 2 - P3 ** 2) / np.maximum(2 * P1 * P3, 1e-300), -1.0, 1.0)
    s13 = np.sqrt(1.0 - c13 ** 2)
    v1 = np.stack([np.zeros(n), np.zeros(n), P1], 1)
    v3 = np.stack([P3 * s13, np.zeros(n), P3 * c13], 1)
    v2 = -(v1 + v3)
    # uniform random rotation from a uniform unit quaternion
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    qw = np.sqrt(1 - u1) * np.sin(TWO_PI * u2)
    qx = np.sqrt(1 - u1) * np.cos(TWO_PI * u2)
    qy = np.sqrt(u1) * np.sin(TWO_PI * u3)
    qz = np.sqrt(u1) * np.cos(TWO_PI * u3)
    Rm = np.empty((n, 3, 3))
    Rm[:, 0, 0] = 1 - 2 * (qy * qy + qz * qz); Rm[:, 0, 1] = 2 * (qx * qy - qz * qw); Rm[:, 0, 2] = 2 * (qx * qz + qy * qw)
    Rm[:, 1, 0] = 2 * (qx * qy + qz * qw); Rm[:, 1, 1] = 1 - 2 * (qx * qx + qz * qz); Rm[:, 1, 2] = 2 * (qy * qz - qx * qw)
    Rm[:, 2, 0] = 2 * (qx * qz - qy * qw); Rm[:, 2, 1] = 2 * (qy * qz + qx * qw); Rm[:, 2, 2] = 1 - 2 * (qx * qx + qy * qy)
    out = np.stack([v1, v2, v3], 1)  # (n, 3 particles, 3)
    return np.einsum("nij,npj->npi", Rm, out)


def _digitise(geo: Geometry, L: int, x, y, z):
    phi = np.mod(np.arctan2(y, x), TWO_PI)
    g = np.clip(np.floor(phi / TWO_PI * geo.ntot[L]).astype(np.int64), 0, geo.ntot[L] - 1)
    row = np.clip(np.floor((z + geo.H[L]) / geo.pitch).astype(np.int64), 0, geo.nrow[L] - 1)
    return encode(np.full(g.shape, L), g // geo.ncol[L], g % geo.ncol[L], row)


# --------------------------------------------------------------------------- frames

def _gen_chunk(geo, rng, f0, nf, n_tracks, signal_mask, noise_mean, ms, digitise, noise, p_range,
               cos_range, align=None):
    # background tracks
    nt = int(n_tracks.sum())
    tf = np.repeat(np.arange(f0, f0 + nf), n_tracks)
    vx, vy, vz = _target_points(rng, nt, geo)
    p = p_range[0] + (p_range[1] - p_range[0]) * rng.random(nt)
    cth = cos_range[0] + (cos_range[1] - cos_range[0]) * rng.random(nt)
    theta = np.arccos(cth)
    psi = rng.random(nt) * TWO_PI
    q = np.where(rng.random(nt) < 0.5, 1.0, -1.0)
    sig = np.zeros(nt, bool)
    # signal decays: 3 tracks from one vertex
    sf = np.nonzero(signal_mask)[0] + f0
    ns = sf.size
    if ns:
        mom = _decay_momenta(rng, ns, geo).reshape(-1, 3)
        sx, sy, sz = _target_points(rng, ns, geo)
        pm = np.linalg.norm(mom, axis=1)
        tf = np.concatenate([tf, np.repeat(sf, 3)])
        vx = np.concatenate([vx, np.repeat(sx, 3)])
        vy = np.concatenate([vy, np.repeat(sy, 3)])
        vz = np.concatenate([vz, np.repeat(sz, 3)])
        p = np.concatenate([p, pm])
        theta = np.concatenate([theta, np.arccos(np.clip(mom[:, 2] / np.maximum(pm, 1e-300), -1, 1))])
        psi = np.concatenate([psi, np.arctan2(mom[:, 1], mom[:, 0])])
        q = np.concatenate([q, np.tile([1.0, -1.0, 1.0], ns)])
        sig = np.concatenate([sig, np.ones(3 * ns, bool)])
    ntr = tf.size
    layers = _propagate(geo, vx, vy, vz, np.maximum(p, 1e-6), theta, psi, q, rng, ms, align)
    h_frame, h_addr, h_trk, h_pos, h_layer = [], [], [], [], []
    nh = np.zeros(ntr, np.int32)
    for L, (ok, x, y, z, xl, yl, zl) in enumerate(layers):
        idx = np.nonzero(ok)[0]
        nh[idx] += 1
        h_frame.append(tf[idx]); h_trk.append(idx); h_layer.append(np.full(idx.size, L, np.int8))
        h_addr.append(_digitise(geo, L, xl[idx], yl[idx], zl[idx]))
        h_pos.append(np.stack([x[idx], y[idx], z[idx]], 1))
    if noise:
        for L in range(4):
            cnt = rng.poisson(noise_mean, nf) if np.ndim(noise_mean) == 0 else rng.poisson(noise_mean)
            m = int(cnt.sum())
            g = rng.integers(0, geo.ntot[L], m)
            row = rng.integers(0, geo.nrow[L], m)
            h_frame.append(np.repeat(np.arange(f0, f0 + nf), cnt))
            h_trk.append(np.full(m, -1, np.int64))
            h_layer.append(np.full(m, L, np.int8))
            h_addr.append(encode(np.full(m, L), g // geo.ncol[L], g % geo.ncol[L], row))
            phi = (g + 0.5) * TWO_PI / geo.ntot[L]
            h_pos.append(np.stack([geo.r[L] * np.cos(phi), geo.r[L] * np.sin(phi),
                                   -geo.H[L] + (row + 0.5) * geo.pitch], 1))
    fr = np.concatenate(h_frame); ad = np.concatenate(h_addr); tr = np.concatenate(h_trk)
    ly = np.concatenate(h_layer); pos = np.concatenate(h_pos)
    order = np.lexsort((rng.random(fr.size), fr))  # shuffle hits within each frame
    tracks = dict(frame=tf, p=p, theta=theta, psi=psi, q=q.astype(np.int8), vx=vx, vy=vy, vz=vz,
                  signal=sig, n_hits=nh)
    return fr[order], ad[order], tr[order], ly[order], pos[order], tracks


def _chunk_job(job):
    """One independently seeded chunk of frames (a process-pool task)."""
    cfg, seed, c0, nf, counts, fsig, lam, ms, digitise, noise, p_range, cos_range, align, b_scale = job
    rng = np.random.default_rng([seed, 1 + c0 // CHUNK_FRAMES])
    geo = Geometry(cfg)
    geo.B *= b_scale
    return _gen_chunk(geo, rng, c0, nf, counts, fsig, lam, ms, digitise, noise, p_range, cos_range, align)


def generate(n_frames: int, mean_tracks=10.0, noise_per_layer=0.5, signal_every: int | None = 10,
             seed: int = 1, ms: bool = True, digitise: bool = True, noise: bool = True,
             track_counts: np.ndarray | None = None, noise_scale: np.ndarray | None = None,
             p_range=(15.0, 53.0), cos_range=(-0.8, 0.8), cfg: dict | None = None,
             workers: int | None = None, align=None, b_scale: float = 1.0) -> dict:
    """Draw ``n_frames`` frames.

    mean_tracks      Poisson mean of background tracks per frame (ignored if track_counts given)
    noise_per_layer  Poisson mean of uniform noise hits per layer per frame
    signal_every     frame f carries a signal decay when f % signal_every == 0 (None: never)
    ms / digitise / noise  switch multiple scattering, pixel digitisation, noise off
    track_counts     explicit background tracks per frame (lognormal mixes and the like)
    noise_scale      per-frame multiplier of noise_per_layer
    workers          processes for chunks of 65,536 frames (spawned; the output does
                     not depend on it)
    align            4 x 6 true displacement of the layers (dx, dy, dz [mm], wx, wy, wz
                     [rad], layer L moved to R(w) x + d, R = Rz Ry Rx); hits are
                     digitised in each layer's own frame
    b_scale          true field / nominal field
    Returns dict with ``hits`` (int32), ``off`` (int64, F+1), per-hit truth ``hit_track``
    (global track id or -1), ``hit_layer``, ``hit_pos`` (float64 true crossing points of
    track hits, pixel centres of noise hits), per-track truth ``trk_*`` and
    ``frame_signal``.  With digitise=False the addresses still carry layer and pixel
    but ``hit_pos`` is the position to fit.
    """
    cfg = cfg or load_config()
    geo = Geometry(cfg)
    if track_counts is None:
        rng0 = np.random.default_rng([seed, 0x7ac])
        track_counts = rng0.poisson(mean_tracks, n_frames)
    track_counts = np.asarray(track_counts, np.int64)
    fsig = np.zeros(n_frames, bool)
    if signal_every:
        fsig[::signal_every] = True
    frames, addrs, trks, lays, poss = [], [], [], [], []
    tr_all = {}
    base_track = 0
    jobs = []
    for c0 in range(0, n_frames, CHUNK_FRAMES):
        nf = min(CHUNK_FRAMES, n_frames - c0)
        lam = noise_per_layer if noise_scale is None else noise_per_layer * np.asarray(noise_scale[c0:c0 + nf], float)
        jobs.append((cfg, seed, c0, nf, track_counts[c0:c0 + nf], fsig[c0:c0 + nf], lam, ms, digitise, noise,
                     p_range, cos_range, None if align is None else np.asarray(align, float), float(b_scale)))
    if workers is None:
        import sys
        main_file = getattr(sys.modules.get("__main__"), "__file__", None)
        spawnable = main_file is None or os.path.exists(main_file)  # spawn re-imports the main script
        workers = min(len(jobs), os.cpu_count() or 1, 16) if spawnable and len(jobs) >= 4 else 1
    if workers > 1 and len(jobs) > 1:
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
            results = list(ex.map(_chunk_job, jobs))
    else:
        results = [_chunk_job(j) for j in jobs]
    for fr, ad, tr, ly, pos, tracks in results:
        tr = np.where(tr >= 0, tr + base_track, -1)
        base_track += tracks["frame"].size
        frames.append(fr); addrs.append(ad); trks.append(tr); lays.append(ly); poss.append(pos)
        for k, v in tracks.items():
            tr_all.setdefault(k, []).append(v)
    fr = np.concatenate(frames) if frames else np.zeros(0, np.int64)
    off = np.zeros(n_frames + 1, np.int64)
    np.cumsum(np.bincount(fr, minlength=n_frames), out=off[1:])
    out = dict(hits=np.concatenate(addrs) if addrs else np.zeros(0, np.int32), off=off,
               hit_track=np.concatenate(trks).astype(np.int64) if trks else np.zeros(0, np.int64),
               hit_layer=np.concatenate(lays) if lays else np.zeros(0, np.int8),
               hit_pos=np.concatenate(poss) if poss else np.zeros((0, 3)),
               frame_signal=fsig, digitised=digitise)
    for k, v in tr_all.items():
        out["trk_" + k] = np.concatenate(v)
    return out


# --------------------------------------------------------------------------- named workloads

def c4_truth(seed: int = 4) -> dict:
    """Injected misalignment of the c4 workload: per layer N(0, 50 um) in x, y, z and
    N(0, 0.5 mrad) in the three rotations, field scale 1 + N(0, 1e-3)."""
    rng = np.random.default_rng([seed, 0xa119])
    align = np.concatenate([rng.normal(0.0, 0.050, (4, 3)), rng.normal(0.0, 0.5e-3, (4, 3))], 1)
    return dict(align=align, b_scale=1.0 + rng.normal(0.0, 1e-3))


def workload(name: str, n_frames: int | None = None, seed: int | None = None) -> dict:
    """The synthetic workloads: ``c1`` (parity: Poisson(10) tracks, 0.5 noise/layer,
    signal every 10th frame), ``c2`` (throughput: Poisson(20), 2 noise/layer, signal in
    0.1% of frames), ``c3`` (uneven: lognormal(median 15, sigma 1) tracks capped at 400,
    0.5 noise/layer, 1% of frames at 100x noise), ``c5`` (streaming: the c1 frame mix,
    signal every 10th frame, 1,000,000 frames, seed 5; the arrival process is the
    replay's)."""
    if name == "c4":
        # the c1 mix with the layers displaced and the field off nominal (seed 4)
        s = seed if seed is not None else 4
        truth = c4_truth(s)
        out = generate(n_frames or 100_000, 10.0, 0.5, 10, s, align=truth["align"], b_scale=truth["b_scale"])
        out.update(truth_align=truth["align"], truth_b_scale=truth["b_scale"])
        return out
    if name == "c5":
        return generate(n_frames or 1_000_000, 10.0, 0.5, 10, seed if seed is not None else 5)
    if name == "c1":
        return generate(n_frames or 1000, 10.0, 0.5, 10, seed if seed is not None else 1)
    if name == "c2":
        return generate(n_frames or 1_000_000, 20.0, 2.0, 1000, seed if seed is not None else 2)
    if name == "c3":
        nf = n_frames or 200_000
        s = seed if seed is not None else 3
        rng = np.random.default_rng([s, 0xc3])
        counts = np.minimum(400, np.round(rng.lognormal(math.log(15.0), 1.0, nf))).astype(np.int64)
        scale = np.where(rng.random(nf) < 0.01, 100.0, 1.0)
        return generate(nf, track_counts=counts, noise_per_layer=0.5, signal_every=1000, seed=s,
                        noise_scale=scale)
    raise ValueError(name)
