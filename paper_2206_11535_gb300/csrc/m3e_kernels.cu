// Selection kernels of libm3e: the whole per-frame method of the paper
// (Algorithm 1: load, selection cuts, track reconstruction, vertex fit, store)
// in FP32 with IEEE division and square root.
//
// One routine, process_frame<Group>, runs a frame on a group of threads: a warp
// (persistent kernel, warp per frame, frames from a device work queue) or a
// whole CTA (frames too large for a warp's shared-memory stage, and the plain
// per-frame form).  Per frame:
//   A  decode the int32 pixel addresses and histogram them by (layer, phi bin)
//   B  counting sort into shared memory: x, y, z, phi from FP64-built tables
//   C  selection cuts: for each layer-1 hit, layer-0 and layer-2 partners from
//      the phi bins that can pass the Phi cuts, then Delta lambda and r_tc
//   D  triplet fit, layer-3 extrapolation and closest hit, second triplet fit,
//      global curvature and chi2 cut (one thread per selected triplet)
//   E  energy test of every e+ e+ e- combination
//   F  vertex of each surviving combination, early exit once one passes
#include <cfloat>

#include "m3e_internal.cuh"

namespace m3e {
namespace {

constexpr float PI_F = 3.14159265358979323846f;
constexpr float TWO_PI_F = 6.28318530717958647692f;
constexpr unsigned FULL = 0xffffffffu;

// ------------------------------------------------------------------ thread groups

struct WarpGroup {
  static constexpr int N = 32;
  __device__ __forceinline__ int rank() const { return threadIdx.x & 31; }
  __device__ __forceinline__ void sync() const { __syncwarp(); }
  __device__ __forceinline__ bool any(bool p) const { return __any_sync(FULL, p) != 0; }
  __device__ __forceinline__ bool leader() const { return (threadIdx.x & 31) == 0; }
};

template <int NT>
struct CtaGroup {
  static constexpr int N = NT;
  __device__ __forceinline__ int rank() const { return threadIdx.x; }
  __device__ __forceinline__ void sync() const { __syncthreads(); }
  __device__ __forceinline__ bool any(bool p) const { return __syncthreads_or(p) != 0; }
  __device__ __forceinline__ bool leader() const { return threadIdx.x == 0; }
};

// ------------------------------------------------------------------ shared-memory stage

struct TrkS {          // a kept track, as the vertex stage needs it
  float cx, cy, rt;    // transverse circle through the layer-0 and layer-1 hits
  float R, ct, st;     // 3D radius and cos/sin of the first segment's polar angle
  float p, E, sms;     // momentum, energy, MS width at layer 0
  float h0x, h0y, h0z; // layer-0 hit
  float ah0;           // angle of the layer-0 hit seen from the circle centre
  float eps;           // turning sense, +1 clockwise (positive charge)
  int tid;             // index of the triplet it came from
  int pad;
};

template <int CH, int CT, int CK, int CC>
struct FrameSm {
  float x[CH], y[CH], z[CH], phi[CH];
  uint32_t addr[CH];
  uint16_t inidx[CH];
  uint8_t bin[CH];
  uint16_t bstart[NBK + 1];
  int bcur[NBK];
  TrkS trk[CK];                 // positives from the front, negatives from the back
  union {
    ushort4 trip[CT];           // selected triplets (sorted-hit indices)
    uint32_t combo[CC];         // e+ e+ e- combinations (track indices), after the fits
  } u;
  int ntrip, npos, nneg, ncombo, flag, bad;
  unsigned long long acc[ST_REASON0 + 8];  // statistics of this group's frames
  unsigned long long facc[ST_REASON0];     // statistics of the current frame
};

using SmWarp = FrameSm<W_HITS, W_TRIP, W_TRK, W_COMBO>;
using SmCta = FrameSm<C_HITS, C_TRIP, C_TRK, C_COMBO>;

// ------------------------------------------------------------------ small helpers

struct Dec {
  int L, g, row, b;
  bool ok;
};

__device__ __forceinline__ Dec decode(const DevCfg& C, uint32_t a) {
  Dec d;
  d.L = (a >> 26) & 3;
  const int lad = (a >> 21) & 31, col = (a >> 13) & 255;
  d.row = a & 8191;
  d.ok = (a >> 28) == 0 && lad < C.nlad[d.L] && col < C.ncol[d.L] && d.row < C.nrow[d.L];
  d.g = lad * C.ncol[d.L] + col;
  d.b = d.ok ? (d.g * NB) / C.ntot[d.L] : 0;
  return d;
}

__device__ __forceinline__ float wrap_2pi(float a) {  // (-2 pi, 2 pi) -> [0, 2 pi)
  if (a < 0.f) a += TWO_PI_F;
  if (a >= TWO_PI_F) a -= TWO_PI_F;
  return a;
}

__device__ __forceinline__ float wrap_pi(float a) {  // (-2 pi, 2 pi) -> [-pi, pi]
  if (a > PI_F) a -= TWO_PI_F;
  if (a < -PI_F) a += TWO_PI_F;
  return a;
}

// sin(x) - x cos(x) for x in (0, pi].  For small x the two terms cancel to
// x^3/3, so the Taylor series sum_k (-1)^(k+1) 2k x^(2k+1) / (2k+1)! is used
// below 0.5 (five terms: truncation below FP32 rounding).
__device__ __forceinline__ float sin_minus_xcos(float x) {
  if (x < 0.5f) {
    const float x2 = x * x;
    float s = 1.f / 3991680.f;
    s = s * x2 - 1.f / 45360.f;
    s = s * x2 + 1.f / 840.f;
    s = s * x2 - 1.f / 30.f;
    s = s * x2 + 1.f / 3.f;
    return s * x2 * x;
  }
  float sx, cx;
  sincosf(x, &sx, &cx);
  return sx - x * cx;
}

// ------------------------------------------------------------------ triplet fit

struct SegF {
  float phi, RC, th, dphi, dth;
};

// One segment of the circle solution: chord d, axial length z, transverse radius
// Rct of the circle through the triplet.  Helix relations d = 2 R_t sin(Phi/2),
// z = R_t Phi cot(theta), R_t = R sin(theta) give the 3D radius R_C, the polar
// angle theta_C and the derivatives dPhi/dR, dtheta/dR at the circle solution.
__device__ __forceinline__ SegF segment(float d, float z, float Rct, bool obtuse) {
  SegF s;
  float ph = 2.f * asinf(fminf(1.f, d / (2.f * Rct)));
  if (obtuse) ph = TWO_PI_F - ph;
  const float zp = z / ph;
  s.RC = sqrtf(Rct * Rct + zp * zp);
  s.th = atan2f(Rct * ph, z);
  float sh, ch;
  sincosf(0.5f * ph, &sh, &ch);
  const float sh2 = sh * sh;
  const float dRdphi = -(d * d * ch / (8.f * sh2 * sh) + zp * zp / ph) / s.RC;
  s.dphi = 1.f / dRdphi;
  const float g = ph / (2.f * sh);
  const float gp = sin_minus_xcos(0.5f * ph) / (2.f * sh2);
  const float dg = d * g;
  s.dth = z * d * gp / (z * z + dg * dg) * s.dphi;
  s.phi = ph;
  return s;
}

struct TFitF {
  bool valid;
  float eps, Rct, ccx, ccy;
  float Rref;                  // expansion point of the kink model: R_C of segment 0
  float alpha, a0p, beta, b0p; // Phi_MS ~ alpha u + a0p, Theta_MS ~ beta u + b0p, u = R - Rref
  float s2;                    // sin^2 of the mean polar angle
  float kappa, skappa;
  float thC0, thC1, RC0, dth0;
};

// Single triplet fit, hits a -> b -> c, scattering at b (Sec. "Single Triplet
// Fit"): linear kink model around the circle solution and its closed-form
// minimum in the 3D radius.  The model is written in u = R - R_C0 so that the
// small offsets (R_C0 - R_C1, theta_C1 - theta_C0) enter directly instead of as
// differences of large products; the algebra equals the minimum of
// [Phi_MS^2 sin^2(theta) + Theta_MS^2] / sigma_MS^2.
__device__ __forceinline__ TFitF fit_triplet(float ax, float ay, float az, float bx, float by, float bz,
                                             float cx, float cy, float cz, float hl, float kB) {
  TFitF f;
  f.valid = false;
  const float ux = ax - bx, uy = ay - by, vx = cx - bx, vy = cy - by;
  const float cross = ux * vy - uy * vx;
  const float u2 = ux * ux + uy * uy, v2 = vx * vx + vy * vy;
  const float wx = cx - ax, wy = cy - ay;
  const float d01 = sqrtf(u2), d12 = sqrtf(v2), d20 = sqrtf(wx * wx + wy * wy);
  if (!(cross != 0.f)) return f;
  const float rtc = d01 * d12 * d20 / (2.f * cross);
  if (!isfinite(rtc) || rtc == 0.f) return f;
  f.Rct = fabsf(rtc);
  f.eps = rtc > 0.f ? 1.f : -1.f;
  f.ccx = bx + (vy * u2 - uy * v2) / (2.f * cross);
  f.ccy = by + (ux * v2 - vx * u2) / (2.f * cross);
  const bool ob0 = ((ax - cx) * (bx - cx) + (ay - cy) * (by - cy)) < 0.f;
  const bool ob1 = ((bx - ax) * (cx - ax) + (by - ay) * (cy - ay)) < 0.f;
  const SegF s0 = segment(d01, bz - az, f.Rct, ob0);
  const SegF s1 = segment(d12, cz - bz, f.Rct, ob1);
  const float dR = s0.RC - s1.RC;
  f.Rref = s0.RC;
  f.alpha = 0.5f * (s0.dphi + s1.dphi);
  f.a0p = 0.5f * s1.dphi * dR;
  f.beta = s1.dth - s0.dth;
  f.b0p = (s1.th - s0.th) + s1.dth * dR;
  const float sn = sinf(0.5f * (s0.th + s1.th));
  f.s2 = sn * sn;
  const float den = f.alpha * f.alpha * f.s2 + f.beta * f.beta;
  const float u = -(f.alpha * f.a0p * f.s2 + f.beta * f.b0p) / den;
  const float Rs = f.Rref + u;
  if (!(Rs > 0.f) || !isfinite(Rs)) return f;
  const float sms = hl / (kB * Rs);
  f.kappa = f.eps / Rs;
  f.skappa = sms / sqrtf(den) / (Rs * Rs);
  if (!isfinite(f.kappa) || !isfinite(f.skappa) || !(f.skappa > 0.f)) return f;
  f.thC0 = s0.th;
  f.thC1 = s1.th;
  f.RC0 = s0.RC;
  f.dth0 = s0.dth;
  f.valid = true;
  return f;
}

__device__ __forceinline__ float kink_chi2(const TFitF& f, float R, float sg) {
  const float u = R - f.Rref;
  const float kp = f.alpha * u + f.a0p, kt = f.beta * u + f.b0p;
  return (kp * kp * f.s2 + kt * kt) / (sg * sg);
}

// ------------------------------------------------------------------ track reconstruction

struct TrackOut {
  int status, i3;
  float kbar, th01, chi2, mbest;
};

// Algorithm 3 for one selected triplet (sorted-hit indices i0, i1, i2): fit,
// estimate the layer-3 point from the first triplet's circle and the second
// segment's polar angle, take the closest layer-3 hit ((r3 dphi)^2 + dz^2, ties
// to the smaller address), fit (h1, h2, h3), weighted mean curvature and chi2 of
// both triplets at it, chi2 cut.  On success fills *t for the vertex stage.
template <class S>
__device__ TrackOut build_track(const S& sm, const DevCfg& C, int i0, int i1, int i2, TrkS* t) {
  TrackOut o;
  o.status = 0;
  o.i3 = -1;
  o.kbar = o.th01 = o.chi2 = o.mbest = 0.f;
  const float x0 = sm.x[i0], y0 = sm.y[i0], z0 = sm.z[i0];
  const float x1 = sm.x[i1], y1 = sm.y[i1], z1 = sm.z[i1];
  const float x2 = sm.x[i2], y2 = sm.y[i2], z2 = sm.z[i2];
  const TFitF f1 = fit_triplet(x0, y0, z0, x1, y1, z1, x2, y2, z2, C.hl[1], C.kB);
  if (!f1.valid) return o;
  const float r3 = C.r3;
  const float D = sqrtf(f1.ccx * f1.ccx + f1.ccy * f1.ccy);
  o.status = 1;
  if (!(D > 0.f) || D > f1.Rct + r3 || D < fabsf(f1.Rct - r3)) return o;
  const float a = (r3 * r3 - (f1.Rct - D) * (f1.Rct + D)) / (2.f * D);
  const float hh = sqrtf(fmaxf((r3 - a) * (r3 + a), 0.f));
  const float ux = f1.ccx / D, uy = f1.ccy / D;
  const float qx0 = a * ux - hh * uy, qy0 = a * uy + hh * ux;
  const float qx1 = a * ux + hh * uy, qy1 = a * uy - hh * ux;
  const float a2 = atan2f(y2 - f1.ccy, x2 - f1.ccx);
  const float al0 = wrap_2pi(f1.eps * (a2 - atan2f(qy0 - f1.ccy, qx0 - f1.ccx)));
  const float al1 = wrap_2pi(f1.eps * (a2 - atan2f(qy1 - f1.ccy, qx1 - f1.ccx)));
  const bool take1 = al1 < al0;
  const float al = take1 ? al1 : al0;
  const float qx = take1 ? qx1 : qx0, qy = take1 ? qy1 : qy0;
  float s12, c12;
  sincosf(f1.thC1, &s12, &c12);
  const float z3 = z2 + f1.Rct * al * c12 / s12;
  const float phi3 = atan2f(qy, qx);
  int best = -1;
  float mb = FLT_MAX;
  uint32_t ab = 0;
  const int l3a = sm.bstart[3 * NB], l3b = sm.bstart[4 * NB];
  for (int j = l3a; j < l3b; ++j) {
    const float dphi = wrap_pi(sm.phi[j] - phi3);
    const float dz = sm.z[j] - z3;
    const float m = (r3 * dphi) * (r3 * dphi) + dz * dz;
    const uint32_t aj = sm.addr[j];
    if (best < 0 || m < mb || (m == mb && aj < ab)) {
      best = j;
      mb = m;
      ab = aj;
    }
  }
  o.status = 2;
  if (best < 0) return o;
  o.i3 = best;
  o.mbest = mb;
  const float x3 = sm.x[best], y3 = sm.y[best], z3h = sm.z[best];
  const TFitF f2 = fit_triplet(x1, y1, z1, x2, y2, z2, x3, y3, z3h, C.hl[2], C.kB);
  o.status = 3;
  if (!f2.valid) return o;
  const float w1 = 1.f / (f1.skappa * f1.skappa), w2 = 1.f / (f2.skappa * f2.skappa);
  const float kb = (f1.kappa * w1 + f2.kappa * w2) / (w1 + w2);
  o.kbar = kb;
  if (!(kb != 0.f) || !isfinite(kb)) return o;
  const float Rb = 1.f / fabsf(kb);
  const float pb = C.kB * Rb;
  const float chi2 = kink_chi2(f1, Rb, C.hl[1] / pb) + kink_chi2(f2, Rb, C.hl[2] / pb);
  o.chi2 = chi2;
  o.th01 = f1.thC0 + f1.dth0 * (Rb - f1.RC0);
  if (!isfinite(chi2)) return o;
  o.status = 4;
  if (!(chi2 < C.chi2_trk)) return o;
  o.status = 5;
  // track for the vertex stage: transverse circle of radius R sin(theta01) through
  // the layer-0 and layer-1 hits, centre on the side the track turns to
  float st, ct;
  sincosf(o.th01, &st, &ct);
  t->R = Rb;
  t->ct = ct;
  t->st = st;
  t->rt = Rb * st;
  t->p = pb;
  t->E = sqrtf(pb * pb + C.me2);
  t->sms = C.hl[0] / pb;
  t->eps = kb > 0.f ? 1.f : -1.f;
  t->h0x = x0;
  t->h0y = y0;
  t->h0z = z0;
  const float dx = x1 - x0, dy = y1 - y0;
  const float d = sqrtf(dx * dx + dy * dy);
  const float ex = dx / d, ey = dy / d;
  const float hd = 0.5f * d;
  const float off = sqrtf(fmaxf((t->rt - hd) * (t->rt + hd), 0.f));
  const float mx = 0.5f * (x0 + x1), my = 0.5f * (y0 + y1);
  t->cx = mx + t->eps * ey * off;
  t->cy = my - t->eps * ex * off;
  t->ah0 = atan2f(y0 - t->cy, x0 - t->cx);
  return o;
}

// ------------------------------------------------------------------ vertex

__device__ __forceinline__ float arc_to_h0(const TrkS& t, float x, float y) {
  return wrap_2pi(t.eps * (atan2f(y - t.cy, x - t.cx) - t.ah0));
}

__device__ __forceinline__ float point_var(const TrkS& t, float x, float y, float sp2) {
  const float s = t.rt * arc_to_h0(t, x, y);
  return t.sms * t.sms * s * s + sp2;
}

__device__ __forceinline__ float target_distance(const DevCfg& C, float x, float y, float z) {
  const float px = sqrtf(x * x + y * y), pz = fabsf(z);
  const float ex = -C.tgt_r, ez = C.tgt_h;
  float t = ((px - C.tgt_r) * ex + pz * ez) / (ex * ex + ez * ez);
  t = fminf(1.f, fmaxf(0.f, t));
  const float dx = px - (C.tgt_r + t * ex), dz = pz - t * ez;
  return sqrtf(dx * dx + dz * dz);
}

struct VtxOut {
  int status, pass;
  float chi2, tdist, ptot;
};

// Vertex of one e+ e+ e- combination (Sec. "Vertex Fit", "Signal Estimation"):
// pairwise circle intersections, target-disk filter, error-weighted transverse
// mean for each choice of one point per pair, closest points, z projection,
// chi2; the smallest-chi2 choice is cut on chi2, target distance and |sum p|.
__device__ VtxOut vertex(const TrkS& A, const TrkS& B, const TrkS& E, const DevCfg& C) {
  const TrkS* V[3] = {&A, &B, &E};
  VtxOut o;
  o.status = 2;
  o.pass = 0;
  o.chi2 = o.tdist = o.ptot = FLT_MAX;
  float px[3][2], py[3][2], pv[3][2];
  int npt[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const TrkS& a = *V[k == 2 ? 1 : 0];
    const TrkS& b = *V[k == 0 ? 1 : 2];
    float ex = b.cx - a.cx, ey = b.cy - a.cy;
    const float D = sqrtf(ex * ex + ey * ey);
    npt[k] = 0;
    if (!(D > 0.f)) {
      o.status = 0;
      return o;
    }
    const float aa = ((a.rt - b.rt) * (a.rt + b.rt) + D * D) / (2.f * D);
    const float h2 = (a.rt - aa) * (a.rt + aa);
    if (h2 < 0.f) {
      o.status = 0;
      return o;
    }
    ex /= D;
    ey /= D;
    const float bx = a.cx + aa * ex, by = a.cy + aa * ey;
    const float h = sqrtf(h2);
    const int nc = h2 == 0.f ? 1 : 2;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      if (j >= nc) break;
      const float sg = j == 0 ? 1.f : -1.f;
      const float qx = bx - sg * h * ey, qy = by + sg * h * ex;
      if (sqrtf(qx * qx + qy * qy) > C.isect_lim) continue;
      const int m = npt[k];
      px[k][m] = qx;
      py[k][m] = qy;
      pv[k][m] = point_var(a, qx, qy, C.sig_pix2) + point_var(b, qx, qy, C.sig_pix2);
      npt[k] = m + 1;
    }
  }
  if (npt[0] == 0 || npt[1] == 0 || npt[2] == 0) {
    o.status = 1;
    return o;
  }
  float bmx = 0.f, bmy = 0.f, bmz = 0.f;
  float bpx[3] = {0.f, 0.f, 0.f}, bpy[3] = {0.f, 0.f, 0.f};
  float best = FLT_MAX;
  bool have = false;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int s0 = (c >> 2) & 1, s1 = (c >> 1) & 1, s2 = c & 1;  // s2 fastest
    if (s0 >= npt[0] || s1 >= npt[1] || s2 >= npt[2]) continue;
    const float w0 = 1.f / pv[0][s0], w1 = 1.f / pv[1][s1], w2 = 1.f / pv[2][s2];
    const float ws = w0 + w1 + w2;
    const float mx = (px[0][s0] * w0 + px[1][s1] * w1 + px[2][s2] * w2) / ws;
    const float my = (py[0][s0] * w0 + py[1][s1] * w1 + py[2][s2] * w2) / ws;
    float cx[3], cy[3], zi[3], vi[3];
    bool bad = false;
    float wz = 0.f, wzs = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const TrkS& t = *V[i];
      const float dx = mx - t.cx, dy = my - t.cy;
      const float dn = sqrtf(dx * dx + dy * dy);
      if (!(dn > 0.f)) bad = true;
      cx[i] = t.cx + t.rt * dx / dn;
      cy[i] = t.cy + t.rt * dy / dn;
      const float dphi = arc_to_h0(t, cx[i], cy[i]);
      zi[i] = t.h0z - dphi * t.R * t.ct;
      const float s = t.rt * dphi;
      vi[i] = t.sms * t.sms * s * s + C.sig_pix2;
      wz += zi[i] / vi[i];
      wzs += 1.f / vi[i];
    }
    if (bad) continue;
    const float mz = wz / wzs;
    float chi2 = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const float dx = cx[i] - mx, dy = cy[i] - my, dz = zi[i] - mz;
      chi2 += (dx * dx + dy * dy + dz * dz) / vi[i];
    }
    if (!have || chi2 < best) {
      have = true;
      best = chi2;
      bmx = mx;
      bmy = my;
      bmz = mz;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        bpx[i] = cx[i];
        bpy[i] = cy[i];
      }
    }
  }
  if (!have || !isfinite(best)) {
    o.status = 1;
    return o;
  }
  o.chi2 = best;
  o.tdist = target_distance(C, bmx, bmy, bmz);
  float Px = 0.f, Py = 0.f, Pz = 0.f;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const TrkS& t = *V[i];
    const float ux = (bpx[i] - t.cx) / t.rt, uy = (bpy[i] - t.cy) / t.rt;
    const float pt = t.p * t.st;
    Px += pt * t.eps * uy;
    Py -= pt * t.eps * ux;
    Pz += t.p * t.ct;
  }
  o.ptot = sqrtf(Px * Px + Py * Py + Pz * Pz);
  o.pass = o.chi2 <= C.vtx_chi2 && o.tdist <= C.tgt_dist && o.ptot <= C.ptot_max;
  return o;
}

// ------------------------------------------------------------------ one frame

template <class G>
__device__ __forceinline__ void bucket_scan(const G& g, int* bcur, uint16_t* bstart) {
  if (g.rank() < 32) {
    const int lane = g.rank();
    int v[NBK / 32];
    int s = 0;
#pragma unroll
    for (int k = 0; k < NBK / 32; ++k) {
      v[k] = bcur[lane * (NBK / 32) + k];
      s += v[k];
    }
    int inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(FULL, inc, o);
      if (lane >= o) inc += t;
    }
    int ex = inc - s;
#pragma unroll
    for (int k = 0; k < NBK / 32; ++k) {
      bstart[lane * (NBK / 32) + k] = (uint16_t)ex;
      bcur[lane * (NBK / 32) + k] = ex;
      ex += v[k];
    }
    if (lane == 31) bstart[NBK] = (uint16_t)inc;
  }
  g.sync();
}

template <class G, class S, int CH, int CT, int CK, int CC, bool DEFER, bool DEBUG>
__device__ int process_frame(const G& g, S& sm, const DevCfg& C, const KParams& P, int f) {
  const bool stats = P.stats != nullptr;
  const int64_t base = P.off[f] - P.off_base;
  const int64_t n64 = P.off[f + 1] - P.off[f];
  if (DEBUG && g.leader()) {
    P.dump.n_trip[f] = 0;
    P.dump.n_combo[f] = 0;
  }
  if (n64 < 0) {
    if (g.leader()) atomicOr(P.err, ERR_NEGSIZE);
    return M3E_ERR_BADHIT;
  }
  if (DEFER && n64 > CH) return DEFERRED;
  const int n = (int)(n64 > 0x7fffffff ? 0x7fffffff : n64);
  const int32_t* hp = P.hits + base;

  // ---- A: decode and histogram
  for (int k = g.rank(); k < NBK; k += G::N) sm.bcur[k] = 0;
  if (g.leader()) {
    sm.bad = 0;
    sm.ntrip = 0;
    sm.npos = 0;
    sm.nneg = 0;
    sm.ncombo = 0;
    sm.flag = 0;
    if (stats)
      for (int k = 0; k < ST_REASON0; ++k) sm.facc[k] = 0;
  }
  g.sync();
  for (int i = g.rank(); i < n; i += G::N) {
    const Dec d = decode(C, (uint32_t)__ldg(hp + i));
    if (!d.ok) sm.bad = 1;
    else if (n <= CH) atomicAdd(&sm.bcur[d.L * NB + d.b], 1);
  }
  g.sync();
  if (sm.bad) {
    if (g.leader()) atomicOr(P.err, ERR_BADHIT);
    return M3E_ERR_BADHIT;
  }
  if (n > C.max_hits || n > CH) return M3E_HIT_OVERFLOW;
  if (stats && g.leader()) {
    sm.facc[ST_FRAMES] += 1;
    sm.facc[ST_HITS] += n;
  }

  // ---- B: counting sort by (layer, phi bin)
  bucket_scan(g, sm.bcur, sm.bstart);
  for (int i = g.rank(); i < n; i += G::N) {
    const uint32_t a = (uint32_t)__ldg(hp + i);
    const Dec d = decode(C, a);
    const int key = d.L * NB + d.b;
    const int pos = atomicAdd(&sm.bcur[key], 1);
    const float4 cl = __ldg(P.col_lut + C.col_off[d.L] + d.g);
    sm.x[pos] = cl.x;
    sm.y[pos] = cl.y;
    sm.phi[pos] = cl.z;
    sm.z[pos] = __ldg(P.row_lut + C.row_off[d.L] + d.row);
    sm.addr[pos] = a;
    sm.inidx[pos] = (uint16_t)i;
    sm.bin[pos] = (uint8_t)d.b;
  }
  g.sync();

  // ---- C: selection cuts (Algorithm 2), pairs restricted to reachable phi bins
  {
    unsigned npair = 0, ntt = 0;
    const int l1a = sm.bstart[NB], l1b = sm.bstart[2 * NB];
    const int nb0 = min(2 * C.k01 + 1, NB), nb2 = min(2 * C.k12 + 1, NB);
    for (int i1 = l1a + g.rank(); i1 < l1b; i1 += G::N) {
      const float x1 = sm.x[i1], y1 = sm.y[i1], z1 = sm.z[i1];
      const int b1 = sm.bin[i1];
      const int s0 = nb0 == NB ? 0 : (b1 - C.k01 + NB) & (NB - 1);
      const int s2 = nb2 == NB ? 0 : (b1 - C.k12 + NB) & (NB - 1);
      for (int w0 = 0; w0 < nb0; ++w0) {
        const int bb0 = (s0 + w0) & (NB - 1);
        const int e0 = sm.bstart[bb0 + 1];
        for (int i0 = sm.bstart[bb0]; i0 < e0; ++i0) {
          const float x0 = sm.x[i0], y0 = sm.y[i0];
          ++npair;
          if (!(x0 * x1 + y0 * y1 >= C.c01)) continue;
          const float tl01 = (z1 - sm.z[i0]) * C.inv_dr01;
          for (int w2 = 0; w2 < nb2; ++w2) {
            const int bb2 = 2 * NB + ((s2 + w2) & (NB - 1));
            const int e2 = sm.bstart[bb2 + 1];
            for (int i2 = sm.bstart[bb2]; i2 < e2; ++i2) {
              const float x2 = sm.x[i2], y2 = sm.y[i2];
              ++npair;
              if (!(x1 * x2 + y1 * y2 >= C.c12)) continue;
              ++ntt;
              const float dl = (sm.z[i2] - z1) * C.inv_dr12 - tl01;
              if (!(fabsf(dl) <= C.dl_max)) continue;
              const float ax = x0 - x1, ay = y0 - y1, bx = x2 - x1, by = y2 - y1;
              const float cr = ax * by - ay * bx;
              const float ex = x2 - x0, ey = y2 - y0;
              const float Pq = (ax * ax + ay * ay) * (bx * bx + by * by) * (ex * ex + ey * ey);
              const float Qq = cr * cr;
              if (!(cr != 0.f && Pq >= C.rtc_lo2 * Qq && Pq <= C.rtc_hi2 * Qq)) continue;
              const int k = atomicAdd(&sm.ntrip, 1);
              if (k < CT) sm.u.trip[k] = make_ushort4((uint16_t)i0, (uint16_t)i1, (uint16_t)i2, 0);
            }
          }
        }
      }
    }
    if (stats) {
      atomicAdd(&sm.facc[ST_PAIRS], (unsigned long long)npair);
      atomicAdd(&sm.facc[ST_TTESTS], (unsigned long long)ntt);
    }
  }
  g.sync();
  const int ntrip = sm.ntrip;
  if (DEBUG && g.leader()) P.dump.n_trip[f] = ntrip;
  if (ntrip > C.max_trip) return M3E_TRIPLET_OVERFLOW;
  if (DEFER && ntrip > CT) return DEFERRED;
  if (stats && g.leader()) sm.facc[ST_TRIP] += ntrip;

  // ---- D: track reconstruction (Algorithm 3), one thread per triplet
  for (int t = g.rank(); t < ntrip; t += G::N) {
    const ushort4 tr = sm.u.trip[t];
    TrkS tk;
    const TrackOut o = build_track(sm, C, tr.x, tr.y, tr.z, &tk);
    if (o.status == 5) {
      tk.tid = t;
      int slot = -1;
      if (tk.eps > 0.f) {
        const int k = atomicAdd(&sm.npos, 1);
        if (k < CK) slot = k;
      } else {
        const int k = atomicAdd(&sm.nneg, 1);
        if (k < CK) slot = CK - 1 - k;
      }
      if (slot >= 0) sm.trk[slot] = tk;
    }
    if (DEBUG && t < P.dump.cap_trip) {
      const int64_t r = (int64_t)f * P.dump.cap_trip + t;
      P.dump.trip[4 * r + 0] = sm.inidx[tr.x];
      P.dump.trip[4 * r + 1] = sm.inidx[tr.y];
      P.dump.trip[4 * r + 2] = sm.inidx[tr.z];
      P.dump.trip[4 * r + 3] = o.i3 >= 0 ? (int)sm.inidx[o.i3] : -1;
      P.dump.trk_status[r] = o.status;
      P.dump.trk_val[4 * r + 0] = o.kbar;
      P.dump.trk_val[4 * r + 1] = o.th01;
      P.dump.trk_val[4 * r + 2] = o.chi2;
      P.dump.trk_val[4 * r + 3] = o.mbest;
    }
  }
  g.sync();
  const int npos = sm.npos, nneg = sm.nneg;
  const int ntrk = npos + nneg;
  if (ntrk > C.max_trk) return M3E_TRACK_OVERFLOW;
  if (DEFER && ntrk > CK) return DEFERRED;
  if (stats && g.leader()) sm.facc[ST_TRK] += ntrk;

  // ---- E: energy test of every (e+ pair, e-) combination (Algorithm 4, part 1)
  {
    const int npair = npos * (npos - 1) / 2;
    const int ntest = npair * nneg;
    for (int t = g.rank(); t < ntest; t += G::N) {
      const int pr = t / nneg, c = t - pr * nneg;
      int b = (int)((1.f + sqrtf(1.f + 8.f * (float)pr)) * 0.5f);
      while (b * (b - 1) / 2 > pr) --b;
      while ((b + 1) * b / 2 <= pr) ++b;
      const int a = pr - b * (b - 1) / 2;
      const int ci = CK - 1 - c;
      const float e = sm.trk[a].E + sm.trk[b].E + sm.trk[ci].E - C.m_mu;
      if (fabsf(e) <= C.e_win) {
        const int k = atomicAdd(&sm.ncombo, 1);
        if (k < CC) sm.u.combo[k] = (uint32_t)a | ((uint32_t)b << 8) | ((uint32_t)ci << 16);
      }
    }
    if (stats && g.leader()) sm.facc[ST_ETEST] += ntest;
  }
  g.sync();
  const int ncombo = sm.ncombo;
  if (DEBUG && g.leader()) P.dump.n_combo[f] = ncombo;
  if (ncombo > C.max_combo) return M3E_COMBO_OVERFLOW;
  if (DEFER && ncombo > CC) return DEFERRED;
  if (stats && g.leader()) sm.facc[ST_COMBO] += ncombo;

  // ---- F: vertex of each combination (Algorithm 4, part 2), early exit
  bool found = false;
  unsigned nv = 0;
  for (int c0 = 0; c0 < ncombo; c0 += G::N) {
    const int c = c0 + g.rank();
    bool pass = false;
    if (c < ncombo) {
      const uint32_t cb = sm.u.combo[c];
      const int a = cb & 255, b = (cb >> 8) & 255, e = (cb >> 16) & 255;
      const VtxOut v = vertex(sm.trk[a], sm.trk[b], sm.trk[e], C);
      pass = v.pass != 0;
      nv += v.status == 2;
      if (DEBUG && c < P.dump.cap_combo) {
        const int64_t r = (int64_t)f * P.dump.cap_combo + c;
        P.dump.combo[4 * r + 0] = sm.trk[a].tid;
        P.dump.combo[4 * r + 1] = sm.trk[b].tid;
        P.dump.combo[4 * r + 2] = sm.trk[e].tid;
        P.dump.combo[4 * r + 3] = v.status | (v.pass << 8);
        P.dump.combo_val[4 * r + 0] = sm.trk[a].E + sm.trk[b].E + sm.trk[e].E - C.m_mu;
        P.dump.combo_val[4 * r + 1] = v.chi2;
        P.dump.combo_val[4 * r + 2] = v.tdist;
        P.dump.combo_val[4 * r + 3] = v.ptot;
      }
    }
    found = g.any(pass) || found;
    if (found && !DEBUG) break;
  }
  if (stats && nv) atomicAdd(&sm.facc[ST_VTX], (unsigned long long)nv);
  return found ? M3E_VERTEX : M3E_DROP;
}

// Store the frame's decision (store_frame of Algorithm 1) and commit its statistics.
template <class G, class S>
__device__ __forceinline__ void finish_frame(const G& g, S& sm, const KParams& P, int f, int r) {
  g.sync();
  if (g.leader()) {
    P.keep[f] = (uint8_t)(r != M3E_DROP);
    P.reason[f] = (uint8_t)r;
    if (P.stats) {
      sm.acc[ST_REASON0 + r] += 1;
      for (int k = 0; k < ST_REASON0; ++k) sm.acc[k] += sm.facc[k];
    }
  }
}

template <class G, class S>
__device__ __forceinline__ void flush_stats(const G& g, S& sm, const KParams& P) {
  g.sync();
  if (P.stats)
    for (int k = g.rank(); k < ST_REASON0 + 8; k += G::N)
      if (sm.acc[k]) atomicAdd(P.stats + k, sm.acc[k]);
}

template <class G, class S>
__device__ __forceinline__ void clear_stats(const G& g, S& sm) {
  for (int k = g.rank(); k < ST_REASON0 + 8; k += G::N) sm.acc[k] = 0;
  g.sync();
}

// ------------------------------------------------------------------ kernels

// Persistent warp-per-frame kernel: each warp takes `grab` frames at a time from
// the device work queue; a frame that outgrows the warp's shared-memory stage is
// appended to the deferred list for the CTA kernel.
template <bool DEBUG>
__global__ void __launch_bounds__(WARPS_PER_CTA * 32)
    k_select_warp(const __grid_constant__ DevCfg C, const __grid_constant__ KParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmWarp& sm = reinterpret_cast<SmWarp*>(smem_raw)[threadIdx.x >> 5];
  const WarpGroup g;
  clear_stats(g, sm);
  const int nf = (int)P.n_frames;
  for (;;) {
    int f0 = 0;
    if (g.leader()) f0 = atomicAdd(&P.work[0], P.grab);
    f0 = __shfl_sync(FULL, f0, 0);
    if (f0 >= nf) break;
    const int f1 = min(f0 + P.grab, nf);
    for (int f = f0; f < f1; ++f) {
      const int r = process_frame<WarpGroup, SmWarp, W_HITS, W_TRIP, W_TRK, W_COMBO, true, DEBUG>(g, sm, C, P, f);
      if (r == DEFERRED) {
        if (g.leader()) {
          const int k = atomicAdd(&P.work[1], 1);
          P.defer_list[k] = f;
          if (P.stats) sm.acc[ST_DEFER] += 1;
        }
      } else {
        finish_frame(g, sm, P, f, r);
      }
      g.sync();
    }
  }
  flush_stats(g, sm, P);
}

// CTA-per-frame kernel.  LIST: frames from the deferred list written by the warp
// kernel earlier on the same stream; otherwise frames 0..n-1, one CTA each
// (grid-stride when the grid is smaller).
template <int NT, bool DEBUG, bool LIST>
__global__ void __launch_bounds__(NT) k_select_cta(const __grid_constant__ DevCfg C, const __grid_constant__ KParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmCta& sm = *reinterpret_cast<SmCta*>(smem_raw);
  const CtaGroup<NT> g;
  clear_stats(g, sm);
  const int count = LIST ? P.work[1] : (int)P.n_frames;
  for (int i = blockIdx.x; i < count; i += gridDim.x) {
    const int f = LIST ? P.defer_list[i] : i;
    const int r = process_frame<CtaGroup<NT>, SmCta, C_HITS, C_TRIP, C_TRK, C_COMBO, false, DEBUG>(g, sm, C, P, f);
    finish_frame(g, sm, P, f, r);
    g.sync();
  }
  flush_stats(g, sm, P);
}

template <class K>
cudaError_t set_smem(K k, size_t bytes) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

size_t select_smem_bytes() { return sizeof(SmWarp) * WARPS_PER_CTA; }
size_t cta_smem_bytes() { return sizeof(SmCta); }

int select_blocks_per_sm() {
  int nb = 0;
  set_smem(k_select_warp<false>, select_smem_bytes());
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_select_warp<false>, WARPS_PER_CTA * 32,
                                                    select_smem_bytes()) != cudaSuccess)
    return 1;
  return nb > 0 ? nb : 1;
}

cudaError_t launch_select(const DevCfg& c, const KParams& p, int grid, bool debug, cudaStream_t s) {
  const size_t sm = select_smem_bytes();
  if (debug) {
    cudaError_t e = set_smem(k_select_warp<true>, sm);
    if (e != cudaSuccess) return e;
    k_select_warp<true><<<grid, WARPS_PER_CTA * 32, sm, s>>>(c, p);
  } else {
    cudaError_t e = set_smem(k_select_warp<false>, sm);
    if (e != cudaSuccess) return e;
    k_select_warp<false><<<grid, WARPS_PER_CTA * 32, sm, s>>>(c, p);
  }
  return cudaGetLastError();
}

cudaError_t launch_deferred(const DevCfg& c, const KParams& p, int grid, bool debug, cudaStream_t s) {
  const size_t sm = cta_smem_bytes();
  if (debug) {
    cudaError_t e = set_smem(k_select_cta<CTA_THREADS, true, true>, sm);
    if (e != cudaSuccess) return e;
    k_select_cta<CTA_THREADS, true, true><<<grid, CTA_THREADS, sm, s>>>(c, p);
  } else {
    cudaError_t e = set_smem(k_select_cta<CTA_THREADS, false, true>, sm);
    if (e != cudaSuccess) return e;
    k_select_cta<CTA_THREADS, false, true><<<grid, CTA_THREADS, sm, s>>>(c, p);
  }
  return cudaGetLastError();
}

cudaError_t launch_plain(const DevCfg& c, const KParams& p, bool debug, cudaStream_t s) {
  const size_t sm = cta_smem_bytes();
  const int grid = (int)(p.n_frames < 0x7fffffff ? p.n_frames : 0x7fffffff);
  if (grid == 0) return cudaSuccess;
  if (debug) {
    cudaError_t e = set_smem(k_select_cta<PLAIN_THREADS, true, false>, sm);
    if (e != cudaSuccess) return e;
    k_select_cta<PLAIN_THREADS, true, false><<<grid, PLAIN_THREADS, sm, s>>>(c, p);
  } else {
    cudaError_t e = set_smem(k_select_cta<PLAIN_THREADS, false, false>, sm);
    if (e != cudaSuccess) return e;
    k_select_cta<PLAIN_THREADS, false, false><<<grid, PLAIN_THREADS, sm, s>>>(c, p);
  }
  return cudaGetLastError();
}

}  // namespace m3e
