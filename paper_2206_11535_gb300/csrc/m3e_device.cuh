// Device code shared by the fused and the staged selection kernels: thread
// groups, the shared-memory frame stage, decode, the triplet fit, track
// reconstruction and the vertex, all in FP32 (the build uses the approximate
// division and square root, a few ulp; exact comparisons that decide an integer
// use explicitly rounded intrinsics).
#pragma once

#include <cfloat>
#include <type_traits>

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

// Kept tracks as structure of arrays: the energy test reads E[] with one index for
// all lanes (broadcast) and the vertex stage gathers by track index without the
// bank conflicts of a 64-byte record stride.
template <int CK>
struct TrkSoA {
  float cx[CK], cy[CK], rt[CK];     // transverse circle through the layer-0 and layer-1 hits
  float R[CK], ct[CK], st[CK];      // 3D radius and cos/sin of the first segment's polar angle
  float p[CK], E[CK], sms[CK];      // momentum, energy, MS width at layer 0
  float h0x[CK], h0y[CK], h0z[CK];  // layer-0 hit
  float ah0[CK];                    // angle of the layer-0 hit seen from the circle centre
  float eps[CK];                    // turning sense, +1 clockwise (positive charge)
  int tid[CK];                      // index of the triplet it came from
};

// PHI / IDX: whether the stage keeps each hit's phi (the layer-3 search of the
// fused track stage reads it) and its input index (candidate record only); a
// stage without them holds more frames in flight per SM.  Triplets of a stage of
// at most 256 hits are kept as 8-bit indices.
template <int CH, int CT, int CK, int CC, bool PHI = true, bool IDX = true, bool ADDR = true,
          int CH32 = (CH <= W_HITS ? CH : 1)>
struct FrameSm {
  static constexpr bool kPhi = PHI, kIdx = IDX, kAddr = ADDR;
  static constexpr bool kPackB = CH < 256;  // bucket cursors as bytes, four to a word
  using TripT = typename std::conditional<(CH <= 256), uchar4, ushort4>::type;
  float x[CH], y[CH], z[CH], phi[PHI ? CH : 1];
  uint32_t addr[ADDR ? CH : 1];
  uint16_t inidx[IDX ? CH : 1];
  uint16_t bstart[NBK + 1];
  uint32_t bcur[kPackB ? NBK / 4 : NBK];  // bucket counts, then cursors
  // warp stage, selection cuts (warp_cuts): the layer-2 hits in z-bin order (bin
  // starts zbs), the (layer-1 hit, Phi01 partner) pairs of a chunk of 32 layer-1 hits
  // (their layer-0 hits) and the candidate triplets of one round of pairs
  float4 zq[CH32 == 1 ? 1 : W_L2];  // layer-2 hits in z-bin order: x, y, z, sorted index (as int bits)
  uint8_t p01[CH32 == 1 ? 1 : W_P01];
  uint8_t zbs[CH32 == 1 ? 1 : NZB + 1];
  alignas(16) uint16_t cand[CH32 == 1 ? 1 : W_CAND];  // also the z-bin counters (32-bit words)
  // CTA stage, selection cuts: the layer-2 hits in z-bin order (sorted-hit indices),
  // the bin starts of that order and the bin cursors of its counting sort
  uint16_t zidx[CH32 == 1 ? CH : 1];
  uint16_t zbs2[CH32 == 1 ? NZB + 1 : 1];
  uint32_t zcur[CH32 == 1 ? NZB : 1];
  TrkSoA<CK> t;                 // positives from the front, negatives from the back
  union {
    TripT trip[CT];             // selected triplets (sorted-hit indices)
    uint32_t combo[CC];         // e+ e+ e- combinations (track indices), after the fits
  } u;
  int ntrip, npos, nneg, ncombo, nstore, flag, bad;
  unsigned long long acc[ST_REASON0 + 8];  // statistics of this group's frames
  unsigned long long facc[ST_REASON0];     // statistics of the current frame
};

using SmWarp = FrameSm<W_HITS, W_TRIP, W_TRK, W_COMBO>;
using SmCta = FrameSm<C_HITS, C_TRIP, C_TRK, C_COMBO>;

// ------------------------------------------------------------------ small helpers

// Asynchronous 4-byte copy from global to shared memory (no register holds the
// value), and the wait for all of this thread's copies.
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

template <class T>
__device__ __forceinline__ T make_trip(int i0, int i1, int i2) {  // a triplet of sorted-hit indices
  T t;
  t.x = (decltype(t.x))i0;
  t.y = (decltype(t.y))i1;
  t.z = (decltype(t.z))i2;
  t.w = 0;
  return t;
}

struct Dec {
  int L, g, row, b;
  int ci, ri;  // indices of the hit's column and row in the look-up tables
  bool ok;
};

// A per-layer constant selected by the (data-dependent) layer: selects over the
// four values instead of an indexed load, which the constant cache would serialise
// over the distinct layers of a warp.
template <class T>
__device__ __forceinline__ T by_layer(const T (&v)[4], int L) {
  return L == 0 ? v[0] : (L == 1 ? v[1] : (L == 2 ? v[2] : v[3]));
}
// a 16-bit field of a packed per-layer word
__device__ __forceinline__ int field16(unsigned long long w, int L) { return (int)((w >> (16 * L)) & 0xffffull); }

__device__ __forceinline__ Dec decode(const DevCfg& C, uint32_t a) {
  Dec d;
  d.L = (a >> 26) & 3;
  const int lad = (a >> 21) & 31, col = (a >> 13) & 255;
  d.row = a & 8191;
  d.ok = (a >> 28) == 0 && lad < C.nlad[d.L] && col < C.ncol[d.L] && d.row < C.nrow[d.L];
  d.g = lad * C.ncol[d.L] + col;
  d.ci = C.col_off[d.L] + d.g;
  d.ri = C.row_off[d.L] + d.row;
  // phi bin floor(g NB / ntot) without an integer division: g NB < 2^24 is exact in
  // FP32, and (g NB + 1/2) / ntot lies at least 1/(2 ntot) >= 6e-5 from an integer,
  // far more than the two roundings (< 4e-6 at values below NB)
  d.b = d.ok ? (int)__fmul_rn(__fadd_rn((float)(d.g * NB), 0.5f), C.intot[d.L]) : 0;
  return d;
}

// decode() with the per-layer constants from the 16-byte entries of a table in shared
// memory (DevCfg::ltab): one load per hit, where the constant cache would serialise
// the loads of a warp's several layers.  The same values as decode().
__device__ __forceinline__ Dec decode_s(const uint4* tab, uint32_t a) {
  Dec d;
  d.L = (a >> 26) & 3;
  const uint4 t = tab[d.L];
  const int lad = (a >> 21) & 31, col = (a >> 13) & 255;
  d.row = a & 8191;
  const int nlad = (int)(t.x & 63u), ncol = (int)((t.x >> 6) & 511u), nrow = (int)(t.x >> 15);
  d.ok = (a >> 28) == 0 && lad < nlad && col < ncol && d.row < nrow;
  d.g = lad * ncol + col;
  d.ci = (int)t.y + d.g;
  d.ri = (int)t.z + d.row;
  d.b = d.ok ? (int)__fmul_rn(__fadd_rn((float)(d.g * NB), 0.5f), __uint_as_float(t.w)) : 0;
  return d;
}

// decode without the phi bin and without loads indexed by the hit's layer: the
// per-layer integers come from packed 16-bit fields.  For a kernel that does little
// else per hit (the ingest), where loads of per-layer constants at the warp's
// several layers would serialise in the constant cache and bound the kernel.
__device__ __forceinline__ Dec decode_packed(const DevCfg& C, uint32_t a) {
  Dec d;
  d.L = (a >> 26) & 3;
  const int lad = (a >> 21) & 31, col = (a >> 13) & 255;
  d.row = a & 8191;
  const int nlad = field16(C.pk_nlad, d.L), ncol = field16(C.pk_ncol, d.L);
  d.ok = (a >> 28) == 0 && lad < nlad && col < ncol && d.row < field16(C.pk_nrow, d.L);
  d.g = lad * ncol + col;
  d.ci = field16(C.pk_coloff, d.L) + d.g;
  d.ri = field16(C.pk_rowoff, d.L) + d.row;
  d.b = 0;
  return d;
}

// Azimuth of the centre of global column g of layer L, (g + 1/2) 2 pi / ntot: the
// step 2 pi / ntot is held as a sum of two floats and the product's rounding error
// is recovered by a fused multiply-add, which gives the FP64 value rounded once to
// FP32 for every column of the detector (the look-up table's value, checked
// exhaustively by the tests).
template <bool SEL = false>
__device__ __forceinline__ float column_phi(const DevCfg& C, int L, int g) {
  const float p = (float)g + 0.5f;  // exact: g < 2^23
  const float sh = SEL ? by_layer(C.phs_hi, L) : C.phs_hi[L], sl = SEL ? by_layer(C.phs_lo, L) : C.phs_lo[L];
  const float hi = __fmul_rn(p, sh);
  const float lo = __fmaf_rn(p, sh, -hi);
  return __fadd_rn(hi, __fmaf_rn(p, sl, lo));
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

// sin(x) - x cos(x) for x in (0, pi], given s = sin x and c = cos x.  For small x
// the two terms cancel to x^3/3, so the Taylor series
// sum_k (-1)^(k+1) 2k x^(2k+1) / (2k+1)! is used below 0.5 (five terms:
// truncation below FP32 rounding).
__device__ __forceinline__ float sin_minus_xcos(float x, float s, float c) {
  if (x < 0.5f) {
    const float x2 = x * x;
    float t = 1.f / 3991680.f;
    t = t * x2 - 1.f / 45360.f;
    t = t * x2 + 1.f / 840.f;
    t = t * x2 - 1.f / 30.f;
    t = t * x2 + 1.f / 3.f;
    return t * x2 * x;
  }
  return s - x * c;
}

// ------------------------------------------------------------------ triplet fit

struct SegF {
  float phi, RC, th, dphi, dth, zp;
};

// One segment of the circle solution: chord d, axial length z, transverse radius
// Rct of the circle through the triplet, and the arc angle Phi travelled along the
// segment with sh = sin(Phi/2) and ch = cos(Phi/2).  Helix relations
// d = 2 R_t sin(Phi/2), z = R_t Phi cot(theta), R_t = R sin(theta) give the 3D
// radius R_C, the polar angle theta_C and the derivatives dPhi/dR, dtheta/dR at
// the circle solution.  The divisions share the reciprocals of Phi and of
// sin(Phi/2): dPhi/dR = -R_C / (d^2 cos(Phi/2) / (8 sin^3(Phi/2)) + zp^2 / Phi).
__device__ __forceinline__ SegF segment_core(float d, float z, float Rct, float sh, float ch, float ph) {
  SegF s;
  const float iph = 1.f / ph, ish = 1.f / sh;
  const float zp = z * iph;
  s.RC = sqrtf(Rct * Rct + zp * zp);
  s.th = 0.f;  // the polar angle atan2(Rct, zp) itself: computed where it is needed
  const float ish2 = ish * ish;
  s.dphi = -s.RC / (0.125f * d * d * ch * ish2 * ish + zp * zp * iph);
  const float g = 0.5f * ph * ish;
  const float gp = 0.5f * sin_minus_xcos(0.5f * ph, sh, ch) * ish2;
  const float dg = d * g;
  s.dth = z * d * gp * s.dphi / (z * z + dg * dg);
  s.phi = ph;
  s.zp = zp;
  return s;
}

// The same from the chord alone: sin(Phi/2) = d / 2R_t on either arc (the long arc
// turns by 2 pi minus the short one, which leaves the sine of the half angle and
// flips its cosine); inv2R = 1 / (2 R_t).  Near a half turn (d -> 2 R_t) the arc
// sine loses half the digits of its argument; the triplet fit therefore takes the
// angle from the triangle (fit_triplet), and this form serves the reverse sweep of
// the alignment gradient, which differentiates it.
__device__ __forceinline__ SegF segment(float d, float z, float Rct, float inv2R, bool obtuse) {
  const float sh = fminf(1.f, d * inv2R);
  float ph = 2.f * asinf(sh);
  float ch = sqrtf(fmaxf((1.f - sh) * (1.f + sh), 0.f));
  if (obtuse) {
    ph = TWO_PI_F - ph;
    ch = -ch;
  }
  SegF s = segment_core(d, z, Rct, sh, ch, ph);
  s.th = atan2f(Rct * ph, z);
  return s;
}

struct TFitF {
  float eps, Rct, ccx, ccy;
  float Rref;                  // expansion point of the kink model: R_C of segment 0
  float alpha, a0p, beta, b0p; // Phi_MS ~ alpha u + a0p, Theta_MS ~ beta u + b0p, u = R - Rref
  float s2;                    // sin^2 of the mean polar angle
  float kappa, skappa;
  float zp0, RC0, dth0;         // segment 0: z / Phi (theta_C0 = atan2(Rct, zp0)), R_C, dtheta/dR
  float zp1;                   // z / Phi of segment 1 = R_t cot(theta_C1)
  int valid;
};

// Single triplet fit, hits a -> b -> c, scattering at b (Sec. "Single Triplet
// Fit"): linear kink model around the circle solution and its closed-form
// minimum in the 3D radius.  The model is written in u = R - R_C0 so that the
// small offsets (R_C0 - R_C1, theta_C1 - theta_C0) enter directly instead of as
// differences of large products; the algebra equals the minimum of
// [Phi_MS^2 sin^2(theta) + Theta_MS^2] / sigma_MS^2.  Inlined at both calls of a
// track: as a call, its 18-float result and the caller's live values went through
// local memory.
__device__ __forceinline__ TFitF fit_triplet(float ax, float ay, float az, float bx, float by, float bz, float cx,
                                          float cy, float cz, float hl, float kB) {
  TFitF f;
  f.valid = 0;
  const float ux = ax - bx, uy = ay - by, vx = cx - bx, vy = cy - by;
  const float cross = ux * vy - uy * vx;
  const float u2 = ux * ux + uy * uy, v2 = vx * vx + vy * vy;
  const float wx = cx - ax, wy = cy - ay;
  const float d01 = sqrtf(u2), d12 = sqrtf(v2), d20 = sqrtf(wx * wx + wy * wy);
  if (!(cross != 0.f)) return f;
  const float i2c = 0.5f / cross;
  const float rtc = d01 * d12 * d20 * i2c;
  if (!isfinite(rtc) || rtc == 0.f) return f;
  f.Rct = fabsf(rtc);
  f.eps = rtc > 0.f ? 1.f : -1.f;
  f.ccx = bx + (vy * u2 - uy * v2) * i2c;
  f.ccy = by + (ux * v2 - vx * u2) * i2c;
  // Arc angle of each segment from the triangle: the track's arc from a to b is
  // the one that does not hold c, so it turns by twice the inscribed angle at c,
  // Phi01 = 2 atan2(|cross|, (a - c).(b - c)) (more than pi when that angle is
  // obtuse), and Phi12 likewise by twice the angle at a.  sin(Phi/2) and
  // cos(Phi/2) are that angle's sine and cosine, |cross| / (lengths) and
  // dot / (lengths): full precision up to a half turn and beyond, where the arc
  // sine of d / 2R_t would lose half its digits.
  const float acr = fabsf(cross);
  const float dotc = (ax - cx) * (bx - cx) + (ay - cy) * (by - cy);
  const float dota = (bx - ax) * (cx - ax) + (by - ay) * (cy - ay);
  const float il0 = 1.f / (d20 * d12), il1 = 1.f / (d01 * d20);
  const SegF s0 = segment_core(d01, bz - az, f.Rct, acr * il0, dotc * il0, 2.f * atan2f(acr, dotc));
  const SegF s1 = segment_core(d12, cz - bz, f.Rct, acr * il1, dota * il1, 2.f * atan2f(acr, dota));
  const float dR = s0.RC - s1.RC;
  f.Rref = s0.RC;
  f.alpha = 0.5f * (s0.dphi + s1.dphi);
  f.a0p = 0.5f * s1.dphi * dR;
  f.beta = s1.dth - s0.dth;
  // polar angles from cos = zp / R_C, sin = R_t / R_C of each segment: their difference
  // as one well-conditioned atan2, and sin^2 of their mean from cos(theta0 + theta1)
  // (the common factor 1 / (R_C0 R_C1) drops out of the atan2)
  const float R2 = f.Rct * f.Rct;
  f.b0p = atan2f(f.Rct * (s0.zp - s1.zp), fmaf(s0.zp, s1.zp, R2)) + s1.dth * dR;
  f.s2 = 0.5f * (1.f - (s0.zp * s1.zp - R2) / (s0.RC * s1.RC));
  const float den = f.alpha * f.alpha * f.s2 + f.beta * f.beta;
  const float u = -(f.alpha * f.a0p * f.s2 + f.beta * f.b0p) / den;
  const float Rs = f.Rref + u;
  if (!(Rs > 0.f) || !isfinite(Rs)) return f;
  const float iRs = 1.f / Rs;
  f.kappa = f.eps * iRs;
  f.skappa = hl * iRs * iRs * iRs / (kB * sqrtf(den));  // sigma_MS(p*) / sqrt(den) / R*^2
  if (!isfinite(f.kappa) || !isfinite(f.skappa) || !(f.skappa > 0.f)) return f;
  f.zp0 = s0.zp;
  f.RC0 = s0.RC;
  f.dth0 = s0.dth;
  f.zp1 = s1.zp;
  f.valid = 1;
  return f;
}

// [Phi_MS^2 sin^2(theta) + Theta_MS^2] / sigma_MS^2 of the kink model at R, with
// isg = 1 / sigma_MS.
__device__ __forceinline__ float kink_chi2(const TFitF& f, float R, float isg) {
  const float u = R - f.Rref;
  const float kp = f.alpha * u + f.a0p, kt = f.beta * u + f.b0p;
  return (kp * kp * f.s2 + kt * kt) * (isg * isg);
}

// ------------------------------------------------------------------ hit views

// Hits of one frame, sorted by (layer, phi bin), as build_track reads them: from
// the shared-memory stage of a fused kernel, or from global memory in the staged
// form (pointers already offset to the frame).
// pos(i) = (x, y, z, phi) of sorted hit i.
template <class S>
struct SmHits {
  static constexpr bool kPark = false;
  const S& s;
  __device__ __forceinline__ float4 pos(int i) const { return make_float4(s.x[i], s.y[i], s.z[i], s.phi[i]); }
  __device__ __forceinline__ uint32_t addr(int i) const { return s.addr[i]; }
  __device__ __forceinline__ int l3(int b) const { return s.bstart[3 * NB + b]; }  // layer-3 bin starts
};

// The first triplet fit's values that the global fit and the track record need,
// parked in shared memory across the layer-3 search and the second fit (staged form,
// one slot per thread of a 128-thread CTA): fewer live registers in the track stage.
struct FitPark {
  float v[11][128];
};

__device__ __forceinline__ void park_fit(FitPark& pk, const TFitF& f) {
  volatile float* q = &pk.v[0][threadIdx.x & 127];
  q[0 * 128] = f.skappa;
  q[1 * 128] = f.kappa;
  q[2 * 128] = f.alpha;
  q[3 * 128] = f.a0p;
  q[4 * 128] = f.beta;
  q[5 * 128] = f.b0p;
  q[6 * 128] = f.s2;
  q[7 * 128] = f.Rref;
  q[8 * 128] = f.Rct;
  q[9 * 128] = f.zp0;
  q[10 * 128] = f.dth0;
}

__device__ __forceinline__ TFitF unpark_fit(const FitPark& pk) {
  const volatile float* q = &pk.v[0][threadIdx.x & 127];
  TFitF f;
  f.skappa = q[0 * 128];
  f.kappa = q[1 * 128];
  f.alpha = q[2 * 128];
  f.a0p = q[3 * 128];
  f.beta = q[4 * 128];
  f.b0p = q[5 * 128];
  f.s2 = q[6 * 128];
  f.Rref = q[7 * 128];
  f.Rct = q[8 * 128];
  f.zp0 = q[9 * 128];
  f.dth0 = q[10 * 128];
  f.RC0 = f.Rref;  // R_C of segment 0 is the expansion point
  f.eps = f.ccx = f.ccy = f.zp1 = 0.f;
  f.valid = 1;
  return f;
}

struct GHits {                       // one 16-byte load per hit
  static constexpr bool kPark = true;
  const float4* __restrict__ ps;
  const uint32_t* __restrict__ as;
  const uint16_t* __restrict__ l3s;  // NB + 1 layer-3 bin starts, frame-relative
  FitPark* park;
  __device__ __forceinline__ float4 pos(int i) const { return __ldg(ps + i); }
  __device__ __forceinline__ uint32_t addr(int i) const { return __ldg(as + i); }
  __device__ __forceinline__ int l3(int b) const { return __ldg(l3s + b); }
};

// ------------------------------------------------------------------ track reconstruction

constexpr int SCAN3_MAX = 96;

struct TrackOut {
  int status, i3;
  float kbar, th01, chi2, mbest;
  float Rct, zp0, dth0, RC0;  // of the first triplet's fit: what the track record needs besides kbar
};

// Global fit of a track from its two triplet fits (weighted mean curvature, chi2 of
// both kink models at it, chi2 cut) and what the track record needs.
__device__ __forceinline__ TrackOut global_fit(TrackOut o, const TFitF& f1, const TFitF& f2, const DevCfg& C) {
  const float w1 = 1.f / (f1.skappa * f1.skappa), w2 = 1.f / (f2.skappa * f2.skappa);
  const float kb = (f1.kappa * w1 + f2.kappa * w2) / (w1 + w2);
  o.kbar = kb;
  if (!(kb != 0.f) || !isfinite(kb)) return o;
  const float Rb = 1.f / fabsf(kb);
  const float pb = C.kB * Rb;
  const float chi2 = kink_chi2(f1, Rb, pb * C.ihl[1]) + kink_chi2(f2, Rb, pb * C.ihl[2]);
  o.chi2 = chi2;
  if (!isfinite(chi2)) return o;
  o.status = 4;
  if (!(chi2 < C.chi2_trk)) return o;
  o.status = 5;
  o.th01 = atan2f(f1.Rct, f1.zp0) + f1.dth0 * (Rb - f1.RC0);  // theta01 (candidate record)
  o.Rct = f1.Rct;
  o.zp0 = f1.zp0;
  o.dth0 = f1.dth0;
  o.RC0 = f1.RC0;
  return o;
}

// Algorithm 3 for one selected triplet (sorted-hit indices i0, i1, i2): fit,
// estimate the layer-3 point from the first triplet's circle and the second
// segment's polar angle, take the closest layer-3 hit ((r3 dphi)^2 + dz^2, ties
// to the smaller address), fit (h1, h2, h3), weighted mean curvature and chi2 of
// both triplets at it, chi2 cut.  The caller turns a kept track (status 5) into
// its record with track_record.
//
// Closest hit: a frame with at most SCAN3_MAX layer-3 hits scans them all (the
// loads are independent, so their latencies overlap); a larger one visits them
// by phi bin in rings around the bin of the estimated point.  Every hit of ring m >= 3 lies at least (m - 2) bin widths
// minus one column from the estimated phi (one ring of slack covers a bin index
// rounded across an edge), so once (r3 * that)^2 exceeds the best metric no
// farther hit can win: the search returns the same hit as a scan of all hits.
template <class V>
__device__ __forceinline__ TrackOut build_track(const V& v, const DevCfg& C, int i0, int i1, int i2) {
  TrackOut o;
  o.status = 0;
  o.i3 = -1;
  o.kbar = o.th01 = o.chi2 = o.mbest = 0.f;
  o.Rct = o.zp0 = o.dth0 = o.RC0 = 0.f;
  const float4 p0 = v.pos(i0), p1 = v.pos(i1), p2 = v.pos(i2);
  const float x0 = p0.x, y0 = p0.y, z0 = p0.z;
  const float x1 = p1.x, y1 = p1.y, z1 = p1.z;
  const float x2 = p2.x, y2 = p2.y, z2 = p2.z;
  const TFitF f1 = fit_triplet(x0, y0, z0, x1, y1, z1, x2, y2, z2, C.hl[1], C.kB);
  if (!f1.valid) return o;
  if constexpr (V::kPark) park_fit(*v.park, f1);
  const float r3 = C.r3;
  const float D = sqrtf(f1.ccx * f1.ccx + f1.ccy * f1.ccy);
  o.status = 1;
  if (!(D > 0.f) || D > f1.Rct + r3 || D < fabsf(f1.Rct - r3)) return o;
  const float iD = 1.f / D;
  const float a = (r3 * r3 - (f1.Rct - D) * (f1.Rct + D)) * (0.5f * iD);
  const float hh = sqrtf(fmaxf((r3 - a) * (r3 + a), 0.f));
  const float ux = f1.ccx * iD, uy = f1.ccy * iD;
  const float qx0 = a * ux - hh * uy, qy0 = a * uy + hh * ux;
  const float qx1 = a * ux + hh * uy, qy1 = a * uy - hh * ux;
  // turning angle from h2 to each crossing q in the turning sense: the angle from
  // (h2 - c) to (q - c) is atan2(cross, dot); clockwise turning decreases it.  The
  // crossing reached first is found without the angles: with (dot, -eps cross) as
  // the direction of the turn, a turn of less than a half (-eps cross >= 0) comes
  // before one of more, and within a half the turn of q1 is the smaller one when
  // the direction of q1 lies clockwise of that of q0 (negative 2D cross product).
  // Only the chosen turn is evaluated.
  const float wx = x2 - f1.ccx, wy = y2 - f1.ccy;
  const float vx0 = qx0 - f1.ccx, vy0 = qy0 - f1.ccy, vx1 = qx1 - f1.ccx, vy1 = qy1 - f1.ccy;
  const float cr0 = wx * vy0 - wy * vx0, dt0 = wx * vx0 + wy * vy0;
  const float cr1 = wx * vy1 - wy * vx1, dt1 = wx * vx1 + wy * vy1;
  const float t0 = -f1.eps * cr0, t1 = -f1.eps * cr1;
  const bool lo0 = !(t0 < 0.f), lo1 = !(t1 < 0.f);
  const bool take1 = (lo1 && !lo0) || (lo1 == lo0 && dt0 * t1 - t0 * dt1 < 0.f);
  const float al = wrap_2pi(-f1.eps * atan2f(take1 ? cr1 : cr0, take1 ? dt1 : dt0));
  const float qx = take1 ? qx1 : qx0, qy = take1 ? qy1 : qy0;
  const float z3 = z2 + al * f1.zp1;  // R_t * dPhi * cot(theta_C12)
  float phi3 = atan2f(qy, qx);
  if (phi3 < 0.f) phi3 += TWO_PI_F;
  int b3 = (int)(phi3 * (NB / TWO_PI_F));
  b3 = b3 < 0 ? 0 : (b3 >= NB ? NB - 1 : b3);
  int best = -1;
  float mb = FLT_MAX;
  uint32_t ab = 0;
  // (r3 dphi)^2 + dz^2, rounded in one fixed order wherever it is inlined; dphi is
  // the difference of the azimuths (both in [0, 2 pi)) less the nearest multiple of
  // 2 pi, which one fused multiply-add subtracts exactly as a subtraction of 2 pi
  // would (the two choices at |dphi| = pi give the same metric)
  auto metric = [&](const float4& q) {
    const float d = __fsub_rn(q.w, phi3);
    const float rd = __fmul_rn(r3, __fmaf_rn(-TWO_PI_F, rintf(__fmul_rn(d, 1.f / TWO_PI_F)), d));
    const float dz = __fsub_rn(q.z, z3);
    return __fmaf_rn(rd, rd, __fmul_rn(dz, dz));
  };
  // the full rule: an equal metric goes to the smaller address
  auto visit = [&](int j) {
    const float4 q = v.pos(j);
    const uint32_t aj = v.addr(j);
    const float mm = metric(q);
    if (best < 0 || mm < mb || (mm == mb && aj < ab)) {
      best = j;
      mb = mm;
      ab = aj;
    }
  };
  const int l3a = v.l3(0), l3e = v.l3(NB);
  if (l3e - l3a <= SCAN3_MAX) {
    // few layer-3 hits: a straight scan, whose loads do not depend on each other.
    // It reads no addresses: it notes whether another hit has the same metric as
    // the best so far, and only then (rarely) repeats the scan with the full rule.
    bool tie = false;
    if (l3a < l3e) {
      best = l3a;
      mb = metric(v.pos(l3a));
    }
#pragma unroll 4
    for (int j = l3a + 1; j < l3e; ++j) {
      const float mm = metric(v.pos(j));
      if (mm < mb) {
        best = j;
        mb = mm;
        tie = false;
      } else if (mm == mb) {
        tie = true;
      }
    }
    if (tie) {
      best = -1;
      mb = FLT_MAX;
      for (int j = l3a; j < l3e; ++j) visit(j);
    }
  } else {
    for (int m = 0; m <= NB / 2; ++m) {
      if (m >= 3) {
        const float dmin = (float)(m - 2) * (TWO_PI_F / NB) - C.colw3;
        if (dmin > 0.f && (r3 * dmin) * (r3 * dmin) > mb) break;
      }
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        if (side == 1 && (m == 0 || m == NB / 2)) continue;
        const int bb = (b3 + (side ? -m : m)) & (NB - 1);
        const int e = v.l3(bb + 1);
        for (int j = v.l3(bb); j < e; ++j) visit(j);
      }
    }
  }
  o.status = 2;
  if (best < 0) return o;
  o.i3 = best;
  o.mbest = mb;
  const float4 p3 = v.pos(best);
  const TFitF f2 = fit_triplet(x1, y1, z1, x2, y2, z2, p3.x, p3.y, p3.z, C.hl[2], C.kB);
  o.status = 3;
  if (!f2.valid) return o;
  if constexpr (V::kPark) return global_fit(o, unpark_fit(*v.park), f2, C);
  else return global_fit(o, f1, f2, C);
}


// Record of a kept track for the vertex stage (layout below), from the layer-0 and
// layer-1 hits p0, p1 and the reconstruction o: transverse circle of radius
// R sin(theta01) through the two hits, centre on the side the track turns to.
// theta01 = theta_C0 + dtheta/dR (R - R_C0) enters through its cosine and sine,
// the rotation of (cos, sin) theta_C0 = (zp0, R_t) / R_C0 by the small correction.
__device__ __forceinline__ void track_record(const float4& p0, const float4& p1, const TrackOut& o, const DevCfg& C,
                                             float* tr) {
  const float x0 = p0.x, y0 = p0.y, x1 = p1.x, y1 = p1.y;
  const float Rb = 1.f / fabsf(o.kbar);
  const float pb = C.kB * Rb;
  float sd, cd;
  __sincosf(o.dth0 * (Rb - o.RC0), &sd, &cd);
  const float iRC = 1.f / o.RC0;
  const float ct = (o.zp0 * cd - o.Rct * sd) * iRC, st = (o.Rct * cd + o.zp0 * sd) * iRC;
  const float eps = o.kbar > 0.f ? 1.f : -1.f;
  const float rt = Rb * st;
  const float dx = x1 - x0, dy = y1 - y0;
  const float d = sqrtf(dx * dx + dy * dy);
  const float ex = dx / d, ey = dy / d;
  const float hd = 0.5f * d;
  const float off = sqrtf(fmaxf((rt - hd) * (rt + hd), 0.f));
  const float cx = 0.5f * (x0 + x1) + eps * ey * off;
  const float cy = 0.5f * (y0 + y1) - eps * ex * off;
  tr[0] = cx;
  tr[1] = cy;
  tr[2] = rt;
  tr[3] = Rb;
  tr[4] = ct;
  tr[5] = st;
  tr[6] = pb;
  tr[7] = sqrtf(pb * pb + C.me2);
  tr[8] = C.hl[0] / pb;
  tr[9] = x0;
  tr[10] = y0;
  tr[11] = p0.z;
  tr[12] = atan2f(y0 - cy, x0 - cx);
  tr[13] = eps;
}

// Track record layout (16 floats, also the global record of the staged form):
// cx cy rt R ct st p E sms h0x h0y h0z ah0 eps - -
template <int CK>
__device__ __forceinline__ void store_track(TrkSoA<CK>& T, int k, const float* tr, int tid) {
  T.cx[k] = tr[0];
  T.cy[k] = tr[1];
  T.rt[k] = tr[2];
  T.R[k] = tr[3];
  T.ct[k] = tr[4];
  T.st[k] = tr[5];
  T.p[k] = tr[6];
  T.E[k] = tr[7];
  T.sms[k] = tr[8];
  T.h0x[k] = tr[9];
  T.h0y[k] = tr[10];
  T.h0z[k] = tr[11];
  T.ah0[k] = tr[12];
  T.eps[k] = tr[13];
  T.tid[k] = tid;
}

// ------------------------------------------------------------------ vertex

struct TrackR {  // one kept track in registers (record layout above)
  float cx, cy, rt, R, ct, st, p, E, sms, h0x, h0y, h0z, ah0, eps;
};

template <int CK>
__device__ __forceinline__ TrackR load_track(const TrkSoA<CK>& T, int k) {
  TrackR t;
  t.cx = T.cx[k]; t.cy = T.cy[k]; t.rt = T.rt[k]; t.R = T.R[k]; t.ct = T.ct[k]; t.st = T.st[k];
  t.p = T.p[k]; t.E = T.E[k]; t.sms = T.sms[k]; t.h0x = T.h0x[k]; t.h0y = T.h0y[k]; t.h0z = T.h0z[k];
  t.ah0 = T.ah0[k]; t.eps = T.eps[k];
  return t;
}

__device__ __forceinline__ TrackR load_track(const float4* __restrict__ rec, int64_t k) {
  const float4 a = __ldg(rec + 4 * k), b = __ldg(rec + 4 * k + 1), c = __ldg(rec + 4 * k + 2),
               d = __ldg(rec + 4 * k + 3);
  TrackR t;
  t.cx = a.x; t.cy = a.y; t.rt = a.z; t.R = a.w;
  t.ct = b.x; t.st = b.y; t.p = b.z; t.E = b.w;
  t.sms = c.x; t.h0x = c.y; t.h0y = c.z; t.h0z = c.w;
  t.ah0 = d.x; t.eps = d.y;
  return t;
}

// Turning angle travelled from point (x, y) forward to the track's layer-0 hit.
__device__ __forceinline__ float arc_to_h0(const TrackR& t, float x, float y) {
  return wrap_2pi(t.eps * (atan2f(y - t.cy, x - t.cx) - t.ah0));
}

__device__ __forceinline__ float point_var(const TrackR& t, float x, float y, float sp2) {
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

// Longitudinal momentum sum of a combination (the z part of |sum p|, Sec. "Vertex
// Fit"), rounded in one fixed order, so that the vertex and the early test below
// see the same value.  It does not depend on the vertex position.
__device__ __forceinline__ float pz_track(float p, float ct) { return __fmul_rn(p, ct); }
__device__ __forceinline__ float pz_sum(float pa, float pb, float pe) { return __fadd_rn(__fadd_rn(pa, pb), pe); }

// |sum p| >= |P_z|: the vertex's sum of squares only adds non-negative terms and
// rounding is monotone, so its |sum p| is at least sqrt(fl(P_z^2)).  When P_z^2
// exceeds the squared momentum cut by a relative 1e-4 (far more than any rounding
// of the cut or the square root), the combination fails the cut whatever its
// vertex, and the decision-only runs skip its vertex.  Runs that report each
// combination's status (debug records, statistics) still fit it.
__device__ __forceinline__ bool pz_fails_ptot(float Pz, float ptot_max) {
  return __fmul_rn(Pz, Pz) > ptot_max * ptot_max * 1.0001f;
}

struct VtxOut {
  int status, pass;
  float chi2, tdist, ptot;
  float chi2_second;  // second-smallest chi2 over the choices (candidate record only)
};

// Whether the transverse circles (centre, radius) of two tracks intersect, with
// the distance D of the centres, the foot aa of the chord on the centre line and
// the squared half chord h2.
__device__ __forceinline__ bool circles_meet(float acx, float acy, float ar, float bcx, float bcy, float br, float& D,
                                             float& aa, float& h2) {
  const float ex = bcx - acx, ey = bcy - acy;
  D = sqrtf(ex * ex + ey * ey);
  if (!(D > 0.f)) return false;
  aa = ((ar - br) * (ar + br) + D * D) / (2.f * D);
  h2 = (ar - aa) * (ar + aa);
  return !(h2 < 0.f);
}

// Intersection points of the circles of tracks a and b, in two fixed slots (q0
// first, as the oracle orders them), each with its target-filter flag.  Returns
// false when the circles do not intersect.  One routine for the prefilter of the
// vertex stage and for the vertex itself, so both take the same decisions.
__device__ __forceinline__ bool pair_geometry(float acx, float acy, float ar, float bcx, float bcy, float br,
                                              float lim, float& x0, float& y0, bool& k0, float& x1, float& y1,
                                              bool& k1) {
  k0 = k1 = false;
  float D, aa, h2;
  if (!circles_meet(acx, acy, ar, bcx, bcy, br, D, aa, h2)) return false;
  const float ex = (bcx - acx) / D, ey = (bcy - acy) / D;
  const float bx = acx + aa * ex, by = acy + aa * ey;
  const float h = sqrtf(h2);
  x0 = bx - h * ey;
  y0 = by + h * ex;
  x1 = bx + h * ey;
  y1 = by - h * ex;
  k0 = sqrtf(x0 * x0 + y0 * y0) <= lim;
  k1 = h2 != 0.f && sqrtf(x1 * x1 + y1 * y1) <= lim;
  return true;
}

// The quantities that decide the geometric steps of the vertex, over all three
// pairs whatever the status (candidate record only, for the boundary bands of a
// parity check): the smallest squared half chord relative to the product of the
// two radii, and the smallest distance of an intersection point from the filter
// radius.  Symmetric in the tracks, so independent of their order.
__device__ __forceinline__ void vertex_soft(const TrackR& A, const TrackR& B, const TrackR& E, float lim, float& disc,
                                            float& margin) {
  disc = margin = FLT_MAX;
  const TrackR* V[3] = {&A, &B, &E};
#pragma unroll 1
  for (int k = 0; k < 3; ++k) {
    const TrackR& a = *V[k == 2 ? 1 : 0];
    const TrackR& b = *V[k == 0 ? 1 : 2];
    float D, aa, h2;
    const bool meet = circles_meet(a.cx, a.cy, a.rt, b.cx, b.cy, b.rt, D, aa, h2);
    if (!(D > 0.f)) continue;
    disc = fminf(disc, fabsf(h2) / (a.rt * b.rt));
    if (!meet) continue;
    float x0, y0, x1, y1;
    bool k0, k1;
    pair_geometry(a.cx, a.cy, a.rt, b.cx, b.cy, b.rt, lim, x0, y0, k0, x1, y1, k1);
    margin = fminf(margin, fabsf(sqrtf(x0 * x0 + y0 * y0) - lim));
    if (h2 != 0.f) margin = fminf(margin, fabsf(sqrtf(x1 * x1 + y1 * y1) - lim));
  }
}

// Status of a combination after the first two vertex steps: 0 a pair of circles
// does not intersect, 1 the target filter leaves a pair without points, 2 go on.
__device__ __forceinline__ int vertex_prefilter(const float* a, const float* b, const float* e, float lim) {
  float x0, y0, x1, y1;
  bool k0, k1, k2, k3, k4, k5;
  if (!pair_geometry(a[0], a[1], a[2], b[0], b[1], b[2], lim, x0, y0, k0, x1, y1, k1)) return 0;
  if (!pair_geometry(a[0], a[1], a[2], e[0], e[1], e[2], lim, x0, y0, k2, x1, y1, k3)) return 0;
  if (!pair_geometry(b[0], b[1], b[2], e[0], e[1], e[2], lim, x0, y0, k4, x1, y1, k5)) return 0;
  return (k0 || k1) && (k2 || k3) && (k4 || k5) ? 2 : 1;
}

// pair_geometry plus the error of each surviving point (sum of both tracks' errors).
__device__ __forceinline__ int pair_points(const TrackR& a, const TrackR& b, const DevCfg& C, float& x0, float& y0,
                                           float& v0, bool& k0, float& x1, float& y1, float& v1, bool& k1) {
  v0 = v1 = 1.f;
  if (!pair_geometry(a.cx, a.cy, a.rt, b.cx, b.cy, b.rt, C.isect_lim, x0, y0, k0, x1, y1, k1)) return 0;
  if (k0) v0 = point_var(a, x0, y0, C.sig_pix2) + point_var(b, x0, y0, C.sig_pix2);
  if (k1) v1 = point_var(a, x1, y1, C.sig_pix2) + point_var(b, x1, y1, C.sig_pix2);
  return 1;
}

// Closest point of track t to (mx, my), its z on the helix and its error.  The
// closest point lies on the ray from the centre through (mx, my), so its angle
// seen from the centre is that of (mx - cx, my - cy).
__device__ __forceinline__ void closest(const TrackR& t, float mx, float my, float sp2, float& px, float& py,
                                        float& z, float& var, bool& bad) {
  const float dx = mx - t.cx, dy = my - t.cy;
  const float dn = sqrtf(dx * dx + dy * dy);
  if (!(dn > 0.f)) bad = true;
  const float sc = t.rt / dn;
  px = t.cx + sc * dx;
  py = t.cy + sc * dy;
  const float dphi = wrap_2pi(t.eps * (atan2f(dy, dx) - t.ah0));
  z = t.h0z - dphi * t.R * t.ct;
  const float s = t.rt * dphi;
  var = t.sms * t.sms * s * s + sp2;
}

// Vertex of one e+ e+ e- combination (Sec. "Vertex Fit", "Signal Estimation"):
// pairwise circle intersections, target-disk filter, error-weighted transverse
// mean for each choice of one point per pair, closest points, z projection, chi2;
// the smallest-chi2 choice is cut on chi2, target distance and |sum p|.  The loop
// over the (at most 8) choices stays rolled: its body is large, and one copy keeps
// the kernel's instruction footprint small.
__device__ __forceinline__ VtxOut vertex(const TrackR& A, const TrackR& B, const TrackR& E, const DevCfg& C) {
  VtxOut o;
  o.status = 0;
  o.pass = 0;
  o.chi2 = o.tdist = o.ptot = FLT_MAX;
  o.chi2_second = FLT_MAX;
  float x00, y00, v00, x01, y01, v01, x10, y10, v10, x11, y11, v11, x20, y20, v20, x21, y21, v21;
  bool k00, k01, k10, k11, k20, k21;
  if (!pair_points(A, B, C, x00, y00, v00, k00, x01, y01, v01, k01)) return o;
  if (!pair_points(A, E, C, x10, y10, v10, k10, x11, y11, v11, k11)) return o;
  if (!pair_points(B, E, C, x20, y20, v20, k20, x21, y21, v21, k21)) return o;
  o.status = 1;
  if (!(k00 || k01) || !(k10 || k11) || !(k20 || k21)) return o;
  float best = FLT_MAX, bmx = 0.f, bmy = 0.f, bmz = 0.f;
  bool have = false;
  // the valid choices as a bit set, visited in increasing order (s2 fastest, as the
  // oracle's loops), so each lane runs only its own choices
  unsigned valid = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const bool s0 = (c >> 2) & 1, s1 = (c >> 1) & 1, s2 = c & 1;
    if ((s0 ? k01 : k00) && (s1 ? k11 : k10) && (s2 ? k21 : k20)) valid |= 1u << c;
  }
#pragma unroll 1
  while (valid) {
    const int c = __ffs(valid) - 1;
    valid &= valid - 1;
    const bool s0 = (c >> 2) & 1, s1 = (c >> 1) & 1, s2 = c & 1;
    const float w0 = 1.f / (s0 ? v01 : v00), w1 = 1.f / (s1 ? v11 : v10), w2 = 1.f / (s2 ? v21 : v20);
    const float iws = 1.f / (w0 + w1 + w2);
    const float mx = ((s0 ? x01 : x00) * w0 + (s1 ? x11 : x10) * w1 + (s2 ? x21 : x20) * w2) * iws;
    const float my = ((s0 ? y01 : y00) * w0 + (s1 ? y11 : y10) * w1 + (s2 ? y21 : y20) * w2) * iws;
    float pa, qa, za, va, pb, qb, zb, vb, pe, qe, ze, ve;
    bool bad = false;
    closest(A, mx, my, C.sig_pix2, pa, qa, za, va, bad);
    closest(B, mx, my, C.sig_pix2, pb, qb, zb, vb, bad);
    closest(E, mx, my, C.sig_pix2, pe, qe, ze, ve, bad);
    if (bad) continue;
    const float ia = 1.f / va, ib = 1.f / vb, ie = 1.f / ve;
    const float mz = (za * ia + zb * ib + ze * ie) / (ia + ib + ie);
    const float chi2 = ((pa - mx) * (pa - mx) + (qa - my) * (qa - my) + (za - mz) * (za - mz)) * ia +
                       ((pb - mx) * (pb - mx) + (qb - my) * (qb - my) + (zb - mz) * (zb - mz)) * ib +
                       ((pe - mx) * (pe - mx) + (qe - my) * (qe - my) + (ze - mz) * (ze - mz)) * ie;
    if (!have || chi2 < best) {
      if (have) o.chi2_second = best;
      have = true;
      best = chi2;
      bmx = mx;
      bmy = my;
      bmz = mz;
    } else if (chi2 < o.chi2_second) {
      o.chi2_second = chi2;
    }
  }
  if (!have || !isfinite(best)) return o;
  o.status = 2;
  o.chi2 = best;
  o.tdist = target_distance(C, bmx, bmy, bmz);
  float Px = 0.f, Py = 0.f;
  const TrackR* V[3] = {&A, &B, &E};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const TrackR& t = *V[i];
    const float dx = bmx - t.cx, dy = bmy - t.cy;
    const float idn = 1.f / sqrtf(dx * dx + dy * dy);
    const float ux = dx * idn, uy = dy * idn;  // direction of the closest point from the centre
    const float pt = t.p * t.st;
    Px += pt * t.eps * uy;
    Py -= pt * t.eps * ux;
  }
  const float Pz = pz_sum(pz_track(A.p, A.ct), pz_track(B.p, B.ct), pz_track(E.p, E.ct));
  o.ptot = sqrtf(Px * Px + Py * Py + Pz * Pz);
  o.pass = o.chi2 <= C.vtx_chi2 && o.tdist <= C.tgt_dist && o.ptot <= C.ptot_max;
  return o;
}

// ------------------------------------------------------------------ one frame


// The exact cut tests, written with explicitly rounded operations so that every
// stage and tier takes the same decision whatever the compiler contracts:
// Phi cut between two hits: h_a . h_b >= cos(phi_max) r_a r_b.
__device__ __forceinline__ bool phi_pass(float xa, float ya, float xb, float yb, float c) {
  return fmaf(xa, xb, __fmul_rn(ya, yb)) >= c;
}
// Delta lambda: |tan(lambda12) - tan(lambda01)| <= dl_max, with tan(lambda01) given.
__device__ __forceinline__ bool dl_pass(float z1, float z2, float tl01, const DevCfg& C) {
  return fabsf(fmaf(__fsub_rn(z2, z1), C.inv_dr12, -tl01)) <= C.dl_max;
}
__device__ __forceinline__ float tan_l01(float z0, float z1, const DevCfg& C) {
  return __fmul_rn(__fsub_rn(z1, z0), C.inv_dr01);
}
// r_tc window without division or root: (d01 d12 d20)^2 against (2 r cross)^2.
__device__ __forceinline__ bool rtc_pass(float x0, float y0, float x1, float y1, float x2, float y2,
                                         const DevCfg& C) {
  const float ax = __fsub_rn(x0, x1), ay = __fsub_rn(y0, y1), bx = __fsub_rn(x2, x1), by = __fsub_rn(y2, y1);
  const float cr = fmaf(ax, by, -__fmul_rn(ay, bx));
  const float ex = __fsub_rn(x2, x0), ey = __fsub_rn(y2, y0);
  const float Pq = __fmul_rn(__fmul_rn(fmaf(ax, ax, __fmul_rn(ay, ay)), fmaf(bx, bx, __fmul_rn(by, by))),
                             fmaf(ex, ex, __fmul_rn(ey, ey)));
  const float Qq = __fmul_rn(cr, cr);
  return cr != 0.f && Pq >= __fmul_rn(C.rtc_lo2, Qq) && Pq <= __fmul_rn(C.rtc_hi2, Qq);
}
// z bin of a layer-2 point in the warp stage: monotone in z, so every hit with z in
// [zlo, zhi] lies in bins zbin(zlo) .. zbin(zhi).
__device__ __forceinline__ int zbin2(float z, const DevCfg& C) {
  const int b = (int)__fmul_rn(__fadd_rn(z, C.zoff2), C.izw2);
  return b < 0 ? 0 : (b > NZB - 1 ? NZB - 1 : b);
}

// The phi bin of sorted layer-1 hit i: the last bin whose start is at most i (bins
// are in order; an empty bin shares its start with the next one).
__device__ __forceinline__ int layer1_bin(const uint16_t* bstart, int i) {
  int lo = 0, hi = NB - 1;
#pragma unroll
  for (int step = 0; step < 5; ++step) {  // NB = 32
    const int mid = (lo + hi + 1) >> 1;
    if ((int)bstart[NB + mid] <= i) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Add one hit to bucket key; returns the bucket's count (cursor) before it.  With
// packed cursors a bucket is one byte of a word: counts and starts stay below the
// 256 hits such a frame can hold, so no byte carries into the next.
template <class S>
__device__ __forceinline__ int bucket_add(S& sm, int key) {
  if constexpr (S::kPackB) {
    const int sh = 8 * (key & 3);
    return (int)((atomicAdd(&sm.bcur[key >> 2], 1u << sh) >> sh) & 255u);
  } else {
    return (int)atomicAdd(&sm.bcur[key], 1u);
  }
}

// Exclusive prefix of the bucket counts: bucket starts into bstart and, as the
// placement cursors, back into bcur.
template <class G, class S>
__device__ __forceinline__ void bucket_scan(const G& g, S& sm) {
  static_assert(NBK == 4 * 32, "one word of four packed buckets per lane");
  if (g.rank() < 32) {
    const int lane = g.rank();
    int v[NBK / 32];
    int s = 0;
#pragma unroll
    for (int k = 0; k < NBK / 32; ++k) {
      if constexpr (S::kPackB) v[k] = (int)((sm.bcur[lane] >> (8 * k)) & 255u);
      else v[k] = (int)sm.bcur[lane * (NBK / 32) + k];
      s += v[k];
    }
    int inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(FULL, inc, o);
      if (lane >= o) inc += t;
    }
    int ex = inc - s;
    uint32_t w = 0;
#pragma unroll
    for (int k = 0; k < NBK / 32; ++k) {
      sm.bstart[lane * (NBK / 32) + k] = (uint16_t)ex;
      if constexpr (S::kPackB) w |= (uint32_t)ex << (8 * k);
      else sm.bcur[lane * (NBK / 32) + k] = (uint32_t)ex;
      ex += v[k];
    }
    if constexpr (S::kPackB) sm.bcur[lane] = w;
    if (lane == 31) sm.bstart[NBK] = (uint16_t)inc;
  }
  g.sync();
}

// Selection cuts of a warp-stage frame (Algorithm 2), on the hits sorted by (layer,
// phi bin).  The layer-2 hits are also put in z-bin order (x, y, z and index packed
// in one record), so that for a (layer-1 hit, Phi01 partner) pair the Delta lambda
// cut, seen as a z window on the layer-2 hit, becomes a contiguous range of that
// order.  Per chunk of 32 layer-1 hits (a lane each):
//   1. the Phi01 partners as a bit mask over the layer-0 hits and the Phi12
//      partners as a bit mask over the z-ordered layer-2 hits, from passes over
//      those hits that all lanes take together (one broadcast load per hit);
//   2. the pairs of layer-1 hits that have Phi12 partners, numbered by a prefix sum
//      and listed with their layer-0 hit;
//   3. the pairs, 32 at a time: each lane finds its pair's layer-1 hit (a search
//      over the lanes' prefix), forms the z window (widened by 1e-3 mm against
//      rounding) and its bin range, and keeps the Phi12 partners inside it: the
//      candidate triplets, numbered by a prefix sum and listed;
//   4. the candidates, 32 at a time, through the exact Delta lambda and r_tc tests,
//      the survivors appended in a fixed order by ballot.
// The exact tests are the expressions every other stage uses (phi_pass, dl_pass,
// rtc_pass), and the z window contains every hit that passes Delta lambda, so the
// selected set equals the brute-force one.  sm.bad = 2 when a capacity is exceeded
// (the frame goes to a larger stage).  npair / ntt: this lane's share of the pair
// tests within the reachable phi bins (counted, with stats, as the other stages
// count them) and of the candidate triplets (Phi01 partners times Phi12 partners).
template <class S, int CT>
__device__ __forceinline__ void warp_cuts(S& sm, const DevCfg& C, bool stats, unsigned& npair, unsigned& ntt) {
  const int lane = threadIdx.x & 31;
  const int n0 = sm.bstart[NB], l1a = n0, l1b = sm.bstart[2 * NB], l2b = sm.bstart[3 * NB];
  const int n1 = l1b - l1a, n2 = l2b - l1b;
  bool over = n0 > W_L0 || n2 > W_L2;
  int nt = 0;
  if (!over) {
    // layer-2 hits in z-bin order: counting sort with byte counters packed four to a
    // word (in the candidate buffer, free until step 3), two hits per lane
    uint32_t* zc = reinterpret_cast<uint32_t*>(sm.cand);
    if (lane < NZB / 4) zc[lane] = 0u;
    __syncwarp();
    const int bq0 = lane < n2 ? zbin2(sm.z[l1b + lane], C) : -1;
    const int bq1 = lane + 32 < n2 ? zbin2(sm.z[l1b + lane + 32], C) : -1;
    if (bq0 >= 0) atomicAdd(&zc[bq0 >> 2], 1u << (8 * (bq0 & 3)));
    if (bq1 >= 0) atomicAdd(&zc[bq1 >> 2], 1u << (8 * (bq1 & 3)));
    __syncwarp();
    const uint32_t w = zc[lane >> 1];  // bins 2 lane, 2 lane + 1
    const int ca = (int)((w >> (16 * (lane & 1))) & 255u), cb = (int)((w >> (16 * (lane & 1) + 8)) & 255u);
    int inc = ca + cb;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(FULL, inc, o);
      if (lane >= o) inc += t;
    }
    const int ex = inc - ca - cb;
    sm.zbs[2 * lane] = (uint8_t)ex;
    sm.zbs[2 * lane + 1] = (uint8_t)(ex + ca);
    if (lane == 31) sm.zbs[NZB] = (uint8_t)inc;
    __syncwarp();
    if (lane < NZB / 4) {
      uint32_t cw = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) cw |= (uint32_t)sm.zbs[4 * lane + k] << (8 * k);
      zc[lane] = cw;  // placement cursors
    }
    __syncwarp();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int bq = h ? bq1 : bq0;
      if (bq >= 0) {
        const int i2 = l1b + lane + 32 * h;
        const int pos = (int)((atomicAdd(&zc[bq >> 2], 1u << (8 * (bq & 3))) >> (8 * (bq & 3))) & 255u);
        sm.zq[pos] = make_float4(sm.x[i2], sm.y[i2], sm.z[i2], __int_as_float(i2));
      }
    }
    __syncwarp();
  }
  for (int j0 = 0; j0 < n1 && !over; j0 += 32) {
    const int j = j0 + lane;
    const bool has = j < n1;
    const int i1 = l1a + j;
    float x1 = 0.f, y1 = 0.f, z1 = 0.f;
    if (has) {
      x1 = sm.x[i1];
      y1 = sm.y[i1];
      z1 = sm.z[i1];
      if (stats) {  // the pair tests within the reachable phi bins, as the other stages count them
        const int nb0 = min(2 * C.k01 + 1, NB), nb2 = min(2 * C.k12 + 1, NB);
        const int b1 = layer1_bin(sm.bstart, i1);
        const int s0 = nb0 == NB ? 0 : (b1 - C.k01 + NB) & (NB - 1);
        const int s2 = nb2 == NB ? 0 : (b1 - C.k12 + NB) & (NB - 1);
        npair += sm.bstart[min(s0 + nb0, NB)] - sm.bstart[s0] + (s0 + nb0 > NB ? sm.bstart[s0 + nb0 - NB] : 0);
        npair += sm.bstart[2 * NB + min(s2 + nb2, NB)] - sm.bstart[2 * NB + s2] +
                 (s2 + nb2 > NB ? sm.bstart[2 * NB + s2 + nb2 - NB] - sm.bstart[2 * NB] : 0);
      }
    }
    // 1. Phi01 and Phi12 partners as bit masks (lanes without a layer-1 hit test
    // (0, 0), which passes neither cut)
    uint32_t a0 = 0u, a1 = 0u, b0 = 0u, b1 = 0u;
    const int n0a = min(n0, 32), n2a = min(n2, 32);
    for (int q = 0; q < n0a; ++q)
      if (phi_pass(sm.x[q], sm.y[q], x1, y1, C.c01)) a0 |= 1u << q;
    for (int q = 32; q < n0; ++q)
      if (phi_pass(sm.x[q], sm.y[q], x1, y1, C.c01)) a1 |= 1u << (q - 32);
    for (int q = 0; q < n2a; ++q) {
      const float4 h = sm.zq[q];
      if (phi_pass(x1, y1, h.x, h.y, C.c12)) b0 |= 1u << q;
    }
    for (int q = 32; q < n2; ++q) {
      const float4 h = sm.zq[q];
      if (phi_pass(x1, y1, h.x, h.y, C.c12)) b1 |= 1u << (q - 32);
    }
    const int c01 = __popc(a0) + __popc(a1), c12all = __popc(b0) + __popc(b1);
    ntt += (unsigned)(c01 * c12all);
    // 2. the pairs whose layer-1 hit has Phi12 partners, listed by their layer-0 hit
    const int pc = c12all ? c01 : 0;
    int pe = pc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(FULL, pe, o);
      if (lane >= o) pe += t;
    }
    const int pre = pe - pc;
    const int T = __shfl_sync(FULL, pe, 31);
    if (T > W_P01) {
      over = true;
      break;
    }
    if (pc) {
      int wpos = pre;
      for (uint32_t m = a0; m; m &= m - 1u) sm.p01[wpos++] = (uint8_t)(__ffs(m) - 1);
      for (uint32_t m = a1; m; m &= m - 1u) sm.p01[wpos++] = (uint8_t)(__ffs(m) + 31);
    }
    __syncwarp();
    // 3. the pairs, 32 at a time
    for (int k0 = 0; k0 < T; k0 += 32) {
      const int k = k0 + lane;
      int ow = 0;  // the last lane whose pairs start at or before k
#pragma unroll
      for (int st = 16; st; st >>= 1) {
        const int pv = __shfl_sync(FULL, pre, ow + st);
        if (pv <= k) ow += st;
      }
      const float px1 = __shfl_sync(FULL, x1, ow), py1 = __shfl_sync(FULL, y1, ow), pz1 = __shfl_sync(FULL, z1, ow);
      const uint32_t pml = __shfl_sync(FULL, b0, ow), pmh = __shfl_sync(FULL, b1, ow);
      int i0 = 0;
      float x0 = 0.f, y0 = 0.f, tl01 = 0.f;
      unsigned long long cm = 0ull;
      if (k < T) {
        i0 = sm.p01[k];
        x0 = sm.x[i0];
        y0 = sm.y[i0];
        tl01 = tan_l01(sm.z[i0], pz1, C);
        const float zlo = pz1 + (tl01 - C.dl_max) * C.dr12 - 1e-3f;
        const float zhi = pz1 + (tl01 + C.dl_max) * C.dr12 + 1e-3f;
        const int lo = sm.zbs[zbin2(zlo, C)], hi = sm.zbs[zbin2(zhi, C) + 1];
        const unsigned long long below_hi = hi >= 64 ? ~0ull : (1ull << hi) - 1ull;
        const unsigned long long below_lo = lo >= 64 ? ~0ull : (1ull << lo) - 1ull;
        cm = (below_hi & ~below_lo) & (((unsigned long long)pmh << 32) | pml);
      }
      const int tri01 = i0 | ((l1a + j0 + ow) << 8);  // the pair's layer-0 and layer-1 sorted indices
      const int cnt = __popcll(cm);
      int ce = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(FULL, ce, o);
        if (lane >= o) ce += t;
      }
      const int cpre = ce - cnt, ctot = __shfl_sync(FULL, ce, 31);
      for (int c0 = 0; c0 < ctot; c0 += W_CAND) {
        // each lane lists its candidates numbered c0 .. c0 + W_CAND - 1: pair lane, z-order position
        unsigned long long m = cm;
        for (int idx = cpre; m; ++idx) {
          const int q = __ffsll((long long)m) - 1;
          m &= m - 1ull;
          if (idx >= c0 && idx < c0 + W_CAND) sm.cand[idx - c0] = (uint16_t)((lane << 6) | q);
        }
        __syncwarp();
        // 4. the exact tests, 32 candidates at a time
        const int ne = min(ctot - c0, W_CAND);
        for (int e0 = 0; e0 < ne; e0 += 32) {
          const int e = e0 + lane;
          const int ent = e < ne ? sm.cand[e] : 0;
          const int pl = ent >> 6;
          const float cx0 = __shfl_sync(FULL, x0, pl), cy0 = __shfl_sync(FULL, y0, pl);
          const float cx1 = __shfl_sync(FULL, px1, pl), cy1 = __shfl_sync(FULL, py1, pl);
          const float cz1 = __shfl_sync(FULL, pz1, pl), ctl = __shfl_sync(FULL, tl01, pl);
          const int ct = __shfl_sync(FULL, tri01, pl);
          const float4 h = sm.zq[ent & 63];
          const bool pass = e < ne && dl_pass(cz1, h.z, ctl, C) && rtc_pass(cx0, cy0, cx1, cy1, h.x, h.y, C);
          const unsigned bm = __ballot_sync(FULL, pass);
          const int kk = nt + __popc(bm & ((1u << lane) - 1u));
          if (pass && kk < CT) sm.u.trip[kk] = make_trip<typename S::TripT>(ct & 255, ct >> 8, __float_as_int(h.w));
          nt += __popc(bm);
        }
        __syncwarp();
        if (nt > C.max_trip) break;  // the frame overflows: its decision is known
      }
      if (nt > C.max_trip) break;
    }
    if (nt > C.max_trip) break;
  }
  if (over) npair = ntt = 0;  // the frame is counted by the stage that takes it over
  if (lane == 0) {
    sm.ntrip = nt;
    sm.bad = over ? 2 : 0;
  }
  __syncwarp();
}

constexpr int PENDING = -2;  // frame_front result: triplets selected, later stages to run

// Stages A-C of one frame (load, sort, selection cuts).  Returns a final reason,
// DEFERRED (frame too large for this stage), or PENDING with the selected
// triplets in sm.u.trip and their count in sm.ntrip.
// LIVE: the hits sit in a ring that the host rewrites while the kernel runs
// (streaming), so they are read with loads that bypass the caches instead of
// the read-only path.
// prefetch_next: the group takes frame f + 1 next; its addresses are fetched into
// L1 while this frame is processed.
// NOST: compiled for runs without statistics (P.stats is null).  TAB: the warp stage
// decodes with the per-layer constants from a shared-memory table (decode_s) instead of
// the constant cache (the staged form's stage 1 measured faster so, the fused kernels
// slower).
template <class G, class S, int CH, int CT, bool DEFER, bool DEBUG, bool LIVE = false, bool NOST = false,
          bool TAB = false>
__device__ int frame_front(const G& g, S& sm, const DevCfg& C, const KParams& P, int f, bool prefetch_next = false) {
  const bool stats = !NOST && P.stats != nullptr;
  const int64_t base = P.off[f] - P.off_base;
  const int64_t n64 = P.off[f + 1] - P.off[f];
  if constexpr (G::N == 32 && !LIVE) {
    if (prefetch_next) {
      const int64_t nb = P.off[f + 1] - P.off_base, ne = P.off[f + 2] - P.off_base;
      const int64_t a = nb + 32 * g.rank();
      if (g.rank() < 8 && a < ne) prefetch_l1(P.hits + a);
    }
  }
  if (DEBUG && g.leader()) {
    P.dump.n_trip[f] = 0;
    P.dump.n_combo[f] = 0;
  }
  if (n64 < 0) {
    if (g.leader()) atomicOr(P.err, ERR_NEGSIZE);
    return M3E_ERR_BADHIT;
  }
  if (DEFER && n64 > (CH < P.defer_hits ? CH : P.defer_hits)) return DEFERRED;
  const int n = (int)(n64 > 0x7fffffff ? 0x7fffffff : n64);
  const int32_t* hp = P.hits + base;

  // ---- A: decode and histogram
  for (int k = g.rank(); k < (S::kPackB ? NBK / 4 : NBK); k += G::N) sm.bcur[k] = 0;
  // warp stage: the per-layer decode table (DevCfg::ltab) for parts A and B, in the
  // space of the layer-2 z order, which part C fills later
  uint4* const ltab = reinterpret_cast<uint4*>(sm.zq);
  if constexpr (G::N == 32 && DEFER && TAB) {
    static_assert(sizeof(sm.zq) >= 4 * sizeof(uint4), "room for the decode table");
    if (g.rank() < 4) ltab[g.rank()] = C.ltab[g.rank()];
  }
  if (g.leader()) {
    sm.bad = 0;
    sm.ntrip = 0;
    sm.npos = 0;
    sm.nneg = 0;
    sm.ncombo = 0;
    sm.nstore = 0;
    sm.flag = 0;
    if (stats)
      for (int k = 0; k < ST_REASON0; ++k) sm.facc[k] = 0;
  }
  g.sync();
  if constexpr (G::N == 32 && DEFER) {
    // warp stage (n <= CH): each lane holds its hits' addresses in registers, so the
    // loads of a frame (addresses, then the table entries) are all in flight at once
    constexpr int K = (CH + 31) / 32;
    const int lane = g.rank();
    uint32_t av[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int i = lane + 32 * k;
      av[k] = i < n ? (uint32_t)(LIVE ? __ldcv(hp + i) : __ldg(hp + i)) : 0u;
    }
    bool bad = false;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (lane + 32 * k < n) {
        const Dec d = TAB ? decode_s(ltab, av[k]) : decode(C, av[k]);
        if (!d.ok) bad = true;
        else bucket_add(sm, d.L * NB + d.b);
      }
    }
    if (__any_sync(FULL, bad)) {
      if (g.leader()) atomicOr(P.err, ERR_BADHIT);
      return M3E_ERR_BADHIT;
    }
    if (n > C.max_hits) return M3E_HIT_OVERFLOW;
    if (stats && g.leader()) {
      sm.facc[ST_FRAMES] += 1;
      sm.facc[ST_HITS] += n;
    }
    // ---- B: counting sort by (layer, phi bin); the table entries go straight from
    // global to shared memory (asynchronous 4-byte copies, all of the lane's in flight)
    bucket_scan(g, sm);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int i = lane + 32 * k;
      if (i < n) {
        const Dec d = TAB ? decode_s(ltab, av[k]) : decode(C, av[k]);
        const int pos = bucket_add(sm, d.L * NB + d.b);
        const float* cl = reinterpret_cast<const float*>(P.col_lut + d.ci);
        cp_async4(&sm.x[pos], cl);
        cp_async4(&sm.y[pos], cl + 1);
        if constexpr (S::kPhi) cp_async4(&sm.phi[pos], cl + 2);
        cp_async4(&sm.z[pos], P.row_lut + d.ri);
        if constexpr (S::kAddr) sm.addr[pos] = av[k];
        if constexpr (S::kIdx) sm.inidx[pos] = (uint16_t)i;
      }
    }
    cp_async_wait_all();
  } else {
    for (int i = g.rank(); i < n; i += G::N) {
      const Dec d = decode(C, (uint32_t)(LIVE ? __ldcv(hp + i) : __ldg(hp + i)));
      if (!d.ok) sm.bad = 1;
      else if (n <= CH) bucket_add(sm, d.L * NB + d.b);
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
    bucket_scan(g, sm);
    for (int i = g.rank(); i < n; i += G::N) {
      const uint32_t a = (uint32_t)(LIVE ? __ldcv(hp + i) : __ldg(hp + i));
      const Dec d = decode(C, a);
      const int key = d.L * NB + d.b;
      const int pos = bucket_add(sm, key);
      const float4 c4 = __ldg(P.col_lut + d.ci);
      sm.x[pos] = c4.x;
      sm.y[pos] = c4.y;
      if constexpr (S::kPhi) sm.phi[pos] = c4.z;
      sm.z[pos] = __ldg(P.row_lut + d.ri);
      if constexpr (S::kAddr) sm.addr[pos] = a;
      if constexpr (S::kIdx) sm.inidx[pos] = (uint16_t)i;
    }
  }
  g.sync();

  // ---- C: selection cuts (Algorithm 2), pairs restricted to reachable phi bins.
  // The bins of a window are contiguous in the sorted order, so a window is one
  // index range, or two when it wraps past phi = 2 pi.
  {
    unsigned npair = 0, ntt = 0;
    const int l1a = sm.bstart[NB], l1b = sm.bstart[2 * NB];
    const int nb0 = min(2 * C.k01 + 1, NB), nb2 = min(2 * C.k12 + 1, NB);
    if constexpr (G::N == 32) {
      warp_cuts<S, CT>(sm, C, stats, npair, ntt);
    } else {
      // CTA stage.  The layer-2 hits are first put in z-bin order, so that the Delta
      // lambda cut of a (layer-0, layer-1) pair, seen as a z window on the layer-2 hit
      // (widened by 1e-3 mm against rounding), is one contiguous range of that order.
      // Each warp holds 32 layer-1 hits at a time and tests the entries of their Phi01
      // windows 32 at a time (each lane finds its hit by a search over the lanes'
      // prefix of window sizes); the z ranges of the pairs that pass are numbered by a
      // prefix sum, and their candidates are tested 32 at a time (a second search)
      // with the exact Phi12, Delta lambda and r_tc expressions of the warp stage.  The z window holds every hit that
      // passes Delta lambda, so the selected set equals the brute-force one.  A frame
      // whose triplet count passed max_trip overflows whatever follows: the warps stop.
      constexpr int NW = G::N / 32;
      const int lane = g.rank() & 31, wid = g.rank() >> 5;
      const int l2b = sm.bstart[3 * NB];
      static_assert(NZB == 64, "two z bins per lane in the prefix sum");
      for (int k = g.rank(); k < NZB; k += G::N) sm.zcur[k] = 0u;
      g.sync();
      for (int i = l1b + g.rank(); i < l2b; i += G::N) atomicAdd(&sm.zcur[zbin2(sm.z[i], C)], 1u);
      g.sync();
      if (g.rank() < 32) {
        const int ca = (int)sm.zcur[2 * lane], cb = (int)sm.zcur[2 * lane + 1];
        int inc = ca + cb;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int t = __shfl_up_sync(FULL, inc, o);
          if (lane >= o) inc += t;
        }
        const int ex = inc - ca - cb;
        sm.zbs2[2 * lane] = (uint16_t)ex;
        sm.zbs2[2 * lane + 1] = (uint16_t)(ex + ca);
        sm.zcur[2 * lane] = (uint32_t)ex;
        sm.zcur[2 * lane + 1] = (uint32_t)(ex + ca);
        if (lane == 31) sm.zbs2[NZB] = (uint16_t)inc;
      }
      g.sync();
      for (int i = l1b + g.rank(); i < l2b; i += G::N) sm.zidx[atomicAdd(&sm.zcur[zbin2(sm.z[i], C)], 1u)] = (uint16_t)i;
      g.sync();
      auto overflowed = [&]() {
        int ov = 0;
        if (lane == 0) ov = *(volatile int*)&sm.ntrip > C.max_trip;
        return __shfl_sync(FULL, ov, 0) != 0;
      };
      // a warp takes every NW-th layer-1 hit, 32 of them at a time (a lane each);
      // the Phi01 windows of those hits are tested 32 entries at a time
      const int nh = l1b - l1a > wid ? (l1b - l1a - wid + NW - 1) / NW : 0;
      bool stop = false;
      for (int mb = 0; mb < nh && !stop; mb += 32) {
        const bool has = mb + lane < nh;
        const int i1 = l1a + wid + NW * (mb + lane);
        float x1 = 0.f, y1 = 0.f, z1 = 0.f;
        int a0 = 0, n0a = 0, n0w = 0, c12 = 0;
        if (has) {
          x1 = sm.x[i1];
          y1 = sm.y[i1];
          z1 = sm.z[i1];
          const int b1 = layer1_bin(sm.bstart, i1);
          const int s0 = nb0 == NB ? 0 : (b1 - C.k01 + NB) & (NB - 1);
          a0 = sm.bstart[s0];
          n0a = sm.bstart[min(s0 + nb0, NB)] - a0;
          n0w = n0a + (s0 + nb0 > NB ? sm.bstart[s0 + nb0 - NB] : 0);
          if (stats) {  // the pair tests within the reachable phi bins, and the Phi12 partners
            const int s2 = nb2 == NB ? 0 : (b1 - C.k12 + NB) & (NB - 1);
            const int a2 = sm.bstart[2 * NB + s2], n2a = sm.bstart[2 * NB + min(s2 + nb2, NB)] - a2;
            const int w2 = sm.bstart[2 * NB];
            npair += n0w + n2a + (s2 + nb2 > NB ? sm.bstart[2 * NB + s2 + nb2 - NB] - w2 : 0);
            for (int k = l1b; k < l2b; ++k) c12 += phi_pass(x1, y1, sm.x[k], sm.y[k], C.c12);
          }
        }
        int pe = n0w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int t = __shfl_up_sync(FULL, pe, o);
          if (lane >= o) pe += t;
        }
        const int pre1 = pe - n0w, T1 = __shfl_sync(FULL, pe, 31);
        for (int e0 = 0; e0 < T1 && !stop; e0 += 32) {
          const int e = e0 + lane;
          int ow = 0;  // the last lane whose window entries start at or before e
#pragma unroll
          for (int st = 16; st; st >>= 1) {
            const int pv = __shfl_sync(FULL, pre1, ow + st);
            if (pv <= e) ow += st;
          }
          const int oa0 = __shfl_sync(FULL, a0, ow), on0a = __shfl_sync(FULL, n0a, ow);
          const int opre = __shfl_sync(FULL, pre1, ow), oi1 = __shfl_sync(FULL, i1, ow);
          const float ox1 = __shfl_sync(FULL, x1, ow), oy1 = __shfl_sync(FULL, y1, ow), oz1 = __shfl_sync(FULL, z1, ow);
          const int oc12 = __shfl_sync(FULL, c12, ow);
          int i0 = 0;
          bool p01 = false;
          if (e < T1) {
            const int k = e - opre;
            i0 = k < on0a ? oa0 + k : k - on0a;
            p01 = phi_pass(sm.x[i0], sm.y[i0], ox1, oy1, C.c01);
          }
          if (p01) ntt += oc12;
          // the Phi01 pairs' z ranges in the z order of layer 2, then their candidates
          float tl01 = 0.f;
          int lo = 0, cnt = 0;
          if (p01) {
            tl01 = tan_l01(sm.z[i0], oz1, C);
            const float zlo = oz1 + (tl01 - C.dl_max) * C.dr12 - 1e-3f;
            const float zhi = oz1 + (tl01 + C.dl_max) * C.dr12 + 1e-3f;
            lo = sm.zbs2[zbin2(zlo, C)];
            cnt = sm.zbs2[zbin2(zhi, C) + 1] - lo;
          }
          int ce = cnt;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(FULL, ce, o);
            if (lane >= o) ce += t;
          }
          const int pre2 = ce - cnt, T2 = __shfl_sync(FULL, ce, 31);
          for (int c0 = 0; c0 < T2 && !stop; c0 += 32) {
            const int c = c0 + lane;
            int pw = 0;  // the last lane whose candidates start at or before c
#pragma unroll
            for (int st = 16; st; st >>= 1) {
              const int pv = __shfl_sync(FULL, pre2, pw + st);
              if (pv <= c) pw += st;
            }
            const int pi0 = __shfl_sync(FULL, i0, pw), pi1 = __shfl_sync(FULL, oi1, pw);
            const int plo = __shfl_sync(FULL, lo, pw), ppre = __shfl_sync(FULL, pre2, pw);
            const float ptl = __shfl_sync(FULL, tl01, pw);
            const float px1 = __shfl_sync(FULL, ox1, pw), py1 = __shfl_sync(FULL, oy1, pw), pz1 = __shfl_sync(FULL, oz1, pw);
            if (c < T2) {
              const int i2 = sm.zidx[plo + c - ppre];
              const float x2 = sm.x[i2], y2 = sm.y[i2], z2 = sm.z[i2];
              if (phi_pass(px1, py1, x2, y2, C.c12) && dl_pass(pz1, z2, ptl, C) &&
                  rtc_pass(sm.x[pi0], sm.y[pi0], px1, py1, x2, y2, C)) {
                const int kk = atomicAdd(&sm.ntrip, 1);
                if (kk < CT) sm.u.trip[kk] = make_trip<typename S::TripT>(pi0, pi1, i2);
              }
            }
            stop = overflowed();
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
  if (DEFER && sm.bad == 2) return DEFERRED;  // partner lists beyond the warp stage's capacity
  const int ntrip = sm.ntrip;
  if (DEBUG && g.leader()) P.dump.n_trip[f] = ntrip;
  if (ntrip > C.max_trip) return M3E_TRIPLET_OVERFLOW;
  if (DEFER && ntrip > CT) return DEFERRED;
  if (stats && g.leader()) sm.facc[ST_TRIP] += ntrip;
  return PENDING;
}

// Stages D-F of one frame after frame_front returned PENDING: track
// reconstruction, energy test and vertex.  Returns a final reason or DEFERRED.
template <class G, class S, int CT, int CK, int CC, bool DEFER, bool DEBUG>
__device__ int frame_back(const G& g, S& sm, const DevCfg& C, const KParams& P, int f) {
  const bool stats = P.stats != nullptr;
  const int ntrip = sm.ntrip;
  const SmHits<S> view{sm};
  // ---- D: track reconstruction (Algorithm 3), one thread per triplet
  for (int t = g.rank(); t < ntrip; t += G::N) {
    const auto tr = sm.u.trip[t];
    const TrackOut o = build_track(view, C, tr.x, tr.y, tr.z);
    if (o.status == 5) {
      float tk[14];
      track_record(view.pos(tr.x), view.pos(tr.y), o, C, tk);
      int slot = -1;
      if (tk[13] > 0.f) {
        const int k = atomicAdd(&sm.npos, 1);
        if (k < CK) slot = k;
      } else {
        const int k = atomicAdd(&sm.nneg, 1);
        if (k < CK) slot = CK - 1 - k;
      }
      if (slot >= 0) store_track(sm.t, slot, tk, t);
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

  // ---- E: energy test of every (e+ pair, e-) combination (Algorithm 4, part 1):
  // one e+ pair per thread, the e- loop uniform across the group (broadcast reads).
  // All passing combinations count towards the cap; a decision-only run stores only
  // those whose P_z leaves the momentum cut open (pz_fails_ptot).
  const bool prune = !DEBUG && !stats;
  {
    const int npair = npos * (npos - 1) / 2;
    for (int pr = g.rank(); pr < npair; pr += G::N) {
      int b = (int)((1.f + sqrtf(1.f + 8.f * (float)pr)) * 0.5f);
      while (b * (b - 1) / 2 > pr) --b;
      while ((b + 1) * b / 2 <= pr) ++b;
      const int a = pr - b * (b - 1) / 2;
      const float eab = sm.t.E[a] + sm.t.E[b];
      const float pzab = __fadd_rn(pz_track(sm.t.p[a], sm.t.ct[a]), pz_track(sm.t.p[b], sm.t.ct[b]));
      for (int c = 0; c < nneg; ++c) {
        const int ci = CK - 1 - c;
        const float e = (eab + sm.t.E[ci]) - C.m_mu;
        if (fabsf(e) <= C.e_win) {
          const int k = atomicAdd(&sm.ncombo, 1);
          const uint32_t code = (uint32_t)a | ((uint32_t)b << 8) | ((uint32_t)ci << 16);
          const bool open = !pz_fails_ptot(__fadd_rn(pzab, pz_track(sm.t.p[ci], sm.t.ct[ci])), C.ptot_max);
          if (!prune) {
            if (k < CC) sm.u.combo[k] = code;
            if (stats && open) atomicAdd(&sm.facc[ST_PZOPEN], 1ull);
          } else if (open) {
            const int k2 = atomicAdd(&sm.nstore, 1);
            if (k2 < CC) sm.u.combo[k2] = code;
          }
        }
      }
    }
    if (stats && g.leader()) sm.facc[ST_ETEST] += (unsigned long long)npair * nneg;
  }
  g.sync();
  const int ncombo = sm.ncombo;
  const int nvtx = prune ? sm.nstore : ncombo;  // combinations to fit
  if (DEBUG && g.leader()) P.dump.n_combo[f] = ncombo;
  if (ncombo > C.max_combo) {
    if (stats && g.leader()) sm.facc[ST_PZOPEN] = 0;  // counted, as the combinations, only when fitted
    return M3E_COMBO_OVERFLOW;
  }
  if (DEFER && nvtx > CC) return DEFERRED;
  if (stats && g.leader()) sm.facc[ST_COMBO] += ncombo;

  // ---- F: vertex of each combination (Algorithm 4, part 2), early exit
  bool found = false;
  unsigned nv = 0, nvo = 0;
  for (int c0 = 0; c0 < nvtx; c0 += G::N) {
    const int c = c0 + g.rank();
    bool pass = false;
    if (c < nvtx) {
      const uint32_t cb = sm.u.combo[c];
      const int a = cb & 255, b = (cb >> 8) & 255, e = (cb >> 16) & 255;
      const VtxOut v = vertex(load_track(sm.t, a), load_track(sm.t, b), load_track(sm.t, e), C);
      pass = v.pass != 0;
      nv += v.status == 2;
      if (stats && v.status == 2)
        nvo += !pz_fails_ptot(pz_sum(pz_track(sm.t.p[a], sm.t.ct[a]), pz_track(sm.t.p[b], sm.t.ct[b]),
                                     pz_track(sm.t.p[e], sm.t.ct[e])), C.ptot_max);
      if (DEBUG && c < P.dump.cap_combo) {
        const int64_t r = (int64_t)f * P.dump.cap_combo + c;
        P.dump.combo[4 * r + 0] = sm.t.tid[a];
        P.dump.combo[4 * r + 1] = sm.t.tid[b];
        P.dump.combo[4 * r + 2] = sm.t.tid[e];
        P.dump.combo[4 * r + 3] = v.status | (v.pass << 8);
        P.dump.combo_val[4 * r + 0] = (sm.t.E[a] + sm.t.E[b] + sm.t.E[e]) - C.m_mu;
        P.dump.combo_val[4 * r + 1] = v.chi2;
        P.dump.combo_val[4 * r + 2] = v.tdist;
        P.dump.combo_val[4 * r + 3] = v.ptot;
        if (P.dump.combo_aux) {
          float dm, fm;
          vertex_soft(load_track(sm.t, a), load_track(sm.t, b), load_track(sm.t, e), C.isect_lim, dm, fm);
          P.dump.combo_aux[4 * r + 0] = dm;
          P.dump.combo_aux[4 * r + 1] = fm;
          P.dump.combo_aux[4 * r + 2] = v.chi2_second;
          P.dump.combo_aux[4 * r + 3] = 0.f;
        }
      }
    }
    found = g.any(pass) || found;
    if (found && !DEBUG) break;
  }
  if (stats && nv) atomicAdd(&sm.facc[ST_VTX], (unsigned long long)nv);
  if (stats && nvo) atomicAdd(&sm.facc[ST_VTXOPEN], (unsigned long long)nvo);
  return found ? M3E_VERTEX : M3E_DROP;
}

template <class G, class S, bool NOST = false>
__device__ __forceinline__ void finish_frame(const G& g, S& sm, const KParams& P, int f, int r) {
  g.sync();
  if (g.leader()) {
    P.keep[f] = (uint8_t)(r != M3E_DROP);
    P.reason[f] = (uint8_t)r;
    if (!NOST && P.stats) {
      sm.acc[ST_REASON0 + r] += 1;
      for (int k = 0; k < ST_REASON0; ++k) sm.acc[k] += sm.facc[k];
    }
  }
}

template <class G, class S>
__device__ __forceinline__ void flush_stats(const G& g, S& sm, unsigned long long* stats) {
  g.sync();
  if (stats)
    for (int k = g.rank(); k < ST_REASON0 + 8; k += G::N)
      if (sm.acc[k]) atomicAdd(stats + k, sm.acc[k]);
}

template <class G, class S>
__device__ __forceinline__ void clear_stats(const G& g, S& sm) {
  for (int k = g.rank(); k < ST_REASON0 + 8; k += G::N) sm.acc[k] = 0;
  g.sync();
}

}  // namespace
}  // namespace m3e
