// Gradient of the summed track chi2 of frozen candidates with respect to the
// rigid alignment of the four layers and the field scale (libm3e).
//
// A candidate is a quadruplet of hits (layers 0..3) whose track the selection
// found (Sec. "Track Reconstruction": two triplet fits and the global chi2 at the
// inverse-variance mean curvature).  The hit measured at nominal position x_nom
// on layer L sits at R(w_L) x_nom + d_L, R = Rz(wz) Ry(wy) Rx(wx); the field is
// scaled by params[24].  The selection of the quadruplet is discrete and stays
// fixed; chi2 is differentiable in the positions, so the gradient is exact for
// the frozen set.
//
// One thread per candidate: forward fit (the same fit_triplet as the selection,
// so that the chi2 equals the selection's at nominal alignment), then the
// reverse sweep by hand, recomputing each triplet's intermediate values instead
// of storing them.  d chi2 / d(field scale) = 2 chi2 / scale exactly: the scale
// enters only through sigma_MS ~ 1/p and the two triplets' weights scale alike.
// Sums: per-thread FP32 over its candidates, per-block FP64, then one block in a
// fixed order (deterministic for a given grid).
#include "m3e_device.cuh"

namespace m3e {
namespace {

constexpr int GT = 128;            // threads per block
constexpr int NG = 26;             // chi2, 24 alignment gradients, field-scale gradient

struct AlignSm {
  float R[4][9];                   // rotation of each layer (row-major)
  float dR[4][3][9];               // derivative with respect to wx, wy, wz
  float d[4][3];
  float scale;
};

__device__ void rotation_and_derivatives(const float* w, float* R, float* dR) {
  float sx, cx, sy, cy, sz, cz;
  sincosf(w[0], &sx, &cx);
  sincosf(w[1], &sy, &cy);
  sincosf(w[2], &sz, &cz);
  const float Rx[9] = {1, 0, 0, 0, cx, -sx, 0, sx, cx}, dRx[9] = {0, 0, 0, 0, -sx, -cx, 0, cx, -sx};
  const float Ry[9] = {cy, 0, sy, 0, 1, 0, -sy, 0, cy}, dRy[9] = {-sy, 0, cy, 0, 0, 0, -cy, 0, -sy};
  const float Rz[9] = {cz, -sz, 0, sz, cz, 0, 0, 0, 1}, dRz[9] = {-sz, -cz, 0, cz, -sz, 0, 0, 0, 0};
  auto mul = [](const float* A, const float* B, float* out) {
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) out[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
  };
  float T[9];
  mul(Ry, Rx, T);
  mul(Rz, T, R);
  mul(Rz, Ry, T);                  // d/dwx = Rz Ry dRx
  mul(T, dRx, dR);
  float U[9];
  mul(dRy, Rx, U);                 // d/dwy = Rz dRy Rx
  mul(Rz, U, dR + 9);
  mul(Ry, Rx, U);                  // d/dwz = dRz Ry Rx
  mul(dRz, U, dR + 18);
}

// ------------------------------------------------------------------ reverse sweep

// One segment of the circle solution (segment() in the shared device code):
// adjoints of (R_C, theta_C, dPhi/dR, dtheta/dR) to adjoints of (d, z, R_t, Phi).
// The outputs are written as functions of d, z, R_t and the arc angle Phi, with
// sin(Phi/2) and cos(Phi/2) functions of Phi: the arc angle is a smooth function
// of the hits (twice the triangle's angle at the third hit), whereas its form
// 2 asin(d / 2 R_t) has an infinite slope at a half turn, where the branch
// switches.
__device__ void segment_bwd(float d, float z, float Rct, bool obtuse, float RC_b, float th_b, float dphi_b,
                            float dth_b, float& d_b, float& z_b, float& Rct_b, float& phi_b) {
  const float sh = fminf(1.f, d / (2.f * Rct));
  float ph = 2.f * asinf(sh);
  float ch = sqrtf(fmaxf((1.f - sh) * (1.f + sh), 0.f));
  if (obtuse) {
    ph = TWO_PI_F - ph;
    ch = -ch;
  }
  const float zp = z / ph;
  const float RC = sqrtf(Rct * Rct + zp * zp);
  const float Y = Rct * ph;
  const float sh2 = sh * sh;
  const float Q = d * d * ch / (8.f * sh2 * sh) + zp * zp / ph;
  const float dRdphi = -Q / RC;
  const float dphi = 1.f / dRdphi;
  const float g = ph / (2.f * sh);
  const float gp = sin_minus_xcos(0.5f * ph, sh, ch) / (2.f * sh2);
  const float dg = d * g;
  const float Dz = z * z + dg * dg;
  const float T = z * d * gp / Dz;
  // dth = T * dphi
  float ph_b = 0.f, sh_b = 0.f, ch_b = 0.f, zp_b = 0.f;
  d_b = 0.f;
  z_b = 0.f;
  Rct_b = 0.f;
  const float T_b = dth_b * dphi;
  dphi_b += dth_b * T;
  z_b += T_b * d * gp / Dz;
  d_b += T_b * z * gp / Dz;
  const float gp_b = T_b * z * d / Dz;
  const float Dz_b = -T_b * T / Dz;
  z_b += 2.f * z * Dz_b;
  const float dg_b = 2.f * dg * Dz_b;
  d_b += dg_b * g;
  const float g_b = dg_b * d;
  ph_b += g_b / (2.f * sh);
  sh_b -= g_b * g / sh;
  const float smx_b = gp_b / (2.f * sh2);          // gp = (sin x - x cos x) / (2 sh^2), x = ph / 2
  sh_b -= gp_b * 2.f * gp / sh;
  ph_b += smx_b * 0.25f * ph * sh;                 // d/dph (sin x - x cos x) = (ph / 4) sin(ph / 2)
  // dphi = 1 / dRdphi, dRdphi = -Q / RC
  const float dRdphi_b = -dphi_b * dphi * dphi;
  const float Q_b = -dRdphi_b / RC;
  RC_b -= dRdphi_b * dRdphi / RC;
  d_b += Q_b * d * ch / (4.f * sh2 * sh);
  ch_b += Q_b * d * d / (8.f * sh2 * sh);
  sh_b -= Q_b * 3.f * d * d * ch / (8.f * sh2 * sh2);
  zp_b += Q_b * 2.f * zp / ph;
  ph_b -= Q_b * zp * zp / (ph * ph);
  // th = atan2(Rct * ph, z)
  const float r2 = Y * Y + z * z;
  const float Y_b = th_b * z / r2;
  z_b -= th_b * Y / r2;
  Rct_b += Y_b * ph;
  ph_b += Y_b * Rct;
  // RC = sqrt(Rct^2 + zp^2), zp = z / ph
  Rct_b += RC_b * Rct / RC;
  zp_b += RC_b * zp / RC;
  z_b += zp_b / ph;
  ph_b -= zp_b * zp / ph;
  // sh = sin(ph / 2), ch = cos(ph / 2) on both branches (ch carries the sign)
  phi_b = ph_b + 0.5f * (sh_b * ch - ch_b * sh);
}

// Angle at r between p - r and q - r, atan2(|X|, D), X = (p-r) x (q-r), D = (p-r).(q-r):
// adds the adjoints of the transverse coordinates of p, q, r.
__device__ __forceinline__ void angle_bwd(const float* p, const float* q, const float* r, float ang_b, float* gp,
                                          float* gq, float* gr) {
  const float ex = p[0] - r[0], ey = p[1] - r[1], fx = q[0] - r[0], fy = q[1] - r[1];
  const float X = ex * fy - ey * fx, D = ex * fx + ey * fy;
  const float n2 = X * X + D * D;
  const float X_b = ang_b * (X >= 0.f ? D : -D) / n2, D_b = -ang_b * fabsf(X) / n2;
  const float ex_b = X_b * fy + D_b * fx, ey_b = -X_b * fx + D_b * fy;
  const float fx_b = -X_b * ey + D_b * ex, fy_b = X_b * ex + D_b * ey;
  gp[0] += ex_b;
  gp[1] += ey_b;
  gq[0] += fx_b;
  gq[1] += fy_b;
  gr[0] -= ex_b + fx_b;
  gr[1] -= ey_b + fy_b;
}

struct TripBar {                   // adjoints of a triplet fit's outputs
  float alpha, a0p, beta, b0p, s2, Rref, kappa, w;
};

// Reverse sweep of fit_triplet for hits a -> b -> c: recomputes the forward values
// and returns the adjoints of the nine coordinates.
__device__ void fit_triplet_bwd(const float* a, const float* b, const float* c, float hl, float kB, const TripBar& o,
                                float* ga, float* gb, float* gc) {
  const float ux = a[0] - b[0], uy = a[1] - b[1], vx = c[0] - b[0], vy = c[1] - b[1];
  const float wx = c[0] - a[0], wy = c[1] - a[1];
  const float cross = ux * vy - uy * vx;
  const float d01 = sqrtf(ux * ux + uy * uy), d12 = sqrtf(vx * vx + vy * vy), d20 = sqrtf(wx * wx + wy * wy);
  const float rtc = d01 * d12 * d20 / (2.f * cross);
  const float Rct = fabsf(rtc);
  const float eps = rtc > 0.f ? 1.f : -1.f;
  const bool ob0 = ((a[0] - c[0]) * (b[0] - c[0]) + (a[1] - c[1]) * (b[1] - c[1])) < 0.f;
  const bool ob1 = ((b[0] - a[0]) * (c[0] - a[0]) + (b[1] - a[1]) * (c[1] - a[1])) < 0.f;
  const float z01 = b[2] - a[2], z12 = c[2] - b[2];
  const SegF s0 = segment(d01, z01, Rct, 0.5f / Rct, ob0);
  const SegF s1 = segment(d12, z12, Rct, 0.5f / Rct, ob1);
  const float dR = s0.RC - s1.RC;
  const float alpha = 0.5f * (s0.dphi + s1.dphi);
  const float a0p = 0.5f * s1.dphi * dR;
  const float beta = s1.dth - s0.dth;
  const float b0p = (s1.th - s0.th) + s1.dth * dR;
  float sn, cm;
  sincosf(0.5f * (s0.th + s1.th), &sn, &cm);
  const float s2 = sn * sn;
  const float den = alpha * alpha * s2 + beta * beta;
  const float N = alpha * a0p * s2 + beta * b0p;
  const float u = -N / den;
  const float Rs = s0.RC + u;
  const float kappa = eps / Rs;
  const float kr = kB * Rs * Rs * Rs / hl;
  const float w = kr * kr * den;   // 1 / sigma_kappa^2
  // kappa = eps / Rs, w = kB^2 Rs^6 den / hl^2
  const float Rs_b = o.kappa * (-kappa / Rs) + o.w * (6.f * w / Rs);
  float den_b = o.w * (w / den);
  float Rref_b = o.Rref + Rs_b;    // Rs = R_C0 + u
  const float u_b = Rs_b;
  const float N_b = -u_b / den;    // u = -N / den
  den_b -= u_b * u / den;
  const float alpha_b = o.alpha + N_b * a0p * s2 + den_b * 2.f * alpha * s2;
  const float a0p_b = o.a0p + N_b * alpha * s2;
  const float s2_b = o.s2 + N_b * alpha * a0p + den_b * alpha * alpha;
  const float beta_b = o.beta + N_b * b0p + den_b * 2.f * beta;
  const float b0p_b = o.b0p + N_b * beta;
  const float m_b = s2_b * 2.f * sn * cm;  // s2 = sin^2(m), m = (th0 + th1) / 2
  float th0_b = 0.5f * m_b - b0p_b, th1_b = 0.5f * m_b + b0p_b;
  float dth1_b = b0p_b * dR + beta_b;
  const float dth0_b = -beta_b;
  float dR_b = b0p_b * s1.dth + 0.5f * a0p_b * s1.dphi;
  const float dphi1_b = 0.5f * a0p_b * dR + 0.5f * alpha_b;
  const float dphi0_b = 0.5f * alpha_b;
  const float RC0_b = Rref_b + dR_b, RC1_b = -dR_b;
  float d01_b, z01_b, Rct0_b, d12_b, z12_b, Rct1_b, phi0_b, phi1_b;
  segment_bwd(d01, z01, Rct, ob0, RC0_b, th0_b, dphi0_b, dth0_b, d01_b, z01_b, Rct0_b, phi0_b);
  segment_bwd(d12, z12, Rct, ob1, RC1_b, th1_b, dphi1_b, dth1_b, d12_b, z12_b, Rct1_b, phi1_b);
  const float rtc_b = eps * (Rct0_b + Rct1_b);    // R_t = |rtc|
  d01_b += rtc_b * rtc / d01;      // rtc = d01 d12 d20 / (2 cross)
  d12_b += rtc_b * rtc / d12;
  const float d20_b = rtc_b * rtc / d20;
  const float cross_b = -rtc_b * rtc / cross;
  float ux_b = d01_b * ux / d01 + cross_b * vy, uy_b = d01_b * uy / d01 - cross_b * vx;
  float vx_b = d12_b * vx / d12 - cross_b * uy, vy_b = d12_b * vy / d12 + cross_b * ux;
  const float wx_b = d20_b * wx / d20, wy_b = d20_b * wy / d20;
  ga[0] = ux_b - wx_b;
  ga[1] = uy_b - wy_b;
  ga[2] = -z01_b;
  gb[0] = -ux_b - vx_b;
  gb[1] = -uy_b - vy_b;
  gb[2] = z01_b - z12_b;
  gc[0] = vx_b + wx_b;
  gc[1] = vy_b + wy_b;
  gc[2] = z12_b;
  // arc angles (inscribed-angle theorem): Phi_01 = 2 x angle at c, Phi_12 = 2 x angle at a
  angle_bwd(a, b, c, 2.f * phi0_b, ga, gb, gc);
  angle_bwd(b, c, a, 2.f * phi1_b, gb, gc, ga);
}

struct GradParams {
  const int32_t* hits;
  const int64_t* off;              // off[n_frames] = number of hits (bound of the indices)
  int64_t n_frames;
  const int4* cand;
  int64_t n_cand;
  const float* params;             // 25
  const float4* col_lut;
  const float* row_lut;
  double* partial;                 // [gridDim.x][NG]
  float* chi2_each;                // or nullptr
  float* kappa_each;               // or nullptr: the weighted mean curvature of each fit
  unsigned long long* n_valid;     // candidates with a finite chi2 and gradient
  int grad;
};

template <bool GRAD>
__global__ void __launch_bounds__(GT) k_fit_grad(const __grid_constant__ DevCfg C, const __grid_constant__ GradParams G) {
  __shared__ AlignSm A;
  __shared__ double red[GT / 32][NG];
  if (threadIdx.x < 4) {
    const int L = threadIdx.x;
    float w[3] = {G.params[6 * L + 3], G.params[6 * L + 4], G.params[6 * L + 5]};
    rotation_and_derivatives(w, A.R[L], &A.dR[L][0][0]);
    for (int k = 0; k < 3; ++k) A.d[L][k] = G.params[6 * L + k];
  }
  if (threadIdx.x == 0) A.scale = G.params[24];
  __syncthreads();
  const int64_t n_hits = G.off[G.n_frames];
  const float kB = C.kB * A.scale;
  float acc[NG];
#pragma unroll
  for (int k = 0; k < NG; ++k) acc[k] = 0.f;
  unsigned nvalid = 0;
  for (int64_t i = blockIdx.x * (int64_t)GT + threadIdx.x; i < G.n_cand; i += (int64_t)gridDim.x * GT) {
    const int4 q = G.cand[i];
    const int qi[4] = {q.x, q.y, q.z, q.w};
    float P[4][3], X[4][3];
    bool ok = true;
#pragma unroll
    for (int L = 0; L < 4; ++L) {
      const int h = qi[L];
      ok = ok && h >= 0 && h < n_hits;
      const Dec dd = decode(C, ok ? (uint32_t)__ldg(G.hits + h) : 0u);
      ok = ok && dd.ok && dd.L == L;
      if (ok) {
        const float4 cl = __ldg(G.col_lut + C.col_off[L] + dd.g);
        X[L][0] = cl.x;
        X[L][1] = cl.y;
        X[L][2] = __ldg(G.row_lut + C.row_off[L] + dd.row);
      } else {
        X[L][0] = X[L][1] = X[L][2] = 0.f;
      }
      const float* R = A.R[L];
#pragma unroll
      for (int r = 0; r < 3; ++r) P[L][r] = R[3 * r] * X[L][0] + R[3 * r + 1] * X[L][1] + R[3 * r + 2] * X[L][2] + A.d[L][r];
    }
    float chi2 = __int_as_float(0x7fc00000);  // NaN unless the fit succeeds
    float kb_out = __int_as_float(0x7fc00000);
    if (ok) {
      const TFitF f1 = fit_triplet(P[0][0], P[0][1], P[0][2], P[1][0], P[1][1], P[1][2], P[2][0], P[2][1], P[2][2],
                                   C.hl[1], kB);
      const TFitF f2 = fit_triplet(P[1][0], P[1][1], P[1][2], P[2][0], P[2][1], P[2][2], P[3][0], P[3][1], P[3][2],
                                   C.hl[2], kB);
      ok = f1.valid && f2.valid;
      float kb = 0.f, w1 = 0.f, w2 = 0.f;
      if (ok) {
        w1 = 1.f / (f1.skappa * f1.skappa);
        w2 = 1.f / (f2.skappa * f2.skappa);
        kb = (f1.kappa * w1 + f2.kappa * w2) / (w1 + w2);
        ok = kb != 0.f && isfinite(kb);
      }
      if (ok) {
        kb_out = kb;
        const float Rb = 1.f / fabsf(kb);
        const float pb = kB * Rb;
        chi2 = kink_chi2(f1, Rb, pb * C.ihl[1]) + kink_chi2(f2, Rb, pb * C.ihl[2]);
        ok = isfinite(chi2);
        if (GRAD && ok) {
          // chi2 = sum_t (A_t^2 s2_t + B_t^2) q_t, A = alpha u + a0p, B = beta u + b0p,
          // u = Rb - Rref, q = (kB Rb / hl)^2
          const TFitF* ft[2] = {&f1, &f2};
          TripBar tb[2];
          float Rb_b = 0.f;
#pragma unroll
          for (int t = 0; t < 2; ++t) {
            const TFitF& f = *ft[t];
            const float u = Rb - f.Rref;
            const float Aq = f.alpha * u + f.a0p, Bq = f.beta * u + f.b0p;
            const float kq = pb * (t == 0 ? C.ihl[1] : C.ihl[2]);
            const float qt = kq * kq;
            tb[t].alpha = 2.f * Aq * u * f.s2 * qt;
            tb[t].a0p = 2.f * Aq * f.s2 * qt;
            tb[t].beta = 2.f * Bq * u * qt;
            tb[t].b0p = 2.f * Bq * qt;
            tb[t].s2 = Aq * Aq * qt;
            const float lin = (2.f * Aq * f.alpha * f.s2 + 2.f * Bq * f.beta) * qt;
            tb[t].Rref = -lin;
            Rb_b += lin + (Aq * Aq * f.s2 + Bq * Bq) * 2.f * qt / Rb;
          }
          // Rb = 1 / |kb|, kb = (k1 w1 + k2 w2) / (w1 + w2)
          const float kb_b = -Rb_b * Rb * Rb * (kb > 0.f ? 1.f : -1.f);
          const float W = w1 + w2;
          tb[0].kappa = kb_b * w1 / W;
          tb[1].kappa = kb_b * w2 / W;
          tb[0].w = kb_b * (f1.kappa - kb) / W;
          tb[1].w = kb_b * (f2.kappa - kb) / W;
          float g[4][3] = {};
          float ga[3], gb[3], gc[3];
          fit_triplet_bwd(P[0], P[1], P[2], C.hl[1], kB, tb[0], ga, gb, gc);
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            g[0][r] += ga[r];
            g[1][r] += gb[r];
            g[2][r] += gc[r];
          }
          fit_triplet_bwd(P[1], P[2], P[3], C.hl[2], kB, tb[1], ga, gb, gc);
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            g[1][r] += ga[r];
            g[2][r] += gb[r];
            g[3][r] += gc[r];
          }
          // validity and the chi2 sum are the forward's; a gradient that is not finite
          // (coincident hits) is left out of the gradient only
          bool fin = true;
#pragma unroll
          for (int L = 0; L < 4; ++L)
            for (int r = 0; r < 3; ++r) fin = fin && isfinite(g[L][r]);
          if (fin) {
            // P = R(w) X + d: d P / d d = I, d P / d w_k = dR_k X
#pragma unroll
            for (int L = 0; L < 4; ++L) {
#pragma unroll
              for (int r = 0; r < 3; ++r) acc[1 + 6 * L + r] += g[L][r];
#pragma unroll
              for (int k = 0; k < 3; ++k) {
                const float* D = A.dR[L][k];
                float s = 0.f;
#pragma unroll
                for (int r = 0; r < 3; ++r) s += g[L][r] * (D[3 * r] * X[L][0] + D[3 * r + 1] * X[L][1] + D[3 * r + 2] * X[L][2]);
                acc[1 + 6 * L + 3 + k] += s;
              }
            }
            acc[25] += 2.f * chi2 / A.scale;
          }
        }
      }
    }
    if (ok) {
      acc[0] += chi2;
      ++nvalid;
    }
    if (G.chi2_each) G.chi2_each[i] = ok ? chi2 : __int_as_float(0x7fc00000);
    if (G.kappa_each) G.kappa_each[i] = ok ? kb_out : __int_as_float(0x7fc00000);
  }
  // block sums in FP64, fixed order
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NG; ++k) {
    double v = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
    if (lane == 0) red[wp][k] = v;
  }
  const unsigned nv = __reduce_add_sync(FULL, nvalid);
  if (lane == 0 && nv) atomicAdd(G.n_valid, (unsigned long long)nv);
  __syncthreads();
  if (threadIdx.x < NG) {
    double v = 0.0;
    for (int k = 0; k < GT / 32; ++k) v += red[k][threadIdx.x];
    G.partial[(int64_t)blockIdx.x * NG + threadIdx.x] = v;
  }
}

// Sum of the block partials, one thread per output in block order.
__global__ void k_fit_reduce(const double* partial, int nblocks, float* chi2_sum, float* grad) {
  const int k = threadIdx.x;
  if (k >= NG) return;
  double v = 0.0;
  for (int b = 0; b < nblocks; ++b) v += partial[(int64_t)b * NG + k];
  if (k == 0) {
    if (chi2_sum) *chi2_sum = (float)v;
  } else if (grad) {
    grad[k - 1] = (float)v;
  }
}

}  // namespace

int fit_grad_blocks(int sms, int64_t n_cand) {
  int64_t nb = (n_cand + GT - 1) / GT;
  const int64_t cap = (int64_t)sms * 16;
  if (nb > cap) nb = cap;
  return nb < 1 ? 1 : (int)nb;
}

int fit_grad_partial_size() { return NG; }

cudaError_t launch_fit_grad(const DevCfg& c, const int32_t* hits, const int64_t* off, int64_t n_frames,
                            const int32_t* cand, int64_t n_cand, const float* params, const float4* col_lut,
                            const float* row_lut, double* partial, int nblocks, unsigned long long* n_valid,
                            float* chi2_each, float* kappa_each, float* chi2_sum, float* grad, cudaStream_t s) {
  GradParams g{};
  g.hits = hits;
  g.off = off;
  g.n_frames = n_frames;
  g.cand = reinterpret_cast<const int4*>(cand);
  g.n_cand = n_cand;
  g.params = params;
  g.col_lut = col_lut;
  g.row_lut = row_lut;
  g.partial = partial;
  g.chi2_each = chi2_each;
  g.kappa_each = kappa_each;
  g.n_valid = n_valid;
  if (grad) k_fit_grad<true><<<nblocks, GT, 0, s>>>(c, g);
  else k_fit_grad<false><<<nblocks, GT, 0, s>>>(c, g);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_fit_reduce<<<1, 32, 0, s>>>(partial, nblocks, chi2_sum, grad);
  return cudaGetLastError();
}

}  // namespace m3e
