/* FP64 CPU oracle of the Mu3e online event selection (arXiv:2206.11535).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark, never by the library.  Plain, slow and
 * direct: brute force over every n0*n1*n2 hit triplet, every formula in double
 * precision, steps in the order the paper gives them:
 *   Sec. "Selection Cuts"        -> orc_cut_vars, select_triplets
 *   Sec. "Track Reconstruction"  -> orc_fit_triplet, build_track
 *   Sec. "Vertex Fit"            -> vertex_combination, select_vertex
 *   Sec. "Parallelization" (Algorithms 1-4: caps and keep-on-overflow)
 *                                -> orc_select_frame
 * Where the paper is silent or garbled, the reading taken is stated at the spot.
 * Parity status per function: every function here is pinned by the "not gpu"
 * tests (closed forms, brute force, finite differences, invariants) except the
 * vertex cut VALUES, which the paper does not print (calibrated, see config).
 */
#include "m3e_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define PI 3.14159265358979323846
#define TWO_PI (2.0 * PI)

/* ------------------------------------------------------------------ helpers */

static double wrap_2pi(double a) {  /* into [0, 2pi) */
  double r = fmod(a, TWO_PI);
  if (r < 0) r += TWO_PI;
  if (r >= TWO_PI) r = 0.0;
  return r;
}

static double wrap_pi(double a) {  /* into [-pi, pi] */
  double r = wrap_2pi(a + PI) - PI;
  return r;
}

static double field(const orc_config* c) { return c->B * c->field_scale; }

/* Highland width of the projected multiple-scattering angle, beta = 1
 * (the MS variance of Sec. "Single Triplet Fit", after Highland and Lynch-Dahl). */
double orc_highland(const orc_config* c, double p, int layer) {
  double x = c->x_over_X0[layer];
  return 13.6 / p * sqrt(x) * (1.0 + 0.038 * log(x));
}

/* ------------------------------------------------------------------ decode */

/* Pixel address -> layer/ladder/column/row and the pixel centre on the nominal
 * cylinder of that layer (the detector simplification of Sec. "Selection Cuts":
 * four concentric cylinders, so the transverse radius of every hit of layer i is
 * r_i).  Returns -1 for an address outside the detector. */
int orc_decode(const orc_config* c, uint32_t addr, orc_hit* h) {
  if ((addr >> 28) != 0) return -1;
  int L = (int)((addr >> 26) & 3u);
  int lad = (int)((addr >> 21) & 31u);
  int col = (int)((addr >> 13) & 255u);
  int row = (int)(addr & 8191u);
  if (lad >= c->nlad[L] || col >= c->ncol[L] || row >= c->nrow[L]) return -1;
  int ntot = c->nlad[L] * c->ncol[L];
  int g = lad * c->ncol[L] + col;
  double phi = ((double)g + 0.5) * TWO_PI / (double)ntot;
  h->x = c->r[L] * cos(phi);
  h->y = c->r[L] * sin(phi);
  h->z = -c->H[L] + ((double)row + 0.5) * c->pitch;
  h->phi = phi;
  h->layer = L; h->ladder = lad; h->col = col; h->row = row;
  h->addr = addr;
  return 0;
}

/* Order of hits inside a frame: by (layer, address); equal addresses keep their
 * input order (the chunk layout of Sec. "Memory Layout" sorts hits by frame and
 * layer).  The layer is the top field of the address, so the address alone orders. */
static int cmp_hit(const void* a, const void* b) {
  const orc_hit* x = (const orc_hit*)a;
  const orc_hit* y = (const orc_hit*)b;
  if (x->addr != y->addr) return x->addr < y->addr ? -1 : 1;
  return x->in_idx < y->in_idx ? -1 : (x->in_idx > y->in_idx);
}

/* ------------------------------------------------------------------ selection cuts */

/* The four cut variables of Sec. "Selection Cuts":
 *  v[0] = Delta lambda = tan(lambda_12) - tan(lambda_01), tan(lambda_ij) = (z_j - z_i)/(r_j - r_i)
 *         with the nominal layer radii (Eq. sel-cut-delta-lambda);
 *  v[1] = cos(Phi_01) = h_t0 . h_t1 / (r_0 r_1)   (Eq. sel-cut-phi; the garbled "h_{t,k} = r_{r,i}"
 *  v[2] = cos(Phi_12) = h_t1 . h_t2 / (r_1 r_2)    is read as |h_t| = r_i for layer i);
 *  v[3] = r_tc = d01 d12 d20 / (2 [(h0 - h1) x (h2 - h1)]_z)   (Eq. rt-cut), signed:
 *         positive for clockwise turning.  Collinear points give +-inf (or NaN). */
static double cos_phi(const orc_config* c, const double* hi, const double* hj, int li, int lj) {
  return (hi[0] * hj[0] + hi[1] * hj[1]) / (c->r[li] * c->r[lj]);
}

void orc_cut_vars(const orc_config* c, const double* h0, const double* h1, const double* h2, double* v) {
  double tl01 = (h1[2] - h0[2]) / (c->r[1] - c->r[0]);
  double tl12 = (h2[2] - h1[2]) / (c->r[2] - c->r[1]);
  v[0] = tl12 - tl01;
  v[1] = cos_phi(c, h0, h1, 0, 1);
  v[2] = cos_phi(c, h1, h2, 1, 2);
  double d01 = hypot(h0[0] - h1[0], h0[1] - h1[1]);
  double d12 = hypot(h1[0] - h2[0], h1[1] - h2[1]);
  double d20 = hypot(h2[0] - h0[0], h2[1] - h0[1]);
  double cross = (h0[0] - h1[0]) * (h2[1] - h1[1]) - (h0[1] - h1[1]) * (h2[0] - h1[0]);
  v[3] = d01 * d12 * d20 / (2.0 * cross);
}

/* Each cut, inclusive comparisons (the paper prints no strictness). */
static int cut1(const orc_config* c, const double* v) { return fabs(v[0]) <= c->dlambda_max; }
static int cut2(const orc_config* c, const double* v) { return v[1] >= cos(c->phi01_max); }
static int cut3(const orc_config* c, const double* v) { return v[2] >= cos(c->phi12_max); }
static int cut4(const orc_config* c, const double* v) {
  double a = fabs(v[3]);
  return a >= c->rtc_min && a <= c->rtc_max;
}

/* ------------------------------------------------------------------ triplet fit */

/* Centre of the circle through three transverse points. */
static void circumcentre(const double* a, const double* b, const double* p, double* cx, double* cy) {
  double bx = b[0] - a[0], by = b[1] - a[1];
  double px = p[0] - a[0], py = p[1] - a[1];
  double den = 2.0 * (bx * py - by * px);
  double b2 = bx * bx + by * by, p2 = px * px + py * py;
  *cx = a[0] + (py * b2 - by * p2) / den;
  *cy = a[1] + (bx * p2 - px * b2) / den;
}

/* Single triplet fit (Sec. "Single Triplet Fit", Eq. objective-function), hits
 * a -> b -> c with the scattering at b.  The paper linearises chi2 around the
 * solution without transverse kink (a circle through the three hits, radius r_tc)
 * and cites the formulas; they are derived here from the helix relations
 *   chord d = 2 R_t sin(Phi/2),  z = R_t Phi cot(theta),  R_t = R sin(theta),
 * so that for one segment with chord d and length z along the axis the 3D
 * radius R and the turning angle Phi obey R^2 = d^2 / (4 sin^2(Phi/2)) + z^2 / Phi^2.
 * Steps:
 *  1. circle solution: R_t = |r_tc|, turning sense eps = sign(r_tc), per segment
 *     Phi_C = 2 asin(d / 2R_t) (2 pi minus that when the third hit sees the chord
 *     at an obtuse angle: the arc not containing it), R_C = sqrt(R_t^2 + z^2/Phi_C^2),
 *     theta_C = atan2(R_t Phi_C, z);
 *  2. first-order expansion in the common 3D radius R: Phi'(R) = 1/(dR/dPhi),
 *     theta'(R) = dtheta/dPhi * Phi'(R);
 *  3. kink angles Phi_MS = -(eps/2) sum_i (Phi_i(R) - Phi_C,i) ~ alpha R + a0 (the
 *     transverse direction change at b) and Theta_MS = theta_12(R) - theta_01(R)
 *     ~ beta R + b0;
 *  4. chi2(R) = [Phi_MS^2 sin^2(theta) + Theta_MS^2] / sigma_MS^2: sigma_Phi =
 *     sigma_MS / sin(theta) with theta the polar angle (the paper prints sin(lambda),
 *     read as the sine of the polar angle, the mean of the two segment angles);
 *  5. minimum R* = -(alpha a0 s^2 + beta b0)/(alpha^2 s^2 + beta^2) with sigma_MS
 *     frozen at p* = k B R*; sigma_R^2 = sigma_MS^2 / (alpha^2 s^2 + beta^2);
 *     curvature kappa = eps / R*, sigma_kappa = sigma_R / R*^2. */
int orc_fit_triplet(const orc_config* c, const double* ha, const double* hb, const double* hc,
                    int mid_layer, orc_tfit* f) {
  memset(f, 0, sizeof(*f));
  const double* P[3] = {ha, hb, hc};
  double d01 = hypot(ha[0] - hb[0], ha[1] - hb[1]);
  double d12 = hypot(hb[0] - hc[0], hb[1] - hc[1]);
  double d20 = hypot(hc[0] - ha[0], hc[1] - ha[1]);
  double cross = (ha[0] - hb[0]) * (hc[1] - hb[1]) - (ha[1] - hb[1]) * (hc[0] - hb[0]);
  f->rtc = d01 * d12 * d20 / (2.0 * cross);
  if (!(cross != 0.0) || !isfinite(f->rtc) || f->rtc == 0.0) return 0;
  f->Rct = fabs(f->rtc);
  f->eps = f->rtc > 0 ? 1.0 : -1.0;
  circumcentre(ha, hb, hc, &f->cx, &f->cy);
  for (int i = 0; i < 2; i++) {
    const double* s0 = P[i];
    const double* s1 = P[i + 1];
    const double* o = P[i == 0 ? 2 : 0];  /* the third hit */
    double d = hypot(s1[0] - s0[0], s1[1] - s0[1]);
    double z = s1[2] - s0[2];
    double phi = 2.0 * asin(fmin(1.0, d / (2.0 * f->Rct)));
    double dot = (s0[0] - o[0]) * (s1[0] - o[0]) + (s0[1] - o[1]) * (s1[1] - o[1]);
    if (dot < 0) phi = TWO_PI - phi;
    double R = sqrt(f->Rct * f->Rct + z * z / (phi * phi));
    double th = atan2(f->Rct * phi, z);
    double sh = sin(0.5 * phi), ch = cos(0.5 * phi);
    double dRdphi = -(d * d * ch / (8.0 * sh * sh * sh) + z * z / (phi * phi * phi)) / R;
    double dphi = 1.0 / dRdphi;
    double g = phi / (2.0 * sh);
    double gp = (2.0 * sh - phi * ch) / (4.0 * sh * sh);
    double dthdphi = z * d * gp / (z * z + d * d * g * g);
    f->d[i] = d; f->zs[i] = z; f->phiC[i] = phi; f->RC[i] = R; f->thetaC[i] = th;
    f->dphi[i] = dphi; f->dtheta[i] = dthdphi * dphi;
  }
  f->alpha = 0.5 * (f->dphi[0] + f->dphi[1]);
  f->a0 = -0.5 * (f->dphi[0] * f->RC[0] + f->dphi[1] * f->RC[1]);
  f->beta = f->dtheta[1] - f->dtheta[0];
  f->b0 = (f->thetaC[1] - f->thetaC[0]) - f->dtheta[1] * f->RC[1] + f->dtheta[0] * f->RC[0];
  f->s = sin(0.5 * (f->thetaC[0] + f->thetaC[1]));
  double s2 = f->s * f->s;
  double den = f->alpha * f->alpha * s2 + f->beta * f->beta;
  f->Rstar = -(f->alpha * f->a0 * s2 + f->beta * f->b0) / den;
  if (!isfinite(f->Rstar) || !(f->Rstar > 0.0)) return 0;
  double pstar = c->k * field(c) * f->Rstar;
  f->sigma_ms = orc_highland(c, pstar, mid_layer);
  f->sigmaR = f->sigma_ms / sqrt(den);
  f->kappa = f->eps / f->Rstar;
  f->sigma_kappa = f->sigmaR / (f->Rstar * f->Rstar);
  double kp = f->alpha * f->Rstar + f->a0, kt = f->beta * f->Rstar + f->b0;
  f->chi2min = (kp * kp * s2 + kt * kt) / (f->sigma_ms * f->sigma_ms);
  f->valid = isfinite(f->kappa) && isfinite(f->sigma_kappa) && f->sigma_kappa > 0;
  return f->valid;
}

/* chi2 of one fitted triplet at a common 3D radius R with the width of momentum
 * p (Eq. objective-function-global: each triplet's term at the global curvature). */
static double triplet_chi2_at(const orc_config* c, const orc_tfit* f, double R, double p, int mid_layer) {
  double kp = f->alpha * R + f->a0, kt = f->beta * R + f->b0;
  double sg = orc_highland(c, p, mid_layer);
  return (kp * kp * f->s * f->s + kt * kt) / (sg * sg);
}

/* ------------------------------------------------------------------ exact minimiser (pin only) */

/* Turning angle Phi in (0, pi] of a segment with chord d and axial length z on a
 * helix of 3D radius R: the root of d^2/(4 sin^2(Phi/2)) + z^2/Phi^2 = R^2 (which
 * decreases monotonically on (0, pi]); NaN when R is too small for the segment. */
static double seg_phi_of_R(double d, double z, double R) {
  double lo = 1e-12, hi = PI;
  double fhi = d * d / 4.0 + z * z / (PI * PI) - R * R;
  if (fhi > 0) return NAN;
  for (int it = 0; it < 200; it++) {
    double m = 0.5 * (lo + hi);
    double s = sin(0.5 * m);
    double fm = d * d / (4.0 * s * s) + z * z / (m * m) - R * R;
    if (fm > 0) lo = m; else hi = m;
  }
  return 0.5 * (lo + hi);
}

static double exact_chi2(const orc_config* c, const orc_tfit* f, double R, int mid_layer, double p_sig) {
  double ph[2], th[2];
  for (int i = 0; i < 2; i++) {
    ph[i] = seg_phi_of_R(f->d[i], f->zs[i], R);
    if (!isfinite(ph[i])) return INFINITY;
    double Rt = f->d[i] / (2.0 * sin(0.5 * ph[i]));
    th[i] = atan2(Rt * ph[i], f->zs[i]);
  }
  double pms = -0.5 * f->eps * ((ph[0] - f->phiC[0]) + (ph[1] - f->phiC[1]));
  double tms = th[1] - th[0];
  double s = sin(0.5 * (th[0] + th[1]));
  double sg = orc_highland(c, p_sig, mid_layer);
  return (pms * pms * s * s + tms * tms) / (sg * sg);
}

int orc_fit_triplet_exact(const orc_config* c, const double* ha, const double* hb, const double* hc,
                          int mid_layer, double r_lo, double r_hi, double* R_out) {
  orc_tfit f;
  if (!orc_fit_triplet(c, ha, hb, hc, mid_layer, &f)) return -1;
  if (f.phiC[0] > PI || f.phiC[1] > PI) return -1;
  double p_sig = c->k * field(c) * f.Rstar;
  const double gr = 0.5 * (sqrt(5.0) - 1.0);
  double a = r_lo, b = r_hi;
  double x1 = b - gr * (b - a), x2 = a + gr * (b - a);
  double f1 = exact_chi2(c, &f, x1, mid_layer, p_sig), f2 = exact_chi2(c, &f, x2, mid_layer, p_sig);
  for (int it = 0; it < 300; it++) {
    if (f1 < f2) { b = x2; x2 = x1; f2 = f1; x1 = b - gr * (b - a); f1 = exact_chi2(c, &f, x1, mid_layer, p_sig); }
    else { a = x1; x1 = x2; f1 = f2; x2 = a + gr * (b - a); f2 = exact_chi2(c, &f, x2, mid_layer, p_sig); }
  }
  *R_out = 0.5 * (a + b);
  return 0;
}

/* ------------------------------------------------------------------ track reconstruction */

typedef struct {
  double kappa_bar, R_bar, theta01, chi2, p;
  double eps;
  int32_t h0, h1;         /* sorted-hit indices of the layer-0 and layer-1 hits */
} otrack;

/* Global fit of two triplets (Sec. "Triplets Fit"): kappa_bar is the mean of the
 * signed triplet curvatures weighted by 1/sigma_kappa^2 (the signs make triplets
 * that turn in opposite senses fail the chi2 cut); chi2_global is the sum of the
 * two triplets' chi2 evaluated at R_bar = 1/|kappa_bar| with the MS width of
 * p_bar = k B R_bar.  theta01 is the first segment's polar angle at R_bar from the
 * linear model of triplet 1. */
static int global_fit(const orc_config* c, const orc_tfit* t1, const orc_tfit* t2, orc_track_rec* r) {
  double w1 = 1.0 / (t1->sigma_kappa * t1->sigma_kappa);
  double w2 = 1.0 / (t2->sigma_kappa * t2->sigma_kappa);
  double kb = (t1->kappa * w1 + t2->kappa * w2) / (w1 + w2);
  r->kappa1 = t1->kappa; r->kappa2 = t2->kappa; r->sk1 = t1->sigma_kappa; r->sk2 = t2->sigma_kappa;
  r->kappa_bar = kb;
  if (!(kb != 0.0) || !isfinite(kb)) return 0;
  double Rb = 1.0 / fabs(kb);
  double pb = c->k * field(c) * Rb;
  r->R_bar = Rb;
  r->theta01 = t1->thetaC[0] + t1->dtheta[0] * (Rb - t1->RC[0]);
  r->chi2 = triplet_chi2_at(c, t1, Rb, pb, 1) + triplet_chi2_at(c, t2, Rb, pb, 2);
  return isfinite(r->chi2);
}

/* Track reconstruction of one selected triplet (Sec. "Triplets Fit", Algorithm 3):
 * fit (h0,h1,h2); estimate the layer-3 point from that helix; take the closest
 * layer-3 hit; fit (h1,h2,h3); global fit; keep if chi2 < chi2_track_max.
 *  - Estimated point: the circle through h0,h1,h2 (centre c, radius |r_tc|) meets the
 *    layer-3 cylinder; the first crossing reached from h2 in the turning sense; its z
 *    follows the second segment's polar angle: z3 = z2 + R_t * dPhi * cot(theta_C12).
 *  - Closest hit: smallest (r3 dphi)^2 + dz^2 on the cylinder surface, ties to the
 *    smaller address (the paper names no window; the chi2 cut rejects far hits). */
static void build_track(const orc_config* c, const orc_hit* H, const int32_t* lay_start,
                        int i0, int i1, int i2, orc_track_rec* r, otrack* out) {
  memset(r, 0, sizeof(*r));
  r->i[0] = H[i0].in_idx; r->i[1] = H[i1].in_idx; r->i[2] = H[i2].in_idx; r->i[3] = -1;
  r->m_best = INFINITY; r->m_second = INFINITY;
  double p0[3] = {H[i0].x, H[i0].y, H[i0].z};
  double p1[3] = {H[i1].x, H[i1].y, H[i1].z};
  double p2[3] = {H[i2].x, H[i2].y, H[i2].z};
  orc_tfit t1, t2;
  if (!orc_fit_triplet(c, p0, p1, p2, 1, &t1)) { r->status = 0; return; }
  /* crossing of the triplet circle with r = r3 */
  double r3 = c->r[3];
  double D = hypot(t1.cx, t1.cy);
  if (!(D > 0) || D > t1.Rct + r3 || D < fabs(t1.Rct - r3)) { r->status = 1; return; }
  double a = (r3 * r3 - t1.Rct * t1.Rct + D * D) / (2.0 * D);
  double hh = sqrt(fmax(r3 * r3 - a * a, 0.0));
  double ux = t1.cx / D, uy = t1.cy / D;
  double q[2][2] = {{a * ux - hh * uy, a * uy + hh * ux}, {a * ux + hh * uy, a * uy - hh * ux}};
  double a2 = atan2(p2[1] - t1.cy, p2[0] - t1.cx);
  double best_al = INFINITY, px = 0, py = 0;
  for (int k = 0; k < 2; k++) {
    double al = wrap_2pi(t1.eps * (a2 - atan2(q[k][1] - t1.cy, q[k][0] - t1.cx)));
    if (al < best_al) { best_al = al; px = q[k][0]; py = q[k][1]; }
  }
  double th12 = t1.thetaC[1];
  double z3 = p2[2] + t1.Rct * best_al * cos(th12) / sin(th12);
  double phi3 = atan2(py, px);
  int best = -1;
  for (int j = lay_start[3]; j < lay_start[4]; j++) {
    double dphi = wrap_pi(atan2(H[j].y, H[j].x) - phi3);
    double dz = H[j].z - z3;
    double m = (r3 * dphi) * (r3 * dphi) + dz * dz;
    if (best < 0 || m < r->m_best || (m == r->m_best && H[j].addr < H[best].addr)) { best = j; r->m_best = m; }
  }
  if (best < 0) { r->status = 2; return; }
  for (int j = lay_start[3]; j < lay_start[4]; j++) {  /* runner-up among other pixels */
    if (H[j].addr == H[best].addr) continue;
    double dphi = wrap_pi(atan2(H[j].y, H[j].x) - phi3);
    double dz = H[j].z - z3;
    r->m_second = fmin(r->m_second, (r3 * dphi) * (r3 * dphi) + dz * dz);
  }
  r->i[3] = H[best].in_idx;
  double p3[3] = {H[best].x, H[best].y, H[best].z};
  if (!orc_fit_triplet(c, p1, p2, p3, 2, &t2)) { r->status = 3; return; }
  if (!global_fit(c, &t1, &t2, r)) { r->status = 3; return; }
  if (!(r->chi2 < c->chi2_track_max)) { r->status = 4; return; }
  r->status = 5;
  out->kappa_bar = r->kappa_bar; out->R_bar = r->R_bar; out->theta01 = r->theta01;
  out->chi2 = r->chi2; out->p = c->k * field(c) * r->R_bar;
  out->eps = r->kappa_bar > 0 ? 1.0 : -1.0;
  out->h0 = i0; out->h1 = i1;
}

/* ------------------------------------------------------------------ vertex fit */

typedef struct {
  double cx, cy, rt;       /* transverse circle */
  double R, ct, st, p, eps, sms;
  double h0[3];
} vtrack;

/* Transverse circle of a track (Sec. "Vertex Fit"): radius r_t = 1/kappa_t, i.e. the
 * transverse radius R_bar sin(theta01) of the fitted helix, through the layer-0 and
 * layer-1 hits, centre on the side the track turns to (right for clockwise). */
static void make_vtrack(const orc_config* c, const orc_hit* H, const otrack* t, vtrack* v) {
  const orc_hit* a = &H[t->h0];
  const orc_hit* b = &H[t->h1];
  v->R = t->R_bar; v->ct = cos(t->theta01); v->st = sin(t->theta01);
  v->rt = t->R_bar * v->st; v->p = t->p; v->eps = t->eps;
  v->sms = orc_highland(c, t->p, 0);
  v->h0[0] = a->x; v->h0[1] = a->y; v->h0[2] = a->z;
  double dx = b->x - a->x, dy = b->y - a->y;
  double d = hypot(dx, dy);
  double ux = dx / d, uy = dy / d;
  double off = sqrt(fmax(v->rt * v->rt - 0.25 * d * d, 0.0));
  double mx = 0.5 * (a->x + b->x), my = 0.5 * (a->y + b->y);
  /* left normal (-uy, ux); clockwise (eps = +1) puts the centre on the right */
  v->cx = mx - v->eps * (-uy) * off;
  v->cy = my - v->eps * ux * off;
}

/* Turning angle travelled from point (x,y) forward to the layer-0 hit, in [0, 2 pi). */
static double arc_to_h0(const vtrack* v, double x, double y) {
  double ap = atan2(y - v->cy, x - v->cx);
  double ah = atan2(v->h0[1] - v->cy, v->h0[0] - v->cx);
  return wrap_2pi(v->eps * (ap - ah));
}

/* Track error at a point (Eq. track-error): sigma^2 = sigma_MS^2 s^2 + sigma_pixel^2 with
 * s the transverse path length from the layer-0 hit; the printed "+ sigma_Pixel" is
 * read as the squared pixel resolution pitch^2/12. */
static double point_var(const orc_config* c, const vtrack* v, double x, double y) {
  double s = v->rt * arc_to_h0(v, x, y);
  return v->sms * v->sms * s * s + c->pitch * c->pitch / 12.0;
}

/* Distance from (rho, |z|) to the target surface, the generating segment
 * (target_r, 0)-(0, target_half_len) of the hollow double cone. */
static double target_distance(const orc_config* c, double x, double y, double z) {
  double px = hypot(x, y), pz = fabs(z);
  double ax = c->target_r, az = 0.0, bx = 0.0, bz = c->target_half_len;
  double ex = bx - ax, ez = bz - az;
  double t = ((px - ax) * ex + (pz - az) * ez) / (ex * ex + ez * ez);
  t = fmin(1.0, fmax(0.0, t));
  return hypot(px - (ax + t * ex), pz - (az + t * ez));
}

/* Vertex of one e+ e+ e- combination (Sec. "Vertex Fit", "Signal Estimation").
 *  1. Circle-circle intersections of the three track pairs; a pair that does not
 *     intersect skips the combination (a tangent pair gives one point).
 *  2. Points farther than target_r + isect_margin from the axis are dropped (the
 *     19 mm target disk); a pair left without points skips the combination.
 *  3. For every choice of one point per pair (<= 8): mu_t = sum(p_i/sigma_i^2) /
 *     sum(1/sigma_i^2) (the printed sum to 3 is read as the three pairs), the error of a
 *     point on two tracks being the sum of both tracks' errors.
 *  4. Closest point of each circle to mu_t; turning angle dPhi back to the layer-0 hit;
 *     z_i = z_h0 - dPhi sin(lambda01)/kappa = z_h0 - dPhi R cos(theta01); errors again
 *     by Eq. track-error; mu_z the error-weighted mean of the z_i.
 *  5. chi2 = sum_i |(p_ca,i, z_i) - mu|^2 / sigma_i^2 (the printed "mu_i/sigma_i^2" read as
 *     the squared distance); the choice with the smallest chi2 is the vertex.
 *  6. Signal cuts at that vertex: chi2 <= vtx_chi2_max, distance to the target surface
 *     <= target_dist_max (Algorithm 4 prints the comparison inverted; read as reject
 *     when too far), |sum of momenta at the closest points| <= ptot_max. */
static void vertex_combination(const orc_config* c, const vtrack* V[3], orc_combo_rec* rec) {
  static const int pr[3][2] = {{0, 1}, {0, 2}, {1, 2}};
  double pts[3][2][2], var[3][2];
  int npt[3];
  rec->status = 2; rec->pass = 0;
  rec->chi2 = INFINITY; rec->chi2_second = INFINITY; rec->tdist = INFINITY; rec->ptot = INFINITY;
  rec->disc_min = INFINITY; rec->filt_margin = INFINITY;
  double lim = c->target_r + c->isect_margin;
  /* Diagnostics for a comparison with another implementation (no decision uses
   * them): over all three pairs, whatever the status, the smallest squared half
   * chord relative to the product of the two radii (how close a pair is to not
   * meeting) and the smallest distance of an intersection point from the filter
   * radius.  Both are symmetric in the tracks, hence independent of their order. */
  for (int k = 0; k < 3; k++) {
    const vtrack* A = V[pr[k][0]];
    const vtrack* B = V[pr[k][1]];
    double ex = B->cx - A->cx, ey = B->cy - A->cy;
    double D = hypot(ex, ey);
    if (!(D > 0)) continue;
    double a = (A->rt * A->rt - B->rt * B->rt + D * D) / (2.0 * D);
    double h2 = A->rt * A->rt - a * a;
    rec->disc_min = fmin(rec->disc_min, fabs(h2) / (A->rt * B->rt));
    if (h2 < 0) continue;
    double h = sqrt(h2), bx = A->cx + a * ex / D, by = A->cy + a * ey / D;
    rec->filt_margin = fmin(rec->filt_margin, fabs(hypot(bx - h * ey / D, by + h * ex / D) - lim));
    if (h2 > 0) rec->filt_margin = fmin(rec->filt_margin, fabs(hypot(bx + h * ey / D, by - h * ex / D) - lim));
  }
  for (int k = 0; k < 3; k++) {
    const vtrack* A = V[pr[k][0]];
    const vtrack* B = V[pr[k][1]];
    double ex = B->cx - A->cx, ey = B->cy - A->cy;
    double D = hypot(ex, ey);
    npt[k] = 0;
    if (!(D > 0)) { rec->status = 0; return; }
    double a = (A->rt * A->rt - B->rt * B->rt + D * D) / (2.0 * D);
    double h2 = A->rt * A->rt - a * a;
    if (h2 < 0) { rec->status = 0; return; }
    ex /= D; ey /= D;
    double bx = A->cx + a * ex, by = A->cy + a * ey;
    double cand[2][2];
    int nc;
    if (h2 == 0) { cand[0][0] = bx; cand[0][1] = by; nc = 1; }
    else {
      double h = sqrt(h2);
      cand[0][0] = bx - h * ey; cand[0][1] = by + h * ex;
      cand[1][0] = bx + h * ey; cand[1][1] = by - h * ex;
      nc = 2;
    }
    for (int j = 0; j < nc; j++) {
      double rr = hypot(cand[j][0], cand[j][1]);
      if (rr > lim) continue;
      pts[k][npt[k]][0] = cand[j][0]; pts[k][npt[k]][1] = cand[j][1];
      var[k][npt[k]] = point_var(c, A, cand[j][0], cand[j][1]) + point_var(c, B, cand[j][0], cand[j][1]);
      npt[k]++;
    }
  }
  for (int k = 0; k < 3; k++)
    if (npt[k] == 0) { rec->status = 1; return; }
  double best_mu[3] = {0, 0, 0}, best_pca[3][2];
  for (int s0 = 0; s0 < npt[0]; s0++)
    for (int s1 = 0; s1 < npt[1]; s1++)
      for (int s2 = 0; s2 < npt[2]; s2++) {
        int sel[3] = {s0, s1, s2};
        double wx = 0, wy = 0, ws = 0;
        for (int k = 0; k < 3; k++) {
          wx += pts[k][sel[k]][0] / var[k][sel[k]];
          wy += pts[k][sel[k]][1] / var[k][sel[k]];
          ws += 1.0 / var[k][sel[k]];
        }
        double mx = wx / ws, my = wy / ws;
        double pca[3][2], zi[3], vi[3];
        int bad = 0;
        double wz = 0, wzs = 0;
        for (int i = 0; i < 3; i++) {
          double dx = mx - V[i]->cx, dy = my - V[i]->cy;
          double dn = hypot(dx, dy);
          if (!(dn > 0)) { bad = 1; break; }
          pca[i][0] = V[i]->cx + V[i]->rt * dx / dn;
          pca[i][1] = V[i]->cy + V[i]->rt * dy / dn;
          double dphi = arc_to_h0(V[i], pca[i][0], pca[i][1]);
          zi[i] = V[i]->h0[2] - dphi * V[i]->R * V[i]->ct;
          double s = V[i]->rt * dphi;
          vi[i] = V[i]->sms * V[i]->sms * s * s + c->pitch * c->pitch / 12.0;
          wz += zi[i] / vi[i]; wzs += 1.0 / vi[i];
        }
        if (bad) continue;
        double mz = wz / wzs;
        double chi2 = 0;
        for (int i = 0; i < 3; i++) {
          double dx = pca[i][0] - mx, dy = pca[i][1] - my, dz = zi[i] - mz;
          chi2 += (dx * dx + dy * dy + dz * dz) / vi[i];
        }
        if (chi2 < rec->chi2) {
          rec->chi2_second = rec->chi2;
          rec->chi2 = chi2;
          best_mu[0] = mx; best_mu[1] = my; best_mu[2] = mz;
          for (int i = 0; i < 3; i++) { best_pca[i][0] = pca[i][0]; best_pca[i][1] = pca[i][1]; }
        } else if (chi2 < rec->chi2_second) {
          rec->chi2_second = chi2;
        }
      }
  if (!isfinite(rec->chi2)) { rec->status = 1; return; }
  rec->mu[0] = best_mu[0]; rec->mu[1] = best_mu[1]; rec->mu[2] = best_mu[2];
  rec->tdist = target_distance(c, best_mu[0], best_mu[1], best_mu[2]);
  double P[3] = {0, 0, 0};
  for (int i = 0; i < 3; i++) {
    double ux = (best_pca[i][0] - V[i]->cx) / V[i]->rt;
    double uy = (best_pca[i][1] - V[i]->cy) / V[i]->rt;
    double tx = V[i]->eps * uy, ty = -V[i]->eps * ux;  /* direction of travel */
    rec->pvec[i][0] = V[i]->p * V[i]->st * tx;
    rec->pvec[i][1] = V[i]->p * V[i]->st * ty;
    rec->pvec[i][2] = V[i]->p * V[i]->ct;
    for (int k = 0; k < 3; k++) P[k] += rec->pvec[i][k];
  }
  rec->ptot = sqrt(P[0] * P[0] + P[1] * P[1] + P[2] * P[2]);
  rec->pass = rec->chi2 <= c->vtx_chi2_max && rec->tdist <= c->target_dist_max && rec->ptot <= c->ptot_max;
}

/* ------------------------------------------------------------------ one frame */

typedef struct {
  orc_hit* H;
  int32_t* trip;        /* kept triplets, 3 sorted-hit indices each */
  otrack* trk;
  int32_t* combo;       /* 3 kept-track indices each */
  double* combo_de;
  size_t cap_trip, cap_trk, cap_combo;
} orc_work;

static int grow(void** p, size_t* cap, size_t need, size_t elem) {
  if (need <= *cap) return 0;
  size_t n = *cap ? *cap : 64;
  while (n < need) n *= 2;
  void* q = realloc(*p, n * elem);
  if (!q) return -1;
  *p = q; *cap = n;
  return 0;
}

static void work_free(orc_work* w) {
  free(w->H); free(w->trip); free(w->trk); free(w->combo); free(w->combo_de);
  memset(w, 0, sizeof(*w));
}

/* Algorithm 1 for one frame: load, selection cuts (Algorithm 2), track
 * reconstruction (Algorithm 3), vertex fit (Algorithm 4), store.  A frame whose
 * triplets, tracks or combinations exceed the caps is kept without further
 * processing ("higher than 768" read as: 769 or more overflow).  A frame with an
 * address outside the detector is kept with reason ERR_BADHIT; a frame with more
 * hits than max_hits (the staging capacity) is kept with reason HIT_OVERFLOW. */
static int select_frame_w(const orc_config* c, const int32_t* addrs, const orc_hit* given, int32_t n,
                          orc_frame_out* out, orc_work* w, int64_t* cnt) {
  int32_t trips_cap = out->trips_cap, trks_cap = out->trks_cap, kept_cap = out->kept_cap,
          combos_cap = out->combos_cap;
  orc_trip_rec* trips = out->trips;
  orc_track_rec* trks = out->trks;
  int32_t* kept_trk = out->kept_trk;
  orc_combo_rec* combos = out->combos;
  memset(out, 0, sizeof(*out));
  out->trips = trips; out->trips_cap = trips_cap;
  out->trks = trks; out->trks_cap = trks_cap;
  out->kept_trk = kept_trk; out->kept_cap = kept_cap;
  out->combos = combos; out->combos_cap = combos_cap;
  out->n_hits = n;
  if (cnt) { for (int i = 0; i < 8; i++) cnt[i] = 0; cnt[0] = n; }
  /* load: decode every hit (or take the caller's decoded hits) */
  free(w->H);
  w->H = (orc_hit*)malloc(sizeof(orc_hit) * (size_t)(n > 0 ? n : 1));
  if (!w->H) return -1;
  for (int i = 0; i < n; i++) {
    if (given) { w->H[i] = given[i]; }
    else if (orc_decode(c, (uint32_t)addrs[i], &w->H[i]) != 0) {
      out->reason = ORC_ERR_BADHIT; out->keep = 1;
      return 0;
    }
    w->H[i].in_idx = i;
  }
  if (n > c->max_hits) { out->reason = ORC_HIT_OVERFLOW; out->keep = 1; return 0; }
  qsort(w->H, (size_t)n, sizeof(orc_hit), cmp_hit);
  int32_t ls[5] = {0, 0, 0, 0, 0};
  for (int i = 0; i < n; i++) out->n_layer[w->H[i].layer]++;
  for (int L = 0; L < 4; L++) ls[L + 1] = ls[L] + out->n_layer[L];
  const orc_hit* H = w->H;

  /* ---- selection cuts: every triplet of layers 0, 1, 2 */
  out->n_tested = (int64_t)out->n_layer[0] * out->n_layer[1] * out->n_layer[2];
  int64_t ntrip = 0;
  for (int a = ls[0]; a < ls[1]; a++)
    for (int b = ls[1]; b < ls[2]; b++)
      for (int d = ls[2]; d < ls[3]; d++) {
        double h0[3] = {H[a].x, H[a].y, H[a].z}, h1[3] = {H[b].x, H[b].y, H[b].z},
               h2[3] = {H[d].x, H[d].y, H[d].z};
        double v[4];
        orc_cut_vars(c, h0, h1, h2, v);
        int p1 = cut1(c, v), p2 = cut2(c, v), p3 = cut3(c, v), p4 = cut4(c, v);
        if (p1) out->n_pass[0]++;
        if (p1 && p2) out->n_pass[1]++;
        if (p1 && p2 && p3) out->n_pass[2]++;
        if (!(p1 && p2 && p3 && p4)) continue;
        out->n_pass[3]++;
        if (ntrip < c->max_triplets) {
          if (grow((void**)&w->trip, &w->cap_trip, (size_t)(ntrip + 1) * 3, sizeof(int32_t))) return -1;
          w->trip[3 * ntrip] = a; w->trip[3 * ntrip + 1] = b; w->trip[3 * ntrip + 2] = d;
          if (out->trips && ntrip < out->trips_cap) {
            orc_trip_rec* r = &out->trips[ntrip];
            r->i[0] = H[a].in_idx; r->i[1] = H[b].in_idx; r->i[2] = H[d].in_idx;
            r->dlambda = v[0]; r->cos01 = v[1]; r->cos12 = v[2]; r->rtc = v[3];
            out->trips_n = (int32_t)(ntrip + 1);
          }
        }
        ntrip++;
      }
  out->n_triplets = (int32_t)(ntrip > 0x7fffffff ? 0x7fffffff : ntrip);
  if (cnt) {
    /* algorithmic work after the pair cuts: sum over layer-1 hits of the products of
     * the layer-0 and layer-2 partners that pass the two Phi cuts */
    int64_t T = 0;
    for (int b = ls[1]; b < ls[2]; b++) {
      int64_t n0 = 0, n2 = 0;
      double h1[3] = {H[b].x, H[b].y, H[b].z};
      for (int a = ls[0]; a < ls[1]; a++) {
        double h0[3] = {H[a].x, H[a].y, H[a].z};
        n0 += cos_phi(c, h0, h1, 0, 1) >= cos(c->phi01_max);
      }
      for (int d = ls[2]; d < ls[3]; d++) {
        double h2[3] = {H[d].x, H[d].y, H[d].z};
        n2 += cos_phi(c, h1, h2, 1, 2) >= cos(c->phi12_max);
      }
      T += n0 * n2;
    }
    cnt[1] = (int64_t)out->n_layer[0] * out->n_layer[1] + (int64_t)out->n_layer[1] * out->n_layer[2];
    cnt[2] = T;
    cnt[3] = ntrip;
  }
  if (ntrip > c->max_triplets) { out->reason = ORC_TRIPLET_OVERFLOW; out->keep = 1; return 0; }

  /* ---- track reconstruction: every kept triplet */
  int ntrk = 0;
  for (int t = 0; t < ntrip; t++) {
    orc_track_rec rec;
    otrack tk;
    build_track(c, H, ls, w->trip[3 * t], w->trip[3 * t + 1], w->trip[3 * t + 2], &rec, &tk);
    if (out->trks && t < out->trks_cap) { out->trks[t] = rec; out->trks_n = t + 1; }
    if (rec.status != 5) continue;
    if (grow((void**)&w->trk, &w->cap_trk, (size_t)ntrk + 1, sizeof(otrack))) return -1;
    w->trk[ntrk] = tk;
    if (out->kept_trk && ntrk < out->kept_cap) { out->kept_trk[ntrk] = t; out->kept_n = ntrk + 1; }
    ntrk++;
  }
  out->n_tracks = ntrk;
  if (cnt) cnt[4] = ntrk;
  if (ntrk > c->max_tracks) { out->reason = ORC_TRACK_OVERFLOW; out->keep = 1; return 0; }

  /* ---- vertex fit, part 1: energy test of every e+ e+ e- combination */
  int64_t ncombo = 0, netest = 0;
  for (int a = 0; a < ntrk; a++) {
    if (!(w->trk[a].eps > 0)) continue;
    for (int b = a + 1; b < ntrk; b++) {
      if (!(w->trk[b].eps > 0)) continue;
      for (int e = 0; e < ntrk; e++) {
        if (!(w->trk[e].eps < 0)) continue;
        netest++;
        double me = c->m_e;
        double E = sqrt(w->trk[a].p * w->trk[a].p + me * me) + sqrt(w->trk[b].p * w->trk[b].p + me * me)
                 + sqrt(w->trk[e].p * w->trk[e].p + me * me);
        double de = E - c->m_mu;
        if (!(fabs(de) <= c->e_window)) continue;
        if (ncombo < c->max_combos) {
          if (grow((void**)&w->combo, &w->cap_combo, (size_t)(ncombo + 1) * 3, sizeof(int32_t))) return -1;
          size_t cap_de = w->cap_combo / 3;
          double* q = (double*)realloc(w->combo_de, cap_de * sizeof(double));
          if (!q) return -1;
          w->combo_de = q;
          w->combo[3 * ncombo] = a; w->combo[3 * ncombo + 1] = b; w->combo[3 * ncombo + 2] = e;
          w->combo_de[ncombo] = de;
        }
        ncombo++;
      }
    }
  }
  out->n_combos = (int32_t)(ncombo > 0x7fffffff ? 0x7fffffff : ncombo);
  if (cnt) { cnt[5] = netest; cnt[6] = ncombo; }
  if (ncombo > c->max_combos) { out->reason = ORC_COMBO_OVERFLOW; out->keep = 1; return 0; }

  /* ---- vertex fit, part 2: every combination (Algorithm 4 keeps the frame when any
   * combination passes; the text's single smallest-chi2 vertex is recorded too) */
  int found = 0;
  for (int k = 0; k < ncombo; k++) {
    vtrack va, vb, ve;
    make_vtrack(c, H, &w->trk[w->combo[3 * k]], &va);
    make_vtrack(c, H, &w->trk[w->combo[3 * k + 1]], &vb);
    make_vtrack(c, H, &w->trk[w->combo[3 * k + 2]], &ve);
    const vtrack* V[3] = {&va, &vb, &ve};
    orc_combo_rec rec;
    memset(&rec, 0, sizeof(rec));
    rec.t[0] = w->combo[3 * k]; rec.t[1] = w->combo[3 * k + 1]; rec.t[2] = w->combo[3 * k + 2];
    rec.de = w->combo_de[k];
    vertex_combination(c, V, &rec);
    if (rec.status == 2) out->n_vertexed++;
    if (rec.pass) found = 1;
    if (out->combos && k < out->combos_cap) { out->combos[k] = rec; out->combos_n = k + 1; }
  }
  if (cnt) cnt[7] = out->n_vertexed;
  out->reason = found ? ORC_VERTEX : ORC_DROP;
  out->keep = found;
  return 0;
}

int orc_select_frame(const orc_config* c, const int32_t* addrs, int32_t n, orc_frame_out* out) {
  orc_work w;
  memset(&w, 0, sizeof(w));
  int rc = select_frame_w(c, addrs, NULL, n, out, &w, NULL);
  work_free(&w);
  return rc;
}

/* The same selection on caller-decoded hits (FP64 positions, for the closed-form
 * pins with digitisation switched off).  The order key is hits[i].addr. */
int orc_select_frame_hits(const orc_config* c, const orc_hit* hits, int32_t n, orc_frame_out* out) {
  orc_work w;
  memset(&w, 0, sizeof(w));
  int rc = select_frame_w(c, NULL, hits, n, out, &w, NULL);
  work_free(&w);
  return rc;
}

/* Track fit from FP64 positions (layers 0..3), for the exact-recovery pin. */
int orc_fit_track_positions(const orc_config* c, const double* h, double* out) {
  orc_tfit t1, t2;
  orc_track_rec r;
  memset(&r, 0, sizeof(r));
  if (!orc_fit_triplet(c, h, h + 3, h + 6, 1, &t1)) return -1;
  if (!orc_fit_triplet(c, h + 3, h + 6, h + 9, 2, &t2)) return -1;
  if (!global_fit(c, &t1, &t2, &r)) return -1;
  out[0] = r.kappa_bar; out[1] = r.R_bar; out[2] = r.theta01; out[3] = r.chi2;
  return 0;
}

/* ------------------------------------------------------------------ batch */

typedef struct {
  const orc_config* c;
  const int32_t* hits;
  const int64_t* off;
  int64_t f0, f1;
  uint8_t *keep, *reason;
  int64_t* counts;
  int rc;
} orc_job;

static void* run_job(void* p) {
  orc_job* j = (orc_job*)p;
  orc_work w;
  memset(&w, 0, sizeof(w));
  for (int64_t f = j->f0; f < j->f1; f++) {
    orc_frame_out o;
    memset(&o, 0, sizeof(o));
    int64_t a = j->off[f], b = j->off[f + 1];
    if (select_frame_w(j->c, j->hits + a, NULL, (int32_t)(b - a), &o, &w, j->counts ? j->counts + 8 * f : NULL)) {
      j->rc = -1;
      break;
    }
    j->keep[f] = (uint8_t)o.keep;
    j->reason[f] = (uint8_t)o.reason;
  }
  work_free(&w);
  return NULL;
}

/* Frames are independent (Sec. "Parallelization"): threads take disjoint
 * contiguous frame ranges.  counts, when given, receives 8 int64 per frame:
 * hits, pair tests n0*n1 + n1*n2, triplet tests after the two Phi cuts, kept
 * triplets, kept tracks, energy tests, combinations, vertexed combinations. */
int orc_select_frames(const orc_config* c, const int32_t* hits, const int64_t* off, int64_t n_frames,
                      uint8_t* keep, uint8_t* reason, int32_t n_threads, int64_t* counts) {
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  if (n_threads > n_frames) n_threads = (int32_t)(n_frames > 0 ? n_frames : 1);
  pthread_t th[256];
  orc_job jobs[256];
  for (int t = 0; t < n_threads; t++) {
    jobs[t].c = c; jobs[t].hits = hits; jobs[t].off = off;
    jobs[t].f0 = n_frames * t / n_threads; jobs[t].f1 = n_frames * (t + 1) / n_threads;
    jobs[t].keep = keep; jobs[t].reason = reason; jobs[t].counts = counts; jobs[t].rc = 0;
  }
  if (n_threads == 1) { run_job(&jobs[0]); return jobs[0].rc; }
  for (int t = 0; t < n_threads; t++) pthread_create(&th[t], NULL, run_job, &jobs[t]);
  int rc = 0;
  for (int t = 0; t < n_threads; t++) { pthread_join(th[t], NULL); rc |= jobs[t].rc; }
  return rc;
}

/* ------------------------------------------------------------------ alignment and fit chi2 */

/* R = Rz(wz) Ry(wy) Rx(wx), row-major. */
static void rotation(const double* w, double* R) {
  const double cx = cos(w[0]), sx = sin(w[0]), cy = cos(w[1]), sy = sin(w[1]), cz = cos(w[2]), sz = sin(w[2]);
  const double Rx[9] = {1, 0, 0, 0, cx, -sx, 0, sx, cx};
  const double Ry[9] = {cy, 0, sy, 0, 1, 0, -sy, 0, cy};
  const double Rz[9] = {cz, -sz, 0, sz, cz, 0, 0, 0, 1};
  double T[9];
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      T[3 * i + j] = 0;
      for (int k = 0; k < 3; k++) T[3 * i + j] += Ry[3 * i + k] * Rx[3 * k + j];
    }
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      R[3 * i + j] = 0;
      for (int k = 0; k < 3; k++) R[3 * i + j] += Rz[3 * i + k] * T[3 * k + j];
    }
}

void orc_align_point(const double* p6, const double* xn, double* x) {
  double R[9];
  rotation(p6 + 3, R);
  for (int i = 0; i < 3; i++) x[i] = R[3 * i] * xn[0] + R[3 * i + 1] * xn[1] + R[3 * i + 2] * xn[2] + p6[i];
}

static double fit_chi2_one(const orc_config* c, const int32_t* hits, int64_t n_hits, const int32_t* q,
                           const double* params) {
  double h[12];
  for (int L = 0; L < 4; L++) {
    orc_hit d;
    if (q[L] < 0 || q[L] >= n_hits || orc_decode(c, (uint32_t)hits[q[L]], &d) != 0 || d.layer != L) return NAN;
    const double xn[3] = {d.x, d.y, d.z};
    orc_align_point(params + 6 * L, xn, h + 3 * L);
  }
  double out[4];
  if (orc_fit_track_positions(c, h, out) != 0 || !isfinite(out[3])) return NAN;
  return out[3];
}

typedef struct {
  const orc_config* c;
  const int32_t* hits;
  int64_t n_hits;
  const int32_t* cand;
  int64_t k0, k1;
  const double* params;
  double* chi2;
  int64_t n_ok;
} orc_fit_job;

static void* run_fit_job(void* p) {
  orc_fit_job* j = (orc_fit_job*)p;
  for (int64_t k = j->k0; k < j->k1; k++) {
    j->chi2[k] = fit_chi2_one(j->c, j->hits, j->n_hits, j->cand + 4 * k, j->params);
    j->n_ok += isfinite(j->chi2[k]);
  }
  return NULL;
}

int64_t orc_fit_chi2(const orc_config* c, const int32_t* hits, int64_t n_hits, const int32_t* cand, int64_t n_cand,
                     const double* params, double* chi2, int32_t n_threads) {
  orc_config cs = *c;
  cs.field_scale = c->field_scale * params[24];
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  pthread_t th[256];
  orc_fit_job jobs[256];
  for (int t = 0; t < n_threads; t++) {
    jobs[t].c = &cs; jobs[t].hits = hits; jobs[t].n_hits = n_hits; jobs[t].cand = cand;
    jobs[t].k0 = n_cand * t / n_threads; jobs[t].k1 = n_cand * (t + 1) / n_threads;
    jobs[t].params = params; jobs[t].chi2 = chi2; jobs[t].n_ok = 0;
    if (n_threads > 1) pthread_create(&th[t], NULL, run_fit_job, &jobs[t]);
    else run_fit_job(&jobs[t]);
  }
  int64_t n_ok = 0;
  for (int t = 0; t < n_threads; t++) {
    if (n_threads > 1) pthread_join(th[t], NULL);
    n_ok += jobs[t].n_ok;
  }
  return n_ok;
}
