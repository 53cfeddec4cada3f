/* FP64 CPU oracle of the Mu3e online event selection (arXiv:2206.11535).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library.  It shares no code, header,
 * table or helper with the CUDA library; both read the same JSON parameters.
 *
 * Units: mm, MeV, T, rad.  Hits are packed int32 pixel addresses:
 *   [31:28] zero, [27:26] layer, [25:21] ladder, [20:13] column, [12:0] row.
 * Indices in the record structs below are INPUT indices: the position of the hit
 * inside its frame's packet, so that they can be compared with any other
 * implementation regardless of its internal hit order.
 */
#ifndef M3E_ORACLE_H
#define M3E_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  double r[4], H[4];
  int32_t nlad[4], ncol[4], nrow[4];
  double pitch;
  double B, field_scale, x_over_X0[4];
  double k, m_mu, m_e;
  double target_r, target_half_len;
  double dlambda_max, phi01_max, phi12_max, rtc_min, rtc_max, chi2_track_max;
  double e_window, isect_margin, vtx_chi2_max, target_dist_max, ptot_max;
  int32_t max_hits, max_triplets, max_tracks, max_combos;
} orc_config;

enum { ORC_DROP = 0, ORC_VERTEX = 1, ORC_TRIPLET_OVERFLOW = 2, ORC_TRACK_OVERFLOW = 3,
       ORC_COMBO_OVERFLOW = 4, ORC_HIT_OVERFLOW = 5, ORC_ERR_BADHIT = 6 };

typedef struct {          /* one decoded hit */
  double x, y, z;
  int32_t layer, ladder, col, row;
  uint32_t addr;
  int32_t in_idx;
  double phi;             /* azimuth of the pixel column centre, [0, 2 pi) (decode only) */
} orc_hit;

typedef struct {          /* result of the single triplet fit (Sec. Track Reconstruction) */
  int32_t valid;
  double rtc, Rct, eps, cx, cy;           /* circle through the three hits (transverse) */
  double d[2], zs[2], phiC[2], RC[2], thetaC[2], dphi[2], dtheta[2];
  double alpha, a0, beta, b0, s;           /* linear kink model and sin(mean polar angle) */
  double Rstar, sigmaR, kappa, sigma_kappa, chi2min, sigma_ms;
} orc_tfit;

typedef struct {          /* kept triplet (selection cuts) */
  int32_t i[3];
  double dlambda, cos01, cos12, rtc;
} orc_trip_rec;

typedef struct {          /* track reconstruction of one kept triplet */
  int32_t i[4];           /* i[3] = chosen layer-3 hit or -1 */
  int32_t status;         /* 0 fit1 invalid, 1 no layer-3 crossing, 2 no layer-3 hit,
                             3 fit2 invalid, 4 chi2 >= cut, 5 kept */
  double m_best, m_second;/* 4th-hit metric of the winner and of the best other address */
  double kappa1, kappa2, sk1, sk2, kappa_bar, R_bar, theta01, chi2;
} orc_track_rec;

typedef struct {          /* one e+ e+ e- combination that passed the energy test */
  int32_t t[3];           /* indices into the frame's kept-track list: e+, e+, e- */
  double de;              /* sum of energies minus the muon mass */
  int32_t status;         /* 0 a pair has no intersection, 1 target filter emptied a pair,
                             2 vertexed */
  int32_t pass;           /* 1 when the three signal cuts pass */
  double chi2, tdist, ptot;
  double chi2_second;     /* second-smallest chi2 over intersection choices (or inf) */
  double disc_min;        /* smallest |h^2| / (r_a r_b) over the three pairs (h: half chord) */
  double filt_margin;     /* smallest | |p| - (target_r + margin) | over all intersection points */
  double mu[3];
  double pvec[3][3];      /* momentum of each track at its closest point (MeV) */
} orc_combo_rec;

typedef struct {
  int32_t reason, keep;
  int32_t n_hits, n_layer[4];
  int64_t n_tested;       /* n0*n1*n2 */
  int64_t n_pass[4];      /* survivors after cut 1, 1-2, 1-3, 1-4 in the paper's order */
  int32_t n_triplets, n_tracks, n_combos, n_vertexed;
  /* optional record buffers (may be NULL); the counts written are capped by the capacities */
  orc_trip_rec* trips;  int32_t trips_cap;  int32_t trips_n;
  orc_track_rec* trks;  int32_t trks_cap;   int32_t trks_n;   /* one per kept triplet */
  int32_t* kept_trk;    int32_t kept_cap;   int32_t kept_n;   /* track rec index of each kept track */
  orc_combo_rec* combos; int32_t combos_cap; int32_t combos_n;
} orc_frame_out;

int  orc_decode(const orc_config* c, uint32_t addr, orc_hit* out);
void orc_cut_vars(const orc_config* c, const double* h0, const double* h1, const double* h2,
                  double* v /* dlambda, cos01, cos12, rtc */);
int  orc_fit_triplet(const orc_config* c, const double* ha, const double* hb, const double* hc,
                     int mid_layer, orc_tfit* f);
double orc_highland(const orc_config* c, double p, int layer);
int  orc_select_frame(const orc_config* c, const int32_t* addrs, int32_t n, orc_frame_out* out);
int  orc_select_frame_hits(const orc_config* c, const orc_hit* hits, int32_t n, orc_frame_out* out);
int  orc_select_frames(const orc_config* c, const int32_t* hits, const int64_t* off, int64_t n_frames,
                       uint8_t* keep, uint8_t* reason, int32_t n_threads, int64_t* counts /* F x 8 or NULL */);
/* Track fit from FP64 positions of four hits (layers 0..3): writes kappa_bar, R_bar,
 * theta01 and chi2 into out[0..3]; returns 0 on success. */
int  orc_fit_track_positions(const orc_config* c, const double* h /* 4 x 3 */, double* out);
/* Exact nonlinear single-triplet minimiser on the 3D radius (golden-section search of the
 * unlinearised chi2 of the triplet fit); writes R at the minimum. */
int  orc_fit_triplet_exact(const orc_config* c, const double* ha, const double* hb, const double* hc,
                           int mid_layer, double r_lo, double r_hi, double* R_out);

/* ------------------------------------------------------------------ alignment
 * Rigid alignment of the four layers (the detector model of the track fit,
 * Sec. "Track Reconstruction", with each cylinder displaced): the hit measured at
 * nominal position x_nom on layer L sits at R(w_L) x_nom + d_L in the global
 * frame, R(w) = Rz(wz) Ry(wy) Rx(wx) (rotations about the global axes through the
 * origin, x first), params[6L .. 6L+5] = dx, dy, dz [mm], wx, wy, wz [rad].
 * params[24] scales the field (B * field_scale * params[24]). */
void orc_align_point(const double* p6, const double* x_nom, double* x);
/* chi2 of each frozen candidate: cand[4k .. 4k+3] are global indices into hits of a
 * layer-0, -1, -2, -3 hit; the chi2 of the track fit (global chi2 at the mean
 * curvature, as for a selected track) at the given alignment.  chi2[k] = NaN when a
 * hit is invalid, on the wrong layer, or a fit fails.  Threads over candidate
 * ranges.  Returns the number of finite chi2. */
int64_t orc_fit_chi2(const orc_config* c, const int32_t* hits, int64_t n_hits, const int32_t* cand, int64_t n_cand,
                     const double* params /* 25 */, double* chi2, int32_t n_threads);

#ifdef __cplusplus
}
#endif
#endif
