// C ABI of libm3e: context, parameter checks, look-up tables, launches.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "m3e_internal.cuh"

using namespace m3e;

void noalloc_forget(int dev);  // defined with m3e_select_frames_noalloc below

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

#define CUDA_TRY(x)                                                                    \
  do {                                                                                 \
    cudaError_t e_ = (x);                                                              \
    if (e_ != cudaSuccess) return fail(M3E_ECUDA, "%s: %s", #x, cudaGetErrorString(e_)); \
  } while (0)

// Restores the caller's current device on scope exit.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// Chunks of the host entry point (double-buffered): at most 4, of at least 200,000
// frames, so that the copy of the next chunk hides behind the kernels of this one
// while the fixed cost per chunk (launches, kernel tails) stays small.
constexpr int GATE_MAX = 64;                  // chunks of the host entry point, at most
constexpr int64_t GATE_MIN_FRAMES = 50000;    // frames per chunk, at least (unless the batch is smaller)

}  // namespace

int m3e::m3e_set_error(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

// Device scratch of one launch sequence: work queue, deferred-frame list and the
// global candidate arrays of the staged form.  The context holds one set for the
// device entry points and two for the double-buffered host entry point.
struct Scratch {
  int* work = nullptr;                      // [0] work-queue head, [1] list-1 count, [2] list-2 count
  unsigned long long* counters = nullptr;   // staged: [0] triplets, [1] combinations, [2] stage-3 queue, [3] hits
  int* defer = nullptr;                     // list 1: deferred frames
  int* defer2 = nullptr;                    // list 2 (staged form)
  int* defer1b = nullptr;                   // list 1b (staged form)
  int64_t defer_cap = 0;
  float* hf = nullptr;                      // hx, hy, hz, hphi
  uint32_t* haddr = nullptr;
  uint16_t* hidx = nullptr;
  int64_t hits_cap = 0;
  uint16_t* l3 = nullptr;
  int* fint = nullptr;                      // fstate, ftbase, fntrip, ffound, fncombo
  long long* fcbase = nullptr;              // per frame: first combination
  int64_t frames_cap = 0;
  int4* trip = nullptr;
  float2* tek = nullptr;
  float4* trec = nullptr;
  int64_t trip_cap = 0;
  int4* combo = nullptr;
  int64_t combo_cap = 0;
};

struct m3e_ctx {
  int device = 0;
  int sms = 1;
  int fused_bpsm = 1, s1_bpsm = 1, s2_bpsm = 1, s3_bpsm = 1, s4_bpsm = 1, s1c_bpsm = 1, s1m_bpsm = 1, ingest_bpsm = 1;
  int grab = 4;
  int defer_hits = W_HITS;
  int mid_threads = CTA_THREADS;  // threads of a stage-1 middle-tier CTA
  m3e_config cfg{};
  DevCfg dc{};
  float4* col_lut = nullptr;
  float* row_lut = nullptr;
  int* err = nullptr;           // latched error flags
  int* h_err = nullptr;         // pinned error-flag readback
  int last_launches = 0;
  Scratch main;
  // host entry point staging
  Scratch hsc[2];
  cudaStream_t hs[2] = {nullptr, nullptr};
  cudaEvent_t he[2] = {nullptr, nullptr};
  int32_t* d_hits[2] = {nullptr, nullptr};
  int64_t* d_off[2] = {nullptr, nullptr};
  uint8_t* d_out[2] = {nullptr, nullptr};
  int64_t cap_hits[2] = {0, 0}, cap_frames[2] = {0, 0};
  unsigned* d_gate = nullptr;   // per-chunk arrival flags
  unsigned* h_gate = nullptr;   // pinned constants the copy engine writes into them: GATE_MAX zeros, then a one
  cudaEvent_t ge[2] = {nullptr, nullptr};  // flags cleared; every copy of the call done
  int gate_chunks = 16, gate_ms = 2000, gate_drop = -1;
  // kernel timing
  bool prof = false;
  bool prof_valid = false;
  int prof_kind = 0;            // 0 staged, 1 fused, 2 plain
  cudaEvent_t pe[10] = {};
  // streaming
  StreamEngine* stream = nullptr;
  // fit gradient: per-block partial sums and the valid-candidate counter
  double* fit_partial = nullptr;
  int fit_partial_blocks = 0;
  unsigned long long* fit_nvalid = nullptr;
  unsigned long long* h_fit_nvalid = nullptr;
};

namespace {

int check_config(const m3e_config* c) {
  if (!c) return fail(M3E_EINVAL, "config is NULL");
  if (c->size != sizeof(m3e_config))
    return fail(M3E_EINVAL, "config.size %u != sizeof(m3e_config) %zu", c->size, sizeof(m3e_config));
  for (int L = 0; L < 4; ++L) {
    if (!(c->r_mm[L] > 0) || !(c->half_len_mm[L] > 0)) return fail(M3E_EINVAL, "layer %d: radius/length", L);
    if (L && !(c->r_mm[L] > c->r_mm[L - 1])) return fail(M3E_EINVAL, "layer radii must increase");
    if (c->n_ladders[L] < 1 || c->n_ladders[L] > 32) return fail(M3E_EINVAL, "layer %d: n_ladders 1..32", L);
    if (c->n_cols[L] < 1 || c->n_cols[L] > 256) return fail(M3E_EINVAL, "layer %d: n_cols 1..256", L);
    if (c->n_rows[L] < 1 || c->n_rows[L] > 8192) return fail(M3E_EINVAL, "layer %d: n_rows 1..8192", L);
    if (!(c->x_over_X0[L] > 0) || !(c->x_over_X0[L] < 1)) return fail(M3E_EINVAL, "layer %d: x/X0", L);
  }
  if (!(c->pitch_mm > 0) || !(c->B_T > 0) || !(c->field_scale > 0) || !(c->k_MeV_per_T_mm > 0))
    return fail(M3E_EINVAL, "pitch, field and k must be positive");
  if (!(c->m_mu_MeV > 0) || !(c->m_e_MeV >= 0)) return fail(M3E_EINVAL, "masses");
  if (c->max_hits < 1 || c->max_hits > C_HITS) return fail(M3E_EINVAL, "max_hits must be 1..%d", C_HITS);
  if (c->max_triplets < 0 || c->max_triplets > C_TRIP)
    return fail(M3E_EINVAL, "max_triplets must be 0..%d", C_TRIP);
  if (c->max_tracks < 0 || c->max_tracks > C_TRK) return fail(M3E_EINVAL, "max_tracks must be 0..%d", C_TRK);
  if (c->max_combos < 0 || c->max_combos > C_COMBO) return fail(M3E_EINVAL, "max_combos must be 0..%d", C_COMBO);
  const double cuts[] = {c->dlambda_max, c->phi01_max, c->phi12_max, c->rtc_min, c->rtc_max, c->chi2_track_max,
                         c->e_window, c->isect_margin, c->vtx_chi2_max, c->target_dist_max, c->ptot_max,
                         c->target_r_mm, c->target_half_len_mm};
  for (double v : cuts)
    if (!(v >= 0) || std::isnan(v)) return fail(M3E_EINVAL, "cut values must be >= 0");
  return M3E_OK;
}

// Everything the kernels need, computed in FP64 and rounded once.
void make_devcfg(const m3e_config& c, DevCfg& d) {
  const double TWO_PI = 2.0 * M_PI;
  for (int L = 0; L < 4; ++L) {
    d.r[L] = (float)c.r_mm[L];
    d.ncol[L] = c.n_cols[L];
    d.nlad[L] = c.n_ladders[L];
    d.nrow[L] = c.n_rows[L];
    d.ntot[L] = c.n_ladders[L] * c.n_cols[L];
    d.intot[L] = (float)(1.0 / d.ntot[L]);
    const double x = c.x_over_X0[L];
    d.hl[L] = (float)(13.6 * std::sqrt(x) * (1.0 + 0.038 * std::log(x)));
    d.ihl[L] = (float)(1.0 / (13.6 * std::sqrt(x) * (1.0 + 0.038 * std::log(x))));
  }
  int co = 0, ro = 0;
  for (int L = 0; L < 4; ++L) {
    d.col_off[L] = co;
    d.row_off[L] = ro;
    co += d.ntot[L];
    ro += d.nrow[L];
  }
  for (int L = 0; L < 4; ++L) {
    const double st = TWO_PI / d.ntot[L];
    d.phs_hi[L] = (float)st;
    d.phs_lo[L] = (float)(st - (double)d.phs_hi[L]);
  }
  d.pk_nlad = d.pk_ncol = d.pk_nrow = d.pk_coloff = d.pk_rowoff = 0ull;
  for (int L = 0; L < 4; ++L) {
    d.pk_nlad |= (unsigned long long)d.nlad[L] << (16 * L);
    d.pk_ncol |= (unsigned long long)d.ncol[L] << (16 * L);
    d.pk_nrow |= (unsigned long long)d.nrow[L] << (16 * L);
    d.pk_coloff |= (unsigned long long)d.col_off[L] << (16 * L);
    d.pk_rowoff |= (unsigned long long)d.row_off[L] << (16 * L);
    uint32_t ib;
    std::memcpy(&ib, &d.intot[L], 4);
    d.ltab[L] = make_uint4((uint32_t)d.nlad[L] | (uint32_t)d.ncol[L] << 6 | (uint32_t)d.nrow[L] << 15,
                           (uint32_t)d.col_off[L], (uint32_t)d.row_off[L], ib);
  }
  d.inv_dr01 = (float)(1.0 / (c.r_mm[1] - c.r_mm[0]));
  d.inv_dr12 = (float)(1.0 / (c.r_mm[2] - c.r_mm[1]));
  d.dr12 = (float)(c.r_mm[2] - c.r_mm[1]);
  d.zoff2 = (float)c.half_len_mm[2];
  d.izw2 = (float)(NZB / (2.0 * c.half_len_mm[2]));
  d.c01 = (float)(std::cos(c.phi01_max) * c.r_mm[0] * c.r_mm[1]);
  d.c12 = (float)(std::cos(c.phi12_max) * c.r_mm[1] * c.r_mm[2]);
  d.dl_max = (float)c.dlambda_max;
  d.rtc_lo2 = (float)(4.0 * c.rtc_min * c.rtc_min);
  d.rtc_hi2 = (float)(4.0 * c.rtc_max * c.rtc_max);
  // Phi-bin windows: bins of width w = 2 pi / NB; a bin's hits reach at most one
  // column width beyond its nominal edges.  Two hits whose bins are m apart are
  // at least (m - 1) w - 2 colw apart in phi, so a pair within phi_max needs
  // m <= 1 + (phi_max + 2 colw) / w; 1e-3 rad covers FP32 rounding of the cosine.
  int ntmin = d.ntot[0];
  for (int L = 1; L < 4; ++L) ntmin = ntmin < d.ntot[L] ? ntmin : d.ntot[L];
  const double w = TWO_PI / NB, colw = TWO_PI / ntmin;
  auto win = [&](double phimax) {
    if (phimax >= M_PI) return NB;
    const double k = 1.0 + std::floor((phimax + 2.0 * colw + 1e-3) / w);
    return k >= NB ? NB : (int)k;
  };
  d.k01 = win(c.phi01_max);
  d.k12 = win(c.phi12_max);
  d.kB = (float)(c.k_MeV_per_T_mm * c.B_T * c.field_scale);
  d.chi2_trk = (float)c.chi2_track_max;
  d.r3 = (float)c.r_mm[3];
  d.colw3 = (float)(TWO_PI / d.ntot[3] + 1e-4);
  d.me2 = (float)(c.m_e_MeV * c.m_e_MeV);
  d.m_mu = (float)c.m_mu_MeV;
  d.e_win = (float)c.e_window;
  d.isect_lim = (float)(c.target_r_mm + c.isect_margin);
  d.tgt_r = (float)c.target_r_mm;
  d.tgt_h = (float)c.target_half_len_mm;
  d.vtx_chi2 = (float)c.vtx_chi2_max;
  d.tgt_dist = (float)c.target_dist_max;
  d.ptot_max = (float)c.ptot_max;
  d.sig_pix2 = (float)(c.pitch_mm * c.pitch_mm / 12.0);
  d.max_hits = c.max_hits;
  d.max_trip = c.max_triplets;
  d.max_trk = c.max_tracks;
  d.max_combo = c.max_combos;
}

KParams base_params(m3e_ctx* x, Scratch& sc) {
  KParams p{};
  p.col_lut = x->col_lut;
  p.row_lut = x->row_lut;
  p.work = sc.work;
  p.err = x->err;
  p.defer_list = sc.defer;
  p.defer_count = sc.work + 1;
  p.in_list = sc.defer;
  p.in_count = sc.work + 1;
  p.grab = x->grab;
  p.defer_hits = x->defer_hits;
  return p;
}

template <class T>
int grow(T*& ptr, int64_t& cap, int64_t need, size_t elem, const char* what) {
  if (need <= cap) return M3E_OK;
  if (ptr) CUDA_TRY(cudaFree(ptr));
  ptr = nullptr;
  cap = 0;
  if (cudaMalloc(&ptr, elem * (size_t)need) != cudaSuccess) return fail(M3E_ENOMEM, "%s: %lld entries", what, (long long)need);
  cap = need;
  return M3E_OK;
}

// Scratch for a batch of nf frames (staged arrays only when staged; the sorted
// hits of pending frames take HITS_PER_FRAME entries per frame on average, frames
// beyond that are deferred to the CTA-per-frame kernel).
constexpr int64_t HITS_PER_FRAME = 128;

int ensure_scratch(Scratch& sc, int64_t nf, bool staged) {
  // sorted-hit indices travel as int32 in the triplet records: at most 2^31 - 2^16 of them
  const int64_t nh_want = nf * HITS_PER_FRAME > (1 << 16) ? nf * HITS_PER_FRAME : (1 << 16);
  const int64_t nh = nh_want < ((int64_t)1 << 31) - (1 << 16) ? nh_want : ((int64_t)1 << 31) - (1 << 16);
  int64_t one = sc.work ? 1 : 0;
  int rc = grow(sc.work, one, 1, 4 * sizeof(int), "work counters");
  if (rc) return rc;
  int64_t one2 = sc.counters ? 1 : 0;
  rc = grow(sc.counters, one2, 1, 4 * sizeof(unsigned long long), "counters");
  if (rc) return rc;
  {
    const int64_t dc = nf > 4096 ? nf : 4096;
    if (dc > sc.defer_cap) {
      int64_t c0 = sc.defer_cap, c1 = sc.defer_cap, c2 = sc.defer_cap;
      rc = grow(sc.defer, c0, dc, sizeof(int), "deferred list");
      if (!rc) rc = grow(sc.defer2, c1, dc, sizeof(int), "deferred list 2");
      if (!rc) rc = grow(sc.defer1b, c2, dc, sizeof(int), "deferred list 1b");
      if (rc) return rc;
      sc.defer_cap = dc;
    }
  }
  if (!staged) return M3E_OK;
  int64_t hc = sc.hits_cap;
  if (nh > hc) {
    int64_t c0 = hc, c1 = hc, c2 = hc;
    rc = grow(sc.hf, c0, nh, 4 * sizeof(float), "sorted hits");
    if (!rc) rc = grow(sc.haddr, c1, nh, sizeof(uint32_t), "sorted addresses");
    if (!rc) rc = grow(sc.hidx, c2, nh, sizeof(uint16_t), "sorted input indices");
    if (rc) return rc;
    sc.hits_cap = nh;
  }
  if (nf > sc.frames_cap) {
    int64_t c0 = sc.frames_cap, c1 = sc.frames_cap, c2 = sc.frames_cap;
    rc = grow(sc.l3, c0, nf, (NB + 1) * sizeof(uint16_t), "layer-3 bins");
    if (!rc) rc = grow(sc.fint, c1, nf, 5 * sizeof(int), "frame state");
    if (!rc) rc = grow(sc.fcbase, c2, nf, sizeof(long long), "frame combination bases");
    if (rc) return rc;
    sc.frames_cap = nf;
  }
  const int64_t lim = ((int64_t)1 << 31) - (1 << 16);
  int64_t tc = 64 * nf > (1 << 16) ? 64 * nf : (1 << 16);
  tc = tc < lim ? tc : lim;
  if (tc > sc.trip_cap) {
    int64_t c0 = sc.trip_cap, c1 = sc.trip_cap, c2 = sc.trip_cap;
    rc = grow(sc.trip, c0, tc, sizeof(int4), "triplets");
    if (!rc) rc = grow(sc.tek, c1, tc, sizeof(float2), "track energies");
    if (!rc) rc = grow(sc.trec, c2, tc, 4 * sizeof(float4), "track records");
    if (rc) return rc;
    sc.trip_cap = tc;
  }
  int64_t cc = 192 * nf > (1 << 16) ? 192 * nf : (1 << 16);
  cc = cc < lim ? cc : lim;
  return grow(sc.combo, sc.combo_cap, cc, sizeof(int4), "combinations");
}

void free_scratch(Scratch& sc) {
  cudaFree(sc.work);
  cudaFree(sc.counters);
  cudaFree(sc.defer);
  cudaFree(sc.defer2);
  cudaFree(sc.defer1b);
  cudaFree(sc.hf);
  cudaFree(sc.haddr);
  cudaFree(sc.hidx);
  cudaFree(sc.l3);
  cudaFree(sc.fint);
  cudaFree(sc.fcbase);
  cudaFree(sc.trip);
  cudaFree(sc.tek);
  cudaFree(sc.trec);
  cudaFree(sc.combo);
  sc = Scratch();
}

SParams staged_params(const Scratch& sc) {
  SParams s{};
  const int64_t H = sc.hits_cap, F = sc.frames_cap;
  s.hp = reinterpret_cast<float4*>(sc.hf);
  s.haddr = sc.haddr;
  s.hidx = sc.hidx;
  s.l3 = sc.l3;
  s.fstate = sc.fint;
  s.ftbase = sc.fint + F;
  s.fntrip = sc.fint + 2 * F;
  s.ffound = sc.fint + 3 * F;
  s.fncombo = sc.fint + 4 * F;
  s.fcbase = sc.fcbase;
  s.list1 = sc.defer;
  s.list2 = sc.defer2;
  s.list1b = sc.defer1b;
  s.lcount = sc.work + 1;
  s.hits_cap = H;
  s.trip = sc.trip;
  s.tek = sc.tek;
  s.trec = sc.trec;
  s.combo = sc.combo;
  s.counters = sc.counters;
  s.trip_cap = sc.trip_cap;
  s.combo_cap = sc.combo_cap;
  return s;
}

int check_batch(const int32_t* hits, const int64_t* off, int64_t n, const uint8_t* keep, const uint8_t* reason) {
  if (n < 0 || n > (int64_t)1 << 30) return fail(M3E_EINVAL, "n_frames %lld out of range", (long long)n);
  if (n > 0 && (!off || !keep || !reason)) return fail(M3E_EINVAL, "NULL frame_off/keep/reason");
  (void)hits;
  return M3E_OK;
}

enum { FORM_STAGED = 0, FORM_FUSED = 1, FORM_PLAIN = 2 };

// Enqueue one batch on stream s: form 0 staged (5 kernels), 1 fused warp kernel,
// 2 plain CTA-per-frame kernel; forms 0 and 1 finish with the deferred-frame
// kernel.  Timing events are recorded when `timed`.
int enqueue(m3e_ctx* x, Scratch& sc, KParams p, int form, bool debug, cudaStream_t s, bool timed,
            cudaEvent_t after_s1 = nullptr) {
  if (form == FORM_PLAIN) {
    if (timed) CUDA_TRY(cudaEventRecord(x->pe[0], s));
    CUDA_TRY(launch_plain(x->dc, p, debug, s));
    if (timed) CUDA_TRY(cudaEventRecord(x->pe[1], s));
    x->last_launches = 1;
    return M3E_OK;
  }
  CUDA_TRY(cudaMemsetAsync(sc.work, 0, 4 * sizeof(int), s));  // queue head and the three list counts
  if (form == FORM_FUSED) {
    if (timed) CUDA_TRY(cudaEventRecord(x->pe[0], s));
    CUDA_TRY(launch_fused(x->dc, p, x->sms * x->fused_bpsm, debug, s));
    if (timed) CUDA_TRY(cudaEventRecord(x->pe[1], s));
    CUDA_TRY(launch_deferred(x->dc, p, 2 * x->sms, debug, s));
    if (timed) CUDA_TRY(cudaEventRecord(x->pe[2], s));
    x->last_launches = 2;
    return M3E_OK;
  }
  CUDA_TRY(cudaMemsetAsync(sc.counters, 0, 4 * sizeof(unsigned long long), s));
  const int grids[6] = {x->sms * x->s1_bpsm, x->sms * x->s2_bpsm,  x->sms * x->s3_bpsm,
                        x->sms * x->s4_bpsm, x->sms * x->s1c_bpsm, x->sms * x->s1m_bpsm};
  const SParams sp = staged_params(sc);
  if (p.gate) CUDA_TRY(cudaMemsetAsync(sp.fstate, 0x7f, sizeof(int) * (size_t)p.n_frames, s));  // no stale states
  CUDA_TRY(launch_staged(x->dc, p, sp, grids, debug, s, timed ? x->pe : nullptr, after_s1, x->mid_threads));
  KParams pd = p;  // frames no stage could finish: the CTA-per-frame kernel
  pd.in_list = sp.list2;
  pd.in_count = sp.lcount + 1;
  CUDA_TRY(launch_deferred(x->dc, pd, 2 * x->sms, debug, s));
  if (timed) CUDA_TRY(cudaEventRecord(x->pe[8], s));
  x->last_launches = 8;
  return M3E_OK;
}

}  // namespace

extern "C" {

int m3e_version(void) { return M3E_VERSION; }

const char* m3e_last_error_string(void) { return g_err; }

int m3e_create(const m3e_config* cfg, int cuda_device, m3e_ctx** out) {
  if (!out) return fail(M3E_EINVAL, "out is NULL");
  *out = nullptr;
  int rc = check_config(cfg);
  if (rc) return rc;
  int ndev = 0;
  CUDA_TRY(cudaGetDeviceCount(&ndev));
  if (cuda_device < 0 || cuda_device >= ndev) return fail(M3E_EINVAL, "device %d of %d", cuda_device, ndev);
  DeviceGuard guard(cuda_device);
  m3e_ctx* x = new (std::nothrow) m3e_ctx();
  if (!x) return fail(M3E_ENOMEM, "context");
  x->device = cuda_device;
  x->cfg = *cfg;
  make_devcfg(*cfg, x->dc);
  noalloc_forget(cuda_device);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, cuda_device) != cudaSuccess) {
    delete x;
    return fail(M3E_ECUDA, "cudaGetDeviceProperties");
  }
  x->sms = prop.multiProcessorCount;
  x->fused_bpsm = fused_blocks_per_sm();
  x->s1_bpsm = stage_blocks_per_sm(1);
  x->s2_bpsm = stage_blocks_per_sm(2);
  x->s3_bpsm = stage_blocks_per_sm(3);
  x->s4_bpsm = stage_blocks_per_sm(4);
  x->s1c_bpsm = stage_blocks_per_sm(5);
  x->s1m_bpsm = stage_blocks_per_sm(6);
  x->ingest_bpsm = ingest_blocks_per_sm();
  // look-up tables in FP64, rounded once
  int ncolt = 0, nrowt = 0;
  for (int L = 0; L < 4; ++L) {
    ncolt += x->dc.ntot[L];
    nrowt += x->dc.nrow[L];
  }
  std::vector<float4> cl(ncolt);
  std::vector<float> rl(nrowt);
  for (int L = 0; L < 4; ++L) {
    const int nt = x->dc.ntot[L];
    for (int g = 0; g < nt; ++g) {
      const double ph = ((double)g + 0.5) * 2.0 * M_PI / (double)nt;
      cl[x->dc.col_off[L] + g] = make_float4((float)(cfg->r_mm[L] * std::cos(ph)),
                                             (float)(cfg->r_mm[L] * std::sin(ph)), (float)ph, 0.f);
    }
    for (int w = 0; w < x->dc.nrow[L]; ++w)
      rl[x->dc.row_off[L] + w] = (float)(-cfg->half_len_mm[L] + ((double)w + 0.5) * cfg->pitch_mm);
  }
  bool ok = cudaMalloc(&x->col_lut, sizeof(float4) * ncolt) == cudaSuccess &&
            cudaMalloc(&x->row_lut, sizeof(float) * nrowt) == cudaSuccess &&
            cudaMalloc(&x->err, sizeof(int)) == cudaSuccess && cudaMallocHost(&x->h_err, sizeof(int)) == cudaSuccess;
  if (ok)
    ok = cudaMemcpy(x->col_lut, cl.data(), sizeof(float4) * ncolt, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(x->row_lut, rl.data(), sizeof(float) * nrowt, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemset(x->err, 0, sizeof(int)) == cudaSuccess;
  if (ok) ok = ensure_scratch(x->main, 1 << 12, false) == M3E_OK;
  if (!ok) {
    m3e_destroy(x);
    return fail(M3E_ENOMEM, "device allocation in m3e_create");
  }
  *out = x;
  return M3E_OK;
}

int m3e_destroy(m3e_ctx* x) {
  if (!x) return M3E_OK;
  DeviceGuard guard(x->device);
  if (x->stream) stream_destroy(x->stream);
  x->stream = nullptr;
  cudaDeviceSynchronize();
  cudaFree(x->fit_partial);
  cudaFree(x->fit_nvalid);
  if (x->h_fit_nvalid) cudaFreeHost(x->h_fit_nvalid);
  cudaFree(x->col_lut);
  cudaFree(x->row_lut);
  cudaFree(x->err);
  if (x->h_err) cudaFreeHost(x->h_err);
  free_scratch(x->main);
  for (int i = 0; i < 2; ++i) {
    free_scratch(x->hsc[i]);
    cudaFree(x->d_hits[i]);
    cudaFree(x->d_off[i]);
    cudaFree(x->d_out[i]);
    if (x->hs[i]) cudaStreamDestroy(x->hs[i]);
    if (x->he[i]) cudaEventDestroy(x->he[i]);
    if (x->ge[i]) cudaEventDestroy(x->ge[i]);
  }
  cudaFree(x->d_gate);
  if (x->h_gate) cudaFreeHost(x->h_gate);
  for (int i = 0; i < 10; ++i)
    if (x->pe[i]) cudaEventDestroy(x->pe[i]);
  delete x;
  return M3E_OK;
}

int m3e_set_launch(m3e_ctx* x, int frames_per_grab, int ctas_per_sm) {
  if (!x) return fail(M3E_EINVAL, "ctx is NULL");
  if (frames_per_grab < 1 || frames_per_grab > 64) return fail(M3E_EINVAL, "frames_per_grab 1..64");
  DeviceGuard guard(x->device);
  const int maxb = fused_blocks_per_sm();
  if (ctas_per_sm < 0 || ctas_per_sm > maxb) return fail(M3E_EINVAL, "ctas_per_sm 0..%d", maxb);
  x->grab = frames_per_grab;
  x->fused_bpsm = ctas_per_sm ? ctas_per_sm : maxb;
  return M3E_OK;
}

int m3e_last_launch_count(const m3e_ctx* x) { return x ? x->last_launches : 0; }

int m3e_set_profiling(m3e_ctx* x, int on) {
  if (!x) return fail(M3E_EINVAL, "ctx is NULL");
  DeviceGuard guard(x->device);
  for (int i = 0; i < 10 && on; ++i)
    if (!x->pe[i]) CUDA_TRY(cudaEventCreate(&x->pe[i]));
  x->prof = on != 0;
  x->prof_valid = false;
  return M3E_OK;
}

int m3e_kernel_times(m3e_ctx* x, float* main_ms, float* deferred_ms) {
  if (!x || !main_ms || !deferred_ms) return fail(M3E_EINVAL, "NULL argument");
  if (!x->prof_valid) return fail(M3E_ESTATE, "no timed select call since profiling was enabled");
  DeviceGuard guard(x->device);
  const int last = x->prof_kind == FORM_STAGED ? 8 : (x->prof_kind == FORM_FUSED ? 2 : 1);
  const int mid = x->prof_kind == FORM_STAGED ? 7 : 1;
  CUDA_TRY(cudaEventSynchronize(x->pe[last]));
  CUDA_TRY(cudaEventElapsedTime(main_ms, x->pe[0], x->pe[mid]));
  *deferred_ms = 0.f;
  if (last != mid) CUDA_TRY(cudaEventElapsedTime(deferred_ms, x->pe[mid], x->pe[last]));
  return M3E_OK;
}

int m3e_stage_times(m3e_ctx* x, float* ms, int n) {
  if (!x || !ms || n < 1) return fail(M3E_EINVAL, "bad argument");
  if (!x->prof_valid || x->prof_kind != FORM_STAGED) return fail(M3E_ESTATE, "no timed staged select call");
  DeviceGuard guard(x->device);
  CUDA_TRY(cudaEventSynchronize(x->pe[8]));
  for (int i = 0; i < n && i < 8; ++i) CUDA_TRY(cudaEventElapsedTime(&ms[i], x->pe[i], x->pe[i + 1]));
  return M3E_OK;
}

static int select_common(m3e_ctx* x, const int32_t* hits, const int64_t* off, int64_t n, uint8_t* keep,
                         uint8_t* reason, m3e_stats* stats, const m3e_dump* dump, int form, cudaStream_t s) {
  if (!x) return fail(M3E_EINVAL, "ctx is NULL");
  int rc = check_batch(hits, off, n, keep, reason);
  if (rc) return rc;
  if (form < FORM_STAGED || form > FORM_PLAIN) return fail(M3E_EINVAL, "form must be 0, 1 or 2");
  x->last_launches = 0;
  x->prof_valid = false;
  if (n == 0) return M3E_OK;
  DeviceGuard guard(x->device);
  rc = ensure_scratch(x->main, n, form == FORM_STAGED);
  if (rc) return rc;
  KParams p = base_params(x, x->main);
  p.hits = hits;
  p.off = off;
  p.n_frames = n;
  p.off_base = 0;
  p.keep = keep;
  p.reason = reason;
  p.stats = reinterpret_cast<unsigned long long*>(stats);
  if (dump) {
    if (dump->cap_trip < 0 || dump->cap_combo < 0 || !dump->n_trip || !dump->n_combo ||
        (dump->cap_trip && (!dump->trip || !dump->trk_status || !dump->trk_val)) ||
        (dump->cap_combo && (!dump->combo || !dump->combo_val)))
      return fail(M3E_EINVAL, "incomplete m3e_dump");
    p.dump = *dump;
  }
  const bool timed = x->prof && dump == nullptr;
  rc = enqueue(x, x->main, p, form, dump != nullptr, s, timed);
  x->prof_valid = timed && rc == M3E_OK;
  x->prof_kind = form;
  return rc;
}

int m3e_select_frames(m3e_ctx* x, const int32_t* d_hits, const int64_t* d_off, int64_t n, uint8_t* d_keep,
                      uint8_t* d_reason, m3e_stats* d_stats, cudaStream_t s) {
  return select_common(x, d_hits, d_off, n, d_keep, d_reason, d_stats, nullptr, FORM_STAGED, s);
}

int m3e_select_frames_fused(m3e_ctx* x, const int32_t* d_hits, const int64_t* d_off, int64_t n, uint8_t* d_keep,
                            uint8_t* d_reason, m3e_stats* d_stats, cudaStream_t s) {
  return select_common(x, d_hits, d_off, n, d_keep, d_reason, d_stats, nullptr, FORM_FUSED, s);
}

int m3e_select_frames_plain(m3e_ctx* x, const int32_t* d_hits, const int64_t* d_off, int64_t n, uint8_t* d_keep,
                            uint8_t* d_reason, m3e_stats* d_stats, cudaStream_t s) {
  return select_common(x, d_hits, d_off, n, d_keep, d_reason, d_stats, nullptr, FORM_PLAIN, s);
}

int m3e_select_frames_debug(m3e_ctx* x, int form, const int32_t* d_hits, const int64_t* d_off, int64_t n,
                            uint8_t* d_keep, uint8_t* d_reason, const m3e_dump* dump, cudaStream_t s) {
  if (!dump) return fail(M3E_EINVAL, "dump is NULL");
  return select_common(x, d_hits, d_off, n, d_keep, d_reason, nullptr, dump, form, s);
}

int m3e_check(m3e_ctx* x, cudaStream_t s) {
  if (!x) return fail(M3E_EINVAL, "ctx is NULL");
  DeviceGuard guard(x->device);
  CUDA_TRY(cudaMemcpyAsync(x->h_err, x->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  const int e = *x->h_err;
  if (e) {
    CUDA_TRY(cudaMemsetAsync(x->err, 0, sizeof(int), s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (e & ERR_GATE) return fail(M3E_ETIMEOUT, "a chunk of the host entry point did not arrive in time");
    return fail(M3E_EBADHIT, "invalid pixel address or frame size seen (flags %d)", e);
  }
  return M3E_OK;
}

// End to end from host memory.  One staged selection over the whole batch on
// internal stream 0, while internal stream 1 copies the offsets and then the hits
// in chunks of frames, each followed by a 4-byte copy that sets the chunk's arrival
// flag.  Stage 1 takes a frame only once its chunk has arrived (a bounded wait), so
// the selection starts after the first chunk instead of after the whole batch; the
// kernels after stage 1 wait for the last copy.  The flags are cleared and set by
// the copy engine from constant page-locked words, so no host write races them.
int m3e_select_frames_host(m3e_ctx* x, const int32_t* h_hits, const int64_t* h_off, int64_t n, uint8_t* h_keep,
                           uint8_t* h_reason, cudaStream_t s) {
  if (!x) return fail(M3E_EINVAL, "ctx is NULL");
  int rc = check_batch(h_hits, h_off, n, h_keep, h_reason);
  if (rc) return rc;
  x->last_launches = 0;
  x->prof_valid = false;
  if (n == 0) return M3E_OK;
  if (h_off[n] < h_off[0]) return fail(M3E_EINVAL, "frame_off must be non-decreasing");
  if (h_off[n] > h_off[0] && !h_hits) return fail(M3E_EINVAL, "hits is NULL");
  DeviceGuard guard(x->device);
  for (int i = 0; i < 2; ++i) {
    if (!x->hs[i]) CUDA_TRY(cudaStreamCreateWithFlags(&x->hs[i], cudaStreamNonBlocking));
    if (!x->he[i]) CUDA_TRY(cudaEventCreateWithFlags(&x->he[i], cudaEventDisableTiming));
  }
  // the internal streams start after the work already on the caller's stream
  CUDA_TRY(cudaEventRecord(x->he[0], s));
  for (int i = 0; i < 2; ++i) CUDA_TRY(cudaStreamWaitEvent(x->hs[i], x->he[0], 0));
  const int64_t total = h_off[n] - h_off[0];
  if (!x->d_gate) {
    if (cudaMalloc(&x->d_gate, sizeof(unsigned) * GATE_MAX) != cudaSuccess) return fail(M3E_ENOMEM, "chunk flags");
  }
  if (!x->h_gate) {
    if (cudaMallocHost(&x->h_gate, sizeof(unsigned) * (GATE_MAX + 1)) != cudaSuccess)
      return fail(M3E_ENOMEM, "chunk flag constants");
    for (int k = 0; k < GATE_MAX; ++k) x->h_gate[k] = 0u;
    x->h_gate[GATE_MAX] = 1u;
  }
  for (int i = 0; i < 2; ++i)
    if (!x->ge[i]) CUDA_TRY(cudaEventCreateWithFlags(&x->ge[i], cudaEventDisableTiming));
  rc = grow(x->d_hits[0], x->cap_hits[0], total + total / 4 + 1024, sizeof(int32_t), "staging hits");
  if (rc) return rc;
  if (n + 1 > x->cap_frames[0]) {
    cudaFree(x->d_off[0]);
    cudaFree(x->d_out[0]);
    x->d_off[0] = nullptr;
    x->d_out[0] = nullptr;
    x->cap_frames[0] = 0;
    const int64_t cap = n + n / 4 + 1024;
    if (cudaMalloc(&x->d_off[0], sizeof(int64_t) * (cap + 1)) != cudaSuccess ||
        cudaMalloc(&x->d_out[0], 2 * cap) != cudaSuccess)
      return fail(M3E_ENOMEM, "staging frames");
    x->cap_frames[0] = cap;
  }
  rc = ensure_scratch(x->hsc[0], n, true);
  if (rc) return rc;
  // chunks of about equal frame counts
  const int64_t by_size = n / GATE_MIN_FRAMES;
  const int nch = (int)(by_size < 1 ? 1 : (by_size > x->gate_chunks ? x->gate_chunks : by_size));
  const int64_t fpc = (n + nch - 1) / nch;
  cudaStream_t ps = x->hs[0], cs = x->hs[1];
  // copy stream: clear the flags, then the offsets, then each chunk's hits and its flag
  CUDA_TRY(cudaMemcpyAsync(x->d_gate, x->h_gate, sizeof(unsigned) * nch, cudaMemcpyHostToDevice, cs));
  CUDA_TRY(cudaEventRecord(x->ge[0], cs));
  CUDA_TRY(cudaMemcpyAsync(x->d_off[0], h_off, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, cs));
  for (int k = 0; k < nch; ++k) {
    const int64_t f0 = k * fpc, f1 = f0 + fpc < n ? f0 + fpc : n;
    const int64_t nh = f0 < n ? h_off[f1] - h_off[f0] : 0;
    if (nh > 0)
      CUDA_TRY(cudaMemcpyAsync(x->d_hits[0] + (h_off[f0] - h_off[0]), h_hits + h_off[f0], sizeof(int32_t) * nh,
                               cudaMemcpyHostToDevice, cs));
    if (k != x->gate_drop)
      CUDA_TRY(cudaMemcpyAsync(x->d_gate + k, x->h_gate + GATE_MAX, sizeof(unsigned), cudaMemcpyHostToDevice, cs));
  }
  CUDA_TRY(cudaEventRecord(x->ge[1], cs));
  // compute stream: starts once the flags are clear; the kernels after stage 1
  // also wait for the last copy
  CUDA_TRY(cudaStreamWaitEvent(ps, x->ge[0], 0));
  KParams p = base_params(x, x->hsc[0]);
  p.hits = x->d_hits[0];
  p.off = x->d_off[0];
  p.off_base = h_off[0];
  p.n_frames = n;
  p.keep = x->d_out[0];
  p.reason = x->d_out[0] + x->cap_frames[0];
  p.gate = x->d_gate;
  p.gate_frames = (int)fpc;
  p.gate_ms = x->gate_ms;
  rc = enqueue(x, x->hsc[0], p, FORM_STAGED, false, ps, false, x->ge[1]);
  if (rc) return rc;
  const int launches = x->last_launches;
  CUDA_TRY(cudaMemcpyAsync(h_keep, p.keep, n, cudaMemcpyDeviceToHost, ps));
  CUDA_TRY(cudaMemcpyAsync(h_reason, p.reason, n, cudaMemcpyDeviceToHost, ps));
  for (int i = 0; i < 2; ++i) {
    CUDA_TRY(cudaEventRecord(x->he[i], x->hs[i]));
    CUDA_TRY(cudaStreamWaitEvent(s, x->he[i], 0));
  }
  x->last_launches = launches;
  return M3E_OK;
}

int m3e_set_host_pipeline(m3e_ctx* x, int max_chunks, int wait_ms, int drop_chunk) {
  if (!x) return fail(M3E_EINVAL, "ctx is NULL");
  if (max_chunks < 1 || max_chunks > GATE_MAX) return fail(M3E_EINVAL, "max_chunks 1..%d", GATE_MAX);
  if (wait_ms < 1 || wait_ms > 60000) return fail(M3E_EINVAL, "wait_ms 1..60000");
  if (drop_chunk < -1) return fail(M3E_EINVAL, "drop_chunk >= -1");
  x->gate_chunks = max_chunks;
  x->gate_ms = wait_ms;
  x->gate_drop = drop_chunk;
  return M3E_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ hit ingest

extern "C" int m3e_ingest(m3e_ctx* x, const int32_t* d_hits, int64_t n_hits, float* d_x, float* d_y, float* d_z,
                          float* d_phi, cudaStream_t s) {
  if (!x) return fail(M3E_EINVAL, "ctx is NULL");
  if (n_hits < 0) return fail(M3E_EINVAL, "n_hits < 0");
  x->last_launches = 0;
  x->prof_valid = false;
  if (n_hits == 0) return M3E_OK;
  if (!d_hits || !d_x || !d_y || !d_z) return fail(M3E_EINVAL, "NULL hit or coordinate array");
  DeviceGuard guard(x->device);
  CUDA_TRY(launch_ingest(x->dc, d_hits, n_hits, x->col_lut, x->row_lut, d_x, d_y, d_z, d_phi, x->err,
                         x->sms * x->ingest_bpsm, s));
  x->last_launches = 1;
  return M3E_OK;
}

// ------------------------------------------------------------------ selection without allocation
//
// m3e_select_frames_noalloc runs the fused kernels with their scratch (work-queue
// head, deferred-frame count, deferred-frame list) in the static device array
// below instead of context memory that grows with the batch.  It exists for
// callers that must not allocate device memory once they are running: a filter
// process that reads out frames at a fixed rate cannot afford the implicit device
// synchronisation and the milliseconds of a cudaMalloc/cudaFree in its loop, and
// a process that shares the GPU under a fixed memory budget reserves everything at
// start-up.  The price is a fixed upper bound on the frames of one call.

namespace {

constexpr int64_t NOALLOC_MAX_FRAMES = 1 << 18;  // frames per call (1 MB of scratch)
constexpr int NOALLOC_HEAD = 4;                  // [0] queue head, [1] deferred count, [2..3] unused

// Shared by every call on a device, holding the last call's contents; calls that
// overlap on the GPU race on it.
static __device__ __align__(256) int g_noalloc_scratch[NOALLOC_HEAD + NOALLOC_MAX_FRAMES];

std::mutex g_noalloc_mu;
int* g_noalloc_ptr[256] = {};  // device address of g_noalloc_scratch, per device

// Device address of the scratch array on `dev` (current device), looked up once.
int noalloc_scratch(int dev, int** out) {
  if (dev < 0 || dev >= 256) return fail(M3E_EINVAL, "device %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return fail(M3E_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    g_noalloc_ptr[dev] = static_cast<int*>(ptr);
  }
  *out = g_noalloc_ptr[dev];
  return M3E_OK;
}

}  // namespace

// Forget the cached address of `dev` so that the next call looks it up again: a
// context created after the device's primary context was reset
// (cudaDeviceReset) sees the array at its new address.
void noalloc_forget(int dev) {
  if (dev < 0 || dev >= 256) return;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  g_noalloc_ptr[dev] = nullptr;
}

extern "C" int m3e_select_frames_noalloc(m3e_ctx* x, const int32_t* d_hits, const int64_t* d_frame_off,
                                         int64_t n_frames, uint8_t* d_keep, uint8_t* d_reason, cudaStream_t s) {
  if (!x) return fail(M3E_EINVAL, "ctx is NULL");
  if (n_frames > NOALLOC_MAX_FRAMES)
    return fail(M3E_EINVAL, "m3e_select_frames_noalloc takes at most %lld frames per call, got %lld",
                (long long)NOALLOC_MAX_FRAMES, (long long)n_frames);
  int rc = check_batch(d_hits, d_frame_off, n_frames, d_keep, d_reason);
  if (rc) return rc;
  x->last_launches = 0;
  x->prof_valid = false;
  if (n_frames == 0) return M3E_OK;
  DeviceGuard guard(x->device);
  int* scratch = nullptr;
  rc = noalloc_scratch(x->device, &scratch);
  if (rc) return rc;
  KParams p{};
  p.col_lut = x->col_lut;
  p.row_lut = x->row_lut;
  p.err = x->err;
  p.work = scratch;
  p.defer_list = scratch + NOALLOC_HEAD;
  p.defer_count = scratch + 1;
  p.in_list = scratch + NOALLOC_HEAD;
  p.in_count = scratch + 1;
  p.defer_hits = x->defer_hits;  // the same warp/CTA split as the fused entry point
  p.grab = x->grab;
  p.hits = d_hits;
  p.off = d_frame_off;
  p.n_frames = n_frames;
  p.keep = d_keep;
  p.reason = d_reason;
  // the queue head and the deferred count start at zero; the list is written before it is read
  CUDA_TRY(cudaMemsetAsync(scratch, 0, 2 * sizeof(int), s));
  CUDA_TRY(launch_fused(x->dc, p, x->sms * x->fused_bpsm, false, s));
  CUDA_TRY(launch_deferred(x->dc, p, 2 * x->sms, false, s));
  x->last_launches = 2;
  return M3E_OK;
}

// ------------------------------------------------------------------ persistent batched form

struct m3e_graph {
  m3e_ctx* ctx = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

extern "C" int m3e_prepare(m3e_ctx* x, int64_t max_frames) {
  if (!x) return fail(M3E_EINVAL, "ctx is NULL");
  if (max_frames < 0 || max_frames > (int64_t)1 << 30) return fail(M3E_EINVAL, "max_frames out of range");
  DeviceGuard guard(x->device);
  return ensure_scratch(x->main, max_frames > 1 ? max_frames : 1, true);
}

extern "C" int m3e_graph_create(m3e_ctx* x, int form, const int32_t* d_hits, const int64_t* d_off, int64_t n,
                                uint8_t* d_keep, uint8_t* d_reason, m3e_graph** out) {
  if (!x || !out) return fail(M3E_EINVAL, "NULL argument");
  *out = nullptr;
  if (form != FORM_STAGED && form != FORM_FUSED) return fail(M3E_EINVAL, "graph form must be 0 (staged) or 1 (fused)");
  int rc = check_batch(d_hits, d_off, n, d_keep, d_reason);
  if (rc) return rc;
  if (n < 1) return fail(M3E_EINVAL, "a graph needs at least one frame");
  if (n > x->main.defer_cap || (form == FORM_STAGED && n > x->main.frames_cap))
    return fail(M3E_ESTATE, "call m3e_prepare(ctx, %lld) before capturing", (long long)n);
  DeviceGuard guard(x->device);
  m3e_graph* gr = new (std::nothrow) m3e_graph();
  if (!gr) return fail(M3E_ENOMEM, "graph");
  gr->ctx = x;
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
    delete gr;
    return fail(M3E_ECUDA, "capture stream");
  }
  KParams p = base_params(x, x->main);
  p.hits = d_hits;
  p.off = d_off;
  p.n_frames = n;
  p.keep = d_keep;
  p.reason = d_reason;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    rc = enqueue(x, x->main, p, form, false, cs, false);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    gr->graph = g;
    if (rc == M3E_OK && e2 != cudaSuccess) rc = fail(M3E_ECUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e2));
    if (rc == M3E_OK) {
      e = cudaGraphInstantiate(&gr->exec, gr->graph, 0);
      if (e != cudaSuccess) rc = fail(M3E_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
    }
  } else {
    rc = fail(M3E_ECUDA, "cudaStreamBeginCapture: %s", cudaGetErrorString(e));
  }
  cudaStreamDestroy(cs);
  if (rc) {
    m3e_graph_destroy(gr);
    return rc;
  }
  *out = gr;
  return M3E_OK;
}

extern "C" int m3e_graph_launch(m3e_graph* gr, cudaStream_t s) {
  if (!gr || !gr->exec) return fail(M3E_EINVAL, "graph is NULL");
  DeviceGuard guard(gr->ctx->device);
  CUDA_TRY(cudaGraphLaunch(gr->exec, s));
  return M3E_OK;
}

extern "C" int m3e_graph_destroy(m3e_graph* gr) {
  if (!gr) return M3E_OK;
  if (gr->exec) cudaGraphExecDestroy(gr->exec);
  if (gr->graph) cudaGraphDestroy(gr->graph);
  delete gr;
  return M3E_OK;
}

// Autotuner: time the staged form on the calibration batch for each point of a
// small grid of launch parameters (median of three runs after one warm-up on a
// private stream) and keep the fastest.
extern "C" int m3e_autotune(m3e_ctx* x, const int32_t* d_hits, const int64_t* d_off, int64_t n, uint8_t* d_keep,
                            uint8_t* d_reason, m3e_tuning* out) {
  if (!x || !out) return fail(M3E_EINVAL, "NULL argument");
  int rc = check_batch(d_hits, d_off, n, d_keep, d_reason);
  if (rc) return rc;
  if (n < 1) return fail(M3E_EINVAL, "calibration batch is empty");
  DeviceGuard guard(x->device);
  rc = ensure_scratch(x->main, n, true);
  if (rc) return rc;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  constexpr float AUTOTUNE_MARGIN = 0.02f;
  const int s1max = stage_blocks_per_sm(1);
  const int grabs[] = {1, 2, 4, 8, 16};
  const int dhits[] = {96, 128, W_HITS};
  const int s1s[] = {s1max, s1max > 2 ? (s1max + 1) / 2 : s1max};
  const int g0 = x->grab, d0 = x->defer_hits, b0 = x->s1_bpsm;
  auto run = [&](float* ms) -> int {
    KParams p = base_params(x, x->main);
    p.hits = d_hits;
    p.off = d_off;
    p.n_frames = n;
    p.keep = d_keep;
    p.reason = d_reason;
    float t[5];
    int r = enqueue(x, x->main, p, FORM_STAGED, false, st, false);  // warm-up
    for (int k = 0; k < 5 && r == M3E_OK; ++k) {
      CUDA_TRY(cudaEventRecord(e0, st));
      r = enqueue(x, x->main, p, FORM_STAGED, false, st, false);
      CUDA_TRY(cudaEventRecord(e1, st));
      CUDA_TRY(cudaEventSynchronize(e1));
      CUDA_TRY(cudaEventElapsedTime(&t[k], e0, e1));
    }
    if (r) return r;
    std::sort(t, t + 5);
    *ms = t[2];
    return M3E_OK;
  };
  float ms_def = 0.f;
  rc = run(&ms_def);
  float best = ms_def;
  int bg = g0, bd = d0, bb = b0, tried = 1;
  for (int g : grabs)
    for (int d : dhits)
      for (int b : s1s) {
        if (rc) break;
        x->grab = g;
        x->defer_hits = d;
        x->s1_bpsm = b;
        float ms = 0.f;
        rc = run(&ms);
        ++tried;
        // a configuration replaces the current choice only when it is clearly faster:
        // differences within the run-to-run spread of a short batch are noise
        if (rc == M3E_OK && ms < best * (1.f - AUTOTUNE_MARGIN)) {
          best = ms;
          bg = g;
          bd = d;
          bb = b;
        }
      }
  x->grab = bg;
  x->defer_hits = bd;
  x->s1_bpsm = bb;
  // then, one axis at a time from that point: the middle tier's CTA size and the
  // track stage's resident CTAs per SM
  float worst = best;
  int bm = x->mid_threads, b2 = x->s2_bpsm;
  const int s2max = stage_blocks_per_sm(2);
  const int mids[] = {128, 256, 512};
  for (int m : mids) {
    if (rc || m == bm) continue;
    const int pm = x->mid_threads, pb = x->s1m_bpsm;
    x->mid_threads = m;
    x->s1m_bpsm = stage1_mid_blocks_per_sm(m);
    float ms = 0.f;
    rc = run(&ms);
    ++tried;
    worst = ms > worst ? ms : worst;
    if (rc == M3E_OK && ms < best * (1.f - AUTOTUNE_MARGIN)) {
      best = ms;
      bm = m;
    } else {
      x->mid_threads = pm;
      x->s1m_bpsm = pb;
    }
  }
  const int s2s[] = {s2max, s2max - 1, (s2max + 1) / 2};
  for (int b : s2s) {
    if (rc || b < 1 || b == b2) continue;
    const int pb = x->s2_bpsm;
    x->s2_bpsm = b;
    float ms = 0.f;
    rc = run(&ms);
    ++tried;
    worst = ms > worst ? ms : worst;
    if (rc == M3E_OK && ms < best * (1.f - AUTOTUNE_MARGIN)) {
      best = ms;
      b2 = b;
    } else {
      x->s2_bpsm = pb;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  if (rc) return rc;
  out->frames_per_grab = bg;
  out->defer_hits = bd;
  out->s1_ctas_per_sm = bb;
  out->configs_tried = tried;
  out->ms_default = ms_def;
  out->ms_best = best;
  out->mid_cta_threads = x->mid_threads;
  out->s2_ctas_per_sm = x->s2_bpsm;
  out->ms_worst = worst;
  return M3E_OK;
}

// ------------------------------------------------------------------ streaming

namespace {

KParams stream_base(m3e_ctx* x) {
  KParams p{};
  p.col_lut = x->col_lut;
  p.row_lut = x->row_lut;
  p.err = x->err;
  p.defer_hits = W_HITS;
  p.grab = 1;
  return p;
}

}  // namespace

int m3e_stream_open(m3e_ctx* x, const m3e_stream_params* params) {
  if (!x) return fail(M3E_EINVAL, "ctx is NULL");
  if (x->stream) return fail(M3E_ESTATE, "stream already open");
  DeviceGuard guard(x->device);
  return stream_create(x->device, x->sms, x->dc, stream_base(x), params, &x->stream);
}

int m3e_stream_submit(m3e_ctx* x, const int32_t* h_packet, int32_t n_hits, uint64_t tag, m3e_result* h_result_slot) {
  if (!x) return fail(M3E_EINVAL, "ctx is NULL");
  if (!x->stream) {
    DeviceGuard guard(x->device);
    const int rc = stream_create(x->device, x->sms, x->dc, stream_base(x), nullptr, &x->stream);
    if (rc) return rc;
  }
  return stream_submit(x->stream, h_packet, n_hits, tag, h_result_slot);
}

int m3e_stream_submit_many(m3e_ctx* x, const int32_t* h_hits, const int64_t* h_frame_off, int64_t n_frames,
                           const uint64_t* tags, m3e_result* h_results, int64_t* n_admitted) {
  if (n_admitted) *n_admitted = 0;
  if (!x) return fail(M3E_EINVAL, "ctx is NULL");
  if (!x->stream) {
    DeviceGuard guard(x->device);
    const int rc = stream_create(x->device, x->sms, x->dc, stream_base(x), nullptr, &x->stream);
    if (rc) return rc;
  }
  return stream_submit_many(x->stream, h_hits, h_frame_off, n_frames, tags, h_results, n_admitted);
}

int m3e_stream_poll(m3e_ctx* x, m3e_stream_status* out) {
  if (!x || !out) return fail(M3E_EINVAL, "ctx or out is NULL");
  if (!x->stream) return fail(M3E_ESTATE, "stream not open");
  return stream_poll(x->stream, out);
}

int m3e_stream_drain(m3e_ctx* x, int64_t timeout_ms) {
  if (!x) return fail(M3E_EINVAL, "ctx is NULL");
  if (!x->stream) return M3E_OK;
  if (timeout_ms < 0) return fail(M3E_EINVAL, "timeout_ms < 0");
  return stream_drain(x->stream, timeout_ms);
}

int m3e_stream_close(m3e_ctx* x) {
  if (!x) return fail(M3E_EINVAL, "ctx is NULL");
  if (!x->stream) return M3E_OK;
  DeviceGuard guard(x->device);
  const int rc = stream_destroy(x->stream);
  x->stream = nullptr;
  return rc;
}

int m3e_stream_replay(m3e_ctx* x, const int32_t* h_hits, const int64_t* h_frame_off, int64_t n_frames,
                      double rate_hz, uint64_t seed, uint8_t* out_keep, uint8_t* out_reason,
                      int64_t* out_lat_submit_ns, int64_t* out_lat_arrival_ns, m3e_replay_stats* out) {
  if (!x) return fail(M3E_EINVAL, "ctx is NULL");
  if (!x->stream) {
    DeviceGuard guard(x->device);
    const int rc = stream_create(x->device, x->sms, x->dc, stream_base(x), nullptr, &x->stream);
    if (rc) return rc;
  }
  return stream_replay(x->stream, h_hits, h_frame_off, n_frames, rate_hz, seed, out_keep, out_reason,
                       out_lat_submit_ns, out_lat_arrival_ns, out);
}

// ------------------------------------------------------------------ fit gradient

namespace {

int fit_call(m3e_ctx* x, const int32_t* d_hits, const int64_t* d_off, int64_t n_frames, const int32_t* d_cand,
             int64_t n_cand, const float* d_params, float* chi2_each, float* chi2_sum, float* grad, cudaStream_t s,
             float* kappa_each = nullptr) {
  if (!x) return fail(M3E_EINVAL, "ctx is NULL");
  if (n_frames < 0 || n_cand < 0) return fail(M3E_EINVAL, "n_frames and n_cand must be >= 0");
  if (!d_off || !d_params || (n_cand > 0 && (!d_cand || !d_hits)))
    return fail(M3E_EINVAL, "frame_off, params, cand and hits must not be NULL");
  if (((uintptr_t)d_cand & 15) != 0) return fail(M3E_EINVAL, "cand must be 16-byte aligned (rows of 4 int32)");
  DeviceGuard guard(x->device);
  const int nb = fit_grad_blocks(x->sms, n_cand);
  if (nb > x->fit_partial_blocks) {
    cudaFree(x->fit_partial);
    x->fit_partial = nullptr;
    x->fit_partial_blocks = 0;
    CUDA_TRY(cudaMalloc(&x->fit_partial, sizeof(double) * fit_grad_partial_size() * (size_t)nb));
    x->fit_partial_blocks = nb;
  }
  if (!x->fit_nvalid) CUDA_TRY(cudaMalloc(&x->fit_nvalid, sizeof(unsigned long long)));
  CUDA_TRY(cudaMemsetAsync(x->fit_nvalid, 0, sizeof(unsigned long long), s));
  CUDA_TRY(launch_fit_grad(x->dc, d_hits, d_off, n_frames, d_cand, n_cand, d_params, x->col_lut, x->row_lut,
                           x->fit_partial, nb, x->fit_nvalid, chi2_each, kappa_each, chi2_sum, grad, s));
  return M3E_OK;
}

}  // namespace

int m3e_fit_grad(m3e_ctx* x, const int32_t* d_hits, const int64_t* d_frame_off, int64_t n_frames,
                 const int32_t* d_cand, int64_t n_cand, const float* d_params, float* d_chi2_sum, float* d_grad,
                 cudaStream_t stream) {
  if (!d_chi2_sum) return fail(M3E_EINVAL, "chi2_sum must not be NULL");
  return fit_call(x, d_hits, d_frame_off, n_frames, d_cand, n_cand, d_params, nullptr, d_chi2_sum, d_grad, stream);
}

int m3e_fit_chi2(m3e_ctx* x, const int32_t* d_hits, const int64_t* d_frame_off, int64_t n_frames,
                 const int32_t* d_cand, int64_t n_cand, const float* d_params, float* d_chi2_each,
                 cudaStream_t stream) {
  if (!d_chi2_each && n_cand > 0) return fail(M3E_EINVAL, "chi2_each must not be NULL");
  return fit_call(x, d_hits, d_frame_off, n_frames, d_cand, n_cand, d_params, d_chi2_each, nullptr, nullptr,
                  stream);
}

int m3e_fit_kappa(m3e_ctx* x, const int32_t* d_hits, const int64_t* d_frame_off, int64_t n_frames,
                  const int32_t* d_cand, int64_t n_cand, const float* d_params, float* d_kappa_each,
                  cudaStream_t stream) {
  if (!d_kappa_each && n_cand > 0) return fail(M3E_EINVAL, "kappa_each must not be NULL");
  return fit_call(x, d_hits, d_frame_off, n_frames, d_cand, n_cand, d_params, nullptr, nullptr, nullptr, stream,
                  d_kappa_each);
}

int m3e_fit_valid_count(m3e_ctx* x, cudaStream_t stream, int64_t* out) {
  if (!x || !out) return fail(M3E_EINVAL, "ctx or out is NULL");
  *out = 0;
  if (!x->fit_nvalid) return M3E_OK;
  DeviceGuard guard(x->device);
  if (!x->h_fit_nvalid) CUDA_TRY(cudaMallocHost(&x->h_fit_nvalid, sizeof(unsigned long long)));
  CUDA_TRY(cudaMemcpyAsync(x->h_fit_nvalid, x->fit_nvalid, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                           stream));
  CUDA_TRY(cudaStreamSynchronize(stream));
  *out = (int64_t)*x->h_fit_nvalid;
  return M3E_OK;
}
