// C ABI of libm3e: context, parameter checks, look-up tables, launches.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "m3e_internal.cuh"

using namespace m3e;

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

constexpr int HOST_CHUNKS = 8;  // chunks of the host entry point (double-buffered)

}  // namespace

struct m3e_ctx {
  int device = 0;
  int sms = 1;
  int blocks_per_sm = 1;
  int grab = 4;
  m3e_config cfg{};
  DevCfg dc{};
  float4* col_lut = nullptr;
  float* row_lut = nullptr;
  int* work = nullptr;          // [0] queue head, [1] deferred count, [2] error flags
  int* defer_list = nullptr;
  int64_t defer_cap = 0;
  int* h_err = nullptr;         // pinned error-flag readback
  int last_launches = 0;
  // host entry point staging
  cudaStream_t hs[2] = {nullptr, nullptr};
  cudaEvent_t he[2] = {nullptr, nullptr};
  int32_t* d_hits[2] = {nullptr, nullptr};
  int64_t* d_off[2] = {nullptr, nullptr};
  uint8_t* d_out[2] = {nullptr, nullptr};
  int* d_work2[2] = {nullptr, nullptr};
  int* d_defer2[2] = {nullptr, nullptr};
  int64_t cap_hits[2] = {0, 0}, cap_frames[2] = {0, 0};
  // kernel timing
  bool prof = false;
  bool prof_valid = false;
  bool prof_plain = false;
  cudaEvent_t pe[3] = {nullptr, nullptr, nullptr};
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
    const double x = c.x_over_X0[L];
    d.hl[L] = (float)(13.6 * std::sqrt(x) * (1.0 + 0.038 * std::log(x)));
  }
  int co = 0, ro = 0;
  for (int L = 0; L < 4; ++L) {
    d.col_off[L] = co;
    d.row_off[L] = ro;
    co += d.ntot[L];
    ro += d.nrow[L];
  }
  d.inv_dr01 = (float)(1.0 / (c.r_mm[1] - c.r_mm[0]));
  d.inv_dr12 = (float)(1.0 / (c.r_mm[2] - c.r_mm[1]));
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

KParams base_params(m3e_ctx* x) {
  KParams p{};
  p.col_lut = x->col_lut;
  p.row_lut = x->row_lut;
  p.work = x->work;
  p.err = x->work + 2;
  p.defer_list = x->defer_list;
  p.grab = x->grab;
  return p;
}

int ensure_defer(m3e_ctx* x, int64_t n) {
  if (n <= x->defer_cap) return M3E_OK;
  int64_t cap = x->defer_cap ? x->defer_cap : 4096;
  while (cap < n) cap *= 2;
  if (x->defer_list) CUDA_TRY(cudaFree(x->defer_list));
  x->defer_list = nullptr;
  x->defer_cap = 0;
  if (cudaMalloc(&x->defer_list, sizeof(int) * cap) != cudaSuccess)
    return fail(M3E_ENOMEM, "deferred list of %lld frames", (long long)cap);
  x->defer_cap = cap;
  return M3E_OK;
}

int check_batch(const int32_t* hits, const int64_t* off, int64_t n, const uint8_t* keep, const uint8_t* reason) {
  if (n < 0 || n > (int64_t)1 << 30) return fail(M3E_EINVAL, "n_frames %lld out of range", (long long)n);
  if (n > 0 && (!off || !keep || !reason)) return fail(M3E_EINVAL, "NULL frame_off/keep/reason");
  (void)hits;
  return M3E_OK;
}

// Enqueue the persistent kernel and the deferred-frame kernel on stream s with
// the given work/deferred scratch.
int enqueue_select(m3e_ctx* x, KParams p, bool debug, cudaStream_t s, bool timed) {
  CUDA_TRY(cudaMemsetAsync(p.work, 0, 2 * sizeof(int), s));
  const int grid = x->sms * x->blocks_per_sm;
  if (timed) CUDA_TRY(cudaEventRecord(x->pe[0], s));
  CUDA_TRY(launch_select(x->dc, p, grid, debug, s));
  if (timed) CUDA_TRY(cudaEventRecord(x->pe[1], s));
  CUDA_TRY(launch_deferred(x->dc, p, 2 * x->sms, debug, s));
  if (timed) CUDA_TRY(cudaEventRecord(x->pe[2], s));
  x->last_launches = 2;
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
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, cuda_device) != cudaSuccess) {
    delete x;
    return fail(M3E_ECUDA, "cudaGetDeviceProperties");
  }
  x->sms = prop.multiProcessorCount;
  x->blocks_per_sm = select_blocks_per_sm();
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
            cudaMalloc(&x->work, 4 * sizeof(int)) == cudaSuccess &&
            cudaMallocHost(&x->h_err, sizeof(int)) == cudaSuccess;
  if (ok)
    ok = cudaMemcpy(x->col_lut, cl.data(), sizeof(float4) * ncolt, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(x->row_lut, rl.data(), sizeof(float) * nrowt, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemset(x->work, 0, 4 * sizeof(int)) == cudaSuccess;
  if (ok) ok = ensure_defer(x, 1 << 16) == M3E_OK;
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
  cudaDeviceSynchronize();
  cudaFree(x->col_lut);
  cudaFree(x->row_lut);
  cudaFree(x->work);
  cudaFree(x->defer_list);
  if (x->h_err) cudaFreeHost(x->h_err);
  for (int i = 0; i < 2; ++i) {
    cudaFree(x->d_hits[i]);
    cudaFree(x->d_off[i]);
    cudaFree(x->d_out[i]);
    cudaFree(x->d_work2[i]);
    cudaFree(x->d_defer2[i]);
    if (x->hs[i]) cudaStreamDestroy(x->hs[i]);
    if (x->he[i]) cudaEventDestroy(x->he[i]);
  }
  for (int i = 0; i < 3; ++i)
    if (x->pe[i]) cudaEventDestroy(x->pe[i]);
  delete x;
  return M3E_OK;
}

int m3e_set_launch(m3e_ctx* x, int frames_per_grab, int ctas_per_sm) {
  if (!x) return fail(M3E_EINVAL, "ctx is NULL");
  if (frames_per_grab < 1 || frames_per_grab > 64) return fail(M3E_EINVAL, "frames_per_grab 1..64");
  DeviceGuard guard(x->device);
  const int maxb = select_blocks_per_sm();
  if (ctas_per_sm < 0 || ctas_per_sm > maxb) return fail(M3E_EINVAL, "ctas_per_sm 0..%d", maxb);
  x->grab = frames_per_grab;
  x->blocks_per_sm = ctas_per_sm ? ctas_per_sm : maxb;
  return M3E_OK;
}

int m3e_last_launch_count(const m3e_ctx* x) { return x ? x->last_launches : 0; }

int m3e_set_profiling(m3e_ctx* x, int on) {
  if (!x) return fail(M3E_EINVAL, "ctx is NULL");
  DeviceGuard guard(x->device);
  for (int i = 0; i < 3 && on; ++i)
    if (!x->pe[i]) CUDA_TRY(cudaEventCreate(&x->pe[i]));
  x->prof = on != 0;
  x->prof_valid = false;
  return M3E_OK;
}

int m3e_kernel_times(m3e_ctx* x, float* main_ms, float* deferred_ms) {
  if (!x || !main_ms || !deferred_ms) return fail(M3E_EINVAL, "NULL argument");
  if (!x->prof_valid) return fail(M3E_ESTATE, "no timed select call since profiling was enabled");
  DeviceGuard guard(x->device);
  CUDA_TRY(cudaEventSynchronize(x->pe[x->prof_plain ? 1 : 2]));
  CUDA_TRY(cudaEventElapsedTime(main_ms, x->pe[0], x->pe[1]));
  *deferred_ms = 0.f;
  if (!x->prof_plain) CUDA_TRY(cudaEventElapsedTime(deferred_ms, x->pe[1], x->pe[2]));
  return M3E_OK;
}

static int select_common(m3e_ctx* x, const int32_t* hits, const int64_t* off, int64_t n, uint8_t* keep,
                         uint8_t* reason, m3e_stats* stats, const m3e_dump* dump, bool plain, cudaStream_t s) {
  if (!x) return fail(M3E_EINVAL, "ctx is NULL");
  int rc = check_batch(hits, off, n, keep, reason);
  if (rc) return rc;
  x->last_launches = 0;
  if (n == 0) return M3E_OK;
  DeviceGuard guard(x->device);
  KParams p = base_params(x);
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
  x->prof_valid = false;
  if (plain) {
    if (timed) CUDA_TRY(cudaEventRecord(x->pe[0], s));
    CUDA_TRY(launch_plain(x->dc, p, dump != nullptr, s));
    if (timed) CUDA_TRY(cudaEventRecord(x->pe[1], s));
    x->last_launches = 1;
    x->prof_valid = timed;
    x->prof_plain = true;
    return M3E_OK;
  }
  rc = ensure_defer(x, n);
  if (rc) return rc;
  p.defer_list = x->defer_list;
  rc = enqueue_select(x, p, dump != nullptr, s, timed);
  x->prof_valid = timed && rc == M3E_OK;
  x->prof_plain = false;
  return rc;
}

int m3e_select_frames(m3e_ctx* x, const int32_t* d_hits, const int64_t* d_off, int64_t n, uint8_t* d_keep,
                      uint8_t* d_reason, m3e_stats* d_stats, cudaStream_t s) {
  return select_common(x, d_hits, d_off, n, d_keep, d_reason, d_stats, nullptr, false, s);
}

int m3e_select_frames_plain(m3e_ctx* x, const int32_t* d_hits, const int64_t* d_off, int64_t n, uint8_t* d_keep,
                            uint8_t* d_reason, m3e_stats* d_stats, cudaStream_t s) {
  return select_common(x, d_hits, d_off, n, d_keep, d_reason, d_stats, nullptr, true, s);
}

int m3e_select_frames_debug(m3e_ctx* x, const int32_t* d_hits, const int64_t* d_off, int64_t n, uint8_t* d_keep,
                            uint8_t* d_reason, const m3e_dump* dump, cudaStream_t s) {
  if (!dump) return fail(M3E_EINVAL, "dump is NULL");
  return select_common(x, d_hits, d_off, n, d_keep, d_reason, nullptr, dump, false, s);
}

int m3e_check(m3e_ctx* x, cudaStream_t s) {
  if (!x) return fail(M3E_EINVAL, "ctx is NULL");
  DeviceGuard guard(x->device);
  CUDA_TRY(cudaMemcpyAsync(x->h_err, x->work + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  const int e = *x->h_err;
  if (e) {
    CUDA_TRY(cudaMemsetAsync(x->work + 2, 0, sizeof(int), s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return fail(M3E_EBADHIT, "invalid pixel address or frame size seen (flags %d)", e);
  }
  return M3E_OK;
}

// End to end from host memory.  Frames are cut into chunks of about equal hit
// count; chunk k uses buffer set k % 2 and internal stream k % 2, so the copies
// of one chunk overlap the kernels of the other.
int m3e_select_frames_host(m3e_ctx* x, const int32_t* h_hits, const int64_t* h_off, int64_t n, uint8_t* h_keep,
                           uint8_t* h_reason, cudaStream_t s) {
  if (!x) return fail(M3E_EINVAL, "ctx is NULL");
  int rc = check_batch(h_hits, h_off, n, h_keep, h_reason);
  if (rc) return rc;
  x->last_launches = 0;
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
  const int nch = (int)(n < HOST_CHUNKS ? n : HOST_CHUNKS);
  int64_t f0 = 0;
  int launches = 0;
  for (int k = 0; k < nch; ++k) {
    int64_t f1 = n;
    if (k + 1 < nch) {  // chunk end: first frame whose start reaches (k+1)/nch of the hits
      const int64_t target = h_off[0] + total * (k + 1) / nch;
      int64_t lo = f0 + 1, hi = n - (nch - k - 1);
      while (lo < hi) {
        const int64_t mid = (lo + hi) / 2;
        if (h_off[mid] >= target) hi = mid; else lo = mid + 1;
      }
      f1 = lo;
    }
    const int b = k & 1;
    const int64_t nf = f1 - f0, nh = h_off[f1] - h_off[f0];
    cudaStream_t hs = x->hs[b];
    if (nh > x->cap_hits[b]) {
      if (x->d_hits[b]) CUDA_TRY(cudaFree(x->d_hits[b]));
      x->d_hits[b] = nullptr;
      x->cap_hits[b] = 0;
      const int64_t cap = nh + nh / 4 + 1024;
      if (cudaMalloc(&x->d_hits[b], sizeof(int32_t) * cap) != cudaSuccess) return fail(M3E_ENOMEM, "staging hits");
      x->cap_hits[b] = cap;
    }
    if (nf > x->cap_frames[b]) {
      cudaFree(x->d_off[b]);
      cudaFree(x->d_out[b]);
      cudaFree(x->d_work2[b]);
      cudaFree(x->d_defer2[b]);
      x->d_off[b] = nullptr;
      x->d_out[b] = nullptr;
      x->d_work2[b] = nullptr;
      x->d_defer2[b] = nullptr;
      x->cap_frames[b] = 0;
      const int64_t cap = nf + nf / 4 + 1024;
      if (cudaMalloc(&x->d_off[b], sizeof(int64_t) * (cap + 1)) != cudaSuccess ||
          cudaMalloc(&x->d_out[b], 2 * cap) != cudaSuccess || cudaMalloc(&x->d_work2[b], 4 * sizeof(int)) != cudaSuccess ||
          cudaMalloc(&x->d_defer2[b], sizeof(int) * cap) != cudaSuccess)
        return fail(M3E_ENOMEM, "staging frames");
      CUDA_TRY(cudaMemsetAsync(x->d_work2[b], 0, 4 * sizeof(int), hs));
      x->cap_frames[b] = cap;
    }
    CUDA_TRY(cudaMemcpyAsync(x->d_hits[b], h_hits + h_off[f0], sizeof(int32_t) * nh, cudaMemcpyHostToDevice, hs));
    CUDA_TRY(cudaMemcpyAsync(x->d_off[b], h_off + f0, sizeof(int64_t) * (nf + 1), cudaMemcpyHostToDevice, hs));
    KParams p = base_params(x);
    p.hits = x->d_hits[b];
    p.off = x->d_off[b];
    p.off_base = h_off[f0];
    p.n_frames = nf;
    p.keep = x->d_out[b];
    p.reason = x->d_out[b] + x->cap_frames[b];
    p.work = x->d_work2[b];
    p.defer_list = x->d_defer2[b];
    rc = enqueue_select(x, p, false, hs, false);
    if (rc) return rc;
    launches += x->last_launches;
    CUDA_TRY(cudaMemcpyAsync(h_keep + f0, p.keep, nf, cudaMemcpyDeviceToHost, hs));
    CUDA_TRY(cudaMemcpyAsync(h_reason + f0, p.reason, nf, cudaMemcpyDeviceToHost, hs));
    f0 = f1;
  }
  for (int i = 0; i < 2; ++i) {
    CUDA_TRY(cudaEventRecord(x->he[i], x->hs[i]));
    CUDA_TRY(cudaStreamWaitEvent(s, x->he[i], 0));
  }
  x->last_launches = launches;
  return M3E_OK;
}

}  // extern "C"
