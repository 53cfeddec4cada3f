// Internal definitions shared by the kernels and the C ABI of libm3e.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "m3e.h"

namespace m3e {

constexpr int NB = 32;            // phi bins per layer (power of two)
constexpr int NBK = 4 * NB;       // (layer, bin) buckets
constexpr int DEFERRED = -1;      // process_frame result: frame too large for the warp stage

// Shared-memory capacities of the two frame stages.  The warp stage holds
// typical frames; anything above its capacities is re-run by the CTA stage,
// whose capacities are the configuration limits.
constexpr int W_HITS = 160, W_TRIP = 160, W_TRK = 48, W_COMBO = 512;
constexpr int W_P01 = 384;        // warp stage: Phi01 partners of 32 layer-1 hits
constexpr int W_L0 = 64, W_L2 = 64;  // warp stage: layer-0 / layer-2 hits (bit masks of two words)
constexpr int NZB = 64;           // warp stage: z bins of the layer-2 order
constexpr int W_CAND = 256;       // warp stage: candidate triplets written per step
constexpr int C_HITS = 4096, C_TRIP = 1024, C_TRK = 128, C_COMBO = 1024;
constexpr int WARPS_PER_CTA = 4;  // persistent warp kernel: warps (frames in flight) per CTA
constexpr int CTA_THREADS = 256;  // large-frame kernel
constexpr int PLAIN_THREADS = 128;  // plain per-frame kernel

// Geometry and cuts, precomputed on the host in FP64 and rounded once.
struct DevCfg {
  float r[4];
  float inv_dr01, inv_dr12;   // 1/(r1 - r0), 1/(r2 - r1), nominal radii
  float dr12;                 // r2 - r1
  float zoff2, izw2;          // layer-2 z bin of the warp stage: (z + zoff2) * izw2, NZB bins over the length
  float c01, c12;             // cos(phi_max) * r_i * r_j: a pair passes when h_i . h_j >= c
  float dl_max;               // |Delta lambda| <= dl_max
  float rtc_lo2, rtc_hi2;     // (2 rtc_min)^2, (2 rtc_max)^2 against (d01 d12 d20)^2 / cross^2
  int k01, k12;               // phi-bin half windows of the two pair cuts
  int ntot[4], ncol[4], nlad[4], nrow[4];
  float intot[4];             // 1 / ntot, rounded once (phi bin of a column, decode)
  float phs_hi[4], phs_lo[4]; // 2 pi / ntot as a sum of two floats (phi of a column by exact FP32 steps)
  int col_off[4], row_off[4]; // offsets of each layer in the look-up tables
  // the same per-layer integers packed as 16-bit fields (layer L in bits 16 L ..), read
  // by decode with shifts instead of loads indexed by the hit's layer
  unsigned long long pk_nlad, pk_ncol, pk_nrow, pk_coloff, pk_rowoff;
  // the decode constants of layer L in one 16-byte entry, copied to shared memory by
  // the selection kernels: {nlad | ncol << 6 | nrow << 15, col_off, row_off, 1/ntot bits}
  uint4 ltab[4];
  float kB;                   // p [MeV] = kB * R [mm]
  float hl[4];                // Highland width numerator: sigma_MS(p) = hl[layer] / p
  float ihl[4];               // 1 / hl
  float chi2_trk;
  float r3;
  float colw3;                // one layer-3 column in phi plus rounding slack (4th-hit ring search)
  float me2, m_mu, e_win;
  float isect_lim;            // target_r + isect_margin
  float tgt_r, tgt_h, vtx_chi2, tgt_dist, ptot_max;
  float sig_pix2;             // pitch^2 / 12
  int max_hits, max_trip, max_trk, max_combo;
};

struct KParams {
  const int32_t* hits;
  const int64_t* off;
  int64_t n_frames;
  int64_t off_base;           // subtracted from off[] (chunked host entry point)
  uint8_t* keep;
  uint8_t* reason;
  unsigned long long* stats;  // m3e_stats viewed as an array, or nullptr
  const float4* col_lut;      // per global column: x, y, phi, 0
  const float* row_lut;       // per row: z
  int* work;                  // [0] work-queue head of a frame-parallel kernel
  int* err;                   // error flags (ERR_*), latched until m3e_check
  int* defer_list;            // frames a kernel cannot finish are appended here ...
  int* defer_count;           // ... and counted here
  const int* in_list;         // list-driven kernels: the frames to run ...
  const int* in_count;        // ... and their number
  int grab;                   // frames per work-queue grab
  int defer_hits;             // warp stages defer frames with more hits (<= W_HITS)
  const unsigned* gate;       // host entry point: per-chunk arrival flags (written by the copy engine), or null
  int gate_frames;            // frames per chunk
  int gate_ms;                // longest wait for one chunk
  m3e_dump dump;              // all pointers null unless debugging
};

// Global scratch of the staged form (see m3e_staged.cu), sized per batch.
struct SParams {
  float4* hp;                  // sorted hits of the pending frames (from the hit allocator): x, y, z, phi
  uint32_t* haddr;
  uint16_t* hidx;              // input index of each sorted hit (candidate record only)
  int* list1;                  // frames deferred by the warp tier of stage 1
  int* list1b;                 // frames deferred by the middle tier of stage 1
  int* list2;                  // frames deferred by the top tier of stage 1 and by stage 3
  int* lcount;                 // [0] list1 count, [1] list2 count, [2] list1b count
  uint16_t* l3;                // [F][NB + 1] layer-3 phi-bin starts, frame-relative
  int *fstate, *ftbase, *fntrip, *ffound;  // per frame: state, triplet range, vertex found
  long long* fcbase;           // per frame: first combination
  int* fncombo;
  int4* trip;                  // {frame, first sorted hit, i0 | i1 << 16, i2} (frame-relative indices), frame -1 = unused
  float2* tek;                 // per triplet: (eps E, P_z) of a kept track, (0, 0) otherwise
  float4* trec;                // per triplet: 16-float track record when kept
  int4* combo;                 // {frame, triplet a, triplet b, triplet e-}, frame -1 = unused
  unsigned long long* counters;  // [0] triplets, [1] combinations, [2] stage-3 queue, [3] sorted hits
  int64_t trip_cap, combo_cap, hits_cap;
};

enum { ST_FRAMES = 0, ST_HITS, ST_PAIRS, ST_TTESTS, ST_TRIP, ST_TRK, ST_ETEST, ST_COMBO, ST_VTX, ST_DEFER,
       ST_PZOPEN, ST_VTXOPEN, ST_REASON0 };

enum { ERR_BADHIT = 1, ERR_NEGSIZE = 2, ERR_GATE = 4 };

// Host-side launchers (m3e_fused.cu, m3e_staged.cu).
cudaError_t launch_fused(const DevCfg& c, const KParams& p, int grid, bool debug, cudaStream_t s);
cudaError_t launch_deferred(const DevCfg& c, const KParams& p, int grid, bool debug, cudaStream_t s);
cudaError_t launch_plain(const DevCfg& c, const KParams& p, bool debug, cudaStream_t s);
cudaError_t launch_staged(const DevCfg& c, const KParams& p, const SParams& s, const int grids[6], bool debug,
                          cudaStream_t st, cudaEvent_t* ev, cudaEvent_t after_s1 = nullptr, int mid_threads = 256);
int stage1_mid_blocks_per_sm(int threads);  // resident CTAs per SM of the stage-1 middle tier
size_t stage1c_smem_bytes();
int fused_blocks_per_sm();
int stage_blocks_per_sm(int stage);
size_t fused_smem_bytes();
size_t cta_smem_bytes();

// Hit ingest (m3e_ingest.cu): addresses -> FP32 x, y, z (and phi unless null) as SoA.
int ingest_blocks_per_sm();
cudaError_t launch_ingest(const DevCfg& c, const int32_t* hits, int64_t n, const float4* col_lut, const float* row_lut,
                          float* x, float* y, float* z, float* phi, int* err, int grid, cudaStream_t s);

// Gradient of the fit chi2 (m3e_grad.cu).
int fit_grad_blocks(int sms, int64_t n_cand);
int fit_grad_partial_size();
cudaError_t launch_fit_grad(const DevCfg& c, const int32_t* hits, const int64_t* off, int64_t n_frames,
                            const int32_t* cand, int64_t n_cand, const float* params, const float4* col_lut,
                            const float* row_lut, double* partial, int nblocks, unsigned long long* n_valid,
                            float* chi2_each, float* kappa_each, float* chi2_sum, float* grad, cudaStream_t s);

// Records the calling thread's error message (m3e_last_error_string) and returns code.
int m3e_set_error(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));

// Streaming engine (m3e_stream.cu).
struct StreamEngine;
int stream_create(int device, int sms, const DevCfg& dc, const KParams& base, const m3e_stream_params* sp,
                  StreamEngine** out);
int stream_submit(StreamEngine* e, const int32_t* pkt, int32_t n_hits, uint64_t tag, m3e_result* res);
int stream_submit_many(StreamEngine* e, const int32_t* hits, const int64_t* off, int64_t n_frames,
                       const uint64_t* tags, m3e_result* res, int64_t* admitted);
int stream_poll(StreamEngine* e, m3e_stream_status* out);
int stream_drain(StreamEngine* e, int64_t timeout_ms);
int stream_destroy(StreamEngine* e);
int stream_replay(StreamEngine* e, const int32_t* hits, const int64_t* off, int64_t n_frames, double rate_hz,
                  uint64_t seed, uint8_t* out_keep, uint8_t* out_reason, int64_t* lat_submit, int64_t* lat_arrival,
                  m3e_replay_stats* st);

}  // namespace m3e
