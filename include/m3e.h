/* m3e: GB300-native Mu3e online event selection (arXiv:2206.11535).
 *
 * The problem statement is the paper's (Sec. "Online Event Selection",
 * Sec. "Implementation"): a batch of frames of detector hits goes in, and one
 * keep/drop decision per frame comes out.  Per frame the library runs the three
 * steps of the paper: the selection cuts on hit triplets of layers 0-2
 * (Sec. "Selection Cuts", Algorithm 2), the triplet-fit track reconstruction
 * with the fourth layer and a chi2 < 32 cut (Sec. "Track Reconstruction",
 * Algorithm 3) and the geometric e+ e+ e- vertex selection (Sec. "Vertex Fit",
 * Algorithm 4).  Frames whose candidate lists overflow the caps are kept
 * unprocessed (Algorithms 2-4).
 *
 * Conventions of every entry point:
 *   - Return value: M3E_OK (0) or a negative M3E_E* code; the message of the
 *     last failure of the calling thread is m3e_last_error_string().
 *   - Pointers named d_* are DEVICE pointers owned by the caller, on the
 *     context's device; h_* are HOST pointers owned by the caller (pinned memory
 *     gives overlapped copies, pageable memory still works).
 *   - Work is enqueued asynchronously on the caller's stream; no call
 *     synchronises the device.  Results are valid once the stream has reached
 *     the call.  The context allocates only its own scratch (look-up tables,
 *     work queue, deferred-frame list, staging buffers of the host entry point).
 *   - A context is not safe for concurrent use by several host threads.
 *
 * Input format.  Frame f owns hits[frame_off[f] .. frame_off[f+1]) of a CSR
 * batch; frame_off has n_frames + 1 entries, non-decreasing.  A hit is a packed
 * int32 pixel address:
 *   bits [31:28] zero, [27:26] layer 0..3, [25:21] ladder, [20:13] column,
 *   [12:0] row.
 * Global column g = ladder * n_cols[layer] + column counts around the cylinder
 * from phi = 0; the pixel centre is (r cos phi, r sin phi, -H + (row + 1/2) pitch)
 * with phi = (g + 1/2) 2 pi / (n_ladders n_cols) (the paper's detector model of
 * four concentric cylinders, Sec. "Selection Cuts").  The hit order inside a
 * frame is arbitrary and does not change any result; duplicate addresses are
 * distinct hits.
 *
 * Output.  keep[f] is 1 for a frame to store, 0 to drop; reason[f] is one of
 * enum m3e_reason.  A frame holding an address outside the detector (or a
 * negative size) is kept with reason M3E_ERR_BADHIT and M3E_EBADHIT is latched
 * in the context (read it with m3e_check).
 */
#ifndef M3E_H
#define M3E_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

#define M3E_VERSION 100

enum m3e_status {
  M3E_OK = 0,
  M3E_EINVAL = -1,    /* bad argument or configuration */
  M3E_ENOMEM = -2,    /* device or host allocation failed */
  M3E_EBADHIT = -3,   /* a frame held an invalid pixel address (latched, see m3e_check) */
  M3E_ECUDA = -4,     /* a CUDA runtime call failed */
  M3E_EBUSY = -5,     /* admission refused (streaming) */
  M3E_ETIMEOUT = -6,  /* a bounded device wait expired */
  M3E_ESTATE = -7     /* call not valid in the context's current state */
};

enum m3e_reason {
  M3E_DROP = 0,             /* no signal-like vertex: drop the frame */
  M3E_VERTEX = 1,           /* an e+ e+ e- combination passed the vertex cuts */
  M3E_TRIPLET_OVERFLOW = 2, /* more than max_triplets selected triplets */
  M3E_TRACK_OVERFLOW = 3,   /* more than max_tracks tracks */
  M3E_COMBO_OVERFLOW = 4,   /* more than max_combos combinations passed the energy test */
  M3E_HIT_OVERFLOW = 5,     /* more than max_hits hits (staging capacity) */
  M3E_ERR_BADHIT = 6        /* invalid address or frame size */
};

/* Parameters.  Units mm, MeV, T, rad.  Plain data, versioned by its size. */
typedef struct {
  uint32_t size;                     /* must be sizeof(m3e_config) */
  double r_mm[4], half_len_mm[4];    /* layer radii and half lengths */
  int32_t n_ladders[4], n_cols[4], n_rows[4];
  double pitch_mm;
  double B_T, field_scale;           /* solenoid field along +z and its scale */
  double x_over_X0[4];               /* material per layer crossing (Highland width) */
  double k_MeV_per_T_mm, m_mu_MeV, m_e_MeV;
  double target_r_mm, target_half_len_mm;  /* hollow double-cone target */
  /* selection cuts (Sec. "Selection Cuts"), inclusive */
  double dlambda_max, phi01_max, phi12_max, rtc_min, rtc_max;
  double chi2_track_max;             /* strict: keep chi2 < chi2_track_max (32 in the paper) */
  /* vertex cuts (Sec. "Vertex Fit"), inclusive */
  double e_window, isect_margin, vtx_chi2_max, target_dist_max, ptot_max;
  int32_t max_hits;                  /* <= 4096 */
  int32_t max_triplets;              /* <= 1024 (768 in the paper) */
  int32_t max_tracks;                /* <= 128 */
  int32_t max_combos;                /* <= 1024 */
} m3e_config;

/* Per-batch counters, accumulated by atomics into caller-owned DEVICE memory
 * that the caller zeroes.  Work counts are per-frame sums. */
typedef struct {
  unsigned long long frames, hits;
  unsigned long long pair_tests;     /* Phi tests of layer-0/1 and layer-1/2 hit pairs */
  unsigned long long triplet_tests;  /* Delta-lambda tests after both Phi cuts */
  unsigned long long triplets;       /* selected triplets of frames that do not overflow (fits run);
                                        the cuts of an overflowing frame stop once it overflows */
  unsigned long long tracks;         /* tracks kept by the chi2 cut */
  unsigned long long energy_tests;   /* e+ e+ e- combinations tested for energy */
  unsigned long long combos;         /* combinations passing the energy test */
  unsigned long long vertexed;       /* combinations vertexed */
  unsigned long long deferred;       /* frames re-run by the large-frame path */
  unsigned long long pz_open;        /* combinations whose longitudinal momentum sum alone does not
                                        fail the |sum p| cut: the only ones whose vertex a run
                                        without statistics or candidate record evaluates */
  unsigned long long vertexed_pz_open; /* vertexed combinations among those */
  unsigned long long reasons[8];     /* frames per m3e_reason */
} m3e_stats;

/* Optional per-frame record of the candidates (parity checks and debugging):
 * caller-owned DEVICE arrays, frame f at offset f * cap.  Hit indices are INPUT
 * indices, the position of the hit within its frame's packet. */
typedef struct {
  int32_t cap_trip;        /* records kept per frame for triplets (<= max_triplets) */
  int32_t cap_combo;       /* records kept per frame for combinations (<= max_combos) */
  int32_t* n_trip;         /* [F] selected triplets (full count) */
  int32_t* trip;           /* [F][cap_trip][4] i0, i1, i2, i3 (i3 = -1 when no 4th hit; among
                              hits with equal address, which one is reported is unspecified) */
  int32_t* trk_status;     /* [F][cap_trip] 0 fit1 invalid, 1 no layer-3 crossing, 2 no layer-3
                              hit, 3 fit2 invalid, 4 chi2 >= cut, 5 kept */
  float* trk_val;          /* [F][cap_trip][4] kappa_bar, theta01, chi2, 4th-hit metric */
  int32_t* n_combo;        /* [F] combinations passing the energy test (full count) */
  int32_t* combo;          /* [F][cap_combo][4] triplet record index of e+, e+, e-, and
                              status | pass << 8 (status 0 no intersection, 1 emptied by the
                              target filter, 2 vertexed) */
  float* combo_val;        /* [F][cap_combo][4] energy sum - m_mu, chi2, target distance, |sum p| */
  float* combo_aux;        /* [F][cap_combo][4] or NULL: the values that decide the vertex status and
                              choice, for the boundary bands of a parity check: smallest relative
                              discriminant |h^2|/r_a^2 of the three circle pairs, smallest distance
                              (mm) of an intersection point from target_r + isect_margin, the
                              second-smallest chi2 over the intersection choices, 0 (FLT_MAX where
                              the vertex stopped before the quantity) */
} m3e_dump;

typedef struct m3e_ctx m3e_ctx;

/* Create a context on CUDA device cuda_device: checks the configuration, builds
 * the pixel look-up tables in FP64 (rounded once to FP32) and uploads them. */
int m3e_create(const m3e_config* cfg, int cuda_device, m3e_ctx** out);

/* Release the context and its device memory (synchronises the context's device). */
int m3e_destroy(m3e_ctx* ctx);

/* Select frames (the whole method of the paper, every step in CUDA kernels),
 * the throughput form: five persistent kernels that regroup the batch by
 * candidate (frames -> selected triplets -> tracks -> combinations -> decisions,
 * the candidates in device scratch); frames larger than a stage's capacity are
 * re-run by a CTA-per-frame kernel with identical decisions.  d_stats may be
 * NULL.  n_frames may be 0. */
int m3e_select_frames(m3e_ctx* ctx, const int32_t* d_hits, const int64_t* d_frame_off, int64_t n_frames,
                      uint8_t* d_keep, uint8_t* d_reason, m3e_stats* d_stats, cudaStream_t stream);

/* The same decisions through the fused form: one persistent kernel in which a
 * warp runs every stage of a frame in shared memory, frames from a device work
 * queue (lowest latency per frame; the form the streaming path uses). */
int m3e_select_frames_fused(m3e_ctx* ctx, const int32_t* d_hits, const int64_t* d_frame_off, int64_t n_frames,
                            uint8_t* d_keep, uint8_t* d_reason, m3e_stats* d_stats, cudaStream_t stream);

/* The same decisions through the plain per-frame form: one CTA per frame, one
 * launch per batch (the layout of the paper's main kernel, Algorithm 1). */
int m3e_select_frames_plain(m3e_ctx* ctx, const int32_t* d_hits, const int64_t* d_frame_off, int64_t n_frames,
                            uint8_t* d_keep, uint8_t* d_reason, m3e_stats* d_stats, cudaStream_t stream);

/* A selection with the candidate record filled in, through form 0 (staged, as
 * m3e_select_frames), 1 (fused) or 2 (plain); the vertex stage then evaluates
 * every combination instead of stopping at the first passing one. */
int m3e_select_frames_debug(m3e_ctx* ctx, int form, const int32_t* d_hits, const int64_t* d_frame_off,
                            int64_t n_frames, uint8_t* d_keep, uint8_t* d_reason, const m3e_dump* dump,
                            cudaStream_t stream);

/* End to end from HOST memory: copies the offsets and then the hits to the
 * device in chunks of frames on an internal copy stream, while one staged
 * selection over the whole batch runs on an internal compute stream, and copies
 * keep/reason back.  After each chunk the copy engine writes that chunk's arrival
 * flag; stage 1 takes a frame only once its chunk's flag is set, so it starts on
 * the first chunk while the later ones are still on their way.  A wait for a
 * chunk is bounded (m3e_set_host_pipeline); when it runs out the call's results
 * are undefined and M3E_ETIMEOUT is latched (m3e_check).  Returns after
 * enqueueing; the results are in h_keep/h_reason once `stream` has reached the
 * call (the caller's stream waits for both internal streams).  Host buffers that
 * are page-locked copy at full speed; others work, more slowly.  Consecutive calls
 * on one context must be ordered by the caller's stream. */
/* Settings of m3e_select_frames_host: at most max_chunks chunks (1..64, default
 * 16; a chunk holds at least 50,000 frames unless the batch is smaller), a wait of
 * at most wait_ms (1..60,000, default 2,000) for one chunk, and drop_chunk: -1 in
 * normal use; k >= 0 leaves chunk k's flag unset, so that stage 1 runs out of its
 * wait (a test of the bounded wait; the call then latches M3E_ETIMEOUT). */
int m3e_set_host_pipeline(m3e_ctx* ctx, int max_chunks, int wait_ms, int drop_chunk);

int m3e_select_frames_host(m3e_ctx* ctx, const int32_t* h_hits, const int64_t* h_frame_off, int64_t n_frames,
                           uint8_t* h_keep, uint8_t* h_reason, cudaStream_t stream);

/* Synchronise `stream` and return M3E_EBADHIT if any earlier call saw an invalid
 * address or frame size (and clear the latch), else M3E_OK. */
int m3e_check(m3e_ctx* ctx, cudaStream_t stream);

/* Tuning of the persistent kernel: frames taken per work-queue grab (1..64) and
 * resident CTAs per SM (0 = as many as fit). */
int m3e_set_launch(m3e_ctx* ctx, int frames_per_grab, int ctas_per_sm);

/* Size the context's scratch for batches of up to max_frames frames, so that the
 * select calls that follow allocate nothing (required before m3e_graph_create). */
int m3e_prepare(m3e_ctx* ctx, int64_t max_frames);

/* One batch as a CUDA graph (the persistent batched form, captured once and
 * relaunched): form 0 staged, 1 fused.  The graph holds the given pointers and
 * frame count; relaunching it reruns the selection on whatever those buffers hold.
 * Needs m3e_prepare(ctx, >= n_frames) beforehand.  The graph shares the context's
 * scratch: do not run it concurrently with other calls on the same context. */
typedef struct m3e_graph m3e_graph;
int m3e_graph_create(m3e_ctx* ctx, int form, const int32_t* d_hits, const int64_t* d_frame_off, int64_t n_frames,
                     uint8_t* d_keep, uint8_t* d_reason, m3e_graph** out);
int m3e_graph_launch(m3e_graph* graph, cudaStream_t stream);
int m3e_graph_destroy(m3e_graph* graph);

/* Launch parameters chosen by m3e_autotune and in force in the context. */
typedef struct {
  int32_t frames_per_grab;   /* work-queue granularity of the frame-parallel kernels */
  int32_t defer_hits;        /* frames with more hits go from the warp tier to the CTA tiers */
  int32_t s1_ctas_per_sm;    /* resident CTAs per SM of the stage-1 warp tier */
  int32_t configs_tried;
  float ms_default, ms_best; /* calibration batch time at the defaults and at the choice */
  int32_t mid_cta_threads;   /* threads of a CTA of the stage-1 middle tier (frames of 161..1024 hits) */
  int32_t s2_ctas_per_sm;    /* resident CTAs per SM of the track stage */
  float ms_worst;            /* calibration batch time at the slowest configuration tried */
} m3e_tuning;

/* Time the staged form on a calibration batch (device buffers as for
 * m3e_select_frames) over launch parameters and keep the fastest in the
 * context: a grid of frames_per_grab (1..16) x defer_hits (96, 128, 160) x
 * stage-1 CTAs per SM (all, half), then, one axis at a time from that point, the
 * middle tier's CTA size (128, 256, 512 threads) and the track stage's CTAs per
 * SM.  Synchronises the context's device; decisions do not depend on the
 * parameters.  Each configuration is timed as the median of five runs after a
 * warm-up; one replaces the current choice only when it is more than 2% faster,
 * so a calibration batch of a few ms keeps the defaults unless a change clearly
 * pays. */
int m3e_autotune(m3e_ctx* ctx, const int32_t* d_hits, const int64_t* d_frame_off, int64_t n_frames, uint8_t* d_keep,
                 uint8_t* d_reason, m3e_tuning* out);

/* Number of kernel launches the last select call enqueued. */
int m3e_last_launch_count(const m3e_ctx* ctx);

/* Kernel timing.  With on = 1, each m3e_select_frames / _fused / _plain call
 * records CUDA events on the caller's stream around its kernels.
 * m3e_kernel_times waits for the events of the last call and returns the
 * duration in ms of the main kernels (the five staged kernels, the fused kernel
 * or the plain kernel) and of the deferred-frame kernel (0 for the plain form).
 * m3e_stage_times returns up to 8 durations of the last staged call: stage 1
 * (warp tier), stage 1 (middle and top CTA tiers), stages 2-5 and the
 * deferred-frame kernel.
 * Timing adds no device sync. */
int m3e_set_profiling(m3e_ctx* ctx, int on);
int m3e_kernel_times(m3e_ctx* ctx, float* main_ms, float* deferred_ms);
int m3e_stage_times(m3e_ctx* ctx, float* ms, int n);

/* Hit ingest (Sec. "Memory Layout": hits as points (x, y, z), loaded per frame
 * for the selection; Sec. "Selection Cuts": the azimuth phi the cuts bin on):
 * decodes n_hits packed int32 pixel addresses into FP32 coordinates, as
 * structure of arrays, through the context's look-up tables (built in FP64,
 * rounded once), so every value equals the FP64 pixel centre rounded once to FP32:
 *   x = r_L cos(phi), y = r_L sin(phi), z = -H_L + (row + 1/2) pitch   [mm],
 *   phi = (ladder * n_cols_L + col + 1/2) 2 pi / (n_ladders_L n_cols_L) [rad].
 * d_hits [n_hits] and d_x, d_y, d_z, d_phi [n_hits] are caller-owned DEVICE
 * arrays; d_phi may be NULL (not written).  Hits keep their order (hit i of the
 * input is element i of each output); a frame's hits are a contiguous range, so
 * the frame offsets of the selection apply unchanged.  An invalid address gives
 * NaN in every output of that hit and latches M3E_EBADHIT (m3e_check).  One
 * kernel launch on `stream`; 16-byte-aligned arrays take the vectorised path.
 * The selection entry points do not need this call (they decode as they load a
 * frame); it serves callers that want the decoded hits themselves. */
int m3e_ingest(m3e_ctx* ctx, const int32_t* d_hits, int64_t n_hits, float* d_x, float* d_y, float* d_z,
               float* d_phi, cudaStream_t stream);

/* Selection without any device allocation in the call (the paper has no
 * counterpart; this is a deployment aid).  Same decisions as m3e_select_frames,
 * through the fused kernels, with their scratch in a fixed static device array
 * instead of context memory that grows with the batch.  For callers that must
 * not allocate once running: a filter loop at a fixed frame rate cannot take the
 * device synchronisation of cudaMalloc/cudaFree, and a process sharing the GPU
 * under a fixed memory budget reserves all memory at start-up.  The context must
 * exist already (m3e_create allocates; create it during initialisation).
 *   - At most 262,144 frames per call; more returns M3E_EINVAL.
 *   - The first call on a device looks up the array's device address (set-up);
 *     make that first call before any stream capture.  The address is cached per
 *     device; m3e_create clears the cache, so after a cudaDeviceReset create a
 *     new context before calling again.
 *   - Frames above the context's warp-tier size (set by m3e_autotune)
 *     go to the CTA-per-frame kernel, as in m3e_select_frames_fused.
 *   - The array is shared by all calls on a device and keeps the last call's
 *     contents; the call clears what must start at zero.  Calls that overlap on
 *     the GPU (other streams, other contexts of the same device, other threads)
 *     race on it: serialise them.
 *   - No statistics or candidate record. */
int m3e_select_frames_noalloc(m3e_ctx* ctx, const int32_t* d_hits, const int64_t* d_frame_off, int64_t n_frames,
                              uint8_t* d_keep, uint8_t* d_reason, cudaStream_t stream);

/* ------------------------------------------------------------------ fit gradient
 *
 * Gradient of the summed track chi2 of frozen candidates with respect to the
 * rigid alignment of the four layers and the field scale (an extension for
 * detector alignment; the paper's track fit, Sec. "Track Reconstruction", is the
 * forward model, the paper itself fits no alignment).
 *   - d_cand: n_cand rows of 4 int32, the global indices into d_hits of a
 *     layer-0, -1, -2 and -3 hit (16-byte aligned), e.g. the quadruplets of
 *     tracks the selection kept.  The selection is discrete: the rows stay
 *     fixed while the parameters move.
 *   - d_params: 25 floats.  Layer L: params[6L .. 6L+5] = dx, dy, dz [mm],
 *     wx, wy, wz [rad]; the hit measured at nominal position x on layer L is
 *     placed at R(w) x + d, R = Rz(wz) Ry(wy) Rx(wx) (rotations about the global
 *     axes through the origin).  params[24] scales the field (1 = nominal).
 *   - chi2 of a candidate: the track chi2 of the selection (two triplet fits,
 *     global chi2 at the inverse-variance mean curvature) at the moved hits;
 *     candidates whose fit fails, or whose hits are invalid, out of range
 *     (index >= d_frame_off[n_frames]) or on the wrong layer, are left out.
 *   - *d_chi2_sum (device float) = sum of chi2 over the valid candidates;
 *     d_grad (device float[25], or NULL for the sum alone) = its gradient.
 * The gradient is reverse mode, recomputing each candidate's fit (nothing per
 * candidate is stored).  A common translation of all layers and a common
 * rotation about z leave every chi2 unchanged (the gradient has no component
 * along them), and chi2 is quadratic in the field scale.  Sums are accumulated in
 * FP64 per block and added in a fixed order: repeated calls give equal results.
 * Asynchronous on `stream`. */
int m3e_fit_grad(m3e_ctx* ctx, const int32_t* d_hits, const int64_t* d_frame_off, int64_t n_frames,
                 const int32_t* d_cand, int64_t n_cand, const float* d_params, float* d_chi2_sum, float* d_grad,
                 cudaStream_t stream);

/* chi2 of each candidate (NaN for those left out) into d_chi2_each[n_cand]. */
int m3e_fit_chi2(m3e_ctx* ctx, const int32_t* d_hits, const int64_t* d_frame_off, int64_t n_frames,
                 const int32_t* d_cand, int64_t n_cand, const float* d_params, float* d_chi2_each,
                 cudaStream_t stream);

/* Weighted mean curvature kappa_bar (1/mm, signed: positive = clockwise turning)
 * of each frozen candidate's track fit at the given alignment (Sec. "Track
 * Reconstruction": the inverse-variance mean of the two triplet curvatures), in
 * d_kappa_each[n_cand] (device float; NaN where the chi2 of m3e_fit_chi2 would be
 * NaN).  The momentum is p = k B field_scale / |kappa_bar|; a caller fits the field
 * scale with it (for example from the energy sum of signal decays), since the
 * chi2 sum cannot (it grows as the square of the scale). */
int m3e_fit_kappa(m3e_ctx* ctx, const int32_t* d_hits, const int64_t* d_frame_off, int64_t n_frames,
                  const int32_t* d_cand, int64_t n_cand, const float* d_params, float* d_kappa_each,
                  cudaStream_t stream);
/* Number of valid candidates of the last m3e_fit_grad / m3e_fit_chi2 / m3e_fit_kappa call
 * (synchronises `stream`). */
int m3e_fit_valid_count(m3e_ctx* ctx, cudaStream_t stream, int64_t* out);

/* ------------------------------------------------------------------ streaming
 *
 * Frame-by-frame submission with continuous batching: the filter-farm setting
 * of the paper (Sec. "Implementation": frames arrive continuously from the
 * readout and are selected as they come).  Every 64 ns frame is handed over as
 * its own packet; a resident kernel selects frames while new ones are admitted,
 * so there is no batch boundary to wait for.
 *
 * How it works:
 *   - m3e_stream_submit copies the packet into a ring of pinned host memory and
 *     publishes a descriptor with a store-release.  It never calls CUDA.
 *   - A resident kernel (one warp per frame, the fused per-frame code) takes
 *     frames in submission order.  One warp of it moves new descriptors into a
 *     device ring; each worker warp waits, with bounded back-off, for the frame
 *     of the ticket it drew, reads the hits over the host link and writes a
 *     completion word into a pinned completion queue, in completion order.
 *   - A library thread delivers completions into the caller's result slots,
 *     frees ring space in submission order and relaunches the resident kernel
 *     when it has exited while frames are waiting.
 *   - Frames with more than 160 hits (beyond the warp stage) are gathered by the
 *     same thread and run by a CTA-per-frame kernel (same decisions).
 *
 * Every device wait is bounded: the resident kernel exits after idle_us
 * without work and after lifetime_ms in any case, and a worker that waits
 * longer than wait_limit_ms for a published frame gives up, latches an error
 * and exits.  Decisions are those of m3e_select_frames_fused for the same
 * frame, alone or among others. */

/* Result slot of one submitted frame: caller-owned host memory, written by the
 * library.  done turns from 0 to 1 (store-release) when the other fields are
 * valid; t_submit_ns is set by m3e_stream_submit, t_done_ns when the library
 * thread delivers the result (CLOCK_MONOTONIC nanoseconds). */
typedef struct {
  volatile uint32_t done;
  uint8_t keep, reason;      /* as in m3e_select_frames */
  uint16_t reserved;
  int32_t err;               /* M3E_OK, M3E_EBADHIT (invalid address), M3E_ETIMEOUT (stream failed) */
  uint64_t tag;              /* the caller's tag */
  uint64_t t_submit_ns, t_done_ns;
} m3e_result;

/* Stream parameters; zero fields take the defaults. */
typedef struct {
  uint32_t size;             /* sizeof(m3e_stream_params) */
  int32_t slots;             /* frames in flight, a power of two (default 65536) */
  int64_t ring_bytes;        /* host ring of packet bytes (default 64 MiB) */
  int32_t ctas_per_sm;       /* resident kernel: CTAs of 4 warps per SM (default 2) */
  int32_t idle_us;           /* resident kernel exits after this long without work (default 20000) */
  int32_t lifetime_ms;       /* ... and after this long in any case; relaunched while work remains (default 2000) */
  int32_t wait_limit_ms;     /* a worker's wait for a published frame (default lifetime_ms + 1000) */
  int32_t no_feeder;         /* test only: 1 = nothing publishes frames to the workers, so their waits expire */
} m3e_stream_params;

typedef struct {
  uint64_t submitted, completed, busy_refusals;
  uint64_t kernel_launches;  /* resident kernel launches so far */
  uint64_t heavy_frames;     /* frames run by the CTA-per-frame kernel */
  uint64_t delivery_passes;  /* passes of the library thread that delivered results */
  uint64_t tail_publications; /* stores of the descriptor tail seen by the GPU */
  int32_t kernel_running;    /* resident kernel currently on the GPU */
  int32_t failed;            /* a device wait expired: frames in flight were lost (M3E_ETIMEOUT) */
} m3e_stream_status;

/* Start the streaming machinery (pinned rings, device rings, library thread).
 * params may be NULL for the defaults.  M3E_ESTATE if already open. */
int m3e_stream_open(m3e_ctx* ctx, const m3e_stream_params* params);

/* Submit one frame: h_packet[0 .. n_hits) packed addresses (any host memory;
 * copied before return, so the buffer may be reused at once).  h_result_slot
 * must stay valid until its done flag is 1.  Opens the stream with the defaults
 * if it is not open.  Returns M3E_EBUSY without side effects when the slots or
 * the ring bytes are all in use (retry later), M3E_EINVAL for a packet larger
 * than the ring or a NULL slot, M3E_ETIMEOUT once the stream has failed.
 * Safe to call from several threads (internally locked). */
int m3e_stream_submit(m3e_ctx* ctx, const int32_t* h_packet, int32_t n_hits, uint64_t tag,
                      m3e_result* h_result_slot);

/* Submit a CSR batch of host frames at once: frame f is h_hits[h_frame_off[f]
 * .. h_frame_off[f+1]), its result slot h_results[f], its tag tags[f] (tags may
 * be NULL: tag = f).  Frames are admitted in order until one does not fit; one
 * lock, one clock reading (t_submit_ns) and one publication serve the whole
 * batch, so a host that receives frames in bursts pays the fixed cost once.
 * *n_admitted (may be NULL) receives the number admitted; returns M3E_OK when
 * all were, M3E_EBUSY when only the first *n_admitted were (resubmit the rest
 * later), M3E_EINVAL for bad sizes or NULL pointers (nothing admitted). */
int m3e_stream_submit_many(m3e_ctx* ctx, const int32_t* h_hits, const int64_t* h_frame_off, int64_t n_frames,
                           const uint64_t* tags, m3e_result* h_results, int64_t* n_admitted);

/* Counters of the stream (no wait). */
int m3e_stream_poll(m3e_ctx* ctx, m3e_stream_status* out);

/* Wait until every submitted frame has its result, at most timeout_ms;
 * M3E_ETIMEOUT if the time ran out or the stream failed. */
int m3e_stream_drain(m3e_ctx* ctx, int64_t timeout_ms);

/* Drain (bounded), stop the resident kernel and free the stream.  Results of
 * frames still in flight after the bounded drain are written with err =
 * M3E_ETIMEOUT.  Also done by m3e_destroy. */
int m3e_stream_close(m3e_ctx* ctx);

typedef struct {
  double offered_hz;         /* arrival rate asked for */
  double sustained_hz;       /* frames / (last result time - first arrival time) */
  double submit_hz;          /* frames / (last submit time - first arrival time) */
  uint64_t busy_retries;     /* submission calls not fully admitted (M3E_EBUSY), rest retried */
  uint64_t kernel_launches;
  int64_t duration_ns;
} m3e_replay_stats;

/* Latency harness: replay a CSR batch of host frames as an open-loop Poisson
 * arrival process of rate_hz (exponential gaps from a seeded counter-based
 * generator, splitmix64).  One submitting thread waits for the next arrival
 * time and submits every frame that has arrived by then in one call (as
 * m3e_stream_submit_many, at most 1024), retrying what the stream refused;
 * below the host's per-call rate that is one frame per call.  Per frame it returns
 * keep and reason, the latency from submission to result (out_lat_submit_ns)
 * and from the scheduled arrival to result (out_lat_arrival_ns, which includes
 * any wait for admission).  Any output pointer may be NULL.  Waits at most
 * 30 s beyond the last arrival for the results (M3E_ETIMEOUT). */
int m3e_stream_replay(m3e_ctx* ctx, const int32_t* h_hits, const int64_t* h_frame_off, int64_t n_frames,
                      double rate_hz, uint64_t seed, uint8_t* out_keep, uint8_t* out_reason,
                      int64_t* out_lat_submit_ns, int64_t* out_lat_arrival_ns, m3e_replay_stats* out);

const char* m3e_last_error_string(void);
int m3e_version(void);

#ifdef __cplusplus
}
#endif
#endif
