// Fused selection kernels of libm3e: the whole per-frame method of the paper
// (Algorithm 1: load, selection cuts, track reconstruction, vertex fit, store)
// run by one group of threads per frame:
//   k_select_warp  persistent, one warp per frame, frames from a device work
//                  queue (lowest latency per frame; frames too large for a warp's
//                  shared-memory stage go to the deferred list);
//   k_select_cta   one CTA per frame: the deferred frames, and the plain
//                  per-frame form over a whole batch.
#include "m3e_device.cuh"

namespace m3e {
namespace {

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
      int r = frame_front<WarpGroup, SmWarp, W_HITS, W_TRIP, true, DEBUG>(g, sm, C, P, f);
      if (r == PENDING) r = frame_back<WarpGroup, SmWarp, W_TRIP, W_TRK, W_COMBO, true, DEBUG>(g, sm, C, P, f);
      if (r == DEFERRED) {
        if (g.leader()) {
          const int k = atomicAdd(P.defer_count, 1);
          P.defer_list[k] = f;
          if (P.stats) sm.acc[ST_DEFER] += 1;
        }
      } else {
        finish_frame(g, sm, P, f, r);
      }
      g.sync();
    }
  }
  flush_stats(g, sm, P.stats);
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
  const int count = LIST ? *P.in_count : (int)P.n_frames;
  for (int i = blockIdx.x; i < count; i += gridDim.x) {
    const int f = LIST ? P.in_list[i] : i;
    int r = frame_front<CtaGroup<NT>, SmCta, C_HITS, C_TRIP, false, DEBUG>(g, sm, C, P, f);
    if (r == PENDING) r = frame_back<CtaGroup<NT>, SmCta, C_TRIP, C_TRK, C_COMBO, false, DEBUG>(g, sm, C, P, f);
    finish_frame(g, sm, P, f, r);
    g.sync();
  }
  flush_stats(g, sm, P.stats);
}

template <class K>
cudaError_t set_smem(K k, size_t bytes) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

size_t fused_smem_bytes() { return sizeof(SmWarp) * WARPS_PER_CTA; }
size_t cta_smem_bytes() { return sizeof(SmCta); }

int fused_blocks_per_sm() {
  int nb = 0;
  set_smem(k_select_warp<false>, fused_smem_bytes());
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_select_warp<false>, WARPS_PER_CTA * 32,
                                                    fused_smem_bytes()) != cudaSuccess)
    return 1;
  return nb > 0 ? nb : 1;
}

cudaError_t launch_fused(const DevCfg& c, const KParams& p, int grid, bool debug, cudaStream_t s) {
  const size_t sm = fused_smem_bytes();
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
