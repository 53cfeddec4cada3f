// Hit ingest of libm3e: packed int32 pixel addresses -> FP32 hit coordinates as
// structure of arrays (Sec. "Memory Layout": a hit is the point (x, y, z) of its
// pixel; the azimuth phi of the pixel column is the quantity the selection cuts
// bin on, Sec. "Selection Cuts").
//
// The work is a stream: 4 bytes read and 16 bytes written per hit, so HBM
// bandwidth bounds it once the table look-ups stay on chip.  Each CTA (one per SM)
// first copies the (x, y) of every pixel column and the z of every pixel row into
// shared memory (183 KB); phi is computed, not looked up: (g + 1/2) times 2 pi/ntot
// held as a sum of two floats, in exact FP32 steps (the product's rounding error
// recovered by a fused multiply-add), which reproduces the FP64 value rounded once
// for every column of the detector (checked exhaustively).  Each thread then moves
// four consecutive hits per step (one 16-byte load of addresses, one 16-byte
// store into each output array) with INGEST_UNROLL steps in flight; the streams
// are read and written with evict-first hints.
#include "m3e_device.cuh"

namespace m3e {
namespace {

constexpr int INGEST_THREADS = 1024;
constexpr int INGEST_UNROLL = 4;

struct Coord {
  float x, y, z, phi;
};

template <bool PHI>
__device__ __forceinline__ Coord ingest_one(const DevCfg& C, const float2* __restrict__ xy, const float* __restrict__ zr,
                                            uint32_t a, bool& bad) {
  const Dec d = decode_packed(C, a);
  Coord c;
  if (d.ok) {
    const float2 q = xy[d.ci];
    c.x = q.x;
    c.y = q.y;
    c.z = zr[d.ri];
    c.phi = PHI ? column_phi<true>(C, d.L, d.g) : 0.f;
  } else {
    bad = true;
    c.x = c.y = c.z = c.phi = __int_as_float(0x7fc00000);  // quiet NaN
  }
  return c;
}

// VEC: every pointer is 16-byte aligned; threads move int4/float4 units of four
// hits, the last n % 4 hits are taken by the scalar loop of the first threads.
template <bool VEC, bool PHI>
__global__ void __launch_bounds__(INGEST_THREADS, 1)
    k_ingest(const __grid_constant__ DevCfg C, const int32_t* __restrict__ hits, int64_t n,
             const float4* __restrict__ col_lut, const float* __restrict__ row_lut, float* __restrict__ x,
             float* __restrict__ y, float* __restrict__ z, float* __restrict__ phi, int* err) {
  extern __shared__ __align__(16) float2 s_xy[];
  const int ncol = C.col_off[3] + C.ntot[3], nrow = C.row_off[3] + C.nrow[3];
  float* s_z = reinterpret_cast<float*>(s_xy + ncol);
  for (int i = threadIdx.x; i < ncol; i += INGEST_THREADS) {
    const float4 q = __ldg(col_lut + i);
    s_xy[i] = make_float2(q.x, q.y);
  }
  for (int i = threadIdx.x; i < nrow; i += INGEST_THREADS) s_z[i] = __ldg(row_lut + i);
  __syncthreads();
  bool bad = false;
  const int64_t tid = (int64_t)blockIdx.x * INGEST_THREADS + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * INGEST_THREADS;
  int64_t done = 0;
  if constexpr (VEC) {
    const int64_t nv = n >> 2;
    const int4* hv = reinterpret_cast<const int4*>(hits);
    float4* xv = reinterpret_cast<float4*>(x);
    float4* yv = reinterpret_cast<float4*>(y);
    float4* zv = reinterpret_cast<float4*>(z);
    float4* pv = reinterpret_cast<float4*>(phi);
    for (int64_t v0 = tid; v0 < nv; v0 += nth * INGEST_UNROLL) {
      int4 a[INGEST_UNROLL];
#pragma unroll
      for (int u = 0; u < INGEST_UNROLL; ++u) {
        const int64_t v = v0 + u * nth;
        a[u] = v < nv ? __ldcs(hv + v) : make_int4(0, 0, 0, 0);
      }
#pragma unroll
      for (int u = 0; u < INGEST_UNROLL; ++u) {
        const int64_t v = v0 + u * nth;
        if (v < nv) {
          const Coord c0 = ingest_one<PHI>(C, s_xy, s_z, (uint32_t)a[u].x, bad);
          const Coord c1 = ingest_one<PHI>(C, s_xy, s_z, (uint32_t)a[u].y, bad);
          const Coord c2 = ingest_one<PHI>(C, s_xy, s_z, (uint32_t)a[u].z, bad);
          const Coord c3 = ingest_one<PHI>(C, s_xy, s_z, (uint32_t)a[u].w, bad);
          __stcs(xv + v, make_float4(c0.x, c1.x, c2.x, c3.x));
          __stcs(yv + v, make_float4(c0.y, c1.y, c2.y, c3.y));
          __stcs(zv + v, make_float4(c0.z, c1.z, c2.z, c3.z));
          if constexpr (PHI) __stcs(pv + v, make_float4(c0.phi, c1.phi, c2.phi, c3.phi));
        }
      }
    }
    done = nv << 2;
  }
  for (int64_t i = done + tid; i < n; i += nth) {
    const Coord c = ingest_one<PHI>(C, s_xy, s_z, (uint32_t)__ldcs(hits + i), bad);
    __stcs(x + i, c.x);
    __stcs(y + i, c.y);
    __stcs(z + i, c.z);
    if constexpr (PHI) __stcs(phi + i, c.phi);
  }
  if (__any_sync(FULL, bad) && (threadIdx.x & 31) == 0) atomicOr(err, ERR_BADHIT);
}

size_t ingest_smem_bytes(const DevCfg& c) {
  return (size_t)(c.col_off[3] + c.ntot[3]) * sizeof(float2) + (size_t)(c.row_off[3] + c.nrow[3]) * sizeof(float);
}

template <bool VEC, bool PHI>
cudaError_t launch_ingest_t(const DevCfg& c, const int32_t* hits, int64_t n, const float4* col_lut,
                            const float* row_lut, float* x, float* y, float* z, float* phi, int* err, int grid,
                            cudaStream_t s) {
  const size_t sm = ingest_smem_bytes(c);
  cudaError_t e = cudaFuncSetAttribute(k_ingest<VEC, PHI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_ingest<VEC, PHI><<<grid, INGEST_THREADS, sm, s>>>(c, hits, n, col_lut, row_lut, x, y, z, phi, err);
  return cudaGetLastError();
}

}  // namespace

int ingest_blocks_per_sm() { return 1; }  // one CTA per SM: the tables take most of its shared memory

cudaError_t launch_ingest(const DevCfg& c, const int32_t* hits, int64_t n, const float4* col_lut, const float* row_lut,
                          float* x, float* y, float* z, float* phi, int* err, int grid, cudaStream_t s) {
  auto al = [](const void* p) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  const bool vec = al(hits) && al(x) && al(y) && al(z) && al(phi);
  if (vec)
    return phi ? launch_ingest_t<true, true>(c, hits, n, col_lut, row_lut, x, y, z, phi, err, grid, s)
               : launch_ingest_t<true, false>(c, hits, n, col_lut, row_lut, x, y, z, phi, err, grid, s);
  return phi ? launch_ingest_t<false, true>(c, hits, n, col_lut, row_lut, x, y, z, phi, err, grid, s)
             : launch_ingest_t<false, false>(c, hits, n, col_lut, row_lut, x, y, z, phi, err, grid, s);
}

}  // namespace m3e
