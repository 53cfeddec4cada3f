// Staged selection kernels of libm3e: the same method as the fused kernels,
// with the work of a batch regrouped by candidate instead of by frame.
//   stage 1  warp per frame: decode, phi-bin sort, selection cuts (Algorithm 2);
//            the sorted hits and the selected triplets go to global memory
//   stage 2  thread per triplet of the whole batch: track reconstruction (Algorithm 3)
//   stage 3  warp per frame: track cap, energy test (Algorithm 4, part 1);
//            combinations go to global memory
//   stage 4  thread per combination of the whole batch: vertex (Algorithm 4, part 2)
//   stage 5  thread per frame: decision (store_frame of Algorithm 1)
// Every kernel is small and runs one kind of work, so warps share their
// instructions and lanes; a frame's candidates stay contiguous, so its hits and
// tracks are read from L2 by neighbouring threads.  Frames that exceed a stage's
// capacity are deferred to the CTA-per-frame kernel with identical decisions.
#include "m3e_device.cuh"

namespace m3e {
namespace {

constexpr int NL3 = NB + 1;                        // layer-3 bin starts per frame
constexpr int S1_TRIP = 160;                       // stage-1 warp-tier triplet capacity
// the address of each hit at hand for the emit (its phi is computed there); input
// indices only for the candidate record
using SmFront = FrameSm<W_HITS, S1_TRIP, 1, 1, false, false, true>;
using SmFrontD = FrameSm<W_HITS, S1_TRIP, 1, 1, false, true, true>;
constexpr int M_HITS = 1024;                       // stage-1 middle tier (CTA per frame)
using SmFrontMid = FrameSm<M_HITS, C_TRIP, 1, 1>;
using SmFrontCta = FrameSm<C_HITS, C_TRIP, 1, 1>;
constexpr int S3_WARPS = 4;
constexpr int S3_BUF = 128;  // combinations a frame of stage 3 collects before writing

struct S3Sm {                                      // stage 3, per warp
  int pidx[C_TRK], nidx[C_TRK];                    // triplet index of each e+ / e- track
  float pE[C_TRK], nE[C_TRK];
  float pPz[C_TRK], nPz[C_TRK];                    // p cos(theta) of each track
  uint32_t wbuf[S3_BUF];                           // combinations to write: a | b << 8 | c << 16
  int npos, nneg;
  unsigned long long acc[ST_REASON0 + 8];
};

__device__ __forceinline__ int warp_count_add(int* ctr, bool pred) {  // ordered warp compaction
  const unsigned m = __ballot_sync(FULL, pred);
  int base = 0;
  if ((threadIdx.x & 31) == 0 && m) base = atomicAdd(ctr, __popc(m));
  base = __shfl_sync(FULL, base, 0);
  return base + __popc(m & ((1u << (threadIdx.x & 31)) - 1u));
}

// ---- stage 1: write-out of a frame whose cuts selected triplets
// The sorted hits of frame f take the places of its input hits (off[f] - off_base
// onwards, so no allocator is needed); its triplets go to a range taken from the
// triplet allocator, whose atomic is issued first and waited for only after the
// hits are written.  A frame that does not fit is deferred (returns false).
template <class G, class Sm, bool DEBUG, bool LIVE = false>
__device__ __forceinline__ bool emit_frame(const G& g, Sm& sm, const DevCfg& C, const KParams& P, const SParams& S,
                                           int f, int n, int ntrip, long long* bcast) {
  long long tb = 0;
  if (g.leader()) tb = (long long)atomicAdd(&S.counters[0], (unsigned long long)ntrip);
  const long long hb = P.off[f] - P.off_base;
  const bool hits_fit = hb + n <= S.hits_cap;
  // phi and the address of a sorted hit serve only the layer-3 search of stage 2
  const int l3s = sm.bstart[3 * NB];
  const int32_t* hin = P.hits + hb;
  for (int i = g.rank(); hits_fit && i < n; i += G::N) {
    float phi = 0.f;
    if (i >= l3s) {
      uint32_t a;
      if constexpr (Sm::kAddr) a = sm.addr[i];
      else a = (uint32_t)(LIVE ? __ldcv(hin + sm.inidx[i]) : __ldg(hin + sm.inidx[i]));
      if constexpr (Sm::kPhi) {
        phi = sm.phi[i];
      } else {
        const Dec d = decode(C, a);
        phi = column_phi(C, d.L, d.g);
      }
      S.haddr[hb + i] = a;
    }
    S.hp[hb + i] = make_float4(sm.x[i], sm.y[i], sm.z[i], phi);
    if constexpr (DEBUG) {
      static_assert(Sm::kIdx, "the candidate record needs the input indices");
      S.hidx[hb + i] = sm.inidx[i];
    }
  }
  if constexpr (G::N == 32) {
    tb = __shfl_sync(FULL, tb, 0);
  } else {
    if (g.leader()) bcast[1] = tb;
    g.sync();
    tb = bcast[1];
    g.sync();
  }
  if (!hits_fit || tb + ntrip > S.trip_cap) {
    // out of space: mark the triplet slots this frame owns below the cap as unused
    for (int64_t t = tb + g.rank(); t < S.trip_cap && t < tb + ntrip; t += G::N) S.trip[t] = make_int4(-1, 0, 0, 0);
    return false;
  }
  for (int b = g.rank(); b < NL3; b += G::N) S.l3[(int64_t)f * NL3 + b] = sm.bstart[3 * NB + b];
  for (int t = g.rank(); t < ntrip; t += G::N) {
    const auto q = sm.u.trip[t];
    S.trip[tb + t] = make_int4(f, (int)hb, (int)q.x | ((int)q.y << 16), (int)q.z);
  }
  if (g.leader()) {
    S.fstate[f] = PENDING;
    S.ftbase[f] = (int)tb;
    S.fntrip[f] = ntrip;
    S.ffound[f] = 0;
  }
  return true;
}

// After frame_front: decide, emit, or defer one frame (stage-1 tiers).
template <class G, class Sm, bool DEBUG, bool LIVE = false, bool NOST = false>
__device__ __forceinline__ void stage1_finish(const G& g, Sm& sm, const DevCfg& C, const KParams& P, const SParams& S,
                                              int f, int r, long long* bcast) {
  const int ntrip = sm.ntrip;
  if (r == PENDING && ntrip == 0) r = M3E_DROP;  // no triplet: no track, no vertex
  if (r == PENDING) {
    const int n = (int)(P.off[f + 1] - P.off[f]);
    if (emit_frame<G, Sm, DEBUG, LIVE>(g, sm, C, P, S, f, n, ntrip, bcast)) {
      if (!NOST && g.leader() && P.stats)
        for (int k = 0; k < ST_REASON0; ++k) sm.acc[k] += sm.facc[k];
    } else {
      r = DEFERRED;
    }
  }
  if (r == DEFERRED) {
    if (g.leader()) {
      S.fstate[f] = DEFERRED;
      const int k = atomicAdd(P.defer_count, 1);
      P.defer_list[k] = f;
      if (!NOST && P.stats) sm.acc[ST_DEFER] += 1;
    }
  } else if (r != PENDING) {
    if (g.leader()) S.fstate[f] = r;
    finish_frame<G, Sm, NOST>(g, sm, P, f, r);
  }
  g.sync();
}

__device__ __forceinline__ unsigned ld_acquire_sys_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Host entry point: wait until the copy engine has flagged chunk k as arrived.
// The wait is bounded by P.gate_ms; it also ends once another warp has given up.
// Returns false when it gave up (ERR_GATE latched).
__device__ bool gate_wait(const KParams& P, int k) {
  int ok = 1;
  if ((threadIdx.x & 31) == 0) {
    const unsigned long long t_end = global_ns() + (unsigned long long)P.gate_ms * 1000000ull;
    unsigned ns = 64;
    while (ld_acquire_sys_u32(P.gate + k) == 0u) {
      if ((*(volatile int*)P.err & ERR_GATE) || global_ns() > t_end) {
        atomicOr(P.err, ERR_GATE);
        ok = 0;
        break;
      }
      __nanosleep(ns);
      if (ns < 2048) ns *= 2;
    }
  }
  __syncwarp();
  return __shfl_sync(FULL, ok, 0) != 0;
}

// ---- stage 1, warp tier: one warp per frame, frames from the device queue.
// GATED (host entry point): the hits arrive while the kernel runs; a frame is
// taken only after its chunk's arrival flag, and the hits are read past L1.
// NOST: the instance for runs without statistics (no statistics code at all).
template <bool DEBUG, bool GATED = false, bool NOST = false>
__global__ void __launch_bounds__(WARPS_PER_CTA * 32)
    k_stage1(const __grid_constant__ DevCfg C, const __grid_constant__ KParams P, const __grid_constant__ SParams S) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using Sm = typename std::conditional<DEBUG, SmFrontD, SmFront>::type;
  Sm& sm = reinterpret_cast<Sm*>(smem_raw)[threadIdx.x >> 5];
  __shared__ long long bcast[WARPS_PER_CTA][2];
  const WarpGroup g;
  clear_stats(g, sm);
  const int nf = (int)P.n_frames;
  int arrived = -1;  // chunks up to this one are known to have arrived
  bool stop = false;
  while (!stop) {
    int f0 = 0;
    if (g.leader()) f0 = atomicAdd(&P.work[0], P.grab);
    f0 = __shfl_sync(FULL, f0, 0);
    if (f0 >= nf) break;
    const int f1 = min(f0 + P.grab, nf);
    for (int f = f0; f < f1; ++f) {
      if constexpr (GATED) {
        const int k = f / P.gate_frames;
        if (k > arrived) {
          if (!gate_wait(P, k)) {
            stop = true;
            break;
          }
          arrived = k;
        }
      }
      const int r = frame_front<WarpGroup, Sm, W_HITS, S1_TRIP, true, DEBUG, GATED, NOST, true>(g, sm, C, P, f, f + 1 < f1);
      stage1_finish<WarpGroup, Sm, DEBUG, GATED, NOST>(g, sm, C, P, S, f, r, bcast[threadIdx.x >> 5]);
    }
  }
  if (!NOST) flush_stats(g, sm, P.stats);
}

// ---- stage 1, CTA tiers: one CTA per frame deferred by the tier below (large
// frames); the middle tier stages up to M_HITS hits, the top tier C_HITS.
// NT: threads of a CTA (the middle tier's is a tuning parameter).
template <class Sm, int CH, bool DEBUG, int NT = CTA_THREADS, bool NOST = false>
__global__ void __launch_bounds__(NT)
    k_stage1c(const __grid_constant__ DevCfg C, const __grid_constant__ KParams P, const __grid_constant__ SParams S) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Sm& sm = *reinterpret_cast<Sm*>(smem_raw);
  __shared__ long long bcast[2];
  const CtaGroup<NT> g;
  clear_stats(g, sm);
  const int count = *P.in_count;
  for (int i = blockIdx.x; i < count; i += gridDim.x) {
    const int f = P.in_list[i];
    int r;
    if (CH < C_HITS && P.off[f + 1] - P.off[f] > CH) r = DEFERRED;  // for the next tier
    else r = frame_front<CtaGroup<NT>, Sm, CH, C_TRIP, false, DEBUG, false, NOST>(g, sm, C, P, f);
    stage1_finish<CtaGroup<NT>, Sm, DEBUG, false, NOST>(g, sm, C, P, S, f, r, bcast);
  }
  if (!NOST) flush_stats(g, sm, P.stats);
}

// ---- stage 2: one thread per selected triplet
template <bool DEBUG>
__global__ void __launch_bounds__(128, 8)  // 8 CTAs per SM (64 registers: the first fit parked in shared memory)
    k_stage2(const __grid_constant__ DevCfg C, const __grid_constant__ KParams P, const __grid_constant__ SParams S) {
  static_assert(sizeof(FitPark) == 11 * 128 * sizeof(float), "one slot per thread of a 128-thread CTA");
  __shared__ FitPark park;
  const int64_t n = min((int64_t)S.counters[0], S.trip_cap);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int4 rn = i < n ? S.trip[i] : make_int4(-1, 0, 0, 0);
  for (; i < n; i += stride) {
    // the record carries the frame, its first sorted hit and the three frame-relative
    // indices; the next record is loaded while this triplet is fitted
    const int4 r = rn;
    if (i + stride < n) rn = S.trip[i + stride];
    const int f = r.x;
    if (f < 0) continue;
    const int64_t base = (int64_t)(unsigned)r.y;
    const int i0 = r.z & 0xffff, i1 = (int)((unsigned)r.z >> 16), i2 = r.w;
    const GHits v{S.hp + base, S.haddr + base, S.l3 + (int64_t)f * NL3, &park};
    const TrackOut o = build_track(v, C, i0, i1, i2);
    float2 te = make_float2(0.f, 0.f);
    if (o.status == 5) {
      float tk[14];
      track_record(v.pos(i0), v.pos(i1), o, C, tk);
      te = make_float2(tk[13] * tk[7], pz_track(tk[6], tk[4]));  // what the energy test reads
      float4* q = S.trec + 4 * i;
      q[0] = make_float4(tk[0], tk[1], tk[2], tk[3]);
      q[1] = make_float4(tk[4], tk[5], tk[6], tk[7]);
      q[2] = make_float4(tk[8], tk[9], tk[10], tk[11]);
      q[3] = make_float4(tk[12], tk[13], 0.f, 0.f);
    }
    S.tek[i] = te;
    if (DEBUG) {
      const int t = (int)(i - S.ftbase[f]);
      if (t < P.dump.cap_trip) {
        const int64_t d = (int64_t)f * P.dump.cap_trip + t;
        P.dump.trip[4 * d + 0] = S.hidx[base + i0];
        P.dump.trip[4 * d + 1] = S.hidx[base + i1];
        P.dump.trip[4 * d + 2] = S.hidx[base + i2];
        P.dump.trip[4 * d + 3] = o.i3 >= 0 ? (int)S.hidx[base + o.i3] : -1;
        P.dump.trk_status[d] = o.status;
        P.dump.trk_val[4 * d + 0] = o.kbar;
        P.dump.trk_val[4 * d + 1] = o.th01;
        P.dump.trk_val[4 * d + 2] = o.chi2;
        P.dump.trk_val[4 * d + 3] = o.mbest;
      }
    }
  }
}

// ---- stage 3: warp per frame, track cap and energy test (NOST: the instance for
// runs without statistics)
template <bool DEBUG, bool NOST = false>
__global__ void __launch_bounds__(S3_WARPS * 32)
    k_stage3(const __grid_constant__ DevCfg C, const __grid_constant__ KParams P, const __grid_constant__ SParams S) {
  __shared__ S3Sm smem[S3_WARPS];
  S3Sm& sm = smem[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  for (int k = lane; k < ST_REASON0 + 8; k += 32) sm.acc[k] = 0;
  __syncwarp();
  const int nf = (int)P.n_frames;
  const bool stats = !NOST && P.stats != nullptr;
  for (;;) {
    int f0 = 0;
    if (lane == 0) f0 = (int)atomicAdd(&S.counters[2], (unsigned long long)P.grab);
    f0 = __shfl_sync(FULL, f0, 0);
    if (f0 >= nf) break;
    const int f1 = min(f0 + P.grab, nf);
    for (int f = f0; f < f1; ++f) {
      if (S.fstate[f] != PENDING) continue;
      const int tb = S.ftbase[f], nt = S.fntrip[f];
      if (lane == 0) {
        sm.npos = 0;
        sm.nneg = 0;
      }
      __syncwarp();
      // kept tracks of the frame's triplets, split by charge
      for (int t0 = 0; t0 < nt; t0 += 32) {
        const int t = t0 + lane;
        // (eps E, P_z) of a kept track (E > 0), (0, 0) for a triplet that made none
        const float2 te = t < nt ? __ldg(S.tek + tb + t) : make_float2(0.f, 0.f);
        const float E = fabsf(te.x), pz = te.y;
        const bool pos = te.x > 0.f, neg = te.x < 0.f;
        const int kp = warp_count_add(&sm.npos, pos);
        const int kn = warp_count_add(&sm.nneg, neg);
        if (pos && kp < C_TRK) {
          sm.pidx[kp] = tb + t;
          sm.pE[kp] = E;
          sm.pPz[kp] = pz;
        }
        if (neg && kn < C_TRK) {
          sm.nidx[kn] = tb + t;
          sm.nE[kn] = E;
          sm.nPz[kn] = pz;
        }
        __syncwarp();
      }
      __syncwarp();
      const int npos = sm.npos, nneg = sm.nneg;
      int r = PENDING;
      if (npos + nneg > C.max_trk) r = M3E_TRACK_OVERFLOW;
      const int npair = npos * (npos - 1) / 2;
      // all energy-test survivors count towards the cap; a decision-only run
      // writes only those whose P_z leaves the momentum cut open (pz_fails_ptot)
      const bool prune = !DEBUG && !stats;
      int ncombo = 0, nwrite = 0, nopen = 0;
      if (r == PENDING) {
        if (stats && lane == 0) {
          sm.acc[ST_TRK] += npos + nneg;
          sm.acc[ST_ETEST] += (unsigned long long)npair * nneg;
        }
        // one pass over the (e+ pair, e-) combinations: count those passing the energy
        // test and collect those to write, in (pair, e-) order, in the warp's buffer
        for (int p0 = 0; p0 < npair; p0 += 32) {
          const int pr = p0 + lane;
          const bool act = pr < npair;
          int a = 0, b = 0;
          float eab = 0.f, pzab = 0.f;
          if (act) {
            b = (int)((1.f + sqrtf(1.f + 8.f * (float)pr)) * 0.5f);
            while (b * (b - 1) / 2 > pr) --b;
            while ((b + 1) * b / 2 <= pr) ++b;
            a = pr - b * (b - 1) / 2;
            eab = sm.pE[a] + sm.pE[b];
            pzab = __fadd_rn(sm.pPz[a], sm.pPz[b]);
          }
          int cnt = 0, co = 0;
          for (int c = 0; c < nneg; ++c) {
            const bool e_ok = act && fabsf((eab + sm.nE[c]) - C.m_mu) <= C.e_win;
            cnt += e_ok;
            // few combinations pass the energy window: the P_z test and the write
            // run only for an e- where one of the warp's pairs passes
            if (__any_sync(FULL, e_ok)) {
              const bool open = e_ok && !pz_fails_ptot(__fadd_rn(pzab, sm.nPz[c]), C.ptot_max);
              co += open;
              const bool wr = prune ? open : e_ok;
              const unsigned m = __ballot_sync(FULL, wr);
              const int k = nwrite + __popc(m & ((1u << lane) - 1u));
              if (wr && k < S3_BUF) sm.wbuf[k] = (uint32_t)a | ((uint32_t)b << 8) | ((uint32_t)c << 16);
              nwrite += __popc(m);
            }
          }
          ncombo += __reduce_add_sync(FULL, cnt);
          if (stats) nopen += __reduce_add_sync(FULL, co);
        }
        __syncwarp();
        if (DEBUG && lane == 0) P.dump.n_combo[f] = ncombo;
        if (ncombo > C.max_combo) r = M3E_COMBO_OVERFLOW;
        else if (nwrite == 0) r = M3E_DROP;  // no combination, or none that can pass
      }
      if (r == PENDING) {
        long long cb = 0;
        if (lane == 0) cb = (long long)atomicAdd(&S.counters[1], (unsigned long long)nwrite);
        cb = __shfl_sync(FULL, cb, 0);
        if (cb + nwrite > S.combo_cap) {
          for (int64_t t = cb + lane; t < S.combo_cap; t += 32) S.combo[t] = make_int4(-1, 0, 0, 0);
          r = DEFERRED;
        } else {
          if (nwrite <= S3_BUF) {
            for (int t = lane; t < nwrite; t += 32) {
              const uint32_t v = sm.wbuf[t];
              S.combo[cb + t] = make_int4(f, sm.pidx[v & 255], sm.pidx[(v >> 8) & 255], sm.nidx[v >> 16]);
            }
          } else {
            // more than the buffer holds: a second pass writes them, in the same order
            long long w = cb;
            for (int p0 = 0; p0 < npair; p0 += 32) {
              const int pr = p0 + lane;
              int a = 0, b = 0;
              float eab = 0.f, pzab = 0.f;
              const bool act = pr < npair;
              if (act) {
                b = (int)((1.f + sqrtf(1.f + 8.f * (float)pr)) * 0.5f);
                while (b * (b - 1) / 2 > pr) --b;
                while ((b + 1) * b / 2 <= pr) ++b;
                a = pr - b * (b - 1) / 2;
                eab = sm.pE[a] + sm.pE[b];
                pzab = __fadd_rn(sm.pPz[a], sm.pPz[b]);
              }
              for (int c = 0; c < nneg; ++c) {
                const bool pass = act && fabsf((eab + sm.nE[c]) - C.m_mu) <= C.e_win &&
                                  !(prune && pz_fails_ptot(__fadd_rn(pzab, sm.nPz[c]), C.ptot_max));
                const unsigned m = __ballot_sync(FULL, pass);
                if (pass) S.combo[w + __popc(m & ((1u << lane) - 1u))] = make_int4(f, sm.pidx[a], sm.pidx[b], sm.nidx[c]);
                w += __popc(m);
              }
            }
          }
          if (lane == 0) {
            S.fcbase[f] = cb;
            S.fncombo[f] = nwrite;
            if (stats) {
              sm.acc[ST_COMBO] += ncombo;
              sm.acc[ST_PZOPEN] += nopen;
            }
          }
        }
      }
      if (r == DEFERRED) {
        if (lane == 0) {
          S.fstate[f] = DEFERRED;
          const int k = atomicAdd(P.defer_count, 1);
          P.defer_list[k] = f;
          if (stats) sm.acc[ST_DEFER] += 1;
        }
      } else if (r != PENDING) {
        if (lane == 0) {
          S.fstate[f] = r;
          P.keep[f] = (uint8_t)(r != M3E_DROP);
          P.reason[f] = (uint8_t)r;
          if (stats) sm.acc[ST_REASON0 + r] += 1;
        }
      }
      __syncwarp();
    }
  }
  __syncwarp();
  if (stats)
    for (int k = lane; k < ST_REASON0 + 8; k += 32)
      if (sm.acc[k]) atomicAdd(P.stats + k, sm.acc[k]);
}

// ---- stage 4: vertex of every combination, compacted per warp
// Most combinations stop at the first two steps (a pair of track circles that
// does not intersect, or no intersection inside the target filter).  Each warp
// therefore runs those steps on 32 combinations at a time, appends the survivors
// to a queue in shared memory, and runs the full vertex on 32 queued survivors at
// a time, so that all lanes do the expensive part together.
constexpr int S4_WARPS = 4;

__device__ __forceinline__ void load_circle(const float4* __restrict__ rec, int64_t k, float& cx, float& cy,
                                            float& rt) {
  const float4 a = __ldg(rec + 4 * k);
  cx = a.x;
  cy = a.y;
  rt = a.z;
}

template <bool DEBUG>
__device__ __forceinline__ void stage4_dump(const DevCfg& C, const KParams& P, const SParams& S, int64_t i,
                                            const int4& r, const VtxOut& v, const TrackR& A, const TrackR& B,
                                            const TrackR& E) {
  const float esum = A.E + B.E + E.E;
  const int f = r.x;
  const int c = (int)(i - S.fcbase[f]);
  if (c < P.dump.cap_combo) {
    const int64_t d = (int64_t)f * P.dump.cap_combo + c;
    const int tb = S.ftbase[f];
    P.dump.combo[4 * d + 0] = r.y - tb;
    P.dump.combo[4 * d + 1] = r.z - tb;
    P.dump.combo[4 * d + 2] = r.w - tb;
    P.dump.combo[4 * d + 3] = v.status | (v.pass << 8);
    P.dump.combo_val[4 * d + 0] = esum - C.m_mu;
    P.dump.combo_val[4 * d + 1] = v.chi2;
    P.dump.combo_val[4 * d + 2] = v.tdist;
    P.dump.combo_val[4 * d + 3] = v.ptot;
    if (P.dump.combo_aux) {
      float dm, fm;
      vertex_soft(A, B, E, C.isect_lim, dm, fm);
      P.dump.combo_aux[4 * d + 0] = dm;
      P.dump.combo_aux[4 * d + 1] = fm;
      P.dump.combo_aux[4 * d + 2] = v.chi2_second;
      P.dump.combo_aux[4 * d + 3] = 0.f;
    }
  }
}

template <bool DEBUG, bool NOST = false>
__global__ void __launch_bounds__(S4_WARPS * 32, 8)  // 8 CTAs per SM (64 registers)
    k_stage4(const __grid_constant__ DevCfg C, const __grid_constant__ KParams P, const __grid_constant__ SParams S) {
  __shared__ long long queue[S4_WARPS][64];
  long long* q = queue[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const int64_t n = min((int64_t)S.counters[1], S.combo_cap);
  const int64_t stride = (int64_t)gridDim.x * S4_WARPS * 32;
  int qn = 0;
  unsigned nv = 0, nvo = 0;
  int64_t base = ((int64_t)blockIdx.x * S4_WARPS + (threadIdx.x >> 5)) * 32;
  // the combination records are loaded one step ahead; the three circles are read
  // together with the frame's state, before it is known whether they are needed
  int4 rn = base + lane < n ? S.combo[base + lane] : make_int4(-1, 0, 0, 0);
  for (;; base += stride) {
    const bool more = base < n;  // uniform in the warp
    if (more) {
      const int64_t i = base + lane;
      const int4 r = rn;
      if (i + stride < n) rn = S.combo[i + stride];
      bool cand = false;
      if (i < n && r.x >= 0) {
        const int f = r.x;
        float ca[3], cb[3], ce[3];
        load_circle(S.trec, r.y, ca[0], ca[1], ca[2]);
        load_circle(S.trec, r.z, cb[0], cb[1], cb[2]);
        load_circle(S.trec, r.w, ce[0], ce[1], ce[2]);
        if (S.fstate[f] == PENDING && (DEBUG || !*((volatile int*)S.ffound + f))) {
          const int st = vertex_prefilter(ca, cb, ce, C.isect_lim);
          cand = st == 2;
          if (DEBUG && !cand) {  // record the combination with its early status (the same geometry)
            const TrackR A = load_track(S.trec, r.y), B = load_track(S.trec, r.z), E = load_track(S.trec, r.w);
            stage4_dump<DEBUG>(C, P, S, i, r, vertex(A, B, E, C), A, B, E);
          }
        }
      }
      const unsigned m = __ballot_sync(FULL, cand);
      if (cand) q[qn + __popc(m & ((1u << lane) - 1u))] = i;
      qn += __popc(m);
    }
    __syncwarp();
    while (qn >= 32 || (!more && qn > 0)) {
      const int take = qn < 32 ? qn : 32;
      if (lane < take) {
        const int64_t i = q[qn - take + lane];
        const int4 r = S.combo[i];
        const TrackR A = load_track(S.trec, r.y), B = load_track(S.trec, r.z), E = load_track(S.trec, r.w);
        const VtxOut v = vertex(A, B, E, C);
        nv += v.status == 2;
        if (!NOST && P.stats && v.status == 2)
          nvo += !pz_fails_ptot(pz_sum(pz_track(A.p, A.ct), pz_track(B.p, B.ct), pz_track(E.p, E.ct)), C.ptot_max);
        if (v.pass) S.ffound[r.x] = 1;
        if (DEBUG) stage4_dump<DEBUG>(C, P, S, i, r, v, A, B, E);
      }
      qn -= take;
      __syncwarp();
    }
    if (!more) break;
  }
  if (!NOST && P.stats) {
    const unsigned s = __reduce_add_sync(FULL, nv), so = __reduce_add_sync(FULL, nvo);
    if (lane == 0 && s) atomicAdd(P.stats + ST_VTX, (unsigned long long)s);
    if (lane == 0 && so) atomicAdd(P.stats + ST_VTXOPEN, (unsigned long long)so);
  }
}

// ---- stage 5: decision of the frames still pending
__global__ void __launch_bounds__(256)
    k_stage5(const __grid_constant__ KParams P, const __grid_constant__ SParams S) {
  __shared__ unsigned cnt[2];
  if (threadIdx.x < 2) cnt[threadIdx.x] = 0;
  __syncthreads();
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f < P.n_frames && S.fstate[f] == PENDING) {
    const int r = S.ffound[f] ? M3E_VERTEX : M3E_DROP;
    P.keep[f] = (uint8_t)(r != M3E_DROP);
    P.reason[f] = (uint8_t)r;
    if (P.stats) atomicAdd(&cnt[r], 1u);
  }
  __syncthreads();
  if (P.stats && threadIdx.x < 2 && cnt[threadIdx.x])
    atomicAdd(P.stats + ST_REASON0 + threadIdx.x, (unsigned long long)cnt[threadIdx.x]);
}

template <class K>
cudaError_t set_smem(K k, size_t bytes) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

size_t stage1_smem_bytes(bool debug = false) { return (debug ? sizeof(SmFrontD) : sizeof(SmFront)) * WARPS_PER_CTA; }
size_t stage1c_smem_bytes() { return sizeof(SmFrontCta); }
size_t stage1m_smem_bytes() { return sizeof(SmFrontMid); }

int stage_blocks_per_sm(int stage) {
  int nb = 0;
  cudaError_t e = cudaSuccess;
  if (stage == 1) {
    set_smem(k_stage1<false, false, true>, stage1_smem_bytes());
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_stage1<false, false, true>, WARPS_PER_CTA * 32,
                                                      stage1_smem_bytes());
  } else if (stage == 2) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_stage2<false>, 128, 0);
  } else if (stage == 3) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_stage3<false, true>, S3_WARPS * 32, 0);
  } else if (stage == 4) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_stage4<false, true>, S4_WARPS * 32, 0);
  } else if (stage == 5) {
    set_smem(k_stage1c<SmFrontCta, C_HITS, false, CTA_THREADS, true>, stage1c_smem_bytes());
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_stage1c<SmFrontCta, C_HITS, false, CTA_THREADS, true>, CTA_THREADS,
                                                      stage1c_smem_bytes());
  } else {
    set_smem(k_stage1c<SmFrontMid, M_HITS, false, CTA_THREADS, true>, stage1m_smem_bytes());
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_stage1c<SmFrontMid, M_HITS, false, CTA_THREADS, true>, CTA_THREADS,
                                                      stage1m_smem_bytes());
  }
  return e == cudaSuccess && nb > 0 ? nb : 1;
}

template <int NT>
int mid_blocks_per_sm_t() {
  int nb = 0;
  set_smem(k_stage1c<SmFrontMid, M_HITS, false, NT, true>, stage1m_smem_bytes());
  const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &nb, k_stage1c<SmFrontMid, M_HITS, false, NT, true>, NT, stage1m_smem_bytes());
  return e == cudaSuccess && nb > 0 ? nb : 1;
}

int stage1_mid_blocks_per_sm(int threads) {
  return threads == 128 ? mid_blocks_per_sm_t<128>() : (threads == 512 ? mid_blocks_per_sm_t<512>() : mid_blocks_per_sm_t<256>());
}

// Stage 1 (warp tier; middle CTA tier over the warp tier's deferred frames; top
// CTA tier over the middle tier's), stages 2-5.  grids: stage 1 warp tier, 2, 3,
// 4, stage 1 top tier, stage 1 middle tier.  Frames deferred by the top tier or by
// stage 3 end up in S.list2 for the caller's CTA-per-frame kernel.  ev (9 events or
// null): before stage 1 and after each kernel.
// One launch of a CTA tier of stage 1 (the instance without statistics code when nost).
template <class Sm, int CH, bool DEBUG, int NT>
cudaError_t launch_tier(const DevCfg& c, const KParams& p, const SParams& s, int grid, size_t smem, cudaStream_t st,
                        bool nost) {
  if constexpr (!DEBUG) {
    if (nost) {
      const cudaError_t e = set_smem(k_stage1c<Sm, CH, false, NT, true>, smem);
      if (e == cudaSuccess) k_stage1c<Sm, CH, false, NT, true><<<grid, NT, smem, st>>>(c, p, s);
      return e;
    }
  }
  const cudaError_t e = set_smem(k_stage1c<Sm, CH, DEBUG, NT>, smem);
  if (e == cudaSuccess) k_stage1c<Sm, CH, DEBUG, NT><<<grid, NT, smem, st>>>(c, p, s);
  return e;
}

cudaError_t launch_staged(const DevCfg& c, const KParams& p, const SParams& s, const int grids[6], bool debug,
                          cudaStream_t st, cudaEvent_t* ev, cudaEvent_t after_s1, int mid_threads) {
  const size_t sm1 = stage1_smem_bytes(debug), smc = stage1c_smem_bytes(), smm = stage1m_smem_bytes();
  const bool gated = p.gate != nullptr && !debug;
  const bool nost = p.stats == nullptr;
  cudaError_t e = debug ? set_smem(k_stage1<true>, sm1)
                  : gated ? (nost ? set_smem(k_stage1<false, true, true>, sm1) : set_smem(k_stage1<false, true>, sm1))
                          : (nost ? set_smem(k_stage1<false, false, true>, sm1) : set_smem(k_stage1<false>, sm1));
  if (e != cudaSuccess) return e;
  KParams p1 = p, pm = p, pc = p, p3 = p;
  p1.defer_list = s.list1;
  p1.defer_count = s.lcount;
  pm.in_list = s.list1;
  pm.in_count = s.lcount;
  pm.defer_list = s.list1b;
  pm.defer_count = s.lcount + 2;
  pc.in_list = s.list1b;
  pc.in_count = s.lcount + 2;
  pc.defer_list = s.list2;
  pc.defer_count = s.lcount + 1;
  p3.defer_list = s.list2;
  p3.defer_count = s.lcount + 1;
  if (ev) cudaEventRecord(ev[0], st);
  if (debug) k_stage1<true><<<grids[0], WARPS_PER_CTA * 32, sm1, st>>>(c, p1, s);
  else if (gated && nost) k_stage1<false, true, true><<<grids[0], WARPS_PER_CTA * 32, sm1, st>>>(c, p1, s);
  else if (gated) k_stage1<false, true><<<grids[0], WARPS_PER_CTA * 32, sm1, st>>>(c, p1, s);
  else if (nost) k_stage1<false, false, true><<<grids[0], WARPS_PER_CTA * 32, sm1, st>>>(c, p1, s);
  else k_stage1<false><<<grids[0], WARPS_PER_CTA * 32, sm1, st>>>(c, p1, s);
  // the later kernels read the hits too: order them after every copy of the host entry
  if (after_s1) cudaStreamWaitEvent(st, after_s1, 0);
  if (ev) cudaEventRecord(ev[1], st);
  e = debug ? launch_tier<SmFrontMid, M_HITS, true, CTA_THREADS>(c, pm, s, grids[5], smm, st, false)
            : mid_threads == 128 ? launch_tier<SmFrontMid, M_HITS, false, 128>(c, pm, s, grids[5], smm, st, nost)
            : mid_threads == 512 ? launch_tier<SmFrontMid, M_HITS, false, 512>(c, pm, s, grids[5], smm, st, nost)
                                 : launch_tier<SmFrontMid, M_HITS, false, CTA_THREADS>(c, pm, s, grids[5], smm, st, nost);
  if (e != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev[2], st);
  e = debug ? launch_tier<SmFrontCta, C_HITS, true, CTA_THREADS>(c, pc, s, grids[4], smc, st, false)
            : launch_tier<SmFrontCta, C_HITS, false, CTA_THREADS>(c, pc, s, grids[4], smc, st, nost);
  if (e != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev[3], st);
  if (debug) k_stage2<true><<<grids[1], 128, 0, st>>>(c, p, s);
  else k_stage2<false><<<grids[1], 128, 0, st>>>(c, p, s);
  if (ev) cudaEventRecord(ev[4], st);
  if (debug) k_stage3<true><<<grids[2], S3_WARPS * 32, 0, st>>>(c, p3, s);
  else if (nost) k_stage3<false, true><<<grids[2], S3_WARPS * 32, 0, st>>>(c, p3, s);
  else k_stage3<false><<<grids[2], S3_WARPS * 32, 0, st>>>(c, p3, s);
  if (ev) cudaEventRecord(ev[5], st);
  if (debug) k_stage4<true><<<grids[3], S4_WARPS * 32, 0, st>>>(c, p, s);
  else if (nost) k_stage4<false, true><<<grids[3], S4_WARPS * 32, 0, st>>>(c, p, s);
  else k_stage4<false><<<grids[3], S4_WARPS * 32, 0, st>>>(c, p, s);
  if (ev) cudaEventRecord(ev[6], st);
  const int g5 = (int)((p.n_frames + 255) / 256);
  if (g5 > 0) k_stage5<<<g5, 256, 0, st>>>(p, s);
  if (ev) cudaEventRecord(ev[7], st);
  return cudaGetLastError();
}

}  // namespace m3e
