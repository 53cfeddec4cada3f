// Streaming selection of libm3e: frame-by-frame submission with continuous
// batching (the filter-farm setting of Sec. "Implementation": frames arrive
// continuously from the readout and each is selected on its own).
//
// Data path of one frame:
//   host    m3e_stream_submit copies the packet into a pinned host ring and
//           publishes a descriptor {ring offset, hit count} with a store-release
//           of the descriptor-ring tail;
//   feeder  one warp of the resident kernel sees the tail (acquire, system
//           scope), copies new descriptors into the device ring and releases
//           each slot by writing its sequence number (release, GPU scope);
//   worker  every other warp draws a ticket (the next sequence number), waits
//           with bounded back-off for its slot, reads the hits from the host
//           ring over the host link and runs the per-frame method (the fused
//           warp stage), then writes a completion word {seq, reason, keep} into
//           a pinned completion queue, in completion order (release, system
//           scope);
//   host    the library thread consumes the queue, delivers the results into
//           the caller's slots and frees ring space in submission order.
// Frames with more hits than the warp stage holds are batched by the library
// thread to a CTA-per-frame kernel.  The resident kernel exits when idle or at
// the end of its lifetime (and the thread relaunches it while frames wait);
// every device wait is bounded.
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <mutex>
#include <new>
#include <thread>
#include <time.h>
#include <vector>

#include "m3e_device.cuh"

namespace m3e {

struct HDesc {              // host descriptor ring entry
  long long off;            // first word in the packet ring
  int n;                    // hits
  int pad;
};

struct DDesc {              // device descriptor ring entry
  long long off;
  int n;
  int pad;
};

struct HeavyItem {          // frame run by the CTA-per-frame kernel
  long long off;
  int n;
  int pad;
  unsigned long long gseq;  // global submission number (host bookkeeping)
};

// Control words shared by host and device (pinned, mapped), each on its own line.
struct alignas(64) Control {
  unsigned long long tail;        // light frames published (host store-release)
  char p0[56];
  unsigned stop;                  // host: resident kernel must exit
  char p1[60];
  unsigned long long next_base;   // kernel at exit: first ticket it did not publish
  char p2[56];
  unsigned failed;                // kernel: a worker's wait expired
  char p3[60];
};

struct StreamK {
  KParams p;                      // look-up tables and error word
  const int32_t* ring;            // device view of the host packet ring
  const HDesc* hdesc;             // device view of the host descriptor ring
  Control* ctl;                   // device view of the control block
  unsigned long long* hcomp;      // device view of the host completion queue (completion order)
  DDesc* ddesc;                   // device descriptor ring
  unsigned long long* dseq;       // published sequence number of each device-ring slot
  unsigned long long* dstate;     // [0] tickets drawn in this launch, [1] stop ticket + 1 (0 = running)
  unsigned long long* dcq;        // completions written so far (all launches): the queue's tail
  unsigned long long base;        // first ticket of this launch
  unsigned long long mask;        // slots - 1
  long long idle_ns, life_ns, wait_ns;
  int feeder;                     // 0: nothing publishes (test of the bounded waits)
};

namespace {

__device__ __forceinline__ long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return (long long)t;
}
__device__ __forceinline__ unsigned long long ld_acquire_sys(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_acquire_gpu(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed_gpu(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned ld_relaxed_sys(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_gpu(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_release_sys(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_sys(unsigned* p, unsigned v) {
  asm volatile("st.relaxed.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long completion_word(unsigned long long t, int r) {
  return (t << 16) | ((unsigned long long)(r & 255) << 8) | (unsigned long long)(r != M3E_DROP);
}

// Warp 0 of CTA 0: moves published descriptors from the host ring into the
// device ring until told to stop, idle for idle_ns, or at the end of life_ns;
// then sets the stop ticket so that workers holding later tickets exit.
__device__ void feeder(const StreamK& K) {
  const int lane = threadIdx.x & 31;
  if (!K.feeder) return;  // test mode: the workers' waits must expire
  unsigned long long pub = K.base;
  const long long t0 = now_ns();
  long long last = t0;
  for (;;) {
    unsigned long long tail = 0;
    unsigned stop = 0;
    if (lane == 0) {
      tail = ld_acquire_sys(&K.ctl->tail);
      stop = ld_relaxed_sys(&K.ctl->stop);
    }
    tail = __shfl_sync(FULL, tail, 0);
    stop = __shfl_sync(FULL, stop, 0);
    __syncwarp();  // the lanes' reads of the descriptors follow lane 0's acquire
    const long long now = now_ns();
    if (stop || now - t0 > K.life_ns) break;
    if (tail > pub && tail - pub <= K.mask + 1) {
      // groups of 128 descriptors, four per lane: the four 16-byte loads over the
      // host link are in flight together, and one fence orders the group's
      // device-ring writes before its sequence numbers (release pattern)
      for (unsigned long long b = pub; b < tail; b += 128) {
        int4 v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const unsigned long long i = b + j * 32 + lane;
          v[j] = i < tail ? __ldcv(reinterpret_cast<const int4*>(K.hdesc + (i & K.mask))) : make_int4(0, 0, 0, 0);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const unsigned long long i = b + j * 32 + lane;
          if (i < tail) *reinterpret_cast<int4*>(K.ddesc + (i & K.mask)) = v[j];
        }
        __threadfence();
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const unsigned long long i = b + j * 32 + lane;
          if (i < tail) st_relaxed_gpu(&K.dseq[i & K.mask], i);
        }
      }
      pub = tail;
      last = now;
    } else {
      if (now - last > K.idle_ns) break;
      __nanosleep(128);
    }
  }
  if (lane == 0) {
    atomicExch(&K.dstate[1], pub + 1);
    K.ctl->next_base = pub;
  }
}

__global__ void __launch_bounds__(WARPS_PER_CTA * 32)
    k_stream_warp(const __grid_constant__ DevCfg C, const __grid_constant__ StreamK K) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int64_t soff[WARPS_PER_CTA][2];
  const int w = threadIdx.x >> 5;
  if (blockIdx.x == 0 && w == 0) {
    feeder(K);
    return;
  }
  SmWarp& sm = reinterpret_cast<SmWarp*>(smem_raw)[w];
  const WarpGroup g;
  KParams Q = K.p;
  Q.off = soff[w];
  Q.off_base = 0;
  Q.stats = nullptr;
  Q.defer_hits = W_HITS;
  for (;;) {
    unsigned long long t = 0;
    int go = 0;
    if (g.leader()) {
      t = K.base + atomicAdd(&K.dstate[0], 1ull);
      const long long ws = now_ns();
      unsigned ns = 32;
      for (;;) {
        if (ld_acquire_gpu(&K.dseq[t & K.mask]) == t) {
          go = 1;
          break;
        }
        const unsigned long long sv = ld_relaxed_gpu(&K.dstate[1]);
        if (sv != 0 && t + 1 >= sv) break;  // ticket beyond the last published frame
        if (now_ns() - ws > K.wait_ns) {    // nothing published it in time
          st_relaxed_sys(&K.ctl->failed, 1u);
          break;
        }
        __nanosleep(ns);
        if (ns < 1024) ns <<= 1;
      }
    }
    go = __shfl_sync(FULL, go, 0);
    if (!go) break;
    t = __shfl_sync(FULL, t, 0);
    __syncwarp();  // the lanes' reads of the frame follow the leader's acquire
    const DDesc d = K.ddesc[t & K.mask];
    if (g.leader()) {
      soff[w][0] = 0;
      soff[w][1] = d.n;
    }
    Q.hits = K.ring + d.off;
    g.sync();
    int r = frame_front<WarpGroup, SmWarp, W_HITS, W_TRIP, true, false, true>(g, sm, C, Q, 0);
    if (r == PENDING) r = frame_back<WarpGroup, SmWarp, W_TRIP, W_TRK, W_COMBO, true, false>(g, sm, C, Q, 0);
    // frames above the warp stage never get here (the host routes them to the
    // CTA kernel); keep one conservatively should that ever change
    if (r == DEFERRED) r = M3E_HIT_OVERFLOW;
    g.sync();
    // append to the completion queue: the host consumes it in order, O(1) per frame
    if (g.leader()) {
      const unsigned long long c = atomicAdd(K.dcq, 1ull);
      st_release_sys(&K.hcomp[c & K.mask], completion_word(t, r));
    }
  }
}

// Frames with more hits than the warp stage holds, one CTA per frame, from a
// list written by the host before the launch; results (reason << 8 | keep) into
// mapped host memory, read by the host after the launch completes.
template <int NT>
__global__ void __launch_bounds__(NT)
    k_stream_cta(const __grid_constant__ DevCfg C, const __grid_constant__ StreamK K, const HeavyItem* items,
                 int count, unsigned short* res) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int64_t soff[2];
  SmCta& sm = *reinterpret_cast<SmCta*>(smem_raw);
  const CtaGroup<NT> g;
  KParams Q = K.p;
  Q.off = soff;
  Q.off_base = 0;
  Q.stats = nullptr;
  for (int i = blockIdx.x; i < count; i += gridDim.x) {
    const long long off = __ldcv(&items[i].off);
    const int n = __ldcv(&items[i].n);
    if (g.leader()) {
      soff[0] = 0;
      soff[1] = n;
    }
    Q.hits = K.ring + off;
    g.sync();
    int r = frame_front<CtaGroup<NT>, SmCta, C_HITS, C_TRIP, false, false, true>(g, sm, C, Q, 0);
    if (r == PENDING) r = frame_back<CtaGroup<NT>, SmCta, C_TRIP, C_TRK, C_COMBO, false, false>(g, sm, C, Q, 0);
    g.sync();
    if (g.leader()) res[i] = (unsigned short)(((r & 255) << 8) | (r != M3E_DROP));
    g.sync();
  }
}

int64_t host_ns() {
  timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (int64_t)ts.tv_sec * 1000000000LL + ts.tv_nsec;
}

inline void cpu_relax() {
#if defined(__aarch64__)
  asm volatile("yield" ::: "memory");
#else
  std::atomic_signal_fence(std::memory_order_seq_cst);
#endif
}

// splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014): counter-based, one 64-bit output per index.
inline uint64_t splitmix64(uint64_t x) {
  x += 0x9e3779b97f4a7c15ULL;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ULL;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebULL;
  return x ^ (x >> 31);
}

struct SpinLock {
  std::atomic_flag f = ATOMIC_FLAG_INIT;
  void lock() {
    while (f.test_and_set(std::memory_order_acquire)) cpu_relax();
  }
  void unlock() { f.clear(std::memory_order_release); }
};

}  // namespace

struct StreamEngine {
  int device = 0, sms = 1;
  DevCfg dc{};
  KParams base{};
  m3e_stream_params prm{};
  uint64_t S = 0, mask = 0;
  int64_t W = 0;  // ring words
  // pinned host memory and its device views
  int32_t* ring = nullptr;
  HDesc* hdesc = nullptr;
  Control* ctl = nullptr;
  unsigned long long* hcomp = nullptr;
  HeavyItem* hitems = nullptr;
  unsigned short* hres = nullptr;
  int32_t* d_ring = nullptr;
  HDesc* d_hdesc = nullptr;
  Control* d_ctl = nullptr;
  unsigned long long* d_hcomp = nullptr;
  HeavyItem* d_hitems = nullptr;
  unsigned short* d_hres = nullptr;
  // device rings
  DDesc* ddesc = nullptr;
  unsigned long long* dseq = nullptr;
  unsigned long long* dstate = nullptr;
  unsigned long long* dcq = nullptr;
  uint64_t cq_head = 0;           // next completion-queue entry to consume (library thread)
  cudaStream_t rs = nullptr, hs = nullptr;
  cudaEvent_t re = nullptr, he = nullptr;
  int grid = 1;
  int heavy_cap = 4096;
  // per submitted frame (index: global sequence & mask)
  struct Slot {
    m3e_result* res;
    int64_t word_end;
    std::atomic<uint8_t> state;  // 0 free, 1 in flight, 2 done
  };
  Slot* slots = nullptr;
  uint64_t* lmap = nullptr;   // light sequence -> global sequence
  uint8_t* ldone = nullptr;   // light sequence delivered (library thread only)
  // producer side (under lock)
  SpinLock lock;
  uint64_t gseq = 0, lseq = 0;
  int64_t wpos = 0;
  uint64_t low_seen = 0;          // last values of low and rpos read by the producer: re-read
  int64_t rpos_seen = 0;          // only when the ring looks full (they only grow)
  std::vector<HeavyItem> heavy_pending;
  // written by the producer, read by the library thread (own cache line)
  alignas(64) std::atomic<uint64_t> gseq_pub{0};
  std::atomic<uint64_t> lseq_pub{0};
  std::atomic<uint64_t> heavy_n{0};     // frames in heavy_pending
  std::atomic<bool> asleep{false};      // library thread asleep; set and cleared under the lock
  // written by the library thread, read by the producer (own cache line)
  alignas(64) std::atomic<uint64_t> low{0};   // every frame below is delivered and released
  std::atomic<int64_t> rpos{0};               // ring words below are free
  alignas(64) uint64_t lscan = 0;
  uint64_t tail_pub = 0;          // last tail the library thread stored into the control block
  bool rk_running = false, hk_running = false;
  uint64_t rk_base = 0;
  int hk_count = 0;
  // counters and flags
  std::atomic<uint64_t> completed{0}, busy{0}, launches{0}, heavy{0};
  std::atomic<uint64_t> passes_delivering{0}, tail_stores{0};
  std::atomic<bool> failed{false}, quit{false}, running_flag{false};
  std::mutex mu;
  std::condition_variable cv;
  std::thread th;

  // t_done: the delivery time (read once per pass of the library thread)
  void deliver(uint64_t g, int keep, int reason, int err, int64_t t_done = -1) {
    Slot& s = slots[g & mask];
    m3e_result* r = s.res;
    r->keep = (uint8_t)keep;
    r->reason = (uint8_t)reason;
    r->err = err ? err : (reason == M3E_ERR_BADHIT ? M3E_EBADHIT : M3E_OK);
    r->t_done_ns = (uint64_t)(t_done >= 0 ? t_done : host_ns());
    __atomic_store_n(&r->done, 1u, __ATOMIC_RELEASE);
    s.state.store(2, std::memory_order_relaxed);  // read by this thread only
    completed.store(completed.load(std::memory_order_relaxed) + 1, std::memory_order_relaxed);  // one writer
  }

  // Deliveries of the completion queue, in batches: every field of the batch,
  // one release fence, then the done flags (one fence per batch, not per frame).
  static constexpr int DB = 64;
  uint64_t db_g[DB];
  unsigned long long db_w[DB];
  int db_n = 0;
  void flush_deliveries() {
    if (!db_n) return;
    const uint64_t t = (uint64_t)host_ns();
    for (int i = 0; i < db_n; ++i) {
      m3e_result* r = slots[db_g[i] & mask].res;
      const int reason = (int)((db_w[i] >> 8) & 255);
      r->keep = (uint8_t)(db_w[i] & 1);
      r->reason = (uint8_t)reason;
      r->err = reason == M3E_ERR_BADHIT ? M3E_EBADHIT : M3E_OK;
      r->t_done_ns = t;
    }
    std::atomic_thread_fence(std::memory_order_release);
    for (int i = 0; i < db_n; ++i) {
      Slot& sl = slots[db_g[i] & mask];
      __atomic_store_n(&sl.res->done, 1u, __ATOMIC_RELAXED);
      sl.state.store(2, std::memory_order_relaxed);
    }
    completed.store(completed.load(std::memory_order_relaxed) + (uint64_t)db_n, std::memory_order_relaxed);
    db_n = 0;
    publish_tail();  // keep the feeder supplied during long passes
  }

  cudaError_t launch_resident(uint64_t b) {
    StreamK k{};
    k.p = base;
    k.ring = d_ring;
    k.hdesc = d_hdesc;
    k.ctl = d_ctl;
    k.hcomp = d_hcomp;
    k.ddesc = ddesc;
    k.dseq = dseq;
    k.dstate = dstate;
    k.dcq = dcq;
    k.base = b;
    k.mask = mask;
    k.idle_ns = (long long)prm.idle_us * 1000LL;
    k.life_ns = (long long)prm.lifetime_ms * 1000000LL;
    k.wait_ns = (long long)prm.wait_limit_ms * 1000000LL;
    k.feeder = prm.no_feeder ? 0 : 1;
    cudaError_t e = cudaMemsetAsync(dstate, 0, 2 * sizeof(unsigned long long), rs);
    if (e != cudaSuccess) return e;
    k_stream_warp<<<grid, WARPS_PER_CTA * 32, sizeof(SmWarp) * WARPS_PER_CTA, rs>>>(dc, k);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaEventRecord(re, rs);
  }

  cudaError_t launch_heavy(int count) {
    StreamK k{};
    k.p = base;
    k.ring = d_ring;
    const int g = count < sms ? count : sms;
    k_stream_cta<CTA_THREADS><<<g, CTA_THREADS, sizeof(SmCta), hs>>>(dc, k, d_hitems, count, d_hres);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaEventRecord(he, hs);
  }

  // Light completions written by the resident kernel, consumed from the
  // completion queue in completion order (an entry is written once its index is
  // drawn; the consumer clears it before delivering, so that it is empty again
  // before the queue wraps: at most `slots` frames are undelivered).  With
  // fail_rest, every light frame still in flight afterwards is failed.
  bool scan_light(bool fail_rest) {
    bool any = false;
    for (;;) {
      unsigned long long* e = &hcomp[cq_head & mask];
      const unsigned long long wv = __atomic_load_n(e, __ATOMIC_ACQUIRE);
      if (wv == ~0ULL) break;
      __atomic_store_n(e, ~0ULL, __ATOMIC_RELAXED);
      ++cq_head;
      const uint64_t l = wv >> 16;
      db_g[db_n] = lmap[l & mask];
      db_w[db_n] = wv;
      if (++db_n == DB) flush_deliveries();
      ldone[l & mask] = 1;
      any = true;
    }
    flush_deliveries();
    if (any) passes_delivering.fetch_add(1, std::memory_order_relaxed);
    const uint64_t lp = lseq_pub.load(std::memory_order_acquire);
    if (fail_rest)
      for (uint64_t l = lscan; l < lp; ++l)
        if (!ldone[l & mask]) {
          deliver(lmap[l & mask], 1, M3E_ERR_BADHIT, M3E_ETIMEOUT);
          ldone[l & mask] = 1;
          any = true;
        }
    while (lscan < lp && ldone[lscan & mask]) ldone[lscan++ & mask] = 0;
    return any;
  }

  // With no kernel on the GPU: every frame still in flight gets err =
  // M3E_ETIMEOUT (the stream failed, or it is closing with frames left).
  void fail_pending() {
    scan_light(true);
    std::vector<HeavyItem> left;
    lock.lock();
    left.swap(heavy_pending);
    heavy_n.store(0, std::memory_order_relaxed);
    lock.unlock();
    for (const HeavyItem& h : left) deliver(h.gseq, 1, M3E_ERR_BADHIT, M3E_ETIMEOUT);
  }

  void release_in_order() {
    uint64_t lo = low.load(std::memory_order_relaxed);
    const uint64_t gs = gseq_pub.load(std::memory_order_acquire);
    int64_t rp = -1;
    while (lo < gs && slots[lo & mask].state.load(std::memory_order_acquire) == 2) {
      rp = slots[lo & mask].word_end;
      slots[lo & mask].state.store(0, std::memory_order_relaxed);
      ++lo;
    }
    if (rp >= 0) rpos.store(rp, std::memory_order_release);
    low.store(lo, std::memory_order_release);
  }

  // Make the light frames submitted so far visible to the resident kernel.  The
  // library thread publishes (one store of the polled tail word for any number
  // of submissions), so that the submitting thread never writes the word the
  // GPU is polling.
  void publish_tail() {
    const uint64_t lp = lseq_pub.load(std::memory_order_acquire);
    if (lp != tail_pub) {
      __atomic_store_n(&ctl->tail, (unsigned long long)lp, __ATOMIC_RELEASE);
      tail_pub = lp;
      tail_stores.store(tail_stores.load(std::memory_order_relaxed) + 1, std::memory_order_relaxed);
    }
  }

  void run() {
    cudaSetDevice(device);
    int64_t idle_since = -1;
    for (;;) {
      publish_tail();
      bool progress = scan_light(false);
      publish_tail();
      const uint64_t lp = lseq_pub.load(std::memory_order_acquire);
      // resident kernel: exited?  relaunch while light frames wait
      if (rk_running && cudaEventQuery(re) != cudaErrorNotReady) {
        rk_running = false;
        running_flag.store(false);
        rk_base = __atomic_load_n(&ctl->next_base, __ATOMIC_ACQUIRE);
        if (__atomic_load_n(&ctl->failed, __ATOMIC_ACQUIRE)) failed.store(true);
        progress = scan_light(false) || true;
      }
      if (!rk_running && !failed.load() && !quit.load() && lp > rk_base) {
        if (launch_resident(rk_base) != cudaSuccess) {
          failed.store(true);
        } else {
          rk_running = true;
          running_flag.store(true);
          launches.fetch_add(1);
        }
        progress = true;
      }
      // frames beyond the warp stage
      if (hk_running && cudaEventQuery(he) != cudaErrorNotReady) {
        for (int i = 0; i < hk_count; ++i) {
          const unsigned short v = __atomic_load_n(&hres[i], __ATOMIC_ACQUIRE);
          deliver(hitems[i].gseq, v & 1, v >> 8, 0);
        }
        heavy.fetch_add((uint64_t)hk_count);
        hk_running = false;
        progress = true;
      }
      if (!hk_running && !failed.load() && !quit.load() && heavy_n.load(std::memory_order_relaxed)) {
        int n = 0;
        lock.lock();
        if (!heavy_pending.empty()) {
          n = (int)std::min<size_t>(heavy_pending.size(), (size_t)heavy_cap);
          memcpy(hitems, heavy_pending.data(), sizeof(HeavyItem) * n);
          heavy_pending.erase(heavy_pending.begin(), heavy_pending.begin() + n);
          heavy_n.fetch_sub((uint64_t)n, std::memory_order_relaxed);
        }
        lock.unlock();
        if (n) {
          for (int i = 0; i < n; ++i) hres[i] = 0;
          hk_count = n;
          if (launch_heavy(n) != cudaSuccess) {
            failed.store(true);
            for (int i = 0; i < n; ++i) deliver(hitems[i].gseq, 1, M3E_ERR_BADHIT, M3E_ETIMEOUT);
          } else {
            hk_running = true;
          }
          progress = true;
        }
      }
      const bool none_running = !rk_running && !hk_running;
      if (none_running && (failed.load() || quit.load())) fail_pending();
      release_in_order();
      if (quit.load() && none_running) break;
      if (progress || low.load() != gseq_pub.load()) {
        idle_since = -1;
        if (!progress)
          for (int i = 0; i < 16; ++i) cpu_relax();
        continue;
      }
      // nothing in flight: keep spinning for a while (frames at a steady rate
      // should not pay a wake-up), then sleep until a submission wakes us.  The
      // decision to sleep and the producer's check of it are both made under the
      // producer lock, so a submission cannot slip between them.
      const int64_t now = host_ns();
      if (idle_since < 0) idle_since = now;
      if (now - idle_since < 200000) {
        for (int i = 0; i < 64; ++i) cpu_relax();
        continue;
      }
      lock.lock();
      const bool go = gseq == low.load(std::memory_order_relaxed) && !quit.load();
      if (go) asleep.store(true, std::memory_order_relaxed);
      lock.unlock();
      if (go) {
        // the resident kernel exits by itself when idle; its exit is noticed on
        // wake-up or on the timeout
        std::unique_lock<std::mutex> lk(mu);
        cv.wait_for(lk, std::chrono::milliseconds(rk_running || hk_running ? 1 : 20),
                    [&] { return !asleep.load() || quit.load(); });
        lock.lock();
        asleep.store(false, std::memory_order_relaxed);
        lock.unlock();
      }
    }
  }

  // Admit frames first .. first + count - 1 of a CSR batch (hits of frame f at
  // hits[off[f] .. off[f + 1]), result slot res[f - first], tag tags[f - first]
  // or tag0 + (f - first)) in order, until one does not fit.  One lock, one clock
  // read and one publication for the whole range.  Returns the number admitted.
  int64_t submit_range(const int32_t* hits, const int64_t* off, int64_t first, int64_t count, const uint64_t* tags,
                       uint64_t tag0, m3e_result* res) {
    lock.lock();
    const uint64_t t_submit = (uint64_t)host_ns();
    const uint64_t g0 = gseq, l0 = lseq;
    int64_t k = 0;
    bool heavy_added = false;
    for (; k < count; ++k) {
      const int64_t f = first + k;
      const int64_t n = off[f + 1] - off[f];
      const uint64_t g = gseq;
      if (g - low_seen >= S && g - (low_seen = low.load(std::memory_order_acquire)) >= S) break;
      const int64_t rem = W - (wpos % W);
      const int64_t start = n > rem ? wpos + rem : wpos;
      const int64_t end = start + n;
      if (end - rpos_seen > W && end - (rpos_seen = rpos.load(std::memory_order_acquire)) > W) break;
      wpos = end;
      const int64_t o = start % W;
      if (n) memcpy(ring + o, hits + off[f], sizeof(int32_t) * (size_t)n);
      m3e_result* r = res + k;
      r->keep = 0;
      r->reason = 0;
      r->err = 0;
      r->tag = tags ? tags[k] : tag0 + (uint64_t)k;
      r->t_done_ns = 0;
      r->t_submit_ns = t_submit;
      __atomic_store_n(&r->done, 0u, __ATOMIC_RELAXED);
      Slot& sl = slots[g & mask];
      sl.res = r;
      sl.word_end = end;
      sl.state.store(1, std::memory_order_relaxed);
      gseq = g + 1;
      if (n <= W_HITS) {
        const uint64_t l = lseq;
        hdesc[l & mask].off = o;
        hdesc[l & mask].n = (int)n;
        lmap[l & mask] = g;
        lseq = l + 1;
      } else {
        heavy_pending.push_back(HeavyItem{o, (int)n, 0, g});
        heavy_added = true;
      }
    }
    if (heavy_added) heavy_n.store(heavy_pending.size(), std::memory_order_relaxed);
    if (gseq != g0) gseq_pub.store(gseq, std::memory_order_release);
    if (lseq != l0) lseq_pub.store(lseq, std::memory_order_release);
    // the library thread publishes the tail while it runs; asleep, it is woken
    // and the frames are published here (the thread decides to sleep under this
    // lock, so the check cannot miss them)
    const bool wake = k > 0 && asleep.load(std::memory_order_relaxed);
    if (wake) {
      asleep.store(false, std::memory_order_relaxed);
      __atomic_store_n(&ctl->tail, (unsigned long long)lseq, __ATOMIC_RELEASE);
    }
    lock.unlock();
    if (k < count) busy.fetch_add(1, std::memory_order_relaxed);
    if (wake) {
      std::lock_guard<std::mutex> lk(mu);
      cv.notify_one();
    }
    return k;
  }

  int submit(const int32_t* pkt, int32_t n, uint64_t tag, m3e_result* res) {
    if (failed.load(std::memory_order_relaxed)) return m3e_set_error(M3E_ETIMEOUT, "stream has failed");
    if (quit.load(std::memory_order_relaxed)) return m3e_set_error(M3E_ESTATE, "stream is closing");
    const int64_t off[2] = {0, n};
    return submit_range(pkt, off, 0, 1, nullptr, tag, res) == 1 ? M3E_OK : M3E_EBUSY;
  }

  int drain(int64_t timeout_ms) {
    const int64_t deadline = host_ns() + timeout_ms * 1000000LL;
    for (;;) {
      if (low.load(std::memory_order_acquire) == gseq_pub.load(std::memory_order_acquire))
        return failed.load() ? m3e_set_error(M3E_ETIMEOUT, "stream failed: a device wait expired") : M3E_OK;
      if (host_ns() > deadline) return m3e_set_error(M3E_ETIMEOUT, "drain: results still missing after %lld ms",
                                                       (long long)timeout_ms);
      std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
  }

  void free_all() {
    if (ring) cudaFreeHost(ring);
    if (hdesc) cudaFreeHost(hdesc);
    if (ctl) cudaFreeHost(ctl);
    if (hcomp) cudaFreeHost(hcomp);
    if (hitems) cudaFreeHost(hitems);
    if (hres) cudaFreeHost(hres);
    cudaFree(ddesc);
    cudaFree(dseq);
    cudaFree(dstate);
    cudaFree(dcq);
    if (rs) cudaStreamDestroy(rs);
    if (hs) cudaStreamDestroy(hs);
    if (re) cudaEventDestroy(re);
    if (he) cudaEventDestroy(he);
    delete[] slots;
    delete[] lmap;
    delete[] ldone;
  }
};

#define S_TRY(x)                                                                            \
  do {                                                                                      \
    cudaError_t e_ = (x);                                                                   \
    if (e_ != cudaSuccess) {                                                                \
      E->free_all();                                                                        \
      delete E;                                                                             \
      return m3e_set_error(M3E_ECUDA, "%s: %s", #x, cudaGetErrorString(e_));                \
    }                                                                                       \
  } while (0)

template <class T>
static cudaError_t host_mapped(T** h, T** d, size_t bytes) {
  cudaError_t e = cudaHostAlloc((void**)h, bytes, cudaHostAllocMapped | cudaHostAllocPortable);
  if (e != cudaSuccess) return e;
  return cudaHostGetDevicePointer((void**)d, (void*)*h, 0);
}

int stream_create(int device, int sms, const DevCfg& dc, const KParams& base, const m3e_stream_params* sp,
                  StreamEngine** out) {
  m3e_stream_params p{};
  p.size = sizeof(m3e_stream_params);
  if (sp) {
    if (sp->size != sizeof(m3e_stream_params))
      return m3e_set_error(M3E_EINVAL, "m3e_stream_params.size %u != %zu", sp->size, sizeof(m3e_stream_params));
    p = *sp;
  }
  if (p.slots == 0) p.slots = 65536;
  if (p.ring_bytes == 0) p.ring_bytes = 64LL << 20;
  if (p.ctas_per_sm == 0) p.ctas_per_sm = 2;
  if (p.idle_us == 0) p.idle_us = 20000;
  if (p.lifetime_ms == 0) p.lifetime_ms = 2000;
  if (p.wait_limit_ms == 0) p.wait_limit_ms = p.lifetime_ms + 1000;
  if (p.slots < 2 || p.slots > (1 << 24) || (p.slots & (p.slots - 1)))
    return m3e_set_error(M3E_EINVAL, "slots must be a power of two in 2..2^24");
  if (p.ring_bytes < 4096 || p.ring_bytes > (8LL << 30) || (p.ring_bytes & 3))
    return m3e_set_error(M3E_EINVAL, "ring_bytes must be a multiple of 4 in 4 KiB..8 GiB");
  if (p.ctas_per_sm < 1 || p.ctas_per_sm > 16) return m3e_set_error(M3E_EINVAL, "ctas_per_sm 1..16");
  if (p.idle_us < 1 || p.lifetime_ms < 1 || p.wait_limit_ms < 1 || p.lifetime_ms > 60000 ||
      p.wait_limit_ms > 120000 || p.idle_us > 10000000)
    return m3e_set_error(M3E_EINVAL, "idle_us, lifetime_ms (<= 60 s) and wait_limit_ms (<= 120 s) must be positive");
  StreamEngine* E = new (std::nothrow) StreamEngine();
  if (!E) return m3e_set_error(M3E_ENOMEM, "stream engine");
  E->device = device;
  E->sms = sms;
  E->dc = dc;
  E->base = base;
  E->prm = p;
  E->S = (uint64_t)p.slots;
  E->mask = E->S - 1;
  E->W = p.ring_bytes / 4;
  E->slots = new (std::nothrow) StreamEngine::Slot[E->S];
  E->lmap = new (std::nothrow) uint64_t[E->S];
  E->ldone = new (std::nothrow) uint8_t[E->S];
  if (!E->slots || !E->lmap || !E->ldone) {
    E->free_all();
    delete E;
    return m3e_set_error(M3E_ENOMEM, "stream slots");
  }
  for (uint64_t i = 0; i < E->S; ++i) {
    E->slots[i].res = nullptr;
    E->slots[i].word_end = 0;
    E->slots[i].state.store(0);
    E->ldone[i] = 0;
  }
  S_TRY(host_mapped(&E->ring, &E->d_ring, (size_t)p.ring_bytes));
  S_TRY(host_mapped(&E->hdesc, &E->d_hdesc, sizeof(HDesc) * E->S));
  S_TRY(host_mapped(&E->ctl, &E->d_ctl, sizeof(Control)));
  S_TRY(host_mapped(&E->hcomp, &E->d_hcomp, sizeof(unsigned long long) * E->S));
  S_TRY(host_mapped(&E->hitems, &E->d_hitems, sizeof(HeavyItem) * E->heavy_cap));
  S_TRY(host_mapped(&E->hres, &E->d_hres, sizeof(unsigned short) * E->heavy_cap));
  memset(E->ctl, 0, sizeof(Control));
  memset(E->hcomp, 0xff, sizeof(unsigned long long) * E->S);  // all entries empty
  S_TRY(cudaMalloc(&E->ddesc, sizeof(DDesc) * E->S));
  S_TRY(cudaMalloc(&E->dseq, sizeof(unsigned long long) * E->S));
  S_TRY(cudaMalloc(&E->dstate, 2 * sizeof(unsigned long long)));
  S_TRY(cudaMalloc(&E->dcq, sizeof(unsigned long long)));
  S_TRY(cudaStreamCreateWithFlags(&E->rs, cudaStreamNonBlocking));
  S_TRY(cudaMemsetAsync(E->dseq, 0xff, sizeof(unsigned long long) * E->S, E->rs));
  S_TRY(cudaMemsetAsync(E->dcq, 0, sizeof(unsigned long long), E->rs));
  S_TRY(cudaStreamCreateWithFlags(&E->hs, cudaStreamNonBlocking));
  S_TRY(cudaEventCreateWithFlags(&E->re, cudaEventDisableTiming));
  S_TRY(cudaEventCreateWithFlags(&E->he, cudaEventDisableTiming));
  const size_t smw = sizeof(SmWarp) * WARPS_PER_CTA;
  S_TRY(cudaFuncSetAttribute(k_stream_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smw));
  S_TRY(cudaFuncSetAttribute(k_stream_cta<CTA_THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(SmCta)));
  int nb = 0;
  S_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_stream_warp, WARPS_PER_CTA * 32, smw));
  if (nb < 1) nb = 1;
  E->grid = sms * (p.ctas_per_sm < nb ? p.ctas_per_sm : nb);
  S_TRY(cudaStreamSynchronize(E->rs));
  E->th = std::thread([E] { E->run(); });
  *out = E;
  return M3E_OK;
}

int stream_submit(StreamEngine* E, const int32_t* pkt, int32_t n, uint64_t tag, m3e_result* res) {
  if (!res) return m3e_set_error(M3E_EINVAL, "result slot is NULL");
  if (n < 0 || (n > 0 && !pkt)) return m3e_set_error(M3E_EINVAL, "packet: n_hits < 0 or NULL packet");
  if ((int64_t)n > E->W) return m3e_set_error(M3E_EINVAL, "packet of %d hits is larger than the ring", n);
  return E->submit(pkt, n, tag, res);
}

int stream_submit_many(StreamEngine* E, const int32_t* hits, const int64_t* off, int64_t n_frames,
                       const uint64_t* tags, m3e_result* res, int64_t* admitted) {
  if (admitted) *admitted = 0;
  if (n_frames < 0 || (n_frames > 0 && (!off || !res))) return m3e_set_error(M3E_EINVAL, "submit_many: NULL arguments");
  for (int64_t f = 0; f < n_frames; ++f) {
    const int64_t n = off[f + 1] - off[f];
    if (n < 0 || n > E->W || n > 0x7fffffff) return m3e_set_error(M3E_EINVAL, "submit_many: frame %lld has a bad size", (long long)f);
    if (n > 0 && !hits) return m3e_set_error(M3E_EINVAL, "submit_many: hits is NULL");
  }
  if (E->failed.load(std::memory_order_relaxed)) return m3e_set_error(M3E_ETIMEOUT, "stream has failed");
  if (E->quit.load(std::memory_order_relaxed)) return m3e_set_error(M3E_ESTATE, "stream is closing");
  const int64_t k = n_frames ? E->submit_range(hits, off, 0, n_frames, tags, 0, res) : 0;
  if (admitted) *admitted = k;
  return k == n_frames ? M3E_OK : M3E_EBUSY;
}

int stream_poll(StreamEngine* E, m3e_stream_status* o) {
  o->submitted = E->gseq_pub.load();
  o->completed = E->completed.load();
  o->busy_refusals = E->busy.load();
  o->kernel_launches = E->launches.load();
  o->heavy_frames = E->heavy.load();
  o->kernel_running = E->running_flag.load() ? 1 : 0;
  o->delivery_passes = E->passes_delivering.load();
  o->tail_publications = E->tail_stores.load();
  o->failed = E->failed.load() ? 1 : 0;
  return M3E_OK;
}

int stream_drain(StreamEngine* E, int64_t timeout_ms) { return E->drain(timeout_ms); }

int stream_destroy(StreamEngine* E) {
  if (!E) return M3E_OK;
  int rc = E->drain(10000);
  E->quit.store(true);
  __atomic_store_n(&E->ctl->stop, 1u, __ATOMIC_RELEASE);
  {
    std::lock_guard<std::mutex> lk(E->mu);
    E->cv.notify_one();
  }
  // the library thread stops relaunching, waits for its kernels to return (the
  // resident kernel exits on the stop word), fails any frame still in flight
  // and ends
  E->th.join();
  cudaStreamSynchronize(E->rs);
  cudaStreamSynchronize(E->hs);
  E->free_all();
  delete E;
  return rc;
}

int stream_replay(StreamEngine* E, const int32_t* hits, const int64_t* off, int64_t nf, double rate_hz,
                  uint64_t seed, uint8_t* out_keep, uint8_t* out_reason, int64_t* lat_submit, int64_t* lat_arrival,
                  m3e_replay_stats* st) {
  if (nf < 0 || (nf > 0 && (!hits || !off))) return m3e_set_error(M3E_EINVAL, "replay: empty or NULL batch");
  if (!(rate_hz > 0)) return m3e_set_error(M3E_EINVAL, "replay: rate_hz must be positive");
  for (int64_t f = 0; f < nf; ++f)
    if (off[f + 1] < off[f] || off[f + 1] - off[f] > E->W)
      return m3e_set_error(M3E_EINVAL, "replay: frame %lld has a bad size", (long long)f);
  // result slots of the submitted frames: freed only once every submitted frame
  // has its result (the library thread writes them until then)
  m3e_result* res = new (std::nothrow) m3e_result[nf > 0 ? nf : 1];
  if (!res) return m3e_set_error(M3E_ENOMEM, "replay: result slots");
  int64_t submitted = 0;
  auto settle = [&](int64_t wait_ms) -> bool {  // all submitted results written?
    const int64_t dl = host_ns() + wait_ms * 1000000LL;
    for (int64_t f = 0; f < submitted; ++f)
      while (!__atomic_load_n(&res[f].done, __ATOMIC_ACQUIRE)) {
        if (host_ns() > dl) return false;
        std::this_thread::sleep_for(std::chrono::microseconds(20));
      }
    return true;
  };
  auto bail = [&](int rc) -> int {
    // frames in flight still point at res: free it only once they are settled
    // (a failed stream settles them when its kernels have returned), else leak it
    if (settle(60000)) delete[] res;
    return rc;
  };
  std::vector<int64_t> arr((size_t)nf);
  // exponential gaps by inversion of uniform (0, 1] draws
  double t = 0.0;
  for (int64_t f = 0; f < nf; ++f) {
    const double u = ((splitmix64(seed * 0x2545f4914f6cdd1dULL + (uint64_t)f) >> 11) + 1.0) * 0x1.0p-53;
    t += -std::log(u) / rate_hz;
    arr[f] = (int64_t)(t * 1e9);
  }
  const uint64_t launches0 = E->launches.load();
  uint64_t retries = 0;
  const int64_t t0 = host_ns() + 2000000;  // start 2 ms from now
  int64_t last_submit = t0;
  // every frame whose arrival time has come is submitted in one call (at most
  // 1024): below the host's per-call rate that is one frame per call
  for (int64_t f = 0; f < nf;) {
    int64_t now = host_ns();
    while (now < t0 + arr[f]) {
      cpu_relax();
      now = host_ns();
    }
    int64_t e = f + 1;
    while (e < nf && e - f < 1024 && t0 + arr[e] <= now) ++e;
    if (E->failed.load(std::memory_order_relaxed)) return bail(m3e_set_error(M3E_ETIMEOUT, "stream has failed"));
    const int64_t k = E->submit_range(hits, off, f, e - f, nullptr, (uint64_t)f, res + f);
    if (k < e - f) ++retries;
    f += k;
    submitted = f;
  }
  last_submit = host_ns();
  if (!settle(30000)) return bail(m3e_set_error(M3E_ETIMEOUT, "replay: results missing 30 s after the last arrival"));
  int64_t tmax = t0;
  int err = M3E_OK;
  for (int64_t f = 0; f < nf; ++f) {
    const m3e_result& r = res[f];
    if (r.err == M3E_ETIMEOUT) err = M3E_ETIMEOUT;
    if (out_keep) out_keep[f] = r.keep;
    if (out_reason) out_reason[f] = r.reason;
    if (lat_submit) lat_submit[f] = (int64_t)(r.t_done_ns - r.t_submit_ns);
    if (lat_arrival) lat_arrival[f] = (int64_t)r.t_done_ns - (t0 + arr[f]);
    if ((int64_t)r.t_done_ns > tmax) tmax = (int64_t)r.t_done_ns;
  }
  if (st) {
    st->offered_hz = rate_hz;
    st->duration_ns = tmax - t0;
    st->sustained_hz = nf > 0 ? (double)nf / ((double)(tmax - t0) * 1e-9) : 0.0;
    st->submit_hz = nf > 0 ? (double)nf / ((double)(last_submit - t0) * 1e-9) : 0.0;
    st->busy_retries = retries;
    st->kernel_launches = E->launches.load() - launches0;
  }
  delete[] res;
  if (err) return m3e_set_error(M3E_ETIMEOUT, "replay: the stream failed");
  return M3E_OK;
}

}  // namespace m3e
