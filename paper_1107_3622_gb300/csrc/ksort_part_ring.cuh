// Single partition (Steps 1-4 of Section 1.1) of one array in one launch, through a
// ring of shared-memory tiles: part_ring_kernel.
//
// The array's key is its first element (Step 1). Every other element x goes to the
// right side when key <= x and to the left side otherwise (Step 3); the key lands at
// #{x < key} (Step 4). The output buffer receives the left side from the front, the key,
// then the right side; every key is read once and written once.
//
// A CTA owns a ring of S tile slots in shared memory and has two or three roles:
//   producer  (lane 0 of warp 0) claims tiles by ticket, so that every CTA's tiles
//             ascend and every tile a CTA waits for belongs to a CTA that is running
//             (it claimed it); each tile goes into the next free slot by one bulk copy;
//   data warps (NDW of them) each classify one warp sub-tile of 32 x IPT keys with
//             ballots and compact it in place: less keys to the front of the warp's
//             region, >= keys to its back. The last data warp to finish a tile either
//             takes the tile's output ranges at once (reservation form) or publishes the
//             tile's less count for the look-back (ordered form). Once the tile's global
//             offsets are known, each warp writes its two runs out with 128-bit stores
//             and the slot returns to the producer;
//   look-back warps (ordered form only: NLB of them; the CTA's i-th tile goes to warp
//             i mod NLB) find each
//             tile's prefix, the less keys of all earlier tiles. The prefix of the CTA's
//             tile t_i is its own inclusive count after t_(i-1) plus the aggregates of
//             the tiles strictly between t_(i-1) and t_i, all claimed by other CTAs.
//             Those aggregates come from counting alone, never from another look-back,
//             so no chain of look-backs forms across CTAs; within the CTA, consecutive
//             tiles sum their disjoint ranges at once and only add up in order. The tile
//             that holds the array's last keys learns the total less count and places
//             the key.
// Forms. Ordered (NLB > 0): the tiles' runs appear in the output in tile order, so the
// result depends on the input alone, but a tile's offsets wait for the slowest of the
// tiles claimed before it. Reservation (NLB == 0): the last data warp of a tile adds the
// tile's (>= count << 32 | less count) to one 64-bit counter; the value before its add
// gives the tile's less run its place after the less keys already placed and its >= run
// its place before the >= keys already placed, from the right end. No tile waits for
// another; the order of the tiles' runs within each side follows the order in which
// tiles finished. Only the key's index and the contents of the two sides are defined for
// a partition (the order inside each side is not the paper's in either form), and both
// forms give those exactly. The tile whose range reaches the last key places the key.
// A slot is busy from its copy to its write-out, so the ring holds the keys in flight
// from HBM and the keys that wait for their offsets in the same bytes. Every wait is
// bounded by the tuned time limit; on a timeout the kernel records KSORT_ERR_TIMEOUT,
// stops every CTA of the call and returns.
#pragma once

#include "ksort_device.cuh"

namespace ksort {
namespace dev {

// One compiled configuration: NDW data warps of IPT keys per lane (a tile is NDW * 32
// * IPT keys), S slots, MINB CTAs per SM, look-back windows of 32 * PER descriptors, NLB
// look-back warps (0: the reservation form), and at most DEPTH tiles of a CTA loading or
// waiting to be compacted (more bytes in flight than the memory system needs only queue
// up in it; the other slots hold compacted tiles until they are written out).
template <typename K, int NDW_, int IPT_, int S_, int MINB_, int PER_, int NLB_, int DEPTH_,
          bool RESV_ = false>
struct RingCfg {
  static constexpr int NDW = NDW_, IPT = IPT_, S = S_, MINB = MINB_, PER = PER_, NLB = NLB_;
  // RESV: the NLB role warps take the tiles' output ranges by reservation (one 64-bit
  // atomic add per tile, the role warps taking tiles in turn) instead of by look-back, so
  // the data warps never wait on a global round trip
  static constexpr bool RESV = RESV_;
  static_assert(!RESV_ || NLB_ > 0, "reservation by role warps needs role warps");
  static constexpr int DEPTH = DEPTH_ < S_ ? DEPTH_ : S_;
  static constexpr int WT = 32 * IPT;    // keys of a warp sub-tile
  static constexpr int TILE = NDW * WT;  // keys of a tile
  static constexpr int NT = (NDW + 1 + NLB) * 32;  // producer, look-back, data warps
  static constexpr int R = S + 1;            // tile-index ring (see part_ring_kernel)
  // a slot: the tile, then room for the 16 bytes copy_out_v may read past a run
  static constexpr size_t SLOT = (size_t)TILE * sizeof(K) + 128;
  static constexpr size_t SMEM = (size_t)S * SLOT;
  static_assert(TILE < 65536, "tile counts are packed in 16 bits");
  static_assert((TILE * sizeof(K)) % 128 == 0, "slots stay 128-byte aligned");
  static_assert(S >= 2, "a ring needs two slots");
  // a look-back warp waits for slot s's tiles in order only if it takes every one
  static_assert(NLB >= 0 && (NLB == 0 || S % NLB == 0), "look-back warps must divide the slots");
};

template <int NDW, int S, int R>
struct RingShared {
  unsigned long long full[S];     // slot holds its tile's keys (copy landed)
  unsigned long long empty[S];    // every data warp has written its share out
  unsigned long long counted[S];  // every data warp has compacted its share
  unsigned long long ready[S];    // the tile's global offsets are in lbase / gbase
  long long tix[R];               // tile of the CTA's i-th claim at [i % R]; -1: none left
  unsigned cnt[S][NDW];           // per data warp: (valid keys << 16) | less keys
  unsigned acc[S];                // (data warps done << 20) + less keys of the tile
  int lbase[S][NDW];              // global index of each data warp's first less key
  int gbase[S][NDW];              // global index of each data warp's first >= key
  int stop;                       // nonzero: leave (an error here or in another CTA)
  int end_at;                     // ring index of the end mark (no tiles from there on)
  // (i << 32) | inclusive less count of the CTA's tile i, the last one the look-back
  // warps have added up (i = 2^32 - 1 before the first)
  unsigned long long chain;
};

// Where the ring's waits learn that they must stop: this CTA's flag, and the call's
// generation recorded in Control::ring_abort by a CTA that met an error.
struct RingStop {
  const volatile int *cta;
  const unsigned *call;
  unsigned epoch;
  __device__ __forceinline__ bool now() const {
    return *cta != 0 || ld_relaxed(call) == epoch;
  }
};
// The same for a sort: this CTA's flag, and the sort's abort flag (Control::abort, which
// the seed kernel clears).
struct SortStop {
  const volatile int *cta;
  const unsigned *call;
  __device__ __forceinline__ bool now() const {
    return *cta != 0 || ld_relaxed(call) != 0u;
  }
};

// Waits, with the whole warp, for phase `parity` of `bar`: 0 once it has completed, 1
// after limit_ns, 2 once the CTA or the call stops, 3 once ring index `i` reaches
// *end_at (when end_at is given: the tile will never come). Every lane takes the barrier
// itself (so its later reads see what the arriving threads wrote) with the potentially
// blocking try_wait: the hardware suspends the thread until the phase completes or a
// time limit passes, so a waiting warp takes almost no issue slots from the working
// ones. Waits that only a phase completion ends take a suspend-time hint of
// kRingSleepNs; waits that an end mark may end instead (end_at given) take none, since
// the end mark arrives on no barrier and must be seen by polling. The checks run on every
// return, so no wait depends on the hint being honoured; a stop is seen within a few
// hints. The decision to leave is lane 0's, broadcast, so the warp never splits.
// (Waking such a waiter by completing its barrier's phase at the end mark is not safe:
// the arrival can complete the phase after the one that the same warp has yet to see,
// and a parity wait cannot tell the two apart.)
constexpr unsigned kRingSleepNs = 20000;
template <typename Stop>
__device__ __forceinline__ int ring_wait_warp(unsigned long long *bar, unsigned parity,
                                              unsigned long long limit_ns, const Stop &st,
                                              const volatile int *end_at = nullptr, int i = 0) {
  unsigned long long t0 = 0;
  for (unsigned k = 0;; ++k) {
    const bool done = end_at ? mbar_try_wait(bar, parity)
                             : mbar_try_wait_sleep(bar, parity, kRingSleepNs);
    if (__all_sync(kFull, done)) return 0;
    int r = 0;
    if ((threadIdx.x & 31) == 0) {
      if (end_at && i >= *end_at) r = 3;
      else if (*st.cta) r = 2;
      else if ((k & 7u) == 7u) {
        const unsigned long long now = globaltimer();
        if (t0 == 0) t0 = now;
        else if (now - t0 > limit_ns) r = 1;
        if (!r && st.now()) r = 2;
      }
    }
    r = __shfl_sync(kFull, r, 0);
    if (r) return r;
  }
}

// The same for one thread (the producer lane).
template <typename Stop>
__device__ __forceinline__ int ring_wait_one(unsigned long long *bar, unsigned parity,
                                             unsigned long long limit_ns, const Stop &st) {
  unsigned long long t0 = 0;
  for (unsigned k = 0;; ++k) {
    if (mbar_try_wait_sleep(bar, parity, kRingSleepNs)) return 0;
    if (*st.cta) return 2;
    if ((k & 7u) == 7u) {
      const unsigned long long now = globaltimer();
      if (t0 == 0) t0 = now;
      else if (now - t0 > limit_ns) return 1;
      if (st.now()) return 2;
    }
  }
}

// Orders this thread's generic-proxy accesses to shared memory before later async-proxy
// (bulk copy) accesses to it; unlike the unscoped fence it does not wait for the thread's
// global stores.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Records a device error and stops every CTA of the call, this one first.
__device__ __forceinline__ void ring_fail(Control *ctl, volatile int *stop, unsigned epoch,
                                          unsigned code, unsigned long long info) {
  *stop = 1;
  raise_error(ctl, code, info);
  atomicExch(&ctl->ring_abort, epoch);
}

// Sum of the aggregates (less counts) published for tiles lo < u < hi, by one warp:
// windows of 32 * PER descriptors, read at once and lane-strided, so that a window
// costs one round trip to L2. A descriptor not yet published is polled alone until it
// is. Returns 0 with *S_out set, 1 after limit_ns, 2 once the call stops.
template <int PER>
__device__ __forceinline__ int ring_between(const unsigned long long *lb, long long lo,
                                            long long hi, unsigned epoch,
                                            unsigned long long limit_ns, const RingStop &stp,
                                            unsigned long long *S_out, unsigned *windows) {
  const int lane = threadIdx.x & 31;
  const unsigned long long none = (unsigned long long)epoch << 32;  // present, value 0
  unsigned long long S = 0, t0 = 0;
  for (long long pos = hi - 1; pos > lo; pos -= 32 * PER) {
    unsigned long long d[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const long long idx = pos - (j * 32 + lane);
      d[j] = idx > lo ? ld_relaxed(&lb[idx]) : none;
    }
    ++*windows;
    while (true) {
      bool miss = false;
#pragma unroll
      for (int j = 0; j < PER; ++j) miss |= (unsigned)(d[j] >> 32) != epoch;
      if (!__any_sync(kFull, miss)) break;
      int st = 0;
      if (lane == 0) {
        const unsigned long long now = globaltimer();
        if (t0 == 0) t0 = now;
        else if (now - t0 > limit_ns) st = 1;
        if (!st && stp.now()) st = 2;
      }
      st = __shfl_sync(kFull, st, 0);
      if (st) return st;
      __nanosleep(64);
#pragma unroll
      for (int j = 0; j < PER; ++j)
        if ((unsigned)(d[j] >> 32) != epoch) d[j] = ld_relaxed(&lb[pos - (j * 32 + lane)]);
    }
    unsigned sum = 0;
#pragma unroll
    for (int j = 0; j < PER; ++j) sum += (unsigned)(d[j] & 0x7fffffffull);
    S += __reduce_add_sync(kFull, sum);
  }
  *S_out = S;
  return 0;
}

// Step 3 on one warp sub-tile, in place in its region `reg` of a slot: lane l
// classifies the keys at positions j * 32 + l (positions [a, b) are the array's, the rest
// are skipped), then writes them back, less keys from the front in input order, >= keys
// from the back in reverse input order. Positions come from one ballot per key slot.
// Every key is in registers before the first write, so the region can be overwritten.
template <typename K, int IPT, bool FULL>
__device__ __forceinline__ void ring_compact(K *reg, K key, int a, int b, unsigned *L_out,
                                             unsigned *G_out) {
  constexpr int WT = 32 * IPT;
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  K x[IPT];
#pragma unroll
  for (int j = 0; j < IPT; ++j) x[j] = reg[j * 32 + lane];
  __syncwarp();
  unsigned L = 0, G = 0;
#pragma unroll
  for (int j = 0; j < IPT; ++j) {
    const bool left = goes_left(key, x[j]);
    if constexpr (FULL) {
      const unsigned gm = __ballot_sync(kFull, !left);
      const unsigned pg = __popc(gm & lt);
      const int idx = left ? (int)(L + (unsigned)lane - pg) : WT - 1 - (int)(G + pg);
      reg[idx] = x[j];
      const unsigned ng = __popc(gm);
      G += ng;
      L += 32u - ng;
    } else {
      const int e = j * 32 + lane;
      const bool valid = e >= a && e < b;
      const unsigned gm = __ballot_sync(kFull, valid && !left);
      const unsigned lm = __ballot_sync(kFull, valid && left);
      if (valid) {
        const int idx = left ? (int)(L + __popc(lm & lt)) : WT - 1 - (int)(G + __popc(gm & lt));
        reg[idx] = x[j];
      }
      L += __popc(lm);
      G += __popc(gm);
    }
  }
  *L_out = L;
  *G_out = G;
}

// One partition of buffer 0's [0, total) into buffer 1 (p.scratch); *p.key_index
// receives the key's index. Uses p.lb (one descriptor per tile, ordered form) and, in
// Control, the ticket counter part_ticket, the reservation counter ring_resv and the
// count ring_done of CTAs finished (all 0 at the start of a call: the last CTA to finish
// sets them back and makes this call's generation, the workspace's next one, current),
// and ring_abort.
// Tiles are anchored at the 16-byte boundary at or below element 1 (tile_base), so
// every bulk copy starts aligned; it covers whole 16-byte chunks of the array.
// (In the ordered form, fixed first tiles would save claims, but then a CTA's later
// tiles would wait for the first tiles of CTAs with higher indices, which another kernel
// on the GPU can keep from starting; the reservation forms have no such wait and take
// their first DEPTH tiles fixed.)
template <typename K, int NDW, int IPT, int S, int MINB, int PER, int NLB, int DEPTH_,
          bool RESV = false>
__global__ void __launch_bounds__((NDW + 1 + NLB) * 32, MINB) part_ring_kernel(SortParams p) {
  using C = RingCfg<K, NDW, IPT, S, MINB, PER, NLB, DEPTH_, RESV>;
  constexpr int DEPTH = C::DEPTH;
  constexpr int WT = C::WT, TILE = C::TILE, R = C::R;
  constexpr int VEC = Vec<K>::N;
  extern __shared__ __align__(128) unsigned char ring_smem[];
  __shared__ RingShared<NDW, S, R> sh;
  auto slot = [&](int s) { return reinterpret_cast<K *>(ring_smem + (size_t)s * C::SLOT); };

  Control *const ctl = p.ctl;
  grid_dep_wait();    // the previous launch in the stream is complete
  grid_dep_launch();  // the next one may start launching as CTAs leave
  unsigned epoch = *reinterpret_cast<volatile unsigned *>(&ctl->epoch) + 1u;
  if (epoch == 0u || epoch >= kMaxEpoch) epoch = 1u;
  const K *const src = static_cast<const K *>(p.keys);
  K *const dst = static_cast<K *>(p.scratch);
  const long long n = p.total;
  const long long base = tile_base(src, 0);
  const long long tiles = (n - base + TILE - 1) / TILE;
  const unsigned long long limit = p.spin_limit_ns;
  volatile int *const stop = &sh.stop;
  const RingStop stp{stop, &ctl->ring_abort, epoch};
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const K key = __ldcg(src);  // Step 1: the first element is the key
  // First tiles: in the reservation forms no tile waits for another, so CTA b takes
  // tiles b, b + G, ..., b + (DEPTH - 1) G (G CTAs) without a claim, and its first DEPTH
  // copies leave at once instead of one per claim's round trip; later claims count from
  // DEPTH G. The ordered form's tiles wait for their predecessors, so there every tile
  // is claimed, in the order CTAs run.
  constexpr bool kStaticFirst = NLB == 0 || RESV;
  const unsigned long long t_first =
      kStaticFirst ? (unsigned long long)DEPTH * gridDim.x : 0ull;
  unsigned long long tk = 0;
  if (threadIdx.x == 0)
    tk = kStaticFirst ? (unsigned long long)blockIdx.x : atomicAdd(&ctl->part_ticket, 1ull);

  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < S; ++s) {
      mbar_init(&sh.full[s], 1);
      mbar_init(&sh.empty[s], NDW);
      mbar_init(&sh.counted[s], NDW);
      mbar_init(&sh.ready[s], 1);
      sh.acc[s] = 0;
    }
    sh.stop = 0;
    sh.end_at = 0x7fffffff;
    sh.chain = 0xffffffff00000000ull;  // before tile 0: inclusive count 0
    fence_mbar_init();
  }
  __syncthreads();

  // ring index of the last copy or end mark put in each slot (producer lane)
  int last_use[S];
#pragma unroll
  for (int s = 0; s < S; ++s) last_use[s] = -1;

  if (warp == 0) {
    // ---------------------------------------------------------------- producer
    if (lane == 0) {
      for (int i = 0;; ++i) {
        const int s = i % S;
        if (i >= S) {  // the slot's previous tile must have been written out
          const int st = ring_wait_one(&sh.empty[s], (unsigned)((i / S) - 1) & 1u, limit, stp);
          if (st) {
            if (st == 1) ring_fail(ctl, stop, epoch, kDevTimeout, 0xA00000000ull | (unsigned)i);
            break;
          }
        }
        if (DEPTH < S && i >= DEPTH) {  // tile i - DEPTH must have been compacted
          const int j = i - DEPTH;
          unsigned long long *done = NLB > 0 ? &sh.counted[j % S] : &sh.ready[j % S];
          const int st = ring_wait_one(done, (unsigned)(j / S) & 1u, limit, stp);
          if (st) {
            if (st == 1) ring_fail(ctl, stop, epoch, kDevTimeout, 0x1200000000ull | (unsigned)i);
            break;
          }
        }
#pragma unroll
        for (int u = 0; u < S; ++u)
          if (u == s) last_use[u] = i;
        if (tk >= (unsigned long long)tiles || *stop) {  // no tiles left: end mark
          sh.tix[i % R] = -1;
          *reinterpret_cast<volatile int *>(&sh.end_at) = i;
          mbar_arrive(&sh.full[s]);
          break;
        }
        const long long t = (long long)tk;
        sh.tix[i % R] = t;
        const long long lo = base + t * TILE;
        const int vhi = (int)(n - lo < TILE ? n - lo : TILE);
        const unsigned bytes = (unsigned)((vhi + VEC - 1) / VEC * VEC) * (unsigned)sizeof(K);
        mbar_expect_tx(&sh.full[s], bytes);
        bulk_g2s(slot(s), src + lo, bytes, &sh.full[s]);
        trace_mark(p, (unsigned long long)t, 0);  // copy issued
        if (p.trace && (unsigned long long)t < (unsigned long long)p.trace_cap)
          p.trace[t * kTraceWords + 7] = blockIdx.x | ((unsigned long long)i << 20) |
                                         ((unsigned long long)epoch << 40);
        if (kStaticFirst && i + 1 < DEPTH)
          tk = (unsigned long long)blockIdx.x + (unsigned long long)(i + 1) * gridDim.x;
        else
          tk = t_first + atomicAdd(&ctl->part_ticket, 1ull);  // the next claim overlaps this copy
      }
    }
    __syncwarp();
  } else if (NLB > 0 && warp <= NLB && RESV) {
    // ---------------------------------------------------------------- reservation
    if constexpr (RESV) {
    volatile int *const end_at = &sh.end_at;
    for (int i = warp - 1;; i += NLB) {
      __syncwarp();  // one decision for the whole warp (see the look-back loop)
      if (__any_sync(kFull, i >= *end_at)) break;
      const int s = i % S;
      int st = ring_wait_warp(&sh.counted[s], (unsigned)(i / S) & 1u, limit, stp, end_at, i);
      if (st) {
        if (st == 1 && lane == 0) ring_fail(ctl, stop, epoch, kDevTimeout, 0x1300000000ull | (unsigned)i);
        break;
      }
      const long long t = sh.tix[i % R];
      if (t < 0) break;
      // the data warps' counts: exclusive prefixes of (less, >=) over the warps
      const unsigned c = lane < NDW ? sh.cnt[s][lane] : 0u;
      const unsigned Lw = c & 0xffffu, Gw = (c >> 16) - Lw;
      const unsigned v = Lw | (Gw << 16);
      unsigned inc = v;
#pragma unroll
      for (int d = 1; d < NDW; d <<= 1) {
        const unsigned u = __shfl_up_sync(kFull, inc, d);
        if (lane >= d) inc += u;
      }
      const unsigned tot = __shfl_sync(kFull, inc, NDW - 1);
      const unsigned ex = inc - v;
      const long long A = tot & 0xffffu, GT = tot >> 16;
      // the tile's ranges at once: the (>=, less) keys of the tiles that reserved before
      unsigned long long pre = 0;
      if (lane == 0) pre = atomicAdd(&ctl->ring_resv, ((unsigned long long)GT << 32) | (unsigned long long)A);
      pre = __shfl_sync(kFull, pre, 0);
      const long long PL = (long long)(pre & 0xffffffffull), PG = (long long)(pre >> 32);
      bool ok = PL + PG + A + GT <= n - 1;
      if (lane < NDW) {
        const long long lb = PL + (long long)(ex & 0xffffu);
        const long long gb = n - PG - GT + (long long)(ex >> 16);
        ok = ok && lb >= 0 && lb + Lw <= n && gb >= 1 && gb + Gw <= n;
        sh.lbase[s][lane] = (int)lb;
        sh.gbase[s][lane] = (int)gb;
      }
      if (!__all_sync(kFull, ok)) {  // never released for writing
        if (lane == 0) ring_fail(ctl, stop, epoch, kDevInternal, 0x1400000000ull | (unsigned)t);
        break;
      }
      if (lane == 0) {
        if (PL + PG + A + GT == n - 1) {  // every key placed: Step 4
          dst[PL + A] = key;
          if (p.key_index) *p.key_index = PL + A;
        }
        trace_mark(p, (unsigned long long)t, 3);  // offsets known
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&sh.ready[s]);
    }
    }
  } else if (NLB > 0 && warp <= NLB) {
    // ---------------------------------------------------------------- look-back
    if constexpr (NLB > 0 && !RESV) {
    volatile int *const end_at = &sh.end_at;
    volatile unsigned long long *const chain = &sh.chain;
    unsigned windows = 0;
    for (int i = warp - 1;; i += NLB) {
      // One decision for the whole warp: the lanes read end_at at different times (lane 0
      // may still be arriving on the last tile's barrier), and a warp split here would
      // wait in the next warp-wide vote for lanes that have left.
      __syncwarp();
      if (__any_sync(kFull, i >= *end_at)) break;
      const int s = i % S;
      // the tile's counts (leaves at the end mark: the tile will never come)
      int st = ring_wait_warp(&sh.counted[s], (unsigned)(i / S) & 1u, limit, stp, end_at, i);
      if (st) {
        if (st == 1 && lane == 0) ring_fail(ctl, stop, epoch, kDevTimeout, 0xB00000000ull | (unsigned)i);
        break;
      }
      const long long t = sh.tix[i % R];
      if (t < 0) break;
      const long long t_prev = i == 0 ? -1 : sh.tix[(i - 1) % R];
      if (lane == 0) trace_mark(p, (unsigned long long)t, 5);  // look-back starts
      // the data warps' counts: exclusive prefixes of (less, >=) over the warps
      const unsigned c = lane < NDW ? sh.cnt[s][lane] : 0u;
      const unsigned Lw = c & 0xffffu, Gw = (c >> 16) - Lw;
      const unsigned v = Lw | (Gw << 16);
      unsigned inc = v;
#pragma unroll
      for (int d = 1; d < NDW; d <<= 1) {
        const unsigned u = __shfl_up_sync(kFull, inc, d);
        if (lane >= d) inc += u;
      }
      const unsigned tot = __shfl_sync(kFull, inc, NDW - 1);
      const unsigned ex = inc - v;
      const long long A = tot & 0xffffu, GT = tot >> 16;
      unsigned long long Sb = 0;
      const int bs = ring_between<PER>(p.lb, t_prev, t, epoch, limit, stp, &Sb, &windows);
      if (bs) {
        if (bs == 1 && lane == 0) ring_fail(ctl, stop, epoch, kDevTimeout, 0xC00000000ull | (unsigned)t);
        break;
      }
      if (lane == 0) trace_mark(p, (unsigned long long)t, 6);  // between-sum done
      // the inclusive count of the CTA's previous tile, from the warp that added it up
      unsigned long long prev = 0;
      if (lane == 0) {
        const unsigned long long t0 = globaltimer();
        for (unsigned k = 0;; ++k) {
          const unsigned long long cv = *chain;
          if ((unsigned)(cv >> 32) == (unsigned)(i - 1)) {
            prev = cv & 0xffffffffull;
            break;
          }
          if ((k & 63u) == 63u) {
            if (stp.now()) { st = 2; break; }
            if (globaltimer() - t0 > limit) { st = 1; break; }
          }
          __nanosleep(32);
        }
      }
      st = __shfl_sync(kFull, st, 0);
      if (st) {
        if (st == 1 && lane == 0) ring_fail(ctl, stop, epoch, kDevTimeout, 0x1000000000ull | (unsigned)i);
        break;
      }
      prev = __shfl_sync(kFull, prev, 0);
      const long long E = (long long)(prev + Sb);  // less keys of all earlier tiles
      if (lane == 0) *chain = ((unsigned long long)(unsigned)i << 32) | (unsigned long long)(E + A);
      const long long lo = base + t * TILE;
      const long long PV = t == 0 ? 0 : lo - 1;    // classified keys of all earlier tiles
      const long long PG = PV - E;                 // of which >= key
      bool ok = PG >= 0 && E + A <= n - 1;
      if (lane < NDW) {
        const long long lb = E + (long long)(ex & 0xffffu);
        const long long gb = n - PG - GT + (long long)(ex >> 16);
        ok = ok && lb >= 0 && lb + Lw <= n && gb >= 1 && gb + Gw <= n;
        sh.lbase[s][lane] = (int)lb;
        sh.gbase[s][lane] = (int)gb;
      }
      if (!__all_sync(kFull, ok)) {
        if (lane == 0) ring_fail(ctl, stop, epoch, kDevInternal, 0xD00000000ull | (unsigned)t);
        break;
      }
      if (lane == 0) trace_mark(p, (unsigned long long)t, 3);  // offsets known
      if (t == tiles - 1 && lane == 0) {  // Step 4: the key at #{x < key}
        dst[E + A] = key;
        if (p.key_index) *p.key_index = E + A;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&sh.ready[s]);
    }
    if (lane == 0 && windows) atomicAdd(&ctl->lookback_steps, (unsigned long long)windows);
    }
  } else {
    // ---------------------------------------------------------------- data warps
    const int dw = warp - 1 - NLB;
    // writes out this warp's two runs of the CTA's j-th tile (its offsets are known),
    // then hands the warp's share of the slot back to the producer
    auto write_tile = [&](int j) {
      const int s = j % S;
      if (dw == 0 && lane == 0 && p.trace)
        trace_mark(p, (unsigned long long)sh.tix[j % R], 4);  // written out (first warp)
      const unsigned c = sh.cnt[s][dw];
      const unsigned L = c & 0xffffu, G = (c >> 16) - L;
      const K *reg = slot(s) + dw * WT;
      copy_out_v<K, 32>(reg, dst + sh.lbase[s][dw], L, lane);
      copy_out_v<K, 32>(reg + WT - G, dst + sh.gbase[s][dw], G, lane);
      fence_proxy_async_smem();  // the slot's next keys arrive by a bulk copy
      __syncwarp();
      if (lane == 0) mbar_arrive(&sh.empty[s]);
    };
    int wnext = 0;  // next of the CTA's tiles this warp writes out
    int i = 0;
    bool failed = false;
    for (;; ++i) {
      const int s = i % S;
      // slot s still holds tile i - S: write this warp's share of it out first
      while (wnext <= i - S) {
        const int st = ring_wait_warp(&sh.ready[wnext % S], (unsigned)(wnext / S) & 1u, limit, stp);
        if (st) {
          if (st == 1 && lane == 0) ring_fail(ctl, stop, epoch, kDevTimeout, 0xE00000000ull | (unsigned)wnext);
          failed = true;
          break;
        }
        write_tile(wnext++);
      }
      if (failed) break;
      const int st = ring_wait_warp(&sh.full[s], (unsigned)(i / S) & 1u, limit, stp);
      if (st) {
        if (st == 1 && lane == 0) ring_fail(ctl, stop, epoch, kDevTimeout, 0xF00000000ull | (unsigned)i);
        failed = true;
        break;
      }
      const long long t = sh.tix[i % R];
      if (t < 0) {  // no tiles left: let the look-back warp see the end mark
        __syncwarp();
        if (lane == 0) mbar_arrive(&sh.counted[s]);
        break;
      }
      if (dw == 0 && lane == 0) trace_mark(p, (unsigned long long)t, 1);  // keys landed
      const long long lo = base + t * TILE;
      const int vlo = (int)(1 - lo > 0 ? 1 - lo : 0);
      const int vhi = (int)(n - lo < TILE ? n - lo : TILE);
      const int e0 = dw * WT;
      const int a = min(WT, max(0, vlo - e0)), b = min(WT, max(0, vhi - e0));
      K *reg = slot(s) + e0;
      unsigned L = 0, G = 0;
      if (a == 0 && b == WT) ring_compact<K, IPT, true>(reg, key, a, b, &L, &G);
      else ring_compact<K, IPT, false>(reg, key, a, b, &L, &G);
      __syncwarp();
      if (lane == 0) {
        sh.cnt[s][dw] = ((L + G) << 16) | L;
        // the counts before the tile's completion count (the reservation forms publish
        // them by the arrival on `counted`, which orders them itself)
        if constexpr (!RESV) __threadfence_block();
        const unsigned old = RESV ? 0u : atomicAdd(&sh.acc[s], (1u << 20) + L);
        if (!RESV && (old >> 20) == (unsigned)NDW - 1u) {  // the last warp of the tile
          __threadfence_block();
          sh.acc[s] = 0u;
          if constexpr (NLB > 0) {  // ordered form: publish the tile's aggregate
            st_relaxed(&p.lb[t], lb_pack(epoch, false, (old & 0xfffffu) + L));
            trace_mark(p, (unsigned long long)t, 2);  // aggregate published
          } else {
            // reservation form: the tile's runs take their places now
            unsigned Lt = 0, Gt = 0;
#pragma unroll
            for (int w = 0; w < NDW; ++w) {
              const unsigned cw = sh.cnt[s][w];
              const unsigned lw = cw & 0xffffu, gw = (cw >> 16) - lw;
              sh.lbase[s][w] = (int)Lt;  // offsets within the tile, for now
              sh.gbase[s][w] = (int)Gt;
              Lt += lw;
              Gt += gw;
            }
            const unsigned long long pre =
                atomicAdd(&ctl->ring_resv, ((unsigned long long)Gt << 32) | Lt);
            const long long PL = (long long)(pre & 0xffffffffull), PG = (long long)(pre >> 32);
            const bool ok = PL + PG + Lt + Gt <= n - 1;
#pragma unroll
            for (int w = 0; w < NDW; ++w) {
              sh.lbase[s][w] = (int)(PL + sh.lbase[s][w]);
              sh.gbase[s][w] = (int)(n - PG - Gt + sh.gbase[s][w]);
            }
            if (!ok) {  // never released for writing: the data warps leave on the stop
              ring_fail(ctl, stop, epoch, kDevInternal, 0x1100000000ull | (unsigned)t);
            } else {
              if (PL + PG + Lt + Gt == n - 1) {  // every key placed: Step 4
                dst[PL + Lt] = key;
                if (p.key_index) *p.key_index = PL + Lt;
              }
              trace_mark(p, (unsigned long long)t, 3);  // offsets known
              mbar_arrive(&sh.ready[s]);
            }
          }
        }
        if constexpr (NLB > 0) mbar_arrive(&sh.counted[s]);
      }
      // write out every earlier tile whose offsets are already known
      while (wnext <= i &&
             __all_sync(kFull, mbar_test(&sh.ready[wnext % S], (unsigned)(wnext / S) & 1u)))
        write_tile(wnext++);
    }
    if (!failed) {
      while (wnext < i) {
        const int st = ring_wait_warp(&sh.ready[wnext % S], (unsigned)(wnext / S) & 1u, limit, stp);
        if (st) {
          if (st == 1 && lane == 0) ring_fail(ctl, stop, epoch, kDevTimeout, 0xE00000000ull | (unsigned)wnext);
          break;
        }
        write_tile(wnext++);
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // copies still in flight (after a stop) land before the CTA leaves; bounded
    const unsigned long long t0 = globaltimer();
#pragma unroll
    for (int s = 0; s < S; ++s)
      if (last_use[s] >= 0)
        while (!mbar_test(&sh.full[s], (unsigned)(last_use[s] / S) & 1u) &&
               globaltimer() - t0 < limit)
          __nanosleep(128);
    // The last CTA to finish knows that every CTA has read the generation and that no
    // claim or reservation is left: it resets the counters for the next call and makes
    // this generation current.
    __threadfence();
    if (atomicAdd(&ctl->ring_done, 1u) == gridDim.x - 1u) {
      ctl->ring_done = 0u;
      ctl->part_ticket = 0ull;
      ctl->ring_resv = 0ull;
      ctl->epoch = epoch;
    }
  }
}

}  // namespace dev
}  // namespace ksort
