// Device code of libksort: K-sort (arxiv 1107.3622, Section 1.1) on one GPU.
//
//   Steps 1-4 (partition of a sub-array around its first element) run as tile passes
//   of a single-pass partition with decoupled look-back; Steps 5-6 (the recursion)
//   run as a persistent device work queue; sub-arrays at or below a cutoff are
//   finished inside shared memory by the same first-element key rule.
//
// Element classification is Step 3's: x goes right of the key when key <= x, left
// otherwise. Each pass is out of place between two buffers; the key index and the
// contents of the two sides are those of Steps 1-4, the order inside each side is the
// tile order documented at tile_kernel.
//
// Kernels of a sort, in stream order: seed_kernel (one CTA) starts a generation and
// queues the roots; tile_kernel (phase 1; or its ring and warp-role forms,
// tile_ring_kernel and tile_ws_kernel) runs every tile pass of the sub-arrays above the
// cutoff, queuing sides as sub-arrays complete, until all of them are done;
// small_kernel (phase 2) finishes the queued small sub-arrays in shared memory. The
// wave form runs the upper levels first as wave_count_kernel / wave_scatter_kernel
// pairs, one per level, and hands what remains to tile_kernel with wave_handoff_kernel.
// Single partitions: part_ring_kernel (the default, one launch; ksort_part_ring.cuh),
// part_kernel (one launch), split_count_kernel / split_move_kernel (the wave form's:
// count, then move, no waits between CTAs), exact_*_kernel (the paper's element order),
// and tile_kernel for the fixed-scratch entry point. tile_ring_kernel is in
// ksort_tile_ring.cuh.
#pragma once

#include <cstdint>

#include "ksort_internal.h"

namespace ksort {
namespace dev {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kSmallThreads = 256;  // default small_kernel CTA (512 and 1024 also built)

#ifndef KSORT_LOOKBACK_PER
#define KSORT_LOOKBACK_PER 1
#endif
#ifndef KSORT_PART_LOOKBACK_PER
#define KSORT_PART_LOOKBACK_PER 1  // part_kernel: windows of 32 x this many descriptors
#endif
// tile_kernel CTAs per SM that the register budget is sized for (64 registers a thread)
constexpr int tile_min_blocks(int nt) { return 1024 / nt; }

// ----------------------------------------------------------------------------- PTX
__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may start before the previous kernel in the stream has finished;
// grid_dep_wait() blocks until that kernel has completed and its memory is visible (a
// no-op in a kernel launched without the attribute). grid_dep_launch() lets the next
// such kernel start launching.
__device__ __forceinline__ void grid_dep_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void grid_dep_launch() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned ld_relaxed(const unsigned *p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned long long *p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed(unsigned long long *p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned atom_add_release(unsigned *p, unsigned v) {
  unsigned old;
  asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v)
               : "memory");
  return old;
}
__device__ __forceinline__ void bsync() { __syncthreads(); }

// ----------------------------------------------------------------------------- keys
template <typename K> struct Vec;
template <> struct Vec<float> { using T = float4; static constexpr int N = 4; };
template <> struct Vec<unsigned> { using T = uint4; static constexpr int N = 4; };
template <> struct Vec<double> { using T = double2; static constexpr int N = 2; };

// Step 3: a[p] goes right of the key when key <= a[p]; every other element goes left.
template <typename K>
__device__ __forceinline__ bool goes_left(K key, K x) { return !(key <= x); }

// float64 keys are classified on the integer pipes: this GPU issues FP64 instructions,
// compares included, at a small fraction of the FP32 and integer rates. The IEEE-754
// order of two doubles that are not NaN is the unsigned order of
//     sign ? ~bits : bits | 2^63
// once -0 is read as +0, and `key <= x` is false when either operand is NaN, so the
// result is the same as the floating-point compare for every pair of inputs.
__device__ __forceinline__ unsigned long long f64_order(double v) {
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
  if ((b << 1) == 0ull) b = 0ull;  // -0 == +0
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ bool f64_nan(double v) {
  return ((unsigned long long)__double_as_longlong(v) << 1) > 0xffe0000000000000ull;
}
template <>
__device__ __forceinline__ bool goes_left<double>(double key, double x) {
  return f64_nan(key) | f64_nan(x) | (f64_order(key) > f64_order(x));
}

// NaN test on the key's bits (integer pipes for every type; u32 keys have none).
template <typename K>
__device__ __forceinline__ bool key_is_nan(K) { return false; }
template <>
__device__ __forceinline__ bool key_is_nan<float>(float v) {
  return (__float_as_uint(v) & 0x7fffffffu) > 0x7f800000u;
}
template <>
__device__ __forceinline__ bool key_is_nan<double>(double v) { return f64_nan(v); }

template <typename K>
__device__ __forceinline__ unsigned long long key_bits(K k) {
  unsigned long long b = 0;
  memcpy(&b, &k, sizeof(K));
  return b;
}
template <typename K>
__device__ __forceinline__ K bits_key(unsigned long long b) {
  K k;
  memcpy(&k, &b, sizeof(K));
  return k;
}

// ----------------------------------------------------------------------------- errors
__device__ __forceinline__ void raise_error(Control *ctl, unsigned code, unsigned long long info) {
  if (atomicCAS(&ctl->error, 0u, code) == 0u) atomicExch(&ctl->err_info, info);
  atomicExch(&ctl->abort, 1u);
}

// Every sub-array the kernels record (work items, wave lists) is checked here when it is
// created: inside the caller's buffer and within one partition's size. Records are
// only ever read back, so every range a kernel derives from one (tiles, bulk copies,
// destinations) stays inside the buffers; a violation is reported and not recorded.
// This stands in for a memory checker, which this GPU pool does not offer.
__device__ __forceinline__ bool sub_array_ok(const SortParams &p, long long b, long long e,
                                             unsigned long long where) {
  if (b >= 0 && b < e && e <= p.total && e - b <= kMaxItemKeys) return true;
  raise_error(p.ctl, kDevInternal, 0xF00000000ull | where);
  return false;
}

// ----------------------------------------------------------------------------- tiles
// Tile grid of a sub-array [begin, end) in buffer `buf`: the first classified element
// is begin + 1 (begin holds the key); tiles are anchored at the 16-byte boundary at or
// below it so that whole vectors move with 128-bit accesses.
template <typename K>
__host__ __device__ __forceinline__ long long tile_base(const K *buf, long long begin) {
  const long long first = begin + 1;
  const int mis = (int)((reinterpret_cast<uintptr_t>(buf + first) & 15u) / sizeof(K));
  return first - mis;
}
template <typename K, int TILE>
__host__ __device__ __forceinline__ unsigned tile_count(const K *buf, long long begin,
                                                        long long end) {
  const long long base = tile_base(buf, begin);
  return (unsigned)((end - base + TILE - 1) / TILE);
}

// Look-back descriptor: [63:32] epoch, [31] inclusive-prefix flag, [30:0] value.
// Sort generations are 1 .. 2^31 - 1; zeroed memory (epoch 0) is never valid.
constexpr unsigned kMaxEpoch = 0x80000000u;
__device__ __forceinline__ unsigned long long lb_pack(unsigned epoch, bool inclusive,
                                                       unsigned v) {
  return ((unsigned long long)epoch << 32) | ((unsigned long long)inclusive << 31) |
         (unsigned long long)(v & 0x7fffffffu);
}

// Decoupled look-back (Merrill and Garland, 2016) run by one warp: the less count of
// all tiles before `t`. Many tiles are in flight at once, so the nearest inclusive
// prefix can be a few hundred tiles back: each step reads a window of 32 * kLookbackPer
// descriptors at once, lane-strided so every load instruction reads 32 neighbouring
// descriptors (lane l holds offsets j * 32 + l below `pos`, j < kLookbackPer). A window
// ends the look-back when it holds an inclusive prefix with every nearer descriptor
// present; if the whole window is present, its aggregates are added and the window
// moves down. Otherwise only the nearest missing descriptor is polled (cheap for the
// memory system) until it appears, and the window is read again. Every wait is
// bounded by `limit_ns`. Returns 0 when the prefix was found, 1 on timeout, 2 when the
// call was aborted.
constexpr int kLookbackPer = KSORT_LOOKBACK_PER;
template <int PER = kLookbackPer>
__device__ __forceinline__ int lookback(const unsigned long long *lb, unsigned t, unsigned epoch,
                                        unsigned long long limit_ns, const unsigned *abort_flag,
                                        unsigned long long *E_out,
                                        unsigned long long *steps,
                                        unsigned long long *dbg = nullptr) {
  constexpr int NONE = 32 * PER;
  const int lane = threadIdx.x & 31;
  unsigned long long E = 0;
  long long pos = (long long)t - 1;
  unsigned long long t0 = 0;
  unsigned polls = 0;
  while (true) {
    unsigned long long d[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const long long idx = pos - (j * 32 + lane);
      d[j] = idx >= 0 ? ld_relaxed(&lb[idx]) : lb_pack(epoch, true, 0u);
    }
    int inv = NONE, incl = NONE;  // this lane's nearest missing / inclusive offset
#pragma unroll
    for (int j = PER - 1; j >= 0; --j) {
      const bool ok = (unsigned)(d[j] >> 32) == epoch;
      if (!ok) inv = j * 32 + lane;
      if (ok && ((d[j] >> 31) & 1ull)) incl = j * 32 + lane;
    }
    const int near_inv = __reduce_min_sync(kFull, inv);
    const int near_incl = __reduce_min_sync(kFull, incl);
    ++*steps;
    if (dbg && lane == 0) {
      if (dbg[0] == 0) dbg[0] = globaltimer();  // first window back
      dbg[1] += 1;                               // windows read
    }
    if (near_incl < near_inv || near_inv == NONE) {
      // add every value up to the nearest inclusive one (or the whole window)
      unsigned sum = 0;
#pragma unroll
      for (int j = 0; j < PER; ++j)
        if (j * 32 + lane <= near_incl) sum += (unsigned)(d[j] & 0x7fffffffull);
      E += __reduce_add_sync(kFull, sum);
      if (near_incl < NONE) {
        *E_out = E;
        return 0;
      }
      pos -= NONE;
      continue;
    }
    // poll the nearest missing descriptor alone until it appears (bounded)
    const unsigned long long *wait_on = &lb[pos - near_inv];
    int stop = 0;
    if (lane == 0) {
      unsigned ns = 32;
      while ((unsigned)(ld_relaxed(wait_on) >> 32) != epoch) {
        if (dbg) dbg[2] += 1;  // polls
        if ((++polls & 15u) == 0u) {
          const unsigned long long now = globaltimer();
          if (t0 == 0) t0 = now;
          if (now - t0 > limit_ns) { stop = 1; break; }
          if (ld_relaxed(abort_flag) != 0u) { stop = 2; break; }
        }
        __nanosleep(ns);
        ns = ns < 256 ? ns * 2 : 256;
      }
    }
    stop = __shfl_sync(kFull, stop, 0);
    if (stop) {
      *E_out = 0;
      return stop;
    }
  }
}

// Writes count keys from shared memory so[0..count) to global g[0..count) with NG
// threads (rank r): scalar stores up to g's first 16-byte boundary, then one 128-bit
// store per vector. Every vector is assembled from the two aligned 16-byte chunks of
// shared memory it straddles (all vectors of a call have the same misalignment), so the
// shared-memory reads are whole chunks and do not collide in banks. The reads may touch
// up to 16 bytes past so[count): every buffer passed here carries that much room.
template <typename K, int NG>
__device__ __forceinline__ void copy_out_v(const K *so, K *g, unsigned count, int r) {
  constexpr int VEC = Vec<K>::N;
  using V = typename Vec<K>::T;
  unsigned head = (unsigned)(((16u - (reinterpret_cast<uintptr_t>(g) & 15u)) & 15u) / sizeof(K));
  if (head > count) head = count;
  if (r < (int)head) g[r] = so[r];
  const unsigned nvec = (count - head) / VEC;
  V *gv = reinterpret_cast<V *>(g + head);
  const K *s0 = so + head;
  const unsigned mis = (unsigned)((reinterpret_cast<uintptr_t>(s0) & 15u) / sizeof(K));
  const V *cv = reinterpret_cast<const V *>(s0 - mis);
  for (unsigned v = r; v < nvec; v += NG) {
    const V a = cv[v];
    V q = a;
    if (mis != 0) {
      const V b = cv[v + 1];
      if constexpr (VEC == 4) {
        if (mis == 1) { q.x = a.y; q.y = a.z; q.z = a.w; q.w = b.x; }
        else if (mis == 2) { q.x = a.z; q.y = a.w; q.z = b.x; q.w = b.y; }
        else { q.x = a.w; q.y = b.x; q.z = b.y; q.w = b.z; }
      } else {
        q.x = a.y;
        q.y = b.x;
      }
    }
    gv[v] = q;
  }
  for (unsigned k = head + nvec * VEC + r; k < count; k += NG) g[k] = so[k];
}

// Scatter of one thread's IPT keys into a tile's output (bit j of lessbits / gebits: key
// j goes to the less / >= side), thread by thread: wl0 / wg0 are the output indices of
// the warp's first less / >= key and `excl` packs this thread's exclusive counts within
// the warp (less in the low, >= in the high 16 bits). (A slot-major order, conflict-free
// in shared memory, measured slower: its ballots cost more than the bank conflicts.)
template <typename K, int IPT>
__device__ __forceinline__ void scatter_keys(K *so, const K (&x)[IPT], unsigned lessbits,
                                             unsigned gebits, unsigned wl0, unsigned wg0,
                                             unsigned excl) {
  unsigned rl = wl0 + (excl & 0xffffu), rg = wg0 + (excl >> 16);
#pragma unroll
  for (int j = 0; j < IPT; ++j) {
    if ((lessbits >> j) & 1u) so[rl++] = x[j];
    else if ((gebits >> j) & 1u) so[rg++] = x[j];
  }
}

// Reserved ranges [lbase, lbase + L) and [gbase, gbase + G) inside the sub-array.
__device__ __forceinline__ bool ranges_ok(long long begin, long long end, long long lbase,
                                       unsigned L, long long gbase, unsigned G) {
  return lbase >= begin && lbase + L <= end && gbase >= begin && gbase + G <= end;
}

// Global offsets of the two sides of tile t; false (and an error) if inconsistent.
__device__ __forceinline__ bool tile_dest(long long begin, long long end, long long lo,
                                          unsigned t, unsigned long long E, unsigned L, unsigned G,
                                          long long *lbase, long long *gbase) {
  const long long first = begin + 1;
  const long long PV = t == 0 ? 0 : lo - first;  // classified keys in earlier tiles
  const long long PG = PV - (long long)E;        // of which >= key
  *lbase = begin + (long long)E;
  *gbase = end - PG - (long long)G;
  return *lbase >= begin && *lbase + L <= end && *gbase >= begin && *gbase + G <= end;
}

// ----------------------------------------------------------------------------- smem
// Shared-memory finisher for one small sub-array (m <= cutoff keys) staged in buffer A,
// run by one CTA of 256, 512 or 1024 threads. Its warps apply Steps 1-6: first CTA-wide partitions
// while a segment is larger than block_segment(NT) keys, then one warp per segment (Steps
// 1-4 by ballots from one buffer into the other; Steps 5-6 depth first, the smaller
// side queued for another warp), and sides of at most kLeaf keys become leaves that
// are finished in registers, several per warp (warp_leaf_run). Every key that reaches
// its final index is written there in A; A is copied out at the end.
#ifndef KSORT_LEAF
#define KSORT_LEAF 32  // largest leaf (2 .. 32 keys), for sweeps
#endif
constexpr int kLeaf = KSORT_LEAF;
static_assert(kLeaf >= 2 && kLeaf <= 32, "a leaf fits one warp");
// Queued segments are disjoint; those above kLeaf (or kMarkLeaf) keys number at most
// cutoff / 17 (for leaves of at least 16 keys), and the CTA-wide phase queues at most
// two leaves per partition: 1024 slots suffice for cutoffs up to 16384 keys.
constexpr int kSmallQueue = 1024;
constexpr int kMaxSmallCutoff = 16384;
// Segments above block_segment(NT) keys are partitioned by the whole CTA (a count pass,
// a scan and a scatter pass, three barriers), smaller ones by one warp in a single pass.
// A 256-thread CTA, which serves many items at once, gains from the warp form's single
// pass (7e6 f32 keys, cutoff 4096: 1024 -> 4096 takes the finisher from 0.270 to 0.254
// ms); the larger CTAs, chosen to finish a few items soon, keep their warps busy with
// the CTA form above 1024 keys.
constexpr int kBlockSegmentMin = 1024;
__host__ __device__ constexpr int block_segment(int nt) { return nt == 256 ? 4096 : kBlockSegmentMin; }
constexpr int kBigStack = kMaxSmallCutoff / kBlockSegmentMin + 2;

struct SmallShared {
  unsigned ring[kSmallQueue];         // queued segments: start << 16 | n << 1 | parity
  unsigned big[kBigStack];            // segments for CTA-wide partitions
  unsigned wl[32], wg[32];            // per-warp counts of a CTA-wide partition
  int head, tail, pending, bad, nbig, L;
};

// Steps 1-6 on a warp's worth of leaves (segments of at most 32 keys), one key per
// lane, several leaves side by side. Leaf sides are kept in their order (a stable
// partition), and for a sub-array that small the recursion of Steps 1-6 has a closed
// form. Under the first-element key and the `key <= x` rule with order-keeping sides,
// every key x of a leaf ends at
//     start + #{y in the leaf : y < x} + #{y earlier in the leaf : y == x}:
// the key of a sub-array precedes the keys equal to it (they come after it and go right),
// and each side keeps its order. So each lane counts that index directly, with no
// dependent chain of levels, and keys move once, to their final index.
// The closed form needs the compare to be a total order. A run holding a NaN key runs
// the levels themselves instead: each sub-array's lowest lane is its key, the other
// lanes of its mask go left when !(key <= x) (one ballot), and the masks split until
// every lane is alone; that is exact for any compare.
// Entries of `list` (leaf_pack): start << 12 | first lane << 7 | n << 1 | parity (parity
// 1: the leaf is in B); `used` = lanes the run fills.
template <typename K>
__device__ __forceinline__ void warp_leaf_run(K *A, const K *B, const unsigned *list, int count,
                                              int used) {
  const int lane = threadIdx.x & 31;
  __syncwarp();
  const unsigned ent = lane < count ? list[lane] : 0u;
  const unsigned starts =
      __reduce_or_sync(kFull, lane < count ? (1u << ((ent >> 7) & 31u)) : 0u);
  const bool act = count > 0 && lane < used;
  const unsigned le_mask = lane == 31 ? kFull : ((2u << lane) - 1u);
  const int leaf = act ? __popc(starts & le_mask) - 1 : 0;
  const unsigned e = __shfl_sync(kFull, ent, leaf);
  const int lo = (int)((e >> 7) & 31u);
  const int n = (int)((e >> 1) & 63u);
  const int s0 = (int)(e >> 12);
  const K *src = ((e & 1u) ? B : A) + s0;
  const int me = lane - lo;
  K x = K(0);
  if (act) x = src[me];
  int dst = s0;
  if (__any_sync(kFull, act && key_is_nan(x))) {
    unsigned mask = act ? (((n >= 32) ? kFull : ((1u << n) - 1u)) << lo) : 0u;
    for (int level = 0; level < 32; ++level) {  // a 32-lane sub-array needs at most 31
      const bool big = act && (mask & (mask - 1u)) != 0u;
      if (!__any_sync(kFull, big)) break;
      const int piv = __ffs(mask) - 1;
      const K key = __shfl_sync(kFull, x, piv < 0 ? 0 : piv);  // Step 1
      const bool is_key = lane == piv;
      const bool lf = big && !is_key && goes_left(key, x);  // Step 3
      const unsigned low = __ballot_sync(kFull, lf) & mask;
      if (big) {
        const int Lc = __popc(low);
        if (is_key) {
          dst += Lc;  // Step 4
          mask = 1u << lane;
        } else if (lf) {
          mask = low;
        } else {
          dst += Lc + 1;
          mask &= ~(low | (1u << piv));
        }
      }
    }
  } else if (act) {
    int pos = 0;
#pragma unroll 4
    for (int j = 0; j < n; ++j) {
      const K y = src[j];
      // y < x (y goes left of key x), or y == x and y comes earlier
      pos += (goes_left(x, y) || (j < me && !goes_left(y, x))) ? 1 : 0;
    }
    dst = s0 + pos;
  }
  __syncwarp();  // every lane has read its leaf before any key moves
  if (act) A[dst] = x;
  __syncwarp();
}

__device__ __forceinline__ unsigned seg_pack(int s, int n, int par) {
  return ((unsigned)s << 16) | ((unsigned)n << 1) | (unsigned)par;  // s, n <= 16384
}
// A leaf of a run: start in its buffer, first lane in the run, size (1..32), parity.
__device__ __forceinline__ unsigned leaf_pack(int s, int n, int par, int lane0) {
  return ((unsigned)s << 12) | ((unsigned)lane0 << 7) | ((unsigned)n << 1) | (unsigned)par;
}

// Lane 0 queues a segment.
__device__ __forceinline__ void small_push(SmallShared &q, int s, int n, int par) {
  atomicAdd(&q.pending, 1);
  const int slot = atomicAdd(&q.tail, 1);
  __threadfence_block();
  atomicExch(&q.ring[slot % kSmallQueue], seg_pack(s, n, par));
}

// Lane 0 claims the next queued segment; returns 0 once the CTA's work is done.
__device__ __forceinline__ unsigned small_pop(SmallShared &q) {
  volatile SmallShared &v = q;
  for (unsigned spins = 0;; ++spins) {
    const int h = v.head;
    if (h < v.tail) {
      if (atomicCAS(&q.head, h, h + 1) == h) {
        unsigned e = 0;
        for (unsigned w = 0; (e = atomicExch(&q.ring[h % kSmallQueue], 0u)) == 0u; ++w) {
          if (w > (1u << 24)) {  // the pusher reserved the slot: it cannot stay empty
            q.bad = 1;
            return 0;
          }
        }
        __threadfence_block();
        return e;
      }
    } else if (v.pending == 0 || v.bad) {
      return 0;
    }
    if (spins > (1u << 24)) {
      q.bad = 1;
      return 0;
    }
    __nanosleep(spins < 4 ? 32 : 200);
  }
}

// Steps 1-4 by all warps of the CTA on X[s .. s+n): each warp classifies a contiguous
// run of 32-key chunks twice (count, then scatter after a scan of the warp counts). Same
// layout as warp_partition. Returns L; contains three CTA barriers.
template <typename K, int NT>
__device__ __forceinline__ int block_partition(const K *X, K *Y, int s, int n, K key,
                                               SmallShared &q) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned lt = lanemask_lt();
  const int e = s + n;
  const int nch = (n - 1 + 31) / 32;
  const int per = (nch + NW - 1) / NW;
  const int c0 = w * per, c1 = min(nch, c0 + per);
  unsigned wl = 0, wg = 0;
#pragma unroll 4
  for (int c = c0; c < c1; ++c) {
    const int i = s + 1 + c * 32 + lane;
    const bool v = i < e;
    const bool le = v && goes_left(key, X[i]);
    wl += __popc(__ballot_sync(kFull, le));
    wg += __popc(__ballot_sync(kFull, v && !le));
  }
  if (lane == 0) {
    q.wl[w] = wl;
    q.wg[w] = wg;
  }
  bsync();
  if (w == 0) {
    const unsigned a0 = lane < NW ? q.wl[lane] : 0u, b0 = lane < NW ? q.wg[lane] : 0u;
    unsigned a = a0, b = b0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned ua = __shfl_up_sync(kFull, a, o), ub = __shfl_up_sync(kFull, b, o);
      if (lane >= o) { a += ua; b += ub; }
    }
    if (lane < NW) {
      q.wl[lane] = a - a0;
      q.wg[lane] = b - b0;
    }
    if (lane == 31) q.L = (int)a;
  }
  bsync();
  unsigned rl = q.wl[w], rg = q.wg[w];
#pragma unroll 4
  for (int c = c0; c < c1; ++c) {
    const int i = s + 1 + c * 32 + lane;
    const bool v = i < e;
    const K x = v ? X[i] : K(0);
    const bool le = v && goes_left(key, x);
    const unsigned ml = __ballot_sync(kFull, le), mg = __ballot_sync(kFull, v && !le);
    if (v) Y[le ? s + rl + __popc(ml & lt) : e - 1 - rg - __popc(mg & lt)] = x;
    rl += __popc(ml);
    rg += __popc(mg);
  }
  const int L = q.L;
  bsync();
  return L;
}

// Steps 1-4 by one warp on X[s .. s+n): less keys to Y[s ..] upward, the others to
// Y[s+n-1 ..] downward; returns the number of less keys L (the key's offset).
template <typename K>
__device__ __forceinline__ int warp_partition(const K *X, K *Y, int s, int n, K key) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  const int e = s + n;
  int L = 0, G = 0;
  int i0 = s + 1;
  // groups of four full chunks: every lane has a key, so the >= lanes are the others
  for (; i0 + 128 <= e; i0 += 128) {
    K x[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) x[u] = X[i0 + 32 * u + lane];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const bool l = goes_left(key, x[u]);
      const unsigned ml = __ballot_sync(kFull, l);
      const int rl = __popc(ml & lt);
      Y[l ? s + L + rl : e - 1 - G - (lane - rl)] = x[u];
      const int c = __popc(ml);
      L += c;
      G += 32 - c;
    }
  }
  // the rest one chunk at a time (the same order, so the same layout)
  for (; i0 < e; i0 += 32) {
    const int i = i0 + lane;
    const bool v = i < e;
    const K x = v ? X[i] : K(0);
    const bool l = v && goes_left(key, x);
    const unsigned ml = __ballot_sync(kFull, l), mg = __ballot_sync(kFull, v && !l);
    if (v) Y[l ? s + L + __popc(ml & lt) : e - 1 - G - __popc(mg & lt)] = x;
    L += __popc(ml);
    G += __popc(mg);
  }
  __syncwarp();
  return L;
}

// Sorts A[0..m) (staged keys) with the K-sort rule into out[0..m); B is scratch of at
// least m keys. Run by the whole CTA of NT threads; returns false if a consistency
// check failed.
template <typename K, int NT>
__device__ bool smem_ksort(K *A, K *B, unsigned *leaf_lists, K *__restrict__ out, int m,
                           SmallShared &q, unsigned long long *segments) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned *leaves = leaf_lists + warp * 32;
  for (int i = tid; i < kSmallQueue; i += NT) q.ring[i] = 0u;
  if (tid == 0) {
    q.head = 0;
    q.tail = 0;
    q.pending = 0;
    q.bad = 0;
    q.nbig = 0;
  }
  bsync();
  unsigned long long nseg = 0;

  if (m <= kLeaf) {
    if (warp == 0) {
      if (lane == 0) leaves[0] = leaf_pack(0, m, 0, 0);
      warp_leaf_run(A, B, leaves, 1, m);
    }
    nseg = 1;
  } else {
    // CTA-wide partitions while segments are large (the top levels of the item)
    if (tid == 0) {
      if (m > block_segment(NT)) q.big[q.nbig++] = seg_pack(0, m, 0);
      else small_push(q, 0, m, 0);
    }
    bsync();
    while (q.nbig > 0) {
      const unsigned e = q.big[q.nbig - 1];
      const int s = (int)(e >> 16), n = (int)((e >> 1) & 0x7fffu), par = (int)(e & 1u);
      bsync();
      const K *X = par ? B : A;
      K *Y = par ? A : B;
      const K key = X[s];
      const int L = block_partition<K, NT>(X, Y, s, n, key, q);
      ++nseg;
      const int cp = par ^ 1;
      if (tid == 0) {
        A[s + L] = key;
        --q.nbig;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const int cs = c ? s + L + 1 : s, cn = c ? n - L - 1 : L;
          if (cn > block_segment(NT)) q.big[q.nbig++] = seg_pack(cs, cn, cp);
          else if (cn >= 2) small_push(q, cs, cn, cp);
          else if (cn == 1 && cp) A[cs] = Y[cs];
        }
      }
      bsync();
    }
    // warp-level Steps 1-6 on the queued segments; leaves are gathered per warp into
    // runs of at most 32 keys
    int nleaves = 0, nlanes = 0;
    while (true) {
      unsigned e = 0;
      if (lane == 0) e = small_pop(q);
      e = __shfl_sync(kFull, e, 0);
      if (e == 0u) break;
      int s = (int)(e >> 16), n = (int)((e >> 1) & 0x7fffu), par = (int)(e & 1u);
      while (true) {
        if (n <= kLeaf) {  // a leaf (queued by the CTA-wide phase)
          if (nlanes + n > 32) {
            warp_leaf_run(A, B, leaves, nleaves, nlanes);
            nleaves = nlanes = 0;
          }
          if (lane == 0) leaves[nleaves] = leaf_pack(s, n, par, nlanes);
          ++nleaves;
          nlanes += n;
          break;
        }
        const K *X = par ? B : A;
        K *Y = par ? A : B;
        ++nseg;
        const K key = X[s];  // Step 1
        const int L = warp_partition(X, Y, s, n, key);
        if (lane == 0) A[s + L] = key;  // Step 4: final index
        const int ls = s, ln = L, rs = s + L + 1, rn = n - L - 1, cp = par ^ 1;
        if (cp && ln == 1 && lane == 0) A[ls] = Y[ls];
        if (cp && rn == 1 && lane == 0) A[rs] = Y[rs];
        // Steps 5-6: sides of 2..kLeaf keys become leaves; of the larger sides, the
        // smaller is queued and the warp keeps the other
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const int cs = c ? rs : ls, cn = c ? rn : ln;
          if (cn >= 2 && cn <= kLeaf) {
            if (nlanes + cn > 32) {
              warp_leaf_run(A, B, leaves, nleaves, nlanes);
              nleaves = nlanes = 0;
            }
            if (lane == 0) leaves[nleaves] = leaf_pack(cs, cn, cp, nlanes);
            ++nleaves;
            nlanes += cn;
          }
        }
        const bool bl = ln > kLeaf, br = rn > kLeaf;
        if (bl && br) {
          if (lane == 0) {
            if (ln < rn) small_push(q, ls, ln, cp);
            else small_push(q, rs, rn, cp);
          }
          if (ln < rn) { s = rs; n = rn; } else { s = ls; n = ln; }
          par = cp;
        } else if (bl) {
          s = ls; n = ln; par = cp;
        } else if (br) {
          s = rs; n = rn; par = cp;
        } else {
          break;
        }
      }
      if (lane == 0) {
        __threadfence_block();
        atomicSub(&q.pending, 1);
      }
    }
    if (nleaves) warp_leaf_run(A, B, leaves, nleaves, nlanes);
  }
  bsync();
  copy_out_v<K, NT>(A, out, (unsigned)m, tid);
  if (tid == 0) *segments += nseg;
  return q.bad == 0;
}

// Largest final segment of the marked form (2 .. 32): its closed form costs one compare
// per key of the segment, and segments above it are partitioned by a warp (measured
// best at 20 of 12, 16, 20, 24 and 32).
#ifndef KSORT_MARK_LEAF
#define KSORT_MARK_LEAF 20
#endif
constexpr int kMarkLeaf = KSORT_MARK_LEAF;
static_assert(kMarkLeaf >= 2 && kMarkLeaf <= 32, "a marked segment spans at most two words");

// Marked form of the finisher, for sub-arrays without NaN keys (the closed form of a
// leaf needs a total order). The partitions run as in smem_ksort, but a final segment
// (a key at its index, a one-key side, a leaf of 2..kMarkLeaf keys) is not finished where it
// appears: its first index is marked in the bitmap `seg`, and in `par` when its keys are
// in B. Bit m of `seg` closes the last segment. Once every partition is done, each
// index of the sub-array finds its segment from the marks (a segment spans at most 32
// indices, so the marks around it lie in at most three words), and each key goes
// straight to its final index in `out`: a leaf key by the closed form of warp_leaf_run,
// any other key as it stands. Warps take 32-index windows in turn, so every lane has a
// key whatever the leaf sizes. Nothing in shared memory is written in this pass, so a
// leaf may span windows of two warps. The result equals smem_ksort's.
__device__ __forceinline__ void seg_mark(unsigned *bits, int i) {
  atomicOr(&bits[i >> 5], 1u << (i & 31));
}

// A final side [cs, cs + cn) of 1..kMarkLeaf keys, in B when cp is 1.
__device__ __forceinline__ void mark_final(unsigned *seg, unsigned *par, int cs, int cn, int cp) {
  if (cn < 1) return;
  seg_mark(seg, cs);
  if (cp) seg_mark(par, cs);
}

template <typename K, int NT, typename Pre>
__device__ bool smem_ksort_marked(K *A, K *B, unsigned *seg, unsigned *par,
                                  K *__restrict__ out, int m, SmallShared &q,
                                  unsigned long long *segments, Pre &&pre) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int words = (m >> 5) + 2;
  for (int i = tid; i < kSmallQueue; i += NT) q.ring[i] = 0u;
  for (int i = tid; i < words; i += NT) {
    seg[i] = 0u;
    par[i] = 0u;
  }
  if (tid == 0) {
    q.head = 0;
    q.tail = 0;
    q.pending = 0;
    q.bad = 0;
    q.nbig = 0;
  }
  bsync();
  unsigned long long nseg = m <= kMarkLeaf ? 1 : 0;
  if (tid == 0) {
    seg_mark(seg, m);
    if (m <= kMarkLeaf) mark_final(seg, par, 0, m, 0);
    else if (m > block_segment(NT)) q.big[q.nbig++] = seg_pack(0, m, 0);
    else small_push(q, 0, m, 0);
  }
  bsync();
  // CTA-wide partitions while segments are large (the top levels of the item)
  while (q.nbig > 0) {
    const unsigned e = q.big[q.nbig - 1];
    const int s = (int)(e >> 16), n = (int)((e >> 1) & 0x7fffu), pe = (int)(e & 1u);
    bsync();
    const K *X = pe ? B : A;
    K *Y = pe ? A : B;
    const K key = X[s];
    const int L = block_partition<K, NT>(X, Y, s, n, key, q);
    ++nseg;
    const int cp = pe ^ 1;
    if (tid == 0) {
      A[s + L] = key;
      seg_mark(seg, s + L);
      --q.nbig;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int cs = c ? s + L + 1 : s, cn = c ? n - L - 1 : L;
        if (cn > block_segment(NT)) q.big[q.nbig++] = seg_pack(cs, cn, cp);
        else if (cn > kMarkLeaf) small_push(q, cs, cn, cp);
        else mark_final(seg, par, cs, cn, cp);
      }
    }
    bsync();
  }
  // warp-level Steps 1-6 on the queued segments (all above kMarkLeaf keys)
  while (true) {
    unsigned e = 0;
    if (lane == 0) e = small_pop(q);
    e = __shfl_sync(kFull, e, 0);
    if (e == 0u) break;
    int s = (int)(e >> 16), n = (int)((e >> 1) & 0x7fffu), pe = (int)(e & 1u);
    while (true) {
      const K *X = pe ? B : A;
      K *Y = pe ? A : B;
      ++nseg;
      const K key = X[s];  // Step 1
      const int L = warp_partition(X, Y, s, n, key);
      const int ls = s, ln = L, rs = s + L + 1, rn = n - L - 1, cp = pe ^ 1;
      if (lane == 0) {
        A[s + L] = key;  // Step 4: final index
        seg_mark(seg, s + L);
        if (ln <= kMarkLeaf) mark_final(seg, par, ls, ln, cp);
        if (rn <= kMarkLeaf) mark_final(seg, par, rs, rn, cp);
      }
      // Steps 5-6: of two sides above kMarkLeaf keys the smaller is queued and the warp
      // keeps the other
      const bool bl = ln > kMarkLeaf, br = rn > kMarkLeaf;
      if (bl && br) {
        if (lane == 0) {
          if (ln < rn) small_push(q, ls, ln, cp);
          else small_push(q, rs, rn, cp);
        }
        if (ln < rn) { s = rs; n = rn; } else { s = ls; n = ln; }
        pe = cp;
      } else if (bl) {
        s = ls; n = ln; pe = cp;
      } else if (br) {
        s = rs; n = rn; pe = cp;
      } else {
        break;
      }
    }
    if (lane == 0) {
      __threadfence_block();
      atomicSub(&q.pending, 1);
    }
  }
  bsync();
  // every index: its segment from the marks, its key to the final index; thread 0 first
  // runs `pre` (the claim of the next item), which overlaps the other warps' windows
  if (tid == 0) pre();
  const unsigned le = lane == 31 ? kFull : ((2u << lane) - 1u);
  const int nwin = (m + 31) >> 5;
  bool broken = false;
  for (int w = warp; w < nwin; w += NT / 32) {
    const int i = (w << 5) + lane;
    const unsigned cur = seg[w], nxt = seg[w + 1], prv = w > 0 ? seg[w - 1] : 0u;
    const unsigned below = cur & le, above = cur & ~le;
    const int s0 = below ? (w << 5) + 31 - __clz(below)
                         : (prv ? ((w - 1) << 5) + 31 - __clz(prv) : -1);
    const int e0 = above ? (w << 5) + __ffs(above) - 1
                         : (nxt ? ((w + 1) << 5) + __ffs(nxt) - 1 : -1);
    if (i >= m) continue;
    if (s0 < 0 || e0 < 0 || e0 - s0 > kMarkLeaf) {  // marks do not cover i: report, skip
      broken = true;
      continue;
    }
    const int n = e0 - s0, me = i - s0;
    const K *src = ((par[s0 >> 5] >> (s0 & 31)) & 1u) ? B : A;
    const K x = src[i];
    int pos = me;
    if (n >= 2) {
      pos = 0;
#pragma unroll 4
      for (int j = 0; j < n; ++j) {
        const K y = src[s0 + j];
        // y < x (y goes left of key x), or y == x and y comes earlier
        pos += (goes_left(x, y) || (j < me && !goes_left(y, x))) ? 1 : 0;
      }
    }
    out[s0 + pos] = x;
  }
  if (broken) q.bad = 1;
  bsync();
  if (tid == 0) *segments += nseg;
  return q.bad == 0;
}

// Dynamic shared memory of a finisher CTA of nt threads: A and B (cutoff keys each),
// the per-warp leaf lists, then the two mark bitmaps (cutoff + 64 bits each).
__host__ __device__ constexpr int small_mark_words(int cutoff) { return (cutoff >> 5) + 2; }
template <typename K>
__host__ __device__ constexpr size_t small_smem_bytes(int cutoff, int nt = kSmallThreads) {
  return (size_t)2 * cutoff * sizeof(K) + (size_t)nt * sizeof(unsigned) + 16 +
         2 * small_mark_words(cutoff) * sizeof(unsigned);
}

// The finisher's shared memory carved from one dynamic allocation (at `base`).
template <typename K>
struct SmallSmem {
  K *A, *B;
  unsigned *leaf_lists, *seg, *par;
  __device__ SmallSmem(unsigned char *base, int cutoff, int nt) {
    A = reinterpret_cast<K *>(base);
    B = A + cutoff;
    leaf_lists = reinterpret_cast<unsigned *>(B + cutoff);
    seg = leaf_lists + nt + 4;
    par = seg + small_mark_words(cutoff);
  }
};

// ----------------------------------------------------------------------------- queue
// Work items live in a bump-allocated pool. The sort runs in two phases.
// Phase 1 (Steps 1-4 on items above the cutoff, with Steps 5-6 queuing their sides):
// a large item reserves one ticket per tile pass; tickets index both the look-back
// descriptors and a ticket map that names the item. CTAs claim tickets with
// one atomicAdd, in order, possibly before the item that owns the ticket exists; they
// then wait for it, so a freshly queued item starts without dispatch delay. Phase 2
// starts when every large item has completed: the small items, now a complete list,
// are claimed with atomicAdd and finished in shared memory. Entries carry the sort's
// epoch, so no memset is needed between sorts.
__device__ __forceinline__ unsigned long long q_entry(unsigned epoch, unsigned long long idx) {
  return ((unsigned long long)epoch << 32) | idx;
}

// One thread queues the sub-array [b, e) of buffer (flags & kItemScratch). A small item
// goes straight to the small list. A large item gets its tile tickets; its ticket-map
// entries are written afterwards by publish_tickets (possibly by several threads).
// Returns the ticket range in *t0 / *tiles (tiles = 0: nothing left to publish).
template <typename K, int TILE>
__device__ __forceinline__ unsigned long long reserve_item(const SortParams &p, unsigned epoch,
                                                           long long b, long long e,
                                                           unsigned flags,
                                                           unsigned long long *t0_out,
                                                           unsigned *tiles_out) {
  Control *ctl = p.ctl;
  *tiles_out = 0;
  if (!sub_array_ok(p, b, e, 1)) return 0;
  const long long m = e - b;
  const K *buf = (flags & kItemScratch) ? static_cast<const K *>(p.scratch)
                                        : static_cast<const K *>(p.keys);
  const bool small = m <= p.cutoff && !(flags & kItemPartitionOnly);
  const unsigned tiles = small ? 1u : tile_count<K, TILE>(buf, b, e);
  // a medium item takes one ticket; its CTA runs all of its tile passes
  const bool medium = !small && tiles >= 2 && (int)tiles <= p.medium_tiles;
  const unsigned tickets = medium ? 1u : tiles;
  // the key load and both atomics are independent: all three are in flight at once
  const K first = __ldcg(buf + b);
  const unsigned long long t0 = small ? 0ull : atomicAdd(&ctl->lb_used, (unsigned long long)tickets);
  const unsigned long long idx = atomicAdd(&ctl->pushed, 1ull);
  if (!small && t0 + tickets > p.lb_cap) {
    raise_error(ctl, kDevWorkspaceExhausted, 2);
    return 0;
  }
  if (idx >= p.item_cap) {
    raise_error(ctl, kDevWorkspaceExhausted, 1);
    return 0;
  }
  Item *it = p.items + idx;
  it->begin = b;
  it->end = e;
  it->key = key_bits<K>(first);
  it->tiles = tiles;
  it->lb = (unsigned)t0;
  it->flags = flags | (small ? kItemSmall : 0u) | (medium ? kItemMedium : 0u);
  it->epoch = epoch;
  if (small) {
    __threadfence();
    const unsigned long long qi = atomicAdd(&ctl->sq_tail, 1ull);  // qi <= idx < item_cap
    st_release(&p.small_q[qi], q_entry(epoch, idx));
  } else {
    ItemCtl *c = p.ictl + idx;
    c->done = 0;
    c->less = 0;
    atomicAdd(&ctl->large_pushed, 1ull);  // before any ticket can be served
    __threadfence();
    *t0_out = t0;
    *tiles_out = tickets;
  }
  return idx;
}

// Ticket-map entries of a reserved large item, written by `group` threads (rank r).
// Each entry is a release store, so an acquirer also sees the item record.
__device__ __forceinline__ void publish_tickets(const SortParams &p, unsigned epoch,
                                                unsigned long long idx, unsigned long long t0,
                                                unsigned tiles, int r, int group) {
  const unsigned long long entry = q_entry(epoch, idx);
  for (unsigned j = r; j < tiles; j += group) st_release(&p.tmap[t0 + j], entry);
}

__device__ __forceinline__ void load_item(const Item *ip, Item *it) {
  it->begin = __ldcg(&ip->begin);
  it->end = __ldcg(&ip->end);
  it->key = __ldcg(&ip->key);
  it->tiles = __ldcg(&ip->tiles);
  it->lb = __ldcg(&ip->lb);
  it->flags = __ldcg(&ip->flags);
  it->epoch = 0;
}

// One thread, phase 1: waits for ticket k to be issued. Returns 1 with the item index,
// 0 when phase 1 is over (every large item completed), -1 on abort or timeout.
__device__ __forceinline__ int wait_ticket(const SortParams &p, unsigned epoch,
                                           unsigned long long k, long long *h_out) {
  Control *ctl = p.ctl;
  unsigned ns = 16;
  unsigned long long idle_t0 = 0, last = ~0ull;
  while (true) {
    if (k < p.lb_cap) {
      const unsigned long long v = ld_acquire(&p.tmap[k]);
      if ((unsigned)(v >> 32) == epoch) {
        *h_out = (long long)(v & 0xffffffffull);
        return 1;
      }
    }
    if (ld_relaxed(&ctl->abort)) return -1;
    // `completed` before `pushed`: an item queues its sides before it completes
    const unsigned long long c = ld_acquire(&ctl->large_completed);
    const unsigned long long pu = ld_acquire(&ctl->large_pushed);
    if (c == pu) return 0;
    const unsigned long long now = globaltimer();
    if (c != last) {
      last = c;
      idle_t0 = now;
    } else if (now - idle_t0 > p.spin_limit_ns) {
      raise_error(ctl, kDevTimeout, 0x300000000ull | k);
      return -1;
    }
    __nanosleep(ns);
    ns = ns < 256 ? ns * 2 : 256;
  }
}

// One thread, phase 2: claims the next small item. Returns 1 with the item, 0 when none
// is left, -1 on abort or timeout.
__device__ __forceinline__ int claim_small(const SortParams &p, unsigned epoch, long long *h_out,
                                           Item *it_out) {
  Control *ctl = p.ctl;
  if (ld_relaxed(&ctl->abort)) return -1;
  const unsigned long long j = atomicAdd(&ctl->sq_head, 1ull);
  if (j >= ld_acquire(&ctl->sq_tail) || j >= p.item_cap) return 0;
  unsigned long long t0 = 0;
  for (unsigned spins = 1;; ++spins) {  // queued before phase 2 began: already visible
    const unsigned long long v = ld_acquire(&p.small_q[j]);
    if ((unsigned)(v >> 32) == epoch) {
      const long long idx = (long long)(v & 0xffffffffull);
      load_item(p.items + idx, it_out);
      *h_out = idx;
      return 1;
    }
    if ((spins & 255u) == 0u) {
      const unsigned long long now = globaltimer();
      if (t0 == 0) t0 = now;
      if (now - t0 > p.spin_limit_ns) {
        raise_error(ctl, kDevTimeout, 0x200000000ull | j);
        return -1;
      }
    }
    __nanosleep(32);
  }
}

// A CTA of NT threads, any phase: the small item `it` (index h) is loaded into shared
// memory and finished there by smem_ksort_marked, or by smem_ksort when it holds a NaN
// key; its keys end in buffer 0. Thread 0 runs `pre` once on the way (the next item's
// claim), and the closing CTA barrier makes what it wrote visible.
template <typename K, int NT, typename Pre>
__device__ __forceinline__ void finish_small_item(const SortParams &p, const Item it, long long h,
                                                  K *buf0, const K *buf1, const SmallSmem<K> &sm,
                                                  SmallShared &q, unsigned long long *st_small,
                                                  unsigned long long *st_small_keys,
                                                  unsigned long long *st_segs, Pre &&pre) {
  const int tid = threadIdx.x;
  const K *src = ((it.flags & kItemScratch) ? buf1 : buf0) + it.begin;
  const int m = (int)(it.end - it.begin);
  bool nan = false;
  for (int e = tid; e < m; e += NT) {
    const K v = __ldcg(src + e);
    sm.A[e] = v;
    nan |= key_is_nan(v);
  }
  bool ok;
  if (__syncthreads_or(nan)) {
    ok = smem_ksort<K, NT>(sm.A, sm.B, sm.leaf_lists, buf0 + it.begin, m, q, st_segs);
    if (tid == 0) pre();
  } else {
    ok = smem_ksort_marked<K, NT>(sm.A, sm.B, sm.seg, sm.par, buf0 + it.begin, m, q, st_segs,
                                  pre);
  }
  if (tid == 0) {
    if (!ok) raise_error(p.ctl, kDevInternal, 0x600000000ull | (unsigned)h);
    ++*st_small;
    *st_small_keys += (unsigned long long)m;
  }
  __syncthreads();
}

// One thread, phase 1: claims the next small item only if one is queued now (the list
// is still growing, so the head moves by compare-and-swap and never passes the tail).
// Returns 1 with the item, 0 when none is queued, -1 on abort or timeout.
__device__ __forceinline__ int try_claim_small(const SortParams &p, unsigned epoch,
                                               long long *h_out, Item *it_out) {
  Control *ctl = p.ctl;
  if (ld_relaxed(&ctl->abort)) return -1;
  unsigned long long j = ld_relaxed(&ctl->sq_head);
  while (true) {
    const unsigned long long tail = ld_acquire(&ctl->sq_tail);
    if (j >= tail || j >= p.item_cap) return 0;
    const unsigned long long prev = atomicCAS(&ctl->sq_head, j, j + 1);
    if (prev == j) break;
    j = prev;
  }
  unsigned long long t0 = 0;
  for (unsigned spins = 1;; ++spins) {  // its pusher has taken the slot: the entry follows
    const unsigned long long v = ld_acquire(&p.small_q[j]);
    if ((unsigned)(v >> 32) == epoch) {
      const long long idx = (long long)(v & 0xffffffffull);
      load_item(p.items + idx, it_out);
      *h_out = idx;
      return 1;
    }
    if ((spins & 255u) == 0u) {
      const unsigned long long now = globaltimer();
      if (t0 == 0) t0 = now;
      if (now - t0 > p.spin_limit_ns) {
        raise_error(ctl, kDevTimeout, 0xC00000000ull | j);
        return -1;
      }
    }
    __nanosleep(32);
  }
}

// Diagnostics: timestamp `slot` of ticket k (only when a trace buffer is installed).
__device__ __forceinline__ void trace_mark(const SortParams &p, unsigned long long k, int slot) {
  if (p.trace && k < (unsigned long long)p.trace_cap) p.trace[k * kTraceWords + slot] = globaltimer();
}

// ----------------------------------------------------------------------------- kernels
// Phase 1: tile passes. Each CTA loops: claim a ticket (claimed one ahead, so the
// claim's latency overlaps the previous tile), wait until it is issued, load the
// tile's keys with 128-bit loads straight into registers, and run Steps 1-4 on them:
//   count   Step 3 per key (bit masks), one warp scan of the (less, >=) counts, the
//           tile totals and this thread's offsets; the tile's aggregate is published
//           at once so that later tiles' look-backs need not wait for the rest;
//   scatter this thread's less keys to sout from the front and its >= keys after all
//           less keys (tile-local order: thread by thread), while warp 0 runs the
//           look-back that yields E, the less keys of all earlier tiles of the item;
//   write   less keys of tile t to dst[begin + E ...]; >= keys to the right end,
//           dst[end - PG - G ...] with PG the >= keys of earlier tiles, so the key's
//           index begin + #{x < key} stays free.
// Thread i owns the keys at tile positions (v * NT + i) * VEC + l. The last tile of an
// item to finish places the key (Step 4) and queues both sides (Steps 5-6). The tile
// shape (NT threads x IPT keys) is one of a few compiled variants picked at run time.
template <int NW>
struct TileCtaShared {
  unsigned wl[NW], wg[NW];
  unsigned long long E;
  int abort;
  int r;        // ticket status for the CTA
  unsigned t;   // tile index within the item
  long long h;  // item index
  Item it;      // the item (cached while tickets stay within one item)
  long long lo;
  int vlo, vhi;
  int last;     // this CTA finished the item's last tile
  unsigned long long k;  // ticket
  unsigned long long cidx[2], ct0[2];
  unsigned ctiles[2];
  unsigned long long c_less;  // #{x < key} of the item being finished
  unsigned mL[kMediumMaxTiles], mG[kMediumMaxTiles];  // a medium item's tile counts
};

// Keys [vlo, vhi) of the tile at src + lo (16-byte aligned) into registers, by NG
// threads; rank r holds tile positions (v * NG + r) * VEC + l. Whole vectors inside the
// range move with 128-bit loads, the edges one key at a time; nothing outside the range
// is read.
template <typename K, int NG, int IPT>
__device__ __forceinline__ void tile_load(const K *src, long long lo, int vlo, int vhi,
                                          K (&x)[IPT], int r) {
  constexpr int VEC = Vec<K>::N, NV = IPT / VEC;
  using V = typename Vec<K>::T;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const int k0 = (v * NG + r) * VEC;
    if (k0 >= vlo && k0 + VEC <= vhi) {
      const V q = __ldcg(reinterpret_cast<const V *>(src + lo + k0));
      if constexpr (VEC == 4) {
        x[v * 4 + 0] = q.x; x[v * 4 + 1] = q.y; x[v * 4 + 2] = q.z; x[v * 4 + 3] = q.w;
      } else {
        x[v * 2 + 0] = q.x; x[v * 2 + 1] = q.y;
      }
    } else {
#pragma unroll
      for (int l = 0; l < VEC; ++l) {
        const int k = k0 + l;
        x[v * VEC + l] = (k >= vlo && k < vhi) ? __ldcg(src + lo + k) : K(0);
      }
    }
  }
}

// Whole CTA, once every tile pass of item h is written and c = #{x < key} is known:
// Step 4 (the key to its final index) and Steps 5-6 (both sides queued; the tickets of
// large sides published by every thread), then the item counts as completed.
template <typename K, int TILE, int NW>
__device__ __forceinline__ void finish_item(const SortParams &p, unsigned epoch, const Item &it,
                                            long long h, unsigned long long c,
                                            TileCtaShared<NW> &sh, unsigned long long &st_large,
                                            unsigned long long &st_large_keys) {
  const int tid = threadIdx.x;
  Control *ctl = p.ctl;
  K *const buf0 = static_cast<K *>(p.keys);
  const unsigned par = it.flags & kItemScratch;
  K *dst = static_cast<K *>(par ? p.keys : p.scratch);
  const K key = bits_key<K>(it.key);
  const long long kpos = it.begin + (long long)c;
  const bool bad = kpos >= it.end;
  if (tid < 2) sh.ctiles[tid] = 0;
  if (tid == 0) {
    if (bad) {
      raise_error(ctl, kDevInternal, 0x700000000ull | (unsigned)h);
    } else if (it.flags & kItemPartitionOnly) {
      dst[kpos] = key;  // a single partition: the key index is the result
      if (p.key_index) *p.key_index = (long long)c;
    } else {
      buf0[kpos] = key;  // Step 4
    }
  }
  if (tid < 2 && !bad && !(it.flags & kItemPartitionOnly)) {
    // Steps 5-6: threads 0 and 1 queue the two sides at once (each a chain of atomics)
    const int s = tid;
    const unsigned cflags = par ^ kItemScratch;
    const long long cb = s ? kpos + 1 : it.begin, ce = s ? it.end : kpos;
    const long long mm = ce - cb;
    if (mm == 1) {
      if (cflags & kItemScratch) buf0[cb] = __ldcg(dst + cb);
    } else if (mm >= 2) {
      unsigned long long t0 = 0;
      unsigned tiles = 0;
      sh.cidx[s] = reserve_item<K, TILE>(p, epoch, cb, ce, cflags, &t0, &tiles);
      sh.ct0[s] = t0;
      sh.ctiles[s] = tiles;
    }
  }
  __syncthreads();
#pragma unroll
  for (int s = 0; s < 2; ++s)
    if (sh.ctiles[s]) publish_tickets(p, epoch, sh.cidx[s], sh.ct0[s], sh.ctiles[s], tid, blockDim.x);
  __syncthreads();
  if (tid == 0) {
    ++st_large;
    st_large_keys += (unsigned long long)(it.end - it.begin);
    __threadfence();
    atomicAdd(&ctl->large_completed, 1ull);
  }
}

// FUSE: the CTAs also finish small items (dynamic shared memory: SmallShared, then the
// finisher's buffers for p.cutoff keys). A CTA about to claim a ticket takes a queued
// small item instead while at least p.fuse_park tickets are held beyond the ones issued
// (CTAs already parked for items still to come). The finisher launch that follows takes
// what is left of the small list.
template <typename K, int NT, int IPT, bool FUSE>
__global__ void __launch_bounds__(NT, tile_min_blocks(NT)) tile_kernel(SortParams p) {
  constexpr int TILE = NT * IPT;
  constexpr int VEC = Vec<K>::N;
  constexpr int NV = IPT / VEC;
  constexpr int NW = NT / 32;
  static_assert(IPT % VEC == 0 && IPT <= 32 && NT % 32 == 0, "bad tile shape");
  using V = typename Vec<K>::T;
  __shared__ __align__(16) K sout[TILE + Vec<K>::N];  // + room for copy_out_v's reads
  __shared__ TileCtaShared<NW> sh;
  K *const buf0 = static_cast<K *>(p.keys);
  K *const buf1 = static_cast<K *>(p.scratch);
  Control *ctl = p.ctl;
  grid_dep_wait();    // the seed (or the previous launch) is complete
  grid_dep_launch();  // the finisher may start launching as CTAs leave
  const unsigned epoch = *reinterpret_cast<volatile unsigned *>(&ctl->epoch);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const unsigned lt = lanemask_lt();
  unsigned long long st_tiles = 0, st_lb = 0, st_large = 0, st_large_keys = 0;
  long long cached_h = -1;
  unsigned long long k_next = ~0ull;  // ticket claimed at the end of the previous tile
  extern __shared__ __align__(16) unsigned char fuse_smem[];
  unsigned long long st_small = 0, st_small_keys = 0, st_segs = 0;

  while (true) {
    // ---- claim: tickets are taken only when the CTA is about to load them, so
    // consecutive tickets are worked on at about the same time and look-backs find
    // their predecessors' aggregates already published
    int fr = 0;
    if constexpr (FUSE) {
      if (tid == 0 && k_next == ~0ull) {
        const unsigned long long head = ld_relaxed(&ctl->tq_head);
        const unsigned long long used = ld_relaxed(&ctl->lb_used);
        if (head >= used + (unsigned long long)p.fuse_park) {
          fr = try_claim_small(p, epoch, &sh.h, &sh.it);
          if (fr != 0) {
            sh.r = fr > 0 ? 2 : -1;
            cached_h = -1;
          }
        }
      }
    }
    if (tid == 0 && fr == 0) {
      const unsigned long long k = k_next != ~0ull ? k_next : atomicAdd(&ctl->tq_head, 1ull);
      k_next = ~0ull;
      long long h = 0;
      const unsigned long long tw0 = p.trace ? globaltimer() : 0;
      const int r = wait_ticket(p, epoch, k, &h);
      sh.r = r;
      sh.k = k;
      if (r > 0) {
        if (p.trace && k < (unsigned long long)p.trace_cap) {
          p.trace[k * kTraceWords + 0] = tw0;  // ticket claimed, wait starts
          p.trace[k * kTraceWords + 1] = globaltimer();  // ticket issued
          p.trace[k * kTraceWords + 5] = 0;
          p.trace[k * kTraceWords + 7] = blockIdx.x;
        }
        if (h != cached_h) {
          load_item(p.items + h, &sh.it);
          cached_h = h;
        }
        const K *src = (sh.it.flags & kItemScratch) ? buf1 : buf0;
        const unsigned t = (unsigned)(k - sh.it.lb);
        const long long lo = tile_base(src, sh.it.begin) + (long long)t * TILE;
        const long long first = sh.it.begin + 1;
        sh.h = h;
        sh.t = t;
        sh.lo = lo;
        sh.vlo = (int)(first > lo ? first - lo : 0);
        sh.vhi = (int)(sh.it.end - lo < TILE ? sh.it.end - lo : TILE);
      }
    }
    __syncthreads();
    if constexpr (FUSE) {
      SmallShared &q = *reinterpret_cast<SmallShared *>(fuse_smem);
      const SmallSmem<K> sm(fuse_smem + (sizeof(SmallShared) + 15) / 16 * 16, p.cutoff, NT);
      if (sh.r == 2) {  // a small item, taken while other CTAs wait for tiles
        finish_small_item<K, NT>(p, sh.it, sh.h, buf0, buf1, sm, q, &st_small, &st_small_keys,
                                 &st_segs, [] {});
        continue;
      }

    }
    if (sh.r <= 0) break;
    if (sh.it.flags & kItemMedium) {
      // ---- a medium item: this CTA runs all its tile passes, counting first and then
      // moving, so each tile's prefix is known locally (no look-back, one ticket)
      const Item it = sh.it;
      const long long h = sh.h;
      const unsigned par = it.flags & kItemScratch;
      const K *src = par ? buf1 : buf0;
      K *dst = par ? buf0 : buf1;
      const K key = bits_key<K>(it.key);  // Step 1
      const long long base = tile_base(src, it.begin), first = it.begin + 1;
      const unsigned T = it.tiles;
      if (tid < kMediumMaxTiles) {
        sh.mL[tid] = 0;
        sh.mG[tid] = 0;
      }
      __syncthreads();
      for (unsigned t = 0; t < T; ++t) {  // Step 3: counts of every tile
        const long long lo = base + (long long)t * TILE;
        const int vlo = (int)(first > lo ? first - lo : 0);
        const int vhi = (int)(it.end - lo < TILE ? it.end - lo : TILE);
        K x[IPT];
        tile_load<K, NT, IPT>(src, lo, vlo, vhi, x, tid);
        unsigned cl = 0, cg = 0;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
#pragma unroll
          for (int l = 0; l < VEC; ++l) {
            const int k = (v * NT + tid) * VEC + l;
            if (k >= vlo && k < vhi) {
              if (goes_left(key, x[v * VEC + l])) ++cl;
              else ++cg;
            }
          }
        }
        cl = __reduce_add_sync(kFull, cl);
        cg = __reduce_add_sync(kFull, cg);
        if (lane == 0) {
          atomicAdd(&sh.mL[t], cl);
          atomicAdd(&sh.mG[t], cg);
        }
      }
      __syncthreads();
      unsigned long long E = 0;
      bool bad = false;
      for (unsigned t = 0; t < T && !bad; ++t) {  // Steps 3.1/3.2 per tile, prefix known
        const long long lo = base + (long long)t * TILE;
        const int vlo = (int)(first > lo ? first - lo : 0);
        const int vhi = (int)(it.end - lo < TILE ? it.end - lo : TILE);
        K x[IPT];
        tile_load<K, NT, IPT>(src, lo, vlo, vhi, x, tid);
        unsigned lessbits = 0, gebits = 0;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
#pragma unroll
          for (int l = 0; l < VEC; ++l) {
            const int j = v * VEC + l, k = (v * NT + tid) * VEC + l;
            const bool valid = k >= vlo && k < vhi;
            const bool le = goes_left(key, x[j]);
            lessbits |= (unsigned)(valid && le) << j;
            gebits |= (unsigned)(valid && !le) << j;
          }
        }
        const unsigned mine = (unsigned)__popc(lessbits) | ((unsigned)__popc(gebits) << 16);
        unsigned incl = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const unsigned u = __shfl_up_sync(kFull, incl, o);
          if (lane >= o) incl += u;
        }
        if (lane == 31) {
          sh.wl[w] = incl & 0xffffu;
          sh.wg[w] = incl >> 16;
        }
        __syncthreads();
        unsigned L = 0, G = 0, wlx = 0, wgx = 0;
#pragma unroll
        for (int i = 0; i < NW; ++i) {
          const unsigned a = sh.wl[i], b = sh.wg[i];
          if (i < w) {
            wlx += a;
            wgx += b;
          }
          L += a;
          G += b;
        }
        scatter_keys<K, IPT>(sout, x, lessbits, gebits, wlx, L + wgx, incl - mine);
        __syncthreads();
        long long lbase = 0, gbase = 0;
        if (L != sh.mL[t] || G != sh.mG[t] ||
            !tile_dest(it.begin, it.end, lo, t, E, L, G, &lbase, &gbase)) {
          if (tid == 0) raise_error(ctl, kDevInternal, 0x500000000ull | t);
          bad = true;  // uniform: every thread computed the same values
        } else {
          copy_out_v<K, NT>(sout, dst + lbase, L, tid);
          copy_out_v<K, NT>(sout + L, dst + gbase, G, tid);
          E += L;
        }
        __syncthreads();  // sout and the warp counts are reused by the next tile
      }
      if (bad) break;
      if (tid == 0) {
        if (!FUSE) k_next = atomicAdd(&ctl->tq_head, 1ull);
        st_tiles += T;
      }
      finish_item<K, TILE, NW>(p, epoch, it, h, E, sh, st_large, st_large_keys);
      if (tid == 0) trace_mark(p, sh.k, 6);  // completed
      continue;
    }
    const Item it = sh.it;
    const unsigned t = sh.t;
    const long long lo = sh.lo, h = sh.h;
    const int vlo = sh.vlo, vhi = sh.vhi;
    const unsigned par = it.flags & kItemScratch;
    const K *src = par ? buf1 : buf0;
    K *dst = par ? buf0 : buf1;
    const K key = bits_key<K>(it.key);  // Step 1: the first element is the key

    // ---- load (whole vectors with 128-bit loads, single loads at the edges)
    K x[IPT];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int k0 = (v * NT + tid) * VEC;
      if (k0 >= vlo && k0 + VEC <= vhi) {
        const V q = __ldcg(reinterpret_cast<const V *>(src + lo + k0));
        if constexpr (VEC == 4) {
          x[v * 4 + 0] = q.x; x[v * 4 + 1] = q.y; x[v * 4 + 2] = q.z; x[v * 4 + 3] = q.w;
        } else {
          x[v * 2 + 0] = q.x; x[v * 2 + 1] = q.y;
        }
      } else {
#pragma unroll
        for (int l = 0; l < VEC; ++l) {
          const int k = k0 + l;
          x[v * VEC + l] = (k >= vlo && k < vhi) ? __ldcg(src + lo + k) : K(0);
        }
      }
    }
    // ---- count (Step 3)
    unsigned lessbits = 0, gebits = 0;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
#pragma unroll
      for (int l = 0; l < VEC; ++l) {
        const int j = v * VEC + l, k = (v * NT + tid) * VEC + l;
        const bool valid = k >= vlo && k < vhi;
        const bool le = goes_left(key, x[j]);
        lessbits |= (unsigned)(valid && le) << j;
        gebits |= (unsigned)(valid && !le) << j;
      }
    }
    const unsigned mine = (unsigned)__popc(lessbits) | ((unsigned)__popc(gebits) << 16);
    unsigned incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned u = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += u;
    }
    if (lane == 31) {
      sh.wl[w] = incl & 0xffffu;
      sh.wg[w] = incl >> 16;
    }
    __syncthreads();
    unsigned L = 0, G = 0, wlx = 0, wgx = 0;
#pragma unroll
    for (int i = 0; i < NW; ++i) {
      const unsigned a = sh.wl[i], b = sh.wg[i];
      if (i < w) {
        wlx += a;
        wgx += b;
      }
      L += a;
      G += b;
    }
    unsigned long long *lb = p.lb + it.lb;
    unsigned long long resv = 0;
    if (tid == 0) {
      if (p.reserve) {
        // the tile's ranges at once: one add of (>= << 32 | less) to the item's counter
        // gives the less and >= keys of the tiles that took theirs before; the result is
        // first used after the scatter, so its round trip overlaps it
        resv = atomicAdd(&p.ictl[h].less, ((unsigned long long)G << 32) | L);
      } else {
        st_relaxed(&lb[t], lb_pack(epoch, t == 0, L));  // aggregate (inclusive: tile 0)
      }
      trace_mark(p, sh.k, 2);  // loaded and counted
    }

    // ---- look-back (warp 0) and scatter (everyone)
    if (w == 0 && !p.reserve) {
      unsigned long long E = 0;
      int status = 0;
      if (t > 0) {
        unsigned long long steps = 0;
        unsigned long long dbg[3] = {0, 0, 0};
        const bool tr = p.trace && sh.k < (unsigned long long)p.trace_cap;
        status = lookback(lb, t, epoch, p.spin_limit_ns, &ctl->abort, &E, &steps,
                          tr ? dbg : nullptr);
        if (lane == 0) {
          if (status == 0) st_relaxed(&lb[t], lb_pack(epoch, true, (unsigned)(E + L)));
          st_lb += steps;
          if (tr) {
            p.trace[sh.k * kTraceWords + 5] = dbg[0];
            p.trace[sh.k * kTraceWords + 7] = blockIdx.x | (dbg[1] << 20) | (dbg[2] << 40);
          }
        }
      }
      if (lane == 0) {
        if (status == 1) raise_error(ctl, kDevTimeout, 0x100000000ull | t);
        sh.E = E;
        sh.abort = status == 0 ? 0 : 1;
        trace_mark(p, sh.k, 3);  // look-back done
      }
    }
    scatter_keys<K, IPT>(sout, x, lessbits, gebits, wlx, L + wgx, incl - mine);
    if (tid == 0 && p.reserve) {
      sh.E = resv;
      sh.abort = 0;
    }
    __syncthreads();
    const unsigned long long E = sh.E;
    if (sh.abort) break;

    // ---- write
    long long lbase = 0, gbase = 0;
    if (p.reserve) {
      const long long PL = (long long)(E & 0xffffffffull), PG = (long long)(E >> 32);
      lbase = it.begin + PL;
      gbase = it.end - PG - (long long)G;
    }
    if (p.reserve ? !(ranges_ok(it.begin, it.end, lbase, L, gbase, G))
                  : !tile_dest(it.begin, it.end, lo, t, E, L, G, &lbase, &gbase)) {
      if (tid == 0) raise_error(ctl, kDevInternal, 0x500000000ull | t);
      break;
    }
    copy_out_v<K, NT>(sout, dst + lbase, L, tid);
    copy_out_v<K, NT>(sout + L, dst + gbase, G, tid);
    __syncthreads();

    // ---- completion: the last tile of the item places the key and queues both sides
    if (tid == 0) {
      trace_mark(p, sh.k, 4);  // written
      ++st_tiles;
      if (t == it.tiles - 1 && !p.reserve) atomicExch(&p.ictl[h].less, E + L);
      // release: this tile's writes (ordered before by the barrier) and `less` become
      // visible to whichever CTA observes the count reaching tiles
      const unsigned done_before = atom_add_release(&p.ictl[h].done, 1u);
      if (!FUSE) k_next = atomicAdd(&ctl->tq_head, 1ull);  // the next ticket (its claim overlaps)
      sh.last = done_before == it.tiles - 1;
      if (sh.last) {
        __threadfence();
        const unsigned long long v = ld_acquire(&p.ictl[h].less);
        sh.c_less = p.reserve ? (v & 0xffffffffull) : v;  // every tile has taken its range
      }
    }
    __syncthreads();
    if (sh.last) finish_item<K, TILE, NW>(p, epoch, it, h, sh.c_less, sh, st_large, st_large_keys);
    if (tid == 0) trace_mark(p, sh.k, 6);  // completed
  }
  if (tid == 0) {
    if (st_tiles) atomicAdd(&ctl->tiles, st_tiles);
    if (st_lb) atomicAdd(&ctl->lookback_steps, st_lb);
    if (st_large) atomicAdd(&ctl->large_items, st_large);
    if (st_large_keys) atomicAdd(&ctl->large_keys, st_large_keys);
    if (st_small) atomicAdd(&ctl->small_items, st_small);
    if (st_small_keys) atomicAdd(&ctl->small_keys, st_small_keys);
    if (st_segs) atomicAdd(&ctl->smem_levels, st_segs);
  }
}

// Dynamic shared memory of the fused tile kernel.
template <typename K>
__host__ __device__ constexpr size_t fuse_smem_bytes(int cutoff, int nt) {
  return (sizeof(SmallShared) + 15) / 16 * 16 + small_smem_bytes<K>(cutoff, nt);
}

// ----------------------------------------------------------------------------- staged
// Bulk copies global -> shared (cp.async.bulk) with mbarrier completion.
__device__ __forceinline__ unsigned smem_u32(const void *ptr) {
  return (unsigned)__cvta_generic_to_shared(ptr);
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes,
                                         unsigned long long *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// The same with a suspend-time hint: the thread sleeps until the phase completes or
// about hint_ns pass, instead of returning after the hardware's own short limit, so an
// idle warp does not take issue slots from the warps that work.
__device__ __forceinline__ bool mbar_try_wait_sleep(unsigned long long *bar, unsigned parity,
                                                    unsigned hint_ns) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_test(unsigned long long *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for phase `parity` of `bar` to complete; false if limit_ns passed first.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity,
                                          unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  for (unsigned i = 1;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 31u) == 0u && globaltimer() - t0 > limit_ns) return false;
  }
}

// Geometry of one tile pass (the ring form's slots), written by the producer.
struct PipeTile {
  Item it;
  long long h;              // item index
  long long lo;             // first buffer index of the tile (16-byte aligned)
  unsigned long long k;     // ticket
  unsigned t;               // tile index within the item
  int vlo, vhi;             // classified keys of the tile: [vlo, vhi)
  int agg;                  // its aggregate is published already
};

template <typename K, int TILE>
__device__ __forceinline__ void pipe_geom(const SortParams &p, PipeTile &pt, Item *ci,
                                          long long *ch, unsigned long long k, long long h) {
  if (h != *ch) {
    load_item(p.items + h, ci);
    *ch = h;
  }
  pt.it = *ci;
  const K *src = static_cast<const K *>((pt.it.flags & kItemScratch) ? p.scratch : p.keys);
  pt.k = k;
  pt.h = h;
  pt.t = (unsigned)(k - pt.it.lb);
  pt.lo = tile_base(src, pt.it.begin) + (long long)pt.t * TILE;
  const long long first = pt.it.begin + 1;
  pt.vlo = (int)(first > pt.lo ? first - pt.lo : 0);
  pt.vhi = (int)(pt.it.end - pt.lo < TILE ? pt.it.end - pt.lo : TILE);
  pt.agg = 0;
}

// One bulk copy of the tile's keys, rounded out to whole 16-byte blocks (they hold
// classified keys, so the copy stays inside the buffer's allocation).
template <typename K>
__device__ __forceinline__ void pipe_issue(const SortParams &p, const PipeTile &pt, K *sdst,
                                           unsigned long long *bar) {
  constexpr int VEC = Vec<K>::N;
  const K *src = static_cast<const K *>((pt.it.flags & kItemScratch) ? p.scratch : p.keys);
  const unsigned bytes = (unsigned)((pt.vhi + VEC - 1) / VEC * VEC) * (unsigned)sizeof(K);
  fence_proxy_async();  // earlier generic accesses before the async-proxy copy
  mbar_expect_tx(bar, bytes);
  bulk_g2s(sdst, src + pt.lo, bytes, bar);
}

template <typename K, int TILE>
constexpr size_t pipe_smem_bytes() { return (size_t)3 * TILE * sizeof(K) + 16; }  // + copy_out_v room

// ----------------------------------------------------------------------------- warp roles
// Named barriers (0 is __syncthreads): bar.arrive / bar.sync between warp groups.
__device__ __forceinline__ void nbar_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void nbar_arrive(int id, int count) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}
// bar.sync with an OR over the participants' predicates (the same result in all of them).
__device__ __forceinline__ bool nbar_or(int id, int count, bool pred) {
  unsigned out;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 q, %1, 0;\n\t"
      "bar.red.or.pred p, %2, %3, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(out)
      : "r"((unsigned)pred), "r"(id), "r"(count)
      : "memory");
  return out != 0;
}
__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// An arrival that orders nothing: for a barrier whose waiter needs no data from the
// arriving thread, only the fact that its earlier reads are done (whose results the
// thread has already used).
__device__ __forceinline__ void mbar_arrive_relaxed(unsigned long long *bar) {
  asm volatile("mbarrier.arrive.relaxed.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// `count` arrivals at once.
__device__ __forceinline__ void mbar_arrive_n(unsigned long long *bar, unsigned count) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
// Waits for phase `parity` of `bar`; gives up (false) after limit_ns or once the sort is
// aborted.
__device__ __forceinline__ bool mbar_wait_or_abort(unsigned long long *bar, unsigned parity,
                                                   unsigned long long limit_ns,
                                                   const unsigned *abort_flag) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  for (unsigned i = 1;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 31u) == 0u) {
      if (globaltimer() - t0 > limit_ns) return false;
      if (ld_relaxed(abort_flag) != 0u) return false;
    }
  }
}

// A tile staged in one input buffer (written by the load warp before its copy starts).
struct WsTile {
  Item it;
  long long h, lo;
  unsigned long long k;
  unsigned t;
  int vlo, vhi;
  int end;  // 1: no more tiles, 2: aborted
};

// What the look-back warp needs of a counted tile (written by the first data thread).
struct WsCur {
  Item it;
  long long h, lo;
  unsigned long long k;
  unsigned t;
  unsigned L, G;
  int stop;
  int agg;  // the data warps published the aggregate already (early count)
};

// Records that two consecutive tiles use at once are indexed by tile parity.
template <int ND>
struct WsShared {
  unsigned wl[ND], wg[ND];
  WsCur cur[2];
  unsigned long long E[2];
  int abort[2];
  WsTile rec[2];
  unsigned long long full[2], empty[2];
  unsigned long long cidx[2], ct0[2];
  unsigned ctiles[2];
  long long ch;  // item cached in `ci` (load warp)
  Item ci;
};

// Named barriers; the count and prefix barriers come in two copies, one per tile parity.
constexpr int kWsBarStart = 1, kWsBarData = 2, kWsBarCnt = 3 /* and 4 */, kWsBarE = 5 /* and 6 */,
              kWsBarWritten = 7;

template <typename K, int TILE>
constexpr size_t ws_smem_bytes() { return (size_t)3 * TILE * sizeof(K) + 16; }  // + copy_out_v room

// Phase 1, warp-specialised form of tile_kernel: the same tile passes, Steps and
// output, by three groups of warps of one CTA that wait on each other only through
// named barriers and mbarriers:
//   warp 1 (load)      claims tickets in order, waits until each is issued, and starts
//                      one bulk copy of the tile's keys into the input buffer the data
//                      warps last released (two buffers, full/empty mbarriers). It may
//                      block on a ticket that is not issued yet without stopping the
//                      other warps, which finish the tiles already loaded.
//   warps 2.. (data)   count a tile in shared memory (Step 3), publish its totals,
//                      scatter it into the output tile, and, once the look-back warp has
//                      its prefix, write both sides out. While the look-back runs they
//                      count the next tile early, if its keys have landed, and publish its
//                      aggregate, so that later tiles' look-backs find it sooner.
//   warp 0 (look-back) publishes each tile's aggregate and runs its look-back; once the
//                      data warps have written the tile it runs the completion atomic
//                      (whose release waits for the tile's stores): the last tile of an
//                      item places the key (Step 4) and queues both sides (Steps 5-6).
// The completion of tile i (warp 0) overlaps the loading and counting of tile i+1
// (data warps). Dynamic shared memory: two input tiles and the output tile.
template <typename K, int NT, int IPT>
__global__ void __launch_bounds__(NT, tile_min_blocks(NT)) tile_ws_kernel(SortParams p) {
  constexpr int ND = NT / 32 - 2;  // data warps
  constexpr int NTD = ND * 32;     // data threads
  constexpr int TILE = NTD * IPT;
  constexpr int VEC = Vec<K>::N;
  constexpr int NV = IPT / VEC;
  static_assert(IPT % VEC == 0 && IPT <= 32 && ND >= 2, "bad tile shape");
  using V = typename Vec<K>::T;
  extern __shared__ __align__(128) unsigned char ws_smem[];
  K *const sin0 = reinterpret_cast<K *>(ws_smem);  // input tiles 0, 1
  K *const sout0 = sin0 + 2 * TILE;                // output tile
  __shared__ WsShared<ND> sh;
  K *const buf0 = static_cast<K *>(p.keys);
  Control *ctl = p.ctl;
  grid_dep_wait();
  grid_dep_launch();
  const unsigned epoch = *reinterpret_cast<volatile unsigned *>(&ctl->epoch);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;

  if (tid == 0) {
    mbar_init(&sh.full[0], 1);
    mbar_init(&sh.full[1], 1);
    mbar_init(&sh.empty[0], ND);
    mbar_init(&sh.empty[1], ND);
    fence_mbar_init();
    sh.ch = -1;
  }
  __syncthreads();  // the only CTA-wide barrier

  if (w == 1) {
    // ------------------------------------------------------------------ load warp
    unsigned eph = 0;       // bit j: parity of the next release of buffer j
    int fills[2] = {0, 0};  // copies started into buffer j
    int j = 0;
    while (true) {
      if (fills[j] > 0) {
        // the data warps release buffer j once they hold its keys in registers
        const bool ok = mbar_wait_or_abort(&sh.empty[j], (eph >> j) & 1u, p.spin_limit_ns,
                                           &ctl->abort);
        eph ^= 1u << j;
        if (!ok) break;  // the consumers stopped (abort or an error elsewhere)
      }
      int stop = 0;
      if (lane == 0) {
        const unsigned long long k = atomicAdd(&ctl->tq_head, 1ull);
        trace_mark(p, k, 0);  // claimed
        long long h = 0;
        const int r = wait_ticket(p, epoch, k, &h);
        WsTile &rc = sh.rec[j];
        if (r > 0) {
          if (h != sh.ch) {
            load_item(p.items + h, &sh.ci);
            sh.ch = h;
          }
          rc.it = sh.ci;
          const K *src = static_cast<const K *>((rc.it.flags & kItemScratch) ? p.scratch : p.keys);
          rc.k = k;
          rc.h = h;
          rc.t = (unsigned)(k - rc.it.lb);
          rc.lo = tile_base(src, rc.it.begin) + (long long)rc.t * TILE;
          const long long first = rc.it.begin + 1;
          rc.vlo = (int)(first > rc.lo ? first - rc.lo : 0);
          rc.vhi = (int)(rc.it.end - rc.lo < TILE ? rc.it.end - rc.lo : TILE);
          rc.end = 0;
          // whole 16-byte blocks that hold classified keys: inside the buffer's allocation
          const unsigned bytes = (unsigned)((rc.vhi + VEC - 1) / VEC * VEC) * (unsigned)sizeof(K);
          fence_proxy_async();  // earlier generic accesses before the async-proxy copy
          mbar_expect_tx(&sh.full[j], bytes);
          bulk_g2s(sin0 + j * TILE, src + rc.lo, bytes, &sh.full[j]);
          trace_mark(p, k, 1);  // copy issued
        } else {
          rc.end = r == 0 ? 1 : 2;
          mbar_expect_tx(&sh.full[j], 0u);  // completes the phase without a copy
          stop = 1;
        }
      }
      stop = __shfl_sync(kFull, stop, 0);
      ++fills[j];
      if (stop) break;
      j ^= 1;
    }
    // a copy still in flight lands before the CTA may leave (bounded)
    if (lane == 0) {
      for (int q = 0; q < 2; ++q)
        if (fills[q] > 0) mbar_wait(&sh.full[q], (unsigned)(fills[q] - 1) & 1u, p.spin_limit_ns);
    }
    return;
  }

  if (w == 0) {
    // ------------------------------------------------------------------ look-back warp
    unsigned long long st_tiles = 0, st_lb = 0, st_large = 0, st_large_keys = 0;
    int par = 0;  // parity of the current tile
    while (true) {
      if (par) nbar_sync(kWsBarCnt + 1, NTD + 32);  // the data warps counted the tile
      else nbar_sync(kWsBarCnt, NTD + 32);
      const WsCur c = sh.cur[par];
      if (c.stop) break;
      unsigned long long *lb = p.lb + c.it.lb;
      if (lane == 0) {
        if (!c.agg) st_relaxed(&lb[c.t], lb_pack(epoch, c.t == 0, c.L));  // aggregate
        trace_mark(p, c.k, 2);
      }
      unsigned long long E = 0;
      int status = 0;
      if (c.t > 0) {
        unsigned long long steps = 0;
        status = lookback(lb, c.t, epoch, p.spin_limit_ns, &ctl->abort, &E, &steps);
        if (lane == 0) {
          if (status == 0) st_relaxed(&lb[c.t], lb_pack(epoch, true, (unsigned)(E + c.L)));
          st_lb += steps;
        }
      }
      if (lane == 0) {
        if (status == 1) raise_error(ctl, kDevTimeout, 0x100000000ull | c.t);
        sh.E[par] = E;
        sh.abort[par] = status == 0 ? 0 : 1;
        trace_mark(p, c.k, 3);
      }
      if (par) nbar_arrive(kWsBarE + 1, NTD + 32);
      else nbar_arrive(kWsBarE, NTD + 32);
      if (status != 0) break;  // the data warps see the abort and stop too
      nbar_sync(kWsBarWritten, NTD + 32);  // the data warps wrote the tile
      const unsigned cpar = c.it.flags & kItemScratch;
      K *dst = cpar ? buf0 : static_cast<K *>(p.scratch);
      int last = 0;
      if (lane == 0) {
        trace_mark(p, c.k, 4);
        ++st_tiles;
        if (c.t == c.it.tiles - 1) atomicExch(&p.ictl[c.h].less, E + c.L);
        // release: the tile's writes (ordered before by the named barrier) and `less`
        // become visible to whichever CTA observes the count reaching tiles
        const unsigned done_before = atom_add_release(&p.ictl[c.h].done, 1u);
        last = done_before == c.it.tiles - 1;
        sh.ctiles[0] = sh.ctiles[1] = 0;
        if (last) {
          __threadfence();
          const unsigned long long cc = ld_acquire(&p.ictl[c.h].less);
          const long long kpos = c.it.begin + (long long)cc;
          const K key = bits_key<K>(c.it.key);
          if (kpos >= c.it.end) {
            raise_error(ctl, kDevInternal, 0x700000000ull | (unsigned)c.h);
          } else if (c.it.flags & kItemPartitionOnly) {
            dst[kpos] = key;  // a single partition: the key index is the result
            if (p.key_index) *p.key_index = (long long)cc;
          } else {
            buf0[kpos] = key;  // Step 4
            const unsigned cflags = cpar ^ kItemScratch;
            const long long cb[2] = {c.it.begin, kpos + 1};
            const long long ce[2] = {kpos, c.it.end};
#pragma unroll
            for (int s = 0; s < 2; ++s) {  // Steps 5-6
              const long long mm = ce[s] - cb[s];
              if (mm == 1) {
                if (cflags & kItemScratch) buf0[cb[s]] = __ldcg(dst + cb[s]);
              } else if (mm >= 2) {
                unsigned long long t0 = 0;
                unsigned tiles = 0;
                sh.cidx[s] = reserve_item<K, TILE>(p, epoch, cb[s], ce[s], cflags, &t0, &tiles);
                sh.ct0[s] = t0;
                sh.ctiles[s] = tiles;
              }
            }
          }
        }
      }
      last = __shfl_sync(kFull, last, 0);
      if (last) {
        __syncwarp();
#pragma unroll
        for (int s = 0; s < 2; ++s)
          if (sh.ctiles[s]) publish_tickets(p, epoch, sh.cidx[s], sh.ct0[s], sh.ctiles[s], lane, 32);
        __syncwarp();
        if (lane == 0) {
          ++st_large;
          st_large_keys += (unsigned long long)(c.it.end - c.it.begin);
          __threadfence();
          atomicAdd(&ctl->large_completed, 1ull);
        }
      }
      if (lane == 0) {
        trace_mark(p, c.k, 6);  // completed
        if (p.trace && c.k < (unsigned long long)p.trace_cap)
          p.trace[c.k * kTraceWords + 7] = blockIdx.x;
      }
      par ^= 1;
    }
    if (lane == 0) {
      if (st_tiles) atomicAdd(&ctl->tiles, st_tiles);
      if (st_lb) atomicAdd(&ctl->lookback_steps, st_lb);
      if (st_large) atomicAdd(&ctl->large_items, st_large);
      if (st_large_keys) atomicAdd(&ctl->large_keys, st_large_keys);
    }
    return;
  }

  // -------------------------------------------------------------------- data warps
  const int dt = tid - 64, dw = w - 2;
  unsigned fph = 0;   // bit j: parity of the next completion of input buffer j
  int b = 0;          // input buffer of the current tile
  int par = 0;        // parity of the current tile (its records and barriers)
  int early = 0;      // the current tile's aggregate was published by an early count
  while (true) {
    const bool landed = mbar_wait(&sh.full[b], (fph >> b) & 1u, 4 * p.spin_limit_ns);
    fph ^= 1u << b;
    const WsTile rc = sh.rec[b];
    // the same decision in every data warp: stop on the end of the tiles, an abort or a
    // copy that never landed
    if (nbar_or(kWsBarStart, NTD, !landed || rc.end != 0)) {
      if (dt == 0) {
        if (!landed) raise_error(ctl, kDevTimeout, 0x800000000ull);
        sh.cur[par].stop = 1;
      }
      if (par) nbar_arrive(kWsBarCnt + 1, NTD + 32);  // lets the look-back warp see the stop
      else nbar_arrive(kWsBarCnt, NTD + 32);
      break;
    }
    K *const sin = sin0 + b * TILE;
    const K key = bits_key<K>(rc.it.key);  // Step 1: the first element is the key
    K x[IPT];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const V q = *reinterpret_cast<const V *>(sin + (v * NTD + dt) * VEC);
      if constexpr (VEC == 4) {
        x[v * 4 + 0] = q.x; x[v * 4 + 1] = q.y; x[v * 4 + 2] = q.z; x[v * 4 + 3] = q.w;
      } else {
        x[v * 2 + 0] = q.x; x[v * 2 + 1] = q.y;
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&sh.empty[b]);  // this warp's keys are in registers
    // ---- count (Step 3)
    unsigned lessbits = 0, gebits = 0;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
#pragma unroll
      for (int l = 0; l < VEC; ++l) {
        const int jx = v * VEC + l, kk = (v * NTD + dt) * VEC + l;
        const bool valid = kk >= rc.vlo && kk < rc.vhi;
        const bool le = goes_left(key, x[jx]);
        lessbits |= (unsigned)(valid && le) << jx;
        gebits |= (unsigned)(valid && !le) << jx;
      }
    }
    const unsigned mine = (unsigned)__popc(lessbits) | ((unsigned)__popc(gebits) << 16);
    unsigned incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned u = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += u;
    }
    if (lane == 31) {
      sh.wl[dw] = incl & 0xffffu;
      sh.wg[dw] = incl >> 16;
    }
    nbar_sync(kWsBarData, NTD);
    unsigned L = 0, G = 0, wlx = 0, wgx = 0;
#pragma unroll
    for (int i = 0; i < ND; ++i) {
      const unsigned a = sh.wl[i], c = sh.wg[i];
      if (i < dw) {
        wlx += a;
        wgx += c;
      }
      L += a;
      G += c;
    }
    if (dt == 0) {
      WsCur &c = sh.cur[par];
      c.it = rc.it;
      c.h = rc.h;
      c.lo = rc.lo;
      c.k = rc.k;
      c.t = rc.t;
      c.L = L;
      c.G = G;
      c.stop = 0;
      c.agg = early;
    }
    if (par) nbar_arrive(kWsBarCnt + 1, NTD + 32);
    else nbar_arrive(kWsBarCnt, NTD + 32);
    // ---- scatter into the output tile (its last readers wrote it out before the data
    // warps reached kWsBarData above)
    scatter_keys<K, IPT>(sout0, x, lessbits, gebits, wlx, L + wgx, incl - mine);
    // ---- while the look-back runs: count the next tile early if its keys have landed,
    // and publish its aggregate, so that later tiles' look-backs find it sooner
    {
      const unsigned nb = b ^ 1;
      const bool have = mbar_test(&sh.full[nb], (fph >> nb) & 1u);
      early = 0;
      if (!nbar_or(kWsBarStart, NTD, !have)) {
        const WsTile &rn = sh.rec[nb];
        if (rn.end == 0) {
          const K nkey = bits_key<K>(rn.it.key);
          const K *snb = sin0 + nb * TILE;
          unsigned cnt = 0;
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            const V q = *reinterpret_cast<const V *>(snb + (v * NTD + dt) * VEC);
            K y[VEC];
            if constexpr (VEC == 4) {
              y[0] = q.x; y[1] = q.y; y[2] = q.z; y[3] = q.w;
            } else {
              y[0] = q.x; y[1] = q.y;
            }
#pragma unroll
            for (int l = 0; l < VEC; ++l) {
              const int kk = (v * NTD + dt) * VEC + l;
              cnt += (kk >= rn.vlo && kk < rn.vhi && goes_left(nkey, y[l])) ? 1u : 0u;
            }
          }
          cnt = __reduce_add_sync(kFull, cnt);
          if (lane == 0) sh.wl[dw] = cnt;  // every data warp read its prefixes above
          nbar_sync(kWsBarData, NTD);
          if (dt == 0) {
            unsigned tot = 0;
#pragma unroll
            for (int i = 0; i < ND; ++i) tot += sh.wl[i];
            st_relaxed(&p.lb[rn.it.lb + rn.t], lb_pack(epoch, rn.t == 0, tot));
            trace_mark(p, rn.k, 5);  // aggregate published early
          }
          early = 1;
        }
      }
    }
    // ---- the prefix, then write both sides
    if (par) nbar_sync(kWsBarE + 1, NTD + 32);  // all scatters done, prefix known
    else nbar_sync(kWsBarE, NTD + 32);
    if (sh.abort[par]) break;
    const unsigned long long E = sh.E[par];
    long long lbase = 0, gbase = 0;
    K *dst = (rc.it.flags & kItemScratch) ? buf0 : static_cast<K *>(p.scratch);
    if (!tile_dest(rc.it.begin, rc.it.end, rc.lo, rc.t, E, L, G, &lbase, &gbase)) {
      // impossible prefixes: record, and write nothing (the other warps decide the same)
      if (dt == 0) raise_error(ctl, kDevInternal, 0x500000000ull | rc.t);
    } else {
      copy_out_v<K, NTD>(sout0, dst + lbase, L, dt);
      copy_out_v<K, NTD>(sout0 + L, dst + gbase, G, dt);
    }
    nbar_arrive(kWsBarWritten, NTD + 32);
    par ^= 1;
    b ^= 1;
  }
}

// ----------------------------------------------------------------------------- partition
// One partition (Steps 1-4) of buffer 0's [0, total) into buffer 1, in a single launch
// and without the work queue: CTA c handles tiles c, c + G, c + 2G, ... of the one item,
// so every CTA knows its next tile in advance and stages it into shared memory by a bulk
// copy while the current tile is finished. Per tile: count in shared memory (Step 3),
// publish the aggregate, decoupled look-back by warp 0 while the other warps scatter and
// count the CTA's next tile early (publishing its aggregate too), then write both sides.
// The tile that holds the last keys learns the total less count from its own look-back
// and places the key there (Step 4): no per-tile completion count is needed.
// The generation (epoch) is the workspace's next one; the last CTA to finish makes it
// the current one and clears the partition's own stop flag and CTA count.
// Dynamic shared memory: two input tiles and the output tile.
template <typename K, int NT, int IPT>
__global__ void __launch_bounds__(NT, tile_min_blocks(NT)) part_kernel(SortParams p) {
  constexpr int TILE = NT * IPT;
  constexpr int VEC = Vec<K>::N;
  constexpr int NV = IPT / VEC;
  constexpr int NW = NT / 32;
  static_assert(IPT % VEC == 0 && IPT <= 32 && NT % 32 == 0 && NW > 1, "bad tile shape");
  using V = typename Vec<K>::T;
  extern __shared__ __align__(128) unsigned char part_smem[];
  K *const sin0 = reinterpret_cast<K *>(part_smem);
  K *const sout = sin0 + 2 * TILE;
  __shared__ unsigned wl[NW], wg[NW];
  __shared__ unsigned long long bar[2];
  __shared__ unsigned long long sE;
  __shared__ int sabort, sfail;
  __shared__ unsigned early_L;
  Control *ctl = p.ctl;
  unsigned epoch = *reinterpret_cast<volatile unsigned *>(&ctl->epoch) + 1u;
  if (epoch == 0u || epoch >= kMaxEpoch) epoch = 1u;
  const K *const src = static_cast<const K *>(p.keys);
  K *const dst = static_cast<K *>(p.scratch);
  const long long n = p.total;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int G = gridDim.x;
  const long long base = tile_base(src, 0);  // the key is src[0]; tiles start here
  const long long tiles = (n - base + TILE - 1) / TILE;
  const K key = __ldcg(src);  // Step 1: the first element is the key
  unsigned long long *lb = p.lb;
  unsigned long long st_lb = 0;

  auto geom = [&](long long t, int *vlo, int *vhi, long long *lo) {
    *lo = base + t * TILE;
    *vlo = (int)(1 > *lo ? 1 - *lo : 0);
    *vhi = (int)(n - *lo < TILE ? n - *lo : TILE);
  };
  auto issue = [&](long long t, int j) {
    int vlo, vhi;
    long long lo;
    geom(t, &vlo, &vhi, &lo);
    const unsigned bytes = (unsigned)((vhi + VEC - 1) / VEC * VEC) * (unsigned)sizeof(K);
    fence_proxy_async();
    mbar_expect_tx(&bar[j], bytes);
    bulk_g2s(sin0 + j * TILE, src + lo, bytes, &bar[j]);
  };

  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
    sfail = 0;
    early_L = 0;
    if (blockIdx.x < tiles) issue(blockIdx.x, 0);
    if (blockIdx.x + G < tiles) issue(blockIdx.x + G, 1);
  }
  __syncthreads();
  unsigned phase = 0;
  int b = 0, early = 0;
  // on a stop, the copies still in flight: this tile's (if it never landed) and the next
  int drain_cur = 0, drain_next = 0;
  for (long long t = blockIdx.x; t < tiles; t += G) {
    if (tid == 0) trace_mark(p, (unsigned long long)t, 0);  // tile starts
    const bool landed = mbar_wait(&bar[b], (phase >> b) & 1u, p.spin_limit_ns);
    phase ^= 1u << b;
    if (tid == 0) trace_mark(p, (unsigned long long)t, 1);  // keys in shared memory
    int vlo, vhi;
    long long lo;
    geom(t, &vlo, &vhi, &lo);
    const K *sin = sin0 + b * TILE;
    K x[IPT];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const V q = *reinterpret_cast<const V *>(sin + (v * NT + tid) * VEC);
      if constexpr (VEC == 4) {
        x[v * 4 + 0] = q.x; x[v * 4 + 1] = q.y; x[v * 4 + 2] = q.z; x[v * 4 + 3] = q.w;
      } else {
        x[v * 2 + 0] = q.x; x[v * 2 + 1] = q.y;
      }
    }
    unsigned lessbits = 0, gebits = 0;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
#pragma unroll
      for (int l = 0; l < VEC; ++l) {
        const int jx = v * VEC + l, kk = (v * NT + tid) * VEC + l;
        const bool valid = kk >= vlo && kk < vhi;
        const bool le = goes_left(key, x[jx]);
        lessbits |= (unsigned)(valid && le) << jx;
        gebits |= (unsigned)(valid && !le) << jx;
      }
    }
    const unsigned mine = (unsigned)__popc(lessbits) | ((unsigned)__popc(gebits) << 16);
    unsigned incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned u = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += u;
    }
    if (lane == 31) {
      wl[w] = incl & 0xffffu;
      wg[w] = incl >> 16;
    }
    const bool has_next = t + G < tiles;
    if (__syncthreads_or(!landed)) {
      if (tid == 0) {
        raise_error(ctl, kDevTimeout, 0x900000000ull | (unsigned)t);
        atomicExch(&ctl->part_abort, 1u);
      }
      drain_cur = landed ? 0 : 1;
      drain_next = has_next ? 1 : 0;
      break;
    }
    unsigned L = 0, Gc = 0, wlx = 0, wgx = 0;
#pragma unroll
    for (int i = 0; i < NW; ++i) {
      const unsigned a = wl[i], c = wg[i];
      if (i < w) {
        wlx += a;
        wgx += c;
      }
      L += a;
      Gc += c;
    }
    const unsigned tt = (unsigned)t;
    if (tid == 0 && !early) st_relaxed(&lb[tt], lb_pack(epoch, tt == 0, L));
    if (tid == 0) trace_mark(p, (unsigned long long)t, 2);  // counted
    if (w == 0) {
      unsigned long long E = 0;
      int status = 0;
      if (tt > 0) {
        unsigned long long steps = 0;
        // (measured: wider windows cost more than the steps they save)
        status = lookback<KSORT_PART_LOOKBACK_PER>(lb, tt, epoch, p.spin_limit_ns,
                                                   &ctl->part_abort, &E, &steps);
        if (lane == 0) {
          if (status == 0) st_relaxed(&lb[tt], lb_pack(epoch, true, (unsigned)(E + L)));
          st_lb += steps;
        }
      }
      if (lane == 0) {
        if (status == 1) {
          raise_error(ctl, kDevTimeout, 0x100000000ull | tt);
          atomicExch(&ctl->part_abort, 1u);
        }
        sE = E;
        sabort = status == 0 ? 0 : 1;
        trace_mark(p, (unsigned long long)t, 3);  // look-back done
      }
    }
    scatter_keys<K, IPT>(sout, x, lessbits, gebits, wlx, L + wgx, incl - mine);
    // the other warps: count the next tile early if its keys have landed
    const long long tn = t + G;
    early = 0;
    if (w > 0 && tn < tiles) {
      const bool ok = mbar_test(&bar[b ^ 1], (phase >> (b ^ 1)) & 1u);
      if (__all_sync(kFull, ok)) {
        int nvlo, nvhi;
        long long nlo;
        geom(tn, &nvlo, &nvhi, &nlo);
        const K *snx = sin0 + (b ^ 1) * TILE;
        unsigned cnt = 0;
        for (int v = tid - 32; v < TILE / VEC; v += NT - 32) {
          const V q = *reinterpret_cast<const V *>(snx + v * VEC);
          K y[VEC];
          if constexpr (VEC == 4) {
            y[0] = q.x; y[1] = q.y; y[2] = q.z; y[3] = q.w;
          } else {
            y[0] = q.x; y[1] = q.y;
          }
#pragma unroll
          for (int l = 0; l < VEC; ++l) {
            const int kk = v * VEC + l;
            cnt += (kk >= nvlo && kk < nvhi && goes_left(key, y[l])) ? 1u : 0u;
          }
        }
        cnt = __reduce_add_sync(kFull, cnt);
        if (lane == 0) atomicAdd(&early_L, cnt);
      } else if (lane == 0) {
        sfail = 1;
      }
      asm volatile("bar.sync 1, %0;" ::"r"(NT - 32) : "memory");
      if (tid == 32 && !sfail) {
        st_relaxed(&lb[(unsigned)tn], lb_pack(epoch, (unsigned)tn == 0, early_L));
        trace_mark(p, (unsigned long long)tn, 5);  // aggregate published early
      }
    }
    __syncthreads();
    if (tn < tiles) early = !sfail;  // the same value in every thread
    if (sabort) {
      drain_next = has_next ? 1 : 0;
      break;
    }
    const unsigned long long E = sE;
    // write: less keys from the front, >= keys from the back (the key's slot stays free)
    const long long PV = tt == 0 ? 0 : lo - 1;  // classified keys in earlier tiles
    const long long lbase = (long long)E, gbase = n - (PV - (long long)E) - (long long)Gc;
    if (lbase < 0 || lbase + L > n || gbase < 1 || gbase + Gc > n) {
      if (tid == 0) {
        raise_error(ctl, kDevInternal, 0x500000000ull | tt);
        atomicExch(&ctl->part_abort, 1u);
      }
      drain_next = has_next ? 1 : 0;
      break;
    }
    copy_out_v<K, NT>(sout, dst + lbase, L, tid);
    copy_out_v<K, NT>(sout + L, dst + gbase, Gc, tid);
    if (t == tiles - 1 && tid == 0) {
      const long long c = (long long)E + L;  // #{x < key}: Step 4
      dst[c] = key;
      if (p.key_index) *p.key_index = c;
    }
    // this buffer takes the tile after next (once every thread is done reading it)
    __syncthreads();
    if (tid == 0) {
      trace_mark(p, (unsigned long long)t, 4);  // written
      if (p.trace && (unsigned long long)t < (unsigned long long)p.trace_cap)
        p.trace[t * kTraceWords + 7] = blockIdx.x;
      sfail = 0;
      early_L = 0;
      if (t + 2 * (long long)G < tiles) issue(t + 2 * G, b);
    }
    b ^= 1;
  }
  // copies still in flight land before the CTA leaves (bounded); after a normal end none is
  if (tid == 0) {
    if (drain_cur) mbar_wait(&bar[b], ((phase >> b) & 1u) ^ 1u, p.spin_limit_ns);
    if (drain_next) mbar_wait(&bar[b ^ 1], (phase >> (b ^ 1)) & 1u, p.spin_limit_ns);
  }
  if (tid == 0) {
    if (st_lb) atomicAdd(&ctl->lookback_steps, st_lb);
    __threadfence();
    if (atomicAdd(&ctl->part_done, 1u) == (unsigned)G - 1u) {
      // every CTA has read the epoch: the next call gets the one after
      ctl->part_done = 0u;
      ctl->part_abort = 0u;
      ctl->epoch = epoch;
    }
  }
}

// ----------------------------------------------------------------------------- exact
// Steps 1-4 with the paper's own element order: the hole scheme of Step 3 (a front scan
// that moves each element below the key one place left and sends each element >= the key
// to the back hole, and a back scan that leaves elements >= the key in place and sends
// each element below the key to the front hole) has a closed form. Number the elements
// after the key 0..m-1; let F_t be the t-th element >= key from the front and B_t the
// t-th element < key from the back (0-based t), L = #{< key}, and T the number of t with
// F_t before B_t (a prefix of t: F_t is before B_t exactly when at least t+1 elements
// < key follow it). Then, as indices of the sub-array (the key was at 0):
//   the key goes to L;
//   B_t, t < T, goes to the index of F_t; every other element < key at k goes to k;
//   F_0 goes to L + 1 (Step 4's temp);
//   F_t, 1 <= t < T, goes to the index of B_{t-1} plus 1, and so does F_T when T >= 1 and
//   F_T comes before B_{T-1}; every other element >= key at k stays at k + 1.
// Four passes: tile counts, their scan (one CTA), per-element ranks (recording where each
// F_t and B_t is, and counting the pairs), and the placement.
constexpr int kExactThreads = 256, kExactIpt = 4, kExactTile = kExactThreads * kExactIpt;

template <typename K>
__global__ void __launch_bounds__(kExactThreads) exact_count_kernel(const K *a, long long m,
                                                                    unsigned *tile_less) {
  const K key = a[0];
  const K *b = a + 1;
  const long long g = blockIdx.x;
  const long long base = g * kExactTile + (long long)threadIdx.x * kExactIpt;
  unsigned c = 0;
#pragma unroll
  for (int i = 0; i < kExactIpt; ++i)
    if (base + i < m) c += goes_left(key, b[base + i]) ? 1u : 0u;
  c = __reduce_add_sync(kFull, c);
  __shared__ unsigned ws[kExactThreads / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned tot = 0;
    for (int w = 0; w < kExactThreads / 32; ++w) tot += ws[w];
    tile_less[g] = tot;
  }
}

// One CTA: ge_before[g] = elements >= key in tiles before g, less_after[g] = elements < key
// in tiles after g; *L_out = all elements < key.
template <int NT>
__global__ void __launch_bounds__(NT) exact_scan_kernel(const unsigned *tile_less,
                                                          long long tiles, long long m,
                                                          unsigned long long *ge_before,
                                                          unsigned long long *less_after,
                                                          unsigned long long *L_out) {
  __shared__ unsigned long long wsum[32], carry_ge, carry_less;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid == 0) {
    carry_ge = 0;
    carry_less = 0;
  }
  __syncthreads();
  // forward: ge counts
  for (long long c0 = 0; c0 < tiles; c0 += NT) {
    const long long g = c0 + tid;
    unsigned long long v = 0;
    if (g < tiles) {
      const long long sz = (g == tiles - 1) ? m - g * kExactTile : kExactTile;
      v = (unsigned long long)sz - tile_less[g];
    }
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long u = __shfl_up_sync(kFull, x, o);
      if (lane >= o) x += u;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    unsigned long long wb = 0;
    for (int i = 0; i < w; ++i) wb += wsum[i];
    if (g < tiles) ge_before[g] = carry_ge + wb + x - v;
    __syncthreads();
    if (tid == NT - 1) carry_ge += wb + x;
    __syncthreads();
  }
  // backward: less counts after each tile
  for (long long c0 = 0; c0 < tiles; c0 += NT) {
    const long long g = tiles - 1 - (c0 + tid);  // tid 0 takes the last tile
    const unsigned long long v = g >= 0 ? tile_less[g] : 0ull;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long u = __shfl_up_sync(kFull, x, o);
      if (lane >= o) x += u;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    unsigned long long wb = 0;
    for (int i = 0; i < w; ++i) wb += wsum[i];
    if (g >= 0) less_after[g] = carry_less + wb + x - v;
    __syncthreads();
    if (tid == NT - 1) carry_less += wb + x;
    __syncthreads();
  }
  if (tid == 0) *L_out = carry_less;
}

// Ranks inside a tile: element k's exclusive ge count and inclusive less count (thread
// i holds elements base + i*IPT ... + IPT - 1).
struct ExactRanks {
  unsigned ge_excl[kExactIpt], less_incl[kExactIpt];
  unsigned tile_less;
};
template <typename K>
__device__ __forceinline__ void exact_ranks(const K *b, long long m, K key, long long base,
                                            bool (&lf)[kExactIpt], bool (&valid)[kExactIpt],
                                            ExactRanks &r) {
  __shared__ unsigned wl[kExactThreads / 32], wg[kExactThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned nl = 0, ng = 0;
#pragma unroll
  for (int i = 0; i < kExactIpt; ++i) {
    valid[i] = base + i < m;
    lf[i] = valid[i] && goes_left(key, b[base + i]);
    nl += lf[i] ? 1u : 0u;
    ng += (valid[i] && !lf[i]) ? 1u : 0u;
  }
  unsigned xl = nl, xg = ng;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned ul = __shfl_up_sync(kFull, xl, o), ug = __shfl_up_sync(kFull, xg, o);
    if (lane >= o) {
      xl += ul;
      xg += ug;
    }
  }
  if (lane == 31) {
    wl[w] = xl;
    wg[w] = xg;
  }
  __syncthreads();
  unsigned bl = 0, bg = 0, tl = 0;
  for (int i = 0; i < kExactThreads / 32; ++i) {
    if (i < w) {
      bl += wl[i];
      bg += wg[i];
    }
    tl += wl[i];
  }
  unsigned cl = bl + xl - nl, cg = bg + xg - ng;  // before this thread
#pragma unroll
  for (int i = 0; i < kExactIpt; ++i) {
    r.ge_excl[i] = cg;
    cl += lf[i] ? 1u : 0u;
    r.less_incl[i] = cl;
    cg += (valid[i] && !lf[i]) ? 1u : 0u;
  }
  r.tile_less = tl;
}

template <typename K>
__global__ void __launch_bounds__(kExactThreads) exact_rank_kernel(
    const K *a, long long m, const unsigned long long *ge_before,
    const unsigned long long *less_after, int *Fpos, int *Bpos, unsigned long long *T_out) {
  const K key = a[0];
  const K *b = a + 1;
  const long long g = blockIdx.x;
  const long long base = g * kExactTile + (long long)threadIdx.x * kExactIpt;
  bool lf[kExactIpt], valid[kExactIpt];
  ExactRanks r;
  exact_ranks(b, m, key, base, lf, valid, r);
  unsigned pairs = 0;
#pragma unroll
  for (int i = 0; i < kExactIpt; ++i) {
    if (!valid[i]) continue;
    const long long k = base + i;
    const unsigned long long after = less_after[g] + (r.tile_less - r.less_incl[i]);
    if (lf[i]) {
      Bpos[after] = (int)k;  // B_t with t = #{< key after k}
    } else {
      const unsigned long long t = ge_before[g] + r.ge_excl[i];
      Fpos[t] = (int)k;  // F_t
      pairs += after >= t + 1 ? 1u : 0u;  // F_t before B_t
    }
  }
  pairs = __reduce_add_sync(kFull, pairs);
  if ((threadIdx.x & 31) == 0 && pairs) atomicAdd(T_out, (unsigned long long)pairs);
}

template <typename K>
__global__ void __launch_bounds__(kExactThreads) exact_place_kernel(
    const K *a, long long m, const unsigned long long *ge_before,
    const unsigned long long *less_after, const int *Fpos, const int *Bpos,
    const unsigned long long *T_in, const unsigned long long *L_in, K *out, long long *key_index) {
  const K key = a[0];
  const K *b = a + 1;
  const long long g = blockIdx.x;
  const long long base = g * kExactTile + (long long)threadIdx.x * kExactIpt;
  const unsigned long long T = *T_in, L = *L_in;
  bool lf[kExactIpt], valid[kExactIpt];
  ExactRanks r;
  exact_ranks(b, m, key, base, lf, valid, r);
#pragma unroll
  for (int i = 0; i < kExactIpt; ++i) {
    if (!valid[i]) continue;
    const long long k = base + i;
    long long dest;
    if (lf[i]) {
      const unsigned long long t = less_after[g] + (r.tile_less - r.less_incl[i]);
      dest = t < T ? (long long)Fpos[t] : k;
    } else {
      const unsigned long long t = ge_before[g] + r.ge_excl[i];
      if (t == 0) dest = (long long)L + 1;
      else if (t < T) dest = (long long)Bpos[t - 1] + 1;
      else if (t == T && k < (long long)Bpos[T - 1]) dest = (long long)Bpos[T - 1] + 1;
      else dest = k + 1;
    }
    out[dest] = b[k];
  }
  if (g == 0 && threadIdx.x == 0) {
    out[L] = key;  // Step 4
    if (key_index) *key_index = (long long)L;
  }
}

// ----------------------------------------------------------------------------- waves
// Level-synchronous tile passes (the wave form) for the upper recursion levels of a
// sort. The sub-arrays above the cutoff at one depth form the level's list; their
// classified keys (every element but the key, Step 3) are numbered consecutively along
// the list, the level's key space (WaveItem::koff), which is split into equal
// contiguous spans, one per CTA, across sub-array boundaries. A level is two launches:
//   count    each CTA counts the less keys of the first and of the last sub-array its
//            span touches, and publishes both counts;
//   scatter  each CTA takes the less keys before its span in its first sub-array from
//            the counts of the CTAs before it (which hold the rest of that sub-array),
//            then moves its keys tile by tile as tile_kernel does: less keys from the
//            left end, >= keys from the right end. The CTA holding a sub-array's last
//            key places its key (Step 4) and queues both sides (Steps 5-6): small sides
//            for the SMEM finisher, large sides on the next level's list.
// No CTA ever waits for another: the launches are ordered by the stream, and under
// programmatic dependent launch the next launch's CTAs start as this one's leave and
// wait (griddepcontrol.wait) until its memory is complete. After the last wave level,
// the remaining list is handed to tile_kernel's work queue.
// Placement of a key at an even level: the level reads buffer 0, where other CTAs of
// the same launch may still be reading the sub-array, so the key is recorded in
// wave_fin and written to buffer 0 by the next launch (an odd level's count, or the
// hand-off); odd levels read buffer 1 and write the key at once.

// Keys per CTA span: equal shares of the level, at least one tile each.
__device__ __forceinline__ long long wave_span(long long keys, int grid, int tile) {
  const long long per = (keys + grid - 1) / grid;
  return per < tile ? (long long)tile : per;
}

template <int NW>
struct WaveShared {
  unsigned wl[NW], wg[NW];
  unsigned long long red[NW];
  int find[8];
};

// Whole CTA: the list item whose key-space range holds s (koff increases along the
// list, items[0].koff = 0). Each round probes NT evenly spaced items, so m items take
// ceil(log_NT m) rounds.
template <int NT, int NW>
__device__ __forceinline__ long long wave_find(const WaveItem *items, long long m, long long s,
                                               WaveShared<NW> &sh) {
  if (threadIdx.x < 8) sh.find[threadIdx.x] = 0;
  __syncthreads();
  long long lo = 0, hi = m;
  for (int r = 0; hi - lo > 1 && r < 8; ++r) {
    const long long step = (hi - lo + NT - 1) / NT;
    const long long idx = lo + (long long)threadIdx.x * step;
    if (threadIdx.x > 0 && idx < hi && __ldcg(&items[idx].koff) <= s)
      atomicMax(&sh.find[r], (int)threadIdx.x);
    __syncthreads();
    lo += (long long)sh.find[r] * step;
    hi = min(hi, lo + step);
  }
  return lo;
}

// Sum over the CTA (every thread gets it); two barriers.
template <int NW>
__device__ __forceinline__ unsigned long long wave_sum(unsigned long long v, WaveShared<NW> &sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  if ((threadIdx.x & 31) == 0) sh.red[threadIdx.x >> 5] = v;
  __syncthreads();
  unsigned long long t = 0;
#pragma unroll
  for (int i = 0; i < NW; ++i) t += sh.red[i];
  __syncthreads();
  return t;
}

// Keys [vlo, vhi) of the tile at src + lo (16-byte aligned) into registers; thread i
// holds tile positions (v * NT + i) * VEC + l. Whole vectors inside the range move
// with 128-bit loads, the edges one key at a time; nothing outside the range is read.
template <typename K, int NT, int IPT>
__device__ __forceinline__ void wave_load(const K *src, long long lo, int vlo, int vhi,
                                          K (&x)[IPT]) {
  constexpr int VEC = Vec<K>::N, NV = IPT / VEC;
  using V = typename Vec<K>::T;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const int k0 = (v * NT + (int)threadIdx.x) * VEC;
    if (k0 >= vlo && k0 + VEC <= vhi) {
      const V q = __ldcg(reinterpret_cast<const V *>(src + lo + k0));
      if constexpr (VEC == 4) {
        x[v * 4 + 0] = q.x; x[v * 4 + 1] = q.y; x[v * 4 + 2] = q.z; x[v * 4 + 3] = q.w;
      } else {
        x[v * 2 + 0] = q.x; x[v * 2 + 1] = q.y;
      }
    } else {
#pragma unroll
      for (int l = 0; l < VEC; ++l) {
        const int k = k0 + l;
        x[v * VEC + l] = (k >= vlo && k < vhi) ? __ldcg(src + lo + k) : K(0);
      }
    }
  }
}

// Keys recorded by the last even level go to their final index in buffer 0.
template <typename K>
__device__ __forceinline__ void wave_place_late_keys(const SortParams &p) {
  unsigned long long n = __ldcg(&p.ctl->wave_fin);
  if (n > p.wave_cap) n = p.wave_cap;  // an overflow was reported when it happened
  K *buf0 = static_cast<K *>(p.keys);
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += stride)
    buf0[__ldcg(&p.wave_fin[2 * i])] = bits_key<K>(__ldcg(&p.wave_fin[2 * i + 1]));
}

// The level's list, its key count, and this CTA's span [*s0, *s1); false: no work.
__device__ __forceinline__ bool wave_level_span(const SortParams &p, int level, int tile,
                                                long long *m, long long *per, long long *s0,
                                                long long *s1) {
  const unsigned long long ctr = __ldcg(&p.ctl->wave_ctr[level & 1]);
  *m = (long long)(ctr >> kWaveKeyBits);
  const long long keys = (long long)(ctr & kWaveKeyMask);
  if (*m == 0 || *m > (long long)p.wave_cap || __ldcg(&p.ctl->abort) != 0u) return false;
  *per = wave_span(keys, (int)gridDim.x, tile);
  *s0 = (long long)blockIdx.x * *per;
  *s1 = min(*s0 + *per, keys);
  return *s0 < keys;
}

template <typename K, int NT, int IPT>
__global__ void __launch_bounds__(NT, tile_min_blocks(NT)) wave_count_kernel(SortParams p,
                                                                             int level) {
  constexpr int TILE = NT * IPT, VEC = Vec<K>::N, NV = IPT / VEC, NW = NT / 32;
  __shared__ WaveShared<NW> sh;
  grid_dep_wait();
  grid_dep_launch();
  Control *ctl = p.ctl;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl->wave_ctr[(level + 1) & 1] = 0ull;  // the next level's list starts empty
    if ((level & 1) == 0) ctl->wave_fin = 0ull;
  }
  if (level & 1) wave_place_late_keys<K>(p);
  long long m = 0, per = 0, s0 = 0, s1 = 0;
  if (!wave_level_span(p, level, TILE, &m, &per, &s0, &s1)) return;
  const WaveItem *items = p.wave_items + (size_t)(level & 1) * p.wave_cap;
  const K *src = static_cast<const K *>((level & 1) ? p.scratch : p.keys);
  long long h = wave_find<NT, NW>(items, m, s0, sh);
  unsigned long long first_cnt = 0, last_cnt = 0;
  bool first_seg = true;
  for (long long s = s0; s < s1 && h < m; ++h) {
    const long long begin = __ldcg(&items[h].begin), end = __ldcg(&items[h].end);
    const long long koff = __ldcg(&items[h].koff);
    const long long a = s - koff, b = min(s1 - koff, end - begin - 1);  // item offsets
    const K key = __ldcg(src + begin);  // Step 1
    const long long f = begin + 1, base = tile_base(src, begin);
    unsigned cnt = 0;
    for (long long lo = base + ((f + a - base) / TILE) * TILE; lo < f + b; lo += TILE) {
      const int vlo = (int)max(f + a - lo, 0ll), vhi = (int)min(f + b - lo, (long long)TILE);
      K x[IPT];
      wave_load<K, NT, IPT>(src, lo, vlo, vhi, x);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
#pragma unroll
        for (int l = 0; l < VEC; ++l) {
          const int k = (v * NT + (int)threadIdx.x) * VEC + l;
          cnt += (k >= vlo && k < vhi && goes_left(key, x[v * VEC + l])) ? 1u : 0u;  // Step 3
        }
      }
    }
    const unsigned long long c = wave_sum<NW>(cnt, sh);
    if (first_seg) first_cnt = c;
    last_cnt = c;
    first_seg = false;
    s = koff + b;
  }
  if (threadIdx.x == 0) {
    p.wave_cnt[2 * blockIdx.x] = first_cnt;
    p.wave_cnt[2 * blockIdx.x + 1] = last_cnt;
  }
}

template <typename K, int NT, int IPT>
__global__ void __launch_bounds__(NT, tile_min_blocks(NT)) wave_scatter_kernel(SortParams p,
                                                                               int level) {
  constexpr int TILE = NT * IPT, VEC = Vec<K>::N, NV = IPT / VEC, NW = NT / 32;
  static_assert(IPT % VEC == 0 && IPT <= 32 && NT % 32 == 0, "bad tile shape");
  __shared__ __align__(16) K sout[TILE + VEC];  // + room for copy_out_v's reads
  __shared__ WaveShared<NW> sh;
  grid_dep_wait();
  grid_dep_launch();
  Control *ctl = p.ctl;
  long long m = 0, per = 0, s0 = 0, s1 = 0;
  if (!wave_level_span(p, level, TILE, &m, &per, &s0, &s1)) return;
  const unsigned epoch = *reinterpret_cast<volatile unsigned *>(&ctl->epoch);
  const WaveItem *items = p.wave_items + (size_t)(level & 1) * p.wave_cap;
  WaveItem *next = p.wave_items + (size_t)((level + 1) & 1) * p.wave_cap;
  K *const buf0 = static_cast<K *>(p.keys);
  const K *src = static_cast<const K *>((level & 1) ? p.scratch : p.keys);
  K *dst = static_cast<K *>((level & 1) ? p.keys : p.scratch);
  const unsigned cflags = (level & 1) ? 0u : kItemScratch;  // the sides live in dst
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  long long h = wave_find<NT, NW>(items, m, s0, sh);

  // less keys of the first sub-array before this span: the last count of the CTA
  // holding its first key, and the (only) count of every CTA in between
  unsigned long long E = 0;
  {
    const long long koff = __ldcg(&items[h].koff);
    if (koff < s0) {
      const long long cf = koff / per;
      unsigned long long part = 0;
      for (long long j = cf + tid; j < (long long)blockIdx.x; j += NT)
        part += __ldcg(&p.wave_cnt[2 * j + (j == cf ? 1 : 0)]);
      E = wave_sum<NW>(part, sh);
    }
  }
  unsigned long long st_items = 0, st_keys = 0, st_tiles = 0;
  for (long long s = s0; s < s1 && h < m; ++h) {
    const long long begin = __ldcg(&items[h].begin), end = __ldcg(&items[h].end);
    const long long koff = __ldcg(&items[h].koff);
    const long long klen = end - begin - 1;
    const long long a = s - koff, b = min(s1 - koff, klen);
    const K key = __ldcg(src + begin);  // Step 1
    const long long f = begin + 1, base = tile_base(src, begin);
    for (long long lo = base + ((f + a - base) / TILE) * TILE; lo < f + b; lo += TILE) {
      const int vlo = (int)max(f + a - lo, 0ll), vhi = (int)min(f + b - lo, (long long)TILE);
      K x[IPT];
      wave_load<K, NT, IPT>(src, lo, vlo, vhi, x);
      // Step 3 per key, then one warp scan of the packed (less, >=) counts
      unsigned lessbits = 0, gebits = 0;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
#pragma unroll
        for (int l = 0; l < VEC; ++l) {
          const int j = v * VEC + l, k = (v * NT + tid) * VEC + l;
          const bool valid = k >= vlo && k < vhi;
          const bool le = goes_left(key, x[j]);
          lessbits |= (unsigned)(valid && le) << j;
          gebits |= (unsigned)(valid && !le) << j;
        }
      }
      const unsigned mine = (unsigned)__popc(lessbits) | ((unsigned)__popc(gebits) << 16);
      unsigned incl = mine;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned u = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += u;
      }
      if (lane == 31) {
        sh.wl[w] = incl & 0xffffu;
        sh.wg[w] = incl >> 16;
      }
      __syncthreads();
      unsigned L = 0, G = 0, wlx = 0, wgx = 0;
#pragma unroll
      for (int i = 0; i < NW; ++i) {
        const unsigned c0 = sh.wl[i], c1 = sh.wg[i];
        if (i < w) {
          wlx += c0;
          wgx += c1;
        }
        L += c0;
        G += c1;
      }
      scatter_keys<K, IPT>(sout, x, lessbits, gebits, wlx, L + wgx, incl - mine);
      __syncthreads();
      // less keys after the E less keys before this tile; >= keys before the >= keys of
      // earlier tiles, counted from the right end
      const long long before = lo + vlo - f;  // keys of the sub-array before this tile
      const long long lbase = begin + (long long)E;
      const long long gbase = end - (before - (long long)E) - (long long)G;
      if (!(lbase >= begin && lbase + L <= end && gbase >= begin && gbase + G <= end)) {
        if (tid == 0) raise_error(ctl, kDevInternal, 0x900000000ull | (unsigned)h);
        break;  // uniform: every thread computed the same bounds
      }
      copy_out_v<K, NT>(sout, dst + lbase, L, tid);
      copy_out_v<K, NT>(sout + L, dst + gbase, G, tid);
      E += L;
      ++st_tiles;
      __syncthreads();  // sout and the warp counts are reused by the next tile
    }
    if (koff + klen <= s1 && tid == 0) {
      // this span holds the sub-array's last key: E = #{x < key}
      const long long kpos = begin + (long long)E;  // Step 4
      if (kpos >= end) {
        raise_error(ctl, kDevInternal, 0x800000000ull | (unsigned)h);
      } else {
        if (level & 1) {
          buf0[kpos] = key;
        } else {
          const unsigned long long i = atomicAdd(&ctl->wave_fin, 1ull);
          if (i < p.wave_cap) {
            p.wave_fin[2 * i] = (unsigned long long)kpos;
            p.wave_fin[2 * i + 1] = key_bits<K>(key);
          } else {
            raise_error(ctl, kDevWorkspaceExhausted, 4);
          }
        }
        ++st_items;
        st_keys += (unsigned long long)(end - begin);
        const long long cb[2] = {begin, kpos + 1}, ce[2] = {kpos, end};
#pragma unroll
        for (int c = 0; c < 2; ++c) {  // Steps 5-6
          const long long mm = ce[c] - cb[c];
          if (mm > p.cutoff && !sub_array_ok(p, cb[c], ce[c], 3)) {
            // reported, not recorded
          } else if (mm > p.cutoff) {
            const unsigned long long old = atomicAdd(
                &ctl->wave_ctr[(level + 1) & 1], (1ull << kWaveKeyBits) | (unsigned long long)(mm - 1));
            const unsigned long long idx = old >> kWaveKeyBits;
            if (idx < p.wave_cap) {
              next[idx].begin = cb[c];
              next[idx].end = ce[c];
              next[idx].koff = (long long)(old & kWaveKeyMask);
            } else {
              raise_error(ctl, kDevWorkspaceExhausted, 3);
            }
          } else if (mm >= 2 || (mm == 1 && cflags)) {
            // small sides (and single keys left in buffer 1) go to the SMEM finisher
            unsigned long long t0 = 0;
            unsigned tiles = 0;
            reserve_item<K, TILE>(p, epoch, cb[c], ce[c], cflags, &t0, &tiles);
          }
        }
      }
    }
    E = 0;  // the next sub-array starts inside this span
    s = koff + b;
  }
  if (tid == 0) {
    if (st_items) atomicAdd(&ctl->large_items, st_items);
    if (st_keys) atomicAdd(&ctl->large_keys, st_keys);
    if (st_tiles) atomicAdd(&ctl->tiles, st_tiles);
  }
}

// After the last wave level: keys still waiting go to buffer 0, and every sub-array on
// the list becomes a work item of tile_kernel's queue (ticket map published).
template <typename K, int TILE>
__global__ void wave_handoff_kernel(SortParams p, int level) {
  grid_dep_wait();
  Control *ctl = p.ctl;
  if (level & 1) wave_place_late_keys<K>(p);
  const unsigned long long ctr = __ldcg(&ctl->wave_ctr[level & 1]);
  const long long m = (long long)(ctr >> kWaveKeyBits);
  if (m == 0 || m > (long long)p.wave_cap || __ldcg(&ctl->abort) != 0u) return;
  const unsigned epoch = *reinterpret_cast<volatile unsigned *>(&ctl->epoch);
  const WaveItem *items = p.wave_items + (size_t)(level & 1) * p.wave_cap;
  const unsigned flags = (level & 1) ? kItemScratch : 0u;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long h = (long long)blockIdx.x * blockDim.x + threadIdx.x; h < m; h += stride) {
    unsigned long long t0 = 0;
    unsigned tiles = 0;
    const unsigned long long idx =
        reserve_item<K, TILE>(p, epoch, __ldcg(&items[h].begin), __ldcg(&items[h].end), flags,
                              &t0, &tiles);
    if (tiles) publish_tickets(p, epoch, idx, t0, tiles, 0, 1);
  }
}

// ----------------------------------------------------------------------------- split
// A single partition (Steps 1-4 of one array) in two launches with no wait between CTAs:
// split_count_kernel, then split_move_kernel under programmatic dependent launch. The
// keys after the key are cut into warp tiles of 32 * IPT keys, anchored at the 16-byte
// boundary at or below index 1 as every tile grid here is; global warp g (CTA c, warp w:
// g = c * NW + w) owns the Q consecutive warp tiles from g * Q on. The count launch
// stores each warp's less count (Step 3's classification) in p.wave_cnt[g]. The move
// launch gives each warp the exclusive prefix of those counts and moves the warp's tiles
// one by one: each is compacted in the warp's own slice of shared memory (less keys,
// then >= keys) and written with 128-bit stores, less keys from the front of the output
// and >= keys from the back, as the tile passes do. A warp walks its tiles from the last
// to the first, so that the ones the count launch read last, still in L2, are read again
// first. The last warp of the grid places the key at the total less count (Step 4).
// Every thread keeps the next tile's loads in flight while it works on the current one.
struct SplitGeom {
  long long base;   // start of warp tile 0 (index 1 rounded down to 16 bytes)
  long long tiles;  // warp tiles
  long long per;    // warp tiles per warp (Q)
};
template <typename K, int WT>
__device__ __forceinline__ SplitGeom split_geom(const K *src, long long n, long long warps) {
  SplitGeom g;
  g.base = tile_base(src, 0);
  g.tiles = (n - g.base + WT - 1) / WT;
  g.per = (g.tiles + warps - 1) / warps;
  return g;
}
// Key range [vlo, vhi) of warp tile s, which starts at *lo.
template <int WT>
__device__ __forceinline__ void split_tile(const SplitGeom &g, long long n, long long s,
                                           long long *lo, int *vlo, int *vhi) {
  *lo = g.base + s * WT;
  *vlo = (int)(1 > *lo ? 1 - *lo : 0);
  *vhi = (int)(n - *lo < WT ? n - *lo : WT);
}
// Step 3 on one lane's keys of a warp tile: bit j of *less / *ge set when key j is
// classified and goes to that side.
template <typename K, int IPT>
__device__ __forceinline__ void split_classify(K key, const K (&x)[IPT], int vlo, int vhi,
                                               int lane, unsigned *less, unsigned *ge) {
  constexpr int VEC = Vec<K>::N, NV = IPT / VEC;
  unsigned lb = 0, gb = 0;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
#pragma unroll
    for (int l = 0; l < VEC; ++l) {
      const int j = v * VEC + l, k = (v * 32 + lane) * VEC + l;
      const bool valid = k >= vlo && k < vhi;
      const bool le = goes_left(key, x[j]);
      lb |= (unsigned)(valid && le) << j;
      gb |= (unsigned)(valid && !le) << j;
    }
  }
  *less = lb;
  *ge = gb;
}

// A full warp tile (every key classified: all but the array's first and last) moves
// with unconditional 128-bit loads.
template <typename K, int IPT>
__device__ __forceinline__ void warp_tile_load_full(const K *t, K (&x)[IPT], int lane) {
  constexpr int VEC = Vec<K>::N, NV = IPT / VEC;
  using V = typename Vec<K>::T;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const V q = __ldcg(reinterpret_cast<const V *>(t + (v * 32 + lane) * VEC));
    if constexpr (VEC == 4) {
      x[v * 4 + 0] = q.x; x[v * 4 + 1] = q.y; x[v * 4 + 2] = q.z; x[v * 4 + 3] = q.w;
    } else {
      x[v * 2 + 0] = q.x; x[v * 2 + 1] = q.y;
    }
  }
}
template <typename K, int WT, int IPT>
__device__ __forceinline__ void split_load(const K *src, const SplitGeom &sg, long long n,
                                           long long s, K (&x)[IPT], int lane) {
  long long lo;
  int vlo, vhi;
  split_tile<WT>(sg, n, s, &lo, &vlo, &vhi);
  if (vlo == 0 && vhi == WT) warp_tile_load_full<K, IPT>(src + lo, x, lane);
  else tile_load<K, 32, IPT>(src, lo, vlo, vhi, x, lane);
}
// Step 3's less count of one lane's keys of warp tile s.
template <typename K, int WT, int IPT>
__device__ __forceinline__ unsigned split_less(K key, const SplitGeom &sg, long long n,
                                               long long s, const K (&x)[IPT], int lane) {
  long long lo;
  int vlo, vhi;
  split_tile<WT>(sg, n, s, &lo, &vlo, &vhi);
  if (vlo == 0 && vhi == WT) {
    unsigned c = 0;
#pragma unroll
    for (int j = 0; j < IPT; ++j) c += goes_left(key, x[j]) ? 1u : 0u;
    return c;
  }
  unsigned lb, gb;
  split_classify<K, IPT>(key, x, vlo, vhi, lane, &lb, &gb);
  return (unsigned)__popc(lb);
}

template <typename K, int NT, int IPT>
__global__ void __launch_bounds__(NT, tile_min_blocks(NT)) split_count_kernel(SortParams p) {
  constexpr int NW = NT / 32, WT = 32 * IPT;
  grid_dep_launch();  // the move launch may start; it waits for this launch's memory
  const K *const src = static_cast<const K *>(p.keys);
  const long long n = p.total;
  const int lane = threadIdx.x & 31;
  const long long g = (long long)blockIdx.x * NW + (threadIdx.x >> 5);
  const SplitGeom sg = split_geom<K, WT>(src, n, (long long)gridDim.x * NW);
  const K key = __ldcg(src);  // Step 1: the first element is the key
  long long s = g * sg.per;
  const long long s_end = s + sg.per < sg.tiles ? s + sg.per : sg.tiles;
  unsigned cl = 0;
  // two key sets in turn: the next tile's loads are in flight while this one is counted
  K xa[IPT], xb[IPT];
  if (s < s_end) split_load<K, WT, IPT>(src, sg, n, s, xa, lane);
  while (s < s_end) {
    if (s + 1 < s_end) split_load<K, WT, IPT>(src, sg, n, s + 1, xb, lane);
    cl += split_less<K, WT, IPT>(key, sg, n, s, xa, lane);
    if (++s >= s_end) break;
    if (s + 1 < s_end) split_load<K, WT, IPT>(src, sg, n, s + 1, xa, lane);
    cl += split_less<K, WT, IPT>(key, sg, n, s, xb, lane);
    ++s;
  }
  cl = __reduce_add_sync(kFull, cl);
  if (lane == 0) p.wave_cnt[g] = cl;
}

// One warp tile of split_move_kernel: Steps 3.1/3.2 for its keys x, given the less keys
// of every earlier warp tile (*Erun holds them for the tiles up to and including this
// one and is lowered by this tile's count). The keys are compacted in the warp's slice
// `so` at offsets that share the destination's 16-byte phase, so both runs are copied
// out with aligned 128-bit loads and stores. False (and an error) if a destination
// falls outside the output.
template <typename K, int WT, int IPT>
__device__ __forceinline__ bool split_move_tile(const SortParams &p, K key, const SplitGeom &sg,
                                                long long n, long long s, const K (&x)[IPT],
                                                K *so, K *dst, unsigned long long *Erun,
                                                int lane) {
  constexpr int VEC = Vec<K>::N;
  long long lo;
  int vlo, vhi;
  split_tile<WT>(sg, n, s, &lo, &vlo, &vhi);
  const bool full = vlo == 0 && vhi == WT;
  unsigned lb = 0, gb = 0, mine;
  if (full && sizeof(K) == 4) {  // one compare per key: recount, and compare again below
    unsigned c = 0;
#pragma unroll
    for (int j = 0; j < IPT; ++j) c += goes_left(key, x[j]) ? 1u : 0u;
    mine = c | ((IPT - c) << 16);
  } else if (full) {  // 8-byte keys compare on the integer pipes: keep the result bits
#pragma unroll
    for (int j = 0; j < IPT; ++j) lb |= (goes_left(key, x[j]) ? 1u : 0u) << j;
    gb = ~lb & (IPT >= 32 ? 0xffffffffu : (1u << (IPT & 31)) - 1u);
    mine = (unsigned)__popc(lb) | ((unsigned)(IPT - __popc(lb)) << 16);
  } else {
    split_classify<K, IPT>(key, x, vlo, vhi, lane, &lb, &gb);
    mine = (unsigned)__popc(lb) | ((unsigned)__popc(gb) << 16);
  }
  unsigned incl = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned u = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += u;
  }
  const unsigned tot = __shfl_sync(kFull, incl, 31);
  const unsigned L = tot & 0xffffu, G = tot >> 16;
  const unsigned long long E = *Erun - L;  // less keys in all earlier warp tiles
  *Erun = E;
  const long long PV = s == 0 ? 0 : lo - 1;  // classified keys in earlier warp tiles
  const long long lbase = (long long)E, gbase = n - (PV - (long long)E) - (long long)G;
  if (lbase < 0 || lbase + L > n || gbase < 1 || gbase + G > n) {
    if (lane == 0) raise_error(p.ctl, kDevInternal, 0xA00000000ull | (unsigned)s);
    return false;
  }
  const unsigned ml = (unsigned)((reinterpret_cast<uintptr_t>(dst + lbase) & 15u) / sizeof(K));
  const unsigned mg = (unsigned)((reinterpret_cast<uintptr_t>(dst + gbase) & 15u) / sizeof(K));
  const unsigned wl0 = ml, wg0 = (ml + L + VEC - 1) / VEC * VEC + mg;
  const unsigned ex = incl - mine;
  if (full && sizeof(K) == 4) {
    unsigned rl = wl0 + (ex & 0xffffu), rg = wg0 + (ex >> 16);
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
      const bool le = goes_left(key, x[j]);
      so[le ? rl : rg] = x[j];
      rl += le ? 1u : 0u;
      rg += le ? 0u : 1u;
    }
  } else {
    scatter_keys<K, IPT>(so, x, lb, gb, wl0, wg0, ex);
  }
  __syncwarp();
  copy_out_v<K, 32>(so + wl0, dst + lbase, L, lane);
  copy_out_v<K, 32>(so + wg0, dst + gbase, G, lane);
  __syncwarp();  // the slice is refilled by the next tile
  return true;
}

template <typename K, int NT, int IPT>
__global__ void __launch_bounds__(NT, tile_min_blocks(NT)) split_move_kernel(SortParams p) {
  constexpr int VEC = Vec<K>::N, NW = NT / 32, WT = 32 * IPT;
  static_assert(IPT % VEC == 0 && IPT <= 32 && WT < 65536, "bad warp tile");
  // per warp: both runs at their destination phase (up to 3 * VEC keys of gaps) plus the
  // 16 bytes copy_out_v may read past a run
  __shared__ __align__(16) K sbuf[NW][WT + 4 * VEC];
  __shared__ unsigned long long spart[NW];
  const K *const src = static_cast<const K *>(p.keys);
  K *const dst = static_cast<K *>(p.scratch);
  const long long n = p.total;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const long long c0 = (long long)blockIdx.x * NW, g = c0 + w;
  const SplitGeom sg = split_geom<K, WT>(src, n, (long long)gridDim.x * NW);
  const K key = __ldcg(src);  // Step 1
  const long long s_begin = g * sg.per < sg.tiles ? g * sg.per : sg.tiles;
  const long long s_end = s_begin + sg.per < sg.tiles ? s_begin + sg.per : sg.tiles;
  K xa[IPT], xb[IPT];
  // the warp's last tile first: its loads do not depend on the count launch
  if (s_begin < s_end) split_load<K, WT, IPT>(src, sg, n, s_end - 1, xa, lane);
  grid_dep_wait();  // every warp's count is written and visible
  const unsigned long long *cnt = p.wave_cnt;
  unsigned long long acc = 0;  // less keys of the warps of earlier CTAs
  for (long long i = tid; i < c0; i += NT) acc += __ldcg(&cnt[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
  if (lane == 0) spart[w] = acc;
  __syncthreads();
  unsigned long long E0 = 0;
#pragma unroll
  for (int i = 0; i < NW; ++i) E0 += spart[i];
  for (int i = 0; i < w; ++i) E0 += __ldcg(&cnt[c0 + i]);  // earlier warps of this CTA
  const unsigned long long mine_cnt = __ldcg(&cnt[g]);
  if (blockIdx.x == gridDim.x - 1 && w == NW - 1 && lane == 0) {
    const unsigned long long c = E0 + mine_cnt;  // #{x < key} over the whole array
    if (c >= (unsigned long long)n) {
      raise_error(p.ctl, kDevInternal, 0xA00000000ull);
    } else {
      dst[c] = key;  // Step 4
      if (p.key_index) *p.key_index = (long long)c;
    }
  }
  unsigned long long Erun = E0 + mine_cnt;  // less keys up to the next tile back
  K *const so = sbuf[w];
  bool ok = true;
  // from the last tile to the first, two key sets in turn (the next loads in flight)
  long long s = s_end - 1;
  while (s >= s_begin) {
    if (s > s_begin) split_load<K, WT, IPT>(src, sg, n, s - 1, xb, lane);
    if (!(ok = split_move_tile<K, WT, IPT>(p, key, sg, n, s, xa, so, dst, &Erun, lane))) break;
    if (--s < s_begin) break;
    if (s > s_begin) split_load<K, WT, IPT>(src, sg, n, s - 1, xa, lane);
    if (!(ok = split_move_tile<K, WT, IPT>(p, key, sg, n, s, xb, so, dst, &Erun, lane))) break;
    --s;
  }
  if (ok && Erun != E0 && lane == 0)  // the counts of both launches disagree
    raise_error(p.ctl, kDevInternal, 0xA00000000ull | 0xFFFFFFFFull);
}

// Phase 2: every small sub-array, claimed from the complete list, is finished by
// finish_small_item.

struct SmallCtaShared {
  SmallShared q;
  int r;
  long long h;
  Item it;
};

template <typename K, int NT>
__global__ void __launch_bounds__(NT) small_kernel(SortParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ SmallCtaShared sh;
  K *const buf0 = static_cast<K *>(p.keys);
  K *const buf1 = static_cast<K *>(p.scratch);
  Control *ctl = p.ctl;
  grid_dep_wait();  // the tile passes are complete
  const unsigned epoch = *reinterpret_cast<volatile unsigned *>(&ctl->epoch);
  const int tid = threadIdx.x;
  const SmallSmem<K> sm(smem, p.cutoff, NT);
  unsigned long long st_small = 0, st_small_keys = 0, st_segs = 0;
  if (tid == 0) sh.r = claim_small(p, epoch, &sh.h, &sh.it);
  __syncthreads();
  while (sh.r > 0) {
    const Item it = sh.it;
    const long long h = sh.h;
    __syncthreads();  // every thread holds the item before thread 0 claims the next
    finish_small_item<K, NT>(p, it, h, buf0, buf1, sm, sh.q, &st_small, &st_small_keys,
                             &st_segs, [&] { sh.r = claim_small(p, epoch, &sh.h, &sh.it); });
  }
  if (tid == 0) {
    if (st_small) atomicAdd(&ctl->small_items, st_small);
    if (st_small_keys) atomicAdd(&ctl->small_keys, st_small_keys);
    if (st_segs) atomicAdd(&ctl->smem_levels, st_segs);
  }
}

// One thread, at the start of a sort: a new generation (which retires every tagged
// entry of earlier sorts) and cleared dispatch counters and statistics. Returns it.
__device__ __forceinline__ unsigned start_generation(Control *ctl) {
  unsigned ep = ctl->epoch + 1u;
  if (ep == 0u || ep >= kMaxEpoch) ep = 1u;
  ctl->epoch = ep;
  ctl->pushed = 0;
  ctl->large_pushed = ctl->large_completed = 0;
  ctl->tq_head = 0;
  ctl->sq_head = ctl->sq_tail = 0;
  ctl->lb_used = 0;
  ctl->abort = 0;
  ctl->large_items = ctl->large_keys = ctl->tiles = 0;
  ctl->small_items = ctl->small_keys = 0;
  ctl->smem_levels = ctl->lookback_steps = 0;
  ctl->wave_ctr[0] = ctl->wave_ctr[1] = 0;
  ctl->wave_fin = 0;
  return ep;
}

// Wave form: a root above the cutoff goes on the level-0 list (true), else false.
__device__ __forceinline__ bool seed_wave_root(const SortParams &p, long long b, long long e) {
  if (!p.wave || e - b <= p.cutoff || (p.root_flags & kItemPartitionOnly)) return false;
  if (!sub_array_ok(p, b, e, 2)) return true;  // reported, not recorded
  Control *ctl = p.ctl;
  const unsigned long long old = atomicAdd(
      &ctl->wave_ctr[0], (1ull << kWaveKeyBits) | (unsigned long long)(e - b - 1));
  const unsigned long long idx = old >> kWaveKeyBits;
  if (idx < p.wave_cap) {
    p.wave_items[idx].begin = b;
    p.wave_items[idx].end = e;
    p.wave_items[idx].koff = (long long)(old & kWaveKeyMask);
  } else {
    raise_error(ctl, kDevWorkspaceExhausted, 5);
  }
  return true;
}

// Seed kernel (one CTA): starts a new generation and queues the roots.
template <typename K, int TILE>
__global__ void seed_kernel(SortParams p) {
  __shared__ unsigned epoch_sh;
  Control *ctl = p.ctl;
  grid_dep_launch();  // the tile kernel may start launching; it waits for this one
  if (threadIdx.x == 0) epoch_sh = start_generation(ctl);
  __syncthreads();
  const unsigned epoch = epoch_sh;
  if (!p.offsets) {
    // one root: thread 0 reserves it, the whole CTA writes its ticket-map entries
    __shared__ unsigned long long idx_sh, t0_sh;
    __shared__ unsigned tiles_sh;
    if (threadIdx.x == 0) {
      tiles_sh = 0;
      if (p.total >= 2) {
        if (p.total > kMaxItemKeys) raise_error(ctl, kDevBadOffsets, 0);
        else if (!seed_wave_root(p, 0, p.total))
          idx_sh = reserve_item<K, TILE>(p, epoch, 0, p.total, p.root_flags, &t0_sh, &tiles_sh);
      }
    }
    __syncthreads();
    if (tiles_sh) publish_tickets(p, epoch, idx_sh, t0_sh, tiles_sh, threadIdx.x, blockDim.x);
    return;
  }
  for (long long r = threadIdx.x; r < p.num_roots; r += blockDim.x) {
    const long long b = p.offsets[r], e = p.offsets[r + 1];
    if (b < 0 || e < b || e > p.total || e - b > kMaxItemKeys) {
      raise_error(ctl, kDevBadOffsets, (unsigned long long)r);
      continue;
    }
    if (e - b >= 2 && !seed_wave_root(p, b, e)) {
      unsigned long long t0 = 0;
      unsigned tiles = 0;
      const unsigned long long idx = reserve_item<K, TILE>(p, epoch, b, e, p.root_flags, &t0, &tiles);
      if (tiles) publish_tickets(p, epoch, idx, t0, tiles, 0, 1);
    }
  }
}

}  // namespace dev
}  // namespace ksort
