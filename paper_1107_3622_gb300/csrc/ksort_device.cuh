// Device code of libksort: the K-sort partition (arxiv 1107.3622, Section 1.1,
// Steps 1-4) as a single-pass tiled kernel with decoupled look-back, the recursion of
// Steps 5-6 as a persistent work queue, and a shared-memory finisher that applies the
// same first-element key rule to small sub-arrays.
//
// Element classification follows Step 3: x stays right of the key when key <= x,
// otherwise it goes left. Unlike the paper's sequential hole scheme, each pass is
// out of place between two buffers; the key index and the two sides' contents are
// those of Steps 1-4, the order inside each side is the tile order described below.
#pragma once

#include <cstdint>

#include "ksort_internal.h"

namespace ksort {
namespace dev {

constexpr unsigned kFull = 0xffffffffu;

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
__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
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
__device__ __forceinline__ void st_release(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release(unsigned long long *p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed(unsigned long long *p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// ----------------------------------------------------------------------------- keys
template <typename K> struct Vec;
template <> struct Vec<float> { using T = float4; static constexpr int N = 4; };
template <> struct Vec<unsigned> { using T = uint4; static constexpr int N = 4; };
template <> struct Vec<double> { using T = double2; static constexpr int N = 2; };

template <typename K>
__device__ __forceinline__ void unpack(const typename Vec<K>::T &q, K *x);
template <> __device__ __forceinline__ void unpack<float>(const float4 &q, float *x) {
  x[0] = q.x; x[1] = q.y; x[2] = q.z; x[3] = q.w;
}
template <> __device__ __forceinline__ void unpack<unsigned>(const uint4 &q, unsigned *x) {
  x[0] = q.x; x[1] = q.y; x[2] = q.z; x[3] = q.w;
}
template <> __device__ __forceinline__ void unpack<double>(const double2 &q, double *x) {
  x[0] = q.x; x[1] = q.y;
}

// Step 3: a[p] goes right of the key when key <= a[p]; every other element goes left.
template <typename K>
__device__ __forceinline__ bool goes_left(K key, K x) { return !(key <= x); }

// ----------------------------------------------------------------------------- errors
__device__ __forceinline__ void raise_error(Control *ctl, unsigned *abort_flag, unsigned code,
                                            unsigned long long info) {
  if (atomicCAS(&ctl->error, 0u, code) == 0u) atomicExch(&ctl->err_info, info);
  atomicExch(abort_flag, 1u);
}

// ----------------------------------------------------------------------------- tiles
// Tile grid of a sub-array [begin, end) in buffer `buf`: the first classified element
// is begin + 1 (begin holds the key); tiles are anchored at the 16-byte boundary at or
// below it so that whole vectors are loaded with 128-bit accesses.
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
// Sorts number their generations 1 .. 2^31 - 1 and standalone partitions
// 2^31 .. 2^32 - 1, so descriptors left by one kind of call never look valid to the
// other; zeroed memory (epoch 0) is never valid.
constexpr unsigned kPartitionEpoch = 0x80000000u;
__host__ __device__ __forceinline__ unsigned partition_epoch(unsigned gen) {
  return kPartitionEpoch | (gen & 0x7fffffffu);
}
__device__ __forceinline__ unsigned long long lb_pack(unsigned epoch, bool inclusive,
                                                       unsigned v) {
  return ((unsigned long long)epoch << 32) | ((unsigned long long)inclusive << 31) |
         (unsigned long long)(v & 0x7fffffffu);
}

template <int BLOCK>
struct TileShared {
  unsigned wl[BLOCK / 32];  // per warp: less count, then its exclusive prefix
  unsigned wg[BLOCK / 32];  // per warp: >= count, then its exclusive prefix
  unsigned L, G;            // tile totals
  unsigned long long E;     // less keys in all earlier tiles of the sub-array
  int abort;
};

// Decoupled look-back (Merrill and Garland, 2016) run by one warp: the less count of
// all tiles before `t`. Lane l inspects descriptor pos - l; windows move down by 32
// until one holds an inclusive prefix. Every wait is bounded by `limit_ns`.
// Returns 0 when the prefix was found, 1 on timeout, 2 when the call was aborted.
__device__ __forceinline__ int lookback(const unsigned long long *lb, unsigned t, unsigned epoch,
                                        unsigned long long limit_ns, const unsigned *abort_flag,
                                        unsigned long long *E_out,
                                        unsigned long long *steps) {
  const int lane = threadIdx.x & 31;
  unsigned long long E = 0;
  long long pos = (long long)t - 1;
  unsigned long long t0 = 0;
  while (true) {
    const long long idx = pos - lane;
    unsigned long long d;
    unsigned spins = 0;
    while (true) {
      d = idx >= 0 ? ld_relaxed(&lb[idx]) : lb_pack(epoch, true, 0u);
      if (__all_sync(kFull, (unsigned)(d >> 32) == epoch)) break;
      ++spins;
      if ((spins & 63u) == 0u) {
        int stop = 0;
        if (lane == 0) {
          const unsigned long long now = globaltimer();
          if (t0 == 0) t0 = now;
          stop = (now - t0 > limit_ns) ? 1 : (ld_relaxed(abort_flag) != 0u ? 2 : 0);
        }
        stop = __shfl_sync(kFull, stop, 0);
        if (stop) {
          *E_out = 0;
          return stop;
        }
      }
      __nanosleep(20);
    }
    ++*steps;
    const bool inclusive = (d >> 31) & 1ull;
    const unsigned v = (unsigned)(d & 0x7fffffffull);
    const unsigned pm = __ballot_sync(kFull, inclusive);
    if (pm) {
      const int p = __ffs(pm) - 1;
      E += __reduce_add_sync(kFull, lane <= p ? v : 0u);
      *E_out = E;
      return 0;
    }
    E += __reduce_add_sync(kFull, v);
    pos -= 32;
  }
}

// Writes count keys from shared memory (sm[0..count)) to global g[0..count): scalar
// stores up to the first 16-byte boundary of g, then one 128-bit store per VEC keys.
template <typename K, int BLOCK>
__device__ __forceinline__ void copy_out(const K *sm, K *g, unsigned count) {
  constexpr int VEC = Vec<K>::N;
  using V = typename Vec<K>::T;
  const int tid = threadIdx.x;
  unsigned head = (unsigned)(((16u - (reinterpret_cast<uintptr_t>(g) & 15u)) & 15u) / sizeof(K));
  if (head > count) head = count;
  if (tid < (int)head) g[tid] = sm[tid];
  const unsigned nvec = (count - head) / VEC;
  V *gv = reinterpret_cast<V *>(g + head);
  for (unsigned v = tid; v < nvec; v += BLOCK) {
    K x[VEC];
#pragma unroll
    for (int l = 0; l < VEC; ++l) x[l] = sm[head + v * VEC + l];
    V q;
    if constexpr (VEC == 4) {
      q.x = x[0]; q.y = x[1]; q.z = x[2]; q.w = x[3];
    } else {
      q.x = x[0]; q.y = x[1];
    }
    gv[v] = q;
  }
  for (unsigned k = head + nvec * VEC + tid; k < count; k += BLOCK) g[k] = sm[k];
}

// One tile pass of the partition of [begin, end) from `src` to `dst` (Steps 1-4 for
// the keys of one tile). The tile is staged in shared memory (`sin`, TILE keys); each
// warp classifies a contiguous TILE/NW slice with ballots, twice: once to count, and,
// after the look-back has given the keys of earlier tiles, again to scatter into
// `sout` in partitioned order. Less keys of tile t land at dst[begin + E_t ...], the
// others at the right end, dst[end - PG_t - G_t ...] with PG_t the >= keys of earlier
// tiles, so the key's index begin + #{x < key} stays free. Returns false if the call
// was aborted or timed out. Needs a __syncthreads() between consecutive calls.
template <typename K, int BLOCK, int IPT>
__device__ __forceinline__ bool partition_tile(
    const K *__restrict__ src, K *__restrict__ dst, long long begin, long long end, unsigned t,
    unsigned long long *__restrict__ lb, unsigned epoch, unsigned long long limit_ns,
    Control *ctl, unsigned *abort_flag, K *sin, TileShared<BLOCK> &sh,
    unsigned long long *less_through_tile, unsigned long long *lb_steps) {
  constexpr int VEC = Vec<K>::N;
  constexpr int TILE = BLOCK * IPT;
  constexpr int NW = BLOCK / 32;
  constexpr int SLICE = TILE / NW;  // keys per warp
  static_assert(IPT % VEC == 0 && SLICE % 32 == 0, "bad tile shape");
  using V = typename Vec<K>::T;
  K *sout = sin + TILE;

  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const K key = __ldcg(src + begin);  // Step 1: the first element is the key
  const long long first = begin + 1;
  const long long base = tile_base(src, begin);
  const long long lo = base + (long long)t * TILE;
  // valid positions of this tile: [vlo, vhi) relative to lo
  const int vlo = (int)(first > lo ? first - lo : 0);
  const int vhi = (int)(end - lo < TILE ? end - lo : TILE);

  // stage the tile: 128-bit loads for whole vectors, single loads at the two edges
  for (int v = tid; v < TILE / VEC; v += BLOCK) {
    const int k0 = v * VEC;
    if (k0 >= vlo && k0 + VEC <= vhi) {
      *reinterpret_cast<V *>(sin + k0) = __ldcg(reinterpret_cast<const V *>(src + lo + k0));
    } else {
#pragma unroll
      for (int l = 0; l < VEC; ++l)
        if (k0 + l >= vlo && k0 + l < vhi) sin[k0 + l] = __ldcg(src + lo + k0 + l);
    }
  }
  __syncthreads();

  // pass 1: Step 3 counts per warp
  const unsigned lt = lanemask_lt();
  unsigned wl = 0, wg = 0;
#pragma unroll 4
  for (int c = 0; c < SLICE; c += 32) {
    const int k = w * SLICE + c + lane;
    const bool valid = k >= vlo && k < vhi;
    const bool le = valid && goes_left(key, sin[k]);
    wl += __popc(__ballot_sync(kFull, le));
    wg += __popc(__ballot_sync(kFull, valid && !le));
  }
  if (lane == 0) {
    sh.wl[w] = wl;
    sh.wg[w] = wg;
  }
  __syncthreads();

  if (w == 0) {
    const unsigned a0 = lane < NW ? sh.wl[lane] : 0u;
    const unsigned b0 = lane < NW ? sh.wg[lane] : 0u;
    unsigned a = a0, b = b0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned ua = __shfl_up_sync(kFull, a, o);
      const unsigned ub = __shfl_up_sync(kFull, b, o);
      if (lane >= o) { a += ua; b += ub; }
    }
    const unsigned L = __shfl_sync(kFull, a, 31);
    const unsigned G = __shfl_sync(kFull, b, 31);
    if (lane < NW) {
      sh.wl[lane] = a - a0;
      sh.wg[lane] = b - b0;
    }
    unsigned long long E = 0;
    int status = 0;
    if (t == 0) {
      if (lane == 0) st_relaxed(&lb[0], lb_pack(epoch, true, L));
    } else {
      if (lane == 0) st_relaxed(&lb[t], lb_pack(epoch, false, L));
      unsigned long long steps = 0;
      status = lookback(lb, t, epoch, limit_ns, abort_flag, &E, &steps);
      if (lane == 0) {
        if (status == 0) st_relaxed(&lb[t], lb_pack(epoch, true, (unsigned)(E + L)));
        *lb_steps += steps;
      }
    }
    if (lane == 0) {
      if (status == 1) raise_error(ctl, abort_flag, kDevTimeout, 0x100000000ull | t);
      sh.L = L;
      sh.G = G;
      sh.E = E;
      sh.abort = status == 0 ? 0 : 1;
    }
  }
  __syncthreads();
  if (sh.abort) return false;

  // pass 2: the same classification, scattered into sout in partitioned order
  const unsigned L = sh.L, G = sh.G;
  const unsigned long long E = sh.E;
  unsigned rl = sh.wl[w], rg = L + sh.wg[w];
#pragma unroll 4
  for (int c = 0; c < SLICE; c += 32) {
    const int k = w * SLICE + c + lane;
    const bool valid = k >= vlo && k < vhi;
    const K x = valid ? sin[k] : K(0);
    const bool le = valid && goes_left(key, x);
    const unsigned ml = __ballot_sync(kFull, le), mg = __ballot_sync(kFull, valid && !le);
    if (valid) sout[le ? rl + __popc(ml & lt) : rg + __popc(mg & lt)] = x;
    rl += __popc(ml);
    rg += __popc(mg);
  }
  __syncthreads();

  const long long PV = t == 0 ? 0 : lo - first;  // classified keys in earlier tiles
  const long long PG = PV - (long long)E;        // of which >= key
  const long long lbase = begin + (long long)E;
  const long long gbase = end - PG - (long long)G;
  if (lbase < begin || lbase + L > end || gbase < begin || gbase + G > end) {
    // only with inconsistent prefixes; never write outside the item
    if (tid == 0) raise_error(ctl, abort_flag, kDevInternal, 0x500000000ull | t);
    return false;
  }
  copy_out<K, BLOCK>(sout, dst + lbase, L);
  copy_out<K, BLOCK>(sout + L, dst + gbase, G);
  *less_through_tile = E + L;
  return true;
}

// ----------------------------------------------------------------------------- smem
// Shared-memory finisher for one small sub-array (m <= cutoff keys), run by one CTA.
// The keys are loaded into buffer A; every recursion level then runs on WARPS, with no
// CTA barrier: a warp takes a segment [s, s + n) from a CTA-local queue and applies
// Steps 1-4 to it (key = its first element; x goes right when key <= x) from one
// shared buffer into the other, then Steps 5-6 depth first: it keeps one side, queues
// the other, and finishes sides of at most 32 keys in registers by the same rule.
// Every key that reaches its final index is written there in buffer A, which is
// copied out once all warps are done.
// Queued segments hold more than 32 keys and are disjoint, so at most cutoff / 33 are
// live at once: 512 slots cover cutoffs up to 16896 keys.
constexpr int kSmallQueue = 512;
constexpr int kMaxSmallCutoff = 16384;
// Segments above this size are partitioned by the whole CTA, smaller ones by one warp.
constexpr int kBlockSegment = 1024;
constexpr int kBigStack = kMaxSmallCutoff / kBlockSegment + 2;

struct SmallShared {
  unsigned long long ring[kSmallQueue];
  unsigned long long big[kBigStack];  // segments for CTA-wide partitions
  unsigned wl[32], wg[32];            // per-warp counts of a CTA-wide partition
  int head, tail, pending, bad, nbig, L;
};

template <typename K>
__host__ __device__ constexpr size_t smem_finisher_bytes(int cap, int warps) {
  // buffers A and B, then per-warp scratch for the 32-key register sorts
  return (size_t)2 * cap * sizeof(K) + (size_t)warps * 32 * (sizeof(K) + sizeof(unsigned)) + 64;
}

// Steps 1-4 by one warp on X[s .. s+n): less keys to Y[s ..] upward, the others to
// Y[s+n-1 ..] downward; returns the number of less keys L (the key's offset).
template <typename K>
__device__ __forceinline__ int warp_partition(const K *X, K *Y, int s, int n, K key) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  const int e = s + n;
  int L = 0, G = 0;
  for (int i0 = s + 1; i0 < e; i0 += 64) {
    const int ia = i0 + lane, ib = ia + 32;
    const bool va = ia < e, vb = ib < e;
    const K xa = va ? X[ia] : K(0);
    const K xb = vb ? X[ib] : K(0);
    const bool la = va && goes_left(key, xa);
    const bool lb = vb && goes_left(key, xb);
    const unsigned mla = __ballot_sync(kFull, la), mga = __ballot_sync(kFull, va && !la);
    const unsigned mlb = __ballot_sync(kFull, lb), mgb = __ballot_sync(kFull, vb && !lb);
    if (va) Y[la ? s + L + __popc(mla & lt) : e - 1 - G - __popc(mga & lt)] = xa;
    L += __popc(mla);
    G += __popc(mga);
    if (vb) Y[lb ? s + L + __popc(mlb & lt) : e - 1 - G - __popc(mgb & lt)] = xb;
    L += __popc(mlb);
    G += __popc(mgb);
  }
  __syncwarp();
  return L;
}

// Steps 1-6 for n <= 32 keys held one per lane: every segment of the warp is
// partitioned around its first element in the same step, until all segments hold one
// key. X[s..s+n) in, A[s..s+n) out (X may equal A).
template <typename K>
__device__ __forceinline__ void warp_tiny_ksort(const K *X, K *A, int s, int n, K *wk,
                                                unsigned *wseg) {
  const int lane = threadIdx.x & 31;
  const bool act = lane < n;
  const unsigned lt = lanemask_lt();
  K x = act ? X[s + lane] : K(0);
  int lo = 0, hi = n;
  for (int level = 0; level < 32; ++level) {
    if (!__any_sync(kFull, act && lane == lo && hi - lo >= 2)) break;
    const K key = __shfl_sync(kFull, x, lo);
    const bool in_big = act && hi - lo >= 2;
    const bool is_key = lane == lo;
    const bool lf = in_big && !is_key && goes_left(key, x);
    const unsigned ml = __ballot_sync(kFull, lf);
    const unsigned segmask = (hi >= 32 ? kFull : ((1u << hi) - 1u)) & ~((1u << lo) - 1u);
    const int Lc = __popc(ml & segmask);
    const int rl = __popc(ml & segmask & lt);
    int dest = lane, nlo = lo, nhi = hi;
    if (in_big) {
      if (is_key) {
        dest = lo + Lc;
        nlo = dest;
        nhi = dest + 1;
      } else if (lf) {
        dest = lo + rl;
        nhi = lo + Lc;
      } else {
        dest = lo + Lc + 1 + (lane - lo - 1 - rl);
        nlo = lo + Lc + 1;
      }
    }
    if (act) {
      wk[dest] = x;
      wseg[dest] = (unsigned)nlo | ((unsigned)nhi << 8);
    }
    __syncwarp();
    if (act) {
      x = wk[lane];
      const unsigned q = wseg[lane];
      lo = (int)(q & 0xffu);
      hi = (int)(q >> 8);
    }
    __syncwarp();
  }
  if (act) A[s + lane] = x;
  __syncwarp();
}

__device__ __forceinline__ unsigned long long seg_pack(int s, int n, int par) {
  return ((unsigned long long)(unsigned)s << 32) | ((unsigned long long)(unsigned)n << 1) |
         (unsigned long long)par;
}

// Lane 0 queues a segment of more than 32 keys.
__device__ __forceinline__ void small_push(SmallShared &q, int s, int n, int par) {
  atomicAdd(&q.pending, 1);
  const int slot = atomicAdd(&q.tail, 1);
  __threadfence_block();
  atomicExch(&q.ring[slot % kSmallQueue], seg_pack(s, n, par));
}

// Lane 0 claims the next queued segment; returns 0 once the CTA's work is done.
__device__ __forceinline__ unsigned long long small_pop(SmallShared &q) {
  volatile SmallShared &v = q;
  for (unsigned spins = 0;; ++spins) {
    const int h = v.head;
    if (h < v.tail) {
      if (atomicCAS(&q.head, h, h + 1) == h) {
        unsigned long long e = 0;
        for (unsigned w = 0; (e = atomicExch(&q.ring[h % kSmallQueue], 0ull)) == 0ull; ++w) {
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
    if (spins > (1u << 26)) {
      q.bad = 1;
      return 0;
    }
    __nanosleep(16);
  }
}

// Steps 1-4 by the whole CTA on X[s .. s+n): each warp classifies a contiguous run of
// 32-key chunks twice (count, then scatter after a scan of the warp counts). Same
// output layout as warp_partition. Returns L; contains three CTA barriers.
template <typename K, int BLOCK>
__device__ __forceinline__ int block_partition(const K *X, K *Y, int s, int n, K key,
                                               SmallShared &q) {
  constexpr int NW = BLOCK / 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned lt = lanemask_lt();
  const int e = s + n;
  const int nch = (n - 1 + 31) / 32;
  const int per = (nch + NW - 1) / NW;
  const int c0 = w * per, c1 = min(nch, c0 + per);
  unsigned wl = 0, wg = 0;
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
  __syncthreads();
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
  __syncthreads();
  unsigned rl = q.wl[w], rg = q.wg[w];
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
  __syncthreads();
  return L;
}

// Sorts src[0..m) into out[0..m) (they may alias) with the K-sort rule.
template <typename K, int BLOCK>
__device__ bool smem_ksort(const K *__restrict__ src, K *__restrict__ out, int m, int cap,
                           unsigned char *smem, SmallShared &q, unsigned long long *segments) {
  constexpr int NW = BLOCK / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  K *A = reinterpret_cast<K *>(smem);
  K *B = A + cap;
  K *wk = B + cap + warp * 32;
  unsigned *wseg = reinterpret_cast<unsigned *>(B + cap + NW * 32) + warp * 32;

  for (int e = tid; e < m; e += BLOCK) A[e] = __ldcg(src + e);
  for (int i = tid; i < kSmallQueue; i += BLOCK) q.ring[i] = 0ull;
  if (tid == 0) {
    q.head = 0;
    q.tail = 0;
    q.pending = 0;
    q.bad = 0;
  }
  __syncthreads();
  unsigned long long nseg = 0;
  if (m <= 32) {
    if (warp == 0) warp_tiny_ksort(A, A, 0, m, wk, wseg);
    nseg = 1;
  } else {
    // CTA-wide partitions while segments are large (the top levels of the item)
    if (tid == 0) {
      q.nbig = 0;
      if (m > kBlockSegment) q.big[q.nbig++] = seg_pack(0, m, 0);
      else small_push(q, 0, m, 0);
    }
    __syncthreads();
    while (q.nbig > 0) {
      const unsigned long long e = q.big[q.nbig - 1];
      const int s = (int)(e >> 32), n = (int)((e >> 1) & 0x7fffffffu), par = (int)(e & 1ull);
      __syncthreads();
      const K *X = par ? B : A;
      K *Y = par ? A : B;
      const K key = X[s];
      const int L = block_partition<K, BLOCK>(X, Y, s, n, key, q);
      ++nseg;
      const int cp = par ^ 1;
      if (tid == 0) {
        A[s + L] = key;
        --q.nbig;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const int cs = c ? s + L + 1 : s, cn = c ? n - L - 1 : L;
          if (cn > kBlockSegment) q.big[q.nbig++] = seg_pack(cs, cn, cp);
          else if (cn > 32) small_push(q, cs, cn, cp);
          else if (cn == 1 && cp) A[cs] = Y[cs];
        }
      }
      if (warp < 2) {  // warps 0 and 1 finish a side of at most 32 keys at once
        const int cs = warp ? s + L + 1 : s, cn = warp ? n - L - 1 : L;
        if (cn >= 2 && cn <= 32) warp_tiny_ksort(Y, A, cs, cn, wk, wseg);
      }
      __syncthreads();
    }
    while (true) {
      unsigned long long e = 0;
      if (lane == 0) e = small_pop(q);
      e = __shfl_sync(kFull, e, 0);
      if (e == 0ull) break;
      int s = (int)(e >> 32), n = (int)((e >> 1) & 0x7fffffffu), par = (int)(e & 1ull);
      while (true) {
        const K *X = par ? B : A;
        K *Y = par ? A : B;
        ++nseg;
        const K key = X[s];  // Step 1
        const int L = warp_partition(X, Y, s, n, key);
        if (lane == 0) A[s + L] = key;  // Step 4: final index
        const int ls = s, ln = L, rs = s + L + 1, rn = n - L - 1, cp = par ^ 1;
        if (cp && ln == 1 && lane == 0) A[ls] = Y[ls];
        if (cp && rn == 1 && lane == 0) A[rs] = Y[rs];
        if (ln >= 2 && ln <= 32) warp_tiny_ksort(Y, A, ls, ln, wk, wseg);
        if (rn >= 2 && rn <= 32) warp_tiny_ksort(Y, A, rs, rn, wk, wseg);
        __syncwarp();
        const bool bl = ln > 32, br = rn > 32;
        if (bl && br) {  // Steps 5-6: queue the smaller side, keep the larger
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
  }
  __syncthreads();
  copy_out<K, BLOCK>(A, out, (unsigned)m);
  if (tid == 0) *segments += nseg;
  return q.bad == 0;
}

// ----------------------------------------------------------------------------- queue
// Work items live in a bump-allocated pool. The sort runs in two phases.
// Phase 1 (Steps 1-4 on items above the cutoff, with Steps 5-6 queuing their sides):
// a large item reserves one ticket per tile pass; tickets index both the look-back
// descriptors and a ticket map that names the item. CTAs claim tickets with one
// atomicAdd, in order, possibly before the item that owns the ticket exists; they then
// wait for it, so a freshly queued item starts without any dispatch delay. Phase 2
// starts when every large item has completed: the small items, now a complete list,
// are claimed with atomicAdd and finished in shared memory. Entries carry the sort's
// epoch, so no memset is needed between sorts.
__device__ __forceinline__ unsigned long long q_entry(unsigned epoch, unsigned long long idx) {
  return ((unsigned long long)epoch << 32) | idx;
}

template <typename K, int TILE>
__device__ __forceinline__ bool push_item(const SortParams &p, unsigned epoch, long long b,
                                          long long e, unsigned parity) {
  Control *ctl = p.ctl;
  const long long m = e - b;
  const K *buf = parity ? static_cast<const K *>(p.scratch) : static_cast<const K *>(p.keys);
  const bool small = m <= p.cutoff;
  const unsigned tiles = small ? 1u : tile_count<K, TILE>(buf, b, e);
  unsigned long long t0 = 0;
  if (!small) {
    t0 = atomicAdd(&ctl->lb_used, (unsigned long long)tiles);
    if (t0 + tiles > p.lb_cap) {
      raise_error(ctl, &ctl->abort, kDevWorkspaceExhausted, 2);
      return false;
    }
  }
  const unsigned long long idx = atomicAdd(&ctl->pushed, 1ull);
  if (idx >= p.item_cap) {
    raise_error(ctl, &ctl->abort, kDevWorkspaceExhausted, 1);
    return false;
  }
  Item *it = p.items + idx;
  it->begin = b;
  it->end = e;
  it->tiles = tiles;
  it->lb = (unsigned)t0;
  it->flags = (parity ? kItemScratch : 0u) | (small ? kItemSmall : 0u);
  it->epoch = epoch;
  if (small) {
    __threadfence();
    const unsigned long long qi = atomicAdd(&ctl->sq_tail, 1ull);  // qi <= idx < item_cap
    st_release(&p.small_q[qi], q_entry(epoch, idx));
  } else {
    ItemCtl *c = p.ictl + idx;
    c->done = 0;
    c->less = 0;
    atomicAdd(&ctl->large_pushed, 1ull);
    __threadfence();
    const unsigned long long entry = q_entry(epoch, idx);
    for (unsigned j = 0; j < tiles; ++j) st_relaxed(&p.tmap[t0 + j], entry);
  }
  return true;
}

__device__ __forceinline__ void load_item(const Item *ip, Item *it) {
  it->begin = __ldcg(&ip->begin);
  it->end = __ldcg(&ip->end);
  it->tiles = __ldcg(&ip->tiles);
  it->lb = __ldcg(&ip->lb);
  it->flags = __ldcg(&ip->flags);
  it->epoch = 0;
}

// Thread 0 of a CTA, phase 1: waits for ticket k to be issued. Returns 1 with the
// item, 0 when phase 1 is over (every large item completed), -1 on abort or timeout.
__device__ __forceinline__ int wait_ticket(const SortParams &p, unsigned epoch,
                                           unsigned long long k, long long *h_out,
                                           unsigned *t_out, Item *it_out) {
  Control *ctl = p.ctl;
  unsigned ns = 16;
  unsigned long long idle_t0 = 0, last = ~0ull;
  while (true) {
    if (k < p.lb_cap) {
      const unsigned long long v = ld_acquire(&p.tmap[k]);
      if ((unsigned)(v >> 32) == epoch) {
        const long long idx = (long long)(v & 0xffffffffull);
        load_item(p.items + idx, it_out);
        *h_out = idx;
        *t_out = (unsigned)(k - it_out->lb);
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
      raise_error(ctl, &ctl->abort, kDevTimeout, 0x300000000ull | k);
      return -1;
    }
    __nanosleep(ns);
    ns = ns < 256 ? ns * 2 : 256;
  }
}

// Thread 0 of a CTA, phase 2: claims the next small item. Returns false when none is left.
__device__ __forceinline__ bool claim_small(const SortParams &p, unsigned epoch, long long *h_out,
                                            Item *it_out) {
  Control *ctl = p.ctl;
  if (ld_relaxed(&ctl->abort)) return false;
  const unsigned long long j = atomicAdd(&ctl->sq_head, 1ull);
  if (j >= ld_acquire(&ctl->sq_tail) || j >= p.item_cap) return false;
  unsigned long long t0 = 0;
  for (unsigned spins = 1;; ++spins) {  // queued before phase 2 began: already visible
    const unsigned long long v = ld_acquire(&p.small_q[j]);
    if ((unsigned)(v >> 32) == epoch) {
      const long long idx = (long long)(v & 0xffffffffull);
      load_item(p.items + idx, it_out);
      *h_out = idx;
      return true;
    }
    if ((spins & 255u) == 0u) {
      const unsigned long long now = globaltimer();
      if (t0 == 0) t0 = now;
      if (now - t0 > p.spin_limit_ns) {
        raise_error(ctl, &ctl->abort, kDevTimeout, 0x200000000ull | j);
        return false;
      }
    }
    __nanosleep(32);
  }
}

template <int BLOCK>
struct SortShared {
  TileShared<BLOCK> tile;
  SmallShared small;
  long long h;
  unsigned t;
  int has_work;
  Item it;
};

// Persistent sort kernel: phase 1 (tile passes of large items) then phase 2 (small
// items), see the queue notes above.
template <typename K, int BLOCK, int IPT, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) sort_kernel(SortParams p) {
  constexpr int TILE = BLOCK * IPT;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ SortShared<BLOCK> sh;
  K *const buf0 = static_cast<K *>(p.keys);
  K *const buf1 = static_cast<K *>(p.scratch);
  Control *ctl = p.ctl;
  const unsigned epoch = *reinterpret_cast<volatile unsigned *>(&ctl->epoch);
  const int tid = threadIdx.x;
  unsigned long long st_tiles = 0, st_lb = 0, st_segs = 0, st_small = 0, st_small_keys = 0;
  unsigned long long st_large = 0, st_large_keys = 0;
  unsigned long long cy_fetch = 0, cy_small = 0, cy_tile = 0, cy_fin = 0;
  long long c0 = clock64();
  bool aborted = false;

  // ---- phase 1
  while (true) {
    if (tid == 0) {
      const unsigned long long k = atomicAdd(&ctl->tq_head, 1ull);
      sh.has_work = wait_ticket(p, epoch, k, &sh.h, &sh.t, &sh.it);
    }
    __syncthreads();
    {
      const long long c1 = clock64();
      cy_fetch += (unsigned long long)(c1 - c0);
      c0 = c1;
    }
    if (sh.has_work <= 0) {
      aborted = sh.has_work < 0;
      break;
    }
    const Item it = sh.it;
    const long long h = sh.h;
    const unsigned t = sh.t;
    const unsigned par = it.flags & kItemScratch;
    K *src = par ? buf1 : buf0;
    K *dst = par ? buf0 : buf1;
    unsigned long long less = 0;
    const bool ok = partition_tile<K, BLOCK, IPT>(
        src, dst, it.begin, it.end, t, p.lb + it.lb, epoch, p.spin_limit_ns, ctl, &ctl->abort,
        reinterpret_cast<K *>(smem), sh.tile, &less, &st_lb);
    if (!ok) {
      aborted = true;
      break;
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();  // release the CTA's tile writes (ordered before by the barrier)
      {
        const long long c1 = clock64();
        cy_tile += (unsigned long long)(c1 - c0);
        c0 = c1;
      }
      ++st_tiles;
      if (t == it.tiles - 1) {
        atomicExch(&p.ictl[h].less, less);
        __threadfence();
      }
      const unsigned old = atomicAdd(&p.ictl[h].done, 1u);
      if (old == it.tiles - 1) {
        __threadfence();
        // Step 4: the key goes to its final index; Steps 5-6: both sides are queued.
        const unsigned long long c = ld_acquire(&p.ictl[h].less);
        const K key = __ldcg(src + it.begin);
        const long long kpos = it.begin + (long long)c;
        if (kpos >= it.end) {
          raise_error(ctl, &ctl->abort, kDevInternal, 0x700000000ull | (unsigned)h);
        } else {
          buf0[kpos] = key;
          const unsigned cpar = par ^ 1u;
          const long long cb[2] = {it.begin, kpos + 1};
          const long long ce[2] = {kpos, it.end};
#pragma unroll
          for (int s = 0; s < 2; ++s) {
            const long long m = ce[s] - cb[s];
            if (m == 1) {
              if (cpar) buf0[cb[s]] = __ldcg(dst + cb[s]);
            } else if (m >= 2) {
              push_item<K, TILE>(p, epoch, cb[s], ce[s], cpar);
            }
          }
        }
        ++st_large;
        st_large_keys += (unsigned long long)(it.end - it.begin);
        __threadfence();
        atomicAdd(&ctl->large_completed, 1ull);
      }
      const long long c1 = clock64();
      cy_fin += (unsigned long long)(c1 - c0);
      c0 = c1;
    }
    __syncthreads();
  }

  // ---- phase 2
  while (!aborted) {
    if (tid == 0) sh.has_work = claim_small(p, epoch, &sh.h, &sh.it) ? 1 : 0;
    __syncthreads();
    {
      const long long c1 = clock64();
      cy_fetch += (unsigned long long)(c1 - c0);
      c0 = c1;
    }
    if (!sh.has_work) break;
    const Item it = sh.it;
    const K *src = (it.flags & kItemScratch) ? buf1 : buf0;
    const int m = (int)(it.end - it.begin);
    const bool fin_ok = smem_ksort<K, BLOCK>(src + it.begin, buf0 + it.begin, m, p.cutoff, smem,
                                             sh.small, &st_segs);
    __syncthreads();
    if (tid == 0) {
      if (!fin_ok) raise_error(ctl, &ctl->abort, kDevInternal, 0x600000000ull | (unsigned)sh.h);
      ++st_small;
      st_small_keys += (unsigned long long)m;
      const long long c1 = clock64();
      cy_small += (unsigned long long)(c1 - c0);
      c0 = c1;
    }
  }

  if (tid == 0) {
    if (st_tiles) atomicAdd(&ctl->tiles, st_tiles);
    if (st_lb) atomicAdd(&ctl->lookback_steps, st_lb);
    if (st_segs) atomicAdd(&ctl->smem_levels, st_segs);
    if (st_small) atomicAdd(&ctl->small_items, st_small);
    if (st_small_keys) atomicAdd(&ctl->small_keys, st_small_keys);
    if (st_large) atomicAdd(&ctl->large_items, st_large);
    if (st_large_keys) atomicAdd(&ctl->large_keys, st_large_keys);
    atomicAdd(&ctl->cyc_fetch, cy_fetch);
    atomicAdd(&ctl->cyc_small, cy_small);
    atomicAdd(&ctl->cyc_tile, cy_tile);
    atomicAdd(&ctl->cyc_finish, cy_fin);
  }
}

// Seed kernel (one CTA): starts a new generation and queues the roots.
template <typename K, int TILE>
__global__ void seed_kernel(SortParams p) {
  __shared__ unsigned epoch_sh;
  Control *ctl = p.ctl;
  if (threadIdx.x == 0) {
    unsigned ep = ctl->epoch + 1u;
    if (ep == 0u || ep >= kPartitionEpoch) ep = 1u;
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
    ctl->cyc_fetch = ctl->cyc_small = ctl->cyc_tile = ctl->cyc_finish = 0;
    epoch_sh = ep;
  }
  __syncthreads();
  const unsigned epoch = epoch_sh;
  for (long long r = threadIdx.x; r < p.num_roots; r += blockDim.x) {
    long long b = 0, e = p.total;
    if (p.offsets) {
      b = p.offsets[r];
      e = p.offsets[r + 1];
    }
    if (b < 0 || e < b || e > p.total || e - b > kMaxItemKeys) {
      raise_error(ctl, &ctl->abort, kDevBadOffsets, (unsigned long long)r);
      continue;
    }
    if (e - b >= 2) push_item<K, TILE>(p, epoch, b, e, 0u);
  }
}

// Standalone out-of-place partition (ksort_partition_out): one CTA per tile, tiles
// claimed in launch order through a ticket so that look-back only waits on CTAs that
// are already running. Every CTA counts itself done, even after an abort, so the last
// one can hand a clean state to the next call.
template <typename K, int BLOCK, int IPT>
__global__ void __launch_bounds__(BLOCK) partition_kernel(PartParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ TileShared<BLOCK> sh;
  __shared__ unsigned t_sh, gen_sh;
  __shared__ unsigned long long base_sh;
  const K *in = static_cast<const K *>(p.in);
  K *out = static_cast<K *>(p.out);
  PartCtl *pc = p.pctl;
  if (threadIdx.x == 0) {
    const unsigned long long base = ld_relaxed(&pc->base);
    gen_sh = ld_relaxed(&pc->gen);
    base_sh = base;
    t_sh = (unsigned)(atomicAdd(&pc->ticket, 1ull) - base);
  }
  __syncthreads();
  const unsigned t = t_sh;
  const unsigned long long base = base_sh;
  const unsigned ntiles = gridDim.x;
  unsigned long long less = 0, steps = 0;
  bool ok = false;
  if (t < ntiles) {
    ok = partition_tile<K, BLOCK, IPT>(in, out, 0, p.n, t, p.lb, partition_epoch(gen_sh),
                                       p.spin_limit_ns, p.ctl, &pc->abort,
                                       reinterpret_cast<K *>(smem), sh, &less, &steps);
  } else if (threadIdx.x == 0) {
    raise_error(p.ctl, &pc->abort, kDevInternal, 0x800000000ull | t);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();  // release the CTA's tile writes (ordered before by the barrier)
    if (ok && t == ntiles - 1) {
      atomicExch(&pc->less, less);
      __threadfence();
    }
    const unsigned long long old = atomicAdd(&pc->done, 1ull) - base;
    if (old == ntiles - 1) {
      __threadfence();
      if (ld_relaxed(&pc->abort) == 0u) {
        const unsigned long long c = ld_acquire(&pc->less);
        out[c] = __ldcg(in);  // Step 4
        *p.key_index = (long long)c;
      }
      // Every CTA of this call has read base and gen and finished: start the next call.
      atomicExch(&pc->base, base + ntiles);
      atomicExch(&pc->gen, gen_sh + 1u);
      atomicExch(&pc->abort, 0u);
    }
  }
}

}  // namespace dev
}  // namespace ksort
