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

// One tile pass of the partition of [begin, end) from `src` to `dst`.
// Less keys of tile t land at dst[begin + E_t ...], >= keys at the right end,
// dst[end - PG_t - G_t ...] with PG_t the >= keys of earlier tiles; so the key's index
// begin + #{x < key} is left free. Returns false if the call was aborted or timed out.
// Requires a __syncthreads() between consecutive calls (shared staging reuse).
template <typename K, int BLOCK, int IPT>
__device__ __forceinline__ bool partition_tile(
    const K *__restrict__ src, K *__restrict__ dst, long long begin, long long end, unsigned t,
    unsigned long long *__restrict__ lb, unsigned epoch, unsigned long long limit_ns,
    Control *ctl, unsigned *abort_flag, K *stage, TileShared<BLOCK> &sh,
    unsigned long long *less_through_tile, unsigned long long *lb_steps) {
  constexpr int VEC = Vec<K>::N;
  constexpr int VPT = IPT / VEC;
  constexpr int TILE = BLOCK * IPT;
  constexpr int NW = BLOCK / 32;
  static_assert(IPT % VEC == 0 && IPT <= 32, "bad IPT");
  using V = typename Vec<K>::T;

  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const K key = __ldcg(src + begin);  // Step 1: the first element is the key
  const long long first = begin + 1;
  const long long base = tile_base(src, begin);
  const long long lo = base + (long long)t * TILE;

  K x[IPT];
#pragma unroll
  for (int v = 0; v < VPT; ++v) {
    const long long e0 = lo + ((long long)v * BLOCK + tid) * VEC;
    if (e0 >= first && e0 + VEC <= end) {
      const V q = __ldcg(reinterpret_cast<const V *>(src + e0));
      unpack<K>(q, &x[v * VEC]);
    } else {
#pragma unroll
      for (int l = 0; l < VEC; ++l) {
        const long long e = e0 + l;
        x[v * VEC + l] = (e >= first && e < end) ? __ldcg(src + e) : K(0);
      }
    }
  }

  // Step 3 for every element; ranks within the warp from ballots.
  const unsigned lt = lanemask_lt();
  unsigned rank[IPT];
  unsigned lessbits = 0, validbits = 0;
  unsigned wl = 0, wg = 0;
#pragma unroll
  for (int v = 0; v < VPT; ++v) {
#pragma unroll
    for (int l = 0; l < VEC; ++l) {
      const int i = v * VEC + l;
      const long long e = lo + ((long long)v * BLOCK + tid) * VEC + l;
      const bool valid = e >= first && e < end;
      const bool le = valid && goes_left(key, x[i]);
      const bool ge = valid && !le;
      const unsigned ml = __ballot_sync(kFull, le);
      const unsigned mg = __ballot_sync(kFull, ge);
      rank[i] = le ? wl + __popc(ml & lt) : wg + __popc(mg & lt);
      wl += __popc(ml);
      wg += __popc(mg);
      lessbits |= (unsigned)le << i;
      validbits |= (unsigned)valid << i;
    }
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
    const bool ok = status == 0;
    if (lane == 0) {
      if (status == 1) raise_error(ctl, abort_flag, kDevTimeout, 0x100000000ull | t);
      sh.L = L;
      sh.G = G;
      sh.E = E;
      sh.abort = ok ? 0 : 1;
    }
  }
  __syncthreads();
  if (sh.abort) return false;

  const unsigned L = sh.L, G = sh.G;
  const unsigned long long E = sh.E;
  const unsigned wlx = sh.wl[w], wgx = sh.wg[w];
#pragma unroll
  for (int i = 0; i < IPT; ++i) {
    if ((validbits >> i) & 1u) {
      const unsigned slot = ((lessbits >> i) & 1u) ? wlx + rank[i] : L + wgx + rank[i];
      stage[slot] = x[i];
    }
  }
  __syncthreads();

  const long long PV = t == 0 ? 0 : lo - first;  // classified elements in earlier tiles
  const long long PG = PV - (long long)E;        // of which >= key
  const long long lbase = begin + (long long)E;
  const long long gbase = end - PG - (long long)G;
  const unsigned total = L + G;
  bool bad = false;
  for (unsigned k = tid; k < total; k += BLOCK) {
    const long long d = k < L ? lbase + k : gbase + (k - L);
    if (d >= begin && d < end) {
      dst[d] = stage[k];
    } else {
      bad = true;  // only with inconsistent prefixes; never write outside the item
    }
  }
  if (bad) raise_error(ctl, abort_flag, kDevInternal, 0x500000000ull | t);
  *less_through_tile = E + L;
  return true;
}

// ----------------------------------------------------------------------------- smem
// Shared-memory finisher: sorts m <= cap keys with the K-sort key rule, all segments of
// one recursion level at a time. Each segment [s, s_end) uses its first element as the
// key; its less keys keep their order at s.., the key lands at s + L, the >= keys keep
// their order after it. Segments of one key are final. The whole level is one
// block-wide pass: ballot counts, one scan, then a scatter into the other buffer.
template <int BLOCK, int JMAX>
struct SmemShared {
  unsigned cnt[JMAX * (BLOCK / 32)];
  int active;
  int next_active;
  int bad;
};

template <typename K>
__host__ __device__ constexpr size_t smem_finisher_bytes(int cap) {
  // two key buffers, two u16 segment-start buffers, one u16 per-segment slot array
  return (size_t)cap * (2 * sizeof(K) + 3 * sizeof(unsigned short)) + 64;
}

// Returns false if a consistency check failed (the output is then not sorted).
template <typename K, int BLOCK, int JMAX>
__device__ bool smem_ksort(const K *__restrict__ src, K *__restrict__ out, int m, int cap,
                           unsigned char *smem, SmemShared<BLOCK, JMAX> &sh,
                           unsigned long long *levels) {
  constexpr int NW = BLOCK / 32;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  K *k0 = reinterpret_cast<K *>(smem);
  K *k1 = k0 + cap;
  unsigned short *s0 = reinterpret_cast<unsigned short *>(k1 + cap);
  unsigned short *s1 = s0 + cap;
  unsigned short *slot = s1 + cap;
  const unsigned lt = lanemask_lt();

  for (int e = tid; e < m; e += BLOCK) {
    k0[e] = __ldcg(src + e);
    s0[e] = 0;
  }
  if (tid == 0) {
    sh.active = m >= 2;
    sh.bad = 0;
  }
  __syncthreads();

  const int J = (m + BLOCK - 1) / BLOCK;
  unsigned long long nlev = 0;
  while (sh.active) {
    // Every level shrinks each unfinished segment by at least its key, so m levels
    // always suffice; more means corrupted state: stop rather than loop.
    if (++nlev > (unsigned long long)m) {
      if (tid == 0) sh.bad = 1;
      break;
    }
    // A: classify against the segment's first element; ballot counts per (chunk, warp).
    unsigned bal[JMAX];
#pragma unroll
    for (int j = 0; j < JMAX; ++j) {
      bal[j] = 0;
      if (j < J) {
        const int e = j * BLOCK + tid;
        bool lf = false;
        if (e < m) {
          const int s = s0[e];
          lf = e != s && goes_left(k0[s], k0[e]);
        }
        bal[j] = __ballot_sync(kFull, lf);
        if (lane == 0) sh.cnt[j * NW + w] = __popc(bal[j]);
      }
    }
    if (tid == 0) sh.next_active = 0;
    __syncthreads();
    // B: exclusive scan of the counts in element order (one warp).
    if (w == 0) {
      const int n = J * NW;
      constexpr int PER = (JMAX * NW + 31) / 32;
      unsigned loc[PER];
      unsigned sum = 0;
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        const int i = lane * PER + q;
        loc[q] = i < n ? sh.cnt[i] : 0u;
        sum += loc[q];
      }
      unsigned inc = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned u = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += u;
      }
      unsigned run = inc - sum;
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        const int i = lane * PER + q;
        if (i < n) sh.cnt[i] = run;
        run += loc[q];
      }
    }
    __syncthreads();
    // C: segment heads record the prefix at their start.
#pragma unroll
    for (int j = 0; j < JMAX; ++j) {
      if (j < J) {
        const int e = j * BLOCK + tid;
        if (e < m && s0[e] == e) slot[e] = (unsigned short)(sh.cnt[j * NW + w] + __popc(bal[j] & lt));
      }
    }
    __syncthreads();
    unsigned ps[JMAX];
#pragma unroll
    for (int j = 0; j < JMAX; ++j) {
      ps[j] = 0;
      if (j < J) {
        const int e = j * BLOCK + tid;
        if (e < m) ps[j] = slot[s0[e]];
      }
    }
    __syncthreads();
    // D: the last element of each segment stores the segment's less count L.
#pragma unroll
    for (int j = 0; j < JMAX; ++j) {
      if (j < J) {
        const int e = j * BLOCK + tid;
        if (e < m) {
          const int s = s0[e];
          if (e == m - 1 || s0[e + 1] != s) {
            const unsigned pre = sh.cnt[j * NW + w] + __popc(bal[j] & lt);
            slot[s] = (unsigned short)(pre + ((bal[j] >> lane) & 1u) - ps[j]);
          }
        }
      }
    }
    __syncthreads();
    // E: scatter into the other buffer; new segment starts travel with the keys.
#pragma unroll
    for (int j = 0; j < JMAX; ++j) {
      if (j < J) {
        const int e = j * BLOCK + tid;
        if (e < m) {
          const int s = s0[e];
          const int L = slot[s];
          const int rl = (int)(sh.cnt[j * NW + w] + __popc(bal[j] & lt) - ps[j]);
          const bool lf = (bal[j] >> lane) & 1u;
          int d, ns;
          if (e == s) {
            d = s + L;
            ns = d;
          } else if (lf) {
            d = s + rl;
            ns = s;
          } else {
            d = s + L + 1 + ((e - s - 1) - rl);
            ns = s + L + 1;
          }
          if ((unsigned)d < (unsigned)m) {
            k1[d] = k0[e];
            s1[d] = (unsigned short)ns;
          } else {
            sh.bad = 1;
          }
          if (e == m - 1 || s0[e + 1] != s) {
            const int size = e - s + 1;
            if (L >= 2 || size - L - 1 >= 2) sh.next_active = 1;
          }
        }
      }
    }
    __syncthreads();
    K *tk = k0; k0 = k1; k1 = tk;
    unsigned short *ts = s0; s0 = s1; s1 = ts;
    if (tid == 0) sh.active = sh.next_active;
    __syncthreads();
  }
  __syncthreads();
  for (int e = tid; e < m; e += BLOCK) out[e] = k0[e];
  if (tid == 0) *levels += nlev;
  return sh.bad == 0;
}

// ----------------------------------------------------------------------------- queue
template <typename K, int TILE>
__device__ __forceinline__ bool push_item(const SortParams &p, unsigned epoch, long long b,
                                          long long e, unsigned parity) {
  Control *ctl = p.ctl;
  const long long m = e - b;
  const K *buf = parity ? static_cast<const K *>(p.scratch) : static_cast<const K *>(p.keys);
  const bool small = m <= p.cutoff;
  const unsigned tiles = small ? 1u : tile_count<K, TILE>(buf, b, e);
  unsigned long long lbi = 0;
  if (!small) {
    lbi = atomicAdd(&ctl->lb_used, (unsigned long long)tiles);
    if (lbi + tiles > p.lb_cap) {
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
  it->lb = (unsigned)lbi;
  it->flags = (parity ? kItemScratch : 0u) | (small ? kItemSmall : 0u);
  ItemCtl *c = p.ictl + idx;
  c->grab = 0;
  c->done = 0;
  c->less = 0;
  __threadfence();
  st_release(&it->ready, epoch);
  return true;
}

// Thread 0 of a CTA: claim the next tile (or small item). Returns false when the
// queue has drained or the call was aborted.
__device__ __forceinline__ bool fetch_work(const SortParams &p, unsigned epoch, long long *h_out,
                                           unsigned *t_out, Item *it_out) {
  Control *ctl = p.ctl;
  unsigned ns = 32;
  unsigned long long idle_t0 = 0, last_completed = ~0ull;
  while (true) {
    if (ld_relaxed(&ctl->abort)) return false;
    const unsigned long long h = ld_relaxed(&ctl->head);
    const unsigned long long tail = ld_acquire(&ctl->pushed);
    if (h < tail && h < p.item_cap) {
      Item *ip = p.items + h;
      unsigned spins = 0;
      unsigned long long t0 = 0;
      while (ld_acquire(&ip->ready) != epoch) {
        if ((++spins & 255u) == 0u) {
          const unsigned long long now = globaltimer();
          if (t0 == 0) t0 = now;
          if (now - t0 > p.spin_limit_ns) {
            raise_error(ctl, &ctl->abort, kDevTimeout, 0x200000000ull | h);
            return false;
          }
          if (ld_relaxed(&ctl->abort)) return false;
        }
        __nanosleep(32);
      }
      Item it;
      it.begin = __ldcg(&ip->begin);
      it.end = __ldcg(&ip->end);
      it.tiles = __ldcg(&ip->tiles);
      it.lb = __ldcg(&ip->lb);
      it.flags = __ldcg(&ip->flags);
      it.ready = epoch;
      const unsigned t = atomicAdd(&p.ictl[h].grab, 1u);
      if (t < it.tiles) {
        *h_out = (long long)h;
        *t_out = t;
        *it_out = it;
        return true;
      }
      atomicCAS(&ctl->head, h, h + 1);
      ns = 32;
      continue;
    }
    // Nothing visible: finished when every pushed item has completed. `completed` is
    // read before `pushed`: items push their children before they count as completed.
    const unsigned long long c = ld_acquire(&ctl->completed);
    const unsigned long long pu = ld_acquire(&ctl->pushed);
    if (c == pu) return false;
    const unsigned long long now = globaltimer();
    if (c != last_completed) {
      last_completed = c;
      idle_t0 = now;
    } else if (now - idle_t0 > p.spin_limit_ns) {
      raise_error(ctl, &ctl->abort, kDevTimeout, 0x300000000ull | c);
      return false;
    }
    __nanosleep(ns);
    ns = ns < 1024 ? ns * 2 : 1024;
  }
}

template <int BLOCK, int JMAX>
struct SortShared {
  TileShared<BLOCK> tile;
  SmemShared<BLOCK, JMAX> fin;
  long long h;
  unsigned t;
  int has_work;
  int finisher;
  Item it;
};

// Persistent sort kernel: every CTA loops over the work queue until it drains.
template <typename K, int BLOCK, int IPT, int JMAX>
__global__ void __launch_bounds__(BLOCK) sort_kernel(SortParams p) {
  constexpr int TILE = BLOCK * IPT;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ SortShared<BLOCK, JMAX> sh;
  K *const buf0 = static_cast<K *>(p.keys);
  K *const buf1 = static_cast<K *>(p.scratch);
  Control *ctl = p.ctl;
  const unsigned epoch = *reinterpret_cast<volatile unsigned *>(&ctl->epoch);
  const int tid = threadIdx.x;
  unsigned long long st_tiles = 0, st_lb = 0, st_levels = 0, st_small = 0, st_small_keys = 0;
  unsigned long long st_large = 0, st_large_keys = 0;

  while (true) {
    if (tid == 0) sh.has_work = fetch_work(p, epoch, &sh.h, &sh.t, &sh.it) ? 1 : 0;
    __syncthreads();
    if (!sh.has_work) break;
    const Item it = sh.it;
    const long long h = sh.h;
    const unsigned t = sh.t;
    const unsigned par = it.flags & kItemScratch;
    K *src = par ? buf1 : buf0;
    K *dst = par ? buf0 : buf1;

    if (it.flags & kItemSmall) {
      const int m = (int)(it.end - it.begin);
      const bool fin_ok = smem_ksort<K, BLOCK, JMAX>(src + it.begin, buf0 + it.begin, m,
                                                     p.cutoff, smem, sh.fin, &st_levels);
      __threadfence();
      __syncthreads();
      if (tid == 0) {
        if (!fin_ok) raise_error(ctl, &ctl->abort, kDevInternal, 0x600000000ull | (unsigned)h);
        ++st_small;
        st_small_keys += (unsigned long long)m;
        atomicAdd(&ctl->completed, 1ull);
      }
    } else {
      unsigned long long less = 0;
      const bool ok = partition_tile<K, BLOCK, IPT>(
          src, dst, it.begin, it.end, t, p.lb + it.lb, epoch, p.spin_limit_ns, ctl, &ctl->abort,
          reinterpret_cast<K *>(smem), sh.tile, &less, &st_lb);
      if (!ok) break;
      __threadfence();
      __syncthreads();
      if (tid == 0) {
        ++st_tiles;
        if (t == it.tiles - 1) {
          atomicExch(&p.ictl[h].less, less);
          __threadfence();
        }
        const unsigned old = atomicAdd(&p.ictl[h].done, 1u);
        sh.finisher = old == it.tiles - 1;
        if (sh.finisher) {
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
          atomicAdd(&ctl->completed, 1ull);
        }
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (st_tiles) atomicAdd(&ctl->tiles, st_tiles);
    if (st_lb) atomicAdd(&ctl->lookback_steps, st_lb);
    if (st_levels) atomicAdd(&ctl->smem_levels, st_levels);
    if (st_small) atomicAdd(&ctl->small_items, st_small);
    if (st_small_keys) atomicAdd(&ctl->small_keys, st_small_keys);
    if (st_large) atomicAdd(&ctl->large_items, st_large);
    if (st_large_keys) atomicAdd(&ctl->large_keys, st_large_keys);
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
    ctl->completed = 0;
    ctl->head = 0;
    ctl->lb_used = 0;
    ctl->abort = 0;
    ctl->large_items = ctl->large_keys = ctl->tiles = 0;
    ctl->small_items = ctl->small_keys = 0;
    ctl->smem_levels = ctl->lookback_steps = 0;
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
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
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
