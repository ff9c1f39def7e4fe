// ksort_cluster.cuh — the upper recursion levels of one array inside a thread-block
// cluster (Steps 1-6 of Section 1.1 on every sub-array above the cutoff).
//
// A work-queue level costs a chain of dependent global round trips (claim, load,
// reserve, write, completion, queueing the sides: about 8 us per level on this two-die
// GPU), which dominates sorts of small arrays. Here one cluster of C CTAs keeps the
// whole array in shared memory: CTA r holds indices [r * sl, (r + 1) * sl) in two
// buffers, and every CTA keeps the same table of the active sub-arrays (those above
// the cutoff) of the current level. One level partitions all of them at once:
//
//   1. each thread classifies a contiguous chunk of its CTA's slice, every key against
//      the key of the sub-array it lies in (Step 3: key <= x goes right);
//   2. a CTA-wide exclusive scan of the (less, >=) counts. Sub-arrays are contiguous
//      ranges, so the count of one sub-array's keys before a position equals the scan
//      there minus the scan at the sub-array's first classified key in this CTA;
//   3. cluster barrier; each CTA reads every CTA's per-sub-array counts through
//      distributed shared memory and sums those of the CTAs before it;
//   4. each key is stored, through distributed shared memory, into the other buffer of
//      the CTA that owns its destination: less keys from the sub-array's front in index
//      order, >= keys from its back in index order (the layout of the tile passes), the
//      key at begin + #less (Step 4); keys outside every active sub-array are copied
//      in place;
//   5. cluster barrier; every CTA builds the next table from the same counts and keys
//      (Steps 5-6): sides above the cutoff stay active, sides of 2 .. cutoff keys go to
//      the small-item list of the work queue (CTA 0 queues them).
//
// When no sub-array is left above the cutoff, each CTA writes its slice back to buffer 0
// and the finisher (small_kernel) takes the small items as usual. Nothing waits except
// at the cluster and CTA barriers, so any input, however unbalanced its partitions,
// only takes more levels.
#pragma once

#include <cooperative_groups.h>

namespace ksort {
namespace dev {

namespace cg = cooperative_groups;

constexpr int kClusterThreads = 1024;
constexpr int kClusterMaxChunk = 32;  // keys per thread: a 32-bit mask per thread
constexpr int kClusterMaxCtas = 16;   // largest cluster launched
constexpr int kClusterMaxSmall = 512;  // small sides CTA 0 keeps to queue at the end

template <typename K>
struct ClusterShared {
  int tb[2][kClusterMaxSegs], te[2][kClusterMaxSegs];  // active sub-arrays [b, e), by parity
  K tk[2][kClusterMaxSegs];                            // and their keys (first elements)
  unsigned long long cnt[kClusterMaxSegs];   // this CTA's (>= << 32 | less) per sub-array
  unsigned long long base[kClusterMaxSegs];  // scan at its first classified key here
  unsigned long long endp[kClusterMaxSegs];  // scan just after its last classified key here
  unsigned long long pre[kClusterMaxSegs];   // counts of the CTAs before this one
  unsigned long long tot[kClusterMaxSegs];   // counts of all CTAs
  unsigned long long wsum[32];
  int sb[kClusterMaxSmall], se[kClusterMaxSmall];  // CTA 0: small sides to queue at the end
  K sk[kClusterMaxSmall];
  int nsmall;
  int nseg[2];
  unsigned long long level_keys;
  unsigned epoch;
};

// First active sub-array with end > gi (ns if none): TE is ascending.
__device__ __forceinline__ int seg_after(const int *TE, int ns, int gi) {
  int lo = 0, hi = ns;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (TE[mid] <= gi) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// CTA-wide exclusive scan of one 64-bit value per thread (two 32-bit counts that never
// carry into each other), kClusterThreads threads. Contains two CTA barriers.
__device__ __forceinline__ unsigned long long cluster_block_scan(unsigned long long v,
                                                                 unsigned long long *wsum) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long u = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const unsigned long long w = wsum[lane];
    unsigned long long wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long u = __shfl_up_sync(kFull, wi, o);
      if (lane >= o) wi += u;
    }
    wsum[lane] = wi - w;
  }
  __syncthreads();
  return wsum[warp] + incl - v;
}

// One thread of CTA 0: queues [b, e) (2 .. cutoff keys, in buffer 0 once the kernel has
// written its slices back) on the small-item list.
template <typename K>
__device__ __forceinline__ void cluster_push_small(const SortParams &p, unsigned epoch,
                                                   long long b, long long e, K key) {
  Control *ctl = p.ctl;
  if (!sub_array_ok(p, b, e, 1)) return;
  const unsigned long long idx = atomicAdd(&ctl->pushed, 1ull);
  if (idx >= p.item_cap) {
    raise_error(ctl, kDevWorkspaceExhausted, 9);
    return;
  }
  Item *it = p.items + idx;
  it->begin = b;
  it->end = e;
  it->key = key_bits<K>(key);
  it->tiles = 1;
  it->lb = 0;
  it->flags = kItemSmall;
  it->epoch = epoch;
  __threadfence();
  const unsigned long long qi = atomicAdd(&ctl->sq_tail, 1ull);  // qi <= idx < item_cap
  st_release(&p.small_q[qi], q_entry(epoch, idx));
}

// Diagnostics (ksort_debug_trace): stamp j of level k, by CTA 0's thread 0.
__device__ __forceinline__ void cluster_mark(const SortParams &p, bool on, unsigned long long k,
                                             int j) {
  if (on && k < (unsigned long long)p.trace_cap) p.trace[k * kTraceWords + j] = globaltimer();
}

// One cluster of C CTAs (cluster dimension C, grid C), kClusterThreads threads each;
// `sl` keys per CTA slice (a multiple of 4, at most kClusterMaxChunk per thread), dynamic
// shared memory 2 * sl keys. p.total <= C * sl, and fewer than kClusterMaxSegs
// sub-arrays above p.cutoff can exist at once (both host-checked).
template <typename K>
__global__ void __launch_bounds__(kClusterThreads, 1) cluster_kernel(SortParams p, int sl) {
  extern __shared__ __align__(16) unsigned char csmem[];
  __shared__ ClusterShared<K> sh;
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int r = (int)cl.block_rank();
  const int tid = threadIdx.x;
  K *const s0 = reinterpret_cast<K *>(csmem);
  K *const s1 = s0 + sl;
  K *const g = static_cast<K *>(p.keys);
  const int n = (int)p.total;
  const int lo = r * sl;
  const int hi = min(n, lo + sl);
  const int len = max(0, hi - lo);
  Control *ctl = p.ctl;
  grid_dep_wait();    // the previous launch in the stream is complete
  grid_dep_launch();  // the finisher may start launching; it waits for this one
  if (r == 0 && tid == 0) sh.epoch = start_generation(ctl);
  for (int i = tid; i < len; i += kClusterThreads) s0[i] = __ldcg(g + lo + i);
  if (tid == 0) {
    sh.nseg[0] = 1;
    sh.tb[0][0] = 0;
    sh.te[0][0] = n;
    sh.nsmall = 0;
  }
  cl.sync();  // every slice is loaded; the root's key (Step 1) is element 0, in CTA 0
  if (tid == 0) sh.tk[0][0] = *cl.map_shared_rank(s0, 0);
  __syncthreads();

  // chunk of q keys per thread; q odd, so a warp's 32 chunk starts fall in 32 different
  // shared-memory banks
  const int q = ((len + kClusterThreads - 1) / kClusterThreads) | 1;
  const int c0 = min(len, tid * q), c1 = min(len, c0 + q);
  int cur = 0, tp = 0;
  unsigned long long st_items = 0, st_keys = 0, st_levels = 0;
  bool bad = false;
  const bool tr = p.trace != nullptr && r == 0 && tid == 0;
  while (sh.nseg[tp] > 0) {
    const int ns = sh.nseg[tp];
    const int *TB = sh.tb[tp], *TE = sh.te[tp];
    const K *TK = sh.tk[tp];
    const K *X = cur ? s1 : s0;
    K *Y = cur ? s0 : s1;
    for (int s = tid; s < ns; s += kClusterThreads) {
      sh.base[s] = 0;
      sh.endp[s] = 0;
    }
    if (tid == 0) sh.level_keys = 0;
    cluster_mark(p, tr, st_levels, 0);
    if (tr && st_levels < (unsigned long long)p.trace_cap) p.trace[st_levels * kTraceWords + 7] = ns;
    __syncthreads();

    // 1. classify the chunk (bit k of act / left: position c0 + k is a classified key /
    //    goes left of its sub-array's key), noting where a sub-array's classified keys in
    //    this slice start or end: a chunk of at most 32 keys meets at most two of each,
    //    since active sub-arrays have more than cutoff >= 64 keys
    unsigned act = 0, left = 0;
    unsigned long long run = 0, bv[2] = {0, 0}, ev[2] = {0, 0};
    int bs[2] = {-1, -1}, es[2] = {-1, -1}, nb = 0, ne = 0;
    {
      int s = seg_after(TE, ns, lo + c0);
      for (int i = c0; i < c1; ++i) {
        const int gi = lo + i;
        while (s < ns && TE[s] <= gi) ++s;
        if (s < ns && TB[s] < gi) {  // the key itself, at TB[s], is not classified
          if (gi == max(TB[s] + 1, lo)) {
            if (nb == 0) { bs[0] = s; bv[0] = run; }
            else { bs[1] = s; bv[1] = run; }
            ++nb;
          }
          act |= 1u << (i - c0);
          if (goes_left(TK[s], X[i])) {
            left |= 1u << (i - c0);
            run += 1ull;
          } else {
            run += 1ull << 32;
          }
          if (gi == min(TE[s], hi) - 1) {
            if (ne == 0) { es[0] = s; ev[0] = run; }
            else { es[1] = s; ev[1] = run; }
            ++ne;
          }
        }
      }
    }
    const unsigned long long excl = cluster_block_scan(run, sh.wsum);
    cluster_mark(p, tr, st_levels, 1);

    // 2. the scan at each sub-array's first classified key in this slice, and after its
    //    last; their difference is this CTA's (>=, less) count of the sub-array
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      if (bs[k] >= 0) sh.base[bs[k]] = excl + bv[k];
      if (es[k] >= 0) sh.endp[es[k]] = excl + ev[k];
    }
    __syncthreads();
    for (int s = tid; s < ns; s += kClusterThreads) sh.cnt[s] = sh.endp[s] - sh.base[s];
    cl.sync();  // 3. every CTA's counts are ready
    cluster_mark(p, tr, st_levels, 2);

    for (int s = tid; s < ns; s += kClusterThreads) {
      unsigned long long v[kClusterMaxCtas], before = 0, all = 0;
#pragma unroll
      for (int rr = 0; rr < kClusterMaxCtas; ++rr)  // all loads in flight at once
        v[rr] = rr < C ? *cl.map_shared_rank(&sh.cnt[s], rr) : 0ull;
#pragma unroll
      for (int rr = 0; rr < kClusterMaxCtas; ++rr) {
        if (rr < r) before += v[rr];
        all += v[rr];
      }
      sh.pre[s] = before;
      sh.tot[s] = all;
      atomicAdd(&sh.level_keys, (unsigned long long)(TE[s] - TB[s]));
    }
    __syncthreads();
    cluster_mark(p, tr, st_levels, 3);

    // 4. every key of the chunk to its place in the other buffer of the CTA that owns it
    {
      int s = seg_after(TE, ns, lo + c0);
      unsigned long long run = excl;
      for (int i = c0; i < c1; ++i) {
        const int gi = lo + i;
        while (s < ns && TE[s] <= gi) ++s;
        const unsigned bit = 1u << (i - c0);
        int d = gi, db = 0, de = n;
        if (act & bit) {
          const unsigned long long within = run - sh.base[s];
          const unsigned long long pr = sh.pre[s];
          const int L = (int)(sh.tot[s] & 0xffffffffull);
          if (left & bit) {  // Step 3.1: from the front, in index order
            d = TB[s] + (int)(pr & 0xffffffffull) + (int)(within & 0xffffffffull);
            db = TB[s];
            de = TB[s] + L;
            run += 1ull;
          } else {  // Step 3.2: from the back, in index order
            d = TE[s] - 1 - (int)(pr >> 32) - (int)(within >> 32);
            db = TB[s] + L + 1;
            de = TE[s];
            run += 1ull << 32;
          }
        } else if (s < ns && TB[s] == gi) {
          d = gi + (int)(sh.tot[s] & 0xffffffffull);  // Step 4: the key's final index
        }
        if (d < db || d >= de) {  // inconsistent counts: report, store nothing
          bad = true;
          continue;
        }
        const int owner = d / sl;
        if (owner == r) Y[d - lo] = X[i];
        else *cl.map_shared_rank(Y + (d - owner * sl), owner) = X[i];
      }
    }
    cluster_mark(p, tr, st_levels, 4);
    cl.sync();  // 5. every key of the level has landed
    cluster_mark(p, tr, st_levels, 5);

    // Steps 5-6: the sides of sub-array s are candidates 2 s and 2 s + 1
    {
      const int j = tid;
      int keep = 0, cb = 0, ce = 0;
      K ck = K(0);
      if (j < 2 * ns) {
        const int s = j >> 1;
        const int L = (int)(sh.tot[s] & 0xffffffffull);
        cb = (j & 1) ? TB[s] + L + 1 : TB[s];
        ce = (j & 1) ? TE[s] : TB[s] + L;
        const int m = ce - cb;
        if (m >= 2) {
          const int owner = cb / sl;
          ck = *cl.map_shared_rank(Y + (cb - owner * sl), owner);  // the side's first key
        }
        if (m > p.cutoff) {
          keep = 1;
        } else if (m >= 2 && r == 0) {  // a small side: queued when the kernel ends
          const int k = atomicAdd(&sh.nsmall, 1);
          if (k < kClusterMaxSmall) {
            sh.sb[k] = cb;
            sh.se[k] = ce;
            sh.sk[k] = ck;
          } else {
            cluster_push_small<K>(p, sh.epoch, cb, ce, ck);  // the list is full: now
          }
        }
      }
      const unsigned long long pos = cluster_block_scan((unsigned long long)keep, sh.wsum);
      const int nt = tp ^ 1;
      if (keep && pos < (unsigned long long)kClusterMaxSegs) {
        sh.tb[nt][pos] = cb;
        sh.te[nt][pos] = ce;
        sh.tk[nt][pos] = ck;
      } else if (keep) {
        bad = true;  // more active sub-arrays than the table holds: the host bound failed
      }
      if (j == 2 * ns - 1) sh.nseg[nt] = (int)min(pos + keep, (unsigned long long)kClusterMaxSegs);
      if (tid == 0) {
        st_items += (unsigned long long)ns;
        st_keys += sh.level_keys;
        cluster_mark(p, tr, st_levels, 6);
        ++st_levels;
      }
    }
    __syncthreads();
    cur ^= 1;
    tp ^= 1;
  }

  const K *F = cur ? s1 : s0;
  for (int i = tid; i < len; i += kClusterThreads) g[lo + i] = F[i];
  if (r == 0)
    for (int k = tid; k < min(sh.nsmall, kClusterMaxSmall); k += kClusterThreads)
      cluster_push_small<K>(p, sh.epoch, sh.sb[k], sh.se[k], sh.sk[k]);
  if (bad) raise_error(ctl, kDevInternal, 0xD00000000ull | (unsigned)r);
  if (r == 0 && tid == 0) {
    atomicAdd(&ctl->large_items, st_items);
    atomicAdd(&ctl->large_keys, st_keys);
    atomicAdd(&ctl->tiles, st_levels);  // the cluster form counts levels as its passes
  }
  cl.sync();  // no CTA leaves while another may still read its shared memory
}

}  // namespace dev
}  // namespace ksort
