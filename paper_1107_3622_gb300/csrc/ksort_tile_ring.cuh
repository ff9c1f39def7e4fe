// Phase 1 of a sort (the tile passes of Steps 1-4 on every sub-array above the cutoff,
// with Steps 5-6 queuing their sides) through a ring of shared-memory tile slots:
// tile_ring_kernel, the staged form of the tile passes.
//
// Work comes from the same queue as tile_kernel: one ticket per tile pass, issued when
// the sub-array that owns it is queued. A CTA has three roles:
//   producer  (lane 0 of warp 0) claims tickets in order, waits until each is issued,
//             and stages the tile's keys into the next free slot by one bulk copy, with
//             at most DEPTH tiles of the CTA loading or waiting to be compacted;
//   data warps (NDW of them) each classify one warp sub-tile of 32 x IPT keys with
//             ballots and compact it in place (less keys to the front of the warp's
//             region, >= keys to its back), and publish their counts;
//   reservation warp (warp 1), tile by tile once every data warp has counted it: adds
//             the tile's (>= count << 32 | less count) to its sub-array's counter; the
//             value before the add places the tile's runs: less keys after the less keys
//             already placed, >= keys before the >= keys already placed, from the right
//             end. (When the last data warp did this itself, it fell behind on every
//             round trip and became the last warp of the next tile too.)
// Each data warp then writes its two runs with 128-bit stores. The last warp to write a
// tile counts it done in its sub-array; the one that completes the sub-array places its
// key at begin + #{x < key} (Step 4, the counter's final less count) and queues both
// sides (Steps 5-6).
// No tile waits for another tile, only for its own keys and its ticket; the order of the
// tiles' runs inside each side follows the order in which tiles finished (only the key
// index and the two sides' contents are defined). A data warp writes out every tile
// whose ranges are known before it waits for anything else, so a warp never holds
// unwritten keys while it waits for a ticket that only their sub-array can issue.
// Every wait is bounded by the tuned time limit; a timeout records KSORT_ERR_TIMEOUT,
// sets the sort's abort flag, and every CTA leaves.
#pragma once

#include "ksort_device.cuh"
#include "ksort_part_ring.cuh"

namespace ksort {
namespace dev {

// One compiled shape of the ring tile passes: NDW data warps of IPT keys per lane (a
// tile is NDW * 32 * IPT keys), S slots, MINB CTAs per SM, at most DEPTH tiles loading
// or waiting to be compacted.
template <typename K, int NDW_, int IPT_, int S_, int MINB_, int DEPTH_>
struct TileRingCfg {
  static constexpr int NDW = NDW_, IPT = IPT_, S = S_, MINB = MINB_;
  static constexpr int DEPTH = DEPTH_ < S_ ? DEPTH_ : S_;
  static constexpr int WT = 32 * IPT;
  static constexpr int TILE = NDW * WT;
  static constexpr int NT = (NDW + 2) * 32;  // producer, reservation warp, data warps
  static constexpr size_t SLOT = (size_t)TILE * sizeof(K) + 128;  // + copy_out_v's over-read
  static constexpr size_t SMEM = (size_t)S * SLOT;
  static_assert(TILE < 65536 && (TILE * sizeof(K)) % 128 == 0 && S >= 2, "bad ring shape");
};

template <int NDW, int S>
struct TileRingShared {
  unsigned long long full[S];   // slot holds its tile's keys (copy landed), or the end mark
  unsigned long long empty[S];  // every data warp has written its share out
  unsigned long long counted[S];  // every data warp has compacted its share (or seen the end)
  unsigned long long ready[S];  // the tile's output ranges are in lbase / gbase
  PipeTile info[S];             // the slot's tile: item, ticket, geometry (h < 0: end mark)
  unsigned cnt[S][NDW];         // per data warp: (valid keys << 16) | less keys
  unsigned wdone[S];            // data warps done writing the tile out
  long long lbase[S][NDW];      // buffer index of each data warp's first less key
  long long gbase[S][NDW];      // buffer index of each data warp's first >= key
  long long ch;                 // item whose record is cached in ci (producer)
  Item ci;
  int stop;                     // nonzero: leave (an error here or in another CTA)
};

// One warp, once every tile pass of item h is written and c = #{x < key} is known:
// Step 4 (the key to its final index) and Steps 5-6 (both sides queued, their tickets
// published by the warp's lanes), then the item counts as completed.
template <typename K, int TILE>
__device__ __forceinline__ void finish_item_warp(const SortParams &p, unsigned epoch,
                                                 const Item &it, long long h,
                                                 unsigned long long c) {
  const int lane = threadIdx.x & 31;
  Control *ctl = p.ctl;
  K *const buf0 = static_cast<K *>(p.keys);
  const unsigned par = it.flags & kItemScratch;
  K *dst = static_cast<K *>(par ? p.keys : p.scratch);
  const K key = bits_key<K>(it.key);
  unsigned long long cidx = 0, ct0 = 0;
  unsigned ctiles = 0;
  const long long kpos = it.begin + (long long)c;
  const bool bad = kpos >= it.end;
  if (lane == 0) {
    if (bad) {
      raise_error(ctl, kDevInternal, 0x700000000ull | (unsigned)h);
    } else if (it.flags & kItemPartitionOnly) {
      dst[kpos] = key;  // a single partition: the key index is the result
      if (p.key_index) *p.key_index = (long long)c;
    } else {
      buf0[kpos] = key;  // Step 4
    }
  }
  if (lane < 2 && !bad && !(it.flags & kItemPartitionOnly)) {
    // Steps 5-6: lanes 0 and 1 queue the two sides at once (each a chain of atomics)
    const unsigned cflags = par ^ kItemScratch;
    const long long cb = lane ? kpos + 1 : it.begin, ce = lane ? it.end : kpos;
    const long long mm = ce - cb;
    if (mm == 1) {
      if (cflags & kItemScratch) buf0[cb] = __ldcg(dst + cb);
    } else if (mm >= 2) {
      cidx = reserve_item<K, TILE>(p, epoch, cb, ce, cflags, &ct0, &ctiles);
    }
  }
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const unsigned long long ci = __shfl_sync(kFull, cidx, s);
    const unsigned long long t0 = __shfl_sync(kFull, ct0, s);
    const unsigned nt = __shfl_sync(kFull, ctiles, s);
    if (nt) publish_tickets(p, epoch, ci, t0, nt, lane, 32);
  }
  __syncwarp();
  if (lane == 0) {
    __threadfence();
    atomicAdd(&ctl->large_completed, 1ull);
  }
}

template <typename K, int NDW, int IPT, int S, int MINB, int DEPTH_>
__global__ void __launch_bounds__((NDW + 2) * 32, MINB) tile_ring_kernel(SortParams p) {
  using C = TileRingCfg<K, NDW, IPT, S, MINB, DEPTH_>;
  constexpr int WT = C::WT, TILE = C::TILE, DEPTH = C::DEPTH;
  extern __shared__ __align__(128) unsigned char tring_smem[];
  __shared__ TileRingShared<NDW, S> sh;
  auto slot = [&](int s) { return reinterpret_cast<K *>(tring_smem + (size_t)s * C::SLOT); };
  Control *const ctl = p.ctl;
  grid_dep_wait();
  grid_dep_launch();
  const unsigned epoch = *reinterpret_cast<volatile unsigned *>(&ctl->epoch);
  const unsigned long long limit = p.spin_limit_ns;
  volatile int *const stop = &sh.stop;
  const SortStop stp{stop, &ctl->abort};
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto fail = [&](unsigned code, unsigned long long info) {
    *stop = 1;
    raise_error(ctl, code, info);  // also sets the sort's abort flag
  };

  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < S; ++s) {
      mbar_init(&sh.full[s], 1);
      mbar_init(&sh.empty[s], NDW);
      mbar_init(&sh.counted[s], NDW);
      mbar_init(&sh.ready[s], 1);
      sh.wdone[s] = 0;
    }
    sh.stop = 0;
    sh.ch = -1;
    fence_mbar_init();
  }
  __syncthreads();

  int last_use[S];  // ring index of the last copy or end mark put in each slot (producer)
#pragma unroll
  for (int s = 0; s < S; ++s) last_use[s] = -1;
  unsigned long long st_tiles = 0, st_large = 0, st_large_keys = 0;

  if (warp == 0) {
    // ---------------------------------------------------------------- producer
    if (lane == 0) {
      unsigned long long k = atomicAdd(&ctl->tq_head, 1ull);
      for (int i = 0;; ++i) {
        const int s = i % S;
        int st = 0;
        if (i >= S)  // the slot's previous tile must have been written out
          st = ring_wait_one(&sh.empty[s], (unsigned)((i / S) - 1) & 1u, limit, stp);
        if (!st && DEPTH < S && i >= DEPTH)  // tile i - DEPTH must have been compacted
          st = ring_wait_one(&sh.counted[(i - DEPTH) % S], (unsigned)((i - DEPTH) / S) & 1u,
                             limit, stp);
        if (st) {
          if (st == 1) fail(kDevTimeout, 0x1300000000ull | (unsigned)i);
          break;
        }
        long long h = 0;
        const int r = *stop ? -1 : wait_ticket(p, epoch, k, &h);
#pragma unroll
        for (int u = 0; u < S; ++u)
          if (u == s) last_use[u] = i;
        if (r <= 0) {  // phase 1 is over (or stopped): end mark
          sh.info[s].h = -1;
          mbar_arrive(&sh.full[s]);
          if (r < 0) *stop = 1;
          break;
        }
        pipe_geom<K, TILE>(p, sh.info[s], &sh.ci, &sh.ch, k, h);
        trace_mark(p, k, 0);  // ticket issued, copy starts
        pipe_issue<K>(p, sh.info[s], slot(s), &sh.full[s]);
        k = atomicAdd(&ctl->tq_head, 1ull);  // the next claim overlaps this copy
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------------------------------------------------------- reservation
    // Tile by tile, once every data warp has compacted its share: the tile's output
    // ranges in its item by one 64-bit add of (>= << 32 | less) to the item's counter
    // (the value before it counts the tiles that reserved earlier), then the tile is
    // released for writing. The data warps never wait on this round trip themselves.
    for (int i = 0;; ++i) {
      const int s = i % S;
      const int st = ring_wait_warp(&sh.counted[s], (unsigned)(i / S) & 1u, limit, stp);
      if (st) {
        if (st == 1 && lane == 0) fail(kDevTimeout, 0x1600000000ull | (unsigned)i);
        break;
      }
      const PipeTile &pt = sh.info[s];
      if (pt.h < 0) break;  // the end mark
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
      const unsigned Lt = tot & 0xffffu, Gt = tot >> 16;
      unsigned long long pre = 0;
      if (lane == 0) pre = atomicAdd(&p.ictl[pt.h].less, ((unsigned long long)Gt << 32) | Lt);
      pre = __shfl_sync(kFull, pre, 0);
      const long long PL = (long long)(pre & 0xffffffffull), PG = (long long)(pre >> 32);
      const long long lb0 = pt.it.begin + PL, gb0 = pt.it.end - PG - (long long)Gt;
      if (!ranges_ok(pt.it.begin, pt.it.end, lb0, Lt, gb0, Gt)) {
        if (lane == 0) fail(kDevInternal, 0x1400000000ull | (unsigned)pt.t);  // never released
        break;
      }
      if (lane < NDW) {
        sh.lbase[s][lane] = lb0 + (long long)(ex & 0xffffu);
        sh.gbase[s][lane] = gb0 + (long long)(ex >> 16);
      }
      __syncwarp();
      if (lane == 0) {
        trace_mark(p, pt.k, 3);  // ranges known
        mbar_arrive(&sh.ready[s]);
      }
    }
  } else {
    // ---------------------------------------------------------------- data warps
    const int dw = warp - 2;
    K *const buf0 = static_cast<K *>(p.keys);
    K *const buf1 = static_cast<K *>(p.scratch);
    // this warp's two runs of the CTA's j-th tile go out; the last warp to write a tile
    // counts it done in its item, and the warp that completes the item finishes it
    auto write_tile = [&](int j) {
      const int s = j % S;
      const unsigned c = sh.cnt[s][dw];
      const unsigned L = c & 0xffffu, G = (c >> 16) - L;
      const K *reg = slot(s) + dw * WT;
      K *dst = (sh.info[s].it.flags & kItemScratch) ? buf0 : buf1;
      copy_out_v<K, 32>(reg, dst + sh.lbase[s][dw], L, lane);
      copy_out_v<K, 32>(reg + WT - G, dst + sh.gbase[s][dw], G, lane);
      __syncwarp();
      int last = 0;
      if (lane == 0) {
        __threadfence_block();  // this warp's stores before its count
        last = atomicAdd(&sh.wdone[s], 1u) == (unsigned)NDW - 1u;
      }
      last = __shfl_sync(kFull, last, 0);
      if (last) {  // every warp has written the tile: it is done in its item
        const Item it = sh.info[s].it;
        const long long h = sh.info[s].h;
        int fin = 0;
        unsigned long long less = 0;
        if (lane == 0) {
          sh.wdone[s] = 0;
          trace_mark(p, sh.info[s].k, 4);  // written
          __threadfence();  // the tile's stores, and the other warps' before them
          fin = atom_add_release(&p.ictl[h].done, 1u) == it.tiles - 1u;
          if (fin) {
            __threadfence();
            less = ld_acquire(&p.ictl[h].less) & 0xffffffffull;  // every tile has added
          }
        }
        fin = __shfl_sync(kFull, fin, 0);
        less = __shfl_sync(kFull, less, 0);
        ++st_tiles;
        if (fin) {
          finish_item_warp<K, TILE>(p, epoch, it, h, less);
          ++st_large;
          st_large_keys += (unsigned long long)(it.end - it.begin);
        }
      }
      fence_proxy_async_smem();  // the slot's next keys arrive by a bulk copy
      __syncwarp();
      if (lane == 0) mbar_arrive(&sh.empty[s]);
    };
    int i = 0;       // next of the CTA's tiles to compact
    int wnext = 0;   // next of them this warp writes out
    int end = -1;    // ring index of the end mark, once seen
    unsigned long long t0 = 0;
    for (unsigned k = 0;; ++k) {
      bool progress = false;
      // every tile whose ranges are known goes out first
      while (wnext < i && __all_sync(kFull, mbar_test(&sh.ready[wnext % S], (unsigned)(wnext / S) & 1u))) {
        write_tile(wnext++);
        progress = true;
      }
      if (end >= 0) {
        if (wnext == end) break;
      } else if (__all_sync(kFull, mbar_test(&sh.full[i % S], (unsigned)(i / S) & 1u))) {
        const int s = i % S;
        const PipeTile &pt = sh.info[s];
        if (pt.h < 0) {
          end = i;
          __syncwarp();
          if (lane == 0) mbar_arrive(&sh.counted[s]);  // the reservation warp sees it too
          continue;
        }
        const int e0 = dw * WT;
        const int a = min(WT, max(0, pt.vlo - e0)), b = min(WT, max(0, pt.vhi - e0));
        const K key = bits_key<K>(pt.it.key);  // Step 1: the item's first element
        K *reg = slot(s) + e0;
        unsigned L = 0, G = 0;
        if (a == 0 && b == WT) ring_compact<K, IPT, true>(reg, key, a, b, &L, &G);
        else ring_compact<K, IPT, false>(reg, key, a, b, &L, &G);
        __syncwarp();
        if (lane == 0) {
          sh.cnt[s][dw] = ((L + G) << 16) | L;
          mbar_arrive(&sh.counted[s]);  // release: the count before the arrival
        }
        ++i;
        progress = true;
      }
      if (progress) {
        t0 = 0;
        continue;
      }
      // nothing to do: sleep on what comes next (the oldest unwritten tile's ranges, or
      // the next tile's keys), then check the limit and the stop flags
      if (wnext < i) (void)__all_sync(kFull, mbar_try_wait(&sh.ready[wnext % S], (unsigned)(wnext / S) & 1u));
      else if (end < 0) (void)__all_sync(kFull, mbar_try_wait(&sh.full[i % S], (unsigned)(i / S) & 1u));
      int r = 0;
      if (lane == 0) {
        if (*stop) r = 2;
        else if ((k & 7u) == 7u) {
          const unsigned long long now = globaltimer();
          if (t0 == 0) t0 = now;
          else if (now - t0 > limit) r = 1;
          if (!r && stp.now()) r = 2;
        }
      }
      r = __shfl_sync(kFull, r, 0);
      if (r) {
        if (r == 1 && lane == 0) fail(kDevTimeout, 0x1500000000ull | (unsigned)i);
        break;
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
  }
  // statistics of the data warps (lane 0 of each counts what it finished)
  if (warp > 0 && lane == 0) {
    if (st_tiles) atomicAdd(&ctl->tiles, st_tiles);
    if (st_large) atomicAdd(&ctl->large_items, st_large);
    if (st_large_keys) atomicAdd(&ctl->large_keys, st_large_keys);
  }
}

}  // namespace dev
}  // namespace ksort
