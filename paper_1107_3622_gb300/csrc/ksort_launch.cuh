// Host-side launchers for one key type. Included once per key type by
// ksort_f32.cu / ksort_f64.cu / ksort_u32.cu, which each instantiate Launcher<K>.
#pragma once

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

#include "ksort_device.cuh"
#include "ksort_part_ring.cuh"
#include "ksort_tile_ring.cuh"
#include "ksort_cluster.cuh"

namespace ksort {

// Allows `fn` `smem` bytes of dynamic shared memory on the current device and, with
// `carve`, asks for the largest shared-memory carveout. The runtime keeps function
// attributes per device, so the driver calls are made only when the function does not
// yet have this limit there (one launch otherwise pays them every time).
inline cudaError_t allow_smem(void (*fn)(SortParams), size_t smem, bool carve) {
  static std::mutex mu;
  static std::map<std::pair<const void *, int>, size_t> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  const std::pair<const void *, int> key(reinterpret_cast<const void *>(fn), dev);
  auto it = done.find(key);
  if (it != done.end() && it->second == smem) return cudaSuccess;
  if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
      cudaSuccess)
    return e;
  if (carve && (e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         (int)cudaSharedmemCarveoutMaxShared)) != cudaSuccess)
    return e;
  done[key] = smem;
  return cudaSuccess;
}

// Compiled tile shapes (threads x keys per thread) of the tile passes, picked at run
// time by the tuning's tile shape; every shape moves 128-bit vectors. Variant 0 is the
// default: 32 KiB tiles of 512 threads.
template <typename K> struct Shapes;
template <> struct Shapes<float> {
  static constexpr int NT[kTileShapes] = {512, 512, 256};
  static constexpr int IPT[kTileShapes] = {16, 8, 16};
};
template <> struct Shapes<unsigned> {
  static constexpr int NT[kTileShapes] = {512, 512, 256};
  static constexpr int IPT[kTileShapes] = {16, 8, 16};
};
template <> struct Shapes<double> {
  static constexpr int NT[kTileShapes] = {512, 512, 256};
  static constexpr int IPT[kTileShapes] = {8, 4, 8};
};

// Shapes of form 1 (tile_ring_kernel): data warps x keys per lane, slots, CTAs per SM,
// tiles loading or awaiting compaction. 8-byte keys take half the keys per lane.
template <typename K, int SH> struct RingSortOf;
template <typename K> struct RingSortOf<K, 0> {  // 16 KiB tiles, 6 slots, 2 CTAs per SM
  using Cfg = dev::TileRingCfg<K, 8, 64 / (int)sizeof(K), 6, 2, 3>;
};
template <typename K> struct RingSortOf<K, 1> {  // 8 KiB tiles, 8 slots, 3 CTAs per SM
  using Cfg = dev::TileRingCfg<K, 8, 32 / (int)sizeof(K), 8, 3, 3>;
};
template <typename K> struct RingSortOf<K, 2> {  // 32 KiB tiles, 6 slots, 1 CTA per SM
  using Cfg = dev::TileRingCfg<K, 16, 64 / (int)sizeof(K), 6, 1, 3>;
};

// Variant V: CTA shape V % kTileShapes in form V / kTileShapes (0 registers; 1 a ring of
// shared-memory tiles, with its own three shapes; 2 warp roles, whose tile is the data
// warps' share: two warps load and look back; 3 wave levels, whose work queue then runs
// form 0 of the same shape).
template <typename K, int V>
struct ShapeOf {
  static constexpr int FORM = V / kTileShapes;
  using Ring = typename RingSortOf<K, V % kTileShapes>::Cfg;
  static constexpr int NT = FORM == 1 ? Ring::NT : Shapes<K>::NT[V % kTileShapes];
  static constexpr int IPT = FORM == 1 ? Ring::IPT : Shapes<K>::IPT[V % kTileShapes];
  static constexpr int TILE = FORM == 1 ? Ring::TILE : (FORM == 2 ? NT - 64 : NT) * IPT;
  static constexpr bool STAGED = FORM == 1 || FORM == 2;
  static constexpr size_t SMEM = FORM == 2   ? dev::ws_smem_bytes<K, TILE>()
                                 : FORM == 1 ? Ring::SMEM
                                             : 0;
};

// Calls f(ShapeOf<K, v>{}) for the run-time variant v (out-of-range values: variant 0).
template <typename K, typename F>
decltype(auto) with_shape(int v, F &&f) {
  switch (v) {
    case 1: return f(ShapeOf<K, 1>{});
    case 2: return f(ShapeOf<K, 2>{});
    case 3: return f(ShapeOf<K, 3>{});
    case 4: return f(ShapeOf<K, 4>{});
    case 5: return f(ShapeOf<K, 5>{});
    case 6: return f(ShapeOf<K, 6>{});
    case 7: return f(ShapeOf<K, 7>{});
    case 8: return f(ShapeOf<K, 8>{});
    case 9: return f(ShapeOf<K, 9>{});
    case 10: return f(ShapeOf<K, 10>{});
    case 11: return f(ShapeOf<K, 11>{});
    default: return f(ShapeOf<K, 0>{});
  }
}

// The tile-pass kernel of a variant, with its dynamic shared memory allowed.
template <typename K, typename S>
cudaError_t tile_kernel_of(void (**fn)(SortParams)) {
  if constexpr (S::STAGED) {
    if constexpr (S::FORM == 2) {
      *fn = dev::tile_ws_kernel<K, S::NT, S::IPT>;
    } else {
      using R = typename S::Ring;
      *fn = dev::tile_ring_kernel<K, R::NDW, R::IPT, R::S, R::MINB, R::DEPTH>;
    }
    return allow_smem(*fn, S::SMEM, true);
  } else {
    *fn = dev::tile_kernel<K, S::NT, S::IPT, false>;
    return cudaSuccess;
  }
}

// Largest shared-memory cutoff: two staging buffers of cutoff keys must fit in one
// CTA's shared memory (227 KB), so 8-byte keys stop at half the 4-byte limit.
template <typename K>
constexpr int max_cutoff() { return sizeof(K) == 8 ? dev::kMaxSmallCutoff / 2 : dev::kMaxSmallCutoff; }
static_assert(dev::small_smem_bytes<double>(max_cutoff<double>(), 1024) <= 227 * 1024, "smem");
static_assert(dev::small_smem_bytes<float>(max_cutoff<float>(), 1024) <= 227 * 1024, "smem");

// The finisher kernel of nt threads (256, 512 or 1024; anything else: 256), with its
// dynamic shared memory for `cutoff`-key items allowed.
template <typename K>
cudaError_t small_kernel_of(int nt, int cutoff, void (**fn)(SortParams), size_t *smem) {
  *fn = nt == 1024 ? dev::small_kernel<K, 1024>
      : nt == 512  ? dev::small_kernel<K, 512>
                   : dev::small_kernel<K, dev::kSmallThreads>;
  *smem = dev::small_smem_bytes<K>(cutoff, small_threads_of(nt));
  return allow_smem(*fn, *smem, false);
}

template <typename K>
KernelInfo Launcher<K>::info(int variant) {
  return with_shape<K>(variant, [](auto s) {
    using S = decltype(s);
    return KernelInfo{S::NT, S::TILE, max_cutoff<K>(), S::IPT, S::FORM};
  });
}

template <typename K>
size_t Launcher<K>::small_smem_bytes(int cutoff) {
  return dev::small_smem_bytes<K>(cutoff);
}

template <typename K>
long long Launcher<K>::tile_count(int variant, const void *buf, long long begin, long long end) {
  return with_shape<K>(variant, [&](auto s) {
    using S = decltype(s);
    return (long long)dev::tile_count<K, S::TILE>(static_cast<const K *>(buf), begin, end);
  });
}

template <typename K>
cudaError_t Launcher<K>::occupancy(int variant, int cutoff, int nt, int *tile_ctas,
                                   int *small_ctas) {
  cudaError_t e = with_shape<K>(variant, [&](auto s) {
    using S = decltype(s);
    void (*fn)(SortParams) = nullptr;
    cudaError_t e2 = tile_kernel_of<K, S>(&fn);
    if (e2 != cudaSuccess) return e2;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(tile_ctas, fn, S::NT, S::SMEM);
  });
  if (e != cudaSuccess) return e;
  void (*sk)(SortParams) = nullptr;
  size_t smem = 0;
  e = small_kernel_of<K>(nt, cutoff, &sk, &smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(small_ctas, sk, small_threads_of(nt), smem);
}

// Launches fn<<<grid, block, smem, s>>>(p) under programmatic stream serialization: its
// CTAs may become resident while the previous kernel in the stream finishes, and wait
// in grid_dep_wait() until that kernel's memory is complete, so the launch latency
// overlaps the previous kernel's tail.
inline cudaError_t launch_after(void (*fn)(SortParams), int grid, int block, size_t smem,
                                const SortParams &p, cudaStream_t s) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, fn, p);
}

template <typename K>
cudaError_t Launcher<K>::seed(const SortParams &p, int variant, cudaStream_t st) {
  with_shape<K>(variant, [&](auto s) {
    using S = decltype(s);
    dev::seed_kernel<K, S::TILE><<<1, 1024, 0, st>>>(p);
    return 0;
  });
  return cudaGetLastError();
}

template <typename K>
cudaError_t Launcher<K>::tiles(const SortParams &p, int variant, int grid, cudaStream_t st) {
  return with_shape<K>(variant, [&](auto s) {
    using S = decltype(s);
    void (*fn)(SortParams) = nullptr;
    cudaError_t e = tile_kernel_of<K, S>(&fn);
    if (e != cudaSuccess) return e;
    return launch_after(fn, grid, S::NT, S::SMEM, p, st);
  });
}

// The fused tile kernel (queue form, CTA shape 2: 256 threads), with its dynamic shared
// memory for the finisher of `cutoff`-key items allowed.
template <typename K>
cudaError_t fused_kernel_of(int cutoff, void (**fn)(SortParams), size_t *smem) {
  using S = ShapeOf<K, kFusedVariant>;
  static_assert(S::FORM == 0 && S::NT == 256, "fused shape");
  *fn = dev::tile_kernel<K, S::NT, S::IPT, true>;
  *smem = dev::fuse_smem_bytes<K>(cutoff, S::NT);
  return allow_smem(*fn, *smem, false);
}

template <typename K>
cudaError_t Launcher<K>::fused_occupancy(int cutoff, int *ctas) {
  void (*fn)(SortParams) = nullptr;
  size_t smem = 0;
  cudaError_t e = fused_kernel_of<K>(cutoff, &fn, &smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, fn, 256, smem);
}

template <typename K>
cudaError_t Launcher<K>::tiles_fused(const SortParams &p, int grid, cudaStream_t st) {
  void (*fn)(SortParams) = nullptr;
  size_t smem = 0;
  cudaError_t e = fused_kernel_of<K>(p.cutoff, &fn, &smem);
  if (e != cudaSuccess) return e;
  return launch_after(fn, grid, 256, smem, p, st);
}

// part_kernel of CTA shape `shape`, with its dynamic shared memory allowed.
template <typename K, typename S>
cudaError_t part_kernel_of(void (**fn)(SortParams), size_t *smem) {
  *fn = dev::part_kernel<K, S::NT, S::IPT>;
  *smem = dev::pipe_smem_bytes<K, S::NT * S::IPT>();
  return allow_smem(*fn, *smem, true);
}

template <typename K>
cudaError_t Launcher<K>::part_occupancy(int shape, int *ctas) {
  return with_shape<K>(shape % kTileShapes, [&](auto s) {
    using S = decltype(s);
    void (*fn)(SortParams) = nullptr;
    size_t smem = 0;
    cudaError_t e = part_kernel_of<K, S>(&fn, &smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, fn, S::NT, smem);
  });
}

template <typename K>
cudaError_t Launcher<K>::partition(const SortParams &p, int shape, int grid, cudaStream_t st) {
  return with_shape<K>(shape % kTileShapes, [&](auto s) {
    using S = decltype(s);
    void (*fn)(SortParams) = nullptr;
    size_t smem = 0;
    cudaError_t e = part_kernel_of<K, S>(&fn, &smem);
    if (e != cudaSuccess) return e;
    fn<<<grid, S::NT, smem, st>>>(p);
    return cudaGetLastError();
  });
}

// ------------------------------------------------------------------ ring partition
// Compiled configurations of part_ring_kernel (1-based, as in ksort_tuning_t): data
// warps x keys per lane (the tile), slots, CTAs per SM, look-back window of 32 x PER
// descriptors, look-back warps (0: the reservation form; otherwise the ordered form), and
// the tiles a CTA may have loading or awaiting compaction (measured: 3, 4 and 6 equal at
// 5e7 keys, 2 slower) (about the number of CTAs, so that the tiles claimed between two of a
// CTA's own are usually read in one round trip). 8-byte keys take half the keys per
// lane, so every configuration stages the same bytes.
template <typename K, int C>
struct RingOf;
template <typename K> struct RingOf<K, 1> {  // reservation: 16 KiB tiles, 6 slots, 2 CTAs per SM
  using Cfg = dev::RingCfg<K, 8, 64 / (int)sizeof(K), 6, 2, 12, 0, 3>;
};
template <typename K> struct RingOf<K, 2> {  // reservation: 8 KiB tiles, 8 slots, 3 CTAs per SM
  using Cfg = dev::RingCfg<K, 8, 32 / (int)sizeof(K), 8, 3, 10, 0, 3>;
};
template <typename K> struct RingOf<K, 3> {  // reservation: 32 KiB tiles, 6 slots, 1 CTA per SM
  using Cfg = dev::RingCfg<K, 16, 64 / (int)sizeof(K), 6, 1, 6, 0, 3>;
};
template <typename K> struct RingOf<K, 4> {  // ordered: 16 KiB tiles, 6 slots, 2 CTAs per SM, 2 look-back warps
  using Cfg = dev::RingCfg<K, 8, 64 / (int)sizeof(K), 6, 2, 12, 2, 3>;
};
template <typename K> struct RingOf<K, 5> {  // reservation by 2 role warps: 16 KiB tiles, 6 slots, 2 CTAs per SM
  using Cfg = dev::RingCfg<K, 8, 64 / (int)sizeof(K), 6, 2, 12, 2, 3, true>;
};
template <typename K> struct RingOf<K, 6> {  // reservation by 2 role warps: 16 KiB tiles, 6 slots, 2 CTAs per SM, 4 tiles in flight
  using Cfg = dev::RingCfg<K, 8, 64 / (int)sizeof(K), 6, 2, 12, 2, 4, true>;
};

template <typename K, typename F>
decltype(auto) with_ring(int c, F &&f) {
  switch (c) {
    case 2: return f(typename RingOf<K, 2>::Cfg{});
    case 3: return f(typename RingOf<K, 3>::Cfg{});
    case 4: return f(typename RingOf<K, 4>::Cfg{});
    case 5: return f(typename RingOf<K, 5>::Cfg{});
    case 6: return f(typename RingOf<K, 6>::Cfg{});
    default: return f(typename RingOf<K, 1>::Cfg{});
  }
}

template <typename K, typename C>
cudaError_t ring_kernel_of(void (**fn)(SortParams)) {
  *fn = dev::part_ring_kernel<K, C::NDW, C::IPT, C::S, C::MINB, C::PER, C::NLB, C::DEPTH, C::RESV>;
  return allow_smem(*fn, C::SMEM, true);
}

template <typename K>
RingInfo Launcher<K>::ring_info(int cfg) {
  return with_ring<K>(cfg, [](auto c) {
    using C = decltype(c);
    return RingInfo{C::NT, C::TILE, C::MINB, C::NDW, C::IPT};
  });
}

template <typename K>
cudaError_t Launcher<K>::ring_occupancy(int cfg, int *ctas) {
  return with_ring<K>(cfg, [&](auto c) {
    using C = decltype(c);
    void (*fn)(SortParams) = nullptr;
    cudaError_t e = ring_kernel_of<K, C>(&fn);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, fn, C::NT, C::SMEM);
  });
}

template <typename K>
cudaError_t Launcher<K>::ring_partition(const SortParams &p, int cfg, int grid, cudaStream_t st) {
  return with_ring<K>(cfg, [&](auto c) {
    using C = decltype(c);
    void (*fn)(SortParams) = nullptr;
    cudaError_t e = ring_kernel_of<K, C>(&fn);
    if (e != cudaSuccess) return e;
    return launch_after(fn, grid, C::NT, C::SMEM, p, st);
  });
}

// ------------------------------------------------------------------ cluster form
// Largest slice the cluster kernel's dynamic shared memory holds (two buffers), and the
// largest cluster (16, else 8 CTAs of one GPC) that can run: *csize = 0 when none can.
template <typename K>
cudaError_t Launcher<K>::cluster_setup(int *csize, int *max_sl) {
  auto fn = dev::cluster_kernel<K>;
  *csize = 0;
  *max_sl = 0;
  cudaFuncAttributes fa{};
  cudaError_t e = cudaFuncGetAttributes(&fa, fn);
  if (e != cudaSuccess) return e;
  int dev = 0, optin = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) !=
      cudaSuccess)
    return e;
  const long long dyn = (long long)optin - (long long)fa.sharedSizeBytes;
  // chunks are rounded up to an odd length, so at most kClusterMaxChunk - 1 keys each
  int sl = (int)std::min<long long>(dyn / (2 * (long long)sizeof(K)),
                                    (long long)(dev::kClusterMaxChunk - 1) * dev::kClusterThreads);
  sl &= ~3;
  if (sl < 4) return cudaSuccess;
  const size_t smem = (size_t)2 * sl * sizeof(K);
  if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
      cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) !=
      cudaSuccess)
    return e;
  for (int c : {16, 8}) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)c);
    cfg.blockDim = dim3((unsigned)dev::kClusterThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)c;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int num = 0;
    if (cudaOccupancyMaxActiveClusters(&num, fn, &cfg) == cudaSuccess && num >= 1) {
      *csize = c;
      *max_sl = sl;
      return cudaSuccess;
    }
    (void)cudaGetLastError();  // this size cannot run: try the next
  }
  return cudaSuccess;
}

template <typename K>
cudaError_t Launcher<K>::cluster_sort(const SortParams &p, int csize, int sl, cudaStream_t st) {
  auto fn = dev::cluster_kernel<K>;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)csize);
  cfg.blockDim = dim3((unsigned)dev::kClusterThreads);
  cfg.dynamicSmemBytes = (size_t)2 * sl * sizeof(K);
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, fn, p, sl);
}

// ------------------------------------------------------------------ wave form
// One launch of fn(p, level), under programmatic dependent launch when `pdl` (the
// kernel then starts as the previous launch's CTAs leave and waits for its memory).
inline cudaError_t launch_level(void (*fn)(SortParams, int), int grid, int block,
                                const SortParams &p, int level, bool pdl, cudaStream_t s) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, fn, p, level);
}

template <typename K>
cudaError_t Launcher<K>::wave_occupancy(int shape, int *ctas) {
  return with_shape<K>(shape % kTileShapes, [&](auto s) {
    using S = decltype(s);
    int a = 0, b = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &a, dev::wave_scatter_kernel<K, S::NT, S::IPT>, S::NT, 0);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &b, dev::wave_count_kernel<K, S::NT, S::IPT>, S::NT, 0);
    *ctas = a < b ? a : b;
    return e;
  });
}

template <typename K>
cudaError_t Launcher<K>::wave_level(const SortParams &p, int shape, int level, int grid, bool pdl,
                                    cudaStream_t st) {
  return with_shape<K>(shape % kTileShapes, [&](auto s) {
    using S = decltype(s);
    cudaError_t e = launch_level(dev::wave_count_kernel<K, S::NT, S::IPT>, grid, S::NT, p,
                                 level, pdl, st);
    if (e != cudaSuccess) return e;
    return launch_level(dev::wave_scatter_kernel<K, S::NT, S::IPT>, grid, S::NT, p, level, pdl,
                        st);
  });
}

template <typename K>
cudaError_t Launcher<K>::wave_handoff(const SortParams &p, int shape, int level, bool pdl,
                                      cudaStream_t st) {
  return with_shape<K>(shape % kTileShapes, [&](auto s) {
    using S = decltype(s);
    return launch_level(dev::wave_handoff_kernel<K, S::NT * S::IPT>, 64, 256, p, level, pdl, st);
  });
}

// split_count_kernel then split_move_kernel (the latter under programmatic dependent
// launch) with the CTA shape of `shape`: as many CTAs as are co-resident, no more than
// the warp tiles need, and no more warps than p.wave_cnt holds counts.
template <typename K>
cudaError_t Launcher<K>::partition_split(const SortParams &p, int shape, int sms,
                                         cudaStream_t st) {
  return with_shape<K>(shape % kTileShapes, [&](auto s) {
    using S = decltype(s);
    constexpr int NW = S::NT / 32, WT = 32 * S::IPT;
    auto count = dev::split_count_kernel<K, S::NT, S::IPT>;
    auto move = dev::split_move_kernel<K, S::NT, S::IPT>;
    int a = 0, b = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, count, S::NT, 0);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, move, S::NT, 0);
    if (e != cudaSuccess) return e;
    const long long per_sm = std::max(1, std::min(a, b));
    const long long wtiles = (p.total + WT) / WT;  // at least the warp tiles there are
    long long grid = std::min<long long>((long long)sms * per_sm, (wtiles + NW - 1) / NW);
    grid = std::max<long long>(1, std::min<long long>(grid, 2 * kWaveMaxGrid / NW));
    count<<<(int)grid, S::NT, 0, st>>>(p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)S::NT);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, move, p);
  });
}

// Scratch of the exact-layout partition: [tile counts][ge before][less after][T][L]
// [F positions][B positions], each part 16-byte aligned.
struct ExactWork {
  unsigned *tile_less;
  unsigned long long *ge_before, *less_after, *T, *L;
  int *Fpos, *Bpos;
};
inline size_t exact_layout(long long n, char *base, ExactWork *w) {
  const long long m = n - 1;
  const long long tiles = (m + dev::kExactTile - 1) / dev::kExactTile;
  auto up = [](size_t x) { return (x + 15) / 16 * 16; };
  size_t off = 0;
  const size_t o_tl = off; off = up(off + tiles * sizeof(unsigned));
  const size_t o_gb = off; off = up(off + tiles * sizeof(unsigned long long));
  const size_t o_la = off; off = up(off + tiles * sizeof(unsigned long long));
  const size_t o_T = off;  off = up(off + sizeof(unsigned long long));
  const size_t o_L = off;  off = up(off + sizeof(unsigned long long));
  const size_t o_F = off;  off = up(off + m * sizeof(int));
  const size_t o_B = off;  off = up(off + m * sizeof(int));
  if (w) {
    w->tile_less = reinterpret_cast<unsigned *>(base + o_tl);
    w->ge_before = reinterpret_cast<unsigned long long *>(base + o_gb);
    w->less_after = reinterpret_cast<unsigned long long *>(base + o_la);
    w->T = reinterpret_cast<unsigned long long *>(base + o_T);
    w->L = reinterpret_cast<unsigned long long *>(base + o_L);
    w->Fpos = reinterpret_cast<int *>(base + o_F);
    w->Bpos = reinterpret_cast<int *>(base + o_B);
  }
  return off;
}

template <typename K>
size_t Launcher<K>::exact_work_bytes(long long n) {
  return exact_layout(n, nullptr, nullptr);
}

template <typename K>
cudaError_t Launcher<K>::exact(const void *in, void *out, long long n, long long *key_index,
                               void *work, cudaStream_t s) {
  const long long m = n - 1;
  const long long tiles = (m + dev::kExactTile - 1) / dev::kExactTile;
  ExactWork w{};
  exact_layout(n, static_cast<char *>(work), &w);
  const K *a = static_cast<const K *>(in);
  cudaError_t e = cudaMemsetAsync(w.T, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  dev::exact_count_kernel<K><<<(unsigned)tiles, dev::kExactThreads, 0, s>>>(a, m, w.tile_less);
  dev::exact_scan_kernel<1024><<<1, 1024, 0, s>>>(w.tile_less, tiles, m, w.ge_before, w.less_after, w.L);
  dev::exact_rank_kernel<K><<<(unsigned)tiles, dev::kExactThreads, 0, s>>>(
      a, m, w.ge_before, w.less_after, w.Fpos, w.Bpos, w.T);
  dev::exact_place_kernel<K><<<(unsigned)tiles, dev::kExactThreads, 0, s>>>(
      a, m, w.ge_before, w.less_after, w.Fpos, w.Bpos, w.T, w.L, static_cast<K *>(out), key_index);
  return cudaGetLastError();
}

template <typename K>
cudaError_t Launcher<K>::smalls(const SortParams &p, int grid, cudaStream_t s) {
  void (*sk)(SortParams) = nullptr;
  size_t smem = 0;
  cudaError_t e = small_kernel_of<K>(p.small_threads, p.cutoff, &sk, &smem);
  if (e != cudaSuccess) return e;
  return launch_after(sk, grid, small_threads_of(p.small_threads), smem, p, s);
}

}  // namespace ksort
