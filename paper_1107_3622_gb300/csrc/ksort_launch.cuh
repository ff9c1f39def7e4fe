// Host-side launchers for one key type. Included once per key type by
// ksort_f32.cu / ksort_f64.cu / ksort_u32.cu, which each instantiate Launcher<K>.
#pragma once

#include "ksort_device.cuh"

namespace ksort {

// Keys per thread of a tile pass: a tile is kTileThreads * IPT keys (8 KiB).
template <typename K> struct Shape;
template <> struct Shape<float> { static constexpr int IPT = 16; };
template <> struct Shape<unsigned> { static constexpr int IPT = 16; };
template <> struct Shape<double> { static constexpr int IPT = 8; };

template <typename K>
constexpr int tile_keys() { return dev::kTileThreads * Shape<K>::IPT; }

template <typename K>
KernelInfo Launcher<K>::info() {
  return KernelInfo{dev::kTileThreads, tile_keys<K>(), dev::kMaxSmallCutoff};
}

template <typename K>
size_t Launcher<K>::small_smem_bytes(int cutoff) {
  return dev::small_smem_bytes<K>(cutoff);
}

template <typename K>
long long Launcher<K>::tile_count(const void *buf, long long begin, long long end) {
  return dev::tile_count<K, tile_keys<K>()>(static_cast<const K *>(buf), begin, end);
}

template <typename K>
cudaError_t Launcher<K>::occupancy(int cutoff, int *tile_ctas, int *small_ctas) {
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      tile_ctas, dev::tile_kernel<K, Shape<K>::IPT>, dev::kTileThreads, 0);
  if (e != cudaSuccess) return e;
  auto sk = dev::small_kernel<K>;
  const size_t smem = small_smem_bytes(cutoff);
  e = cudaFuncSetAttribute(sk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(small_ctas, sk, dev::kSmallThreads, smem);
}

template <typename K>
cudaError_t Launcher<K>::seed(const SortParams &p, cudaStream_t s) {
  dev::seed_kernel<K, tile_keys<K>()><<<1, 1024, 0, s>>>(p);
  return cudaGetLastError();
}

template <typename K>
cudaError_t Launcher<K>::tiles(const SortParams &p, int grid, cudaStream_t s) {
  dev::tile_kernel<K, Shape<K>::IPT><<<grid, dev::kTileThreads, 0, s>>>(p);
  return cudaGetLastError();
}

template <typename K>
cudaError_t Launcher<K>::smalls(const SortParams &p, int grid, cudaStream_t s) {
  auto sk = dev::small_kernel<K>;
  const size_t smem = small_smem_bytes(p.cutoff);
  cudaError_t e = cudaFuncSetAttribute(sk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  sk<<<grid, dev::kSmallThreads, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace ksort
