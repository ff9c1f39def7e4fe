// Host-side launchers for one key type. Included once per key type by
// ksort_f32.cu / ksort_f64.cu / ksort_u32.cu, which each instantiate Launcher<K>.
#pragma once

#include "ksort_device.cuh"

namespace ksort {

// Compile-time shape of the kernels for a key type: threads per CTA, keys per thread
// in a tile pass, the CTAs per SM the register budget is sized for, and the largest
// shared-memory item.
template <typename K> struct Shape;
template <> struct Shape<float> {
  static constexpr int BLOCK = 256, IPT = 16, MINB = 4, MAX_CUTOFF = dev::kMaxSmallCutoff;
};
template <> struct Shape<unsigned> {
  static constexpr int BLOCK = 256, IPT = 16, MINB = 4, MAX_CUTOFF = dev::kMaxSmallCutoff;
};
template <> struct Shape<double> {
  static constexpr int BLOCK = 256, IPT = 8, MINB = 4, MAX_CUTOFF = 8192;
};

template <typename K>
KernelInfo Launcher<K>::info() {
  using S = Shape<K>;
  return KernelInfo{S::BLOCK, S::BLOCK * S::IPT, S::MAX_CUTOFF};
}

template <typename K>
size_t Launcher<K>::sort_smem_bytes(int cutoff) {
  using S = Shape<K>;
  const size_t stage = (size_t)2 * S::BLOCK * S::IPT * sizeof(K);
  const size_t fin = dev::smem_finisher_bytes<K>(cutoff, S::BLOCK / 32);
  return stage > fin ? stage : fin;
}

template <typename K>
long long Launcher<K>::tile_count(const void *buf, long long begin, long long end) {
  using S = Shape<K>;
  return dev::tile_count<K, S::BLOCK * S::IPT>(static_cast<const K *>(buf), begin, end);
}

template <typename K>
cudaError_t Launcher<K>::max_ctas_per_sm(int cutoff, int *out) {
  using S = Shape<K>;
  auto kern = dev::sort_kernel<K, S::BLOCK, S::IPT, S::MINB>;
  const size_t smem = sort_smem_bytes(cutoff);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, kern, S::BLOCK, smem);
}

template <typename K>
cudaError_t Launcher<K>::partition_out(const PartParams &p, int num_tiles, cudaStream_t s) {
  using S = Shape<K>;
  auto kern = dev::partition_kernel<K, S::BLOCK, S::IPT>;
  const size_t smem = (size_t)2 * S::BLOCK * S::IPT * sizeof(K);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<num_tiles, S::BLOCK, smem, s>>>(p);
  return cudaGetLastError();
}

template <typename K>
cudaError_t Launcher<K>::seed(const SortParams &p, cudaStream_t s) {
  using S = Shape<K>;
  dev::seed_kernel<K, S::BLOCK * S::IPT><<<1, 1024, 0, s>>>(p);
  return cudaGetLastError();
}

template <typename K>
cudaError_t Launcher<K>::sort(const SortParams &p, int grid, cudaStream_t s) {
  using S = Shape<K>;
  auto kern = dev::sort_kernel<K, S::BLOCK, S::IPT, S::MINB>;
  const size_t smem = sort_smem_bytes(p.cutoff);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, S::BLOCK, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace ksort
