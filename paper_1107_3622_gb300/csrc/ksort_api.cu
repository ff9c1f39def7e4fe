// C ABI of libksort (include/ksort.h): argument checks, per-(device, stream)
// workspaces, tuning, and dispatch to the per-key-type launchers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstddef>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>

#include "../../include/ksort.h"
#include "ksort_device.cuh"
#include "ksort_internal.h"

namespace ksort {
namespace {

thread_local char g_cuda_error[256] = "";

ksort_status_t cuda_fail(cudaError_t e) {
  std::snprintf(g_cuda_error, sizeof(g_cuda_error), "%s: %s", cudaGetErrorName(e),
                cudaGetErrorString(e));
  return KSORT_ERR_CUDA;
}

#define KS_CUDA(call)                          \
  do {                                         \
    cudaError_t e_ = (call);                   \
    if (e_ != cudaSuccess) return cuda_fail(e_); \
  } while (0)

size_t key_bytes(ksort_dtype_t dt) { return dt == KSORT_F64 ? 8 : 4; }
bool dtype_ok(int dt) { return dt == KSORT_F32 || dt == KSORT_F64 || dt == KSORT_U32; }

// ------------------------------------------------------------------ per-type dispatch
struct Ops {
  KernelInfo (*info)(int);
  size_t (*small_smem_bytes)(int);
  cudaError_t (*occupancy)(int, int, int, int *, int *);
  cudaError_t (*seed)(const SortParams &, int, cudaStream_t);
  cudaError_t (*tiles)(const SortParams &, int, int, cudaStream_t);
  cudaError_t (*smalls)(const SortParams &, int, cudaStream_t);
  long long (*tile_count)(int, const void *, long long, long long);
  cudaError_t (*part_occupancy)(int, int *);
  cudaError_t (*partition)(const SortParams &, int, int, cudaStream_t);
  size_t (*exact_work_bytes)(long long);
  cudaError_t (*exact)(const void *, void *, long long, long long *, void *, cudaStream_t);
  cudaError_t (*wave_occupancy)(int, int *);
  cudaError_t (*wave_level)(const SortParams &, int, int, int, bool, cudaStream_t);
  cudaError_t (*wave_handoff)(const SortParams &, int, int, bool, cudaStream_t);
  cudaError_t (*partition_split)(const SortParams &, int, int, cudaStream_t);
  RingInfo (*ring_info)(int);
  cudaError_t (*ring_occupancy)(int, int *);
  cudaError_t (*ring_partition)(const SortParams &, int, int, cudaStream_t);
  cudaError_t (*fused_occupancy)(int, int *);
  cudaError_t (*tiles_fused)(const SortParams &, int, cudaStream_t);
  cudaError_t (*cluster_setup)(int *, int *);
  cudaError_t (*cluster_sort)(const SortParams &, int, int, cudaStream_t);
};

template <typename K>
Ops ops_for() {
  return Ops{&Launcher<K>::info,       &Launcher<K>::small_smem_bytes, &Launcher<K>::occupancy,
             &Launcher<K>::seed,       &Launcher<K>::tiles,            &Launcher<K>::smalls,
             &Launcher<K>::tile_count, &Launcher<K>::part_occupancy,   &Launcher<K>::partition,
             &Launcher<K>::exact_work_bytes, &Launcher<K>::exact,
             &Launcher<K>::wave_occupancy, &Launcher<K>::wave_level, &Launcher<K>::wave_handoff,
             &Launcher<K>::partition_split,
             &Launcher<K>::ring_info,  &Launcher<K>::ring_occupancy, &Launcher<K>::ring_partition,
             &Launcher<K>::fused_occupancy, &Launcher<K>::tiles_fused,
             &Launcher<K>::cluster_setup, &Launcher<K>::cluster_sort};
}

const Ops &ops(ksort_dtype_t dt) {
  static const Ops f32 = ops_for<float>(), f64 = ops_for<double>(), u32 = ops_for<unsigned>();
  return dt == KSORT_F64 ? f64 : dt == KSORT_U32 ? u32 : f32;
}

// ------------------------------------------------------------------ tuning
struct Tuning {
  int cutoff;
  int ctas_per_sm;  // 0: as many as fit
  int spin_limit_ms;
  int variant;      // tile shape of the tile passes, 0 .. kTileVariants - 1
  int wave_levels;  // wave form: level-synchronous levels; 0: automatic
  int medium_tiles; // register-form queue: largest item one CTA takes whole; 0: off
  int part_form;    // single partitions: ring configuration 1 .. kRingConfigs; 0: tile shape's form
  int reserve;      // sorts, register and wave forms: tile ranges by reservation (else look-back)
  int fuse_park;    // tile variant kFusedVariant: finisher inside the tile kernel with this
                    // park threshold; 0: separate finisher launch
  int small_threads;  // finisher CTA: 256, 512 or 1024 threads
  int cluster;        // single arrays that fit: upper levels in a thread-block cluster
};

std::mutex g_mu;
unsigned long long *g_trace = nullptr;  // diagnostics: per-ticket timestamps
long long g_trace_cap = 0;
Tuning g_tuning[3] = {{4096, 0, 2000, 0, 0, 0, 5, 1, 0, 256, 0},
                      {2048, 0, 2000, 0, 0, 0, 5, 1, 0, 256, 0},
                      {4096, 0, 2000, 0, 0, 0, 5, 1, 0, 256, 0}};

// ------------------------------------------------------------------ workspaces
struct Workspace {
  void *base = nullptr;
  size_t bytes = 0;
  Control *ctl = nullptr;
  unsigned long long *lb = nullptr;
  unsigned long long lb_cap = 0;
  Item *items = nullptr;
  ItemCtl *ictl = nullptr;
  unsigned long long *tmap = nullptr, *small_q = nullptr;
  unsigned long long item_cap = 0;
  WaveItem *wave_items = nullptr;          // two level lists of item_cap entries
  unsigned long long *wave_cnt = nullptr;  // 2 x kWaveMaxGrid
  unsigned long long *wave_fin = nullptr;  // item_cap (index, key) pairs
  void *scratch = nullptr;
  size_t scratch_bytes = 0;
  unsigned pending_error = 0;  // device error carried over from a replaced allocation
  unsigned long long launches = 0;  // kernels the last sort or partition on it enqueued
};

std::map<std::pair<int, cudaStream_t>, Workspace> g_ws;

// ------------------------------------------------------------------ phase timing
// While enabled, a sort or partition call outside graph capture records CUDA events on
// its stream at the boundaries of its phases (4 for a sort: before the seed, after it,
// after the partition passes, after the finisher; 2 for a partition). The events of the
// last kPhaseRing timed calls per stream are kept, so calls can be enqueued back to back
// and read afterwards.
bool g_time_phases = false;
constexpr int kPhaseMarks = 4, kPhasesOut = kPhaseMarks - 1, kPhaseRing = 64;
struct PhaseEvents {
  cudaEvent_t ev[kPhaseRing][kPhaseMarks] = {};
  int marks[kPhaseRing] = {};  // events recorded by the call in each slot
  long long calls = 0;         // timed calls so far; call c used slot c % kPhaseRing
};
std::map<std::pair<int, cudaStream_t>, PhaseEvents> g_phase;

struct PhaseMarks {
  PhaseEvents *pe = nullptr;  // null: this call is not timed
  int slot = 0;
  cudaStream_t s = nullptr;
  cudaError_t mark() {
    if (!pe || pe->marks[slot] >= kPhaseMarks) return cudaSuccess;
    return cudaEventRecord(pe->ev[slot][pe->marks[slot]++], s);
  }
};

ksort_status_t phase_begin(int dev, cudaStream_t s, PhaseMarks *m) {
  m->pe = nullptr;
  m->s = s;
  if (!g_time_phases) return KSORT_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  KS_CUDA(cudaStreamIsCapturing(s, &cs));
  if (cs != cudaStreamCaptureStatusNone) return KSORT_OK;
  PhaseEvents &pe = g_phase[{dev, s}];
  const int slot = (int)(pe.calls % kPhaseRing);
  for (cudaEvent_t &e : pe.ev[slot])
    if (!e) KS_CUDA(cudaEventCreate(&e));
  pe.marks[slot] = 0;
  ++pe.calls;
  m->pe = &pe;
  m->slot = slot;
  return KSORT_OK;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Bytes past the scratch keys that bulk copies of whole 16-byte chunks may read.
constexpr size_t kScratchPad = 64;

struct Need {
  unsigned long long item_cap, lb_cap;
  size_t scratch_bytes;
};

// Work-queue and look-back capacities. Up to 2^21 keys the queue can hold one entry
// per key, which covers every input (a sort makes at most n - 1 partition calls);
// beyond that it holds n/32 entries, ~100x what random inputs use. Inputs that need
// more (near-O(n^2) orders) stop with KSORT_ERR_WORKSPACE_EXHAUSTED.
Need need_for(ksort_dtype_t dt, long long total, long long arrays, int variant) {
  const KernelInfo ki = ops(dt).info(variant);
  const unsigned long long t = (unsigned long long)std::max<long long>(total, 1);
  const unsigned long long a = (unsigned long long)std::max<long long>(arrays, 1);
  unsigned long long items = t <= (1ull << 21) ? t : std::max(1ull << 21, t / 32);
  items += a + 64;
  const unsigned long long tiles_per_level = (t + ki.tile_keys - 1) / ki.tile_keys + a + 1;
  const unsigned long long lb = std::max(1ull << 21, 64ull * tiles_per_level);
  return Need{items, lb, (size_t)t * key_bytes(dt)};
}

ksort_status_t get_workspace(int dev, cudaStream_t s, const Need &need, Workspace **out) {
  Workspace &ws = g_ws[{dev, s}];
  if (ws.base && ws.item_cap >= need.item_cap && ws.lb_cap >= need.lb_cap &&
      ws.scratch_bytes >= need.scratch_bytes) {
    *out = &ws;
    return KSORT_OK;
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  KS_CUDA(cudaStreamIsCapturing(s, &cap));
  if (cap != cudaStreamCaptureStatusNone) return KSORT_ERR_OUT_OF_MEMORY;

  const unsigned long long item_cap = std::max(need.item_cap, ws.item_cap);
  const unsigned long long lb_cap = std::max(need.lb_cap, ws.lb_cap);
  const size_t scratch_bytes = std::max(need.scratch_bytes, ws.scratch_bytes);

  if (ws.base) {
    KS_CUDA(cudaStreamSynchronize(s));
    unsigned err = 0;
    KS_CUDA(cudaMemcpy(&err, &ws.ctl->error, sizeof(err), cudaMemcpyDeviceToHost));
    if (err && !ws.pending_error) ws.pending_error = err;
    KS_CUDA(cudaFree(ws.base));
    ws.base = nullptr;
  }
  // [Control][look-back][items][item counters][ticket map][small list][wave lists]
  // [wave counts][late keys][scratch keys]
  size_t off = 0;
  const size_t o_ctl = off;
  off = align_up(off + sizeof(Control), 256);
  const size_t o_lb = off;
  off = align_up(off + lb_cap * sizeof(unsigned long long), 256);
  const size_t o_items = off;
  off = align_up(off + item_cap * sizeof(Item), 256);
  const size_t o_ictl = off;
  off = align_up(off + item_cap * sizeof(ItemCtl), 256);
  const size_t o_tmap = off;
  off = align_up(off + lb_cap * sizeof(unsigned long long), 256);
  const size_t o_sq = off;
  off = align_up(off + item_cap * sizeof(unsigned long long), 256);
  const size_t o_wi = off;
  off = align_up(off + 2 * item_cap * sizeof(WaveItem), 256);
  const size_t o_wc = off;
  off = align_up(off + 2 * kWaveMaxGrid * sizeof(unsigned long long), 256);
  const size_t o_wf = off;
  off = align_up(off + 2 * item_cap * sizeof(unsigned long long), 256);
  const size_t meta = off;
  const size_t o_scr = off;
  off = align_up(off + scratch_bytes + kScratchPad, 256);

  void *base = nullptr;
  cudaError_t e = cudaMalloc(&base, off);
  if (e != cudaSuccess) {
    cudaGetLastError();
    ws = Workspace{};
    return KSORT_ERR_OUT_OF_MEMORY;
  }
  KS_CUDA(cudaMemsetAsync(base, 0, meta, s));
  char *b = static_cast<char *>(base);
  const unsigned pending = ws.pending_error;
  const unsigned long long launches = ws.launches;
  ws = Workspace{};
  ws.launches = launches;
  ws.base = base;
  ws.bytes = off;
  ws.ctl = reinterpret_cast<Control *>(b + o_ctl);
  ws.lb = reinterpret_cast<unsigned long long *>(b + o_lb);
  ws.lb_cap = lb_cap;
  ws.items = reinterpret_cast<Item *>(b + o_items);
  ws.ictl = reinterpret_cast<ItemCtl *>(b + o_ictl);
  ws.tmap = reinterpret_cast<unsigned long long *>(b + o_tmap);
  ws.small_q = reinterpret_cast<unsigned long long *>(b + o_sq);
  ws.item_cap = item_cap;
  ws.wave_items = reinterpret_cast<WaveItem *>(b + o_wi);
  ws.wave_cnt = reinterpret_cast<unsigned long long *>(b + o_wc);
  ws.wave_fin = reinterpret_cast<unsigned long long *>(b + o_wf);
  ws.scratch = b + o_scr;
  ws.scratch_bytes = scratch_bytes;
  ws.pending_error = pending;
  *out = &ws;
  return KSORT_OK;
}

ksort_status_t check_device_ptr(const void *p, size_t align, int dev) {
  if (!p) return KSORT_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(p) % align) return KSORT_ERR_INVALID_ARG;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return KSORT_ERR_INVALID_ARG;
  }
  if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return KSORT_ERR_INVALID_ARG;
  if (a.type == cudaMemoryTypeDevice && a.device != dev) return KSORT_ERR_INVALID_ARG;
  return KSORT_OK;
}

struct DeviceProps {
  int sms = 0;
};
std::map<int, DeviceProps> g_props;

ksort_status_t device_sms(int dev, int *sms) {
  DeviceProps &p = g_props[dev];
  if (!p.sms) KS_CUDA(cudaDeviceGetAttribute(&p.sms, cudaDevAttrMultiProcessorCount, dev));
  *sms = p.sms;
  return KSORT_OK;
}

struct Grids {
  int tiles;   // tile_kernel CTAs filling the GPU
  int smalls;  // small_kernel CTAs filling the GPU
};
// (dtype, variant, cutoff) -> CTAs per SM of (tile_kernel, small_kernel)
std::map<std::pair<int, int>, std::pair<int, int>> g_occ;

ksort_status_t full_grids(ksort_dtype_t dt, int dev, const Tuning &tu, Grids *g) {
  int sms = 0;
  ksort_status_t st = device_sms(dev, &sms);
  if (st != KSORT_OK) return st;
  auto key = std::make_pair(((int)dt * kTileVariants + tu.variant) * 4 + tu.small_threads / 256,
                            tu.cutoff);
  auto it = g_occ.find(key);
  std::pair<int, int> occ;
  if (it == g_occ.end()) {
    KS_CUDA(ops(dt).occupancy(tu.variant, tu.cutoff, tu.small_threads, &occ.first, &occ.second));
    g_occ[key] = occ;
  } else {
    occ = it->second;
  }
  if (occ.first < 1 || occ.second < 1) return KSORT_ERR_INTERNAL;
  int small_occ = occ.second;
  if (tu.ctas_per_sm > 0) small_occ = std::min(small_occ, tu.ctas_per_sm);
  g->tiles = sms * occ.first;
  g->smalls = sms * small_occ;
  return KSORT_OK;
}

// (device, dtype) -> (cluster size, largest slice) of the cluster kernel; size 0: none
std::map<std::pair<int, int>, std::pair<int, int>> g_cluster;

ksort_status_t cluster_setup(ksort_dtype_t dt, int dev, int *csize, int *max_sl) {
  auto key = std::make_pair(dev, (int)dt);
  auto it = g_cluster.find(key);
  if (it == g_cluster.end()) {
    std::pair<int, int> v{0, 0};
    KS_CUDA(ops(dt).cluster_setup(&v.first, &v.second));
    it = g_cluster.emplace(key, v).first;
  }
  *csize = it->second.first;
  *max_sl = it->second.second;
  return KSORT_OK;
}

std::map<std::pair<int, int>, int> g_fuse_occ;  // (dtype, cutoff) -> fused tile CTAs per SM

ksort_status_t fused_occupancy(ksort_dtype_t dt, int cutoff, int *occ) {
  auto key = std::make_pair((int)dt, cutoff);
  auto it = g_fuse_occ.find(key);
  if (it != g_fuse_occ.end()) {
    *occ = it->second;
    return KSORT_OK;
  }
  int o = 0;
  KS_CUDA(ops(dt).fused_occupancy(cutoff, &o));
  if (o < 1) return KSORT_ERR_INTERNAL;
  g_fuse_occ[key] = o;
  *occ = o;
  return KSORT_OK;
}

std::map<std::pair<int, int>, int> g_wave_occ;  // (dtype, shape) -> level-pass CTAs per SM

ksort_status_t wave_occupancy(ksort_dtype_t dt, int shape, int *occ) {
  auto key = std::make_pair((int)dt, shape);
  auto it = g_wave_occ.find(key);
  if (it != g_wave_occ.end()) {
    *occ = it->second;
    return KSORT_OK;
  }
  int o = 0;
  KS_CUDA(ops(dt).wave_occupancy(shape, &o));
  if (o < 1) return KSORT_ERR_INTERNAL;
  g_wave_occ[key] = o;
  *occ = o;
  return KSORT_OK;
}

// Wave levels when the tuning leaves it automatic: about the depth at which a random
// array's sub-arrays fall to the cutoff (log2 of the mean array over the cutoff, plus
// two levels for the spread of random keys); what remains goes to the work queue.
int auto_wave_levels(long long total, long long arrays, int cutoff) {
  const double mean = (double)total / (double)std::max<long long>(arrays, 1);
  int w = 0;
  for (double x = mean; x > cutoff && w < 62; x /= 2) ++w;
  return std::max(1, w + 2);
}

std::map<std::pair<int, int>, int> g_part_occ;  // (dtype, shape) -> part_kernel CTAs per SM

ksort_status_t part_occupancy(ksort_dtype_t dt, int shape, int *occ) {
  auto key = std::make_pair((int)dt, shape);
  auto it = g_part_occ.find(key);
  if (it != g_part_occ.end()) {
    *occ = it->second;
    return KSORT_OK;
  }
  int o = 0;
  KS_CUDA(ops(dt).part_occupancy(shape, &o));
  if (o < 1) return KSORT_ERR_INTERNAL;
  g_part_occ[key] = o;
  *occ = o;
  return KSORT_OK;
}

std::map<std::pair<int, int>, int> g_ring_occ;  // (dtype, configuration) -> CTAs per SM

ksort_status_t ring_occupancy(ksort_dtype_t dt, int cfg, int *occ) {
  auto key = std::make_pair((int)dt, cfg);
  auto it = g_ring_occ.find(key);
  if (it != g_ring_occ.end()) {
    *occ = it->second;
    return KSORT_OK;
  }
  int o = 0;
  KS_CUDA(ops(dt).ring_occupancy(cfg, &o));
  if (o < 1) return KSORT_ERR_INTERNAL;
  g_ring_occ[key] = o;
  *occ = o;
  return KSORT_OK;
}

SortParams sort_params(const Workspace &ws, void *keys, const Tuning &tu) {
  SortParams p{};
  p.keys = keys;
  p.scratch = ws.scratch;
  p.ctl = ws.ctl;
  p.items = ws.items;
  p.ictl = ws.ictl;
  p.tmap = ws.tmap;
  p.small_q = ws.small_q;
  p.item_cap = ws.item_cap;
  p.lb = ws.lb;
  p.lb_cap = ws.lb_cap;
  p.cutoff = tu.cutoff;
  p.small_threads = tu.small_threads;
  p.spin_limit_ns = (unsigned long long)tu.spin_limit_ms * 1000000ull;
  p.trace = g_trace;
  p.trace_cap = g_trace_cap;
  p.wave_items = ws.wave_items;
  p.wave_cap = ws.item_cap;
  p.wave_cnt = ws.wave_cnt;
  p.wave_fin = ws.wave_fin;
  p.wave = 0;
  return p;
}

ksort_status_t current_device(int *dev) {
  KS_CUDA(cudaGetDevice(dev));
  return KSORT_OK;
}

ksort_status_t partition_impl(ksort_dtype_t dt, const void *in, void *out, int64_t n,
                              int64_t *key_index, cudaStream_t s, bool in_place) {
  if (!dtype_ok(dt)) return KSORT_ERR_UNSUPPORTED_DTYPE;
  if (n < 1 || n > kMaxItemKeys) return KSORT_ERR_INVALID_ARG;
  int dev = 0;
  ksort_status_t st = current_device(&dev);
  if (st != KSORT_OK) return st;
  const size_t kb = key_bytes(dt);
  if ((st = check_device_ptr(in, kb, dev)) != KSORT_OK) return st;
  if (!in_place && (st = check_device_ptr(out, kb, dev)) != KSORT_OK) return st;
  if ((st = check_device_ptr(key_index, 8, dev)) != KSORT_OK) return st;
  if (!in_place) {
    const char *a = static_cast<const char *>(in), *b = static_cast<const char *>(out);
    if (a < b + n * kb && b < a + n * kb) return KSORT_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  const Tuning tu = g_tuning[dt];
  Workspace *ws = nullptr;
  Need need = need_for(dt, n, 1, tu.variant);
  need.item_cap = 64;
  if (!in_place) need.scratch_bytes = kb;
  st = get_workspace(dev, s, need, &ws);
  if (st != KSORT_OK) return st;
  void *dst = in_place ? ws->scratch : out;
  if (n == 1) {
    KS_CUDA(cudaMemsetAsync(key_index, 0, sizeof(int64_t), s));
    if (!in_place) KS_CUDA(cudaMemcpyAsync(dst, in, kb, cudaMemcpyDeviceToDevice, s));
    return KSORT_OK;
  }
  // One launch of part_ring_kernel (the tuned configuration); or, with the ring turned
  // off, one launch of part_kernel (the CTA shape of the tuned form) or for the wave form
  // the count and move launches of the split partition. Buffer 0 is read, buffer 1
  // receives the result.
  const int shape = tu.variant % kTileShapes;
  int sms = 0;
  if ((st = device_sms(dev, &sms)) != KSORT_OK) return st;
  long long tiles = 0;
  int occ = 0;
  if (tu.part_form > 0) {
    const long long tk = ops(dt).ring_info(tu.part_form).tile_keys;
    // tiles start at the 16-byte boundary at or below element 1 (tile_base)
    const long long mis = (long long)((reinterpret_cast<uintptr_t>(in) + kb) & 15u) / (long long)kb;
    const long long base = 1 - mis;
    tiles = (n - base + tk - 1) / tk;
    if ((st = ring_occupancy(dt, tu.part_form, &occ)) != KSORT_OK) return st;
  } else {
    tiles = ops(dt).tile_count(shape, in, 0, n);  // form-0 variants: plain tiles
    if ((st = part_occupancy(dt, shape, &occ)) != KSORT_OK) return st;
  }
  if ((unsigned long long)tiles > ws->lb_cap) return KSORT_ERR_INVALID_ARG;
  const int grid = (int)std::max<long long>(1, std::min<long long>((long long)sms * occ, tiles));
  SortParams p = sort_params(*ws, const_cast<void *>(in), tu);
  p.scratch = dst;
  p.num_roots = 1;
  p.total = n;
  p.root_flags = kItemPartitionOnly;
  p.key_index = reinterpret_cast<long long *>(key_index);
  p.readable[0] = n;
  p.readable[1] = 0;  // buffer 1 is only written
  PhaseMarks pm;
  if ((st = phase_begin(dev, s, &pm)) != KSORT_OK) return st;
  KS_CUDA(pm.mark());
  if (tu.part_form > 0) {
    KS_CUDA(ops(dt).ring_partition(p, tu.part_form, grid, s));
    ws->launches = 1;
  } else if (ops(dt).info(tu.variant).form == kWaveForm) {
    KS_CUDA(ops(dt).partition_split(p, shape, sms, s));
    ws->launches = 2;
  } else {
    KS_CUDA(ops(dt).partition(p, shape, grid, s));
    ws->launches = 1;
  }
  KS_CUDA(pm.mark());
  if (in_place) KS_CUDA(cudaMemcpyAsync(const_cast<void *>(in), dst, n * kb, cudaMemcpyDeviceToDevice, s));
  return KSORT_OK;
}

ksort_status_t partition_exact_impl(ksort_dtype_t dt, const void *in, void *out, int64_t n,
                                    int64_t *key_index, cudaStream_t s) {
  if (!dtype_ok(dt)) return KSORT_ERR_UNSUPPORTED_DTYPE;
  if (n < 1 || n > kMaxItemKeys) return KSORT_ERR_INVALID_ARG;
  int dev = 0;
  ksort_status_t st = current_device(&dev);
  if (st != KSORT_OK) return st;
  const size_t kb = key_bytes(dt);
  if ((st = check_device_ptr(in, kb, dev)) != KSORT_OK) return st;
  if ((st = check_device_ptr(out, kb, dev)) != KSORT_OK) return st;
  if ((st = check_device_ptr(key_index, 8, dev)) != KSORT_OK) return st;
  {
    const char *a = static_cast<const char *>(in), *b = static_cast<const char *>(out);
    if (a < b + n * kb && b < a + n * kb) return KSORT_ERR_INVALID_ARG;
  }
  if (n == 1) {
    KS_CUDA(cudaMemsetAsync(key_index, 0, sizeof(int64_t), s));
    KS_CUDA(cudaMemcpyAsync(out, in, kb, cudaMemcpyDeviceToDevice, s));
    return KSORT_OK;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  const Tuning tu = g_tuning[dt];
  Need need = need_for(dt, 1, 1, tu.variant);
  need.item_cap = 64;
  need.scratch_bytes = ops(dt).exact_work_bytes(n);
  Workspace *ws = nullptr;
  if ((st = get_workspace(dev, s, need, &ws)) != KSORT_OK) return st;
  KS_CUDA(ops(dt).exact(in, out, n, reinterpret_cast<long long *>(key_index), ws->scratch, s));
  return KSORT_OK;
}

ksort_status_t sort_impl(ksort_dtype_t dt, void *keys, const int64_t *offsets, int64_t num_arrays,
                         int64_t total, cudaStream_t s) {
  if (!dtype_ok(dt)) return KSORT_ERR_UNSUPPORTED_DTYPE;
  if (total < 0 || num_arrays < 0) return KSORT_ERR_INVALID_ARG;
  if (!offsets && total > kMaxItemKeys) return KSORT_ERR_INVALID_ARG;
  if (total <= 1 || num_arrays == 0) return KSORT_OK;
  int dev = 0;
  ksort_status_t st = current_device(&dev);
  if (st != KSORT_OK) return st;
  const size_t kb = key_bytes(dt);
  if ((st = check_device_ptr(keys, kb, dev)) != KSORT_OK) return st;
  if (offsets && (st = check_device_ptr(offsets, 8, dev)) != KSORT_OK) return st;
  std::lock_guard<std::mutex> lk(g_mu);
  const Tuning tu = g_tuning[dt];
  Workspace *ws = nullptr;
  st = get_workspace(dev, s, need_for(dt, total, num_arrays, tu.variant), &ws);
  if (st != KSORT_OK) return st;
  Grids g{};
  if ((st = full_grids(dt, dev, tu, &g)) != KSORT_OK) return st;
  if (!offsets) {
    // one array: no more CTAs than its first level has tiles, or than small items
    const KernelInfo ki = ops(dt).info(tu.variant);
    g.tiles = (int)std::max<long long>(
        1, std::min<long long>(g.tiles, (total + ki.tile_keys - 1) / ki.tile_keys));
    g.smalls = (int)std::max<long long>(
        1, std::min<long long>(g.smalls, 2 * ((total + tu.cutoff - 1) / tu.cutoff)));
  }
  SortParams p = sort_params(*ws, keys, tu);
  p.offsets = reinterpret_cast<const long long *>(offsets);
  {
    // medium items are served by tile_kernel alone (the register form's queue)
    const int form = ops(dt).info(tu.variant).form;
    p.medium_tiles = form == 0 || form == kWaveForm ? tu.medium_tiles : 0;
    p.reserve = (form == 0 || form == kWaveForm) && tu.reserve ? 1 : 0;
  }
  p.num_roots = offsets ? num_arrays : 1;
  p.total = total;
  p.readable[0] = total;
  p.readable[1] = total + (long long)(kScratchPad / kb);
  const KernelInfo kinfo = ops(dt).info(tu.variant);
  if (kinfo.form == kWaveForm && (offsets || total > tu.cutoff)) {
    // level-synchronous passes for the upper levels, then the work queue for the rest
    const int shape = tu.variant % kTileShapes;
    int wocc = 0, sms = 0;
    if ((st = wave_occupancy(dt, shape, &wocc)) != KSORT_OK) return st;
    if ((st = device_sms(dev, &sms)) != KSORT_OK) return st;
    long long grid = std::min<long long>((long long)sms * wocc, kWaveMaxGrid);
    if (!offsets) grid = std::max<long long>(1, std::min<long long>(grid, (total + kinfo.tile_keys - 1) / kinfo.tile_keys));
    const int levels = tu.wave_levels > 0 ? tu.wave_levels
                                          : auto_wave_levels(total, p.num_roots, tu.cutoff);
    p.wave = 1;
    PhaseMarks pm;
    if ((st = phase_begin(dev, s, &pm)) != KSORT_OK) return st;
    KS_CUDA(pm.mark());
    KS_CUDA(ops(dt).seed(p, tu.variant, s));
    KS_CUDA(pm.mark());
    for (int l = 0; l < levels; ++l) KS_CUDA(ops(dt).wave_level(p, shape, l, (int)grid, true, s));
    KS_CUDA(ops(dt).wave_handoff(p, shape, levels, true, s));
    KS_CUDA(ops(dt).tiles(p, tu.variant, g.tiles, s));
    KS_CUDA(pm.mark());
    KS_CUDA(ops(dt).smalls(p, g.smalls, s));
    KS_CUDA(pm.mark());
    ws->launches = 2ull * (unsigned long long)levels + 4ull;
    return KSORT_OK;
  }
  if (tu.cluster && !offsets && total > tu.cutoff && tu.cutoff >= 64 &&
      total < (long long)kClusterMaxSegs * (tu.cutoff + 1)) {
    // the upper levels in one thread-block cluster, when the array fits its shared memory
    int csize = 0, max_sl = 0;
    if ((st = cluster_setup(dt, dev, &csize, &max_sl)) != KSORT_OK) return st;
    const long long sl = ((total + csize - 1) / std::max(csize, 1) + 3) / 4 * 4;
    if (csize > 0 && sl <= max_sl) {
      PhaseMarks pm;
      if ((st = phase_begin(dev, s, &pm)) != KSORT_OK) return st;
      KS_CUDA(pm.mark());
      KS_CUDA(pm.mark());  // no seed launch: the cluster kernel starts the generation
      KS_CUDA(ops(dt).cluster_sort(p, csize, (int)sl, s));
      KS_CUDA(pm.mark());
      KS_CUDA(ops(dt).smalls(p, g.smalls, s));
      KS_CUDA(pm.mark());
      ws->launches = 2;
      return KSORT_OK;
    }
  }
  if (tu.fuse_park > 0 && tu.variant == kFusedVariant && (offsets || total > tu.cutoff)) {
    // the tile kernel finishes small items too: while enough of its CTAs already wait
    // for tiles of items still to come, the others take small items; the finisher
    // launch that follows takes the rest of the small list
    int focc = 0, sms = 0;
    if ((st = fused_occupancy(dt, tu.cutoff, &focc)) != KSORT_OK) return st;
    if ((st = device_sms(dev, &sms)) != KSORT_OK) return st;
    long long grid = (long long)sms * focc;
    if (!offsets) {
      const long long first = (total + kinfo.tile_keys - 1) / kinfo.tile_keys;
      const long long smalls = 2 * ((total + tu.cutoff - 1) / tu.cutoff);
      grid = std::max<long long>(1, std::min<long long>(grid, std::max(first, smalls)));
    }
    p.fuse_park = tu.fuse_park;
    PhaseMarks pm;
    if ((st = phase_begin(dev, s, &pm)) != KSORT_OK) return st;
    KS_CUDA(pm.mark());
    KS_CUDA(ops(dt).seed(p, tu.variant, s));
    KS_CUDA(pm.mark());
    KS_CUDA(ops(dt).tiles_fused(p, (int)grid, s));
    KS_CUDA(pm.mark());
    KS_CUDA(ops(dt).smalls(p, g.smalls, s));
    KS_CUDA(pm.mark());
    ws->launches = 3;
    return KSORT_OK;
  }
  PhaseMarks pm;
  if ((st = phase_begin(dev, s, &pm)) != KSORT_OK) return st;
  KS_CUDA(pm.mark());
  KS_CUDA(ops(dt).seed(p, tu.variant, s));
  KS_CUDA(pm.mark());
  const bool tiles = offsets || total > tu.cutoff;
  if (tiles) KS_CUDA(ops(dt).tiles(p, tu.variant, g.tiles, s));
  KS_CUDA(pm.mark());
  KS_CUDA(ops(dt).smalls(p, g.smalls, s));
  KS_CUDA(pm.mark());
  ws->launches = tiles ? 3ull : 2ull;
  return KSORT_OK;
}

// One warp waits for descriptor 0, which stays at generation 0 (never a live epoch).
__global__ void selftest_wait_kernel(unsigned long long *lb, Control *ctl,
                                     unsigned long long limit_ns) {
  unsigned long long E = 0, steps = 0;
  const int st = dev::lookback(lb, 1u, 0xffffffffu, limit_ns, &ctl->abort, &E, &steps);
  if (threadIdx.x == 0 && st == 1) dev::raise_error(ctl, kDevTimeout, 0x400000000ull);
}

// ------------------------------------------------------------------ fixed-scratch partition
// ksort_partition_out_noalloc makes three launches: the seed kernel, tile_kernel in its
// default shape (variant 0) with a partition-only root, and a one-thread status kernel.
// It keeps their control block, work item, look-back descriptors and ticket map in one
// file-scope device array instead of a per-stream workspace, so that a call allocates
// nothing. (ksort_partition_out's default is the ring partition, part_ring_kernel; the
// two agree on the key index and on both sides as multisets.) Layout: [Control][items]
// [item counters][small list][look-back][ticket map].
constexpr unsigned long long kNoallocItems = 4;  // a single partition queues only its root
// Tile tickets of the largest input: KSORT_NOALLOC_MAX_KEYS keys at the smallest tile
// (4096 float64 keys), plus one for a start that is not tile-aligned, plus slack.
constexpr unsigned long long kNoallocTiles = KSORT_NOALLOC_MAX_KEYS / 4096 + 64;
constexpr size_t kNoallocItemsOff = (sizeof(Control) + 255) / 256 * 256;
constexpr size_t kNoallocIctlOff = kNoallocItemsOff + kNoallocItems * sizeof(Item);
constexpr size_t kNoallocSqOff = kNoallocIctlOff + kNoallocItems * sizeof(ItemCtl);
constexpr size_t kNoallocLbOff = (kNoallocSqOff + kNoallocItems * 8 + 255) / 256 * 256;
constexpr size_t kNoallocTmapOff = kNoallocLbOff + kNoallocTiles * 8;
constexpr size_t kNoallocBytes = kNoallocTmapOff + kNoallocTiles * 8;  // about 67 KB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr int kNoallocMaxDevices = 64;
struct NoallocDevice {
  bool ready = false;
  unsigned char *base = nullptr;  // device address of g_noalloc_scratch on this device
  int sms = 0;
  int tile_ctas[3] = {0, 0, 0};   // tile_kernel CTAs per SM, per dtype
};
NoallocDevice g_noalloc[kNoallocMaxDevices];

// First call on a device (with that device current): look up the array's address,
// read the SM count and the tile kernel's occupancy, and clear the array on `s`.
ksort_status_t noalloc_device(int dev, cudaStream_t s, NoallocDevice **out) {
  if (dev < 0 || dev >= kNoallocMaxDevices) return KSORT_ERR_INVALID_ARG;
  NoallocDevice &d = g_noalloc[dev];
  if (!d.ready) {
    void *base = nullptr;
    KS_CUDA(cudaGetSymbolAddress(&base, g_noalloc_scratch));
    KS_CUDA(cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev));
    for (int t = 0; t < 3; ++t) {
      int small_ctas = 0;
      KS_CUDA(ops((ksort_dtype_t)t).occupancy(0, g_tuning[t].cutoff, 256, &d.tile_ctas[t],
                                              &small_ctas));
      if (d.tile_ctas[t] < 1) return KSORT_ERR_INTERNAL;
    }
    KS_CUDA(cudaMemsetAsync(base, 0, kNoallocBytes, s));
    d.base = static_cast<unsigned char *>(base);
    d.ready = true;
  }
  *out = &d;
  return KSORT_OK;
}

// Runs after the tile pass: a device-side error becomes a negative key index, and the
// next call starts with a clear flag.
__global__ void noalloc_status_kernel(Control *ctl, long long *key_index) {
  const unsigned e = ctl->error;
  if (e) *key_index = -(long long)e;
}

ksort_status_t partition_noalloc_impl(ksort_dtype_t dt, const void *in, void *out, int64_t n,
                                      int64_t *key_index, cudaStream_t s) {
  if (!dtype_ok(dt)) return KSORT_ERR_UNSUPPORTED_DTYPE;
  if (n < 1) return KSORT_ERR_INVALID_ARG;
  if (n > KSORT_NOALLOC_MAX_KEYS) return KSORT_ERR_TOO_LARGE;
  int dev = 0;
  ksort_status_t st = current_device(&dev);
  if (st != KSORT_OK) return st;
  const size_t kb = key_bytes(dt);
  if ((st = check_device_ptr(in, kb, dev)) != KSORT_OK) return st;
  if ((st = check_device_ptr(out, kb, dev)) != KSORT_OK) return st;
  if ((st = check_device_ptr(key_index, 8, dev)) != KSORT_OK) return st;
  {
    const char *a = static_cast<const char *>(in), *b = static_cast<const char *>(out);
    if (a < b + n * kb && b < a + n * kb) return KSORT_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  NoallocDevice *d = nullptr;
  if ((st = noalloc_device(dev, s, &d)) != KSORT_OK) return st;
  if (n == 1) {
    KS_CUDA(cudaMemsetAsync(key_index, 0, sizeof(int64_t), s));
    KS_CUDA(cudaMemcpyAsync(out, in, kb, cudaMemcpyDeviceToDevice, s));
    return KSORT_OK;
  }
  // always the default tile shape (variant 0), whatever the tuning says
  const long long tiles = ops(dt).tile_count(0, in, 0, n);
  if ((unsigned long long)tiles > kNoallocTiles) return KSORT_ERR_TOO_LARGE;
  const Tuning tu = g_tuning[dt];
  unsigned char *b = d->base;
  Control *ctl = reinterpret_cast<Control *>(b);
  SortParams p{};
  p.keys = const_cast<void *>(in);
  p.scratch = out;
  p.ctl = ctl;
  p.items = reinterpret_cast<Item *>(b + kNoallocItemsOff);
  p.ictl = reinterpret_cast<ItemCtl *>(b + kNoallocIctlOff);
  p.small_q = reinterpret_cast<unsigned long long *>(b + kNoallocSqOff);
  p.item_cap = kNoallocItems;
  p.lb = reinterpret_cast<unsigned long long *>(b + kNoallocLbOff);
  p.tmap = reinterpret_cast<unsigned long long *>(b + kNoallocTmapOff);
  p.lb_cap = kNoallocTiles;
  p.num_roots = 1;
  p.total = n;
  p.cutoff = tu.cutoff;
  p.root_flags = kItemPartitionOnly;
  p.spin_limit_ns = (unsigned long long)tu.spin_limit_ms * 1000000ull;
  p.key_index = reinterpret_cast<long long *>(key_index);
  p.readable[0] = n;
  p.readable[1] = 0;  // the output is only written
  // The seed kernel resets every dispatch counter and moves to a new generation, which
  // retires the descriptors and ticket-map entries of earlier calls; only the sticky
  // error word and its info must be cleared here.
  const size_t e0 = offsetof(Control, error), e1 = offsetof(Control, err_info) + 8;
  KS_CUDA(cudaMemsetAsync(b + e0, 0, e1 - e0, s));
  const int grid = (int)std::max<long long>(
      1, std::min<long long>((long long)d->sms * d->tile_ctas[dt], tiles));
  KS_CUDA(ops(dt).seed(p, 0, s));
  KS_CUDA(ops(dt).tiles(p, 0, grid, s));
  noalloc_status_kernel<<<1, 1, 0, s>>>(ctl, p.key_index);
  KS_CUDA(cudaGetLastError());
  return KSORT_OK;
}

// Failure-path check of the fixed-scratch partition: one warp waits, as tile_kernel's
// look-back does, for a descriptor of the fixed array that nothing publishes, gives up
// after the limit (error word := KSORT_ERR_TIMEOUT), and the call's status kernel
// turns the error into a negative key index.
ksort_status_t selftest_noalloc_impl(int32_t limit_ms, int64_t *key_index, cudaStream_t s) {
  if (limit_ms < 1 || limit_ms > 60000) return KSORT_ERR_INVALID_ARG;
  int dev = 0;
  ksort_status_t st = current_device(&dev);
  if (st != KSORT_OK) return st;
  if ((st = check_device_ptr(key_index, 8, dev)) != KSORT_OK) return st;
  std::lock_guard<std::mutex> lk(g_mu);
  NoallocDevice *d = nullptr;
  if ((st = noalloc_device(dev, s, &d)) != KSORT_OK) return st;
  unsigned char *b = d->base;
  Control *ctl = reinterpret_cast<Control *>(b);
  unsigned long long *lb = reinterpret_cast<unsigned long long *>(b + kNoallocLbOff);
  // as at the start of a call: a clear error word; descriptor 0 at generation 0, the
  // state of a fresh array, which the next call's seed kernel retires like any other
  const size_t e0 = offsetof(Control, error), e1 = offsetof(Control, err_info) + 8;
  KS_CUDA(cudaMemsetAsync(b + e0, 0, e1 - e0, s));
  KS_CUDA(cudaMemsetAsync(&ctl->abort, 0, sizeof(unsigned), s));
  KS_CUDA(cudaMemsetAsync(lb, 0, sizeof(unsigned long long), s));
  selftest_wait_kernel<<<1, 32, 0, s>>>(lb, ctl, (unsigned long long)limit_ms * 1000000ull);
  noalloc_status_kernel<<<1, 1, 0, s>>>(ctl, reinterpret_cast<long long *>(key_index));
  KS_CUDA(cudaGetLastError());
  return KSORT_OK;
}

}  // namespace
}  // namespace ksort

using namespace ksort;

extern "C" {

ksort_status_t ksort_partition(ksort_dtype_t dtype, void *keys_dev, int64_t n,
                               int64_t *key_index_dev, ksort_stream_t stream) {
  return partition_impl(dtype, keys_dev, nullptr, n, key_index_dev, (cudaStream_t)stream, true);
}

ksort_status_t ksort_partition_out(ksort_dtype_t dtype, const void *in_dev, void *out_dev,
                                   int64_t n, int64_t *key_index_dev, ksort_stream_t stream) {
  return partition_impl(dtype, in_dev, out_dev, n, key_index_dev, (cudaStream_t)stream, false);
}

ksort_status_t ksort_partition_out_noalloc(ksort_dtype_t dtype, const void *in_dev, void *out_dev,
                                           int64_t n, int64_t *key_index_dev,
                                           ksort_stream_t stream) {
  return partition_noalloc_impl(dtype, in_dev, out_dev, n, key_index_dev, (cudaStream_t)stream);
}

ksort_status_t ksort_partition_exact(ksort_dtype_t dtype, const void *in_dev, void *out_dev,
                                     int64_t n, int64_t *key_index_dev, ksort_stream_t stream) {
  return partition_exact_impl(dtype, in_dev, out_dev, n, key_index_dev, (cudaStream_t)stream);
}

ksort_status_t ksort_sort(ksort_dtype_t dtype, void *keys_dev, int64_t n, ksort_stream_t stream) {
  return sort_impl(dtype, keys_dev, nullptr, 1, n, (cudaStream_t)stream);
}

ksort_status_t ksort_sort_batched(ksort_dtype_t dtype, void *keys_dev, const int64_t *offsets_dev,
                                  int64_t num_arrays, int64_t total_keys, ksort_stream_t stream) {
  if (num_arrays > 0 && !offsets_dev) return KSORT_ERR_INVALID_ARG;
  return sort_impl(dtype, keys_dev, offsets_dev, num_arrays, total_keys, (cudaStream_t)stream);
}

ksort_status_t ksort_reserve_workspace(ksort_dtype_t dtype, int64_t max_total_keys,
                                       int64_t max_arrays, ksort_stream_t stream) {
  if (!dtype_ok(dtype)) return KSORT_ERR_UNSUPPORTED_DTYPE;
  if (max_total_keys < 0 || max_arrays < 0) return KSORT_ERR_INVALID_ARG;
  int dev = 0;
  ksort_status_t st = current_device(&dev);
  if (st != KSORT_OK) return st;
  std::lock_guard<std::mutex> lk(g_mu);
  Workspace *ws = nullptr;
  st = get_workspace(dev, (cudaStream_t)stream,
                     need_for(dtype, max_total_keys, max_arrays, g_tuning[dtype].variant), &ws);
  if (st != KSORT_OK) return st;
  Grids g{};  // also warms the occupancy cache (no queries during graph capture)
  return full_grids(dtype, dev, g_tuning[dtype], &g);
}

ksort_status_t ksort_release_workspace(ksort_stream_t stream) {
  int dev = 0;
  ksort_status_t st = current_device(&dev);
  if (st != KSORT_OK) return st;
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_ws.find({dev, (cudaStream_t)stream});
  auto ph = g_phase.find({dev, (cudaStream_t)stream});
  if (ph != g_phase.end()) {
    KS_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    for (auto &slot : ph->second.ev)
      for (cudaEvent_t e : slot)
        if (e) KS_CUDA(cudaEventDestroy(e));
    g_phase.erase(ph);
  }
  if (it == g_ws.end()) return KSORT_OK;
  KS_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  if (it->second.base) KS_CUDA(cudaFree(it->second.base));
  g_ws.erase(it);
  return KSORT_OK;
}

ksort_status_t ksort_get_device_error(ksort_stream_t stream) {
  int dev = 0;
  ksort_status_t st = current_device(&dev);
  if (st != KSORT_OK) return st;
  KS_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_ws.find({dev, (cudaStream_t)stream});
  if (it == g_ws.end() || !it->second.base) return KSORT_OK;
  Workspace &ws = it->second;
  unsigned err = 0;
  KS_CUDA(cudaMemcpy(&err, &ws.ctl->error, sizeof(err), cudaMemcpyDeviceToHost));
  if (err) KS_CUDA(cudaMemset(&ws.ctl->error, 0, sizeof(err)));
  if (ws.pending_error) {
    err = ws.pending_error;
    ws.pending_error = 0;
  }
  return (ksort_status_t)err;
}

ksort_status_t ksort_get_stats(ksort_stream_t stream, ksort_stats_t *out) {
  if (!out) return KSORT_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  int dev = 0;
  ksort_status_t st = current_device(&dev);
  if (st != KSORT_OK) return st;
  KS_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_ws.find({dev, (cudaStream_t)stream});
  if (it == g_ws.end() || !it->second.base) return KSORT_OK;
  Control c;
  KS_CUDA(cudaMemcpy(&c, it->second.ctl, sizeof(c), cudaMemcpyDeviceToHost));
  out->large_items = c.large_items;
  out->large_keys = c.large_keys;
  out->tiles = c.tiles;
  out->small_items = c.small_items;
  out->small_keys = c.small_keys;
  out->smem_levels = c.smem_levels;
  out->lookback_steps = c.lookback_steps;
  out->items_pushed = c.pushed;  // pool slots: large and small items
  out->launches = it->second.launches;
  return KSORT_OK;
}

ksort_status_t ksort_set_phase_timing(int32_t enable) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_time_phases = enable != 0;
  return KSORT_OK;
}

ksort_status_t ksort_get_phase_times(ksort_stream_t stream, int32_t max_calls, float *out_ms,
                                     int32_t *calls) {
  if (!calls || max_calls < 0 || (max_calls > 0 && !out_ms)) return KSORT_ERR_INVALID_ARG;
  *calls = 0;
  int dev = 0;
  ksort_status_t st = current_device(&dev);
  if (st != KSORT_OK) return st;
  KS_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_phase.find({dev, (cudaStream_t)stream});
  if (it == g_phase.end()) return KSORT_OK;
  const PhaseEvents &pe = it->second;
  const long long kept = std::min<long long>(pe.calls, kPhaseRing);
  const long long n = std::min<long long>(kept, max_calls);
  for (long long c = 0; c < n; ++c) {  // oldest of the last n first
    const int slot = (int)((pe.calls - n + c) % kPhaseRing);
    float *o = out_ms + c * kPhasesOut;
    for (int i = 0; i < kPhasesOut; ++i) {
      float ms = -1.f;
      if (i + 1 < pe.marks[slot]) KS_CUDA(cudaEventElapsedTime(&ms, pe.ev[slot][i], pe.ev[slot][i + 1]));
      o[i] = ms;
    }
  }
  *calls = (int32_t)n;
  return KSORT_OK;
}

int32_t ksort_max_cutoff(ksort_dtype_t dtype) {
  if (!dtype_ok(dtype)) return 0;
  return ops(dtype).info(0).max_cutoff;
}

int32_t ksort_tile_keys(ksort_dtype_t dtype) {
  if (!dtype_ok(dtype)) return 0;
  std::lock_guard<std::mutex> lk(g_mu);
  return ops(dtype).info(g_tuning[dtype].variant).tile_keys;
}

ksort_status_t ksort_tile_shape(ksort_dtype_t dtype, int32_t shape, int32_t *threads,
                                int32_t *keys_per_thread, int32_t *form) {
  if (!dtype_ok(dtype)) return KSORT_ERR_UNSUPPORTED_DTYPE;
  if (shape < 1 || shape > kTileVariants || !threads || !keys_per_thread || !form)
    return KSORT_ERR_INVALID_ARG;
  const KernelInfo ki = ops(dtype).info(shape - 1);
  *threads = ki.block;
  *keys_per_thread = ki.keys_per_thread;
  *form = ki.form;
  return KSORT_OK;
}

ksort_status_t ksort_partition_shape(ksort_dtype_t dtype, int32_t form, int32_t *threads,
                                     int32_t *tile_keys, int32_t *ctas_per_sm) {
  if (!dtype_ok(dtype)) return KSORT_ERR_UNSUPPORTED_DTYPE;
  if (form < 1 || form > kRingConfigs || !threads || !tile_keys || !ctas_per_sm)
    return KSORT_ERR_INVALID_ARG;
  const RingInfo ri = ops(dtype).ring_info(form);
  *threads = ri.block;
  *tile_keys = ri.tile_keys;
  *ctas_per_sm = ri.min_blocks;
  return KSORT_OK;
}

ksort_status_t ksort_set_tuning(ksort_dtype_t dtype, const ksort_tuning_t *t) {
  if (!dtype_ok(dtype)) return KSORT_ERR_UNSUPPORTED_DTYPE;
  if (!t) return KSORT_ERR_INVALID_ARG;
  const int maxc = ops(dtype).info(0).max_cutoff;
  if (t->cutoff < 0 || (t->cutoff > 0 && (t->cutoff < 2 || t->cutoff > maxc))) return KSORT_ERR_INVALID_ARG;
  if (t->ctas_per_sm < -1 || t->spin_limit_ms < 0 || t->spin_limit_ms > 600000)
    return KSORT_ERR_INVALID_ARG;
  if (t->tile_shape < 0 || t->tile_shape > kTileVariants) return KSORT_ERR_INVALID_ARG;
  if (t->wave_levels < -1 || t->wave_levels > 64) return KSORT_ERR_INVALID_ARG;
  if (t->medium_tiles < -1 || t->medium_tiles > kMediumMaxTiles) return KSORT_ERR_INVALID_ARG;
  if (t->partition_form < -1 || t->partition_form > kRingConfigs) return KSORT_ERR_INVALID_ARG;
  if (t->sort_reserve < -1 || t->sort_reserve > 1) return KSORT_ERR_INVALID_ARG;
  if (t->finish_in_tiles < -1 || t->finish_in_tiles > 4096) return KSORT_ERR_INVALID_ARG;
  if (t->finisher_threads != 0 && t->finisher_threads != 256 && t->finisher_threads != 512 &&
      t->finisher_threads != 1024)
    return KSORT_ERR_INVALID_ARG;
  if (t->cluster_sort < -1 || t->cluster_sort > 1) return KSORT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  Tuning &g = g_tuning[dtype];
  if (t->cutoff) g.cutoff = t->cutoff;
  if (t->ctas_per_sm) g.ctas_per_sm = t->ctas_per_sm < 0 ? 0 : t->ctas_per_sm;
  if (t->spin_limit_ms) g.spin_limit_ms = t->spin_limit_ms;
  if (t->tile_shape) g.variant = t->tile_shape - 1;
  if (t->wave_levels) g.wave_levels = t->wave_levels < 0 ? 0 : t->wave_levels;
  if (t->medium_tiles) g.medium_tiles = t->medium_tiles < 0 ? 0 : t->medium_tiles;
  if (t->partition_form) g.part_form = t->partition_form < 0 ? 0 : t->partition_form;
  if (t->sort_reserve) g.reserve = t->sort_reserve > 0 ? 1 : 0;
  if (t->finish_in_tiles) g.fuse_park = t->finish_in_tiles < 0 ? 0 : t->finish_in_tiles;
  if (t->finisher_threads) g.small_threads = t->finisher_threads;
  if (t->cluster_sort) g.cluster = t->cluster_sort > 0 ? 1 : 0;
  return KSORT_OK;
}

ksort_status_t ksort_get_tuning(ksort_dtype_t dtype, ksort_tuning_t *out) {
  if (!dtype_ok(dtype)) return KSORT_ERR_UNSUPPORTED_DTYPE;
  if (!out) return KSORT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  const Tuning &g = g_tuning[dtype];
  out->cutoff = g.cutoff;
  out->ctas_per_sm = g.ctas_per_sm;
  out->spin_limit_ms = g.spin_limit_ms;
  out->tile_shape = g.variant + 1;
  out->wave_levels = g.wave_levels ? g.wave_levels : -1;
  out->medium_tiles = g.medium_tiles ? g.medium_tiles : -1;
  out->partition_form = g.part_form ? g.part_form : -1;
  out->sort_reserve = g.reserve ? 1 : -1;
  out->finish_in_tiles = g.fuse_park ? g.fuse_park : -1;
  out->finisher_threads = g.small_threads;
  out->cluster_sort = g.cluster ? 1 : -1;
  return KSORT_OK;
}

ksort_status_t ksort_debug_trace(uint64_t *trace_dev, int64_t tickets) {
  if (tickets < 0 || (tickets > 0 && !trace_dev)) return KSORT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  g_trace = reinterpret_cast<unsigned long long *>(trace_dev);
  g_trace_cap = trace_dev ? tickets : 0;
  return KSORT_OK;
}

ksort_status_t ksort_selftest_wait_timeout(int32_t limit_ms, ksort_stream_t stream) {
  if (limit_ms < 1 || limit_ms > 60000) return KSORT_ERR_INVALID_ARG;
  int dev = 0;
  ksort_status_t st = current_device(&dev);
  if (st != KSORT_OK) return st;
  std::lock_guard<std::mutex> lk(g_mu);
  Workspace *ws = nullptr;
  Need need = need_for(KSORT_F32, 1, 1, 0);
  need.item_cap = 64;
  need.scratch_bytes = 4;
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = get_workspace(dev, s, need, &ws)) != KSORT_OK) return st;
  KS_CUDA(cudaMemsetAsync(ws->lb, 0, sizeof(unsigned long long), s));
  KS_CUDA(cudaMemsetAsync(&ws->ctl->abort, 0, sizeof(unsigned), s));
  selftest_wait_kernel<<<1, 32, 0, s>>>(ws->lb, ws->ctl,
                                        (unsigned long long)limit_ms * 1000000ull);
  KS_CUDA(cudaGetLastError());
  return KSORT_OK;
}

ksort_status_t ksort_cluster_shape(ksort_dtype_t dtype, int32_t *cluster_ctas, int64_t *max_keys) {
  if (!dtype_ok(dtype)) return KSORT_ERR_UNSUPPORTED_DTYPE;
  if (!cluster_ctas || !max_keys) return KSORT_ERR_INVALID_ARG;
  int dev = 0;
  ksort_status_t st = current_device(&dev);
  if (st != KSORT_OK) return st;
  std::lock_guard<std::mutex> lk(g_mu);
  int csize = 0, max_sl = 0;
  if ((st = cluster_setup(dtype, dev, &csize, &max_sl)) != KSORT_OK) return st;
  *cluster_ctas = csize;
  *max_keys = (int64_t)csize * max_sl;
  return KSORT_OK;
}

ksort_status_t ksort_selftest_noalloc_timeout(int32_t limit_ms, int64_t *key_index_dev,
                                              ksort_stream_t stream) {
  return selftest_noalloc_impl(limit_ms, key_index_dev, (cudaStream_t)stream);
}

const char *ksort_status_string(ksort_status_t s) {
  switch (s) {
    case KSORT_OK: return "ok";
    case KSORT_ERR_INVALID_ARG: return "invalid argument";
    case KSORT_ERR_UNSUPPORTED_DTYPE: return "unsupported dtype";
    case KSORT_ERR_OUT_OF_MEMORY: return "workspace allocation failed (or needed during graph capture)";
    case KSORT_ERR_CUDA: return "CUDA runtime error";
    case KSORT_ERR_TIMEOUT: return "a device-side wait ran past its time limit";
    case KSORT_ERR_BAD_OFFSETS: return "bad offsets";
    case KSORT_ERR_WORKSPACE_EXHAUSTED: return "work queue or look-back arena exhausted";
    case KSORT_ERR_INTERNAL: return "internal error";
    case KSORT_ERR_TOO_LARGE: return "n exceeds the fixed scratch of ksort_partition_out_noalloc (KSORT_NOALLOC_MAX_KEYS = 2^24 keys)";
  }
  return "unknown status";
}

const char *ksort_last_cuda_error(void) { return g_cuda_error; }

}  // extern "C"
