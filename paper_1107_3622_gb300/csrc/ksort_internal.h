// Internal layout shared by the host API and the kernels of libksort.
// Nothing here is part of the public C ABI (include/ksort.h).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace ksort {

// Device status codes; equal to the public ksort_status_t values.
enum : unsigned {
  kDevOk = 0,
  kDevTimeout = 5,
  kDevBadOffsets = 6,
  kDevWorkspaceExhausted = 7,
  kDevInternal = 8,
};

// Item flags.
enum : unsigned {
  kItemScratch = 1u,        // keys of the item live in buffer 1 (else in buffer 0)
  kItemSmall = 2u,          // finished in shared memory by one CTA
  kItemPartitionOnly = 4u,  // Steps 1-4 only: key and sides go to buffer 1, no recursion
  kItemMedium = 8u,         // one ticket: a single CTA runs every tile pass of the item
};

// Largest item (in tile passes) that may go to a single CTA (kItemMedium).
constexpr int kMediumMaxTiles = 16;

// Largest sub-array, in keys, that one partition may handle: tile prefixes are
// carried in 31 bits of a look-back descriptor.
constexpr long long kMaxItemKeys = 0x7fffffffLL;

// Per-workspace control block (device memory). The dispatch fields are reset by the
// seed kernel at every sort; `error` is sticky until the host reads it.
struct alignas(128) Control {
  unsigned long long pushed;           // work items allocated in the pool
  unsigned long long large_pushed;     // large items queued
  unsigned long long large_completed;  // large items fully partitioned
  unsigned long long tq_head;          // tile tickets claimed by CTAs
  unsigned long long lb_used;          // tile tickets (= look-back descriptors) issued
  unsigned long long sq_head, sq_tail; // small-item list: claimed, queued
  unsigned epoch;                // generation of the current sort (never 0)
  unsigned abort;                // nonzero: stop the current call early
  unsigned error;                // first device error since the host last read it
  unsigned pad0;
  unsigned long long err_info;
  // statistics of the last sort
  unsigned long long large_items, large_keys, tiles, small_items, small_keys;
  unsigned long long smem_levels, lookback_steps;
  // single-partition kernel: CTAs finished, and its own stop flag (both back to 0 when
  // the last CTA of a call finishes)
  unsigned part_done, part_abort;
  unsigned long long part_ticket;  // ring partition: tiles claimed (0 between calls)
  // ring partition: CTAs finished (0 between calls), and the generation of the last call
  // that stopped on an error (never cleared)
  unsigned ring_done, ring_abort;
  // ring partition, reservation form: (>= keys << 32) | less keys of the tiles that have
  // taken their output ranges so far (0 between calls)
  unsigned long long ring_resv;
  // level-synchronous passes: per level parity, items << kWaveKeyBits | classified keys
  unsigned long long wave_ctr[2];
  unsigned long long wave_fin;  // keys of an even level waiting for their final index
};

// Level-synchronous partition passes (the wave form): the sub-arrays above the cutoff
// at one recursion depth form a list, and their classified keys (all but each key)
// are numbered consecutively in list order, the level's key space.
constexpr int kWaveKeyBits = 40;
constexpr unsigned long long kWaveKeyMask = (1ull << kWaveKeyBits) - 1ull;
struct alignas(16) WaveItem {
  long long begin;  // sub-array [begin, end); its key is the element at begin
  long long end;
  long long koff;   // level key-space index of the element at begin + 1
  long long pad;
};

// One work item: a sub-array [begin, end) whose first element is its key.
struct alignas(16) Item {
  long long begin;
  long long end;
  unsigned long long key;  // bit pattern of the item's first element (its key, Step 1)
  unsigned tiles;          // tile passes of a large item; 1 for a small item
  unsigned lb;             // first tile ticket (= look-back descriptor) of a large item
  unsigned flags;          // kItemScratch | kItemSmall | kItemPartitionOnly
  unsigned epoch;          // generation of the sort that wrote the item
};

struct alignas(16) ItemCtl {
  unsigned grab;            // tiles handed out
  unsigned done;            // tiles finished
  // #{x < key} of the item, written by its last tile; with reservation, the running
  // (>= keys << 32) | less keys of the tiles that have taken their ranges
  unsigned long long less;
};

struct SortParams {
  void *keys;          // buffer 0: the caller's keys, where every result lands
  void *scratch;       // buffer 1: ping-pong partner of the same size
  Control *ctl;
  Item *items;
  ItemCtl *ictl;
  unsigned long long *small_q;  // item_cap entries: (epoch << 32) | item index
  unsigned long long item_cap;
  unsigned long long *lb;       // lb_cap look-back descriptors, one per tile ticket
  unsigned long long *tmap;     // lb_cap entries: (epoch << 32) | item of the ticket
  unsigned long long lb_cap;
  const long long *offsets;  // roots: offsets[r] .. offsets[r+1]; null = one root [0, n)
  long long num_roots;
  long long total;           // keys in buffer 0 that roots may cover
  int cutoff;                // largest small item
  unsigned root_flags;       // item flags of the roots (kItemPartitionOnly for a partition)
  unsigned long long spin_limit_ns;
  long long *key_index;      // partition only: receives the key's index (device)
  long long readable[2];     // elements [0, readable[j]) of buffer j may be read in bulk
  unsigned long long *trace; // optional: kTraceWords timestamps per tile ticket
  long long trace_cap;       // tickets the trace buffer holds
  // wave form: two level lists of wave_cap items (level parity), two less counts per
  // CTA of a level pass, and wave_cap (index, key bits) pairs of keys placed late
  WaveItem *wave_items;
  unsigned long long wave_cap;
  unsigned long long *wave_cnt;
  unsigned long long *wave_fin;
  int wave;                  // nonzero: the seed queues large roots on the level-0 list
  int medium_tiles;          // items of 2 .. medium_tiles tile passes go to one CTA; 0: off
  int reserve;               // tile_kernel: output ranges by reservation, not look-back
  int small_threads;         // small_kernel CTA: 256, 512 or 1024 threads
  int fuse_park;             // fused tile_kernel: tickets held ahead of the issued ones
                             // before a CTA takes a small item instead of a ticket
};
constexpr int kTraceWords = 8;

// Host-side launch interface, one explicit instantiation per key type. `variant`
// selects one of kTileVariants compiled forms of the tile passes, for three CTA shapes
// each: tile_kernel (variants 0-2, keys loaded into registers), tile_pipe_kernel (3-5,
// staged through shared memory by bulk copies), tile_ws_kernel (6-8, warp roles) and
// the wave form (9-11: level-synchronous passes for the upper levels, then tile_kernel
// of the same shape for what remains).
constexpr int kTileShapes = 3;
constexpr int kTileForms = 4;
constexpr int kWaveForm = 3;
constexpr int kWaveMaxGrid = 4096;  // CTAs of one level pass (two counts each)
constexpr int kTileVariants = kTileForms * kTileShapes;
// The tile variant whose CTAs can also finish small items (queue form, 256 threads).
constexpr int kFusedVariant = 2;
// Cluster form: most sub-arrays above the cutoff that one level can hold (the host
// takes the cluster form only for arrays of fewer than this many times cutoff + 1 keys).
constexpr int kClusterMaxSegs = 512;
// Threads of a finisher CTA: 256 (the default), 512 or 1024.
constexpr int small_threads_of(int nt) { return nt == 1024 || nt == 512 ? nt : 256; }

struct KernelInfo {
  int block;          // threads per tile-pass CTA
  int tile_keys;      // keys per tile pass
  int max_cutoff;     // largest shared-memory item the kernels support
  int keys_per_thread;
  int form;           // 0 tile_kernel, 1 tile_pipe_kernel, 2 tile_ws_kernel, 3 wave
};

// One compiled configuration of the ring partition (part_ring_kernel).
constexpr int kRingConfigs = 6;
struct RingInfo {
  int block;        // threads per CTA (producer warp, look-back warp, data warps)
  int tile_keys;    // keys per tile
  int min_blocks;   // CTAs per SM the kernel is compiled for
  int data_warps;
  int keys_per_lane;
};

template <typename K>
struct Launcher {
  static KernelInfo info(int variant);
  static size_t small_smem_bytes(int cutoff);
  // CTAs per SM of the tile kernel of `variant` and of the finisher of nt threads
  static cudaError_t occupancy(int variant, int cutoff, int nt, int *tile_ctas, int *small_ctas);
  static cudaError_t seed(const SortParams &p, int variant, cudaStream_t s);
  static cudaError_t tiles(const SortParams &p, int variant, int grid, cudaStream_t s);
  static cudaError_t smalls(const SortParams &p, int grid, cudaStream_t s);
  // the upper levels of one array in a thread-block cluster (cluster_kernel): the
  // cluster size that can run (0: none) and the largest slice per CTA; one launch
  static cudaError_t cluster_setup(int *csize, int *max_sl);
  static cudaError_t cluster_sort(const SortParams &p, int csize, int sl, cudaStream_t s);
  // tile_kernel in tile variant kFusedVariant with the finisher inside (no smalls launch)
  static cudaError_t fused_occupancy(int cutoff, int *ctas);
  static cudaError_t tiles_fused(const SortParams &p, int grid, cudaStream_t s);
  static long long tile_count(int variant, const void *buf, long long begin, long long end);
  // single partitions: part_kernel with CTA shape `shape` (0 .. kTileShapes - 1)
  static cudaError_t part_occupancy(int shape, int *ctas);
  static cudaError_t partition(const SortParams &p, int shape, int grid, cudaStream_t s);
  // single partitions: part_ring_kernel in configuration `cfg` (1 .. kRingConfigs)
  static RingInfo ring_info(int cfg);
  static cudaError_t ring_occupancy(int cfg, int *ctas);
  static cudaError_t ring_partition(const SortParams &p, int cfg, int grid, cudaStream_t s);
  // Steps 1-4 in the paper's element order (exact layout), n >= 2; `work` holds
  // exact_work_bytes(n) bytes of device scratch.
  static size_t exact_work_bytes(long long n);
  static cudaError_t exact(const void *in, void *out, long long n, long long *key_index,
                           void *work, cudaStream_t s);
  // wave form, CTA shape `shape`: CTAs per SM of a level pass; one level (count and
  // scatter launches, chained by programmatic dependent launch when `pdl`); hand-off of
  // the list of level `level` to the work queue of tile_kernel
  static cudaError_t wave_occupancy(int shape, int *ctas);
  static cudaError_t wave_level(const SortParams &p, int shape, int level, int grid, bool pdl,
                                cudaStream_t s);
  static cudaError_t wave_handoff(const SortParams &p, int shape, int level, bool pdl,
                                  cudaStream_t s);
  // single partitions of the wave form: split_count_kernel, then split_move_kernel under
  // programmatic dependent launch (n >= 2; the per-warp counts go to p.wave_cnt)
  static cudaError_t partition_split(const SortParams &p, int shape, int sms, cudaStream_t s);
};

}  // namespace ksort
