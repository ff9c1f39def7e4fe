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
  kItemScratch = 1u,  // keys of the item live in the scratch buffer (else in the caller's)
  kItemSmall = 2u,    // finished in shared memory by one CTA
};

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
  // SM cycles spent by the CTAs of the sort kernel, by phase (sum over CTAs)
  unsigned long long cyc_fetch, cyc_small, cyc_tile, cyc_finish;
  unsigned long long pad1[3];
};

// One work item: a sub-array [begin, end) whose first element is its key.
struct alignas(32) Item {
  long long begin;
  long long end;
  unsigned tiles;   // tile passes of a large item; 1 for a small item
  unsigned lb;      // first look-back descriptor of a large item
  unsigned flags;   // kItemScratch | kItemSmall
  unsigned epoch;   // generation of the sort that wrote the item
};

struct alignas(16) ItemCtl {
  unsigned grab;            // tiles handed out
  unsigned done;            // tiles finished
  unsigned long long less;  // #{x < key} of the item, written by its last tile
};

// State of the standalone partition, carried from call to call on one stream: tickets
// and completions count up forever; `base` is their value when the current call
// started and `gen` numbers the call (its look-back descriptors carry the generation).
// The last CTA of a call advances `base` and `gen` and clears `abort`, so no memset is
// needed between calls.
struct alignas(64) PartCtl {
  unsigned long long ticket;
  unsigned long long done;
  unsigned long long base;
  unsigned long long less;
  unsigned gen;
  unsigned abort;
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
  int pad;
  unsigned long long spin_limit_ns;
};

struct PartParams {
  const void *in;
  void *out;
  long long n;
  long long *key_index;
  PartCtl *pctl;
  unsigned long long *lb;
  Control *ctl;  // receives device errors
  unsigned long long spin_limit_ns;
};

// Host-side launch interface, one explicit instantiation per key type.
struct KernelInfo {
  int block;          // threads per CTA
  int tile_keys;      // keys per tile pass
  int max_cutoff;     // largest shared-memory item the kernel supports
};

template <typename K>
struct Launcher {
  static KernelInfo info();
  static size_t sort_smem_bytes(int cutoff);
  static cudaError_t max_ctas_per_sm(int cutoff, int *out);
  static cudaError_t partition_out(const PartParams &p, int num_tiles, cudaStream_t s);
  static cudaError_t seed(const SortParams &p, cudaStream_t s);
  static cudaError_t sort(const SortParams &p, int grid, cudaStream_t s);
  static long long tile_count(const void *buf, long long begin, long long end);
};

}  // namespace ksort
