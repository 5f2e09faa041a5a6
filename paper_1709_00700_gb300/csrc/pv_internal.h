// Host-side interface between the C-ABI layer (pv_api.cu) and the kernel
// translation units: launch configuration, result buffers and the registry
// of compiled pipeline shapes.
#pragma once

#include <cstdint>
#include <string>
#include <utility>
#include <vector>
#include <cuda_runtime.h>

#include "pv.h"
#include "pv_device.cuh"

namespace pv {

enum Mode { MODE_AGGREGATE = 0, MODE_GROUPED = 1, MODE_PROJECT = 2 };

// Launch shape resolved from a pv_variant.
// Internal status of a grouped launch (never returned through the C ABI): the
// 32-bit-field layout would send too many rows to the global table.
constexpr pv_status kNeedWide = static_cast<pv_status>(-15);

struct LaunchCfg {
  cudaStream_t stream;
  int sm_count;
  int block;      // threads per CTA
  int grid_mult;  // 0: fill the GPU once (occupancy-derived)
  int U;          // items per thread per trip
  bool pred;      // predicated
  bool compact;   // compacted: survivors of the first operation queued per warp (grouped pipelines)
  bool chunk;     // chunked access
  bool staged;    // TMA-staged access (grouped predicated pipelines)
  int compact_probes;  // compacted: probes of the first stage (1 or 2)
  int first_items;     // compacted: items a lane takes through the first stage per trip (1 or 2)
  int* launches;  // incremented per kernel launch
  // optional per-kernel timing: called right before and right after a launch
  void (*mark)(void* timer, cudaStream_t s);
  void* timer;
};

// Programmatic dependent launch (sm_90+): a kernel launched with
// pdl_launch() may start while its predecessor on the stream finishes; it
// must call pdl_wait() before touching anything the predecessor wrote
// (griddepcontrol.wait returns once the predecessor grid has completed and
// its memory is visible).  pdl_launch_dependents() lets the dependent grid
// be scheduled before this grid ends.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" :::); }

template <class... KArgs, class... Args>
inline cudaError_t pdl_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

inline void kmark(const LaunchCfg& c) {
  if (c.mark) c.mark(c.timer, c.stream);
}

// Ungrouped AGGREGATE buffers: raw accumulators (zero between runs) and the
// decoded result row.
struct AggOut {
  unsigned long long* acc;  // [n_aggs + 1], last = hidden row count
  int64_t* result;          // [n_aggs]
  unsigned int* done;       // block ticket (zero between runs)
};

// PROJECT buffers.
struct ProjOut {
  void* col[PV_MAX_PROJ];       // typed output columns
  int64_t capacity;             // rows
  unsigned long long* cursor;   // single pass: write cursor (zero between runs)
  int64_t* count;               // rows written (min(total, capacity))
  unsigned int* done;           // single pass: block ticket
  int64_t* tile_count;          // multi pass: matches per tile
  int64_t* tile_offset;         // multi pass: exclusive prefix of tile_count
  int64_t n_tiles;
};

// Grouped aggregation description shared by the group kernels and the host.
struct GroupDesc {
  int n_keys;
  int n_aggs;
  int coded;                     // keys are mixed-radix codes over the part domains (three parts, or two
                                 // parts one of which is 64 bits wide); else packed (one part, or two
                                 // 32-bit halves)
  int count_word;                // slot word holding the group's row count: the first
                                 // COUNT aggregate, else word n_aggs (hidden count)
  int32_t func[PV_MAX_AGGS];
  int key64[PV_MAX_KEYS];        // key part is a 64-bit source (1 part only)
  int64_t key_min[PV_MAX_KEYS];  // perfect array: domain of each part
  int64_t key_span[PV_MAX_KEYS];
};

// Perfect tables of at most kReplicatedSlots slots get kReplicas copies.
constexpr int64_t kReplicatedSlots = 64;
constexpr int kReplicas = 16;

// Grouped aggregation table + extraction buffers (owned by a result).
struct GroupOut {
  // Global table.  Slot s: keys[s] (EMPTY = ~0; perfect: unused) and
  // vals[s * stride + a] for a < n_aggs, vals[s * stride + n_aggs] = row count.
  unsigned long long* keys;
  unsigned long long* vals;
  int64_t cap;        // slots (power of two for hashed tables; domain for perfect)
  int log2cap;
  int stride;         // words per slot in vals
  int ht;             // pv_ht_kind
  int hash;           // pv_hash_fn
  int cuckoo_k;
  int max_evictions;
  uint64_t seed[4];
  int local_slots;    // LOCAL strategy: slots of the per-CTA shared-memory table
  int warp_agg;       // atomic sinks: combine a warp's rows of equal key before updating
  // Perfect tables of few slots are replicated: CTA b adds into replica
  // b % replicas (vals + replica * rep_stride), which spreads the atomics of
  // many CTAs on the same few words; extraction folds the replicas.
  int cluster_log2;   // cluster tables: log2 of the CTAs per cluster (the table's partitions)
  int replicas;       // 1 for hashed tables
  int64_t rep_stride; // words between replicas: (cap + 1) * stride
  // Thread-private tables with 32-bit fields: a row whose field values are
  // all at most narrow_limit = (2^32 - 1) / (rows a thread visits) updates its
  // thread's table; any other row updates the global table directly.  The
  // launch sets narrow_limit.  narrow_max: the largest value of the columns the
  // narrow aggregates sum, from column statistics (all ones when one can be
  // negative); with narrow_check set, a launch whose narrow_limit is below it
  // returns kNeedWide instead, and the wide layout runs.
  uint64_t narrow_limit;
  uint64_t narrow_max;
  int narrow_check;
  // Extraction (dense result columns, int64): out[c * out_cap + row].
  int64_t* out;
  int64_t out_cap;
  unsigned long long* out_count;
};

// A pipeline program as data, for the generic (interpreted) kernels of
// k_generic.cu: the same canonical slots, predicate ranges (KParams lo/hi)
// and probes as the compiled shapes, with the key parts, aggregate terms and
// projected values read from these tables at run time instead of being
// compiled in.
struct GRef {
  int32_t kind;  // PV_REF_COL: fact slot a; PV_REF_PAYLOAD: payload b of probe a
  int32_t a, b;
};
struct GTerm {
  int32_t kind;  // pv_term_kind
  GRef x;
  int64_t c;
};
struct GAgg {
  int32_t func;  // pv_func
  int32_t n_terms;
  GTerm t[PV_MAX_TERMS];
};
struct GenSpec {
  int32_t n_slots, n_preds, n_probes, n_keys, n_aggs, n_proj;
  int32_t slot_type[kMaxSlots];
  int32_t pred_slot[PV_MAX_PREDS];   // predicate i: kp.lo[i] <= slot value <= kp.hi[i]
  int32_t probe_slot[PV_MAX_PROBES]; // probe j: key column slot, table kp.probe[j]
  GRef key[PV_MAX_KEYS];
  GAgg agg[PV_MAX_AGGS];
  GRef proj[PV_MAX_PROJ];
  int32_t proj_type[PV_MAX_PROJ];
  // Probed tables with several payload columns hold the build row in their
  // slots; payload b of probe j is then gathered from pay_col[j][b].
  int32_t indexed[PV_MAX_PROBES];
  const void* pay_col[PV_MAX_PROBES][PV_MAX_PAYLOAD];
  int32_t pay_type[PV_MAX_PROBES][PV_MAX_PAYLOAD];
  // Row count read on the device when the kernel starts (the fact columns are
  // the result of an earlier pipeline), at most KParams::n_rows; null: n_rows.
  const unsigned long long* n_dyn;
};

struct ShapeEntry {
  std::string sig;
  int mode;
  // Launchers return PV_OK or PV_ERR_UNSUPPORTED (no instantiation for the variant).
  pv_status (*aggregate)(const LaunchCfg&, const KParams&, const AggOut&);
  pv_status (*project)(const LaunchCfg&, const KParams&, const ProjOut&, int exec);
  pv_status (*grouped)(const LaunchCfg&, const KParams&, const GroupDesc&, const GroupOut&,
                       const pv_variant&);
};

void register_shape(const ShapeEntry& e);
const ShapeEntry* find_shape(const std::string& sig);
void register_scan_shapes();
void register_group_shapes();

// Generic kernels (k_generic.cu): any pipeline program within the limits of
// pv.h, with the program read from a GenSpec.  Return PV_ERR_UNSUPPORTED for
// the variant axes they do not implement.
pv_status generic_aggregate(const LaunchCfg& c, const KParams& kp, const GenSpec& gs, const AggOut& out);
pv_status generic_project(const LaunchCfg& c, const KParams& kp, const GenSpec& gs, const ProjOut& out, int exec);
pv_status generic_grouped(const LaunchCfg& c, const KParams& kp, const GenSpec& gs, const GroupDesc& gd,
                          const GroupOut& g, const pv_variant& v);
// Exclusive scan of the multi-pass tile counts (k_scan.cu), launched behind
// the count kernel.
pv_status launch_tile_scan(const LaunchCfg& c, const ProjOut& out, int32_t* err);

// Cost-model kernels (k_mlp.cu).
pv_status mlp_forward(cudaStream_t s, int* launches, const float* params, const float* x, const float* mu,
                      const float* sigma, int B, int F, float* y, float* act);
pv_status mlp_backward(cudaStream_t s, int* launches, const float* params, const float* x, const float* mu,
                       const float* sigma, const float* act, const float* y, const float* t, int B, int F,
                       float* dz, float* grad, float* loss);
pv_status mlp_adam(cudaStream_t s, int* launches, float* p, const float* g, float* m, float* v, int64_t n, float lr,
                   float b1, float b2, float eps, int step);

// Grid size: grid_mult * SMs, or the number of CTAs resident at once; never
// more CTAs than there is work for (items_per_cta items each).
int grid_for(const LaunchCfg& c, const void* kernel, size_t smem, int64_t work_items,
             int64_t items_per_cta);

}  // namespace pv
