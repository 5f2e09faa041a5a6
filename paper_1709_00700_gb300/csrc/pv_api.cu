// C-ABI layer of libpv: contexts, column registration, canonicalisation of a
// pipeline program into a compiled shape, result buffers, the pv_sync
// watchdog, CUDA-graph capture and measurement helpers.
#include <algorithm>
#include <chrono>
#include <climits>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pv_internal.h"
#include "pv_build.h"

using namespace pv;

// ---------------------------------------------------------------------------
// Registry of compiled shapes
// ---------------------------------------------------------------------------
namespace pv {
static std::unordered_map<std::string, ShapeEntry>& registry() {
  static std::unordered_map<std::string, ShapeEntry> r;
  return r;
}
void register_shape(const ShapeEntry& e) { registry()[e.sig] = e; }
const ShapeEntry* find_shape(const std::string& sig) {
  auto it = registry().find(sig);
  return it == registry().end() ? nullptr : &it->second;
}
static void init_registry() {
  static std::once_flag once;
  std::call_once(once, [] {
    register_scan_shapes();
    register_group_shapes();
  });
}

int grid_for(const LaunchCfg& c, const void* kernel, size_t smem, int64_t work_items, int64_t items_per_cta) {
  // Per (kernel, block, smem): CTAs resident per SM, 0 if one CTA does not fit
  // (too many registers or too much shared memory for this block size).
  static std::mutex mu;
  static std::map<std::tuple<const void*, int, size_t>, int> cache;
  int nb = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_tuple(kernel, c.block, smem);
    auto it = cache.find(key);
    if (it != cache.end()) {
      nb = it->second;
    } else {
      cudaFuncAttributes fa{};
      if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess || fa.maxThreadsPerBlock < c.block) nb = 0;
      else if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, c.block, smem) != cudaSuccess) nb = 0;
      cache[key] = nb;
    }
  }
  if (nb <= 0) return 0;
  int64_t g = c.grid_mult > 0 ? static_cast<int64_t>(c.grid_mult) * c.sm_count
                              : static_cast<int64_t>(nb) * c.sm_count;
  int64_t need = items_per_cta > 0 ? (work_items + items_per_cta - 1) / items_per_cta : 1;
  if (need < 1) need = 1;
  g = std::min(g, need);
  return static_cast<int>(std::min<int64_t>(g, INT_MAX));
}
}  // namespace pv

// ---------------------------------------------------------------------------
// Context state
// ---------------------------------------------------------------------------
struct Column {
  std::string table, name;
  int type;
  const void* ptr;
  int64_t n_rows;                          // rows; for a result column its capacity
  bool has_stats = false;
  int64_t vmin = 0, vmax = 0;
  const unsigned long long* n_dyn = nullptr;  // result column: row count on the device
  int32_t src_res = 0;                     // result column: the result it belongs to
};

struct Canon {
  std::string sig;
  int mode = 0;
  KParams kp{};
  int64_t n_rows = 0;
  int n_slots = 0;
  int slot_type[kMaxSlots]{};
  pv_col slot_col[kMaxSlots]{};
  int n_aggs = 0;
  int32_t agg_func[PV_MAX_AGGS]{};
  int n_proj = 0;
  int proj_type[PV_MAX_PROJ]{};
  int n_keys = 0;
  int key_type[PV_MAX_KEYS]{};       // pv_type of the key part source
  int key_src_kind[PV_MAX_KEYS]{};   // PV_REF_COL or PV_REF_PAYLOAD
  int key_src[PV_MAX_KEYS][2]{};     // column handle | (probe, payload)
  int64_t pay_min[PV_MAX_PROBES][PV_MAX_PAYLOAD]{};  // payload statistics of each probed table
  int64_t pay_max[PV_MAX_PROBES][PV_MAX_PAYLOAD]{};
  int64_t capacity_hint = 0;
  GenSpec gs{};               // the program as data, for the generic kernels
  bool generic_only = false;  // no compiled shape can run it (see canonicalize)
};

struct Result {
  Canon canon;
  pv_variant var{};
  const ShapeEntry* entry = nullptr;
  bool generic = false;  // runs on the generic kernels
  std::vector<void*> mem;
  AggOut agg{};
  ProjOut proj{};
  GroupDesc gd{};
  GroupOut grp{};
  int n_cols = 0;
  int col_type[PV_MAX_KEYS + PV_MAX_AGGS]{};
  int64_t rows_cached = -1;
};

struct Graph {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
};

struct pv_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  void* (*alloc)(size_t, void*) = nullptr;
  void (*free_)(void*, void*) = nullptr;
  void* user = nullptr;
  std::string err;
  int sm_count = 0;
  int64_t l2_bytes = 0;
  int32_t* d_err = nullptr;
  int32_t* h_err = nullptr;   // pinned
  cudaEvent_t ev = nullptr;
  int64_t timeout_ms = 60000;
  int32_t next = 1;
  std::map<int32_t, Column> cols;
  std::map<int32_t, std::unique_ptr<BuildTable>> tables;
  std::map<int32_t, std::unique_ptr<Result>> results;
  std::map<int32_t, Graph> graphs;
  void* flush_buf = nullptr;
  int64_t flush_bytes = 0;
  int launches = 0;
  bool capturing = false;
  bool ktime = false;
  std::vector<cudaEvent_t> kev;  // timing events, two per kernel
  int kev_used = 0;
  int64_t* d_stats = nullptr;
  int64_t* d_one = nullptr;   // device int64 holding 1 (the row count of ungrouped results)
};

namespace {

pv_status fail(pv_ctx* c, pv_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

pv_status cuda_fail(pv_ctx* c, cudaError_t e, const char* what) {
  return fail(c, PV_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define PV_CUDA(ctx, call)                                \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

void* dalloc(pv_ctx* c, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~size_t(255);
  if (c->alloc) return c->alloc(bytes, c->user);
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, c->stream) != cudaSuccess) return nullptr;
  return p;
}

void dfree(pv_ctx* c, void* p) {
  if (!p) return;
  if (c->free_) c->free_(p, c->user);
  else cudaFreeAsync(p, c->stream);
}

int type_size(int t) { return t == PV_I32 ? 4 : t == PV_I64 ? 8 : 1; }

bool pred_range(const pv_pred& p, int64_t& lo, int64_t& hi) {
  switch (p.op) {
    case PV_LT:
      if (p.c0 == INT64_MIN) { lo = 1; hi = 0; } else { lo = INT64_MIN; hi = p.c0 - 1; }
      return true;
    case PV_LE: lo = INT64_MIN; hi = p.c0; return true;
    case PV_GT:
      if (p.c0 == INT64_MAX) { lo = 1; hi = 0; } else { lo = p.c0 + 1; hi = INT64_MAX; }
      return true;
    case PV_GE: lo = p.c0; hi = INT64_MAX; return true;
    case PV_EQ: lo = hi = p.c0; return true;
    case PV_BETWEEN: lo = p.c0; hi = p.c1; return true;
  }
  return false;
}

void clamp_range(int type, int64_t& lo, int64_t& hi) {
  int64_t tmin = type == PV_I32 ? INT32_MIN : type == PV_U8 ? 0 : INT64_MIN;
  int64_t tmax = type == PV_I32 ? INT32_MAX : type == PV_U8 ? 255 : INT64_MAX;
  if (lo > hi) { lo = 1; hi = 0; return; }
  lo = std::max(lo, tmin);
  hi = std::min(hi, tmax);
  if (lo > hi) { lo = 1; hi = 0; }
}

}  // namespace

// Canonicalises a pipeline spec: assigns slots to the fact columns in order of
// first use (predicates, probe keys, group keys, aggregate terms, projected
// columns), merges predicates on one column into one range, writes the shape
// signature the compiled shapes are registered under, and the same program as
// data (GenSpec) for the generic kernels.  Parts no compiled shape takes
// (int64 probe keys, constant terms over payloads, two-part keys with a 64-bit
// part, tables with several payload columns, result columns) mark the
// program generic_only instead of failing.
static pv_status canonicalize(pv_ctx* c, const pv_pipeline_spec* s, Canon& k) {
  if (!s) return fail(c, PV_ERR_INVALID_ARG, "null spec");
  if (s->n_preds < 0 || s->n_preds > PV_MAX_PREDS || s->n_probes < 0 || s->n_probes > PV_MAX_PROBES ||
      s->n_keys < 0 || s->n_keys > PV_MAX_KEYS || s->n_aggs < 0 || s->n_aggs > PV_MAX_AGGS ||
      s->n_proj < 0 || s->n_proj > PV_MAX_PROJ)
    return fail(c, PV_ERR_INVALID_ARG, "spec count out of range");
  if (s->n_proj > 0 && (s->n_aggs > 0 || s->n_keys > 0))
    return fail(c, PV_ERR_INVALID_ARG, "a pipeline ends in PROJECT or in an aggregation, not both");
  if (s->n_proj == 0 && s->n_aggs == 0) return fail(c, PV_ERR_INVALID_ARG, "pipeline has no sink");
  k = Canon{};
  k.mode = s->n_proj > 0 ? MODE_PROJECT : s->n_keys > 0 ? MODE_GROUPED : MODE_AGGREGATE;
  k.n_rows = -1;
  k.capacity_hint = s->capacity_hint;
  GenSpec& gs = k.gs;
  std::string err;
  bool first_col = true;
  auto col_of = [&](pv_col h) -> const Column* {
    auto it = c->cols.find(h);
    return it == c->cols.end() ? nullptr : &it->second;
  };
  auto slot = [&](pv_col h) -> int {
    const Column* col = col_of(h);
    if (!col) { err = "unknown column handle " + std::to_string(h); return -1; }
    if (first_col) {
      k.n_rows = col->n_rows;
      gs.n_dyn = col->n_dyn;
      first_col = false;
    } else if (k.n_rows != col->n_rows || gs.n_dyn != col->n_dyn) {
      err = "fact columns differ in row count";
      return -1;
    }
    for (int i = 0; i < k.n_slots; ++i) if (k.slot_col[i] == h) return i;
    if (k.n_slots == kMaxSlots) { err = "more than 8 distinct fact columns"; return -2; }
    k.slot_col[k.n_slots] = h;
    k.slot_type[k.n_slots] = col->type;
    gs.slot_type[k.n_slots] = col->type;
    k.kp.col[k.n_slots] = col->ptr;
    return k.n_slots++;
  };
  auto bad = [&](int r) { return fail(c, r == -2 ? PV_ERR_UNSUPPORTED : PV_ERR_INVALID_ARG, err); };

  // FILTER: one closed range per column.
  std::vector<std::pair<int, std::pair<int64_t, int64_t>>> ranges;
  for (int i = 0; i < s->n_preds; ++i) {
    int sl = slot(s->preds[i].col);
    if (sl < 0) return bad(sl);
    int64_t lo, hi;
    if (!pred_range(s->preds[i], lo, hi)) return fail(c, PV_ERR_INVALID_ARG, "bad predicate op");
    bool merged = false;
    for (auto& r : ranges)
      if (r.first == sl) {
        r.second.first = std::max(r.second.first, lo);
        r.second.second = std::min(r.second.second, hi);
        merged = true;
      }
    if (!merged) ranges.push_back({sl, {lo, hi}});
  }
  std::string sw = "|W:";
  gs.n_preds = static_cast<int32_t>(ranges.size());
  for (size_t j = 0; j < ranges.size(); ++j) {
    int64_t lo = ranges[j].second.first, hi = ranges[j].second.second;
    clamp_range(k.slot_type[ranges[j].first], lo, hi);
    k.kp.lo[j] = lo;
    k.kp.hi[j] = hi;
    gs.pred_slot[j] = ranges[j].first;
    sw += std::to_string(ranges[j].first) + ",";
  }
  // HASH_PROBE
  std::string sj = "|J:";
  std::vector<const BuildTable*> probe_tab;
  gs.n_probes = s->n_probes;
  for (int j = 0; j < s->n_probes; ++j) {
    auto it = c->tables.find(s->probes[j].ht);
    if (it == c->tables.end()) return fail(c, PV_ERR_INVALID_ARG, "unknown hash table handle");
    int sl = slot(s->probes[j].fk);
    if (sl < 0) return bad(sl);
    if (k.slot_type[sl] == PV_I64) k.generic_only = true;  // int64 probe keys
    const BuildTable& bt = *it->second;
    k.kp.probe[j] = bt.ht;
    for (int b = 0; b < PV_MAX_PAYLOAD; ++b) {
      k.pay_min[j][b] = b < bt.n_payload ? bt.pay_min[b] : 0;
      k.pay_max[j][b] = b < bt.n_payload ? bt.pay_max[b] : -1;
      gs.pay_col[j][b] = b < bt.n_payload ? bt.pay_col[b] : nullptr;
      gs.pay_type[j][b] = b < bt.n_payload ? bt.pay_type[b] : PV_I32;
    }
    gs.indexed[j] = bt.indexed ? 1 : 0;
    if (bt.indexed) k.generic_only = true;  // payloads gathered by build row
    gs.probe_slot[j] = sl;
    probe_tab.push_back(&bt);
    sj += std::to_string(sl) + ",";
  }
  // A value reference: its signature text, its type, its GenSpec form.
  auto ref_sig = [&](const pv_ref& r, std::string& out, int* type, GRef* g) -> int {
    if (r.kind == PV_REF_COL) {
      int sl = slot(r.a);
      if (sl < 0) return sl;
      out += "x" + std::to_string(sl);
      if (type) *type = k.slot_type[sl];
      if (g) *g = GRef{PV_REF_COL, sl, 0};
      return 0;
    }
    if (r.kind == PV_REF_PAYLOAD) {
      if (r.a < 0 || r.a >= s->n_probes || r.b < 0 || r.b >= probe_tab[r.a]->n_payload) {
        err = "bad payload reference";
        return -1;
      }
      out += "p" + std::to_string(r.a) + "." + std::to_string(r.b);
      if (type) *type = PV_I32;
      if (g) *g = GRef{PV_REF_PAYLOAD, r.a, r.b};
      return 0;
    }
    err = "bad reference kind";
    return -1;
  };
  // HASH_AGGREGATE keys
  std::string sk = "|K:";
  k.n_keys = s->n_keys;
  gs.n_keys = s->n_keys;
  for (int i = 0; i < s->n_keys; ++i) {
    int r = ref_sig(s->keys[i], sk, &k.key_type[i], &gs.key[i]);
    if (r < 0) return bad(r);
    sk += ",";
    k.key_src_kind[i] = s->keys[i].kind;
    k.key_src[i][0] = s->keys[i].a;
    k.key_src[i][1] = s->keys[i].b;
  }
  if (s->n_keys == 2 && (k.key_type[0] == PV_I64 || k.key_type[1] == PV_I64))
    k.generic_only = true;  // a two-part key with a 64-bit part is coded in mixed radix
  // Aggregates and ARITHMETIC terms
  std::string sa = "|A:";
  int nconst = 0;
  k.n_aggs = s->n_aggs;
  gs.n_aggs = s->n_aggs;
  for (int i = 0; i < s->n_aggs; ++i) {
    const pv_agg& a = s->aggs[i];
    if (a.func < PV_SUM || a.func > PV_MAX) return fail(c, PV_ERR_INVALID_ARG, "bad aggregate function");
    k.agg_func[i] = a.func;
    gs.agg[i].func = a.func;
    gs.agg[i].n_terms = 0;
    if (a.func == PV_COUNT) { sa += "N,"; continue; }
    if (a.n_terms < 1 || a.n_terms > PV_MAX_TERMS) return fail(c, PV_ERR_INVALID_ARG, "aggregate needs 1..3 terms");
    gs.agg[i].n_terms = a.n_terms;
    sa += a.func == PV_SUM ? "S(" : a.func == PV_MIN ? "m(" : "M(";
    for (int t = 0; t < a.n_terms; ++t) {
      const pv_term& tm = a.terms[t];
      GTerm& gt = gs.agg[i].t[t];
      gt.kind = tm.kind;
      gt.c = tm.kind == PV_TERM_X ? 0 : tm.c;
      if (tm.kind == PV_TERM_X) {
        int r = ref_sig(tm.x, sa, nullptr, &gt.x);
        if (r < 0) return bad(r);
      } else if (tm.kind == PV_TERM_X_PLUS_C || tm.kind == PV_TERM_C_MINUS_X) {
        std::string ignore;
        int r = ref_sig(tm.x, ignore, nullptr, &gt.x);
        if (r < 0) return bad(r);
        if (tm.x.kind != PV_REF_COL) {
          k.generic_only = true;  // constant terms over payloads
          sa += "?";
        } else if (nconst < kMaxConsts) {
          sa += (tm.kind == PV_TERM_X_PLUS_C ? "xpc" : "cmx") + std::to_string(gt.x.a) + "#" + std::to_string(nconst);
          k.kp.c[nconst++] = tm.c;
        }
      } else {
        return fail(c, PV_ERR_INVALID_ARG, "bad term kind");
      }
      sa += "*";
    }
    sa += "),";
  }
  // PROJECT
  std::string sp = "|P:";
  k.n_proj = s->n_proj;
  gs.n_proj = s->n_proj;
  for (int i = 0; i < s->n_proj; ++i) {
    const pv_ref& r = s->proj[i];
    if (r.kind == PV_REF_PAYLOAD) {  // int32 payload b of probe a
      if (r.a < 0 || r.a >= s->n_probes || r.b < 0 || r.b >= probe_tab[r.a]->n_payload)
        return fail(c, PV_ERR_INVALID_ARG, "bad payload reference");
      sp += "p" + std::to_string(r.a) + (r.b ? "." + std::to_string(r.b) : std::string()) + ",";
      gs.proj[i] = GRef{PV_REF_PAYLOAD, r.a, r.b};
      k.proj_type[i] = PV_I32;
      gs.proj_type[i] = PV_I32;
      continue;
    }
    if (r.kind != PV_REF_COL) return fail(c, PV_ERR_INVALID_ARG, "bad projection reference");
    int sl = slot(r.a);
    if (sl < 0) return bad(sl);
    sp += std::to_string(sl) + ",";
    gs.proj[i] = GRef{PV_REF_COL, sl, 0};
    k.proj_type[i] = k.slot_type[sl];
    gs.proj_type[i] = k.slot_type[sl];
  }
  if (k.n_rows < 0) return fail(c, PV_ERR_INVALID_ARG, "pipeline references no fact column");
  if (gs.n_dyn != nullptr) k.generic_only = true;  // the row count is known on the device only
  gs.n_slots = k.n_slots;
  std::string sc = "C:";
  for (int i = 0; i < k.n_slots; ++i)
    sc += k.slot_type[i] == PV_I32 ? "i32," : k.slot_type[i] == PV_I64 ? "i64," : "u8,";
  k.sig = sc + sw + sj + sk + sa + sp;
  k.kp.n_rows = k.n_rows;
  k.kp.n_items = (k.n_rows + 3) / 4;
  k.kp.err = c->d_err;
  return PV_OK;
}

static void ktimer_mark(void* t, cudaStream_t s) {
  pv_ctx* c = static_cast<pv_ctx*>(t);
  if (c->kev_used >= static_cast<int>(c->kev.size())) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    c->kev.push_back(e);
  }
  cudaEventRecord(c->kev[c->kev_used++], s);
}

static pv_status resolve_launch(pv_ctx* c, const pv_variant& v, LaunchCfg& L) {
  L.stream = c->stream;
  L.sm_count = c->sm_count;
  L.block = v.block ? v.block : 256;
  if (L.block < 64 || L.block > 1024 || L.block % 32) return fail(c, PV_ERR_INVALID_ARG, "block must be 64..1024, multiple of 32");
  L.grid_mult = v.grid_mult;
  if (L.grid_mult < 0) return fail(c, PV_ERR_INVALID_ARG, "grid_mult < 0");
  L.U = v.items_per_thread ? v.items_per_thread : 2;
  if (L.U != 1 && L.U != 2 && L.U != 4) return fail(c, PV_ERR_INVALID_ARG, "items_per_thread must be 1, 2 or 4");
  if (v.pred != PV_BRANCH && v.pred != PV_PREDICATED && v.pred != PV_COMPACTED)
    return fail(c, PV_ERR_INVALID_ARG, "bad pred mode");
  if (v.access != PV_GRID_STRIDE && v.access != PV_CHUNKED && v.access != PV_STAGED)
    return fail(c, PV_ERR_INVALID_ARG, "bad access");
  if (v.exec != PV_EXEC_SINGLE_PASS && v.exec != PV_EXEC_MULTI_PASS) return fail(c, PV_ERR_INVALID_ARG, "bad exec");
  if (v.prefetch < 0 || v.prefetch > 16) return fail(c, PV_ERR_INVALID_ARG, "prefetch must be 0..16 trips");
  if (v.warp_agg != 0 && v.warp_agg != 1) return fail(c, PV_ERR_INVALID_ARG, "warp_agg must be 0 or 1");
  L.pred = v.pred == PV_PREDICATED;
  L.compact = v.pred == PV_COMPACTED;
  L.chunk = v.access == PV_CHUNKED;
  L.staged = v.access == PV_STAGED;
  if (v.compact_probes < 0 || v.compact_probes > 2) return fail(c, PV_ERR_INVALID_ARG, "compact_probes must be 0..2");
  L.compact_probes = v.compact_probes ? v.compact_probes : 1;
  if (L.compact_probes != 1 && !L.compact) return fail(c, PV_ERR_INVALID_ARG, "compact_probes needs pred = compacted");
  if (v.first_items < 0 || v.first_items > 2) return fail(c, PV_ERR_INVALID_ARG, "first_items must be 0..2");
  L.first_items = v.first_items ? v.first_items : 1;
  if (L.first_items != 1 && !L.compact) return fail(c, PV_ERR_INVALID_ARG, "first_items needs pred = compacted");
  L.launches = &c->launches;
  if (c->ktime && !c->capturing) {
    L.mark = ktimer_mark;
    L.timer = c;
  }
  return PV_OK;
}

// Kernels of this translation unit: column statistics, L2 flush, watchdog spin.
template <class T>
__global__ void k_minmax(const T* p, int64_t n, const unsigned long long* n_dyn, unsigned long long* out) {
  if (n_dyn != nullptr) {
    const unsigned long long d = __ldcg(n_dyn);
    n = d < static_cast<unsigned long long>(n) ? static_cast<int64_t>(d) : n;
  }
  uint64_t mx = 0, mn = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = static_cast<int64_t>(p[i]);
    const uint64_t cmax = max_code(v), cmin = min_code(v);
    mx = cmax > mx ? cmax : mx;
    mn = cmin > mn ? cmin : mn;
  }
  mx = warp_reduce<PV_MAX>(mx);
  mn = warp_reduce<PV_MAX>(mn);
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out, mx);
    atomicMax(out + 1, mn);
  }
}

__global__ void k_flush(uint4* p, int64_t n, uint32_t salt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = make_uint4(salt, (uint32_t)i, salt ^ 0x9e3779b9u, (uint32_t)(i >> 32));
}

// Drops the flush buffer's lines from L2 without writing them back, so the
// next kernel starts on a cold and clean L2 instead of paying for the flush's
// write-backs.  The buffer's contents become undefined, which is fine.
__global__ void k_discard(char* p, int64_t bytes) {
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) * 128; i + 128 <= bytes;
       i += (int64_t)gridDim.x * blockDim.x * 128)
    asm volatile("discard.global.L2 [%0], 128;" ::"l"(p + i) : "memory");
}

// Random-slot atomic throughput (measurement support).  Update u adds 1 to
// each of the `words` 64-bit words of slot floor(fmix64(u ^ seed) * slots /
// 2^64) with atomicAdd: the access pattern of a global aggregation table whose
// groups are spread uniformly.
__global__ void k_atomic_rand(unsigned long long* t, int64_t slots, int words, int64_t n, uint64_t seed) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t s = __umul64hi(fmix64(static_cast<uint64_t>(u) ^ seed), static_cast<uint64_t>(slots));
    unsigned long long* p = t + s * static_cast<uint64_t>(words);
    for (int w = 0; w < words; ++w) atomicAdd(p + w, 1ull);
  }
}

__global__ void k_spin(int64_t ns) {
  uint64_t t0, t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  // bounded: stops after ns of GPU time or ns / 8 + 2^20 polls, whichever first
  const uint64_t polls = static_cast<uint64_t>(ns) / 8 + (1ull << 20);
  for (uint64_t it = 0; it < polls; ++it) {
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 >= static_cast<uint64_t>(ns)) break;
    __nanosleep(1000);
  }
}

static pv_status wait_stream(pv_ctx* c) {
  PV_CUDA(c, cudaEventRecord(c->ev, c->stream));
  auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t e = cudaEventQuery(c->ev);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) return cuda_fail(c, e, "kernel execution");
    auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count();
    if (ms > c->timeout_ms) return fail(c, PV_ERR_TIMEOUT, "pv_sync watchdog expired after " + std::to_string(ms) + " ms");
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  return PV_OK;
}

static const char* err_name(int32_t e) {
  switch (e) {
    case PV_ERR_HT_FULL: return "hash table full";
    case PV_ERR_CUCKOO_CYCLE: return "cuckoo eviction chain exceeded its bound";
    case PV_ERR_KEY_OUT_OF_RANGE: return "key outside the perfect-array domain";
    case PV_ERR_DUP_BUILD_KEY: return "duplicate build key";
    case PV_ERR_OUTPUT_OVERFLOW: return "projection output capacity exceeded";
  }
  return "device error";
}

static pv_status sync_and_check(pv_ctx* c) {
  if (c->capturing) return fail(c, PV_ERR_INVALID_ARG, "cannot sync while capturing a graph");
  pv_status s = wait_stream(c);
  if (s != PV_OK) return s;
  PV_CUDA(c, cudaMemcpyAsync(c->h_err, c->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  PV_CUDA(c, cudaStreamSynchronize(c->stream));
  const int32_t e = *c->h_err;
  if (e != 0) {
    PV_CUDA(c, cudaMemsetAsync(c->d_err, 0, sizeof(int32_t), c->stream));
    PV_CUDA(c, cudaStreamSynchronize(c->stream));
    return fail(c, e, err_name(e));
  }
  return PV_OK;
}

// ---------------------------------------------------------------------------
// Result allocation and launch
// ---------------------------------------------------------------------------
static pv_status column_stats(pv_ctx* c, pv_col h, int64_t* mn, int64_t* mx) {
  auto it = c->cols.find(h);
  if (it == c->cols.end()) return fail(c, PV_ERR_INVALID_ARG, "unknown column handle");
  Column& col = it->second;
  if (!col.has_stats) {
    if (c->capturing) return fail(c, PV_ERR_INVALID_ARG, "column statistics needed while capturing");
    unsigned long long* d = reinterpret_cast<unsigned long long*>(c->d_stats);
    PV_CUDA(c, cudaMemsetAsync(d, 0, 16, c->stream));
    const int grid = std::max(1, std::min<int>(c->sm_count * 4, static_cast<int>((col.n_rows + 255) / 256)));
    if (col.n_rows > 0) {
      const unsigned long long* nd = col.n_dyn;
      if (col.type == PV_I32) k_minmax<<<grid, 256, 0, c->stream>>>(static_cast<const int32_t*>(col.ptr), col.n_rows, nd, d);
      else if (col.type == PV_I64) k_minmax<<<grid, 256, 0, c->stream>>>(static_cast<const int64_t*>(col.ptr), col.n_rows, nd, d);
      else k_minmax<<<grid, 256, 0, c->stream>>>(static_cast<const uint8_t*>(col.ptr), col.n_rows, nd, d);
      PV_CUDA(c, cudaGetLastError());
    }
    unsigned long long hbuf[2] = {0, 0};
    PV_CUDA(c, cudaMemcpyAsync(hbuf, d, 16, cudaMemcpyDeviceToHost, c->stream));
    PV_CUDA(c, cudaStreamSynchronize(c->stream));
    // some row was present: a row's max code and min code are not both 0 (that would need the
    // value to be INT64_MIN and INT64_MAX at once)
    if (col.n_rows > 0 && (hbuf[0] != 0 || hbuf[1] != 0)) {
      col.vmax = decode_max(hbuf[0]);
      col.vmin = decode_min(hbuf[1]);
    } else {
      col.vmin = 0;
      col.vmax = -1;
    }
    col.has_stats = true;
  }
  *mn = col.vmin;
  *mx = col.vmax;
  return PV_OK;
}


static pv_status alloc_result(pv_ctx* c, Result& r) {
  const Canon& k = r.canon;
  auto grab = [&](size_t bytes) -> void* {
    void* p = dalloc(c, bytes);
    if (p) r.mem.push_back(p);
    return p;
  };
  if (k.mode == MODE_AGGREGATE) {
    const size_t words = 2 * static_cast<size_t>(k.n_aggs) + 2;
    char* p = static_cast<char*>(grab(words * 8));
    if (!p) return fail(c, PV_ERR_OOM, "allocator returned NULL");
    PV_CUDA(c, cudaMemsetAsync(p, 0, words * 8, c->stream));
    r.agg.acc = reinterpret_cast<unsigned long long*>(p);
    r.agg.result = reinterpret_cast<int64_t*>(p + (k.n_aggs + 1) * 8);
    r.agg.done = reinterpret_cast<unsigned int*>(p + (2 * k.n_aggs + 1) * 8);
    r.n_cols = k.n_aggs;
    for (int i = 0; i < k.n_aggs; ++i) r.col_type[i] = PV_I64;
    return PV_OK;
  }
  if (k.mode == MODE_PROJECT) {
    int64_t cap = k.capacity_hint > 0 ? k.capacity_hint : k.n_rows;
    r.proj.capacity = cap;
    for (int i = 0; i < k.n_proj; ++i) {
      r.proj.col[i] = grab(static_cast<size_t>(std::max<int64_t>(cap, 1)) * type_size(k.proj_type[i]));
      if (!r.proj.col[i]) return fail(c, PV_ERR_OOM, "allocator returned NULL");
      r.col_type[i] = k.proj_type[i];
    }
    r.n_cols = k.n_proj;
    const int U = r.var.items_per_thread ? r.var.items_per_thread : 2;
    const int block = r.var.block ? r.var.block : 256;
    const int64_t tile_items = static_cast<int64_t>(block) * U;
    r.proj.n_tiles = std::max<int64_t>(1, (k.kp.n_items + tile_items - 1) / tile_items);
    const size_t ctl = 32 + 16 * static_cast<size_t>(r.var.exec == PV_EXEC_MULTI_PASS ? r.proj.n_tiles : 0);
    char* p = static_cast<char*>(grab(ctl));
    if (!p) return fail(c, PV_ERR_OOM, "allocator returned NULL");
    PV_CUDA(c, cudaMemsetAsync(p, 0, ctl, c->stream));
    r.proj.cursor = reinterpret_cast<unsigned long long*>(p);
    r.proj.count = reinterpret_cast<int64_t*>(p + 8);
    r.proj.done = reinterpret_cast<unsigned int*>(p + 16);
    if (r.var.exec == PV_EXEC_MULTI_PASS) {
      r.proj.tile_count = reinterpret_cast<int64_t*>(p + 32);
      r.proj.tile_offset = r.proj.tile_count + r.proj.n_tiles;
    }
    return PV_OK;
  }
  // MODE_GROUPED
  GroupDesc& gd = r.gd;
  gd.n_keys = k.n_keys;
  gd.n_aggs = k.n_aggs;
  gd.count_word = k.n_aggs;
  for (int i = k.n_aggs - 1; i >= 0; --i)
    if (k.agg_func[i] == PV_COUNT) gd.count_word = i;
  for (int i = 0; i < k.n_aggs; ++i) gd.func[i] = k.agg_func[i];
  for (int i = 0; i < k.n_keys; ++i) gd.key64[i] = k.key_type[i] == PV_I64;
  gd.coded = k.n_keys > 2 || (k.n_keys == 2 && (gd.key64[0] || gd.key64[1]));
  // Key domains from column statistics / build payload statistics.
  int64_t domain = 1;
  bool domain_ok = true;
  for (int i = 0; i < k.n_keys; ++i) {
    int64_t mn, mx;
    if (k.key_src_kind[i] == PV_REF_COL) {
      pv_status s = column_stats(c, k.key_src[i][0], &mn, &mx);
      if (s != PV_OK) return s;
    } else {
      mn = k.pay_min[k.key_src[i][0]][k.key_src[i][1]];
      mx = k.pay_max[k.key_src[i][0]][k.key_src[i][1]];
    }
    if (mx < mn) { mn = 0; mx = 0; }  // empty source: any domain works
    gd.key_min[i] = mn;
    const __int128 span = static_cast<__int128>(mx) - mn + 1;
    if (span > (static_cast<__int128>(1) << 40)) { domain_ok = false; gd.key_span[i] = 1; }
    else gd.key_span[i] = static_cast<int64_t>(span);
    if (domain_ok && static_cast<__int128>(domain) * gd.key_span[i] <= (static_cast<__int128>(1) << 40))
      domain *= gd.key_span[i];
    else domain_ok = false;
  }
  if (gd.coded && !domain_ok)
    return fail(c, PV_ERR_UNSUPPORTED, "composite group keys need a key domain of at most 2^40 codes");
  GroupOut& g = r.grp;
  g.ht = r.var.ht;
  g.hash = r.var.hash;
  g.cuckoo_k = r.var.cuckoo_k ? r.var.cuckoo_k : 3;
  if (g.cuckoo_k < 2 || g.cuckoo_k > 4) return fail(c, PV_ERR_INVALID_ARG, "cuckoo_k must be 2..4");
  uint64_t sd = r.var.seed ? r.var.seed : 0x5eed1709ull;
  for (int i = 0; i < 4; ++i) { sd = fmix64(sd + 0x9e3779b97f4a7c15ull); g.seed[i] = sd | 1ull; }
  g.stride = k.n_aggs + 1;
  int64_t expected = k.capacity_hint > 0 ? k.capacity_hint : (domain_ok ? domain : k.n_rows);
  expected = std::max<int64_t>(1, std::min(expected, std::max<int64_t>(k.n_rows, 1)));
  if (g.ht == PV_HT_PERFECT) {
    if (!domain_ok || domain > (int64_t(1) << 28))
      return fail(c, PV_ERR_UNSUPPORTED, "perfect array: key domain larger than 2^28 slots");
    g.cap = domain;
    g.log2cap = 0;
  } else if (g.ht == PV_HT_LINEAR || g.ht == PV_HT_CUCKOO) {
    int l = 1;
    while ((int64_t(1) << l) < 2 * expected) ++l;
    g.log2cap = l;
    g.cap = int64_t(1) << l;
  } else {
    return fail(c, PV_ERR_INVALID_ARG, "bad aggregation table kind");
  }
  g.max_evictions = 32 * std::max(1, g.log2cap);
  g.warp_agg = r.var.warp_agg;
  // largest value a narrow aggregate (SUM of one plain column) adds: decides
  // whether thread-private tables may keep 32-bit fields
  g.narrow_max = 0;
  for (int a = 0; a < k.n_aggs; ++a) {
    const GAgg& ag = k.gs.agg[a];
    if (ag.func != PV_SUM || ag.n_terms != 1 || ag.t[0].kind != PV_TERM_X) continue;
    int64_t lo, hi;
    if (ag.t[0].x.kind == PV_REF_COL) {
      pv_status st = column_stats(c, k.slot_col[ag.t[0].x.a], &lo, &hi);
      if (st != PV_OK) return st;
    } else {
      lo = k.pay_min[ag.t[0].x.a][ag.t[0].x.b];
      hi = k.pay_max[ag.t[0].x.a][ag.t[0].x.b];
    }
    if (hi < lo) continue;  // no rows
    g.narrow_max = lo < 0 ? ~0ull : std::max<uint64_t>(g.narrow_max, static_cast<uint64_t>(hi));
  }
  const int64_t slots = g.cap + 1;  // + side slot for the key equal to EMPTY
  g.replicas = g.ht == PV_HT_PERFECT && g.cap <= kReplicatedSlots ? kReplicas : 1;
  g.rep_stride = slots * g.stride;
  const size_t val_bytes = static_cast<size_t>(slots) * g.stride * 8 * g.replicas;
  g.keys = static_cast<unsigned long long*>(grab(static_cast<size_t>(slots) * 8));
  g.vals = static_cast<unsigned long long*>(grab(val_bytes));
  const int ncol = k.n_keys + k.n_aggs;
  g.out_cap = std::min<int64_t>(slots, std::max<int64_t>(k.n_rows, 1));
  g.out = static_cast<int64_t*>(grab(static_cast<size_t>(g.out_cap) * ncol * 8));
  g.out_count = static_cast<unsigned long long*>(grab(16));
  if (!g.keys || !g.vals || !g.out || !g.out_count) return fail(c, PV_ERR_OOM, "allocator returned NULL");
  // Empty table once at allocation; extraction empties every slot it reads.
  PV_CUDA(c, cudaMemsetAsync(g.keys, 0xFF, static_cast<size_t>(slots) * 8, c->stream));
  PV_CUDA(c, cudaMemsetAsync(g.vals, 0, val_bytes, c->stream));
  PV_CUDA(c, cudaMemsetAsync(g.out_count, 0, 16, c->stream));
  r.n_cols = ncol;
  for (int i = 0; i < ncol; ++i) r.col_type[i] = PV_I64;
  return PV_OK;
}

static pv_status launch_result(pv_ctx* c, Result& r) {
  LaunchCfg L{};
  pv_status s = resolve_launch(c, r.var, L);
  if (s != PV_OK) return s;
  c->launches = 0;
  c->kev_used = 0;
  r.rows_cached = -1;
  Canon& k = r.canon;
  k.kp.prefetch = r.var.prefetch;
  if (L.staged && (r.generic || k.mode != MODE_GROUPED))
    return fail(c, PV_ERR_UNSUPPORTED, "TMA-staged access is compiled for grouped shapes only");
  if (r.generic) {
    if (k.mode == MODE_AGGREGATE) s = generic_aggregate(L, k.kp, k.gs, r.agg);
    else if (k.mode == MODE_PROJECT) s = generic_project(L, k.kp, k.gs, r.proj, r.var.exec);
    else s = generic_grouped(L, k.kp, k.gs, r.gd, r.grp, r.var);
    if (s == PV_ERR_UNSUPPORTED) return fail(c, s, "the generic kernels do not implement this variant");
  } else {
    if (k.mode == MODE_AGGREGATE) s = r.entry->aggregate(L, k.kp, r.agg);
    else if (k.mode == MODE_PROJECT) s = r.entry->project(L, k.kp, r.proj, r.var.exec);
    else s = r.entry->grouped(L, k.kp, r.gd, r.grp, r.var);
  }
  if (s == PV_ERR_UNSUPPORTED) return fail(c, s, "no instantiation of this shape for the variant");
  if (s != PV_OK) return fail(c, s, "kernel launch failed");
  return PV_OK;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

pv_status pv_create(pv_ctx** out, int device, void* stream, void* (*alloc)(size_t, void*),
                    void (*free_)(void*, void*), void* user) {
  if (!out) return PV_ERR_INVALID_ARG;
  *out = nullptr;
  if ((alloc == nullptr) != (free_ == nullptr)) return PV_ERR_INVALID_ARG;
  init_registry();
  auto c = std::make_unique<pv_ctx>();
  c->device = device;
  c->stream = static_cast<cudaStream_t>(stream);
  c->alloc = alloc;
  c->free_ = free_;
  c->user = user;
  if (cudaSetDevice(device) != cudaSuccess) return PV_ERR_CUDA;
  int l2 = 0;
  if (cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return PV_ERR_CUDA;
  if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, device) != cudaSuccess) return PV_ERR_CUDA;
  c->l2_bytes = l2;
  if (cudaEventCreateWithFlags(&c->ev, cudaEventDisableTiming) != cudaSuccess) return PV_ERR_CUDA;
  if (cudaMallocHost(&c->h_err, sizeof(int32_t)) != cudaSuccess) return PV_ERR_CUDA;
  c->d_err = static_cast<int32_t*>(dalloc(c.get(), 256));
  if (!c->d_err) return PV_ERR_OOM;
  c->d_stats = reinterpret_cast<int64_t*>(reinterpret_cast<char*>(c->d_err) + 64);
  c->d_one = reinterpret_cast<int64_t*>(reinterpret_cast<char*>(c->d_err) + 192);
  static const int64_t one = 1;
  if (cudaMemsetAsync(c->d_err, 0, 256, c->stream) != cudaSuccess) return PV_ERR_CUDA;
  if (cudaMemcpyAsync(c->d_one, &one, sizeof(one), cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
    return PV_ERR_CUDA;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return PV_ERR_CUDA;
  *out = c.release();
  return PV_OK;
}

pv_status pv_destroy(pv_ctx* c) {
  if (!c) return PV_ERR_INVALID_ARG;
  cudaStreamSynchronize(c->stream);
  for (auto& kv : c->graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.g) cudaGraphDestroy(kv.second.g);
  }
  for (auto& kv : c->results)
    for (void* p : kv.second->mem) dfree(c, p);
  for (auto& kv : c->tables) dfree(c, kv.second->mem);
  for (cudaEvent_t e : c->kev) cudaEventDestroy(e);
  dfree(c, c->flush_buf);
  dfree(c, c->d_err);
  cudaStreamSynchronize(c->stream);
  if (c->h_err) cudaFreeHost(c->h_err);
  if (c->ev) cudaEventDestroy(c->ev);
  delete c;
  return PV_OK;
}

const char* pv_last_error(const pv_ctx* c) { return c ? c->err.c_str() : "null context"; }

pv_status pv_device_info(pv_ctx* c, int32_t* sm_count, int64_t* l2_bytes) {
  if (!c) return PV_ERR_INVALID_ARG;
  if (sm_count) *sm_count = c->sm_count;
  if (l2_bytes) *l2_bytes = c->l2_bytes;
  return PV_OK;
}

pv_status pv_set_l2_fetch_bytes(pv_ctx* c, int32_t bytes, int32_t* previous) {
  if (!c) return PV_ERR_INVALID_ARG;
  if (bytes != 32 && bytes != 64 && bytes != 128)
    return fail(c, PV_ERR_INVALID_ARG, "L2 fetch bytes must be 32, 64 or 128");
  if (c->capturing) return fail(c, PV_ERR_INVALID_ARG, "pv_set_l2_fetch_bytes cannot be captured");
  PV_CUDA(c, cudaSetDevice(c->device));
  size_t old = 0;
  PV_CUDA(c, cudaDeviceGetLimit(&old, cudaLimitMaxL2FetchGranularity));
  PV_CUDA(c, cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, static_cast<size_t>(bytes)));
  if (previous) *previous = static_cast<int32_t>(old);
  return PV_OK;
}

pv_status pv_register_column(pv_ctx* c, const char* table, const char* name, int32_t type,
                             const void* dev_ptr, int64_t n_rows, pv_col* out) {
  if (!c || !out) return PV_ERR_INVALID_ARG;
  if (type != PV_I32 && type != PV_I64 && type != PV_U8) return fail(c, PV_ERR_INVALID_ARG, "bad column type");
  if (n_rows < 0) return fail(c, PV_ERR_INVALID_ARG, "negative row count");
  if (n_rows > 0 && !dev_ptr) return fail(c, PV_ERR_INVALID_ARG, "null column pointer");
  if (reinterpret_cast<uintptr_t>(dev_ptr) % 16) return fail(c, PV_ERR_INVALID_ARG, "column pointer not 16-byte aligned");
  Column col;
  col.table = table ? table : "";
  col.name = name ? name : "";
  col.type = type;
  col.ptr = dev_ptr;
  col.n_rows = n_rows;
  const int32_t h = c->next++;
  c->cols[h] = col;
  *out = h;
  return PV_OK;
}

pv_status pv_register_result_column(pv_ctx* c, pv_res res, int32_t col, const char* table, const char* name,
                                    pv_col* out) {
  if (!c || !out) return PV_ERR_INVALID_ARG;
  auto it = c->results.find(res);
  if (it == c->results.end()) return fail(c, PV_ERR_INVALID_ARG, "unknown result handle");
  Result& r = *it->second;
  if (col < 0 || col >= r.n_cols) return fail(c, PV_ERR_INVALID_ARG, "column index out of range");
  const Canon& k = r.canon;
  Column nc;
  nc.table = table ? table : "";
  nc.name = name ? name : "";
  nc.type = r.col_type[col];
  nc.src_res = res;
  // Statistics of the column's source: a projected fact column or payload keeps
  // its source's value range, a group-key part its domain; aggregates are
  // computed from the rows when first needed.
  auto inherit = [&](int64_t lo, int64_t hi) {
    nc.has_stats = true;
    nc.vmin = lo;
    nc.vmax = hi;
  };
  if (k.mode == MODE_PROJECT) {
    nc.ptr = r.proj.col[col];
    nc.n_rows = r.proj.capacity;
    nc.n_dyn = reinterpret_cast<const unsigned long long*>(r.proj.count);
    const GRef& g = k.gs.proj[col];
    if (g.kind == PV_REF_PAYLOAD) {
      inherit(k.pay_min[g.a][g.b], k.pay_max[g.a][g.b]);
    } else {
      int64_t lo, hi;
      pv_status st = column_stats(c, k.slot_col[g.a], &lo, &hi);
      if (st != PV_OK) return st;
      inherit(lo, hi);
    }
  } else if (k.mode == MODE_GROUPED) {
    nc.ptr = r.grp.out + static_cast<size_t>(col) * r.grp.out_cap;
    nc.n_rows = r.grp.out_cap;
    nc.n_dyn = r.grp.out_count;
    if (col < k.n_keys) {
      int64_t lo, hi;
      if (k.key_src_kind[col] == PV_REF_COL) {
        pv_status st = column_stats(c, k.key_src[col][0], &lo, &hi);
        if (st != PV_OK) return st;
      } else {
        lo = k.pay_min[k.key_src[col][0]][k.key_src[col][1]];
        hi = k.pay_max[k.key_src[col][0]][k.key_src[col][1]];
      }
      inherit(lo, hi);
    }
  } else {
    nc.ptr = r.agg.result + col;
    nc.n_rows = 1;
  }
  const int32_t h = c->next++;
  c->cols[h] = nc;
  *out = h;
  return PV_OK;
}

pv_status pv_column_stats(pv_ctx* c, pv_col h, int64_t* mn, int64_t* mx) {
  if (!c || !mn || !mx) return PV_ERR_INVALID_ARG;
  return column_stats(c, h, mn, mx);
}

pv_status pv_build_hash_table(pv_ctx* c, const pv_build_spec* spec, const pv_ht_variant* var, pv_ht* out) {
  if (!c || !spec || !var || !out) return PV_ERR_INVALID_ARG;
  if (c->capturing) return fail(c, PV_ERR_INVALID_ARG, "builds are not captured");
  BuildInput in{};
  if (spec->n_preds < 0 || spec->n_preds > PV_MAX_PREDS || spec->n_payload < 0 || spec->n_payload > PV_MAX_PAYLOAD)
    return fail(c, PV_ERR_INVALID_ARG, "build spec count out of range");
  auto get = [&](pv_col h) -> const Column* {
    auto it = c->cols.find(h);
    return it == c->cols.end() ? nullptr : &it->second;
  };
  const Column* key = get(spec->key);
  if (!key) return fail(c, PV_ERR_INVALID_ARG, "unknown key column");
  if (key->type == PV_I64) return fail(c, PV_ERR_UNSUPPORTED, "int64 build keys");
  in.n_rows = key->n_rows;
  in.n_dyn = key->n_dyn;
  in.key = key->ptr;
  in.key_type = key->type;
  in.n_preds = spec->n_preds;
  for (int i = 0; i < spec->n_preds; ++i) {
    const Column* pc = get(spec->preds[i].col);
    if (!pc || pc->n_rows != key->n_rows || pc->n_dyn != key->n_dyn)
      return fail(c, PV_ERR_INVALID_ARG, "bad build predicate column");
    int64_t lo, hi;
    if (!pred_range(spec->preds[i], lo, hi)) return fail(c, PV_ERR_INVALID_ARG, "bad predicate op");
    in.pred_col[i] = pc->ptr;
    in.pred_type[i] = pc->type;
    in.lo[i] = lo;
    in.hi[i] = hi;
  }
  in.n_payload = spec->n_payload;
  for (int i = 0; i < spec->n_payload; ++i) {
    const Column* pc = get(spec->payload[i]);
    if (!pc || pc->n_rows != key->n_rows || pc->n_dyn != key->n_dyn)
      return fail(c, PV_ERR_INVALID_ARG, "bad payload column");
    if (pc->type == PV_I64) return fail(c, PV_ERR_UNSUPPORTED, "int64 payloads");
    in.pay_col[i] = pc->ptr;
    in.pay_type[i] = pc->type;
  }
  int64_t kmin = 0, kmax = -1;
  if (var->kind == PV_HT_PERFECT) {
    pv_status s = column_stats(c, spec->key, &kmin, &kmax);
    if (s != PV_OK) return s;
  }
  auto bt = std::make_unique<BuildTable>();
  BuildEnv env{c->stream, c->sm_count, c->d_err, &c->launches,
               [](size_t b, void* u) { return dalloc(static_cast<pv_ctx*>(u), b); }, c};
  c->launches = 0;
  std::string msg;
  pv_status s = build_table(env, in, *var, kmin, kmax, *bt, msg);
  if (s != PV_OK) {
    if (bt->mem) dfree(c, bt->mem);
    return fail(c, s, msg);
  }
  const int32_t h = c->next++;
  c->tables[h] = std::move(bt);
  *out = h;
  return PV_OK;
}

pv_status pv_rebuild_hash_table(pv_ctx* c, pv_ht h) {
  if (!c) return PV_ERR_INVALID_ARG;
  auto it = c->tables.find(h);
  if (it == c->tables.end()) return fail(c, PV_ERR_INVALID_ARG, "unknown hash table handle");
  BuildEnv env{c->stream, c->sm_count, c->d_err, &c->launches,
               [](size_t b, void* u) { return dalloc(static_cast<pv_ctx*>(u), b); }, c};
  c->launches = 0;
  pv_status s = rebuild_table(env, *it->second);
  return s == PV_OK ? s : fail(c, s, "rebuild launch failed");
}

pv_status pv_run_pipeline(pv_ctx* c, const pv_pipeline_spec* spec, const pv_variant* var, pv_res* out) {
  if (!c || !spec || !var || !out) return PV_ERR_INVALID_ARG;
  if (c->capturing) return fail(c, PV_ERR_INVALID_ARG, "pv_run_pipeline allocates; capture pv_rerun instead");
  auto r = std::make_unique<Result>();
  pv_status s = canonicalize(c, spec, r->canon);
  if (s != PV_OK) return s;
  if (var->interp != 0 && var->interp != 1) return fail(c, PV_ERR_INVALID_ARG, "interp must be 0 or 1");
  r->entry = find_shape(r->canon.sig);
  if (r->entry && r->entry->mode != r->canon.mode) r->entry = nullptr;
  r->generic = var->interp == 1 || r->canon.generic_only || r->entry == nullptr;
  r->var = *var;
  LaunchCfg L{};
  s = resolve_launch(c, r->var, L);
  if (s != PV_OK) return s;
  s = alloc_result(c, *r);
  if (s == PV_OK) s = launch_result(c, *r);
  if (s != PV_OK) {
    for (void* p : r->mem) dfree(c, p);
    return s;
  }
  const int32_t h = c->next++;
  c->results[h] = std::move(r);
  *out = h;
  return PV_OK;
}

pv_status pv_rerun(pv_ctx* c, pv_res h) {
  if (!c) return PV_ERR_INVALID_ARG;
  auto it = c->results.find(h);
  if (it == c->results.end()) return fail(c, PV_ERR_INVALID_ARG, "unknown result handle");
  return launch_result(c, *it->second);
}

pv_status pv_sync(pv_ctx* c) {
  if (!c) return PV_ERR_INVALID_ARG;
  return sync_and_check(c);
}

pv_status pv_set_timeout_ms(pv_ctx* c, int64_t ms) {
  if (!c || ms <= 0) return PV_ERR_INVALID_ARG;
  c->timeout_ms = ms;
  return PV_OK;
}

static pv_status result_rows(pv_ctx* c, Result& r, int64_t* rows) {
  if (r.rows_cached < 0) {
    pv_status s = sync_and_check(c);
    if (s != PV_OK) return s;
    if (r.canon.mode == MODE_AGGREGATE) {
      r.rows_cached = 1;
    } else {
      int64_t n = 0;
      const void* src = r.canon.mode == MODE_PROJECT ? static_cast<const void*>(r.proj.count)
                                                      : static_cast<const void*>(r.grp.out_count);
      PV_CUDA(c, cudaMemcpyAsync(&n, src, 8, cudaMemcpyDeviceToHost, c->stream));
      PV_CUDA(c, cudaStreamSynchronize(c->stream));
      r.rows_cached = n;
    }
  }
  *rows = r.rows_cached;
  return PV_OK;
}

pv_status pv_result_shape(pv_ctx* c, pv_res h, int64_t* n_rows, int32_t* n_cols) {
  if (!c) return PV_ERR_INVALID_ARG;
  auto it = c->results.find(h);
  if (it == c->results.end()) return fail(c, PV_ERR_INVALID_ARG, "unknown result handle");
  int64_t rows;
  pv_status s = result_rows(c, *it->second, &rows);
  if (s != PV_OK) return s;
  if (n_rows) *n_rows = rows;
  if (n_cols) *n_cols = it->second->n_cols;
  return PV_OK;
}

pv_status pv_result_col_type(pv_ctx* c, pv_res h, int32_t col, int32_t* type) {
  if (!c || !type) return PV_ERR_INVALID_ARG;
  auto it = c->results.find(h);
  if (it == c->results.end()) return fail(c, PV_ERR_INVALID_ARG, "unknown result handle");
  if (col < 0 || col >= it->second->n_cols) return fail(c, PV_ERR_INVALID_ARG, "column index out of range");
  *type = it->second->col_type[col];
  return PV_OK;
}

// Whether caller memory p is of the kind a copy expects: device (or
// managed) memory when on_device, else host memory (page-locked or not).  A
// copy-engine copy to host memory given device memory, or the reverse, is
// refused before it is issued.
static bool dst_kind_ok(const void* p, bool on_device) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();  // clear the error the query left: memory CUDA does not know is pageable host memory
    return !on_device;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return on_device ? at.type == cudaMemoryTypeDevice
                   : at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

pv_status pv_fetch_result(pv_ctx* c, pv_res h, int32_t col, void* dst, int64_t dst_rows, int32_t on_device) {
  if (!c) return PV_ERR_INVALID_ARG;
  auto it = c->results.find(h);
  if (it == c->results.end()) return fail(c, PV_ERR_INVALID_ARG, "unknown result handle");
  Result& r = *it->second;
  if (col < 0 || col >= r.n_cols) return fail(c, PV_ERR_INVALID_ARG, "column index out of range");
  int64_t rows;
  pv_status s = result_rows(c, r, &rows);
  if (s != PV_OK) return s;
  if (dst_rows < rows) return fail(c, PV_ERR_INVALID_ARG, "destination too small");
  if (rows == 0) return PV_OK;
  if (!dst) return fail(c, PV_ERR_INVALID_ARG, "null destination");
  if (!dst_kind_ok(dst, on_device))
    return fail(c, PV_ERR_INVALID_ARG, "destination memory is not of the kind on_device states");
  const void* src;
  size_t bytes;
  if (r.canon.mode == MODE_AGGREGATE) {
    src = r.agg.result + col;
    bytes = 8;
  } else if (r.canon.mode == MODE_PROJECT) {
    src = r.proj.col[col];
    bytes = static_cast<size_t>(rows) * type_size(r.col_type[col]);
  } else {
    src = r.grp.out + static_cast<size_t>(col) * r.grp.out_cap;
    bytes = static_cast<size_t>(rows) * 8;
  }
  PV_CUDA(c, cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  PV_CUDA(c, cudaStreamSynchronize(c->stream));
  return PV_OK;
}

pv_status pv_fetch_results(pv_ctx* c, pv_res h, int32_t n_cols, void* const* dst, const int64_t* dst_rows,
                           int32_t on_device) {
  if (!c || !dst || !dst_rows) return PV_ERR_INVALID_ARG;
  auto it = c->results.find(h);
  if (it == c->results.end()) return fail(c, PV_ERR_INVALID_ARG, "unknown result handle");
  Result& r = *it->second;
  if (n_cols != r.n_cols) return fail(c, PV_ERR_INVALID_ARG, "n_cols differs from the result's columns");
  int64_t rows;
  pv_status s = result_rows(c, r, &rows);
  if (s != PV_OK) return s;
  for (int32_t col = 0; col < n_cols; ++col) {
    if (dst_rows[col] < rows) return fail(c, PV_ERR_INVALID_ARG, "destination too small");
    if (rows > 0 && !dst[col]) return fail(c, PV_ERR_INVALID_ARG, "null destination");
    if (rows > 0 && !dst_kind_ok(dst[col], on_device))
      return fail(c, PV_ERR_INVALID_ARG, "destination memory is not of the kind on_device states");
  }
  if (rows == 0) return PV_OK;
  for (int32_t col = 0; col < n_cols; ++col) {
    const void* src;
    size_t bytes;
    if (r.canon.mode == MODE_AGGREGATE) {
      src = r.agg.result + col;
      bytes = 8;
    } else if (r.canon.mode == MODE_PROJECT) {
      src = r.proj.col[col];
      bytes = static_cast<size_t>(rows) * type_size(r.col_type[col]);
    } else {
      src = r.grp.out + static_cast<size_t>(col) * r.grp.out_cap;
      bytes = static_cast<size_t>(rows) * 8;
    }
    PV_CUDA(c, cudaMemcpyAsync(dst[col], src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                               c->stream));
  }
  PV_CUDA(c, cudaStreamSynchronize(c->stream));
  return PV_OK;
}

static int64_t result_capacity(const Result& r) {
  if (r.canon.mode == MODE_AGGREGATE) return 1;
  if (r.canon.mode == MODE_PROJECT) return r.proj.capacity;
  return r.grp.out_cap;
}

pv_status pv_result_capacity(pv_ctx* c, pv_res h, int64_t* rows) {
  if (!c || !rows) return PV_ERR_INVALID_ARG;
  auto it = c->results.find(h);
  if (it == c->results.end()) return fail(c, PV_ERR_INVALID_ARG, "unknown result handle");
  *rows = result_capacity(*it->second);
  return PV_OK;
}

pv_status pv_enqueue_fetch(pv_ctx* c, pv_res h, int32_t n_cols, void* const* dst, const int64_t* dst_rows,
                           int64_t* rows_dst, int32_t on_device) {
  if (!c || !dst || !dst_rows || !rows_dst) return PV_ERR_INVALID_ARG;
  auto it = c->results.find(h);
  if (it == c->results.end()) return fail(c, PV_ERR_INVALID_ARG, "unknown result handle");
  Result& r = *it->second;
  if (n_cols != r.n_cols) return fail(c, PV_ERR_INVALID_ARG, "n_cols differs from the result's columns");
  const int64_t cap = result_capacity(r);
  for (int32_t col = 0; col < n_cols; ++col) {
    if (!dst[col] || dst_rows[col] < cap) return fail(c, PV_ERR_INVALID_ARG, "destination smaller than the capacity");
    if (!dst_kind_ok(dst[col], on_device))
      return fail(c, PV_ERR_INVALID_ARG, "destination memory is not of the kind dst_on_device states");
  }
  if (!dst_kind_ok(rows_dst, on_device))
    return fail(c, PV_ERR_INVALID_ARG, "row count destination is not of the kind dst_on_device states");
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  for (int32_t col = 0; col < n_cols; ++col) {
    const void* src;
    size_t bytes;
    if (r.canon.mode == MODE_AGGREGATE) {
      src = r.agg.result + col;
      bytes = 8;
    } else if (r.canon.mode == MODE_PROJECT) {
      src = r.proj.col[col];
      bytes = static_cast<size_t>(cap) * type_size(r.col_type[col]);
    } else {
      src = r.grp.out + static_cast<size_t>(col) * r.grp.out_cap;
      bytes = static_cast<size_t>(cap) * 8;
    }
    PV_CUDA(c, cudaMemcpyAsync(dst[col], src, bytes, kind, c->stream));
  }
  if (r.canon.mode == MODE_AGGREGATE) {
    // one row; device memory is written by a copy, never by the host
    if (on_device) PV_CUDA(c, cudaMemcpyAsync(rows_dst, c->d_one, 8, cudaMemcpyDeviceToDevice, c->stream));
    else *rows_dst = 1;
  } else {
    const void* cnt = r.canon.mode == MODE_PROJECT ? static_cast<const void*>(r.proj.count)
                                                   : static_cast<const void*>(r.grp.out_count);
    PV_CUDA(c, cudaMemcpyAsync(rows_dst, cnt, 8, kind, c->stream));
  }
  return PV_OK;
}

// Live-row copy of a result: column blockIdx.y, its first
// min(*count, cap) rows (one row when count is null), into device-writable
// memory (device memory or page-locked host memory through its device
// address).  16-byte words when both ends are 16-byte aligned, else elements.
struct FetchArgs {
  const void* src[PV_MAX_KEYS + PV_MAX_AGGS];
  void* dst[PV_MAX_KEYS + PV_MAX_AGGS];
  int esize[PV_MAX_KEYS + PV_MAX_AGGS];
  const unsigned long long* count;
  int64_t cap;
  int64_t* rows_dst;
};

__global__ void k_fetch_rows(const __grid_constant__ FetchArgs a) {
  int64_t n = 1;
  if (a.count != nullptr) {
    const unsigned long long c = *a.count;
    n = c < static_cast<unsigned long long>(a.cap) ? static_cast<int64_t>(c) : a.cap;
  }
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *a.rows_dst = n;
  const int col = blockIdx.y;
  const int es = a.esize[col];
  const char* s = static_cast<const char*>(a.src[col]);
  char* d = static_cast<char*>(a.dst[col]);
  const int64_t bytes = n * es;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (((reinterpret_cast<uintptr_t>(s) | reinterpret_cast<uintptr_t>(d)) & 15u) == 0) {
    const int64_t nv = bytes >> 4;
    for (int64_t i = t; i < nv; i += stride)
      reinterpret_cast<uint4*>(d)[i] = __ldg(reinterpret_cast<const uint4*>(s) + i);
    for (int64_t i = (nv << 4) + t; i < bytes; i += stride) d[i] = s[i];
    return;
  }
  for (int64_t i = t; i < n; i += stride) {
    if (es == 8) reinterpret_cast<uint64_t*>(d)[i] = reinterpret_cast<const uint64_t*>(s)[i];
    else if (es == 4) reinterpret_cast<uint32_t*>(d)[i] = reinterpret_cast<const uint32_t*>(s)[i];
    else d[i] = s[i];
  }
}

// Device address of caller memory a kernel may write: device or managed
// memory as is, page-locked host memory through its device alias; null for
// pageable host memory.
static void* device_writable(void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();  // clear the error the query left
    return nullptr;
  }
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) return p;
  if (at.type == cudaMemoryTypeHost) return at.devicePointer;
  return nullptr;
}

pv_status pv_enqueue_fetch_rows(pv_ctx* c, pv_res h, int32_t n_cols, void* const* dst, const int64_t* dst_rows,
                                int64_t* rows_dst) {
  if (!c || !dst || !dst_rows || !rows_dst) return PV_ERR_INVALID_ARG;
  auto it = c->results.find(h);
  if (it == c->results.end()) return fail(c, PV_ERR_INVALID_ARG, "unknown result handle");
  Result& r = *it->second;
  if (n_cols != r.n_cols) return fail(c, PV_ERR_INVALID_ARG, "n_cols differs from the result's columns");
  const int64_t cap = result_capacity(r);
  FetchArgs a{};
  a.cap = cap;
  a.rows_dst = static_cast<int64_t*>(device_writable(rows_dst));
  if (!a.rows_dst) return fail(c, PV_ERR_INVALID_ARG, "row count destination is not device or page-locked memory");
  int64_t max_bytes = 8;
  for (int32_t col = 0; col < n_cols; ++col) {
    if (!dst[col] || dst_rows[col] < cap) return fail(c, PV_ERR_INVALID_ARG, "destination smaller than the capacity");
    a.dst[col] = device_writable(dst[col]);
    if (!a.dst[col]) return fail(c, PV_ERR_INVALID_ARG, "destination is not device or page-locked memory");
    if (r.canon.mode == MODE_AGGREGATE) {
      a.src[col] = r.agg.result + col;
      a.esize[col] = 8;
    } else if (r.canon.mode == MODE_PROJECT) {
      a.src[col] = r.proj.col[col];
      a.esize[col] = static_cast<int>(type_size(r.col_type[col]));
    } else {
      a.src[col] = r.grp.out + static_cast<size_t>(col) * r.grp.out_cap;
      a.esize[col] = 8;
    }
    max_bytes = std::max<int64_t>(max_bytes, cap * a.esize[col]);
  }
  a.count = r.canon.mode == MODE_AGGREGATE ? nullptr
            : r.canon.mode == MODE_PROJECT ? reinterpret_cast<const unsigned long long*>(r.proj.count)
                                           : r.grp.out_count;
  // sized for the capacity: the live rows are not known on the host
  const int64_t want = (max_bytes / 16 + 255) / 256;
  const int gx = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(want, c->sm_count * 4)));
  k_fetch_rows<<<dim3(gx, n_cols), 256, 0, c->stream>>>(a);
  PV_CUDA(c, cudaGetLastError());
  return PV_OK;
}

pv_status pv_result_kernel(pv_ctx* c, pv_res h, int32_t* generic, char* buf, int64_t cap) {
  if (!c || !generic) return PV_ERR_INVALID_ARG;
  auto it = c->results.find(h);
  if (it == c->results.end()) return fail(c, PV_ERR_INVALID_ARG, "unknown result handle");
  *generic = it->second->generic ? 1 : 0;
  if (buf && cap > 0) {
    const std::string& sig = it->second->canon.sig;
    const size_t n = std::min<size_t>(sig.size(), static_cast<size_t>(cap - 1));
    std::memcpy(buf, sig.data(), n);
    buf[n] = 0;
  }
  return PV_OK;
}

pv_status pv_free(pv_ctx* c, int32_t h) {
  if (!c) return PV_ERR_INVALID_ARG;
  if (c->capturing) return fail(c, PV_ERR_INVALID_ARG, "cannot free while capturing");
  if (c->cols.erase(h)) return PV_OK;
  auto t = c->tables.find(h);
  if (t != c->tables.end()) {
    cudaStreamSynchronize(c->stream);
    dfree(c, t->second->mem);
    c->tables.erase(t);
    return PV_OK;
  }
  auto r = c->results.find(h);
  if (r != c->results.end()) {
    cudaStreamSynchronize(c->stream);
    for (void* p : r->second->mem) dfree(c, p);
    c->results.erase(r);
    for (auto it = c->cols.begin(); it != c->cols.end();)  // columns registered from the result
      it = it->second.src_res == h ? c->cols.erase(it) : std::next(it);
    return PV_OK;
  }
  auto g = c->graphs.find(h);
  if (g != c->graphs.end()) {
    if (g->second.exec) cudaGraphExecDestroy(g->second.exec);
    if (g->second.g) cudaGraphDestroy(g->second.g);
    c->graphs.erase(g);
    return PV_OK;
  }
  return fail(c, PV_ERR_INVALID_ARG, "unknown handle");
}

pv_status pv_graph_capture_begin(pv_ctx* c) {
  if (!c) return PV_ERR_INVALID_ARG;
  if (c->capturing) return fail(c, PV_ERR_INVALID_ARG, "already capturing");
  if (c->stream == nullptr) return fail(c, PV_ERR_INVALID_ARG, "graph capture needs a non-default stream");
  PV_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  c->capturing = true;
  return PV_OK;
}

pv_status pv_graph_capture_end(pv_ctx* c, pv_graph* out) {
  if (!c || !out) return PV_ERR_INVALID_ARG;
  if (!c->capturing) return fail(c, PV_ERR_INVALID_ARG, "not capturing");
  c->capturing = false;
  Graph g;
  PV_CUDA(c, cudaStreamEndCapture(c->stream, &g.g));
  cudaError_t e = cudaGraphInstantiate(&g.exec, g.g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g.g);
    return cuda_fail(c, e, "cudaGraphInstantiate");
  }
  const int32_t h = c->next++;
  c->graphs[h] = g;
  *out = h;
  return PV_OK;
}

pv_status pv_graph_launch(pv_ctx* c, pv_graph h) {
  if (!c) return PV_ERR_INVALID_ARG;
  auto g = c->graphs.find(h);
  if (g == c->graphs.end()) return fail(c, PV_ERR_INVALID_ARG, "unknown graph handle");
  PV_CUDA(c, cudaGraphLaunch(g->second.exec, c->stream));
  for (auto& kv : c->results) kv.second->rows_cached = -1;  // the replay may change any result's rows
  return PV_OK;
}

pv_status pv_l2_flush(pv_ctx* c) {
  if (!c) return PV_ERR_INVALID_ARG;
  if (!c->flush_buf) {
    if (c->capturing) return fail(c, PV_ERR_INVALID_ARG, "first pv_l2_flush allocates; call it before capturing");
    c->flush_bytes = std::max<int64_t>(2 * c->l2_bytes, 64 << 20);
    c->flush_buf = dalloc(c, static_cast<size_t>(c->flush_bytes));
    if (!c->flush_buf) return fail(c, PV_ERR_OOM, "allocator returned NULL");
  }
  static uint32_t salt = 1;
  const int64_t n = c->flush_bytes / 16;
  k_flush<<<c->sm_count * 4, 512, 0, c->stream>>>(static_cast<uint4*>(c->flush_buf), n, salt++);
  k_discard<<<c->sm_count * 4, 512, 0, c->stream>>>(static_cast<char*>(c->flush_buf), c->flush_bytes);
  PV_CUDA(c, cudaGetLastError());
  return PV_OK;
}

pv_status pv_last_launch_count(pv_ctx* c, int32_t* n) {
  if (!c || !n) return PV_ERR_INVALID_ARG;
  *n = c->launches;
  return PV_OK;
}

pv_status pv_set_kernel_timing(pv_ctx* c, int32_t enable) {
  if (!c) return PV_ERR_INVALID_ARG;
  c->ktime = enable != 0;
  c->kev_used = 0;
  return PV_OK;
}

pv_status pv_kernel_times(pv_ctx* c, float* ms, int32_t max, int32_t* n) {
  if (!c || !n || (max > 0 && !ms)) return PV_ERR_INVALID_ARG;
  PV_CUDA(c, cudaStreamSynchronize(c->stream));
  const int k = c->kev_used / 2;
  for (int i = 0; i < k && i < max; ++i) {
    float t = 0;
    PV_CUDA(c, cudaEventElapsedTime(&t, c->kev[2 * i], c->kev[2 * i + 1]));
    ms[i] = t;
  }
  *n = k;
  return PV_OK;
}

pv_status pv_mlp_forward(pv_ctx* c, const float* params, const float* x, const float* mu, const float* sigma,
                         int32_t batch, int32_t n_features, float* y, float* act) {
  if (!c) return PV_ERR_INVALID_ARG;
  c->launches = 0;
  pv_status s = mlp_forward(c->stream, &c->launches, params, x, mu, sigma, batch, n_features, y, act);
  return s == PV_OK ? s : fail(c, s, "pv_mlp_forward failed");
}

pv_status pv_mlp_backward(pv_ctx* c, const float* params, const float* x, const float* mu, const float* sigma,
                          const float* act, const float* y, const float* target, int32_t batch, int32_t n_features,
                          float* dz, float* grad, float* loss) {
  if (!c) return PV_ERR_INVALID_ARG;
  c->launches = 0;
  pv_status s = mlp_backward(c->stream, &c->launches, params, x, mu, sigma, act, y, target, batch, n_features, dz,
                             grad, loss);
  return s == PV_OK ? s : fail(c, s, "pv_mlp_backward failed");
}

pv_status pv_mlp_adam(pv_ctx* c, float* params, const float* grad, float* m, float* v, int64_t n, float lr,
                      float beta1, float beta2, float eps, int32_t step) {
  if (!c) return PV_ERR_INVALID_ARG;
  c->launches = 0;
  pv_status s = mlp_adam(c->stream, &c->launches, params, grad, m, v, n, lr, beta1, beta2, eps, step);
  return s == PV_OK ? s : fail(c, s, "pv_mlp_adam failed");
}

pv_status pv_atomic_peak(pv_ctx* c, int64_t slots, int32_t words, int64_t n_updates, float* ms) {
  if (!c || !ms || slots < 1 || words < 1 || words > 16 || n_updates < 1) return PV_ERR_INVALID_ARG;
  if (c->capturing) return fail(c, PV_ERR_INVALID_ARG, "pv_atomic_peak cannot be captured");
  const size_t bytes = static_cast<size_t>(slots) * static_cast<size_t>(words) * 8;
  if (bytes > (size_t{64} << 30)) return fail(c, PV_ERR_INVALID_ARG, "table larger than 64 GB");
  pv_status st = pv_l2_flush(c);  // allocates the flush buffer before the table
  if (st != PV_OK) return st;
  auto* t = static_cast<unsigned long long*>(dalloc(c, bytes));
  if (!t) return fail(c, PV_ERR_OOM, "allocator returned NULL");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(t, 0, bytes, c->stream);
  const int grid = c->sm_count * 8;
  if (ce == cudaSuccess) {
    k_atomic_rand<<<grid, 256, 0, c->stream>>>(t, slots, words, n_updates, 0x9e3779b97f4a7c15ull);  // warm-up
    ce = cudaGetLastError();
  }
  if (ce == cudaSuccess) st = pv_l2_flush(c);
  if (ce == cudaSuccess && st == PV_OK) ce = cudaEventRecord(e0, c->stream);
  if (ce == cudaSuccess && st == PV_OK) {
    k_atomic_rand<<<grid, 256, 0, c->stream>>>(t, slots, words, n_updates, 0x2545f4914f6cdd1dull);
    ce = cudaGetLastError();
  }
  if (ce == cudaSuccess && st == PV_OK) ce = cudaEventRecord(e1, c->stream);
  if (ce == cudaSuccess && st == PV_OK) ce = cudaEventSynchronize(e1);
  if (ce == cudaSuccess && st == PV_OK) ce = cudaEventElapsedTime(ms, e0, e1);
  cudaStreamSynchronize(c->stream);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  dfree(c, t);
  if (st != PV_OK) return st;
  if (ce != cudaSuccess) return fail(c, PV_ERR_CUDA, cudaGetErrorString(ce));
  return PV_OK;
}

pv_status pv_debug_spin(pv_ctx* c, int64_t ns) {
  if (!c || ns < 0 || ns > 60ll * 1000 * 1000 * 1000) return PV_ERR_INVALID_ARG;
  k_spin<<<1, 1, 0, c->stream>>>(ns);
  PV_CUDA(c, cudaGetLastError());
  return PV_OK;
}

}  // extern "C"
