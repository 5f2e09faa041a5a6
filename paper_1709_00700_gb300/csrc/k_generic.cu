// Generic pipeline kernels: any pipeline program of Table 1's operations
// within the limits of pv.h, with the program (which columns the predicates
// test, which probes run on which key column, the key parts, the aggregate
// terms, the projected values) read at run time from a GenSpec instead of
// being compiled into the kernel.  They run a pipeline when no compiled shape
// matches its spec, when its fact columns are an earlier pipeline's result
// (whose row count exists only on the device), or when the variant asks for
// them (pv_variant.interp = 1).
//
// One thread takes one row at a time, grid-stride over rows, so neighbouring
// lanes read neighbouring rows of each column (coalesced scalar loads).
// Branched mode stops at a row's first failing operation; predicated mode
// evaluates every predicate and probe of every row (Section 6).  The sinks
// are those of the compiled kernels with the aggregate functions read at run
// time: AGGREGATE with per-thread accumulators and one atomic per CTA and
// aggregate; PROJECT single pass (warp-aggregated atomics) or multi pass
// (count, prefix sum, scatter in input order); HASH_AGGREGATE into global
// tables (perfect array, linear probing, cuckoo after a key pass) or
// CTA-local tables in shared memory (Section 4.2), extracted as usual.
#include "k_group.cuh"

namespace pv {
namespace {

constexpr int kGW = PV_MAX_AGGS + 1;  // accumulator words: the aggregates, then the row count

__device__ __forceinline__ int64_t gload(const void* p, int type, int64_t r) {
  if (type == PV_I32) return __ldg(static_cast<const int32_t*>(p) + r);
  if (type == PV_I64) return __ldg(static_cast<const int64_t*>(p) + r);
  return __ldg(static_cast<const uint8_t*>(p) + r);
}

// Rows of the pipeline: n_rows, or the count an earlier pipeline left on the
// device (at most n_rows, the capacity of its result columns).
__device__ __forceinline__ int64_t g_rows(const KParams& kp, const GenSpec& gs) {
  if (gs.n_dyn == nullptr) return kp.n_rows;
  const unsigned long long d = __ldcg(gs.n_dyn);
  return d < static_cast<unsigned long long>(kp.n_rows) ? static_cast<int64_t>(d) : kp.n_rows;
}

// FILTER and HASH_PROBE of row r (Table 1, in the program's order): whether
// the row survives, and what each probe binds (the payload, or for tables
// with several payload columns the build row).
__device__ __forceinline__ bool g_row(const KParams& kp, const GenSpec& gs, int64_t r, bool pred,
                                      int32_t (&bind)[PV_MAX_PROBES]) {
  bool ok = true;
#pragma unroll
  for (int i = 0; i < PV_MAX_PREDS; ++i) {
    if (i < gs.n_preds && (pred || ok)) {
      const int s = gs.pred_slot[i];
      const int64_t v = gload(kp.col[s], gs.slot_type[s], r);
      ok = ok && v >= kp.lo[i] && v <= kp.hi[i];
    }
  }
#pragma unroll
  for (int j = 0; j < PV_MAX_PROBES; ++j) {
    bind[j] = 0;
    if (j < gs.n_probes && (pred || ok)) {
      const int s = gs.probe_slot[j];
      int32_t p = 0;
      const bool hit = probe_key(kp.probe[j], gload(kp.col[s], gs.slot_type[s], r), p);
      bind[j] = hit ? p : 0;
      ok = ok && hit;
    }
  }
  return ok;
}

__device__ __forceinline__ int32_t pick4(const int32_t (&v)[PV_MAX_PROBES], int j) {
  return j == 0 ? v[0] : j == 1 ? v[1] : j == 2 ? v[2] : v[3];
}

// Value of a reference for row r: a fact column, or payload b of probe a.
__device__ __forceinline__ int64_t g_ref(const KParams& kp, const GenSpec& gs, const GRef& x, int64_t r,
                                         const int32_t (&bind)[PV_MAX_PROBES]) {
  if (x.kind == PV_REF_COL) return gload(kp.col[x.a], gs.slot_type[x.a], r);
  const int32_t b = pick4(bind, x.a);
  if (!gs.indexed[x.a]) return b;
  return static_cast<int32_t>(gload(gs.pay_col[x.a][x.b], gs.pay_type[x.a][x.b], b));
}

// ARITHMETIC: the product of the aggregate's terms, wrapping int64 (COUNT: 1).
__device__ __forceinline__ int64_t g_value(const KParams& kp, const GenSpec& gs, const GAgg& a, int64_t r,
                                           const int32_t (&bind)[PV_MAX_PROBES]) {
  if (a.func == PV_COUNT) return 1;
  uint64_t v = 1;
#pragma unroll
  for (int t = 0; t < PV_MAX_TERMS; ++t) {
    if (t < a.n_terms) {
      const GTerm& m = a.t[t];
      const uint64_t x = static_cast<uint64_t>(g_ref(kp, gs, m.x, r, bind));
      const uint64_t c = static_cast<uint64_t>(m.c);
      v *= m.kind == PV_TERM_X ? x : m.kind == PV_TERM_X_PLUS_C ? x + c : c - x;
    }
  }
  return static_cast<int64_t>(v);
}

// Accumulator codes (MIN/MAX as order-preserving codes, so that every word
// starts at 0 and merges with add or max).
__device__ __forceinline__ bool is_minmax(int f) { return f == PV_MIN || f == PV_MAX; }
__device__ __forceinline__ uint64_t g_code(int f, int64_t v) {
  return f == PV_MIN ? min_code(v) : f == PV_MAX ? max_code(v) : static_cast<uint64_t>(v);
}
__device__ __forceinline__ uint64_t g_combine(int f, uint64_t a, uint64_t b) {
  return is_minmax(f) ? (a > b ? a : b) : a + b;
}
__device__ __forceinline__ uint64_t g_warp_reduce(int f, uint64_t v) {
  return is_minmax(f) ? warp_reduce<PV_MAX>(v) : warp_reduce<PV_SUM>(v);
}

// Codes of one surviving row: c[a] for the aggregates, c[PV_MAX_AGGS] = 1.
__device__ __forceinline__ void g_codes(const KParams& kp, const GenSpec& gs, int64_t r,
                                        const int32_t (&bind)[PV_MAX_PROBES], uint64_t (&c)[kGW]) {
#pragma unroll
  for (int a = 0; a < PV_MAX_AGGS; ++a)
    c[a] = a < gs.n_aggs ? g_code(gs.agg[a].func, g_value(kp, gs, gs.agg[a], r, bind)) : 0;
  c[PV_MAX_AGGS] = 1;
}

// ---------------------------------------------------------------------------
// AGGREGATE
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_gen_aggregate(const __grid_constant__ KParams kp,
                                                        const __grid_constant__ GenSpec gs,
                                                        const __grid_constant__ AggOut out, int pred) {
  uint64_t acc[kGW];
#pragma unroll
  for (int a = 0; a < kGW; ++a) acc[a] = 0;
  const int64_t n = g_rows(kp, gs);
  for (int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; r < n;
       r += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int32_t bind[PV_MAX_PROBES];
    if (!g_row(kp, gs, r, pred != 0, bind)) continue;
    uint64_t c[kGW];
    g_codes(kp, gs, r, bind, c);
#pragma unroll
    for (int a = 0; a < PV_MAX_AGGS; ++a)
      if (a < gs.n_aggs) acc[a] = g_combine(gs.agg[a].func, acc[a], c[a]);
    acc[PV_MAX_AGGS] += 1;
  }
  // CTA epilogue: warp shuffles, one slot per warp, one atomic per word; the
  // last CTA decodes the result and re-zeroes the accumulators.
  __shared__ unsigned long long red[32][kGW];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int na = gs.n_aggs;
#pragma unroll
  for (int a = 0; a < kGW; ++a) {
    const int f = a < na ? gs.agg[a].func : PV_SUM;
    acc[a] = g_warp_reduce(f, acc[a]);
    if (lane == 0) red[warp][a] = acc[a];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int a = 0; a < kGW; ++a) {
      if (a < na || a == PV_MAX_AGGS) {
        const int f = a < na ? gs.agg[a].func : PV_SUM;
        const uint64_t v = g_warp_reduce(f, lane < nwarps ? red[lane][a] : 0ull);
        unsigned long long* dst = out.acc + (a < na ? a : na);  // the row count is word n_aggs
        if (lane == 0 && v != 0) {
          if (is_minmax(f)) atomicMax(dst, static_cast<unsigned long long>(v));
          else atomicAdd(dst, static_cast<unsigned long long>(v));
        }
      }
    }
  }
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(out.done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    const uint64_t rows = atomicExch(out.acc + na, 0ull);
    for (int a = 0; a < na; ++a) {
      const uint64_t c = atomicExch(out.acc + a, 0ull);
      const int f = gs.agg[a].func;
      out.result[a] = f == PV_MIN ? (rows ? decode_min(c) : 0)
                      : f == PV_MAX ? (rows ? decode_max(c) : 0) : static_cast<int64_t>(c);
    }
    *out.done = 0;
  }
}

// ---------------------------------------------------------------------------
// PROJECT
// ---------------------------------------------------------------------------
__device__ __forceinline__ void g_write_row(const KParams& kp, const GenSpec& gs, const ProjOut& out, int64_t r,
                                            const int32_t (&bind)[PV_MAX_PROBES], int64_t pos) {
#pragma unroll
  for (int i = 0; i < PV_MAX_PROJ; ++i) {
    if (i < gs.n_proj) {
      const int64_t v = g_ref(kp, gs, gs.proj[i], r, bind);
      const int t = gs.proj_type[i];
      if (t == PV_I32) static_cast<int32_t*>(out.col[i])[pos] = static_cast<int32_t>(v);
      else if (t == PV_I64) static_cast<int64_t*>(out.col[i])[pos] = v;
      else static_cast<uint8_t*>(out.col[i])[pos] = static_cast<uint8_t>(v);
    }
  }
}

// Single pass: each warp reserves its surviving rows with one atomicAdd on the
// output cursor (ballot + popc); the last CTA publishes the count.
__global__ void __launch_bounds__(1024) k_gen_project_sp(const __grid_constant__ KParams kp,
                                                         const __grid_constant__ GenSpec gs,
                                                         const __grid_constant__ ProjOut out, int pred) {
  const int64_t n = g_rows(kp, gs);
  const int lane = threadIdx.x & 31;
  const int64_t T = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  bool overflow = false;
  for (int64_t wb = t - lane; wb < n; wb += T) {  // warp-uniform trips
    const int64_t r = wb + lane;
    int32_t bind[PV_MAX_PROBES];
    const bool live = r < n && g_row(kp, gs, r, pred != 0, bind);
    const unsigned b = __ballot_sync(0xffffffffu, live);
    if (b == 0) continue;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(out.cursor, static_cast<unsigned long long>(__popc(b)));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (live) {
      const int64_t pos = static_cast<int64_t>(base) + __popc(b & ((1u << lane) - 1u));
      if (pos < out.capacity) g_write_row(kp, gs, out, r, bind, pos);
      else overflow = true;
    }
  }
  if (overflow) set_error(kp.err, PV_ERR_OUTPUT_OVERFLOW);
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(out.done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    const int64_t c = static_cast<int64_t>(atomicExch(out.cursor, 0ull));
    *out.count = c < out.capacity ? c : out.capacity;
    *out.done = 0;
  }
}

// Block-wide exclusive scan of a 64-bit value (every thread calls it).
__device__ __forceinline__ uint64_t g_block_scan(uint64_t v, uint64_t* total) {
  __shared__ unsigned long long ws[33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  uint64_t incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(0xffffffffu, static_cast<unsigned long long>(incl), o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) ws[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const uint64_t w = lane < nwarps ? ws[lane] : 0;
    uint64_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, static_cast<unsigned long long>(wi), o);
      if (lane >= o) wi += y;
    }
    if (lane < nwarps) ws[lane] = wi - w;
    if (lane == 31) ws[32] = wi;
  }
  __syncthreads();
  const uint64_t ex = ws[warp] + incl - v;
  *total = ws[32];
  __syncthreads();
  return ex;
}

// Multi pass.  A tile is 4 * U * blockDim rows (the tiles the result was
// allocated for); its row k * blockDim + t belongs to thread t, so rows are
// visited in (k, t) order, which is input order.
__global__ void __launch_bounds__(1024) k_gen_project_count(const __grid_constant__ KParams kp,
                                                            const __grid_constant__ GenSpec gs,
                                                            const __grid_constant__ ProjOut out, int U, int pred) {
  const int64_t n = g_rows(kp, gs);
  const int64_t B = blockDim.x;
  for (int64_t tile = blockIdx.x; tile < out.n_tiles; tile += gridDim.x) {
    const int64_t base = tile * B * 4 * U;
    uint64_t cnt = 0;
    for (int k = 0; k < 4 * U; ++k) {
      const int64_t r = base + k * B + threadIdx.x;
      int32_t bind[PV_MAX_PROBES];
      cnt += r < n && g_row(kp, gs, r, pred != 0, bind);
    }
    uint64_t total;
    g_block_scan(cnt, &total);
    if (threadIdx.x == 0) out.tile_count[tile] = static_cast<int64_t>(total);
  }
  pdl_launch_dependents();
}

__global__ void __launch_bounds__(1024) k_gen_project_scatter(const __grid_constant__ KParams kp,
                                                              const __grid_constant__ GenSpec gs,
                                                              const __grid_constant__ ProjOut out, int U,
                                                              int pred) {
  pdl_wait();  // launched early behind the scan kernel
  const int64_t n = g_rows(kp, gs);
  const int64_t B = blockDim.x;
  for (int64_t tile = blockIdx.x; tile < out.n_tiles; tile += gridDim.x) {
    const int64_t base = tile * B * 4 * U;
    int64_t pos = out.tile_offset[tile];
    for (int q = 0; q < U; ++q) {
      // rows k = 4q .. 4q + 3 of every thread, their flags packed in 16-bit
      // fields (each field's block total is at most blockDim <= 1024)
      int32_t bind[4][PV_MAX_PROBES];
      bool live[4];
      uint64_t packed = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int64_t r = base + (4 * q + j) * B + threadIdx.x;
        live[j] = r < n && g_row(kp, gs, r, pred != 0, bind[j]);
        packed |= static_cast<uint64_t>(live[j]) << (16 * j);
      }
      uint64_t total;
      const uint64_t ex = g_block_scan(packed, &total);
      int64_t before = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (live[j]) {
          const int64_t p = pos + before + static_cast<int64_t>((ex >> (16 * j)) & 0xFFFF);
          if (p < out.capacity) g_write_row(kp, gs, out, base + (4 * q + j) * B + threadIdx.x, bind[j], p);
        }
        before += static_cast<int64_t>((total >> (16 * j)) & 0xFFFF);
      }
      pos += before;
    }
  }
}

// ---------------------------------------------------------------------------
// HASH_AGGREGATE
// ---------------------------------------------------------------------------
enum GenSink { GS_GLOBAL_PERFECT = 0, GS_GLOBAL_HASH = 1, GS_LOCAL_PERFECT = 2, GS_LOCAL_HASH = 3 };

// Key of a row: the mixed-radix code of its parts over their domains (the
// perfect-array slot, and the hash key of coded keys: zero when a part is out
// of its domain), else the packed key (one part, or two 32-bit halves).
__device__ __forceinline__ void g_key(const KParams& kp, const GenSpec& gs, const GroupDesc& gd, int64_t r,
                                      const int32_t (&bind)[PV_MAX_PROBES], uint64_t& code, uint64_t& packed,
                                      bool& in_domain) {
  int64_t part[PV_MAX_KEYS];
#pragma unroll
  for (int i = 0; i < PV_MAX_KEYS; ++i) part[i] = i < gs.n_keys ? g_ref(kp, gs, gs.key[i], r, bind) : 0;
  code = 0;
  in_domain = true;
#pragma unroll
  for (int i = 0; i < PV_MAX_KEYS; ++i) {
    if (i < gs.n_keys) {
      const uint64_t a = static_cast<uint64_t>(part[i]) - static_cast<uint64_t>(gd.key_min[i]);
      const uint64_t span = static_cast<uint64_t>(gd.key_span[i]);
      in_domain = in_domain && a < span;
      code = i == 0 ? a : code * span + a;
    }
  }
  if (gd.coded) packed = in_domain ? code : 0;
  else if (gs.n_keys == 1) packed = gd.key64[0] ? static_cast<uint64_t>(part[0]) : static_cast<uint32_t>(part[0]);
  else packed = (static_cast<uint64_t>(static_cast<uint32_t>(part[0])) << 32) | static_cast<uint32_t>(part[1]);
}

// Adds one row's codes (or a local table's slot) into a slot: SUM/COUNT add,
// MIN/MAX take the max of codes; the row count goes to word n_aggs only when
// no COUNT aggregate holds it.  SHARED: the slot is in shared memory.
template <bool SHARED>
__device__ __forceinline__ void g_slot_add(unsigned long long* v, const uint64_t (&c)[kGW], const GroupDesc& gd) {
#pragma unroll
  for (int a = 0; a < PV_MAX_AGGS; ++a) {
    if (a < gd.n_aggs && c[a] != 0) {
      if (is_minmax(gd.func[a])) atomicMax(v + a, static_cast<unsigned long long>(c[a]));
      else if constexpr (SHARED) shared_add64(v + a, c[a]);
      else atomicAdd(v + a, static_cast<unsigned long long>(c[a]));
    }
  }
  if (gd.count_word == gd.n_aggs && c[PV_MAX_AGGS] != 0) {
    if constexpr (SHARED) shared_add64(v + gd.n_aggs, c[PV_MAX_AGGS]);
    else atomicAdd(v + gd.n_aggs, static_cast<unsigned long long>(c[PV_MAX_AGGS]));
  }
}

template <int SK, int GM>
__global__ void __launch_bounds__(1024) k_gen_group(const __grid_constant__ KParams kp,
                                                    const __grid_constant__ GenSpec gs,
                                                    const __grid_constant__ GroupDesc gd,
                                                    const __grid_constant__ GroupOut g, int pred) {
  extern __shared__ unsigned long long smem[];
  if (blockIdx.x == 0 && threadIdx.x == 0) *g.out_count = 0;  // extraction runs after this kernel
  unsigned long long* lk = smem;                               // local hash table: keys, then values
  unsigned long long* lv = smem + (SK == GS_LOCAL_HASH ? g.local_slots : 0);
  if constexpr (SK == GS_LOCAL_PERFECT) {
    for (int64_t i = threadIdx.x; i < g.cap * g.stride; i += blockDim.x) smem[i] = 0;
    __syncthreads();
  } else if constexpr (SK == GS_LOCAL_HASH) {
    for (int i = threadIdx.x; i < g.local_slots; i += blockDim.x) lk[i] = kEmpty64;
    for (int64_t i = threadIdx.x; i < static_cast<int64_t>(g.local_slots) * g.stride; i += blockDim.x) lv[i] = 0;
    __syncthreads();
  }
  const int64_t n = g_rows(kp, gs);
  unsigned long long* rep = g.vals + (blockIdx.x % g.replicas) * g.rep_stride;
  for (int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; r < n;
       r += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int32_t bind[PV_MAX_PROBES];
    if (!g_row(kp, gs, r, pred != 0, bind)) continue;
    uint64_t code, key;
    bool in_domain;
    g_key(kp, gs, gd, r, bind, code, key, in_domain);
    if (!in_domain && (SK == GS_GLOBAL_PERFECT || SK == GS_LOCAL_PERFECT || gd.coded)) {
      set_error(kp.err, PV_ERR_KEY_OUT_OF_RANGE);
      continue;
    }
    uint64_t c[kGW];
    g_codes(kp, gs, r, bind, c);
    if constexpr (SK == GS_GLOBAL_PERFECT) {
      g_slot_add<false>(rep + code * g.stride, c, gd);
    } else if constexpr (SK == GS_LOCAL_PERFECT) {
      g_slot_add<true>(smem + code * g.stride, c, gd);
    } else {
      if constexpr (SK == GS_LOCAL_HASH) {
        if (key != kEmpty64) {
          const uint32_t mask = static_cast<uint32_t>(g.local_slots) - 1;
          uint32_t idx = static_cast<uint32_t>(fmix64(key)) & mask;
          bool placed = false;
          for (int step = 0; step < kLocalProbe && !placed; ++step) {
            unsigned long long cur = *reinterpret_cast<volatile unsigned long long*>(lk + idx);
            if (cur == kEmpty64) cur = atomicCAS(lk + idx, kEmpty64, static_cast<unsigned long long>(key));
            if (cur == kEmpty64 || cur == key) {
              g_slot_add<true>(lv + static_cast<uint64_t>(idx) * g.stride, c, gd);
              placed = true;
            }
            idx = (idx + 1) & mask;
          }
          if (placed) continue;
        }
      }
      const uint64_t s = global_slot<GM>(g, key, kp.err);  // rows that found no local slot, too
      if (s <= static_cast<uint64_t>(g.cap)) g_slot_add<false>(g.vals + s * g.stride, c, gd);
    }
  }
  pdl_launch_dependents();  // the extraction kernel may start launching now
  if constexpr (SK == GS_LOCAL_PERFECT) {
    __syncthreads();
    for (int64_t i = threadIdx.x; i < g.cap * g.stride; i += blockDim.x) {
      const uint64_t v = smem[i];
      if (!v) continue;
      const int a = static_cast<int>(i % g.stride);
      if (a < gd.n_aggs && is_minmax(gd.func[a])) atomicMax(rep + i, static_cast<unsigned long long>(v));
      else atomicAdd(rep + i, static_cast<unsigned long long>(v));
    }
  } else if constexpr (SK == GS_LOCAL_HASH) {
    __syncthreads();
    for (int i = threadIdx.x; i < g.local_slots; i += blockDim.x) {
      const uint64_t key = lk[i];
      if (key == kEmpty64) continue;
      const unsigned long long* w = lv + static_cast<uint64_t>(i) * g.stride;
      uint64_t c[kGW];
#pragma unroll
      for (int a = 0; a < PV_MAX_AGGS; ++a) c[a] = a < gd.n_aggs ? w[a] : 0;
      c[PV_MAX_AGGS] = gd.count_word == gd.n_aggs ? w[gd.n_aggs] : 0;
      if (w[gd.count_word] == 0) continue;
      const uint64_t s = global_slot<GM>(g, key, kp.err);
      if (s <= static_cast<uint64_t>(g.cap)) g_slot_add<false>(g.vals + s * g.stride, c, gd);
    }
  }
}

// Key pass of the multi-pass strategy: the group key of every surviving row
// into the global linear or cuckoo table.
template <int HTK>
__global__ void __launch_bounds__(1024) k_gen_keys(const __grid_constant__ KParams kp,
                                                   const __grid_constant__ GenSpec gs,
                                                   const __grid_constant__ GroupDesc gd,
                                                   const __grid_constant__ GroupOut g, int pred) {
  const int64_t n = g_rows(kp, gs);
  for (int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; r < n;
       r += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int32_t bind[PV_MAX_PROBES];
    if (!g_row(kp, gs, r, pred != 0, bind)) continue;
    uint64_t code, key;
    bool in_domain;
    g_key(kp, gs, gd, r, bind, code, key, in_domain);
    if (!in_domain && gd.coded) {
      set_error(kp.err, PV_ERR_KEY_OUT_OF_RANGE);
      continue;
    }
    if constexpr (HTK == PV_HT_CUCKOO) global_cuckoo_insert(g, key, kp.err);
    else global_linear_slot(g, key, kp.err);
  }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <class K, class... Args>
pv_status g_launch(const LaunchCfg& c, K k, size_t smem, int64_t rows, Args... args) {
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess)
    return PV_ERR_UNSUPPORTED;
  const int grid = grid_for(c, reinterpret_cast<const void*>(k), smem, rows, static_cast<int64_t>(c.block) * 4);
  if (grid <= 0) return PV_ERR_UNSUPPORTED;
  kmark(c);
  k<<<grid, c.block, smem, c.stream>>>(args...);
  kmark(c);
  ++*c.launches;
  return cudaGetLastError() == cudaSuccess ? PV_OK : PV_ERR_CUDA;
}

// The variant axes the generic kernels implement: grid-stride access,
// branched or predicated mode.
bool g_axes_ok(const LaunchCfg& c) { return !c.chunk && !c.compact; }

}  // namespace

pv_status generic_aggregate(const LaunchCfg& c, const KParams& kp, const GenSpec& gs, const AggOut& out) {
  if (!g_axes_ok(c)) return PV_ERR_UNSUPPORTED;
  return g_launch(c, k_gen_aggregate, 0, kp.n_rows, kp, gs, out, c.pred ? 1 : 0);
}

pv_status generic_project(const LaunchCfg& c, const KParams& kp, const GenSpec& gs, const ProjOut& out, int exec) {
  if (!g_axes_ok(c)) return PV_ERR_UNSUPPORTED;
  const int pred = c.pred ? 1 : 0;
  if (exec == PV_EXEC_SINGLE_PASS) return g_launch(c, k_gen_project_sp, 0, kp.n_rows, kp, gs, out, pred);
  const int grid = grid_for(c, reinterpret_cast<const void*>(k_gen_project_count), 0, out.n_tiles, 1);
  if (grid <= 0 || grid_for(c, reinterpret_cast<const void*>(k_gen_project_scatter), 0, 1, 1) <= 0)
    return PV_ERR_UNSUPPORTED;
  kmark(c);
  k_gen_project_count<<<grid, c.block, 0, c.stream>>>(kp, gs, out, c.U, pred);
  kmark(c);
  ++*c.launches;
  pv_status s = launch_tile_scan(c, out, kp.err);
  if (s != PV_OK) return s;
  kmark(c);
  cudaError_t e = c.mark ? (k_gen_project_scatter<<<grid, c.block, 0, c.stream>>>(kp, gs, out, c.U, pred), cudaSuccess)
                         : pdl_launch(k_gen_project_scatter, dim3(grid), dim3(c.block), 0, c.stream, kp, gs, out,
                                      c.U, pred);
  kmark(c);
  ++*c.launches;
  return e == cudaSuccess && cudaGetLastError() == cudaSuccess ? PV_OK : PV_ERR_CUDA;
}

pv_status generic_grouped(const LaunchCfg& c, const KParams& kp, const GenSpec& gs, const GroupDesc& gd,
                          const GroupOut& g0, const pv_variant& v) {
  if (!g_axes_ok(c) || v.threads_per_table == 1 || v.agg == PV_AGG_CLUSTER || v.warp_agg)
    return PV_ERR_UNSUPPORTED;
  if (v.agg != PV_AGG_LOCAL && v.agg != PV_AGG_GLOBAL) return PV_ERR_INVALID_ARG;
  GroupOut g = g0;
  const int pred = c.pred ? 1 : 0;
  const bool multi = v.exec == PV_EXEC_MULTI_PASS;
  const bool local = v.agg == PV_AGG_LOCAL;
  const size_t slot_bytes = static_cast<size_t>(g.stride) * 8;
  pv_status s;
  if (g.ht == PV_HT_PERFECT) {
    if (multi) return PV_ERR_UNSUPPORTED;  // no keys to insert
    if (local) {
      const size_t smem = static_cast<size_t>(g.cap) * slot_bytes;
      if (smem > kLocalPerfectBytes) return PV_ERR_UNSUPPORTED;
      s = g_launch(c, k_gen_group<GS_LOCAL_PERFECT, G_INSERT>, smem, kp.n_rows, kp, gs, gd, g, pred);
    } else {
      s = g_launch(c, k_gen_group<GS_GLOBAL_PERFECT, G_INSERT>, 0, kp.n_rows, kp, gs, gd, g, pred);
    }
    if (s != PV_OK) return s;
    return launch_dedupe_extract(c, gd, g, false);
  }
  const bool cuckoo = g.ht == PV_HT_CUCKOO;
  if (cuckoo && !multi) return PV_ERR_UNSUPPORTED;  // keys move while inserting
  if (multi) {
    s = cuckoo ? g_launch(c, k_gen_keys<PV_HT_CUCKOO>, 0, kp.n_rows, kp, gs, gd, g, pred)
               : g_launch(c, k_gen_keys<PV_HT_LINEAR>, 0, kp.n_rows, kp, gs, gd, g, pred);
    if (s != PV_OK) return s;
    if (cuckoo && (s = launch_dedupe_extract(c, gd, g, true)) != PV_OK) return s;
  }
  if (!local) {
    s = !multi ? g_launch(c, k_gen_group<GS_GLOBAL_HASH, G_INSERT>, 0, kp.n_rows, kp, gs, gd, g, pred)
        : cuckoo ? g_launch(c, k_gen_group<GS_GLOBAL_HASH, G_LOOKUP_CUCKOO>, 0, kp.n_rows, kp, gs, gd, g, pred)
                 : g_launch(c, k_gen_group<GS_GLOBAL_HASH, G_LOOKUP_LINEAR>, 0, kp.n_rows, kp, gs, gd, g, pred);
  } else {
    int ls = 1;
    while (static_cast<size_t>(ls) * 2 * (slot_bytes + 8) <= kLocalBytes) ls *= 2;
    g.local_slots = ls;
    const size_t smem = static_cast<size_t>(ls) * (slot_bytes + 8);
    s = !multi ? g_launch(c, k_gen_group<GS_LOCAL_HASH, G_INSERT>, smem, kp.n_rows, kp, gs, gd, g, pred)
        : cuckoo ? g_launch(c, k_gen_group<GS_LOCAL_HASH, G_LOOKUP_CUCKOO>, smem, kp.n_rows, kp, gs, gd, g, pred)
                 : g_launch(c, k_gen_group<GS_LOCAL_HASH, G_LOOKUP_LINEAR>, smem, kp.n_rows, kp, gs, gd, g, pred);
  }
  if (s != PV_OK) return s;
  return launch_dedupe_extract(c, gd, g, false);
}

}  // namespace pv
