// Stagewise evaluation of the LOOP body over U items per thread and the
// warp-uniform item loop, shared by the scan and the grouped kernels.
#pragma once

#include <type_traits>

#include "pv_internal.h"

namespace pv {

// Evaluates U items stage by stage so that the loads of all U items of one
// stage are in flight together (loop unrolling, Section 6).
template <class SH, bool PRED, int U>
__device__ __forceinline__ void eval_items(Item<SH> (&it)[U], const KParams& kp, const int64_t (&idx)[U]) {
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int64_t left = kp.n_rows - idx[u] * 4;
    it[u].nvalid = left >= 4 ? 4 : (left > 0 ? static_cast<int>(left) : 0);
    it[u].mask = (1u << it[u].nvalid) - 1u;
  }
  using W = typename SH::Where;
  using JP = typename SH::Probes;
  if constexpr (PRED) {
#pragma unroll
    for (int u = 0; u < U; ++u) load_slots<SH, W::slots | JP::slots | SH::rest_slots>(it[u], kp, idx[u]);
#pragma unroll
    for (int u = 0; u < U; ++u)
      static_for<W::N>([&](auto j) { it[u].mask &= pred_bits<SH, decltype(j)::value>(it[u], kp); });
  } else {
    uint32_t loaded = 0;
    static_for<W::N>([&](auto j) {
      constexpr int J = decltype(j)::value;
      constexpr int S = At<J, typename W::L>::type::slot;
      const bool need = !((loaded >> S) & 1u);
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (need && it[u].mask) load_slots<SH, (1u << S)>(it[u], kp, idx[u]);
      loaded |= 1u << S;
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (it[u].mask) it[u].mask &= pred_bits<SH, J>(it[u], kp);
    });
  }
  static_for<JP::N>([&](auto j) {
    constexpr int J = decltype(j)::value;
    constexpr int S = JP::slot_of[J];
    if constexpr (!PRED && !((W::slots >> S) & 1u)) {
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (it[u].mask) load_slots<SH, (1u << S)>(it[u], kp, idx[u]);
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (PRED || it[u].mask) it[u].mask = probe_item(kp.probe[J], VGet<S>::get(it[u].v), it[u].mask, it[u].pay[J], PRED);
  });
  if constexpr (!PRED) {
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (it[u].mask) load_slots<SH, SH::rest_slots>(it[u], kp, idx[u]);
  }
}

// Warp-uniform item loop: every lane of a warp runs the same number of trips
// (items past the end are empty), so warp collectives are safe inside.
template <bool CHUNK, int U, class F>
__device__ __forceinline__ void for_items_uniform(int64_t n_items, F&& f) {
  const int64_t T = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  if constexpr (!CHUNK) {
    for (int64_t wb = t - lane; wb < n_items; wb += U * T) {
      int64_t idx[U];
#pragma unroll
      for (int u = 0; u < U; ++u) idx[u] = wb + lane + u * T;
      f(idx);
    }
  } else {
    const int64_t chunk = (n_items + T - 1) / T;
    const int64_t begin = t * chunk;
    const int64_t end = begin + chunk < n_items ? begin + chunk : n_items;
    for (int64_t k = 0; k < chunk; k += U) {
      int64_t idx[U];
#pragma unroll
      for (int u = 0; u < U; ++u) idx[u] = begin + k + u < end ? begin + k + u : n_items;
      f(idx);
    }
  }
}

// Predicated pipelines split into a load phase (every column of every row
// of the item) and a compute phase (filter bits, probes); with no branch
// between them, the next items' loads can be issued before the current items
// are consumed.
template <class SH, int U>
__device__ __forceinline__ void load_items_all(Item<SH> (&it)[U], const KParams& kp, const int64_t (&idx)[U]) {
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int64_t left = kp.n_rows - idx[u] * 4;
    it[u].nvalid = left >= 4 ? 4 : (left > 0 ? static_cast<int>(left) : 0);
    it[u].mask = (1u << it[u].nvalid) - 1u;
    load_slots<SH, SH::Where::slots | SH::Probes::slots | SH::rest_slots>(it[u], kp, idx[u]);
  }
}

template <class SH, int U>
__device__ __forceinline__ void filter_probe_items(Item<SH> (&it)[U], const KParams& kp) {
  using W = typename SH::Where;
  using JP = typename SH::Probes;
#pragma unroll
  for (int u = 0; u < U; ++u)
    static_for<W::N>([&](auto j) { it[u].mask &= pred_bits<SH, decltype(j)::value>(it[u], kp); });
  static_for<JP::N>([&](auto j) {
    constexpr int J = decltype(j)::value;
    constexpr int S = JP::slot_of[J];
#pragma unroll
    for (int u = 0; u < U; ++u) it[u].mask = probe_item(kp.probe[J], VGet<S>::get(it[u].v), it[u].mask, it[u].pay[J], true);
  });
}

// log2 of the bytes one item (4 rows) of each column occupies, 4 bits per
// column.
template <class L> struct ItemShifts;
template <class... Ts> struct ItemShifts<TList<Ts...>> {
  static constexpr uint32_t log2c(uint32_t x) { return x <= 1 ? 0 : 1 + log2c(x >> 1); }
  static constexpr uint64_t value = [] {
    uint64_t p = 0;
    int i = 0;
    ((p |= static_cast<uint64_t>(log2c(4 * sizeof(typename Ts::T))) << (4 * i++)), ...);
    return p;
  }();
};

// Bulk prefetch into L2 (TMA engine, no registers or shared memory used) of
// the 32 items (128 rows) a warp consumes at one trip, spread over the
// lanes: lane c prefetches column c.  Only whole in-range chunks are
// prefetched (16-byte aligned: column bases are 16-byte aligned and 128 rows
// of any column type are a multiple of 16 bytes).
template <class SH, uint32_t MASK = ~0u>
struct LanePrefetch {
  static_assert(SH::Cols::N <= 16, "one lane per column, 4-bit shifts");
  const char* base = nullptr;
  uint32_t shift = 0;
  __device__ __forceinline__ LanePrefetch(const KParams& kp, int lane) {
    if (lane < SH::Cols::N && ((MASK >> lane) & 1u)) {
      base = static_cast<const char*>(kp.col[lane]);
      shift = static_cast<uint32_t>(ItemShifts<typename SH::Cols::L>::value >> (4 * lane)) & 15u;
    }
  }
  // first_item: the warp's first item of the chunk; n_full: items with 4 rows.
  __device__ __forceinline__ void issue(int64_t first_item, int64_t n_full) const {
    if (base != nullptr && first_item >= 0 && first_item + 32 <= n_full) {
      const char* p = base + (first_item << shift);
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(32u << shift) : "memory");
    }
  }
};

// Columns a branched pipeline reads for every item, before its first branch:
// the filter columns, else the first probe's key column, else all of them.
// Prefetching the others would fetch sectors the lazy loads skip.
template <class SH>
constexpr uint32_t first_stage_slots() {
  if constexpr (SH::Where::N > 0) return SH::Where::slots;
  else if constexpr (SH::Probes::N > 0) return 1u << SH::Probes::slot_of[0];
  else return ~0u;
}

// Grid-stride item loop (as for_items) that also bulk-prefetches into L2
// the chunk of the MASK columns its warp will read kp.prefetch trips later.
// Chunked access: no prefetch.
template <class SH, bool CHUNK, int U, uint32_t MASK = ~0u, class F>
__device__ __forceinline__ void for_items_pf(const KParams& kp, F&& f) {
  const int pf = CHUNK ? 0 : kp.prefetch;
  if (pf == 0) {
    for_items<CHUNK, U>(kp.n_items, f);
    return;
  }
  const int64_t T = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int64_t n_full = kp.n_rows >> 2;
  const LanePrefetch<SH, MASK> lp(kp, lane);
  auto prefetch = [&](int64_t k) {
#pragma unroll
    for (int u = 0; u < U; ++u) lp.issue((t - lane) + (k * U + u) * T, n_full);
  };
  for (int d = 1; d < pf; ++d) prefetch(d);
  int64_t k = 0;
  for (int64_t base = t; base < kp.n_items; base += U * T, ++k) {
    prefetch(k + pf);
    int64_t idx[U];
#pragma unroll
    for (int u = 0; u < U; ++u) idx[u] = base + u * T;
    f(idx);
  }
}

// Predicated grid-stride item loop without register double buffering.
// Trips whose U items all hold 4 rows load every column with no bounds
// checks and call consume(item, std::true_type); the thread's remaining
// items (at most the one partial item of the table and items past the
// full ones) follow with consume(item, std::false_type).  Prefetch as in
// for_items_pf.
template <class SH, int U, class F>
__device__ __forceinline__ void for_items_pred(const KParams& kp, F&& consume) {
  const int64_t T = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int64_t n_full = kp.n_rows >> 2;
  const int pf = kp.prefetch;
  const LanePrefetch<SH> lp(kp, lane);
  constexpr uint32_t all = SH::Where::slots | SH::Probes::slots | SH::rest_slots;
  if (pf > 0) {
    for (int d = 1; d < pf; ++d)
#pragma unroll
      for (int u = 0; u < U; ++u) lp.issue((t - lane) + static_cast<int64_t>(d * U + u) * T, n_full);
  }
  int64_t base = t;
  int64_t pfb = (t - lane) + static_cast<int64_t>(pf) * U * T;  // warp chunk prefetched at this trip
  for (; base + (U - 1) * T < n_full; base += U * T, pfb += U * T) {
    if (pf > 0) {
#pragma unroll
      for (int u = 0; u < U; ++u) lp.issue(pfb + u * T, n_full);
    }
    Item<SH> it[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      it[u].nvalid = 4;
      it[u].mask = 0xFu;
      load_slots<SH, all>(it[u], kp, base + u * T);
    }
    filter_probe_items<SH, U>(it, kp);
#pragma unroll
    for (int u = 0; u < U; ++u) consume(it[u], std::true_type{});
  }
  for (; base < kp.n_items; base += T) {
    Item<SH> one[1];
    const int64_t idx[1] = {base};
    load_items_all<SH, 1>(one, kp, idx);
    filter_probe_items<SH, 1>(one, kp);
    consume(one[0], std::false_type{});
  }
}

// Software-pipelined item loop of predicated pipelines: the loads of trip
// k + 1 are in flight while trip k is filtered, probed and consumed (two
// register buffers used in turn).  Trips and item indices are those of
// for_items.
template <class SH, bool CHUNK, int U, class F>
__device__ __forceinline__ void for_items_pipelined(const KParams& kp, F&& consume) {
  const int64_t n = kp.n_items;
  const int64_t T = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  int64_t cbeg = 0, cend = 0;
  if constexpr (CHUNK) {
    const int64_t chunk = (n + T - 1) / T;
    cbeg = t * chunk;
    cend = cbeg + chunk < n ? cbeg + chunk : n;
  }
  auto valid = [&](int64_t k) { return CHUNK ? k * U < cend - cbeg : t + k * U * T < n; };
  auto idx_of = [&](int64_t k, int64_t (&idx)[U]) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if constexpr (CHUNK) {
        const int64_t i = cbeg + k * U + u;
        idx[u] = i < cend ? i : n;
      } else {
        idx[u] = t + (k * U + u) * T;
      }
    }
  };
  if (!valid(0)) return;
  const int lane = threadIdx.x & 31;
  const int pf = CHUNK ? 0 : kp.prefetch;
  const int64_t n_full = kp.n_rows >> 2;
  const LanePrefetch<SH> lp(kp, lane);
  // trip k of this warp covers items (t - lane) + (k * U + u) * T, 32 per u
  auto prefetch = [&](int64_t k) {
#pragma unroll
    for (int u = 0; u < U; ++u) lp.issue((t - lane) + (k * U + u) * T, n_full);
  };
  if (pf > 0) {
    for (int d = 1; d <= pf; ++d) prefetch(d);
  }
  Item<SH> a[U], b[U];
  int64_t ia[U], ib[U];
  idx_of(0, ia);
  load_items_all<SH, U>(a, kp, ia);
  for (int64_t k = 0;; k += 2) {
    if (pf > 0) prefetch(k + 1 + pf);
    const bool more = valid(k + 1);
    if (more) {
      idx_of(k + 1, ib);
      load_items_all<SH, U>(b, kp, ib);
    }
    filter_probe_items<SH, U>(a, kp);
    consume(a);
    if (!more) break;
    if (pf > 0) prefetch(k + 2 + pf);
    const bool more2 = valid(k + 2);
    if (more2) {
      idx_of(k + 2, ia);
      load_items_all<SH, U>(a, kp, ia);
    }
    filter_probe_items<SH, U>(b, kp);
    consume(b);
    if (!more2) break;
  }
}

// ---------------------------------------------------------------------------
// TMA-staged access (variant access = PV_STAGED), predicated pipelines.  A
// warp's trip covers one chunk of 128 consecutive rows (32 items), as in
// grid-stride access.  Lane 0 of the warp copies the next chunk of every
// column the pipeline reads into the warp's shared-memory stage with bulk
// copies (cp.async.bulk, the TMA engine) that complete on the warp's
// mbarrier; meanwhile the warp filters and aggregates the current chunk from
// registers.  The copies need no registers, so a warp always has its next
// chunk in flight while it computes, which the register-loaded loop can only
// do with a second register set.  Only whole chunks are staged: the last,
// partial chunk of a table is loaded with plain loads.
//
// Row mapping: to read the stage without bank conflicts, lane l takes rows
// 2l, 2l + 1, 64 + 2l and 64 + 2l + 1 of the chunk (every column the same
// way); a grouped aggregation does not depend on which lane holds which row.
// ---------------------------------------------------------------------------
template <class SH>
constexpr uint32_t staged_slots() { return SH::Where::slots | SH::Probes::slots | SH::rest_slots; }

// Bytes of the stage columns before slot S (and of the whole stage, S = N).
template <class SH, int S>
constexpr int stage_offset() {
  if constexpr (S == 0) {
    return 0;
  } else {
    using T = typename At<S - 1, typename SH::Cols::L>::type::T;
    return stage_offset<SH, S - 1>() + (((staged_slots<SH>() >> (S - 1)) & 1u) ? 128 * static_cast<int>(sizeof(T)) : 0);
  }
}
template <class SH>
constexpr int stage_bytes() { return stage_offset<SH, SH::Cols::N>(); }

__device__ __forceinline__ void mbar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Waits for phase `parity` of the mbarrier to complete, for at most about
// `limit_ns` nanoseconds; false when it gave up.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
  uint64_t t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (uint32_t i = 0;; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if ((i & 63u) == 63u) {
      uint64_t t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if (t - t0 > limit_ns) return false;
    }
  }
}

// Lane 0: copies chunk `chunk` (rows 128 * chunk ...) of every staged column
// into the stage at shared address `dst`, completing on mbarrier `bar`.  The
// chunk must lie wholly inside the table.  Column bases are 16-byte aligned
// and a chunk of any column type is a multiple of 128 bytes, as the bulk
// copy requires.
template <class SH>
__device__ __forceinline__ void stage_issue(const KParams& kp, int64_t chunk, uint32_t dst, uint32_t bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(stage_bytes<SH>())
               : "memory");
  static_for<SH::Cols::N>([&](auto c) {
    constexpr int S = decltype(c)::value;
    if constexpr ((staged_slots<SH>() >> S) & 1u) {
      using T = typename At<S, typename SH::Cols::L>::type::T;
      constexpr uint32_t bytes = 128 * sizeof(T);
      const char* src = static_cast<const char*>(kp.col[S]) + chunk * bytes;
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              dst + stage_offset<SH, S>()),
          "l"(src), "r"(bytes), "r"(bar)
          : "memory");
    }
  });
}

// A lane's 4 rows of the staged chunk (row mapping above) into item `it`.
template <class SH>
__device__ __forceinline__ void stage_read(Item<SH>& it, const char* stage, int lane) {
  it.nvalid = 4;
  it.mask = 0xFu;
  static_for<SH::Cols::N>([&](auto c) {
    constexpr int S = decltype(c)::value;
    if constexpr ((staged_slots<SH>() >> S) & 1u) {
      using T = typename At<S, typename SH::Cols::L>::type::T;
      const char* col = stage + stage_offset<SH, S>();
      auto& d = VGet<S>::get(it.v);
      if constexpr (sizeof(T) == 8) {
        const longlong2 a = *reinterpret_cast<const longlong2*>(col + 16 * lane);
        const longlong2 b = *reinterpret_cast<const longlong2*>(col + 512 + 16 * lane);
        d[0] = a.x; d[1] = a.y; d[2] = b.x; d[3] = b.y;
      } else if constexpr (sizeof(T) == 4) {
        const int2 a = *reinterpret_cast<const int2*>(col + 8 * lane);
        const int2 b = *reinterpret_cast<const int2*>(col + 256 + 8 * lane);
        d[0] = a.x; d[1] = a.y; d[2] = b.x; d[3] = b.y;
      } else {
        const uchar2 a = *reinterpret_cast<const uchar2*>(col + 2 * lane);
        const uchar2 b = *reinterpret_cast<const uchar2*>(col + 64 + 2 * lane);
        d[0] = a.x; d[1] = a.y; d[2] = b.x; d[3] = b.y;
      }
    }
  });
}

// Shared memory of the stages: one stage per warp, then one 8-byte mbarrier
// per warp (padded to 16 bytes); whatever follows starts 16-byte aligned.
template <class SH>
__host__ __device__ constexpr size_t stage_smem(int nwarps) {
  return static_cast<size_t>(nwarps) * stage_bytes<SH>() + ((static_cast<size_t>(nwarps) * 8 + 15) & ~size_t(15));
}

// Predicated item loop over TMA-staged chunks: consume(it, full) for each
// lane's item (full: 4 rows of a staged chunk).  All lanes of a warp run
// every trip.  A wait that gives up (after about a second: a copy that never
// completes) sets PV_ERR_TIMEOUT and ends the loop; the warp then waits once
// more, again bounded, for the copy in flight before the caller goes on.
template <class SH, class F>
__device__ __forceinline__ void for_items_staged(const KParams& kp, char* stages, F&& consume) {
  constexpr uint64_t kLimitNs = 1000000000ull;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  char* stage = stages + static_cast<size_t>(warp) * stage_bytes<SH>();
  const uint32_t dst = static_cast<uint32_t>(__cvta_generic_to_shared(stage));
  const uint32_t bar = static_cast<uint32_t>(__cvta_generic_to_shared(stages)) +
                       static_cast<uint32_t>(nwarps * stage_bytes<SH>() + 8 * warp);
  const int64_t TW = static_cast<int64_t>(gridDim.x) * nwarps;
  const int64_t n_chunks = (kp.n_items + 31) >> 5;
  const int64_t n_full = kp.n_rows >> 7;  // chunks of 128 rows inside the table
  int64_t c = static_cast<int64_t>(blockIdx.x) * nwarps + warp;
  if (lane == 0) {
    mbar_init(bar);
    if (c < n_full) stage_issue<SH>(kp, c, dst, bar);
  }
  __syncwarp();
  uint32_t parity = 0;
  bool pending = c < n_full;  // a copy is in flight
  for (; c < n_chunks; c += TW) {
    Item<SH> one[1];
    if (c < n_full) {
      const bool ok = __all_sync(0xffffffffu, mbar_wait(bar, parity, kLimitNs));
      if (!ok) break;
      parity ^= 1u;
      pending = false;
      stage_read<SH>(one[0], stage, lane);
      __syncwarp();
      if (lane == 0) {
        // the warp's reads of the stage precede the next copy into it
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (c + TW < n_full) stage_issue<SH>(kp, c + TW, dst, bar);
      }
      pending = c + TW < n_full;
      filter_probe_items<SH, 1>(one, kp);
      consume(one[0], std::true_type{});
    } else {
      const int64_t idx[1] = {c * 32 + lane};
      load_items_all<SH, 1>(one, kp, idx);
      filter_probe_items<SH, 1>(one, kp);
      consume(one[0], std::false_type{});
    }
  }
  if (c < n_chunks) {  // gave up waiting
    if (lane == 0) set_error(kp.err, PV_ERR_TIMEOUT);
    if (pending) mbar_wait(bar, parity, kLimitNs);
  }
}

// ---------------------------------------------------------------------------
// Compacted execution (variant pred = PV_COMPACTED).  The pipeline's first
// operation (its filters, or else its first probe) runs over whole items as
// in branched mode; the rows it keeps are appended to a queue per warp in
// shared memory, and each 32 * K queued rows are taken K per lane through the
// remaining operations (the probes, the loads of the sink's columns) and
// the sink (a grouped table, or a thread's ungrouped accumulators).  After a
// selective first operation the later operations then run on full warps, not
// on the few live lanes of every warp.  A lane takes its K rows through each
// stage together, so their dependent loads (a key column, then the table, then
// the next key column ...) are in flight together: K = 2 doubles the memory
// requests a warp has outstanding (variant items_per_thread = 2).  Queue
// entries are 32-bit row indices (tables of fewer than 2^32 rows).
// ---------------------------------------------------------------------------
// Queue entries per warp: a drain leaves fewer than 32 * K rows, and one trip
// appends at most 32 lanes x 4 rows.
template <int K>
__host__ __device__ constexpr int queue_cap() { return 32 * K + 128; }

// Whether an expression tree (Key, Aggs, Proj and their terms) reads the
// payload bound by probe J.
template <int J, class T> struct RefPay : std::false_type {};
template <int J, int I> struct RefPay<J, PL<J, I>> : std::true_type {};
template <int J, template <class...> class Tm, class... Ts>
struct RefPay<J, Tm<Ts...>> : std::bool_constant<(RefPay<J, Ts>::value || ...)> {};
// projected values: slot S < 0 is the payload of probe -S - 1
template <int J, int... S> struct RefPay<J, Proj<S...>> : std::bool_constant<((S == -J - 1) || ...)> {};

// RefPay for a probe index known only in a constexpr loop.
template <class SH>
struct RefPayAt {
  static constexpr bool key(int j) {
    return at<0>(j, [](auto J) { return RefPay<decltype(J)::value, typename SH::Key>::value; });
  }
  static constexpr bool aggs(int j) {
    return at<0>(j, [](auto J) { return RefPay<decltype(J)::value, typename SH::Aggs>::value; });
  }
  static constexpr bool proj(int j) {
    return at<0>(j, [](auto J) { return RefPay<decltype(J)::value, typename SH::Proj>::value; });
  }
  template <int I, class F>
  static constexpr bool at(int j, F f) {
    if constexpr (I >= PV_MAX_PROBES) {
      return false;
    } else {
      return j == I ? f(std::integral_constant<int, I>{}) : at<I + 1>(j, f);
    }
  }
};

// Probes of the first stage: none after filters (the filters are the first
// operation), else the first NF (variant compact_probes), which run over
// whole items with their key columns read in full.
template <class SH, int NF>
constexpr int first_probes() {
  return SH::Where::N > 0 ? 0 : (NF < SH::Probes::N ? NF : SH::Probes::N);
}

// The row stage repeats a first-stage probe only to bind its payload: when
// nothing reads that payload, the probe is skipped.
template <class SH, int NF, int J>
constexpr bool compact_skip_probe() {
  return J < first_probes<SH, NF>() && !RefPay<J, typename SH::Key>::value &&
         !RefPay<J, typename SH::Aggs>::value && !RefPay<J, typename SH::Proj>::value;
}

// Key slots of the probes the row stage skips.
template <class SH, int NF>
constexpr uint32_t compact_skipped_slots() {
  uint32_t m = 0;
  for (int j = 0; j < SH::Probes::N && j < first_probes<SH, NF>(); ++j) {
    const bool read = RefPayAt<SH>::key(j) || RefPayAt<SH>::aggs(j) || RefPayAt<SH>::proj(j);
    if (!read) m |= 1u << SH::Probes::slot_of[j];
  }
  return m;
}

// Columns the sink reads for a queued row beyond the probe keys the row stage
// loads (a skipped probe's key column counts as not loaded).
template <class SH, int NF>
constexpr uint32_t compact_row_slots() {
  constexpr uint32_t probed = SH::Probes::slots & ~compact_skipped_slots<SH, NF>();
  return (SH::Key::slots | SH::Aggs::slots | SH::Proj::slots) & ~probed;
}

// First stage of an item (nvalid = 0 past the table): its filters, or else
// its first NF probes, the key column of each read for the whole item
// (compact_first_load); then the filters or probes leave the surviving rows in
// it.mask (compact_first_eval).
template <class SH, int NF>
__device__ __forceinline__ void compact_first_load(Item<SH>& it, const KParams& kp, int64_t item) {
  using W = typename SH::Where;
  using JP = typename SH::Probes;
  const int64_t left = kp.n_rows - item * 4;
  it.nvalid = left >= 4 ? 4 : (left > 0 ? static_cast<int>(left) : 0);
  it.mask = (1u << it.nvalid) - 1u;
  if constexpr (W::N > 0) {
    load_slots<SH, W::slots>(it, kp, item);
  } else {
    constexpr int NP = first_probes<SH, NF>();
    static_for<NP>([&](auto j) {
      constexpr int S = JP::slot_of[decltype(j)::value];
      load_slots<SH, (1u << S)>(it, kp, item);
    });
  }
}
template <class SH, int NF>
__device__ __forceinline__ void compact_first_eval(Item<SH>& it, const KParams& kp) {
  using W = typename SH::Where;
  using JP = typename SH::Probes;
  if constexpr (W::N > 0) {
    static_for<W::N>([&](auto j) { it.mask &= pred_bits<SH, decltype(j)::value>(it, kp); });
  } else {
    constexpr int NP = first_probes<SH, NF>();
    static_for<NP>([&](auto j) {
      constexpr int J = decltype(j)::value;
      constexpr int S = JP::slot_of[J];
      it.mask = probe_item(kp.probe[J], VGet<S>::get(it.v), it.mask, it.pay[J], false);
    });
  }
}

// K queued rows (has[k]: row k exists) as row 0 of K items: the probes stage
// by stage for all K rows (a first-stage probe again only when its payload is
// read), then the loads of the columns the sink reads.  ok[k] is false when a
// probe missed.
template <class SH, int K, int NF>
__device__ __forceinline__ void compact_load_rows(Item<SH> (&it)[K], bool (&ok)[K], const KParams& kp,
                                                  const uint32_t (&row)[K], const bool (&has)[K]) {
  using JP = typename SH::Probes;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    it[k].nvalid = 1;
    it[k].mask = 1u;
    ok[k] = has[k];
  }
  static_for<JP::N>([&](auto j) {
    constexpr int J = decltype(j)::value;
    constexpr int S = JP::slot_of[J];
    using T = typename At<S, typename SH::Cols::L>::type::T;
    if constexpr (compact_skip_probe<SH, NF, J>()) {
#pragma unroll
      for (int k = 0; k < K; ++k) it[k].pay[J][0] = 0;  // ran in the first stage, payload unread
    } else {
      T key[K];
#pragma unroll
      for (int k = 0; k < K; ++k) key[k] = ok[k] ? __ldg(static_cast<const T*>(kp.col[S]) + row[k]) : T(0);
#pragma unroll
      for (int k = 0; k < K; ++k) {
        VGet<S>::get(it[k].v)[0] = key[k];
        int32_t p = 0;
        if (ok[k]) ok[k] = probe_key(kp.probe[J], static_cast<int64_t>(key[k]), p);
        it[k].pay[J][0] = p;
      }
    }
  });
  static_for<SH::Cols::N>([&](auto c) {
    constexpr int S = decltype(c)::value;
    if constexpr ((compact_row_slots<SH, NF>() >> S) & 1u) {
      using T = typename At<S, typename SH::Cols::L>::type::T;
#pragma unroll
      for (int k = 0; k < K; ++k)
        if (ok[k]) VGet<S>::get(it[k].v)[0] = __ldg(static_cast<const T*>(kp.col[S]) + row[k]);
    }
  });
}

// Largest first_items compiled for a shape: 2 for pipelines whose first
// operation is a filter, 1 for probe-first ones (two items in flight were
// measured slower there: the probes' table lookups, not the key loads, bound
// them).
template <class SH>
constexpr int first_items_max() { return SH::Where::N > 0 ? 2 : 1; }

// The item loop of compacted execution (grid-stride, every lane of a warp
// runs every trip): the first operation over whole items, its surviving rows
// appended to the warp's queue q (queue_cap<K>() entries in shared memory),
// and each 32 * K queued rows handed K per lane to row_fn(rows, has) (lane l
// takes entries l, l + 32, ...); the rows left at the end follow.  All lanes of
// the warp call this together.  ALL_LANES: every lane calls row_fn at every
// drain, lanes without a row with has[] all false, so that row_fn may use warp
// collectives; otherwise only lanes holding a row call it.  FI (variant
// first_items): items a lane takes through the first stage per trip, their
// loads issued together before the first is evaluated; each item's survivors
// are appended and drained before the next, so the queue stays within
// queue_cap<K>().
template <class SH, int K, int NF, bool ALL_LANES = false, int FI = 1, class F>
__device__ __forceinline__ void for_rows_compacted(const KParams& kp, uint32_t* q, F&& row_fn) {
  constexpr int QC = queue_cap<K>();
  constexpr int KEEP = (QC - 32 * K + 31) / 32;  // entries a lane moves down after a drain
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  int qlen = 0;  // warp-uniform
  auto drain = [&](int n) {
    uint32_t rows[K];
    bool has[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      has[k] = lane + 32 * k < n;
      rows[k] = has[k] ? q[lane + 32 * k] : 0u;
    }
    if (ALL_LANES || has[0]) row_fn(rows, has);
    __syncwarp();
    uint32_t keep[KEEP];
#pragma unroll
    for (int i = 0; i < KEEP; ++i) {
      const int k = n + lane + 32 * i;
      keep[i] = k < qlen ? q[k] : 0u;
    }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < KEEP; ++i) {
      const int k = lane + 32 * i;
      if (k < qlen - n) q[k] = keep[i];
    }
    __syncwarp();
    qlen -= n;
  };
  const int64_t T = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t n_full = kp.n_rows >> 2;
  const int pf = kp.prefetch;
  const LanePrefetch<SH, first_stage_slots<SH>()> lp(kp, lane);
  // warp chunks (units of T items) pf trips ahead; trip 0 reads chunks 0 .. FI - 1
  for (int d = FI; d < pf * FI; ++d) lp.issue((t - lane) + d * T, n_full);
  for (int64_t wb = t - lane; wb < kp.n_items; wb += FI * T) {
    if (pf > 0) {
#pragma unroll
      for (int f = 0; f < FI; ++f) lp.issue(wb + static_cast<int64_t>(pf * FI + f) * T, n_full);
    }
    Item<SH> it[FI];
#pragma unroll
    for (int f = 0; f < FI; ++f) compact_first_load<SH, NF>(it[f], kp, wb + f * T + lane);
#pragma unroll
    for (int f = 0; f < FI; ++f) {
      compact_first_eval<SH, NF>(it[f], kp);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const bool live = (it[f].mask >> r) & 1u;
        const uint32_t b = __ballot_sync(0xffffffffu, live);
        if (live) q[qlen + __popc(b & lt)] = static_cast<uint32_t>((wb + f * T + lane) * 4 + r);
        qlen += __popc(b);
      }
      __syncwarp();
      while (qlen >= 32 * K) drain(32 * K);
    }
  }
  if (qlen > 0) drain(qlen);
}

}  // namespace pv
