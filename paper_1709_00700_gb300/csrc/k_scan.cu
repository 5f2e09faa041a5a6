// Scan pipelines without a hash-aggregation sink:
//   AGGREGATE (ungrouped, Table 1; Section 7.3 aggregate fragment),
//   PROJECT single pass (Section 4.1 coarse-grained strategy, here with
//     warp-aggregated atomics on one output cursor),
//   PROJECT multi pass (Section 4.1 fine-grained strategy: a filter kernel
//     counts matches, a prefix sum yields unique write positions, a
//     projection kernel repeats filter and probes and writes).
#include <mutex>

#include "pv_eval.cuh"

namespace pv {

// ---------------------------------------------------------------------------
// AGGREGATE: per-thread accumulators (predicated mode folds every row with
// its flag as a 0/-1 mask, the multiplication of Section 6), warp shuffle
// reduction, one shared-memory pass per CTA, one atomic per CTA and
// aggregate; the last CTA decodes the result and re-zeroes the accumulators.
// ---------------------------------------------------------------------------
// CTA epilogue of the ungrouped aggregation: warp shuffles, one slot per warp
// in shared memory, one atomic per aggregate per CTA; the last CTA to finish
// decodes the MIN/MAX codes into the result and resets the accumulators.
template <class SH>
__device__ __forceinline__ void aggregate_epilogue(uint64_t (&acc)[SH::Aggs::N + 1], const AggOut& out) {
  using A = typename SH::Aggs;
  constexpr int NA = A::N;
  __shared__ unsigned long long red[32][NA + 1];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  static_for<NA + 1>([&](auto a) {
    constexpr int I = decltype(a)::value;
    constexpr int F = I < NA ? A::func_of[I < NA ? I : 0] : PV_COUNT;
    acc[I] = warp_reduce<F>(acc[I]);
  });
  if (lane == 0) {
#pragma unroll
    for (int a = 0; a <= NA; ++a) red[warp][a] = acc[a];
  }
  __syncthreads();
  if (warp == 0) {
    static_for<NA + 1>([&](auto a) {
      constexpr int I = decltype(a)::value;
      constexpr int F = I < NA ? A::func_of[I < NA ? I : 0] : PV_COUNT;
      uint64_t v = lane < nwarps ? red[lane][I] : 0;
      v = warp_reduce<F>(v);
      if (lane == 0 && v != 0) acc_atomic<F>(out.acc + I, v);
    });
  }
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(out.done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    const uint64_t rows = atomicExch(out.acc + NA, 0ull);
    static_for<NA>([&](auto a) {
      constexpr int I = decltype(a)::value;
      constexpr int F = A::func_of[I];
      const uint64_t c = atomicExch(out.acc + I, 0ull);
      int64_t v = static_cast<int64_t>(c);
      if constexpr (F == PV_MIN) v = rows ? decode_min(c) : 0;
      if constexpr (F == PV_MAX) v = rows ? decode_max(c) : 0;
      out.result[I] = v;
    });
    *out.done = 0;
  }
}

template <class SH, bool PRED, bool CHUNK, int U>
__global__ void __maxnreg__(128) k_aggregate(const __grid_constant__ KParams kp, const __grid_constant__ AggOut out) {
  using A = typename SH::Aggs;
  constexpr int NA = A::N;
  uint64_t acc[NA + 1];
#pragma unroll
  for (int a = 0; a <= NA; ++a) acc[a] = 0;

  auto consume = [&](Item<SH> (&it)[U]) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const uint32_t live = (it[u].mask >> r) & 1u;
        if constexpr (PRED) {
          const uint64_t m = 0ull - live;
          static_for<NA>([&](auto a) {
            constexpr int I = decltype(a)::value;
            using AG = typename At<I, typename A::L>::type;
            acc[I] = acc_combine<AG::func>(acc[I], acc_code<AG::func>(agg_value<AG>(it[u], kp, r)) & m);
          });
          acc[NA] += live;
        } else if (live) {
          static_for<NA>([&](auto a) {
            constexpr int I = decltype(a)::value;
            using AG = typename At<I, typename A::L>::type;
            acc[I] = acc_combine<AG::func>(acc[I], acc_code<AG::func>(agg_value<AG>(it[u], kp, r)));
          });
          acc[NA] += 1;
        }
      }
    }
  };
  if constexpr (PRED) {
    for_items_pipelined<SH, CHUNK, U>(kp, consume);
  } else {
    for_items_pf<SH, CHUNK, U, first_stage_slots<SH>()>(kp, [&](const int64_t (&idx)[U]) {
      Item<SH> it[U];
      eval_items<SH, PRED, U>(it, kp, idx);
      consume(it);
    });
  }

  aggregate_epilogue<SH>(acc, out);
}

// ---------------------------------------------------------------------------
// PROJECT helpers
// ---------------------------------------------------------------------------
template <class SH>
__device__ __forceinline__ void write_row(const ProjOut& out, Item<SH>& it, int r, int64_t pos) {
  using PJ = typename SH::Proj;
  static_for<PJ::N>([&](auto c) {
    constexpr int C = decltype(c)::value;
    constexpr int S = PJ::slot_of[C];
    if constexpr (S >= 0) {
      using T = typename At<S, typename SH::Cols::L>::type::T;
      static_cast<T*>(out.col[C])[pos] = VGet<S>::get(it.v)[r];
    } else {
      static_cast<int32_t*>(out.col[C])[pos] = it.pay[-S - 1][r];
    }
  });
}

__device__ __forceinline__ int warp_incl_scan(int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  return v;
}

// Block-wide exclusive scan of a 64-bit value; returns the prefix and sets
// *total.  Every thread of the block must call it.
__device__ __forceinline__ uint64_t block_excl_scan(uint64_t v, uint64_t* total) {
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
    uint64_t w = lane < nwarps ? ws[lane] : 0;
    uint64_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, static_cast<unsigned long long>(wi), o);
      if (lane >= o) wi += y;
    }
    if (lane < nwarps) ws[lane] = wi - w;
    if (lane == 31) ws[32] = wi;  // nwarps <= 32: lane 31 holds the grand total
  }
  __syncthreads();
  const uint64_t ex = ws[warp] + incl - v;
  *total = ws[32];
  __syncthreads();
  return ex;
}

// Single pass: every warp reserves its matches with one atomicAdd on the
// output cursor (ballot-free: counts are scanned with shuffles), then each
// lane writes its rows.  Output order is arbitrary across warps.
template <class SH, bool PRED, bool CHUNK, int U>
__global__ void __maxnreg__(128) k_project_sp(const __grid_constant__ KParams kp, const __grid_constant__ ProjOut out) {
  bool overflow = false;
  for_items_uniform<CHUNK, U>(kp.n_items, [&](const int64_t (&idx)[U]) {
    Item<SH> it[U];
    eval_items<SH, PRED, U>(it, kp, idx);
    int cnt = 0;
#pragma unroll
    for (int u = 0; u < U; ++u) cnt += __popc(it[u].mask);
    const int incl = warp_incl_scan(cnt);
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    if (total == 0) return;
    unsigned long long base = 0;
    if ((threadIdx.x & 31) == 31) base = atomicAdd(out.cursor, static_cast<unsigned long long>(total));
    base = __shfl_sync(0xffffffffu, base, 31);
    int64_t pos = static_cast<int64_t>(base) + incl - cnt;
#pragma unroll
    for (int u = 0; u < U; ++u) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        if ((it[u].mask >> r) & 1u) {
          if (pos < out.capacity) write_row<SH>(out, it[u], r, pos);
          else overflow = true;
          ++pos;
        }
      }
    }
  });
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
    const int64_t n = static_cast<int64_t>(atomicExch(out.cursor, 0ull));
    *out.count = n < out.capacity ? n : out.capacity;
    *out.done = 0;
  }
}

// Multi pass.  A tile is blockDim * U items.  Tiles go to CTAs grid-stride
// (coalesced) or as one contiguous range per CTA (chunked); inside a tile the
// item of (thread t, unroll u) is u * blockDim + t (coalesced) or t * U + u
// (chunked).  Count kernel and scatter kernel use the same mapping.
template <bool CHUNK, int U>
__device__ __forceinline__ void tile_items(int64_t tile, int64_t (&idx)[U]) {
  const int64_t base = tile * static_cast<int64_t>(blockDim.x) * U;
#pragma unroll
  for (int u = 0; u < U; ++u)
    idx[u] = CHUNK ? base + static_cast<int64_t>(threadIdx.x) * U + u
                   : base + static_cast<int64_t>(u) * blockDim.x + threadIdx.x;
}

template <bool CHUNK, class F>
__device__ __forceinline__ void for_tiles(int64_t n_tiles, F&& f) {
  if constexpr (!CHUNK) {
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) f(tile);
  } else {
    const int64_t per = (n_tiles + gridDim.x - 1) / gridDim.x;
    const int64_t b = blockIdx.x * per;
    const int64_t e = b + per < n_tiles ? b + per : n_tiles;
    for (int64_t tile = b; tile < e; ++tile) f(tile);
  }
}

template <class SH, bool PRED, bool CHUNK, int U>
__global__ void __maxnreg__(128) k_project_count(const __grid_constant__ KParams kp, const __grid_constant__ ProjOut out) {
  for_tiles<CHUNK>(out.n_tiles, [&](int64_t tile) {
    int64_t idx[U];
    tile_items<CHUNK, U>(tile, idx);
    Item<SH> it[U];
    eval_items<SH, PRED, U>(it, kp, idx);
    uint64_t cnt = 0;
#pragma unroll
    for (int u = 0; u < U; ++u) cnt += __popc(it[u].mask);
    uint64_t total;
    block_excl_scan(cnt, &total);
    if (threadIdx.x == 0) out.tile_count[tile] = static_cast<int64_t>(total);
  });
  pdl_launch_dependents();
}

// Exclusive prefix sum over the tile counts (one CTA of 1024 threads).
__global__ void __launch_bounds__(1024) k_tile_scan(const __grid_constant__ ProjOut out, int32_t* err) {
  pdl_wait();  // launched early behind the count kernel
  const int64_t n = out.n_tiles;
  const int64_t per = (n + blockDim.x - 1) / blockDim.x;
  const int64_t b = threadIdx.x * per;
  const int64_t e = b + per < n ? b + per : n;
  uint64_t s = 0;
  for (int64_t i = b; i < e; ++i) s += out.tile_count[i];
  uint64_t total;
  uint64_t run = block_excl_scan(s, &total);
  for (int64_t i = b; i < e; ++i) {
    out.tile_offset[i] = static_cast<int64_t>(run);
    run += out.tile_count[i];
  }
  pdl_launch_dependents();
  if (threadIdx.x == 0) {
    const int64_t t = static_cast<int64_t>(total);
    *out.count = t < out.capacity ? t : out.capacity;
    if (t > out.capacity) set_error(err, PV_ERR_OUTPUT_OVERFLOW);
  }
}

template <class SH, bool PRED, bool CHUNK, int U>
__global__ void __maxnreg__(128) k_project_scatter(const __grid_constant__ KParams kp, const __grid_constant__ ProjOut out) {
  static_assert(U <= 4, "16-bit scan fields hold at most 4 unroll slots");
  pdl_wait();  // launched early behind the scan kernel
  for_tiles<CHUNK>(out.n_tiles, [&](int64_t tile) {
    int64_t idx[U];
    tile_items<CHUNK, U>(tile, idx);
    Item<SH> it[U];
    eval_items<SH, PRED, U>(it, kp, idx);
    int64_t pos[U];
    const int64_t base = out.tile_offset[tile];
    if constexpr (CHUNK) {
      // row order inside the tile: (thread, u, row)
      uint64_t c = 0;
#pragma unroll
      for (int u = 0; u < U; ++u) c += __popc(it[u].mask);
      uint64_t total;
      int64_t p = base + static_cast<int64_t>(block_excl_scan(c, &total));
#pragma unroll
      for (int u = 0; u < U; ++u) { pos[u] = p; p += __popc(it[u].mask); }
    } else {
      // row order inside the tile: (u, thread, row); one scan of U packed
      // 16-bit counters (each at most 4 * 1024 per tile)
      uint64_t packed = 0;
#pragma unroll
      for (int u = 0; u < U; ++u) packed |= static_cast<uint64_t>(__popc(it[u].mask)) << (16 * u);
      uint64_t total;
      const uint64_t ex = block_excl_scan(packed, &total);
      int64_t before = 0;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        pos[u] = base + before + static_cast<int64_t>((ex >> (16 * u)) & 0xFFFF);
        before += static_cast<int64_t>((total >> (16 * u)) & 0xFFFF);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      int64_t p = pos[u];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        if ((it[u].mask >> r) & 1u) {
          if (p < out.capacity) write_row<SH>(out, it[u], r, p);
          ++p;
        }
      }
    }
  });
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
// Compacted execution of an ungrouped aggregation: the rows that survive the
// first operation are queued per warp and accumulated one per lane.
template <class SH, int K, int FI>
__global__ void __maxnreg__(128) k_aggregate_compact(const __grid_constant__ KParams kp,
                                                     const __grid_constant__ AggOut out) {
  using A = typename SH::Aggs;
  constexpr int NA = A::N;
  extern __shared__ uint32_t qmem[];
  uint64_t acc[NA + 1];
#pragma unroll
  for (int a = 0; a <= NA; ++a) acc[a] = 0;
  for_rows_compacted<SH, K, 1, false, FI>(kp, qmem + (threadIdx.x >> 5) * queue_cap<K>(),
                            [&](const uint32_t (&rows)[K], const bool (&has)[K]) {
    Item<SH> it[K];
    bool ok[K];
    compact_load_rows<SH, K, 1>(it, ok, kp, rows, has);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (!ok[k]) continue;
      static_for<NA>([&](auto a) {
        constexpr int I = decltype(a)::value;
        using AG = typename At<I, typename A::L>::type;
        acc[I] = acc_combine<AG::func>(acc[I], acc_code<AG::func>(agg_value<AG>(it[k], kp, 0)));
      });
      acc[NA] += 1;
    }
  });
  aggregate_epilogue<SH>(acc, out);
}

// Bytes of one projected row before projected column C (source column types;
// payloads are int32); proj_offset<SH, N> is the whole row.
template <class SH, int C>
constexpr int proj_offset() {
  if constexpr (C == 0) {
    return 0;
  } else {
    constexpr int S = SH::Proj::slot_of[C - 1];
    constexpr int sz = S >= 0 ? static_cast<int>(sizeof(typename At<(S >= 0 ? S : 0), typename SH::Cols::L>::type::T)) : 4;
    return proj_offset<SH, C - 1>() + sz;
  }
}

// Output rows a warp stages in shared memory before it reserves their
// positions: a flush starts at 64 rows, and one drain adds at most 32 * K.
template <int K>
__host__ __device__ constexpr int out_stage_rows() { return 32 * (2 + K); }
template <class SH, int K>
__host__ __device__ constexpr size_t out_stage_bytes() {
  return (static_cast<size_t>(out_stage_rows<K>()) * proj_offset<SH, SH::Proj::N>() + 15) & ~size_t(15);
}

// Row `slot` of a warp's output stage (column C at stage + rows * offset(C)).
template <class SH, int K>
__device__ __forceinline__ void stage_out_row(char* st, int slot, Item<SH>& it) {
  using PJ = typename SH::Proj;
  static_for<PJ::N>([&](auto c) {
    constexpr int C = decltype(c)::value;
    constexpr int S = PJ::slot_of[C];
    char* col = st + out_stage_rows<K>() * proj_offset<SH, C>();
    if constexpr (S >= 0) {
      using T = typename At<S, typename SH::Cols::L>::type::T;
      reinterpret_cast<T*>(col)[slot] = VGet<S>::get(it.v)[0];
    } else {
      reinterpret_cast<int32_t*>(col)[slot] = it.pay[-S - 1][0];
    }
  });
}

// The warp's n staged rows to the output at positions reserved with one
// atomicAdd; rows past the capacity are dropped (overflow).  All lanes.
template <class SH, int K>
__device__ __forceinline__ void flush_out_rows(const char* st, int n, const ProjOut& out, bool& overflow) {
  using PJ = typename SH::Proj;
  const int lane = threadIdx.x & 31;
  __syncwarp();
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(out.cursor, static_cast<unsigned long long>(n));
  base = __shfl_sync(0xffffffffu, base, 0);
  for (int i = lane; i < n; i += 32) {
    const int64_t pos = static_cast<int64_t>(base) + i;
    if (pos >= out.capacity) {
      overflow = true;
      continue;
    }
    static_for<PJ::N>([&](auto c) {
      constexpr int C = decltype(c)::value;
      constexpr int S = PJ::slot_of[C];
      const char* col = st + out_stage_rows<K>() * proj_offset<SH, C>();
      if constexpr (S >= 0) {
        using T = typename At<S, typename SH::Cols::L>::type::T;
        static_cast<T*>(out.col[C])[pos] = reinterpret_cast<const T*>(col)[i];
      } else {
        static_cast<int32_t*>(out.col[C])[pos] = reinterpret_cast<const int32_t*>(col)[i];
      }
    });
  }
  __syncwarp();
}

// Compacted single-pass PROJECT: the rows that survive the first operation
// are queued per warp; at each drain every lane takes its queued rows through
// the rest of the pipeline, and the rows that survive are appended to the
// warp's output stage in shared memory (ballot + popc).  Once 64 or more are
// staged the warp reserves their output positions with one atomicAdd and
// writes them out coalesced: one atomic per 64 to 127 output rows, where one
// per drain put the whole grid on one counter.  Output order is arbitrary, as
// for the other single-pass projection.  Held to 48 registers (none of the
// compiled projections spills there): five 256-thread or two 512-thread CTAs
// per SM, more warps to hide the gathers' latency (the best variant of the
// 100M-row filter/project measured 171.7 us against 185.9 us at 128).
template <class SH, int K, int FI>
__global__ void __maxnreg__(48) k_project_compact(const __grid_constant__ KParams kp,
                                                   const __grid_constant__ ProjOut out) {
  extern __shared__ uint32_t qmem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  char* ost = reinterpret_cast<char*>(qmem + nwarps * queue_cap<K>()) + warp * out_stage_bytes<SH, K>();
  bool overflow = false;
  int staged = 0;  // warp-uniform
  for_rows_compacted<SH, K, 1, true, FI>(kp, qmem + warp * queue_cap<K>(),
                                     [&](const uint32_t (&rows)[K], const bool (&has)[K]) {
    Item<SH> it[K];
    bool ok[K];
    compact_load_rows<SH, K, 1>(it, ok, kp, rows, has);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const unsigned b = __ballot_sync(0xffffffffu, ok[k]);
      if (ok[k]) stage_out_row<SH, K>(ost, staged + __popc(b & ((1u << lane) - 1u)), it[k]);
      staged += __popc(b);
    }
    if (staged >= 64) {
      flush_out_rows<SH, K>(ost, staged, out, overflow);
      staged = 0;
    }
  });
  if (staged > 0) flush_out_rows<SH, K>(ost, staged, out, overflow);
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
    const int64_t n = static_cast<int64_t>(atomicExch(out.cursor, 0ull));
    *out.count = n < out.capacity ? n : out.capacity;
    *out.done = 0;
  }
}

template <class SH, int K>
static pv_status launch_proj_compact_k(const LaunchCfg& c, const KParams& kp, const ProjOut& out) {
  auto k = c.first_items == 2 ? k_project_compact<SH, K, first_items_max<SH>()> : k_project_compact<SH, K, 1>;
  const size_t smem = static_cast<size_t>(c.block / 32) * (queue_cap<K>() * 4 + out_stage_bytes<SH, K>());
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess)
    return PV_ERR_UNSUPPORTED;
  const int grid = grid_for(c, reinterpret_cast<const void*>(k), smem, kp.n_items, c.block);
  if (grid <= 0) return PV_ERR_UNSUPPORTED;
  kmark(c);
  k<<<grid, c.block, smem, c.stream>>>(kp, out);
  kmark(c);
  ++*c.launches;
  return cudaGetLastError() == cudaSuccess ? PV_OK : PV_ERR_CUDA;
}

template <class SH>
static pv_status launch_proj_compact(const LaunchCfg& c, const KParams& kp, const ProjOut& out, int exec) {
  if constexpr (SH::Where::N == 0 && SH::Probes::N == 0) {
    return PV_ERR_UNSUPPORTED;  // nothing to compact on
  } else {
    // single pass only: the queues reorder rows, and multi-pass output keeps input order
    if (exec != PV_EXEC_SINGLE_PASS || c.chunk || (c.U != 1 && c.U != 2) ||
        kp.n_rows > static_cast<int64_t>(UINT32_MAX) || c.first_items > first_items_max<SH>())
      return PV_ERR_UNSUPPORTED;
    return c.U == 2 ? launch_proj_compact_k<SH, 2>(c, kp, out) : launch_proj_compact_k<SH, 1>(c, kp, out);
  }
}

template <class SH, int K>
static pv_status launch_agg_compact_k(const LaunchCfg& c, const KParams& kp, const AggOut& out) {
  auto k = c.first_items == 2 ? k_aggregate_compact<SH, K, first_items_max<SH>()> : k_aggregate_compact<SH, K, 1>;
  const size_t smem = static_cast<size_t>(c.block / 32) * queue_cap<K>() * 4;
  const int grid = grid_for(c, reinterpret_cast<const void*>(k), smem, kp.n_items, c.block);
  if (grid <= 0) return PV_ERR_UNSUPPORTED;
  kmark(c);
  k<<<grid, c.block, smem, c.stream>>>(kp, out);
  kmark(c);
  ++*c.launches;
  return cudaGetLastError() == cudaSuccess ? PV_OK : PV_ERR_CUDA;
}

template <class SH>
static pv_status launch_agg_compact(const LaunchCfg& c, const KParams& kp, const AggOut& out) {
  if constexpr (SH::Where::N == 0 && SH::Probes::N == 0) {
    return PV_ERR_UNSUPPORTED;  // nothing to compact on
  } else {
    // items_per_thread: queued rows a lane takes through the row stage at once
    if (c.chunk || (c.U != 1 && c.U != 2) || kp.n_rows > static_cast<int64_t>(UINT32_MAX) ||
        c.first_items > first_items_max<SH>())
      return PV_ERR_UNSUPPORTED;
    return c.U == 2 ? launch_agg_compact_k<SH, 2>(c, kp, out) : launch_agg_compact_k<SH, 1>(c, kp, out);
  }
}

template <class SH, bool P, bool C, int U>
static pv_status launch_agg_t(const LaunchCfg& c, const KParams& kp, const AggOut& out) {
  auto k = k_aggregate<SH, P, C, U>;
  const int grid = grid_for(c, reinterpret_cast<const void*>(k), 0, kp.n_items, static_cast<int64_t>(c.block) * U);
  if (grid <= 0) return PV_ERR_UNSUPPORTED;
  kmark(c);
  k<<<grid, c.block, 0, c.stream>>>(kp, out);
  kmark(c);
  ++*c.launches;
  return cudaGetLastError() == cudaSuccess ? PV_OK : PV_ERR_CUDA;
}

pv_status launch_tile_scan(const LaunchCfg& c, const ProjOut& out, int32_t* err) {
  kmark(c);
  cudaError_t e = c.mark ? (k_tile_scan<<<1, 1024, 0, c.stream>>>(out, err), cudaSuccess)
                         : pdl_launch(k_tile_scan, dim3(1), dim3(1024), 0, c.stream, out, err);
  kmark(c);
  ++*c.launches;
  return e == cudaSuccess && cudaGetLastError() == cudaSuccess ? PV_OK : PV_ERR_CUDA;
}

template <class SH, bool P, bool C, int U>
static pv_status launch_proj_t(const LaunchCfg& c, const KParams& kp, const ProjOut& out, int exec) {
  if (exec == PV_EXEC_SINGLE_PASS) {
    auto k = k_project_sp<SH, P, C, U>;
    const int grid = grid_for(c, reinterpret_cast<const void*>(k), 0, kp.n_items, static_cast<int64_t>(c.block) * U);
    if (grid <= 0) return PV_ERR_UNSUPPORTED;
    kmark(c);
    k<<<grid, c.block, 0, c.stream>>>(kp, out);
    kmark(c);
    ++*c.launches;
  } else {
    auto kc = k_project_count<SH, P, C, U>;
    auto ks = k_project_scatter<SH, P, C, U>;
    const int grid = grid_for(c, reinterpret_cast<const void*>(kc), 0, out.n_tiles, 1);
    if (grid <= 0 || grid_for(c, reinterpret_cast<const void*>(ks), 0, 1, 1) <= 0) return PV_ERR_UNSUPPORTED;
    kmark(c);
    kc<<<grid, c.block, 0, c.stream>>>(kp, out);
    kmark(c);
    kmark(c);
    cudaError_t e1 = c.mark ? (k_tile_scan<<<1, 1024, 0, c.stream>>>(out, kp.err), cudaSuccess)
                            : pdl_launch(k_tile_scan, dim3(1), dim3(1024), 0, c.stream, out, kp.err);
    kmark(c);
    kmark(c);
    cudaError_t e2 = c.mark ? (ks<<<grid, c.block, 0, c.stream>>>(kp, out), cudaSuccess)
                            : pdl_launch(ks, dim3(grid), dim3(c.block), 0, c.stream, kp, out);
    kmark(c);
    *c.launches += 3;
    if (e1 != cudaSuccess || e2 != cudaSuccess) return PV_ERR_CUDA;
  }
  return cudaGetLastError() == cudaSuccess ? PV_OK : PV_ERR_CUDA;
}

template <class SH>
static pv_status launch_agg(const LaunchCfg& c, const KParams& kp, const AggOut& out) {
  using F = pv_status (*)(const LaunchCfg&, const KParams&, const AggOut&);
  static const F tab[2][2][3] = {
      {{launch_agg_t<SH, false, false, 1>, launch_agg_t<SH, false, false, 2>, launch_agg_t<SH, false, false, 4>},
       {launch_agg_t<SH, false, true, 1>, launch_agg_t<SH, false, true, 2>, launch_agg_t<SH, false, true, 4>}},
      {{launch_agg_t<SH, true, false, 1>, launch_agg_t<SH, true, false, 2>, launch_agg_t<SH, true, false, 4>},
       {launch_agg_t<SH, true, true, 1>, launch_agg_t<SH, true, true, 2>, launch_agg_t<SH, true, true, 4>}}};
  if (c.compact) return c.compact_probes != 1 ? PV_ERR_UNSUPPORTED : launch_agg_compact<SH>(c, kp, out);
  const int ui = c.U == 1 ? 0 : c.U == 2 ? 1 : c.U == 4 ? 2 : -1;
  if (ui < 0) return PV_ERR_UNSUPPORTED;
  return tab[c.pred][c.chunk][ui](c, kp, out);
}

template <class SH>
static pv_status launch_proj(const LaunchCfg& c, const KParams& kp, const ProjOut& out, int exec) {
  using F = pv_status (*)(const LaunchCfg&, const KParams&, const ProjOut&, int);
  static const F tab[2][2][3] = {
      {{launch_proj_t<SH, false, false, 1>, launch_proj_t<SH, false, false, 2>, launch_proj_t<SH, false, false, 4>},
       {launch_proj_t<SH, false, true, 1>, launch_proj_t<SH, false, true, 2>, launch_proj_t<SH, false, true, 4>}},
      {{launch_proj_t<SH, true, false, 1>, launch_proj_t<SH, true, false, 2>, launch_proj_t<SH, true, false, 4>},
       {launch_proj_t<SH, true, true, 1>, launch_proj_t<SH, true, true, 2>, launch_proj_t<SH, true, true, 4>}}};
  if (c.compact) return c.compact_probes != 1 ? PV_ERR_UNSUPPORTED : launch_proj_compact<SH>(c, kp, out, exec);
  const int ui = c.U == 1 ? 0 : c.U == 2 ? 1 : c.U == 4 ? 2 : -1;
  if (ui < 0) return PV_ERR_UNSUPPORTED;
  return tab[c.pred][c.chunk][ui](c, kp, out, exec);
}

template <class SH>
static void reg_aggregate() {
  ShapeEntry e{};
  e.sig = SH::signature();
  e.mode = MODE_AGGREGATE;
  e.aggregate = launch_agg<SH>;
  register_shape(e);
}
template <class SH>
static void reg_project() {
  ShapeEntry e{};
  e.sig = SH::signature();
  e.mode = MODE_PROJECT;
  e.project = launch_proj<SH>;
  register_shape(e);
}

// ---- compiled shapes -------------------------------------------------------
// Filter/aggregate/project table (a int32, b int32, price int64):
//   WHERE range(a) AND range(b) -> SUM(price), COUNT(*)   |   -> (a, price)
using ShFilterAgg = Shape<Cols<TI32, TI32, TI64>, Where<P<0>, P<1>>, Probes<>, Key<>,
                          Aggs<Sum<Mul<X<2>>>, Count>, Proj<>>;
using ShFilterProj = Shape<Cols<TI32, TI32, TI64>, Where<P<0>, P<1>>, Probes<>, Key<>, Aggs<>, Proj<0, 2>>;
// Same table, one predicate (projection query with a single filter).
using ShFilterProj1 = Shape<Cols<TI32, TI32, TI64>, Where<P<0>>, Probes<>, Key<>, Aggs<>, Proj<1, 2>>;
// Ungrouped fixed-point aggregation of the low-cardinality table (all 8
// aggregates, no grouping) — the totals of the grouped query.
using ShLowcardTotals =
    Shape<Cols<TI32, TI64, TI64, TI64, TI64>, Where<P<0>>, Probes<>, Key<>,
          Aggs<Sum<Mul<X<1>>>, Sum<Mul<X<2>>>, Sum<Mul<X<3>>>, Sum<Mul<X<4>>>, Sum<Mul<X<2>, CMX<3, 0>>>,
               Sum<Mul<X<2>, CMX<3, 1>, XPC<4, 2>>>, Sum<Mul<X<1>, X<2>>>, Count>,
          Proj<>>;
// key/value table: filtered SUM/COUNT/MIN/MAX of val.
using ShKeyValTotals = Shape<Cols<TI64>, Where<P<0>>, Probes<>, Key<>,
                             Aggs<Sum<Mul<X<0>>>, Count, Min<Mul<X<0>>>, Max<Mul<X<0>>>>, Proj<>>;

// One probe, COUNT(*) of the joining rows (join cardinality).
using ShJoinCount = Shape<Cols<TI32>, Where<>, Probes<0>, Key<>, Aggs<Count>, Proj<>>;
// Join then project: the probe's payload beside a fact column, without and
// with a fact filter in front (Table 2's pipeline shape ending in PROJECT).
using ShJoinProj = Shape<Cols<TI32, TI64>, Where<>, Probes<0>, Key<>, Aggs<>, Proj<-1, 1>>;
using ShFilterJoinProj = Shape<Cols<TI32, TI32, TI64>, Where<P<0>>, Probes<1>, Key<>, Aggs<>, Proj<-1, 2>>;

// The projection steps of the TPC-H Q5-shaped multi-pipeline query: rows
// that pass a probe, projected with their probe key (customers of the
// selected nations: key, nation), and rows that pass a filter and a probe,
// projected with the payload the probe binds (orders of the year: key, the
// customer's nation).
using ShProbeProjKey = Shape<Cols<TI32, TI32>, Where<>, Probes<0>, Key<>, Aggs<>, Proj<1, 0>>;
using ShFilterProbeProjPay = Shape<Cols<TI32, TI32, TI32>, Where<P<0>>, Probes<1>, Key<>, Aggs<>, Proj<2, -1>>;

void register_scan_shapes() {
  reg_project<ShProbeProjKey>();
  reg_project<ShFilterProbeProjPay>();
  reg_aggregate<ShJoinCount>();
  reg_aggregate<ShFilterAgg>();
  reg_project<ShFilterProj>();
  reg_project<ShFilterProj1>();
  reg_project<ShJoinProj>();
  reg_project<ShFilterJoinProj>();
  reg_aggregate<ShLowcardTotals>();
  reg_aggregate<ShKeyValTotals>();
}

// ---------------------------------------------------------------------------
// Allocation-free multi-pass projection.  Same kernels as the multi-pass
// PROJECT above (fixed launch shape: 256 threads, 4 items per thread,
// branched, coalesced), but its scratch -- the error word and the per-tile
// match counts and write offsets -- lives in one file-scope device array
// instead of memory from an allocator.  Every GPU that loads this library
// holds the array until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr int kNoAllocBlock = 256;
constexpr int kNoAllocU = 4;
constexpr int64_t kNoAllocTileRows = 4LL * kNoAllocBlock * kNoAllocU;
constexpr int64_t kNoAllocMaxTiles = (PV_NOALLOC_MAX_ROWS + kNoAllocTileRows - 1) / kNoAllocTileRows;
constexpr int64_t kNoAllocHeader = 32;  // words: [0] error word (int32), rest unused padding

// Scratch of every call: header, then tile counts, then tile offsets (int64).
__device__ __align__(256) int64_t g_noalloc_scratch[kNoAllocHeader + 2 * kNoAllocMaxTiles];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
int64_t* g_noalloc_addr[kNoAllocMaxDevices];  // device address of the array, per device
int g_noalloc_sms[kNoAllocMaxDevices];

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached.
pv_status noalloc_scratch(int64_t** addr, int* sms) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return PV_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return PV_ERR_CUDA;
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PV_ERR_CUDA;
    g_noalloc_addr[dev] = static_cast<int64_t*>(p);
    g_noalloc_sms[dev] = n;
  }
  *addr = g_noalloc_addr[dev];
  *sms = g_noalloc_sms[dev];
  return PV_OK;
}

void clamp_i32_range(int64_t& lo, int64_t& hi) {
  if (lo > hi) { lo = 1; hi = 0; return; }
  lo = lo < INT32_MIN ? INT32_MIN : lo;
  hi = hi > INT32_MAX ? INT32_MAX : hi;
  if (lo > hi) { lo = 1; hi = 0; }
}

}  // namespace
}  // namespace pv

extern "C" pv_status pv_filter_project_noalloc(const int32_t* a, const int32_t* b, const int64_t* price,
                                                int64_t n_rows, int64_t a_lo, int64_t a_hi, int64_t b_lo,
                                                int64_t b_hi, int32_t* out_a, int64_t* out_price,
                                                int64_t out_capacity, int64_t* out_count, int32_t* out_status,
                                                void* stream) {
  using namespace pv;
  if (n_rows < 0 || n_rows > PV_NOALLOC_MAX_ROWS || out_capacity < 0) return PV_ERR_INVALID_ARG;
  if (!out_count || !out_status) return PV_ERR_INVALID_ARG;
  if (n_rows > 0 && (!a || !b || !price)) return PV_ERR_INVALID_ARG;
  if (out_capacity > 0 && (!out_a || !out_price)) return PV_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b) | reinterpret_cast<uintptr_t>(price)) % 16)
    return PV_ERR_INVALID_ARG;
  int64_t* scratch = nullptr;
  int sms = 0;
  pv_status st = noalloc_scratch(&scratch, &sms);
  if (st != PV_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  KParams kp{};
  kp.n_rows = n_rows;
  kp.n_items = (n_rows + 3) / 4;
  kp.col[0] = a;
  kp.col[1] = b;
  kp.col[2] = price;
  clamp_i32_range(a_lo, a_hi);
  clamp_i32_range(b_lo, b_hi);
  kp.lo[0] = a_lo;
  kp.hi[0] = a_hi;
  kp.lo[1] = b_lo;
  kp.hi[1] = b_hi;
  kp.err = reinterpret_cast<int32_t*>(scratch);
  ProjOut out{};
  out.col[0] = out_a;
  out.col[1] = out_price;
  out.capacity = out_capacity;
  out.count = out_count;
  out.n_tiles = (kp.n_items + kNoAllocBlock * kNoAllocU - 1) / (kNoAllocBlock * kNoAllocU);
  if (out.n_tiles < 1) out.n_tiles = 1;
  out.tile_count = scratch + kNoAllocHeader;
  out.tile_offset = scratch + kNoAllocHeader + kNoAllocMaxTiles;
  // the array keeps the previous call's contents: clear the error word
  if (cudaMemsetAsync(scratch, 0, sizeof(int32_t), s) != cudaSuccess) return PV_ERR_CUDA;
  int launches = 0;
  LaunchCfg c{};
  c.stream = s;
  c.sm_count = sms;
  c.block = kNoAllocBlock;
  c.U = kNoAllocU;
  c.launches = &launches;
  st = launch_proj_t<ShFilterProj, false, false, kNoAllocU>(c, kp, out, PV_EXEC_MULTI_PASS);
  if (st != PV_OK) return st;
  if (cudaMemcpyAsync(out_status, scratch, sizeof(int32_t), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return PV_ERR_CUDA;
  return PV_OK;
}
