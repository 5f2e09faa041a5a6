// Stagewise evaluation of the LOOP body over U items per thread and the
// warp-uniform item loop, shared by the scan and the grouped kernels.
#pragma once

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
    for (int u = 0; u < U; ++u) {
      auto& fk = VGet<S>::get(it[u].v);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        it[u].pay[J][r] = 0;
        if (PRED || ((it[u].mask >> r) & 1u)) {
          int32_t p = 0;
          const bool hit = probe_key(kp.probe[J], static_cast<int64_t>(fk[r]), p);
          it[u].pay[J][r] = p;
          if (!hit) it[u].mask &= ~(1u << r);
        }
      }
    }
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

}  // namespace pv
