// Non-template parts of HASH_AGGREGATE: cuckoo duplicate sweep, result
// extraction, and registration of the grouped shapes compiled in the
// k_group_*.cu translation units.
#include "k_group.cuh"

namespace pv {

__global__ void k_cuckoo_dedupe(const __grid_constant__ GroupOut g) {
  for (int64_t s = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; s < g.cap;
       s += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const unsigned long long key = __ldcg(g.keys + s);
    if (key == kEmpty64) continue;
    for (int f = 0; f < g.cuckoo_k; ++f) {
      const uint64_t p = ht_index(key, g.hash, g.seed[f], g.log2cap);
      if (__ldcg(g.keys + p) == key) {
        if (p != static_cast<uint64_t>(s)) g.keys[s] = kEmpty64;
        break;
      }
    }
  }
}

__global__ void k_extract(const __grid_constant__ GroupDesc gd, const __grid_constant__ GroupOut g) {
  pdl_wait();  // launched early behind the aggregation kernel
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t T = static_cast<int64_t>(gridDim.x) * blockDim.x;
  if (g.replicas > 1) extract_replicated(gd, g, t, T);
  else extract_slots(gd, g, t, T);
}

pv_status launch_dedupe_extract(const LaunchCfg& c, const GroupDesc& gd, const GroupOut& g, bool dedupe) {
  const int64_t total = g.cap + 1;
  const int64_t threads = g.replicas > 1 ? total * 32 : total;  // replicated: one warp per slot
  const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(c.sm_count * 8, (threads + 255) / 256)));
  kmark(c);
  cudaError_t e = cudaSuccess;
  if (dedupe) k_cuckoo_dedupe<<<grid, 256, 0, c.stream>>>(g);
  else if (c.mark) k_extract<<<grid, 256, 0, c.stream>>>(gd, g);  // timed: keep the kernels apart
  else e = pdl_launch(k_extract, dim3(grid), dim3(256), 0, c.stream, gd, g);
  kmark(c);
  if (e != cudaSuccess) return PV_ERR_CUDA;
  ++*c.launches;
  return cudaGetLastError() == cudaSuccess ? PV_OK : PV_ERR_CUDA;
}

void register_group_lowcard();
void register_group_keyval();
void register_group_keyval_f();
void register_group_star();
void register_group_join2();
void register_group_join2y();
void register_group_keys3();
void register_group_star3();
void register_group_q5();

void register_group_shapes() {
  register_group_lowcard();
  register_group_keyval();
  register_group_keyval_f();
  register_group_star();
  register_group_join2();
  register_group_join2y();
  register_group_keys3();
  register_group_star3();
  register_group_q5();
}

}  // namespace pv
