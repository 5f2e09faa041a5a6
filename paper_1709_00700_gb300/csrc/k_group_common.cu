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

__device__ __forceinline__ int64_t decode_agg(int func, uint64_t c) {
  if (func == PV_MIN) return decode_min(c);
  if (func == PV_MAX) return decode_max(c);
  return static_cast<int64_t>(c);
}

// Warp-uniform sweep over the cap + 1 slots; non-empty slots are appended to
// the result columns with one atomicAdd per warp, then cleared.
__global__ void k_extract(const __grid_constant__ GroupDesc gd, const __grid_constant__ GroupOut g) {
  const int64_t total = g.cap + 1;
  const int lane = threadIdx.x & 31;
  const int64_t T = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const bool perfect = g.ht == PV_HT_PERFECT;
  const int na = gd.n_aggs;
  for (int64_t wb = t - lane; wb < total; wb += T) {
    const int64_t s = wb + lane;
    bool occ = false, dirty = false;
    uint64_t key = kEmpty64;
    unsigned long long* v = g.vals + s * g.stride;
    if (s < total) {
      if (perfect) {
        occ = s < g.cap && v[gd.count_word] != 0;
        dirty = occ;
      } else if (s < g.cap) {
        key = g.keys[s];
        dirty = key != kEmpty64;
        occ = dirty && v[gd.count_word] != 0;
      } else {
        occ = dirty = v[gd.count_word] != 0;
      }
    }
    const unsigned ball = __ballot_sync(0xffffffffu, occ);
    unsigned long long base = 0;
    if (lane == 0 && ball) base = atomicAdd(g.out_count, static_cast<unsigned long long>(__popc(ball)));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (occ) {
      const int64_t pos = static_cast<int64_t>(base) + __popc(ball & ((1u << lane) - 1u));
      if (pos < g.out_cap) {
        int64_t k0, k1 = 0;
        if (perfect) {
          if (gd.n_keys == 1) {
            k0 = gd.key_min[0] + s;
          } else {
            k0 = gd.key_min[0] + s / gd.key_span[1];
            k1 = gd.key_min[1] + s % gd.key_span[1];
          }
        } else if (gd.n_keys == 1) {
          k0 = gd.key64[0] ? static_cast<int64_t>(key) : static_cast<int64_t>(static_cast<int32_t>(static_cast<uint32_t>(key)));
        } else {
          k0 = static_cast<int32_t>(static_cast<uint32_t>(key >> 32));
          k1 = static_cast<int32_t>(static_cast<uint32_t>(key));
        }
        g.out[pos] = k0;
        if (gd.n_keys == 2) g.out[g.out_cap + pos] = k1;
        for (int a = 0; a < na; ++a) g.out[(gd.n_keys + a) * g.out_cap + pos] = decode_agg(gd.func[a], v[a]);
      }
    }
    if (dirty) {
      for (int a = 0; a <= na; ++a) v[a] = 0;
      if (!perfect && s < g.cap) g.keys[s] = kEmpty64;
    }
  }
}

pv_status launch_dedupe_extract(const LaunchCfg& c, const GroupDesc& gd, const GroupOut& g, bool dedupe) {
  const int64_t total = g.cap + 1;
  const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(c.sm_count * 8, (total + 255) / 256)));
  kmark(c);
  if (dedupe) k_cuckoo_dedupe<<<grid, 256, 0, c.stream>>>(g);
  else k_extract<<<grid, 256, 0, c.stream>>>(gd, g);
  kmark(c);
  ++*c.launches;
  return cudaGetLastError() == cudaSuccess ? PV_OK : PV_ERR_CUDA;
}

void register_group_lowcard();
void register_group_keyval();
void register_group_keyval_f();
void register_group_star();
void register_group_join2();

void register_group_shapes() {
  register_group_lowcard();
  register_group_keyval();
  register_group_keyval_f();
  register_group_star();
  register_group_join2();
}

}  // namespace pv
