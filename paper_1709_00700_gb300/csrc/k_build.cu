// Build pipelines: LOOP over a dimension table, FILTER, HASH_PUT of key ->
// payload (Table 1, Table 2) into one of three table implementations
// (Section 5.1 linear probing and cuckoo hashing; perfect array for a dense
// key domain).  Build and probe share the table layout of DevHT.
#include <algorithm>

#include "pv_build.h"
#include "pv_internal.h"

namespace pv {

__device__ __forceinline__ int64_t load_any(const void* p, int type, int64_t r) {
  if (type == PV_I32) return static_cast<const int32_t*>(p)[r];
  if (type == PV_I64) return static_cast<const int64_t*>(p)[r];
  return static_cast<const uint8_t*>(p)[r];
}

__device__ __forceinline__ uint64_t cuckoo_pos(const DevHT& h, uint32_t k32, int f) {
  return ht_index(k32, h.hash, h.seed[f], h.log2cap);
}

// Linear probing insert of a unique key: claim the first empty slot of the
// probe sequence with a CAS; meeting the key itself means a duplicate.
__device__ __forceinline__ void linear_put(const DevHT& h, uint32_t k32, uint64_t val, int32_t* err) {
  unsigned long long* slots = reinterpret_cast<unsigned long long*>(h.slots);
  const uint64_t mask = static_cast<uint64_t>(h.cap) - 1;
  uint64_t idx = ht_index(k32, h.hash, h.seed[0], h.log2cap);
  for (int64_t step = 0; step < h.cap; ++step) {
    unsigned long long cur = slots[idx];
    while (static_cast<uint32_t>(cur >> 32) == kEmpty32) {
      const unsigned long long old = atomicCAS(slots + idx, cur, static_cast<unsigned long long>(val));
      if (old == cur) return;
      cur = old;
    }
    if (static_cast<uint32_t>(cur >> 32) == k32) {
      set_error(err, PV_ERR_DUP_BUILD_KEY);
      return;
    }
    idx = (idx + 1) & mask;
  }
  set_error(err, PV_ERR_HT_FULL);
}

// Cuckoo insert (one slot per bucket, k hash functions): take any empty
// candidate slot; otherwise swap into the candidate of the next function in
// turn and continue with the evicted element, at most max_evictions times.
__device__ __forceinline__ void cuckoo_put(const DevHT& h, uint64_t val, int max_evictions, int32_t* err) {
  unsigned long long* slots = reinterpret_cast<unsigned long long*>(h.slots);
  unsigned long long cur = val;
  int f = 0;
  for (int e = 0; e <= max_evictions; ++e) {
    const uint32_t k32 = static_cast<uint32_t>(cur >> 32);
    for (int i = 0; i < h.k; ++i) {
      const uint64_t p = cuckoo_pos(h, k32, i);
      unsigned long long s = slots[p];
      if (static_cast<uint32_t>(s >> 32) == kEmpty32 && atomicCAS(slots + p, s, cur) == s) return;
    }
    const uint64_t p = cuckoo_pos(h, k32, f);
    const unsigned long long old = atomicExch(slots + p, cur);
    if (static_cast<uint32_t>(old >> 32) == kEmpty32) return;
    cur = old;
    // continue with the evicted key from the function after the one that
    // placed it at p
    const uint32_t ok = static_cast<uint32_t>(cur >> 32);
    int placed = 0;
    for (int i = 0; i < h.k; ++i)
      if (cuckoo_pos(h, ok, i) == p) { placed = i; break; }
    f = (placed + 1) % h.k;
  }
  set_error(err, PV_ERR_CUCKOO_CYCLE);
}

// One payload column: the slot holds its value.  Two or more: the slot holds
// the build row, and probes gather the payload values from the columns.
// Payload statistics (minimum and maximum of every payload column over the
// surviving rows) feed the perfect-array domains of group keys on payloads.
__global__ void k_build(const __grid_constant__ BuildParams bp) {
  const BuildInput& in = bp.in;
  const DevHT& h = bp.ht;
  unsigned long long* slots = reinterpret_cast<unsigned long long*>(h.slots);
  int64_t n = in.n_rows;
  if (in.n_dyn != nullptr) {
    const unsigned long long d = __ldcg(in.n_dyn);
    n = d < static_cast<unsigned long long>(n) ? static_cast<int64_t>(d) : n;
  }
  uint64_t pmax[PV_MAX_PAYLOAD], pmin[PV_MAX_PAYLOAD];
#pragma unroll
  for (int i = 0; i < PV_MAX_PAYLOAD; ++i) pmax[i] = pmin[i] = 0;
  for (int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; r < n;
       r += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    bool pass = true;
    for (int i = 0; i < in.n_preds && pass; ++i) {
      const int64_t v = load_any(in.pred_col[i], in.pred_type[i], r);
      pass = in.lo[i] <= v && v <= in.hi[i];
    }
    if (!pass) continue;
    const int64_t key = load_any(in.key, in.key_type, r);
    int32_t pay = 0;
#pragma unroll
    for (int i = 0; i < PV_MAX_PAYLOAD; ++i) {
      if (i < in.n_payload) {
        const int32_t v = static_cast<int32_t>(load_any(in.pay_col[i], in.pay_type[i], r));
        if (i == 0) pay = v;
        pmax[i] = max(pmax[i], max_code(v));
        pmin[i] = max(pmin[i], min_code(v));
      }
    }
    if (in.n_payload > 1) pay = static_cast<int32_t>(r);
    if (h.kind == PV_HT_PERFECT) {
      const int64_t i = key - h.kmin;
      if (static_cast<uint64_t>(i) >= static_cast<uint64_t>(h.cap)) {
        set_error(bp.err, PV_ERR_KEY_OUT_OF_RANGE);
        continue;
      }
      const unsigned long long v = (static_cast<unsigned long long>(static_cast<uint32_t>(pay)) << 32) | 1ull;
      if (atomicCAS(slots + i, 0ull, v) != 0ull) set_error(bp.err, PV_ERR_DUP_BUILD_KEY);
      continue;
    }
    const uint32_t k32 = static_cast<uint32_t>(key);
    if (k32 == kEmpty32) {  // the key equal to the empty marker lives in the side slot
      const unsigned long long v = static_cast<uint32_t>(pay);
      if (atomicCAS(slots + h.cap, ~0ull, v) != ~0ull) set_error(bp.err, PV_ERR_DUP_BUILD_KEY);
      continue;
    }
    const uint64_t val = (static_cast<uint64_t>(k32) << 32) | static_cast<uint32_t>(pay);
    if (h.kind == PV_HT_LINEAR) linear_put(h, k32, val, bp.err);
    else cuckoo_put(h, val, bp.max_evictions, bp.err);
  }
#pragma unroll
  for (int i = 0; i < PV_MAX_PAYLOAD; ++i) {
    if (i < in.n_payload) {
      const uint64_t mx = warp_reduce<PV_MAX>(pmax[i]);
      const uint64_t mn = warp_reduce<PV_MAX>(pmin[i]);
      if ((threadIdx.x & 31) == 0 && mx) {
        atomicMax(bp.pay_stats + 2 * i, static_cast<unsigned long long>(mx));
        atomicMax(bp.pay_stats + 2 * i + 1, static_cast<unsigned long long>(mn));
      }
    }
  }
}

// Duplicate check of a cuckoo table: every key stays within its k candidate
// slots, so a key found in two of them was inserted twice.
__global__ void k_cuckoo_dupcheck(const __grid_constant__ DevHT h, int32_t* err) {
  const unsigned long long* slots = reinterpret_cast<const unsigned long long*>(h.slots);
  for (int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; p < h.cap;
       p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const uint32_t k32 = static_cast<uint32_t>(slots[p] >> 32);
    if (k32 == kEmpty32) continue;
    for (int i = 0; i < h.k; ++i) {
      const uint64_t q = cuckoo_pos(h, k32, i);
      if (q != static_cast<uint64_t>(p) && static_cast<uint32_t>(slots[q] >> 32) == k32) {
        set_error(err, PV_ERR_DUP_BUILD_KEY);
        return;
      }
    }
  }
}

// Presence bits of a perfect array: word w holds slots 32w .. 32w+31 (bit j
// set when slot 32w + j is occupied), one warp ballot per word.
__global__ void k_perfect_bits(const uint64_t* slots, int64_t cap, uint32_t* bits) {
  const int64_t words = (cap + 31) / 32;
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  for (int64_t w = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; w < words; w += nwarps) {
    const int64_t i = w * 32 + lane;
    const uint32_t b = __ballot_sync(0xffffffffu, i < cap && slots[i] != 0);
    if (lane == 0) bits[w] = b;
  }
}

// One byte per slot of a perfect array whose payload spans at most 255
// values: 0 for an empty slot, else payload - base (base = smallest payload - 1).
// A payload outside that span (the build columns changed since the first
// build's statistics) is reported as a key outside its domain.
__global__ void k_perfect_codes(const uint64_t* slots, int64_t cap, uint8_t* codes, int32_t base, int32_t* err) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < cap;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const uint64_t s = slots[i];
    uint32_t c = 0;
    if (s != 0) {
      const int64_t d = static_cast<int64_t>(static_cast<int32_t>(s >> 32)) - base;
      if (d < 1 || d > 255) set_error(err, PV_ERR_KEY_OUT_OF_RANGE);
      else c = static_cast<uint32_t>(d);
    }
    codes[i] = static_cast<uint8_t>(c);
  }
}

static void launch_codes(const BuildEnv& env, const DevHT& h) {
  const int g = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(env.sm_count * 8, (h.cap + 255) / 256)));
  k_perfect_codes<<<g, 256, 0, env.stream>>>(h.slots, h.cap, const_cast<uint8_t*>(h.codes), h.code_base, env.err);
  ++*env.launches;
}

pv_status build_table(const BuildEnv& env, const BuildInput& in, const pv_ht_variant& var, int64_t kmin,
                      int64_t kmax, BuildTable& out, std::string& msg) {
  DevHT& h = out.ht;
  h.kind = var.kind;
  h.hash = var.hash;
  if (var.kind != PV_HT_LINEAR && var.kind != PV_HT_CUCKOO && var.kind != PV_HT_PERFECT) {
    msg = "bad hash table kind";
    return PV_ERR_INVALID_ARG;
  }
  if (var.hash != PV_HASH_MURMUR && var.hash != PV_HASH_MULTSHIFT) {
    msg = "bad hash function";
    return PV_ERR_INVALID_ARG;
  }
  h.k = var.cuckoo_k ? var.cuckoo_k : 3;
  if (h.k < 2 || h.k > 4) {
    msg = "cuckoo_k must be 2..4";
    return PV_ERR_INVALID_ARG;
  }
  uint64_t sd = var.seed ? var.seed : 0xb01d1709ull;
  for (int i = 0; i < 4; ++i) {
    sd = fmix64(sd + 0x9e3779b97f4a7c15ull);
    h.seed[i] = sd | 1ull;
  }
  size_t bytes;
  if (var.kind == PV_HT_PERFECT) {
    const int64_t span = kmax >= kmin ? kmax - kmin + 1 : 1;
    if (span > (int64_t(1) << 28)) {
      msg = "perfect array: key domain larger than 2^28 slots";
      return PV_ERR_UNSUPPORTED;
    }
    h.cap = span;
    h.kmin = kmin;
    h.log2cap = 0;
    h.narrow = kmin >= INT32_MIN && kmin + span <= (int64_t(1) << 31) ? 1 : 0;
    bytes = static_cast<size_t>(span) * 8;
  } else {
    const double lf = var.load_factor > 0 && var.load_factor <= 1 ? var.load_factor : 0.5;
    const double want = std::max<double>(2.0, static_cast<double>(in.n_rows) / lf);
    int l = 1;
    while (static_cast<double>(int64_t(1) << l) < want) ++l;
    if (l > 31) {
      msg = "build table too large";
      return PV_ERR_UNSUPPORTED;
    }
    h.log2cap = l;
    h.cap = int64_t(1) << l;
    bytes = static_cast<size_t>(h.cap + 1) * 8;
  }
  const int max_ev = var.max_evictions > 0 ? var.max_evictions : 32 * std::max(1, h.log2cap);
  if (in.n_payload > 1 && in.n_rows > INT32_MAX) {
    msg = "tables with several payload columns index at most 2^31 - 1 build rows";
    return PV_ERR_UNSUPPORTED;
  }
  out.n_payload = in.n_payload;
  out.indexed = in.n_payload > 1;
  for (int i = 0; i < in.n_payload; ++i) {
    out.pay_col[i] = in.pay_col[i];
    out.pay_type[i] = in.pay_type[i];
  }
  // [slots | 16-byte stats | presence bits (perfect arrays without payload or past 64 KB of slots: the
  // bits stay in L1 where the slots would not, and only hits read a slot)]
  const size_t stats_off = (bytes + 15) & ~size_t(15);
  const bool with_bits = var.kind == PV_HT_PERFECT && (in.n_payload == 0 || h.cap * 8 > (64 << 10));
  h.payload = in.n_payload > 0 ? 1 : 0;
  const size_t bits_bytes = with_bits ? static_cast<size_t>((h.cap + 31) / 32) * 4 : 0;
  constexpr size_t stats_bytes = 16 * PV_MAX_PAYLOAD;
  // a perfect array with one payload column may turn out (payload statistics) to fit one byte per slot
  const bool may_code = var.kind == PV_HT_PERFECT && in.n_payload == 1;
  const size_t codes_off = stats_off + stats_bytes + ((bits_bytes + 15) & ~size_t(15));
  const size_t codes_bytes = may_code ? static_cast<size_t>(h.cap) : 0;
  out.mem = env.alloc(codes_off + codes_bytes + 64, env.user);
  if (!out.mem) {
    msg = "allocator returned NULL";
    return PV_ERR_OOM;
  }
  h.slots = static_cast<uint64_t*>(out.mem);
  unsigned long long* stats = reinterpret_cast<unsigned long long*>(static_cast<char*>(out.mem) + stats_off);
  h.bits = with_bits ? reinterpret_cast<const uint32_t*>(static_cast<char*>(out.mem) + stats_off + stats_bytes)
                      : nullptr;
  out.slot_bytes = bytes;
  BuildParams& bp = out.bp;
  bp = BuildParams{};
  bp.in = in;
  bp.ht = h;
  bp.max_evictions = max_ev;
  bp.err = env.err;
  bp.pay_stats = stats;
  pv_status st = rebuild_table(env, out);
  if (st != PV_OK) {
    msg = "build launch failed";
    return st;
  }
  cudaError_t e = cudaSuccess;
  unsigned long long hs[2 * PV_MAX_PAYLOAD] = {};
  e = cudaMemcpyAsync(hs, stats, stats_bytes, cudaMemcpyDeviceToHost, env.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(env.stream);
  if (e != cudaSuccess) {
    msg = cudaGetErrorString(e);
    return PV_ERR_CUDA;
  }
  for (int i = 0; i < in.n_payload; ++i) {
    if (hs[2 * i] == 0) {  // no surviving row
      out.pay_min[i] = 0;
      out.pay_max[i] = -1;
    } else {
      out.pay_max[i] = decode_max(hs[2 * i]);
      out.pay_min[i] = decode_min(hs[2 * i + 1]);
    }
  }
  if (may_code && out.pay_max[0] - out.pay_min[0] <= 254 && out.pay_min[0] > INT32_MIN) {
    // probes read one byte per key instead of an 8-byte slot (and its presence bit)
    h.codes = reinterpret_cast<const uint8_t*>(static_cast<char*>(out.mem) + codes_off);
    h.code_base = static_cast<int32_t>(out.pay_max[0] >= out.pay_min[0] ? out.pay_min[0] - 1 : -1);
    out.bp.ht = h;
    launch_codes(env, h);
  }
  return PV_OK;
}

pv_status rebuild_table(const BuildEnv& env, const BuildTable& t) {
  const BuildParams& bp = t.bp;
  const DevHT& h = bp.ht;
  cudaError_t e = cudaMemsetAsync(h.slots, h.kind == PV_HT_PERFECT ? 0 : 0xFF, t.slot_bytes, env.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(bp.pay_stats, 0, 16 * PV_MAX_PAYLOAD, env.stream);
  if (e != cudaSuccess) return PV_ERR_CUDA;
  if (bp.in.n_rows > 0) {
    const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(env.sm_count * 8, (bp.in.n_rows + 255) / 256)));
    k_build<<<grid, 256, 0, env.stream>>>(bp);
    ++*env.launches;
    if (h.kind == PV_HT_CUCKOO) {
      const int g2 = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(env.sm_count * 8, (h.cap + 255) / 256)));
      k_cuckoo_dupcheck<<<g2, 256, 0, env.stream>>>(h, env.err);
      ++*env.launches;
    }
  }
  if (h.codes != nullptr) launch_codes(env, h);
  if (h.bits != nullptr && h.codes == nullptr) {
    const int64_t words = (h.cap + 31) / 32;
    const int g3 = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(env.sm_count * 8, (words + 7) / 8)));
    k_perfect_bits<<<g3, 256, 0, env.stream>>>(h.slots, h.cap, const_cast<uint32_t*>(h.bits));
    ++*env.launches;
  }
  return cudaGetLastError() == cudaSuccess ? PV_OK : PV_ERR_CUDA;
}

}  // namespace pv
