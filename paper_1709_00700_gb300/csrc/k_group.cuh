// HASH_AGGREGATE (Table 1) and result extraction.
//
// Execution strategies (Section 4.2):
//   global aggregation: every row updates one global table with atomics;
//   local aggregation: rows first update a CTA-local table in shared memory
//     (N tables = the CTAs, M threads per table = the CTA), which is merged
//     into the global table when the CTA finishes; with M = 1 every thread
//     owns a private table (coarse-grained form, no atomics at all).
// Table implementations (Section 5.1): linear probing, cuckoo hashing, and a
// perfect array over a dense key domain.  Single pass inserts keys while
// aggregating; multi pass inserts the keys in a first kernel and aggregates
// with lookups in a second (cuckoo tables move keys while inserting, so they
// always take the two passes, with a duplicate sweep in between).
//
// Global table: keys[cap + 1] (EMPTY = ~0; slot cap holds the key equal to
// EMPTY) and vals[(cap + 1) * stride] with the aggregate codes and, last, the
// row count of the slot.  Extraction compacts non-empty slots into dense int64
// columns and leaves every slot it visits empty again, so a rerun needs no
// clearing pass.
#pragma once

#include "pv_eval.cuh"

namespace pv {

constexpr int kLocalProbe = 16;          // probe-length bound in a local table
constexpr size_t kLocalBytes = 96 << 10; // shared memory of a CTA-local hash table
constexpr size_t kLocalPerfectBytes = 192 << 10;  // of a CTA-local perfect array (one CTA per SM past 113 KB)
constexpr size_t kClusterBytes = 192 << 10;  // shared memory of one CTA's part of a cluster table

// Whether every group-key part is a 32-bit source.
template <class SH, int... I>
constexpr bool key_parts32(std::integer_sequence<int, I...>) {
  return (KeyPart32<SH, typename At<I, typename SH::Key::L>::type>::value && ...);
}
template <class SH>
constexpr bool key_narrow() {
  return key_parts32<SH>(std::make_integer_sequence<int, SH::Key::N>{});
}

// Mixed-radix code of row r's group key: each part minus its minimum, row-
// major over the part spans (the last part varies fastest).  It is the
// perfect-array slot and, for keys of three parts, the hash-table key.  ok is
// false when a part lies outside its span (unsigned differences wrap below
// the minimum).  Without WIDE, keys of 32-bit parts use 32-bit arithmetic:
// a perfect array has at most 2^28 slots.
template <class SH, bool WIDE = !key_narrow<SH>()>
__device__ __forceinline__ uint64_t row_perfect_index(const GroupDesc& gd, Item<SH>& it, const KParams& kp, int r,
                                                      bool& ok) {
  using U = std::conditional_t<WIDE, uint64_t, uint32_t>;
  U code = 0;
  ok = true;
  static_for<SH::Key::N>([&](auto p) {
    constexpr int P = decltype(p)::value;
    const U a = static_cast<U>(key_part<SH, P>(it, kp, r)) - static_cast<U>(gd.key_min[P]);
    ok = ok && a < static_cast<U>(gd.key_span[P]);
    code = P == 0 ? a : code * static_cast<U>(gd.key_span[P]) + a;
  });
  return code;
}

// Hash-table key of row r: the packed key for one or two parts, the mixed-
// radix code for three (0, an in-domain code, when ok is false, so that rows
// outside the domain add no keys).
template <class SH>
__device__ __forceinline__ uint64_t group_key(const GroupDesc& gd, Item<SH>& it, const KParams& kp, int r, bool& ok) {
  if constexpr (SH::Key::N <= 2) {
    ok = true;
    return pack_key<SH>(it, kp, r);
  } else {
    const uint64_t code = row_perfect_index<SH, true>(gd, it, kp, r, ok);
    return ok ? code : 0;
  }
}

// Global linear probing: slot of key, inserting it if absent.  Returns
// cap + 1 on failure (table full; error recorded).
__device__ __forceinline__ uint64_t global_linear_slot(const GroupOut& g, uint64_t key, int32_t* err) {
  if (key == kEmpty64) return static_cast<uint64_t>(g.cap);
  const uint64_t mask = static_cast<uint64_t>(g.cap) - 1;
  uint64_t idx = ht_index(key, g.hash, g.seed[0], g.log2cap);
  for (int64_t step = 0; step < g.cap; ++step) {
    unsigned long long cur = __ldcg(g.keys + idx);  // keys change under us: read L2
    if (cur == key) return idx;
    if (cur == kEmpty64) {
      cur = atomicCAS(g.keys + idx, kEmpty64, static_cast<unsigned long long>(key));
      if (cur == kEmpty64 || cur == key) return idx;
    }
    idx = (idx + 1) & mask;
  }
  set_error(err, PV_ERR_HT_FULL);
  return static_cast<uint64_t>(g.cap) + 1;
}

// Lookup of a key inserted by the key pass (linear or cuckoo).
template <int HTK>
__device__ __forceinline__ uint64_t global_lookup(const GroupOut& g, uint64_t key, int32_t* err) {
  if (key == kEmpty64) return static_cast<uint64_t>(g.cap);
  if constexpr (HTK == PV_HT_CUCKOO) {
    for (int f = 0; f < g.cuckoo_k; ++f) {
      const uint64_t p = ht_index(key, g.hash, g.seed[f], g.log2cap);
      if (g.keys[p] == key) return p;
    }
  } else {
    const uint64_t mask = static_cast<uint64_t>(g.cap) - 1;
    uint64_t idx = ht_index(key, g.hash, g.seed[0], g.log2cap);
    for (int64_t step = 0; step < g.cap; ++step) {
      const unsigned long long cur = g.keys[idx];
      if (cur == key) return idx;
      if (cur == kEmpty64) break;
      idx = (idx + 1) & mask;
    }
  }
  set_error(err, PV_ERR_HT_FULL);  // a key the key pass did not insert: the table overflowed
  return static_cast<uint64_t>(g.cap) + 1;
}

// Cuckoo insertion of a group key (key pass).  Skips keys already present;
// concurrent inserts of one key may leave duplicates, removed by k_cuckoo_dedupe.
__device__ __forceinline__ void global_cuckoo_insert(const GroupOut& g, uint64_t key, int32_t* err) {
  if (key == kEmpty64) return;  // lives in the side slot, found by value
  for (int f = 0; f < g.cuckoo_k; ++f)
    if (__ldcg(g.keys + ht_index(key, g.hash, g.seed[f], g.log2cap)) == key) return;
  unsigned long long cur = key;
  int f = 0;
  for (int e = 0; e <= g.max_evictions; ++e) {
    for (int i = 0; i < g.cuckoo_k; ++i) {
      const uint64_t p = ht_index(cur, g.hash, g.seed[i], g.log2cap);
      unsigned long long s = __ldcg(g.keys + p);
      if (s == cur) return;
      if (s == kEmpty64 && atomicCAS(g.keys + p, kEmpty64, cur) == kEmpty64) return;
    }
    const uint64_t p = ht_index(cur, g.hash, g.seed[f], g.log2cap);
    const unsigned long long old = atomicExch(g.keys + p, cur);
    if (old == kEmpty64 || old == cur) return;
    cur = old;
    int placed = 0;
    for (int i = 0; i < g.cuckoo_k; ++i)
      if (ht_index(cur, g.hash, g.seed[i], g.log2cap) == p) { placed = i; break; }
    f = (placed + 1) % g.cuckoo_k;
  }
  set_error(err, PV_ERR_CUCKOO_CYCLE);
}

// Index of the first COUNT aggregate of a shape, -1 if it has none.
template <class A>
constexpr int count_index() {
  for (int i = 0; i < A::N; ++i)
    if (A::func_of[i] == PV_COUNT) return i;
  return -1;
}

// 64-bit add into shared memory with 32-bit atomics: fetch-add the low word,
// add the high word (plus the carry out of the low word) only when it is not
// zero.  Exact modulo 2^64, also under concurrency (each adder's carry comes
// from its own fetch-add).
__device__ __forceinline__ void shared_add64(unsigned long long* p, uint64_t x) {
  unsigned int* w = reinterpret_cast<unsigned int*>(p);
  const unsigned int lo = static_cast<unsigned int>(x);
  unsigned int hi = static_cast<unsigned int>(x >> 32);
  if (lo) {
    const unsigned int old = atomicAdd(w, lo);
    hi += (old + lo < old) ? 1u : 0u;
  }
  if (hi) atomicAdd(w + 1, hi);
}

// Adds one row's aggregate codes into a slot with atomics; zero codes (dead
// rows, empty MIN/MAX) cost no atomic.  The hidden row count (last word) is
// kept only when the shape has no COUNT aggregate.  SHARED: the slot is in
// shared memory (32-bit atomics for the sums).
template <class SH, bool SHARED = false>
__device__ __forceinline__ void slot_atomic_add(unsigned long long* v, const uint64_t (&c)[SH::Aggs::N + 1]) {
  using A = typename SH::Aggs;
  static_for<A::N + 1>([&](auto a) {
    constexpr int I = decltype(a)::value;
    constexpr int F = I < A::N ? A::func_of[I < A::N ? I : 0] : PV_COUNT;
    if constexpr (I == A::N && count_index<A>() >= 0) return;
    if (c[I]) {
      if constexpr (SHARED && (F == PV_SUM || F == PV_COUNT)) shared_add64(v + I, c[I]);
      else acc_atomic<F>(v + I, c[I]);
    }
  });
}

// Aggregate codes of row r: SUM/COUNT values, MIN/MAX order codes, row count;
// masked to zero for a dead row (software predication).
template <class SH>
__device__ __forceinline__ void row_codes(Item<SH>& it, const KParams& kp, int r, uint64_t live_mask,
                                          uint64_t (&c)[SH::Aggs::N + 1]) {
  using A = typename SH::Aggs;
  static_for<A::N>([&](auto a) {
    constexpr int I = decltype(a)::value;
    using AG = typename At<I, typename A::L>::type;
    c[I] = acc_code<AG::func>(agg_value<AG>(it, kp, r)) & live_mask;
  });
  c[A::N] = 1ull & live_mask;
}

// ---------------------------------------------------------------------------
// Sinks.  Each provides init() (CTA prologue), add() (one row) and finish()
// (CTA epilogue); every thread of the CTA calls init and finish.
// ---------------------------------------------------------------------------
enum GlobalMode { G_INSERT = 0, G_LOOKUP_LINEAR = 1, G_LOOKUP_CUCKOO = 2 };

template <int GM>
__device__ __forceinline__ uint64_t global_slot(const GroupOut& g, uint64_t key, int32_t* err) {
  if constexpr (GM == G_INSERT) return global_linear_slot(g, key, err);
  else if constexpr (GM == G_LOOKUP_LINEAR) return global_lookup<PV_HT_LINEAR>(g, key, err);
  else return global_lookup<PV_HT_CUCKOO>(g, key, err);
}

// Warp pre-aggregation in front of the global and cluster tables (variant
// flag warp_agg; shared-memory tables ignore it: their atomics cost less
// than the matching): the active lanes holding the same group key combine
// their accumulator codes, and the group's lowest lane alone updates the
// table.  The lanes of a group
// form a list in lane order; pointer jumping (each step adds the successor's
// partial and skips to the successor's successor) leaves the whole group's
// combination in its first lane after ceil(log2(group size)) steps.  One
// ballot skips all of it when no key repeats within the warp.  Returns
// whether this lane still updates the table.
template <class SH>
__device__ __forceinline__ bool warp_preaggregate(uint64_t key, uint64_t (&c)[SH::Aggs::N + 1]) {
  constexpr int NA = SH::Aggs::N;
  const unsigned active = __activemask();
  const unsigned peers = __match_any_sync(active, static_cast<unsigned long long>(key));
  const int lane = threadIdx.x & 31;
  const unsigned after = peers & ~((2u << lane) - 1u);  // lane 31: 2u << 31 == 0, nothing after
  if (__ballot_sync(active, after != 0u) == 0u) return true;
  int nxt = after ? __ffs(after) - 1 : lane;
  int more = after != 0u;
  while (__any_sync(active, more)) {
    static_for<NA + 1>([&](auto a) {
      constexpr int I = decltype(a)::value;
      constexpr int F = I < NA ? SH::Aggs::func_of[I < NA ? I : 0] : PV_COUNT;
      const uint64_t o = __shfl_sync(active, static_cast<unsigned long long>(c[I]), nxt);
      if (more) c[I] = acc_combine<F>(c[I], o);
    });
    const int nn = __shfl_sync(active, nxt, nxt);
    const int nm = __shfl_sync(active, more, nxt);
    if (more) {
      nxt = nn;
      more = nm;
    }
  }
  return (peers & ((1u << lane) - 1u)) == 0u;
}

template <class SH, int GM>
struct SinkGlobalHash {
  static constexpr int NA = SH::Aggs::N;
  const GroupDesc& gd; const GroupOut& g; int32_t* err;
  __device__ SinkGlobalHash(const GroupDesc& d, const GroupOut& o, int32_t* e, unsigned long long*) : gd(d), g(o), err(e) {}
  __device__ void init() {}
  __device__ __forceinline__ void add(Item<SH>& it, const KParams& kp, int r, bool live) {
    bool in_domain;
    const uint64_t key = group_key<SH>(gd, it, kp, r, in_domain);
    if (!in_domain && live) set_error(err, PV_ERR_KEY_OUT_OF_RANGE);
    uint64_t c[NA + 1];
    row_codes<SH>(it, kp, r, live && in_domain ? ~0ull : 0ull, c);
    if (g.warp_agg && !warp_preaggregate<SH>(key, c)) return;
    const uint64_t s = global_slot<GM>(g, key, err);
    if (s > static_cast<uint64_t>(g.cap)) return;
    slot_atomic_add<SH>(g.vals + s * g.stride, c);
  }
  __device__ void finish() {}
};

template <class SH>
struct SinkGlobalPerfect {
  static constexpr int NA = SH::Aggs::N;
  const GroupDesc& gd; const GroupOut& g; int32_t* err;
  __device__ SinkGlobalPerfect(const GroupDesc& d, const GroupOut& o, int32_t* e, unsigned long long*) : gd(d), g(o), err(e) {}
  __device__ void init() {}
  __device__ __forceinline__ void add(Item<SH>& it, const KParams& kp, int r, bool live) {
    bool ok;
    uint64_t s = row_perfect_index<SH>(gd, it, kp, r, ok);
    if (!ok) {
      if (live) { set_error(err, PV_ERR_KEY_OUT_OF_RANGE); return; }
      s = 0;
    }
    uint64_t c[NA + 1];
    row_codes<SH>(it, kp, r, live ? ~0ull : 0ull, c);
    if (g.warp_agg && !warp_preaggregate<SH>(s, c)) return;
    slot_atomic_add<SH>(g.vals + (blockIdx.x % g.replicas) * g.rep_stride + s * g.stride, c);
  }
  __device__ void finish() {}
};

// Block-shared perfect array in shared memory (M = CTA threads), merged with
// one atomic per non-zero entry.
template <class SH>
struct SinkLocalPerfect {
  static constexpr int NA = SH::Aggs::N;
  const GroupDesc& gd; const GroupOut& g; int32_t* err; unsigned long long* sm;
  __device__ SinkLocalPerfect(const GroupDesc& d, const GroupOut& o, int32_t* e, unsigned long long* s)
      : gd(d), g(o), err(e), sm(s) {}
  __device__ void init() {
    const int64_t words = g.cap * g.stride;
    for (int64_t i = threadIdx.x; i < words; i += blockDim.x) sm[i] = 0;
    __syncthreads();
  }
  __device__ __forceinline__ void add(Item<SH>& it, const KParams& kp, int r, bool live) {
    bool ok;
    uint64_t s = row_perfect_index<SH>(gd, it, kp, r, ok);
    if (!ok) {
      if (live) { set_error(err, PV_ERR_KEY_OUT_OF_RANGE); return; }
      s = 0;
    }
    uint64_t c[NA + 1];
    row_codes<SH>(it, kp, r, live ? ~0ull : 0ull, c);
    slot_atomic_add<SH, true>(sm + s * g.stride, c);  // (warp_agg applies to global and cluster tables)
  }
  __device__ void finish() {
    __syncthreads();
    const int64_t words = g.cap * g.stride;
    for (int64_t i = threadIdx.x; i < words; i += blockDim.x) {
      const uint64_t v = sm[i];
      if (!v) continue;
      const int a = static_cast<int>(i % g.stride);
      unsigned long long* dst = g.vals + (blockIdx.x % g.replicas) * g.rep_stride + i;
      if (a == NA || gd.func[a] == PV_SUM || gd.func[a] == PV_COUNT) atomicAdd(dst, static_cast<unsigned long long>(v));
      else atomicMax(dst, static_cast<unsigned long long>(v));
    }
  }
};

// Perfect array partitioned over the C = 2^g.cluster_log2 CTAs of a
// thread-block cluster (distributed shared memory): slot s lives in CTA
// s mod C of the cluster, at local slot s / C, so a cluster keeps C times the
// domain one CTA could on chip, and neighbouring (often equally hot) slots
// spread over its CTAs.  The host picks the smallest C (2..16) whose part
// fits in shared memory.  Rows update the owner's words with
// cluster-scope shared-memory atomics: sums as two 32-bit fetch-adds (the
// high word only on a carry or a non-zero high part, as shared_add64), MIN /
// MAX codes with a 64-bit compare-and-swap loop.  Prologue: zero the local part, cluster
// barrier (no update reaches unzeroed memory).  Epilogue: cluster barrier
// (every update has landed), then each CTA merges its part into the global
// table with one atomic per non-zero word.  Every thread of every CTA of the
// cluster reaches both barriers.
constexpr int kMaxClusterCTAs = 16;

// Cluster-wide barrier (not .aligned: the threads of a warp may reach it
// diverged, e.g. after a grid-stride loop).
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// Address of the same shared-memory offset in cluster CTA `rank`.
__device__ __forceinline__ uint32_t cluster_map(uint32_t local, uint32_t rank) {
  uint32_t remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(rank));
  return remote;
}
__device__ __forceinline__ void cluster_add64(uint32_t addr, uint64_t x) {
  const uint32_t lo = static_cast<uint32_t>(x);
  uint32_t hi = static_cast<uint32_t>(x >> 32);
  if (lo) {
    uint32_t old;
    asm volatile("atom.shared::cluster.add.u32 %0, [%1], %2;" : "=r"(old) : "r"(addr), "r"(lo) : "memory");
    hi += (old + lo < old) ? 1u : 0u;
  }
  if (hi) {
    uint32_t old;
    asm volatile("atom.shared::cluster.add.u32 %0, [%1], %2;" : "=r"(old) : "r"(addr + 4), "r"(hi) : "memory");
  }
}
// 64-bit max into a cluster CTA's shared memory by compare-and-swap: on
// sm_103a, atom.shared::cluster.max.u64 lost updates in a probe (339 of 512
// words wrong after 131k updates from one cluster), while 64-bit CAS and the
// 32-bit cluster atomics were exact.  Every failed CAS sees a strictly larger value, so the loop
// ends; the cap only guards it.  Returns false when the cap was reached.
__device__ __forceinline__ bool cluster_max64(uint32_t addr, uint64_t x) {
  unsigned long long cur;
  asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(cur) : "r"(addr) : "memory");
  for (int it = 0; it < (1 << 20) && cur < x; ++it) {
    unsigned long long old;
    asm volatile("atom.shared::cluster.cas.b64 %0, [%1], %2, %3;"
                 : "=l"(old)
                 : "r"(addr), "l"(cur), "l"(static_cast<unsigned long long>(x))
                 : "memory");
    if (old == cur) return true;
    cur = old;
  }
  return cur >= x;
}

template <class SH>
struct SinkClusterPerfect {
  static constexpr int NA = SH::Aggs::N;
  static constexpr bool kCluster = true;
  static __host__ __device__ int64_t part_slots(int64_t cap, int log2c) { return (cap + (1 << log2c) - 1) >> log2c; }
  const GroupDesc& gd; const GroupOut& g; int32_t* err; unsigned long long* sm;
  uint32_t sbase, rank;
  __device__ SinkClusterPerfect(const GroupDesc& d, const GroupOut& o, int32_t* e, unsigned long long* s)
      : gd(d), g(o), err(e), sm(s), sbase(static_cast<uint32_t>(__cvta_generic_to_shared(s))), rank(cluster_rank()) {}
  __device__ void init() {
    const int64_t words = part_slots(g.cap, g.cluster_log2) * g.stride;
    for (int64_t i = threadIdx.x; i < words; i += blockDim.x) sm[i] = 0;
    cluster_sync();
  }
  __device__ __forceinline__ void add(Item<SH>& it, const KParams& kp, int r, bool live) {
    bool ok;
    uint64_t s = row_perfect_index<SH>(gd, it, kp, r, ok);
    if (!ok) {
      if (live) { set_error(err, PV_ERR_KEY_OUT_OF_RANGE); return; }
      s = 0;
    }
    uint64_t c[NA + 1];
    row_codes<SH>(it, kp, r, live ? ~0ull : 0ull, c);
    if (g.warp_agg && !warp_preaggregate<SH>(s, c)) return;
    const uint32_t base = cluster_map(
        sbase + static_cast<uint32_t>(s >> g.cluster_log2) * static_cast<uint32_t>(g.stride) * 8u,
        static_cast<uint32_t>(s & ((1u << g.cluster_log2) - 1u)));
    using A = typename SH::Aggs;
    static_for<NA + 1>([&](auto a) {
      constexpr int I = decltype(a)::value;
      constexpr int F = I < NA ? A::func_of[I < NA ? I : 0] : PV_COUNT;
      if constexpr (I == NA && count_index<A>() >= 0) return;
      if (c[I]) {
        if constexpr (F == PV_SUM || F == PV_COUNT) cluster_add64(base + I * 8, c[I]);
        else if (!cluster_max64(base + I * 8, c[I])) set_error(err, PV_ERR_TIMEOUT);
      }
    });
  }
  __device__ void finish() {
    cluster_sync();
    const int64_t words = part_slots(g.cap, g.cluster_log2) * g.stride;
    for (int64_t i = threadIdx.x; i < words; i += blockDim.x) {
      const uint64_t v = sm[i];
      if (!v) continue;
      const int64_t slot = ((i / g.stride) << g.cluster_log2) + rank;
      const int a = static_cast<int>(i % g.stride);
      if (slot >= g.cap) continue;
      unsigned long long* dst = g.vals + (blockIdx.x % g.replicas) * g.rep_stride + slot * g.stride + a;
      if (a == NA || gd.func[a] == PV_SUM || gd.func[a] == PV_COUNT) atomicAdd(dst, static_cast<unsigned long long>(v));
      else atomicMax(dst, static_cast<unsigned long long>(v));
    }
  }
};

// Word layout of a thread-private slot.  Wide: word a holds aggregate a
// (SUM/COUNT raw, MIN/MAX as codes), then the row count unless a COUNT
// aggregate already counts rows.  NARROW: the narrow aggregates (NarrowAgg:
// SUM of a plain column, COUNT) and the hidden row count are 32-bit fields,
// two to a word (field f in word f / 2, half f % 2), then one word per other
// aggregate.  Both are padded to an even number of words.
struct SlotLayout {
  int word[PV_MAX_AGGS + 1];  // word of aggregate a (index NA: the hidden row count)
  int half[PV_MAX_AGGS + 1];  // 0 / 1: low / high 32-bit field; -1: the whole word
  int agg[2 * PV_MAX_AGGS + 2][2];  // per word, the aggregate of each field (-1: none); wide words use [0]
  int narrow_words;           // words holding 32-bit fields (they come first)
  int sw;                     // words per slot (even)
};

template <class A, bool NARROW>
constexpr SlotLayout make_slot_layout(int na, int ca) {
  SlotLayout L{};
  for (int w = 0; w < 2 * PV_MAX_AGGS + 2; ++w) L.agg[w][0] = L.agg[w][1] = -1;
  const int count_hidden = ca < 0;
  int f = 0;
  if (NARROW) {
    for (int a = 0; a <= na; ++a) {
      const bool narrow = a < na ? A::narrow_of[a < na ? a : 0] : count_hidden;
      if (!narrow) continue;
      L.word[a] = f / 2;
      L.half[a] = f % 2;
      L.agg[f / 2][f % 2] = a;
      ++f;
    }
  }
  L.narrow_words = (f + 1) / 2;
  int w = L.narrow_words;
  for (int a = 0; a <= na; ++a) {
    const bool narrow = NARROW && (a < na ? A::narrow_of[a < na ? a : 0] : count_hidden);
    if (narrow || (a == na && !count_hidden)) continue;
    L.word[a] = w;
    L.half[a] = -1;
    L.agg[w][0] = a;
    ++w;
  }
  L.sw = (w + 1) & ~1;
  return L;
}

// Thread-private perfect arrays (M = 1): no atomics until the CTA epilogue.
// A slot holds SW words (SlotLayout) stored as SW / 2 16-byte pairs,
// interleaved by thread: pair j of slot s of thread t is at 16-byte unit
// (s * SW / 2 + j) * blockDim + t, so the 8 lanes of a memory phase always
// touch 8 distinct bank groups, whatever slot each lane updates.  Dead rows
// skip the update.  With NARROW, the 32-bit fields hold a thread's partial
// sums of the narrow aggregates: a row updates them only when each of its
// narrow values is at most g.narrow_limit = (2^32 - 1) / (rows the thread
// visits), so no field can overflow; any other row adds its codes straight
// into the global table.  The launch takes the wide layout instead when the
// narrow columns' statistics say some values exceed that limit
// (g.narrow_max), so that such rows stay rare.  Fewer words per slot mean
// less shared-memory traffic per row, the limit of this sink.
template <class SH, bool NARROW = false>
struct SinkThreadPerfect {
  // Tables of 256 threads x (cap x 16 B units) let three CTAs share an SM;
  // the predicated loop then runs without register double buffering.
  static constexpr int kRegs = 80;
  static constexpr bool kPipelined = false;
  // TMA-staged access compiled (the loads that miss their register double buffer)
  static constexpr bool kStaged = true;
  using A = typename SH::Aggs;
  static constexpr int NA = A::N;
  static constexpr int CA = count_index<A>();
  static constexpr SlotLayout L = make_slot_layout<A, NARROW>(NA, CA);
  static constexpr int SW = L.sw;
  static constexpr int SP = SW / 2;
  static constexpr int NW = L.narrow_words;
  static __host__ __device__ int64_t units_per_thread(int64_t cap) { return cap * SP; }
  static __host__ __device__ size_t smem_bytes(int64_t cap, int block) {
    return static_cast<size_t>(units_per_thread(cap)) * 16 * block;
  }
  template <int W>
  static __device__ __forceinline__ constexpr int word_func() {
    constexpr int ag = L.agg[W][0];
    if constexpr (W < NW || ag < 0 || ag >= NA) return PV_SUM;
    else return A::func_of[ag < NA && ag >= 0 ? ag : 0];
  }
  const GroupDesc& gd; const GroupOut& g; int32_t* err; ulonglong2* sm;
  uint32_t sbase;        // shared address of this thread's unit 0 of slot 0
  uint32_t ustride;      // bytes between a thread's consecutive units
  bool bad = false;      // a live row's key fell outside the domain
  __device__ SinkThreadPerfect(const GroupDesc& d, const GroupOut& o, int32_t* e, unsigned long long* s)
      : gd(d), g(o), err(e), sm(reinterpret_cast<ulonglong2*>(s)),
        sbase(static_cast<uint32_t>(__cvta_generic_to_shared(s)) + threadIdx.x * 16u), ustride(blockDim.x * 16u) {}
  __device__ void init() {
    const int64_t n = units_per_thread(g.cap);
    for (int64_t u = 0; u < n; ++u) sm[u * blockDim.x + threadIdx.x] = make_ulonglong2(0, 0);
  }
  __device__ __forceinline__ void add(Item<SH>& it, const KParams& kp, int r, bool live) {
    bool ok;
    const uint64_t s = row_perfect_index<SH>(gd, it, kp, r, ok);
    bad |= !ok && live;
    if (!(ok && live)) return;
    uint64_t v[SW];
#pragma unroll
    for (int j = 0; j < SW; ++j) v[j] = 0;
    bool fits = true;  // every narrow value within the limit
    static_for<NA>([&](auto a) {
      constexpr int I = decltype(a)::value;
      using AG = typename At<I, typename A::L>::type;
      constexpr int WI = L.word[I], HI = L.half[I];
      const int64_t x = agg_value<AG>(it, kp, r);
      if constexpr (HI >= 0) {
        fits = fits && static_cast<uint64_t>(x) <= g.narrow_limit;
        v[WI] += static_cast<uint64_t>(static_cast<uint32_t>(x)) << (32 * HI);
      } else {
        v[WI] = acc_code<AG::func>(x);
      }
    });
    if constexpr (CA < 0) {
      constexpr int WC = L.word[NA], HC = L.half[NA];
      v[WC] += HC >= 0 ? (1ull << (32 * HC)) : 1ull;
    }
    if constexpr (NARROW) {
      if (!fits) {  // a value too large for the 32-bit fields: straight to the global table
        uint64_t c[NA + 1];
        row_codes<SH>(it, kp, r, ~0ull, c);
        slot_atomic_add<SH>(g.vals + (blockIdx.x % g.replicas) * g.rep_stride + s * g.stride, c);
        return;
      }
    }
    // unit J of slot s: sbase + (s * SP + J) * ustride; volatile asm keeps
    // each read-modify-write in program order (rows may share a slot).  A
    // narrow word adds both of its fields at once: they cannot carry.
    const uint32_t a = sbase + static_cast<uint32_t>(s) * (SP * ustride);
    const uint32_t us = ustride;
    unsigned long long w[SW];
    static_for<SP>([&](auto j) {
      constexpr int J = decltype(j)::value;
      asm volatile("ld.shared.v2.u64 {%0, %1}, [%2];" : "=l"(w[2 * J]), "=l"(w[2 * J + 1]) : "r"(a + J * us)
                   : "memory");
    });
    static_for<SP>([&](auto j) {
      constexpr int J = decltype(j)::value;
      const unsigned long long x = acc_combine<word_func<2 * J>()>(w[2 * J], v[2 * J]);
      const unsigned long long y = acc_combine<word_func<2 * J + 1>()>(w[2 * J + 1], v[2 * J + 1]);
      asm volatile("st.shared.v2.u64 [%0], {%1, %2};" ::"r"(a + J * us), "l"(x), "l"(y) : "memory");
    });
  }
  // CTA epilogue: one warp per (slot, word) folds the word over the CTA's
  // threads (32-bit fields summed as 64-bit values) and adds the result into
  // the aggregate's word of the global table.
  __device__ void finish() {
    if (bad) set_error(err, PV_ERR_KEY_OUT_OF_RANGE);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const unsigned long long* w64 = reinterpret_cast<const unsigned long long*>(sm);
    int agg0[SW], agg1[SW];  // aggregate of each word's fields
    static_for<SW>([&](auto jj) {
      constexpr int J = decltype(jj)::value;
      constexpr int a0 = L.agg[J][0], a1 = L.agg[J][1];
      agg0[J] = a0;
      agg1[J] = a1;
    });
    for (int64_t w = warp; w < g.cap * SW; w += nwarps) {
      const int64_t slot = w / SW;
      const int j = static_cast<int>(w % SW);
      const int64_t unit = slot * SP + j / 2;
      unsigned long long* dst = g.vals + (blockIdx.x % g.replicas) * g.rep_stride + slot * g.stride;
      if (j < NW) {
        uint64_t lo = 0, hi = 0;
        for (int t = lane; t < static_cast<int>(blockDim.x); t += 32) {
          const uint64_t x = w64[2 * (unit * blockDim.x + t) + (j & 1)];
          lo += x & 0xffffffffull;
          hi += x >> 32;
        }
        lo = warp_reduce<PV_SUM>(lo);
        hi = warp_reduce<PV_SUM>(hi);
        if (lane == 0) {
          if (lo && agg0[j] >= 0) atomicAdd(dst + agg0[j], static_cast<unsigned long long>(lo));
          if (hi && agg1[j] >= 0) atomicAdd(dst + agg1[j], static_cast<unsigned long long>(hi));
        }
        continue;
      }
      const int ag = agg0[j];
      if (ag < 0) continue;  // padding
      const bool add = ag >= NA || gd.func[ag] == PV_SUM || gd.func[ag] == PV_COUNT;
      uint64_t v = 0;
      for (int t = lane; t < static_cast<int>(blockDim.x); t += 32) {
        const uint64_t x = w64[2 * (unit * blockDim.x + t) + (j & 1)];
        v = add ? v + x : (x > v ? x : v);
      }
      v = add ? warp_reduce<PV_SUM>(v) : warp_reduce<PV_MAX>(v);
      if (lane == 0 && v) {
        if (add) atomicAdd(dst + ag, static_cast<unsigned long long>(v));
        else atomicMax(dst + ag, static_cast<unsigned long long>(v));
      }
    }
  }
};
template <class SH> using SinkThreadPerfectW = SinkThreadPerfect<SH, false>;
template <class SH> using SinkThreadPerfectN = SinkThreadPerfect<SH, true>;

// CTA-local linear-probing table in shared memory; rows whose key does not
// find a place within kLocalProbe steps go straight to the global table.
template <class SH, int GM>
struct SinkLocalHash {
  static constexpr int NA = SH::Aggs::N;
  const GroupDesc& gd; const GroupOut& g; int32_t* err; unsigned long long* lk; unsigned long long* lv;
  __device__ SinkLocalHash(const GroupDesc& d, const GroupOut& o, int32_t* e, unsigned long long* s)
      : gd(d), g(o), err(e), lk(s), lv(s + o.local_slots) {}
  __device__ void init() {
    for (int i = threadIdx.x; i < g.local_slots; i += blockDim.x) lk[i] = kEmpty64;
    for (int64_t i = threadIdx.x; i < static_cast<int64_t>(g.local_slots) * g.stride; i += blockDim.x) lv[i] = 0;
    __syncthreads();
  }
  __device__ __forceinline__ void add(Item<SH>& it, const KParams& kp, int r, bool live) {
    bool in_domain;
    const uint64_t key = group_key<SH>(gd, it, kp, r, in_domain);
    if (!in_domain && live) set_error(err, PV_ERR_KEY_OUT_OF_RANGE);
    uint64_t c[NA + 1];
    row_codes<SH>(it, kp, r, live && in_domain ? ~0ull : 0ull, c);
    if (key != kEmpty64) {
      const uint32_t mask = static_cast<uint32_t>(g.local_slots) - 1;
      uint32_t idx = static_cast<uint32_t>(fmix64(key)) & mask;
      for (int step = 0; step < kLocalProbe; ++step) {
        unsigned long long cur = *reinterpret_cast<volatile unsigned long long*>(lk + idx);
        if (cur == kEmpty64) cur = atomicCAS(lk + idx, kEmpty64, static_cast<unsigned long long>(key));
        if (cur == kEmpty64 || cur == key) {
          slot_atomic_add<SH, true>(lv + static_cast<uint64_t>(idx) * g.stride, c);
          return;
        }
        idx = (idx + 1) & mask;
      }
    }
    const uint64_t s = global_slot<GM>(g, key, err);
    if (s <= static_cast<uint64_t>(g.cap)) slot_atomic_add<SH>(g.vals + s * g.stride, c);
  }
  __device__ void finish() {
    __syncthreads();
    for (int i = threadIdx.x; i < g.local_slots; i += blockDim.x) {
      const uint64_t key = lk[i];
      if (key == kEmpty64) continue;
      uint64_t c[NA + 1];
#pragma unroll
      for (int a = 0; a <= NA; ++a) c[a] = lv[static_cast<uint64_t>(i) * g.stride + a];
      if (!c[count_index<typename SH::Aggs>() >= 0 ? count_index<typename SH::Aggs>() : NA]) continue;
      const uint64_t s = global_slot<GM>(g, key, err);
      if (s <= static_cast<uint64_t>(g.cap)) slot_atomic_add<SH>(g.vals + s * g.stride, c);
    }
  }
};

// Extraction: a warp-uniform sweep (thread t of T) over the cap + 1 slots;
// non-empty slots are appended to the dense result columns with one atomicAdd
// per warp, then emptied.  Slot words are read from L2: they were written by
// atomics of other CTAs.
__device__ __forceinline__ int64_t decode_agg(int func, uint64_t c) {
  if (func == PV_MIN) return decode_min(c);
  if (func == PV_MAX) return decode_max(c);
  return static_cast<int64_t>(c);
}

// Key columns of result row pos.  code: v is a mixed-radix slot code (perfect
// arrays, keys of three parts), decoded part by part from the last; else v is
// a packed hash key (one part, or two 32-bit halves).
__device__ __forceinline__ void write_keys(const GroupDesc& gd, const GroupOut& g, int64_t pos, bool code, uint64_t v) {
  if (code) {
    for (int i = gd.n_keys - 1; i > 0; --i) {
      const uint64_t span = static_cast<uint64_t>(gd.key_span[i]);
      g.out[i * g.out_cap + pos] = gd.key_min[i] + static_cast<int64_t>(v % span);
      v /= span;
    }
    g.out[pos] = gd.key_min[0] + static_cast<int64_t>(v);
  } else if (gd.n_keys == 1) {
    g.out[pos] = gd.key64[0] ? static_cast<int64_t>(v) : static_cast<int64_t>(static_cast<int32_t>(static_cast<uint32_t>(v)));
  } else {
    g.out[pos] = static_cast<int32_t>(static_cast<uint32_t>(v >> 32));
    g.out[g.out_cap + pos] = static_cast<int32_t>(static_cast<uint32_t>(v));
  }
}

__device__ __forceinline__ void extract_slots(const GroupDesc& gd, const GroupOut& g, int64_t t, int64_t T) {
  const int64_t total = g.cap + 1;
  const int lane = threadIdx.x & 31;
  const bool perfect = g.ht == PV_HT_PERFECT;
  const int na = gd.n_aggs;
  for (int64_t wb = t - lane; wb < total; wb += T) {
    const int64_t s = wb + lane;
    bool occ = false, dirty = false;
    uint64_t key = kEmpty64;
    unsigned long long* v = g.vals + s * g.stride;
    if (s < total) {
      if (perfect) {
        occ = s < g.cap && __ldcg(v + gd.count_word) != 0;
        dirty = occ;
      } else if (s < g.cap) {
        key = __ldcg(g.keys + s);
        dirty = key != kEmpty64;
        occ = dirty && __ldcg(v + gd.count_word) != 0;
      } else {
        occ = dirty = __ldcg(v + gd.count_word) != 0;
      }
    }
    const unsigned ball = __ballot_sync(0xffffffffu, occ);
    unsigned long long base = 0;
    if (lane == 0 && ball) base = atomicAdd(g.out_count, static_cast<unsigned long long>(__popc(ball)));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (occ) {
      const int64_t pos = static_cast<int64_t>(base) + __popc(ball & ((1u << lane) - 1u));
      if (pos < g.out_cap) {
        write_keys(gd, g, pos, perfect || gd.coded, perfect ? static_cast<uint64_t>(s) : key);
        for (int a = 0; a < na; ++a) g.out[(gd.n_keys + a) * g.out_cap + pos] = decode_agg(gd.func[a], __ldcg(v + a));
      }
    }
    if (dirty) {
      for (int a = 0; a <= na; ++a) v[a] = 0;
      if (!perfect && s < g.cap) g.keys[s] = kEmpty64;
    }
  }
}

// Extraction of a replicated perfect table: one warp per slot (warp w of W
// takes slots w, w + W, ...).  Lane r reads replica r's words (independent
// loads, one round trip), a warp reduction folds them (add, or max of the
// MIN/MAX codes), lane 0 appends the group and each lane empties its replica.
__device__ __forceinline__ void extract_replicated(const GroupDesc& gd, const GroupOut& g, int64_t t, int64_t T) {
  const int lane = threadIdx.x & 31;
  const int na = gd.n_aggs;
  const bool mine = lane < g.replicas;
  for (int64_t s = t >> 5; s < g.cap; s += T >> 5) {
    unsigned long long* v = g.vals + s * g.stride + (mine ? lane : 0) * g.rep_stride;
    uint64_t w[PV_MAX_AGGS + 1];
#pragma unroll
    for (int a = 0; a <= PV_MAX_AGGS; ++a) w[a] = (a <= na && mine) ? __ldcg(v + a) : 0;
#pragma unroll
    for (int a = 0; a <= PV_MAX_AGGS; ++a) {
      if (a > na) break;
      const bool add = a == na || gd.func[a] == PV_SUM || gd.func[a] == PV_COUNT;
      w[a] = add ? warp_reduce<PV_SUM>(w[a]) : warp_reduce<PV_MAX>(w[a]);
    }
    if (w[gd.count_word] == 0) continue;  // the same for every lane after the reduction
    if (lane == 0) {
      const int64_t pos = static_cast<int64_t>(atomicAdd(g.out_count, 1ull));
      if (pos < g.out_cap) {
        write_keys(gd, g, pos, true, static_cast<uint64_t>(s));
        for (int a = 0; a < na; ++a) g.out[(gd.n_keys + a) * g.out_cap + pos] = decode_agg(gd.func[a], w[a]);
      }
    }
    if (mine)
      for (int a = 0; a <= na; ++a) v[a] = 0;
  }
}


// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------
// Register cap and loop form of a sink: 128 registers and the software-
// pipelined predicated loop unless the sink states otherwise.
template <class S, class = void> struct SinkRegs { static constexpr int value = 128; };
template <class S> struct SinkRegs<S, std::void_t<decltype(S::kRegs)>> { static constexpr int value = S::kRegs; };
template <class S, class = void> struct SinkIsCluster { static constexpr bool value = false; };
template <class S> struct SinkIsCluster<S, std::void_t<decltype(S::kCluster)>> {
  static constexpr bool value = S::kCluster;
};
template <class S, class = void> struct SinkStaged { static constexpr bool value = false; };
template <class S> struct SinkStaged<S, std::void_t<decltype(S::kStaged)>> { static constexpr bool value = S::kStaged; };
template <class S, class = void> struct SinkPipelined { static constexpr bool value = true; };
template <class S> struct SinkPipelined<S, std::void_t<decltype(S::kPipelined)>> {
  static constexpr bool value = S::kPipelined;
};

// Branched kernels of small shapes (at most two aggregates) are held to 64
// registers, so two 512-thread CTAs share an SM: they are latency-bound
// (lazy loads and probes), and occupancy hides the latency.
template <class SH, class Sink, bool PRED> struct GroupRegs {
  static constexpr int value = !PRED && SH::Aggs::N <= 2 ? 64 : SinkRegs<Sink>::value;
};

template <class SH, bool PRED, bool CHUNK, int U, class Sink>
__global__ void __maxnreg__((GroupRegs<SH, Sink, PRED>::value)) k_group(const __grid_constant__ KParams kp, const __grid_constant__ GroupDesc gd, const __grid_constant__ GroupOut g) {
  extern __shared__ unsigned long long smem[];
  if (blockIdx.x == 0 && threadIdx.x == 0) *g.out_count = 0;  // extraction runs after this kernel
  Sink sink(gd, g, kp.err, smem);
  sink.init();
  auto consume = [&](Item<SH> (&it)[U]) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (!PRED && !it[u].mask) continue;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const bool live = (it[u].mask >> r) & 1u;
        if (PRED ? r < it[u].nvalid : live) sink.add(it[u], kp, r, live);
      }
    }
  };
  if constexpr (PRED && SinkPipelined<Sink>::value) {
    for_items_pipelined<SH, CHUNK, U>(kp, consume);
  } else if constexpr (PRED && !CHUNK) {
    for_items_pred<SH, U>(kp, [&](Item<SH>& it, auto full) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const bool live = (it.mask >> r) & 1u;
        if constexpr (decltype(full)::value) sink.add(it, kp, r, live);
        else if (r < it.nvalid) sink.add(it, kp, r, live);
      }
    });
  } else if constexpr (PRED) {
    for_items<CHUNK, U>(kp.n_items, [&](const int64_t (&idx)[U]) {
      Item<SH> it[U];
      eval_items<SH, PRED, U>(it, kp, idx);
      consume(it);
    });
  } else {
    for_items_pf<SH, CHUNK, U, first_stage_slots<SH>()>(kp, [&](const int64_t (&idx)[U]) {
      Item<SH> it[U];
      eval_items<SH, PRED, U>(it, kp, idx);
      consume(it);
    });
  }
  pdl_launch_dependents();  // the extraction kernel may start launching now
  sink.finish();
}

// TMA-staged access (predicated): the warps' stages and mbarriers come first
// in shared memory, the sink's tables after them.
template <class SH, class Sink>
__global__ void __maxnreg__((GroupRegs<SH, Sink, true>::value)) k_group_staged(
    const __grid_constant__ KParams kp, const __grid_constant__ GroupDesc gd, const __grid_constant__ GroupOut g) {
  extern __shared__ unsigned long long smem[];
  if (blockIdx.x == 0 && threadIdx.x == 0) *g.out_count = 0;  // extraction runs after this kernel
  char* stages = reinterpret_cast<char*>(smem);
  Sink sink(gd, g, kp.err, reinterpret_cast<unsigned long long*>(stages + stage_smem<SH>(blockDim.x >> 5)));
  sink.init();
  for_items_staged<SH>(kp, stages, [&](Item<SH>& it, auto full) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const bool live = (it.mask >> r) & 1u;
      if constexpr (decltype(full)::value) sink.add(it, kp, r, live);
      else if (r < it.nvalid) sink.add(it, kp, r, live);
    }
  });
  pdl_launch_dependents();
  sink.finish();
}

// Compacted execution of a grouped pipeline: for_rows_compacted queues the
// survivors of the first stage (the filters, else the first NF probes) per
// warp; each queued row runs the other probes, the sink's column loads and
// the sink, K rows per lane.
template <class SH, class Sink, int K, int NF, int FI>
__global__ void __maxnreg__((GroupRegs<SH, Sink, false>::value)) k_group_compact(
    const __grid_constant__ KParams kp, const __grid_constant__ GroupDesc gd, const __grid_constant__ GroupOut g) {
  extern __shared__ unsigned long long smem[];
  const int nwarps = blockDim.x >> 5;
  uint32_t* q = reinterpret_cast<uint32_t*>(smem) + (threadIdx.x >> 5) * queue_cap<K>();
  if (blockIdx.x == 0 && threadIdx.x == 0) *g.out_count = 0;  // extraction runs after this kernel
  Sink sink(gd, g, kp.err, smem + nwarps * queue_cap<K>() / 2);  // the queues, 4 bytes an entry
  sink.init();
  for_rows_compacted<SH, K, NF, false, FI>(kp, q, [&](const uint32_t (&rows)[K], const bool (&has)[K]) {
    Item<SH> it[K];
    bool ok[K];
    compact_load_rows<SH, K, NF>(it, ok, kp, rows, has);
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (ok[k]) sink.add(it[k], kp, 0, true);
  });
  pdl_launch_dependents();
  sink.finish();
}

// Key pass of the multi-pass strategy: insert the group key of every row
// (every valid row when predicated) into the global linear or cuckoo table.
template <class SH, bool PRED, bool CHUNK, int U, int HTK>
__global__ void __maxnreg__(128) k_group_keys(const __grid_constant__ KParams kp, const __grid_constant__ GroupDesc gd, const __grid_constant__ GroupOut g) {
  for_items<CHUNK, U>(kp.n_items, [&](const int64_t (&idx)[U]) {
    Item<SH> it[U];
    eval_items<SH, PRED, U>(it, kp, idx);
#pragma unroll
    for (int u = 0; u < U; ++u) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const bool live = (it[u].mask >> r) & 1u;
        if (PRED ? r < it[u].nvalid : live) {
          bool in_domain;
          const uint64_t key = group_key<SH>(gd, it[u], kp, r, in_domain);
          if (!in_domain && live) set_error(kp.err, PV_ERR_KEY_OUT_OF_RANGE);
          if constexpr (HTK == PV_HT_CUCKOO) global_cuckoo_insert(g, key, kp.err);
          else global_linear_slot(g, key, kp.err);
        }
      }
    }
  });
}

// Removes cuckoo duplicates: a key is kept only at the first of its k
// candidate slots that holds it.
__global__ void k_cuckoo_dedupe(const __grid_constant__ GroupOut g);
// Compacts non-empty slots into the dense result columns and empties them.
__global__ void k_extract(const __grid_constant__ GroupDesc gd, const __grid_constant__ GroupOut g);
pv_status launch_dedupe_extract(const LaunchCfg& c, const GroupDesc& gd, const GroupOut& g, bool dedupe);

template <class SH> using SinkGInsert = SinkGlobalHash<SH, G_INSERT>;
template <class SH> using SinkGLookupLinear = SinkGlobalHash<SH, G_LOOKUP_LINEAR>;
template <class SH> using SinkGLookupCuckoo = SinkGlobalHash<SH, G_LOOKUP_CUCKOO>;
template <class SH> using SinkLInsert = SinkLocalHash<SH, G_INSERT>;
template <class SH> using SinkLLookupLinear = SinkLocalHash<SH, G_LOOKUP_LINEAR>;
template <class SH> using SinkLLookupCuckoo = SinkLocalHash<SH, G_LOOKUP_CUCKOO>;

template <class K>
static pv_status launch_k(const LaunchCfg& c, K k, const KParams& kp, const GroupDesc& gd, const GroupOut& g,
                          size_t smem, int U) {
  if (smem > 48 * 1024) {
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess)
      return PV_ERR_UNSUPPORTED;
  }
  const int grid = grid_for(c, reinterpret_cast<const void*>(k), smem, kp.n_items, static_cast<int64_t>(c.block) * U);
  if (grid <= 0) return PV_ERR_UNSUPPORTED;
  // rows one thread visits, at most: its items (grid-stride, chunked or staged) of 4 rows, or for
  // compacted execution as many queued rows, plus one partial drain
  const int64_t T = static_cast<int64_t>(grid) * c.block;
  GroupOut g2 = g;
  g2.narrow_limit = static_cast<uint64_t>(UINT32_MAX) / static_cast<uint64_t>(4 * ((kp.n_items + T - 1) / T) + 4);
  if (g.narrow_check && g.narrow_max > g2.narrow_limit) return kNeedWide;
  kmark(c);
  k<<<grid, c.block, smem, c.stream>>>(kp, gd, g2);
  kmark(c);
  ++*c.launches;
  return cudaGetLastError() == cudaSuccess ? PV_OK : PV_ERR_CUDA;
}

template <class SH, template <class> class SinkT, int NF, int FI>
static pv_status run_group_compact_fi(const LaunchCfg& c, const KParams& kp, const GroupDesc& gd, const GroupOut& g,
                                      size_t sink_smem) {
  if (c.U == 4) {
    const size_t smem = static_cast<size_t>(c.block / 32) * queue_cap<4>() * 4 + sink_smem;
    return launch_k(c, k_group_compact<SH, SinkT<SH>, 4, NF, FI>, kp, gd, g, smem, FI);
  }
  if (c.U == 2) {
    const size_t smem = static_cast<size_t>(c.block / 32) * queue_cap<2>() * 4 + sink_smem;
    return launch_k(c, k_group_compact<SH, SinkT<SH>, 2, NF, FI>, kp, gd, g, smem, FI);
  }
  const size_t smem = static_cast<size_t>(c.block / 32) * queue_cap<1>() * 4 + sink_smem;
  return launch_k(c, k_group_compact<SH, SinkT<SH>, 1, NF, FI>, kp, gd, g, smem, FI);
}

// first_items 2: filter-first pipelines only (first_items_max).
template <class SH, template <class> class SinkT, int NF>
static pv_status run_group_compact_nf(const LaunchCfg& c, const KParams& kp, const GroupDesc& gd, const GroupOut& g,
                                      size_t sink_smem) {
  if (c.first_items > first_items_max<SH>()) return PV_ERR_UNSUPPORTED;
  if constexpr (first_items_max<SH>() == 2) {
    if (c.first_items == 2) return run_group_compact_fi<SH, SinkT, NF, 2>(c, kp, gd, g, sink_smem);
  }
  return run_group_compact_fi<SH, SinkT, NF, 1>(c, kp, gd, g, sink_smem);
}

template <class SH, template <class> class SinkT>
static pv_status run_group_compact(const LaunchCfg& c, const KParams& kp, const GroupDesc& gd, const GroupOut& g,
                                   size_t sink_smem) {
  if constexpr (SH::Where::N == 0 && SH::Probes::N == 0) {
    return PV_ERR_UNSUPPORTED;  // nothing to compact on
  } else {
    // items_per_thread: queued rows a lane takes through the row stage at once
    if (c.chunk || (c.U != 1 && c.U != 2 && c.U != 4) || kp.n_rows > static_cast<int64_t>(UINT32_MAX))
      return PV_ERR_UNSUPPORTED;
    if (c.compact_probes == 2) {
      // a second first-stage probe: only pipelines of two or more probes and no filters
      if constexpr (SH::Where::N == 0 && SH::Probes::N >= 2) return run_group_compact_nf<SH, SinkT, 2>(c, kp, gd, g, sink_smem);
      else return PV_ERR_UNSUPPORTED;
    }
    return run_group_compact_nf<SH, SinkT, 1>(c, kp, gd, g, sink_smem);
  }
}

// Launch as clusters of C = 2^g.cluster_log2 CTAs: the grid is the
// co-resident clusters times C (or grid_mult x SMs rounded down to whole
// clusters), unsupported when no cluster of this kernel fits.
template <class K>
static pv_status launch_k_cluster(const LaunchCfg& c, K k, const KParams& kp, const GroupDesc& gd,
                                  const GroupOut& g, size_t smem) {
  const int cl = 1 << g.cluster_log2;
  if (smem > 48 * 1024) {
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess)
      return PV_ERR_UNSUPPORTED;
  }
  if (cl > 8 && cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return PV_ERR_UNSUPPORTED;
  }
  cudaLaunchConfig_t cfg{};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(c.block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = c.stream;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3(cl);
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, k, &cfg) != cudaSuccess || clusters <= 0) {
    cudaGetLastError();
    return PV_ERR_UNSUPPORTED;
  }
  int64_t grid = c.grid_mult > 0 ? (static_cast<int64_t>(c.grid_mult) * c.sm_count) / cl * cl
                                 : static_cast<int64_t>(clusters) * cl;
  grid = std::max<int64_t>(cl, std::min<int64_t>(grid, static_cast<int64_t>(clusters) * cl));
  cfg.gridDim = dim3(static_cast<unsigned>(grid));
  kmark(c);
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k, kp, gd, g);
  kmark(c);
  ++*c.launches;
  return e == cudaSuccess ? PV_OK : PV_ERR_CUDA;
}

// UMASK: bit 0 = unroll 1 compiled, bit 1 = unroll 2 compiled.
template <class SH, int UMASK, template <class> class SinkT>
static pv_status run_group(const LaunchCfg& c, const KParams& kp, const GroupDesc& gd, const GroupOut& g, size_t smem) {
  using S = SinkT<SH>;
  if (c.staged) {
    if constexpr (SinkStaged<S>::value) {
      if (c.compact || !c.pred || c.U != 1 || kp.prefetch != 0) return PV_ERR_UNSUPPORTED;
      return launch_k(c, k_group_staged<SH, S>, kp, gd, g, stage_smem<SH>(c.block / 32) + smem, 1);
    } else {
      return PV_ERR_UNSUPPORTED;
    }
  }
  if constexpr (SinkIsCluster<S>::value) {
    if (c.compact || c.U != 1) return PV_ERR_UNSUPPORTED;
    if (c.pred) return c.chunk ? launch_k_cluster(c, k_group<SH, true, true, 1, S>, kp, gd, g, smem)
                               : launch_k_cluster(c, k_group<SH, true, false, 1, S>, kp, gd, g, smem);
    return c.chunk ? launch_k_cluster(c, k_group<SH, false, true, 1, S>, kp, gd, g, smem)
                   : launch_k_cluster(c, k_group<SH, false, false, 1, S>, kp, gd, g, smem);
  } else {
    if (c.compact) return run_group_compact<SH, SinkT>(c, kp, gd, g, smem);
    if constexpr ((UMASK & 1) != 0) if (c.U == 1) {
      if (c.pred) return c.chunk ? launch_k(c, k_group<SH, true, true, 1, S>, kp, gd, g, smem, 1)
                                 : launch_k(c, k_group<SH, true, false, 1, S>, kp, gd, g, smem, 1);
      return c.chunk ? launch_k(c, k_group<SH, false, true, 1, S>, kp, gd, g, smem, 1)
                     : launch_k(c, k_group<SH, false, false, 1, S>, kp, gd, g, smem, 1);
    }
    if constexpr ((UMASK & 2) != 0) if (c.U == 2) {
      if (c.pred) return c.chunk ? launch_k(c, k_group<SH, true, true, 2, S>, kp, gd, g, smem, 2)
                                 : launch_k(c, k_group<SH, true, false, 2, S>, kp, gd, g, smem, 2);
      return c.chunk ? launch_k(c, k_group<SH, false, true, 2, S>, kp, gd, g, smem, 2)
                     : launch_k(c, k_group<SH, false, false, 2, S>, kp, gd, g, smem, 2);
    }
    return PV_ERR_UNSUPPORTED;
  }
}

template <class SH, int UMASK, int HTK>
static pv_status run_keys(const LaunchCfg& c, const KParams& kp, const GroupDesc& gd, const GroupOut& g) {
  if constexpr ((UMASK & 1) != 0) if (c.U == 1) {
    if (c.pred) return c.chunk ? launch_k(c, k_group_keys<SH, true, true, 1, HTK>, kp, gd, g, 0, 1)
                               : launch_k(c, k_group_keys<SH, true, false, 1, HTK>, kp, gd, g, 0, 1);
    return c.chunk ? launch_k(c, k_group_keys<SH, false, true, 1, HTK>, kp, gd, g, 0, 1)
                   : launch_k(c, k_group_keys<SH, false, false, 1, HTK>, kp, gd, g, 0, 1);
  }
  if constexpr ((UMASK & 2) != 0) if (c.U == 2) {
    if (c.pred) return c.chunk ? launch_k(c, k_group_keys<SH, true, true, 2, HTK>, kp, gd, g, 0, 2)
                               : launch_k(c, k_group_keys<SH, true, false, 2, HTK>, kp, gd, g, 0, 2);
    return c.chunk ? launch_k(c, k_group_keys<SH, false, true, 2, HTK>, kp, gd, g, 0, 2)
                   : launch_k(c, k_group_keys<SH, false, false, 2, HTK>, kp, gd, g, 0, 2);
  }
  return PV_ERR_UNSUPPORTED;
}

// HASH_AGGREGATE under one variant: picks the sink (strategy x table kind x
// pass count), enqueues the key pass if any, the aggregation kernel and the
// extraction kernel.
template <class SH, int UMASK>
static pv_status launch_group(const LaunchCfg& c, const KParams& kp, const GroupDesc& gd, const GroupOut& g0,
                              const pv_variant& v) {
  GroupOut g = g0;
  const bool multi = v.exec == PV_EXEC_MULTI_PASS;
  const bool local = v.agg == PV_AGG_LOCAL;
  if (multi && (c.compact || c.staged)) return PV_ERR_UNSUPPORTED;  // the key pass has neither form
  if (v.agg != PV_AGG_LOCAL && v.agg != PV_AGG_GLOBAL && v.agg != PV_AGG_CLUSTER) return PV_ERR_INVALID_ARG;
  if (v.agg == PV_AGG_CLUSTER) {  // perfect arrays in the distributed shared memory of a cluster
    if (g.ht != PV_HT_PERFECT || multi || v.threads_per_table == 1) return PV_ERR_UNSUPPORTED;
    // the smallest cluster (2..16 CTAs) whose part fits: fewer CTAs keep more updates local (8 CTAs with
    // 150 KB parts measured faster than 16 with 75 KB on 5e4 skewed groups)
    int l = 1;
    auto part_bytes = [&](int lg) {
      return static_cast<size_t>(SinkClusterPerfect<SH>::part_slots(g.cap, lg)) * g.stride * 8;
    };
    while ((1 << l) < kMaxClusterCTAs && part_bytes(l) > kClusterBytes) ++l;
    const size_t smem = part_bytes(l);
    if (smem > kClusterBytes) return PV_ERR_UNSUPPORTED;
    g.cluster_log2 = l;
    const pv_status s = run_group<SH, UMASK, SinkClusterPerfect>(c, kp, gd, g, smem);
    if (s != PV_OK) return s;
    return launch_dedupe_extract(c, gd, g, false);
  }
  const size_t slot_bytes = static_cast<size_t>(g.stride) * 8;
  pv_status s;
  if (g.ht == PV_HT_PERFECT) {
    if (multi) return PV_ERR_UNSUPPORTED;  // no keys to insert
    if (!local) {
      s = run_group<SH, UMASK, SinkGlobalPerfect>(c, kp, gd, g, 0);
    } else if (v.threads_per_table == 1) {
      // 32-bit fields for the narrow aggregates when that saves words per slot
      if constexpr (SinkThreadPerfectN<SH>::SW < SinkThreadPerfectW<SH>::SW) {
        const size_t smem = SinkThreadPerfectN<SH>::smem_bytes(g.cap, c.block);
        if (smem > 200 * 1024) return PV_ERR_UNSUPPORTED;
        GroupOut gn = g;
        gn.narrow_check = 1;
        s = run_group<SH, UMASK, SinkThreadPerfectN>(c, kp, gd, gn, smem);
        if (s == kNeedWide) {
          const size_t wsmem = SinkThreadPerfectW<SH>::smem_bytes(g.cap, c.block);
          if (wsmem > 200 * 1024) return PV_ERR_UNSUPPORTED;
          s = run_group<SH, UMASK, SinkThreadPerfectW>(c, kp, gd, g, wsmem);
        }
      } else {
        const size_t smem = SinkThreadPerfectW<SH>::smem_bytes(g.cap, c.block);
        if (smem > 200 * 1024) return PV_ERR_UNSUPPORTED;
        s = run_group<SH, UMASK, SinkThreadPerfectW>(c, kp, gd, g, smem);
      }
    } else {
      const size_t smem = static_cast<size_t>(g.cap) * slot_bytes;
      if (smem > kLocalPerfectBytes) return PV_ERR_UNSUPPORTED;
      s = run_group<SH, UMASK, SinkLocalPerfect>(c, kp, gd, g, smem);
    }
    if (s != PV_OK) return s;
    return launch_dedupe_extract(c, gd, g, false);
  }
  if (v.threads_per_table == 1) return PV_ERR_UNSUPPORTED;
  const bool cuckoo = g.ht == PV_HT_CUCKOO;
  if (cuckoo && !multi) return PV_ERR_UNSUPPORTED;  // keys move while inserting
  if (multi) {
    s = cuckoo ? run_keys<SH, UMASK, PV_HT_CUCKOO>(c, kp, gd, g) : run_keys<SH, UMASK, PV_HT_LINEAR>(c, kp, gd, g);
    if (s != PV_OK) return s;
    if (cuckoo) {
      s = launch_dedupe_extract(c, gd, g, true);
      if (s != PV_OK) return s;
    }
  }
  if (!local) {
    s = !multi ? run_group<SH, UMASK, SinkGInsert>(c, kp, gd, g, 0)
               : cuckoo ? run_group<SH, UMASK, SinkGLookupCuckoo>(c, kp, gd, g, 0)
                        : run_group<SH, UMASK, SinkGLookupLinear>(c, kp, gd, g, 0);
  } else {
    int ls = 1;
    while (static_cast<size_t>(ls) * 2 * (slot_bytes + 8) <= kLocalBytes) ls *= 2;
    g.local_slots = ls;
    const size_t smem = static_cast<size_t>(ls) * (slot_bytes + 8);
    s = !multi ? run_group<SH, UMASK, SinkLInsert>(c, kp, gd, g, smem)
               : cuckoo ? run_group<SH, UMASK, SinkLLookupCuckoo>(c, kp, gd, g, smem)
                        : run_group<SH, UMASK, SinkLLookupLinear>(c, kp, gd, g, smem);
  }
  if (s != PV_OK) return s;
  return launch_dedupe_extract(c, gd, g, false);
}

template <class SH, int UMASK = 3>
static void reg_grouped() {
  ShapeEntry e{};
  e.sig = SH::signature();
  e.mode = MODE_GROUPED;
  e.grouped = launch_group<SH, UMASK>;
  register_shape(e);
}

}  // namespace pv
