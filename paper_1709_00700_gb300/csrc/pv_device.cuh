// Device building blocks of the pipeline kernels: the compile-time pipeline
// shape (which columns, predicates, probes, keys, aggregates and projected
// columns a pipeline program has, Table 1), per-item evaluation, vector
// loaders, hash functions and reductions.
//
// A pipeline program is instantiated once per shape and variant; its
// constants (predicate bounds, arithmetic constants, column pointers, hash
// tables) arrive at run time in KParams.  The host builds the same shape
// signature from a pv_pipeline_spec and looks the instantiation up.
#pragma once

#include <cstdint>
#include <string>
#include <cuda_runtime.h>

#include "pv.h"

namespace pv {

constexpr int kMaxSlots = 8;
constexpr int kMaxConsts = PV_MAX_AGGS * PV_MAX_TERMS;
constexpr uint64_t kEmpty64 = ~0ull;
constexpr uint32_t kEmpty32 = 0xFFFFFFFFu;

// ---------------------------------------------------------------------------
// Runtime parameters
// ---------------------------------------------------------------------------

// A build-side (probe) hash table.  Slots are 64-bit: key in the high half,
// payload in the low half.  Linear/cuckoo: the high half 0xFFFFFFFF marks an
// empty slot, and a real key equal to -1 lives in the side slot slots[cap].
// Perfect: slot (key - kmin) holds (payload << 32) | 1, 0 when empty.
struct DevHT {
  uint64_t* slots;
  const uint32_t* bits;  // perfect array without payload, or past 64 KB of slots: presence bit per
                         // slot (probes test it first, then read the slot of a hit for its payload)
  const uint8_t* codes;  // perfect array whose one payload spans at most 255 values: one byte per
                         // slot, 0 = empty, else payload - code_base (probes read it, not the slots)
  int32_t code_base;
  int32_t kind;      // pv_ht_kind
  int32_t hash;      // pv_hash_fn
  int32_t log2cap;
  int32_t k;         // cuckoo functions
  int32_t narrow;    // perfect: kmin >= INT32_MIN and kmin + cap <= 2^31, so 32-bit keys index in 32 bits
  int32_t payload;   // slots carry a payload
  int64_t cap;       // slots (power of two for linear/cuckoo; domain size for perfect)
  int64_t kmin;      // perfect: smallest key
  uint64_t seed[4];  // per-function hash seeds
};

struct KParams {
  int64_t n_rows;
  int64_t n_items;               // ceil(n_rows / 4)
  const void* col[kMaxSlots];    // fact column of each slot
  int64_t lo[PV_MAX_PREDS];      // inclusive range per predicate (already clamped
  int64_t hi[PV_MAX_PREDS];      //   to the slot's type; empty range: lo > hi)
  int64_t c[kMaxConsts];         // arithmetic constants, in order of appearance
  DevHT probe[PV_MAX_PROBES];
  int32_t* err;                  // device error word (first error wins)
  int32_t prefetch;              // L2 bulk-prefetch distance in loop trips (0 = off)
};

__device__ __forceinline__ void set_error(int32_t* err, int32_t code) {
  if (*reinterpret_cast<volatile int32_t*>(err) == 0) atomicCAS(err, 0, code);
}

// ---------------------------------------------------------------------------
// Hash functions (Section 9.2.2: Murmur or multiply-shift).  Murmur: the
// 64-bit MurmurHash3 finaliser (fmix64) of key ^ seed.  Multiply-shift
// (Dietzfelbinger et al.): odd multiplier a, top bits of a * key.  Both
// return the top log2cap bits.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t fmix64(uint64_t k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return k;
}

__host__ __device__ __forceinline__ uint64_t ht_index(uint64_t key, int fn, uint64_t seed, int log2cap) {
  uint64_t h = fn == PV_HASH_MURMUR ? fmix64(key ^ seed) : key * (seed | 1ull);
  return log2cap == 0 ? 0 : (h >> (64 - log2cap));
}

// ---------------------------------------------------------------------------
// Column type tags and vector loaders.  One "item" is 4 consecutive rows of a
// thread: one 16-byte load for int32, two for int64, one 4-byte load for uint8.
// ---------------------------------------------------------------------------
struct TI32 { using T = int32_t; static constexpr int code = PV_I32; };
struct TI64 { using T = int64_t; static constexpr int code = PV_I64; };
struct TU8 { using T = uint8_t; static constexpr int code = PV_U8; };

template <class Tag>
__device__ __forceinline__ void load_item(typename Tag::T (&d)[4], const void* base, int64_t item,
                                          int nvalid) {
  using T = typename Tag::T;
  const T* p = static_cast<const T*>(base) + item * 4;
  if (nvalid == 4) {
    if constexpr (sizeof(T) == 4) {
      int4 q = __ldg(reinterpret_cast<const int4*>(p));
      d[0] = q.x; d[1] = q.y; d[2] = q.z; d[3] = q.w;
    } else if constexpr (sizeof(T) == 8) {
      longlong2 a = __ldg(reinterpret_cast<const longlong2*>(p));
      longlong2 b = __ldg(reinterpret_cast<const longlong2*>(p) + 1);
      d[0] = a.x; d[1] = a.y; d[2] = b.x; d[3] = b.y;
    } else {
      uchar4 q = __ldg(reinterpret_cast<const uchar4*>(p));
      d[0] = q.x; d[1] = q.y; d[2] = q.z; d[3] = q.w;
    }
  } else {
#pragma unroll
    for (int r = 0; r < 4; ++r) d[r] = r < nvalid ? p[r] : T(0);
  }
}

// ---------------------------------------------------------------------------
// Type lists
// ---------------------------------------------------------------------------
template <class... Ts> struct TList { static constexpr int N = sizeof...(Ts); };

template <int I, class L> struct At;
template <class T0, class... Ts> struct At<0, TList<T0, Ts...>> { using type = T0; };
template <int I, class T0, class... Ts> struct At<I, TList<T0, Ts...>> { using type = typename At<I - 1, TList<Ts...>>::type; };

template <class F, int... I>
__device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, I...>) {
  (f(std::integral_constant<int, I>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void static_for(F&& f) {
  static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// Per-item values of every slot: a tuple of T[4] arrays.
template <class... Ts> struct VStore;
template <> struct VStore<> {};
template <class T0, class... Ts> struct VStore<T0, Ts...> {
  typename T0::T v[4];
  VStore<Ts...> rest;
};
template <int I> struct VGet {
  template <class S> __device__ __forceinline__ static auto& get(S& s) { return VGet<I - 1>::get(s.rest); }
};
template <> struct VGet<0> {
  template <class S> __device__ __forceinline__ static auto& get(S& s) { return s.v; }
};

// ---------------------------------------------------------------------------
// Shape vocabulary.  Signatures are the canonical text the host matcher
// produces from a pv_pipeline_spec (see pv_api.cu).
// ---------------------------------------------------------------------------
template <class... Ts> struct Cols {
  using L = TList<Ts...>;
  using Store = VStore<Ts...>;
  static constexpr int N = sizeof...(Ts);
  static void sig(std::string& s) {
    s += "C:";
    ((s += (Ts::code == PV_I32 ? "i32," : Ts::code == PV_I64 ? "i64," : "u8,")), ...);
  }
};

template <int S> struct P { static constexpr int slot = S; };
template <class... Ps> struct Where {
  static constexpr int N = sizeof...(Ps);
  static constexpr uint32_t slots = (0u | ... | (1u << Ps::slot));
  using L = TList<Ps...>;
  static void sig(std::string& s) { s += "|W:"; ((s += std::to_string(Ps::slot) + ","), ...); }
};

template <int... S> struct Probes {
  static constexpr int N = sizeof...(S);
  static constexpr int slot_of[N > 0 ? N : 1] = {S...};
  static constexpr uint32_t slots = (0u | ... | (1u << S));
  static void sig(std::string& s) { s += "|J:"; ((s += std::to_string(S) + ","), ...); }
};

// Value sources: slot value, x + c, c - x (ARITHMETIC terms), payload of a probe.
template <int S> struct X {
  static constexpr uint32_t slots = 1u << S;
  static void sig(std::string& s) { s += "x" + std::to_string(S); }
};
template <int S, int CI> struct XPC {
  static constexpr uint32_t slots = 1u << S;
  static void sig(std::string& s) { s += "xpc" + std::to_string(S) + "#" + std::to_string(CI); }
};
template <int S, int CI> struct CMX {
  static constexpr uint32_t slots = 1u << S;
  static void sig(std::string& s) { s += "cmx" + std::to_string(S) + "#" + std::to_string(CI); }
};
template <int J, int I> struct PL {
  static constexpr uint32_t slots = 0;
  static void sig(std::string& s) { s += "p" + std::to_string(J) + "." + std::to_string(I); }
};

template <class... Ts> struct Mul {
  static constexpr uint32_t slots = (0u | ... | Ts::slots);
  static void sig(std::string& s) {
    s += "(";
    ((Ts::sig(s), s += "*"), ...);
    s += ")";
  }
};

template <class E> struct Sum {
  static constexpr int func = PV_SUM;
  static constexpr uint32_t slots = E::slots;
  using Expr = E;
  static void sig(std::string& s) { s += "S"; E::sig(s); }
};
struct Count {
  static constexpr int func = PV_COUNT;
  static constexpr uint32_t slots = 0;
  using Expr = Mul<>;
  static void sig(std::string& s) { s += "N"; }
};
template <class E> struct Min {
  static constexpr int func = PV_MIN;
  static constexpr uint32_t slots = E::slots;
  using Expr = E;
  static void sig(std::string& s) { s += "m"; E::sig(s); }
};
template <class E> struct Max {
  static constexpr int func = PV_MAX;
  static constexpr uint32_t slots = E::slots;
  using Expr = E;
  static void sig(std::string& s) { s += "M"; E::sig(s); }
};

// Aggregates whose per-row value is one plain column value (SUM(x)) or 1
// (COUNT): a thread's partial sum of them fits 32 bits whenever every value
// it adds is at most (2^32 - 1) / rows the thread visits, so a thread-private
// table may keep them as 32-bit fields, two to a 64-bit word.
template <class A> struct NarrowAgg : std::false_type {};
template <> struct NarrowAgg<Count> : std::true_type {};
template <int S> struct NarrowAgg<Sum<Mul<X<S>>>> : std::true_type {};

template <class... As> struct Aggs {
  static constexpr int N = sizeof...(As);
  static constexpr uint32_t slots = (0u | ... | As::slots);
  using L = TList<As...>;
  static constexpr int func_of[N > 0 ? N : 1] = {As::func...};
  static constexpr bool narrow_of[N > 0 ? N : 1] = {NarrowAgg<As>::value...};
  static void sig(std::string& s) { s += "|A:"; ((As::sig(s), s += ","), ...); }
};

template <class... Ks> struct Key {
  static constexpr int N = sizeof...(Ks);
  static constexpr uint32_t slots = (0u | ... | Ks::slots);
  using L = TList<Ks...>;
  static void sig(std::string& s) { s += "|K:"; ((Ks::sig(s), s += ","), ...); }
};

// Projected values in output order: S >= 0 is fact slot S, S < 0 the
// payload of probe -S - 1 (an int32 output column).
template <int... S> struct Proj {
  static constexpr int N = sizeof...(S);
  static constexpr int slot_of[N > 0 ? N : 1] = {S...};
  static constexpr uint32_t slots = (0u | ... | (S >= 0 ? (1u << (S >= 0 ? S : 0)) : 0u));
  static void sig(std::string& s) {
    s += "|P:";
    ((s += (S >= 0 ? std::to_string(S) : "p" + std::to_string(-S - 1)) + ","), ...);
  }
};

template <class C, class W, class J, class K, class A, class PJ>
struct Shape {
  using Cols = C;
  using Where = W;
  using Probes = J;
  using Key = K;
  using Aggs = A;
  using Proj = PJ;
  using Store = typename C::Store;
  static constexpr uint32_t rest_slots = (K::slots | A::slots | PJ::slots) & ~(W::slots | J::slots);
  static std::string signature() {
    std::string s;
    C::sig(s); W::sig(s); J::sig(s); K::sig(s); A::sig(s); PJ::sig(s);
    return s;
  }
};

// ---------------------------------------------------------------------------
// Per-item evaluation: LOOP body of Table 1 for 4 consecutive rows.
// ---------------------------------------------------------------------------
template <class SH>
struct Item {
  typename SH::Store v;
  uint32_t mask;     // surviving rows, bit r for row r of the item
  int nvalid;        // rows of the item inside the table (4 except at the tail)
  int32_t pay[SH::Probes::N > 0 ? SH::Probes::N : 1][4];  // payload bound by each probe
};

template <class SH, uint32_t MASK>
__device__ __forceinline__ void load_slots(Item<SH>& it, const KParams& kp, int64_t item) {
  static_for<SH::Cols::N>([&](auto s) {
    constexpr int S = decltype(s)::value;
    if constexpr ((MASK >> S) & 1u) {
      using Tag = typename At<S, typename SH::Cols::L>::type;
      load_item<Tag>(VGet<S>::get(it.v), kp.col[S], item, it.nvalid);
    }
  });
}

// FILTER: conjunction of closed ranges, one per predicated slot.
template <class SH, int J>
__device__ __forceinline__ uint32_t pred_bits(Item<SH>& it, const KParams& kp) {
  constexpr int S = At<J, typename SH::Where::L>::type::slot;
  using T = typename At<S, typename SH::Cols::L>::type::T;
  auto& v = VGet<S>::get(it.v);
  const T lo = static_cast<T>(kp.lo[J]), hi = static_cast<T>(kp.hi[J]);
  uint32_t b = 0;
#pragma unroll
  for (int r = 0; r < 4; ++r) b |= static_cast<uint32_t>((v[r] >= lo) & (v[r] <= hi)) << r;
  return b;
}

// HASH_PROBE of one key; returns hit and the bound payload.
__device__ __forceinline__ bool probe_key(const DevHT& h, int64_t key, int32_t& pay) {
  if (h.kind == PV_HT_PERFECT) {
    const int64_t i = key - h.kmin;
    if (static_cast<uint64_t>(i) >= static_cast<uint64_t>(h.cap)) return false;
    if (h.codes != nullptr) {  // one byte per key
      const uint32_t b = __ldg(h.codes + i);
      pay = b != 0u ? static_cast<int32_t>(b) + h.code_base : 0;
      return b != 0u;
    }
    if (h.bits != nullptr) {  // 1 bit per key instead of 8 bytes: small enough to stay in L1
      const bool hit = (__ldg(h.bits + (i >> 5)) >> (i & 31)) & 1u;
      pay = hit && h.payload ? static_cast<int32_t>(__ldg(reinterpret_cast<const unsigned long long*>(h.slots) + i) >> 32)
                             : 0;
      return hit;
    }
    const uint64_t s = __ldg(reinterpret_cast<const unsigned long long*>(h.slots) + i);
    pay = static_cast<int32_t>(s >> 32);
    return s != 0;
  }
  if (key != static_cast<int64_t>(static_cast<int32_t>(key))) return false;
  const uint32_t k32 = static_cast<uint32_t>(key);
  if (k32 == kEmpty32) {
    const uint64_t s = __ldg(reinterpret_cast<const unsigned long long*>(h.slots) + h.cap);
    pay = static_cast<int32_t>(s);
    return static_cast<uint32_t>(s >> 32) != kEmpty32;
  }
  const uint64_t mask = static_cast<uint64_t>(h.cap) - 1;
  if (h.kind == PV_HT_CUCKOO) {
    for (int f = 0; f < h.k; ++f) {
      const uint64_t idx = ht_index(k32, h.hash, h.seed[f], h.log2cap);
      const uint64_t s = __ldg(reinterpret_cast<const unsigned long long*>(h.slots) + idx);
      if (static_cast<uint32_t>(s >> 32) == k32) { pay = static_cast<int32_t>(s); return true; }
    }
    return false;
  }
  uint64_t idx = ht_index(k32, h.hash, h.seed[0], h.log2cap);
  for (int64_t step = 0; step < h.cap; ++step) {
    const uint64_t s = __ldg(reinterpret_cast<const unsigned long long*>(h.slots) + idx);
    const uint32_t hk = static_cast<uint32_t>(s >> 32);
    if (hk == k32) { pay = static_cast<int32_t>(s); return true; }
    if (hk == kEmpty32) return false;
    idx = (idx + 1) & mask;
  }
  return false;
}

// HASH_PROBE of the 4 rows of an item; returns the mask with the misses
// cleared and binds the payload of each hit in mask (0 otherwise).  Perfect tables
// (the kind is the same for every lane) probe all 4 rows without branches:
// 4 independent read-only loads, a dead row of a live item costing one cache
// hit.  Hashed tables probe the live rows (every row when all_rows) one at a
// time, as their probe sequences differ.
template <class T>
__device__ __forceinline__ uint32_t probe_item(const DevHT& h, const T (&fk)[4], uint32_t mask, int32_t (&pay)[4],
                                               bool all_rows) {
  if (h.kind == PV_HT_PERFECT) {
    uint32_t hit = 0;
    if constexpr (sizeof(T) <= 4) {
      // Domain inside int32: (fk - kmin) mod 2^32 < cap exactly when kmin <= fk < kmin + cap
      // (a wrapped difference would need fk < INT32_MIN or kmin + cap > 2^31).
      if (h.narrow) {
        const uint32_t k0 = static_cast<uint32_t>(h.kmin), cap = static_cast<uint32_t>(h.cap);
        if (h.codes != nullptr) {  // one byte per key: 4 independent loads, no slot reads
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const uint32_t i = static_cast<uint32_t>(static_cast<int32_t>(fk[r])) - k0;
            const uint32_t b = i < cap ? static_cast<uint32_t>(__ldg(h.codes + i)) : 0u;
            hit |= static_cast<uint32_t>(b != 0u) << r;
            pay[r] = b != 0u ? static_cast<int32_t>(b) + h.code_base : 0;
          }
          return mask & hit;
        }
        if (h.bits != nullptr) {
          uint32_t ic[4];
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const uint32_t i = static_cast<uint32_t>(static_cast<int32_t>(fk[r])) - k0;
            const bool in = i < cap;
            ic[r] = in ? i : 0u;
            const uint32_t w = __ldg(h.bits + (ic[r] >> 5));
            hit |= static_cast<uint32_t>(in & ((w >> (ic[r] & 31u)) & 1u)) << r;
            pay[r] = 0;
          }
          if (h.payload) {  // payload slots of the surviving hits only
            const uint32_t need = mask & hit;
#pragma unroll
            for (int r = 0; r < 4; ++r)
              if ((need >> r) & 1u)
                pay[r] = static_cast<int32_t>(__ldg(reinterpret_cast<const unsigned long long*>(h.slots) + ic[r]) >> 32);
          }
        } else {
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const uint32_t i = static_cast<uint32_t>(static_cast<int32_t>(fk[r])) - k0;
            const bool in = i < cap;
            const uint64_t sv = __ldg(reinterpret_cast<const unsigned long long*>(h.slots) + (in ? i : 0u));
            const bool ok = in && sv != 0;
            hit |= static_cast<uint32_t>(ok) << r;
            pay[r] = ok ? static_cast<int32_t>(sv >> 32) : 0;
          }
        }
        return mask & hit;
      }
    }
    if (h.codes != nullptr) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const uint64_t i = static_cast<uint64_t>(static_cast<int64_t>(fk[r]) - h.kmin);
        const uint32_t b = i < static_cast<uint64_t>(h.cap) ? static_cast<uint32_t>(__ldg(h.codes + i)) : 0u;
        hit |= static_cast<uint32_t>(b != 0u) << r;
        pay[r] = b != 0u ? static_cast<int32_t>(b) + h.code_base : 0;
      }
      return mask & hit;
    }
    if (h.bits != nullptr) {
      uint64_t ic[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const uint64_t i = static_cast<uint64_t>(static_cast<int64_t>(fk[r]) - h.kmin);
        const bool in = i < static_cast<uint64_t>(h.cap);
        ic[r] = in ? i : 0;
        const uint32_t w = __ldg(h.bits + (ic[r] >> 5));
        hit |= static_cast<uint32_t>(in && ((w >> (ic[r] & 31)) & 1u)) << r;
        pay[r] = 0;
      }
      if (h.payload) {
        const uint32_t need = mask & hit;
#pragma unroll
        for (int r = 0; r < 4; ++r)
          if ((need >> r) & 1u)
            pay[r] = static_cast<int32_t>(__ldg(reinterpret_cast<const unsigned long long*>(h.slots) + ic[r]) >> 32);
      }
    } else {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const uint64_t i = static_cast<uint64_t>(static_cast<int64_t>(fk[r]) - h.kmin);
        const bool in = i < static_cast<uint64_t>(h.cap);
        const uint64_t sv = __ldg(reinterpret_cast<const unsigned long long*>(h.slots) + (in ? i : 0));
        const bool ok = in && sv != 0;
        hit |= static_cast<uint32_t>(ok) << r;
        pay[r] = ok ? static_cast<int32_t>(sv >> 32) : 0;
      }
    }
    return mask & hit;
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    pay[r] = 0;
    if (all_rows || ((mask >> r) & 1u)) {
      int32_t p = 0;
      if (probe_key(h, static_cast<int64_t>(fk[r]), p)) pay[r] = p;
      else mask &= ~(1u << r);
    }
  }
  return mask;
}

// LOOP body up to the sink: FILTER, then HASH_PROBE in order, then loads of
// the columns the sink needs.  Branched mode (PRED = false) evaluates one
// operation at a time and skips the loads and probes of an item whose rows
// are all dead, as an if-statement per operation would; predicated mode
// (PRED = true) loads every column and probes every row, carrying the
// surviving-row flags (Section 6: software predication).
template <class SH, bool PRED>
__device__ __forceinline__ void eval_item(Item<SH>& it, const KParams& kp, int64_t item) {
  const int64_t rows_left = kp.n_rows - item * 4;
  it.nvalid = rows_left >= 4 ? 4 : static_cast<int>(rows_left);
  it.mask = (1u << it.nvalid) - 1u;
  using W = typename SH::Where;
  if constexpr (PRED) {
    load_slots<SH, W::slots | SH::Probes::slots | SH::rest_slots>(it, kp, item);
    static_for<W::N>([&](auto j) { it.mask &= pred_bits<SH, decltype(j)::value>(it, kp); });
  } else {
    uint32_t loaded = 0;
    static_for<W::N>([&](auto j) {
      constexpr int J = decltype(j)::value;
      constexpr int S = At<J, typename W::L>::type::slot;
      if (it.mask) {
        if (!((loaded >> S) & 1u)) load_slots<SH, (1u << S)>(it, kp, item);
        loaded |= 1u << S;
        it.mask &= pred_bits<SH, J>(it, kp);
      }
    });
  }
  using JP = typename SH::Probes;
  static_for<JP::N>([&](auto j) {
    constexpr int J = decltype(j)::value;
    constexpr int S = JP::slot_of[J];
    if (PRED || it.mask) {
      if constexpr (!PRED && !((W::slots >> S) & 1u)) load_slots<SH, (1u << S)>(it, kp, item);
      it.mask = probe_item(kp.probe[J], VGet<S>::get(it.v), it.mask, it.pay[J], PRED);
    }
  });
  if constexpr (!PRED) {
    if (it.mask) load_slots<SH, SH::rest_slots>(it, kp, item);
  }
}

// Value of an ARITHMETIC term for row r (wrapping two's-complement int64).
template <class T> struct TermEval;
template <int S> struct TermEval<X<S>> {
  template <class SH> __device__ __forceinline__ static int64_t get(Item<SH>& it, const KParams&, int r) {
    return static_cast<int64_t>(VGet<S>::get(it.v)[r]);
  }
};
template <int S, int CI> struct TermEval<XPC<S, CI>> {
  template <class SH> __device__ __forceinline__ static int64_t get(Item<SH>& it, const KParams& kp, int r) {
    return static_cast<int64_t>(static_cast<uint64_t>(static_cast<int64_t>(VGet<S>::get(it.v)[r])) +
                                static_cast<uint64_t>(kp.c[CI]));
  }
};
template <int S, int CI> struct TermEval<CMX<S, CI>> {
  template <class SH> __device__ __forceinline__ static int64_t get(Item<SH>& it, const KParams& kp, int r) {
    return static_cast<int64_t>(static_cast<uint64_t>(kp.c[CI]) -
                                static_cast<uint64_t>(static_cast<int64_t>(VGet<S>::get(it.v)[r])));
  }
};
template <int J, int I> struct TermEval<PL<J, I>> {
  template <class SH> __device__ __forceinline__ static int64_t get(Item<SH>& it, const KParams&, int r) {
    return static_cast<int64_t>(it.pay[J][r]);
  }
};

template <class E> struct ExprEval;
template <class... Ts> struct ExprEval<Mul<Ts...>> {
  template <class SH> __device__ __forceinline__ static int64_t get(Item<SH>& it, const KParams& kp, int r) {
    uint64_t v = 1;
    ((v *= static_cast<uint64_t>(TermEval<Ts>::get(it, kp, r))), ...);
    return static_cast<int64_t>(v);
  }
};

// Value of aggregate A for row r (COUNT contributes 1).
template <class A, class SH>
__device__ __forceinline__ int64_t agg_value(Item<SH>& it, const KParams& kp, int r) {
  if constexpr (A::func == PV_COUNT) return 1;
  else return ExprEval<typename A::Expr>::get(it, kp, r);
}

// Whether a key part is a 32-bit source (packable into half a 64-bit key).
template <class SH, class K> struct KeyPart32 : std::true_type {};
template <class SH, int S> struct KeyPart32<SH, X<S>>
    : std::integral_constant<bool, At<S, typename SH::Cols::L>::type::code != PV_I64> {};

// Group key of row r packed into 64 bits: one part -> the part (32-bit
// sources zero-extended from their 32-bit pattern), two 32-bit parts ->
// high and low halves.
template <class SH>
__device__ __forceinline__ uint64_t pack_key(Item<SH>& it, const KParams& kp, int r) {
  using K = typename SH::Key;
  static_assert(K::N <= 2, "keys of three parts are mixed-radix codes over the part domains");
  if constexpr (K::N == 1) {
    using K0 = typename At<0, typename K::L>::type;
    const int64_t v = TermEval<K0>::get(it, kp, r);
    if constexpr (KeyPart32<SH, K0>::value) return static_cast<uint32_t>(v);
    else return static_cast<uint64_t>(v);
  } else {
    using K0 = typename At<0, typename K::L>::type;
    using K1 = typename At<1, typename K::L>::type;
    const uint32_t a = static_cast<uint32_t>(TermEval<K0>::get(it, kp, r));
    const uint32_t b = static_cast<uint32_t>(TermEval<K1>::get(it, kp, r));
    return (static_cast<uint64_t>(a) << 32) | b;
  }
}

// Key parts as int64 (perfect-array indexing).
template <class SH, int P>
__device__ __forceinline__ int64_t key_part(Item<SH>& it, const KParams& kp, int r) {
  using KP = typename At<P, typename SH::Key::L>::type;
  return TermEval<KP>::get(it, kp, r);
}

// ---------------------------------------------------------------------------
// Item iteration (LOOP, Section 6 memory access pattern).  Grid-stride:
// thread t of T handles items t, t + T, ... (neighbouring threads touch
// neighbouring addresses: coalesced).  Chunked: thread t handles the
// contiguous items [t * ceil(n/T), (t + 1) * ceil(n/T)) (sequential access).
// U items are loaded before any is consumed (loop unrolling).
// ---------------------------------------------------------------------------
template <bool CHUNK, int U, class F>
__device__ __forceinline__ void for_items(int64_t n_items, F&& f) {
  const int64_t T = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if constexpr (!CHUNK) {
    for (int64_t base = t; base < n_items; base += U * T) {
      int64_t idx[U];
#pragma unroll
      for (int u = 0; u < U; ++u) idx[u] = base + u * T;
      f(idx);
    }
  } else {
    const int64_t chunk = (n_items + T - 1) / T;
    const int64_t begin = t * chunk;
    const int64_t end = begin + chunk < n_items ? begin + chunk : n_items;
    for (int64_t base = begin; base < end; base += U) {
      int64_t idx[U];
#pragma unroll
      for (int u = 0; u < U; ++u) idx[u] = base + u < end ? base + u : n_items;
      f(idx);
    }
  }
}

// ---------------------------------------------------------------------------
// Warp / block reductions of 64-bit accumulators.
// ---------------------------------------------------------------------------
// MIN and MAX are kept in an order-preserving unsigned code so that every
// accumulator starts at 0 and merges with an unsigned max:
//   MAX: code(v) = v ^ 2^63 ;  MIN: code(v) = ~(v ^ 2^63)
__device__ __forceinline__ uint64_t max_code(int64_t v) { return static_cast<uint64_t>(v) ^ (1ull << 63); }
__device__ __forceinline__ uint64_t min_code(int64_t v) { return ~(static_cast<uint64_t>(v) ^ (1ull << 63)); }
__host__ __device__ __forceinline__ int64_t decode_max(uint64_t c) { return static_cast<int64_t>(c ^ (1ull << 63)); }
__host__ __device__ __forceinline__ int64_t decode_min(uint64_t c) { return static_cast<int64_t>(~c ^ (1ull << 63)); }

// Accumulator update: SUM/COUNT add, MIN/MAX take the max of codes.
template <int FUNC>
__device__ __forceinline__ uint64_t acc_combine(uint64_t a, uint64_t b) {
  if constexpr (FUNC == PV_SUM || FUNC == PV_COUNT) return a + b;
  else return a > b ? a : b;
}
template <int FUNC>
__device__ __forceinline__ uint64_t acc_code(int64_t v) {
  if constexpr (FUNC == PV_MIN) return min_code(v);
  else if constexpr (FUNC == PV_MAX) return max_code(v);
  else return static_cast<uint64_t>(v);
}
template <int FUNC>
__device__ __forceinline__ void acc_atomic(unsigned long long* p, uint64_t v) {
  if constexpr (FUNC == PV_SUM || FUNC == PV_COUNT) atomicAdd(p, static_cast<unsigned long long>(v));
  else atomicMax(p, static_cast<unsigned long long>(v));
}

template <int FUNC>
__device__ __forceinline__ uint64_t warp_reduce(uint64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    v = acc_combine<FUNC>(v, __shfl_xor_sync(0xffffffffu, static_cast<unsigned long long>(v), o));
  return v;
}

}  // namespace pv
