// CPU oracle for the query-pipeline hot path.  TEST INFRASTRUCTURE ONLY:
// it is the plain, slow, obviously correct definition that the CUDA kernels
// are checked against.  Only the tests, the smoke check and the benchmark's
// CPU-baseline leg may load it; the product path never calls it.
//
// What it computes (Breß et al., "Generating Custom Code for Efficient Query
// Execution on Heterogeneous Processors"):
//   * a pipeline program is an ordered list of pipeline operations
//     (Table 1: LOOP, FILTER, HASH_PUT, HASH_PROBE, ARITHMETIC, AGGREGATE,
//     HASH_AGGREGATE, PROJECT); every code variant of it computes the same
//     relation (Section 3.3-3.5), so the oracle is the definition itself,
//     interpreted one tuple at a time (Section 2.1, produce/consume: each
//     tuple is pushed through all operations before the next one);
//   * build pipelines run first and fill one hash table each; the probe
//     pipeline then probes them in order (Table 2);
//   * a probe miss drops the tuple (inner equi-join on a unique build key);
//   * AGGREGATE / HASH_AGGREGATE use distributive aggregates only
//     (SUM, COUNT, MIN, MAX; Section 7.6);
//   * PROJECT materialises the surviving tuples in input order.
//
// Readings where the paper is silent (kept identical on the CUDA side by
// definition, not by shared code): build keys must be unique (a duplicate is
// an error); arithmetic is two's-complement int64 that wraps mod 2^64 and the
// oracle raises a flag when any operation overflowed; an empty group is
// absent from a grouped result; an ungrouped SUM/COUNT over no tuples is 0.
//
// Plan encoding (int64 words, produced by oracle.py):
//   builds:  n_builds, then per build
//              key_col, n_filters, (col, op, c0, c1) * n_filters,
//              n_payload, payload_col * n_payload
//   fact:    n_filters, (col, op, c0, c1) * n,
//            n_probes,  (build, fk_col) * n,
//            n_keys,    (ref_kind, a, b) * n,
//            n_aggs,    (func, n_terms, (term_kind, ref_kind, a, b, c) * n_terms) * n,
//            n_proj,    (ref_kind, a, b) * n
//   ref_kind 0 = fact column a; 1 = payload b of probe a.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <memory>
#include <stdexcept>
#include <thread>
#include <unordered_map>
#include <vector>

namespace {

enum ColType { T_I32 = 0, T_I64 = 1, T_U8 = 2 };
enum CmpOp { OP_LT = 0, OP_LE = 1, OP_GT = 2, OP_GE = 3, OP_EQ = 4, OP_BETWEEN = 5 };
enum AggFunc { F_SUM = 0, F_COUNT = 1, F_MIN = 2, F_MAX = 3 };
enum TermKind { TK_X = 0, TK_X_PLUS_C = 1, TK_C_MINUS_X = 2 };
enum RefKind { R_COL = 0, R_PAYLOAD = 1 };

enum {
  OK = 0,
  ERR_PLAN = -1,
  ERR_COLUMN = -2,
  ERR_DUP_BUILD_KEY = -6,
};

struct Column {
  const void* ptr;
  int type;
  int64_t len;
  int64_t at(int64_t r) const {
    switch (type) {
      case T_I32: return static_cast<const int32_t*>(ptr)[r];
      case T_I64: return static_cast<const int64_t*>(ptr)[r];
      case T_U8: return static_cast<const uint8_t*>(ptr)[r];
    }
    throw std::runtime_error("bad column type");
  }
};

struct Pred { int col, op; int64_t c0, c1; };
struct Ref { int kind, a, b; };
struct Term { int kind; Ref x; int64_t c; };
struct Agg { int func; std::vector<Term> terms; };
struct Build { int key_col; std::vector<Pred> filters; std::vector<int> payload; };
struct Probe { int build, fk_col; };

struct Plan {
  std::vector<Build> builds;
  std::vector<Pred> filters;
  std::vector<Probe> probes;
  std::vector<Ref> keys;
  std::vector<Agg> aggs;
  std::vector<Ref> proj;
};

struct Reader {
  const int64_t* w; int64_t n; int64_t i = 0;
  int64_t next() {
    if (i >= n) throw std::runtime_error("plan truncated");
    return w[i++];
  }
};

Pred read_pred(Reader& rd) {
  Pred p; p.col = (int)rd.next(); p.op = (int)rd.next(); p.c0 = rd.next(); p.c1 = rd.next();
  return p;
}
Ref read_ref(Reader& rd) {
  Ref r; r.kind = (int)rd.next(); r.a = (int)rd.next(); r.b = (int)rd.next();
  return r;
}

Plan parse(const int64_t* words, int64_t n) {
  Reader rd{words, n};
  Plan p;
  int64_t nb = rd.next();
  for (int64_t i = 0; i < nb; ++i) {
    Build b; b.key_col = (int)rd.next();
    int64_t nf = rd.next();
    for (int64_t j = 0; j < nf; ++j) b.filters.push_back(read_pred(rd));
    int64_t np = rd.next();
    for (int64_t j = 0; j < np; ++j) b.payload.push_back((int)rd.next());
    p.builds.push_back(b);
  }
  int64_t nf = rd.next();
  for (int64_t j = 0; j < nf; ++j) p.filters.push_back(read_pred(rd));
  int64_t npr = rd.next();
  for (int64_t j = 0; j < npr; ++j) { Probe q; q.build = (int)rd.next(); q.fk_col = (int)rd.next(); p.probes.push_back(q); }
  int64_t nk = rd.next();
  for (int64_t j = 0; j < nk; ++j) p.keys.push_back(read_ref(rd));
  int64_t na = rd.next();
  for (int64_t j = 0; j < na; ++j) {
    Agg a; a.func = (int)rd.next();
    int64_t nt = rd.next();
    for (int64_t t = 0; t < nt; ++t) {
      Term tm; tm.kind = (int)rd.next(); tm.x = read_ref(rd); tm.c = rd.next();
      a.terms.push_back(tm);
    }
    p.aggs.push_back(a);
  }
  int64_t nproj = rd.next();
  for (int64_t j = 0; j < nproj; ++j) p.proj.push_back(read_ref(rd));
  if (rd.i != n) throw std::runtime_error("trailing plan words");
  return p;
}

// FILTER semantics: the comparison written in the plan, on the value widened to int64.
bool eval_pred(const Pred& p, int64_t x) {
  switch (p.op) {
    case OP_LT: return x < p.c0;
    case OP_LE: return x <= p.c0;
    case OP_GT: return x > p.c0;
    case OP_GE: return x >= p.c0;
    case OP_EQ: return x == p.c0;
    case OP_BETWEEN: return p.c0 <= x && x <= p.c1;
  }
  throw std::runtime_error("bad predicate op");
}

// Wrapping int64 arithmetic with an overflow flag.
struct Arith {
  bool overflow = false;
  int64_t add(int64_t a, int64_t b) {
    int64_t r;
    if (__builtin_add_overflow(a, b, &r)) overflow = true;
    return (int64_t)((uint64_t)a + (uint64_t)b);
  }
  int64_t sub(int64_t a, int64_t b) {
    int64_t r;
    if (__builtin_sub_overflow(a, b, &r)) overflow = true;
    return (int64_t)((uint64_t)a - (uint64_t)b);
  }
  int64_t mul(int64_t a, int64_t b) {
    int64_t r;
    if (__builtin_mul_overflow(a, b, &r)) overflow = true;
    return (int64_t)((uint64_t)a * (uint64_t)b);
  }
};

using HashTable = std::unordered_map<int64_t, std::vector<int64_t>>;

struct AggState {
  std::vector<int64_t> v;
  std::vector<bool> seen;
  explicit AggState(size_t n = 0) : v(n, 0), seen(n, false) {}
};

struct Partial {
  AggState ungrouped;
  std::map<std::vector<int64_t>, AggState> groups;
  std::vector<std::vector<int64_t>> rows;  // projection, input order
  bool overflow = false;
};

void fold(const Plan& plan, AggState& st, const std::vector<int64_t>& vals, Arith& ar) {
  for (size_t i = 0; i < plan.aggs.size(); ++i) {
    int f = plan.aggs[i].func;
    if (f == F_SUM || f == F_COUNT) {
      st.v[i] = ar.add(st.v[i], vals[i]);
    } else if (!st.seen[i]) {
      st.v[i] = vals[i];
    } else if (f == F_MIN) {
      st.v[i] = std::min(st.v[i], vals[i]);
    } else {
      st.v[i] = std::max(st.v[i], vals[i]);
    }
    st.seen[i] = true;
  }
}

void merge_into(const Plan& plan, AggState& dst, const AggState& src, Arith& ar) {
  for (size_t i = 0; i < plan.aggs.size(); ++i) {
    if (!src.seen[i]) continue;
    int f = plan.aggs[i].func;
    if (f == F_SUM || f == F_COUNT) dst.v[i] = ar.add(dst.v[i], src.v[i]);
    else if (!dst.seen[i]) dst.v[i] = src.v[i];
    else if (f == F_MIN) dst.v[i] = std::min(dst.v[i], src.v[i]);
    else dst.v[i] = std::max(dst.v[i], src.v[i]);
    dst.seen[i] = true;
  }
}

// The probe pipeline over fact rows [lo, hi): LOOP -> FILTER -> HASH_PROBE*
// -> ARITHMETIC -> (HASH_)AGGREGATE or PROJECT, one tuple at a time.
void run_rows(const Plan& plan, const std::vector<Column>& cols, const std::vector<HashTable>& tables,
              int64_t lo, int64_t hi, Partial& out) {
  Arith ar;
  out.ungrouped = AggState(plan.aggs.size());
  std::vector<const std::vector<int64_t>*> bound(plan.probes.size(), nullptr);
  std::vector<int64_t> key(plan.keys.size()), vals(plan.aggs.size());
  auto ref = [&](const Ref& r, int64_t row) -> int64_t {
    if (r.kind == R_COL) return cols[r.a].at(row);
    return (*bound[r.a])[r.b];
  };
  for (int64_t row = lo; row < hi; ++row) {
    bool pass = true;
    for (const Pred& p : plan.filters) {
      if (!eval_pred(p, cols[p.col].at(row))) { pass = false; break; }
    }
    if (!pass) continue;
    for (size_t j = 0; j < plan.probes.size() && pass; ++j) {
      const HashTable& ht = tables[plan.probes[j].build];
      auto it = ht.find(cols[plan.probes[j].fk_col].at(row));
      if (it == ht.end()) pass = false;
      else bound[j] = &it->second;
    }
    if (!pass) continue;
    if (!plan.proj.empty()) {
      std::vector<int64_t> t;
      for (const Ref& r : plan.proj) t.push_back(ref(r, row));
      out.rows.push_back(std::move(t));
      continue;
    }
    for (size_t i = 0; i < plan.aggs.size(); ++i) {
      const Agg& a = plan.aggs[i];
      if (a.func == F_COUNT) { vals[i] = 1; continue; }
      int64_t v = 1;
      for (const Term& t : a.terms) {
        int64_t x = ref(t.x, row);
        int64_t tv = t.kind == TK_X ? x : t.kind == TK_X_PLUS_C ? ar.add(x, t.c) : ar.sub(t.c, x);
        v = ar.mul(v, tv);
      }
      vals[i] = v;
    }
    if (plan.keys.empty()) {
      fold(plan, out.ungrouped, vals, ar);
    } else {
      for (size_t k = 0; k < plan.keys.size(); ++k) key[k] = ref(plan.keys[k], row);
      auto it = out.groups.find(key);
      if (it == out.groups.end()) it = out.groups.emplace(key, AggState(plan.aggs.size())).first;
      fold(plan, it->second, vals, ar);
    }
  }
  out.overflow = ar.overflow;
}

struct Result {
  int kind = 0;  // 0 ungrouped, 1 grouped, 2 projection
  int64_t nrows = 0;
  std::vector<std::vector<int64_t>> cols;
  int flags = 0;  // bit 0: an int64 operation overflowed
};

int run(const int64_t* words, int64_t nwords, const void* const* ptrs, const int32_t* types,
        const int64_t* lens, int32_t ncols, int64_t fact_rows, int32_t nthreads, Result& res) {
  Plan plan = parse(words, nwords);
  std::vector<Column> cols;
  for (int i = 0; i < ncols; ++i) {
    if (types[i] < 0 || types[i] > 2) return ERR_COLUMN;
    cols.push_back(Column{ptrs[i], types[i], lens[i]});
  }
  auto check_col = [&](int c) { if (c < 0 || c >= ncols) throw std::runtime_error("bad column index"); };
  // Build pipelines (Table 2): LOOP -> FILTER -> HASH_PUT of the key with its payload.
  std::vector<HashTable> tables;
  for (const Build& b : plan.builds) {
    check_col(b.key_col);
    HashTable ht;
    for (int64_t r = 0; r < cols[b.key_col].len; ++r) {
      bool pass = true;
      for (const Pred& p : b.filters) {
        check_col(p.col);
        if (!eval_pred(p, cols[p.col].at(r))) { pass = false; break; }
      }
      if (!pass) continue;
      int64_t k = cols[b.key_col].at(r);
      if (ht.count(k)) return ERR_DUP_BUILD_KEY;
      std::vector<int64_t> pay;
      for (int c : b.payload) { check_col(c); pay.push_back(cols[c].at(r)); }
      ht.emplace(k, std::move(pay));
    }
    tables.push_back(std::move(ht));
  }
  // Validate fact references.
  for (const Pred& p : plan.filters) { check_col(p.col); if (cols[p.col].len < fact_rows) return ERR_COLUMN; }
  for (const Probe& q : plan.probes) {
    check_col(q.fk_col);
    if (q.build < 0 || q.build >= (int)tables.size()) return ERR_PLAN;
    if (cols[q.fk_col].len < fact_rows) return ERR_COLUMN;
  }
  auto check_ref = [&](const Ref& r) {
    if (r.kind == R_COL) { check_col(r.a); if (cols[r.a].len < fact_rows) throw std::runtime_error("short column"); }
    else if (r.a < 0 || r.a >= (int)plan.probes.size() ||
             r.b < 0 || r.b >= (int)plan.builds[plan.probes[r.a].build].payload.size())
      throw std::runtime_error("bad payload ref");
  };
  for (const Ref& r : plan.keys) check_ref(r);
  for (const Agg& a : plan.aggs) for (const Term& t : a.terms) check_ref(t.x);
  for (const Ref& r : plan.proj) check_ref(r);
  if (!plan.proj.empty() && !plan.aggs.empty()) return ERR_PLAN;
  if (plan.proj.empty() && plan.aggs.empty()) return ERR_PLAN;

  // Row-partitioned evaluation (one contiguous chunk per thread), merged in chunk order.
  int T = std::max(1, nthreads);
  if (fact_rows < (int64_t)T * 1024) T = 1;
  std::vector<Partial> parts(T);
  std::vector<std::thread> th;
  for (int t = 0; t < T; ++t) {
    int64_t lo = fact_rows * t / T, hi = fact_rows * (t + 1) / T;
    if (T == 1) run_rows(plan, cols, tables, lo, hi, parts[0]);
    else th.emplace_back([&, t, lo, hi] { run_rows(plan, cols, tables, lo, hi, parts[t]); });
  }
  for (auto& x : th) x.join();

  Arith ar;
  bool overflow = false;
  for (auto& p : parts) overflow |= p.overflow;
  if (!plan.proj.empty()) {
    res.kind = 2;
    res.cols.assign(plan.proj.size(), {});
    for (auto& p : parts)
      for (auto& row : p.rows)
        for (size_t c = 0; c < row.size(); ++c) res.cols[c].push_back(row[c]);
    res.nrows = res.cols.empty() ? 0 : (int64_t)res.cols[0].size();
  } else if (plan.keys.empty()) {
    res.kind = 0;
    AggState all(plan.aggs.size());
    for (auto& p : parts) merge_into(plan, all, p.ungrouped, ar);
    res.cols.assign(plan.aggs.size(), {});
    for (size_t i = 0; i < plan.aggs.size(); ++i) res.cols[i].push_back(all.v[i]);
    res.nrows = 1;
  } else {
    res.kind = 1;
    std::map<std::vector<int64_t>, AggState> all;
    for (auto& p : parts)
      for (auto& kv : p.groups) {
        auto it = all.find(kv.first);
        if (it == all.end()) all.emplace(kv.first, kv.second);
        else merge_into(plan, it->second, kv.second, ar);
      }
    size_t nk = plan.keys.size();
    res.cols.assign(nk + plan.aggs.size(), {});
    for (auto& kv : all) {  // std::map iterates in ascending key order
      for (size_t k = 0; k < nk; ++k) res.cols[k].push_back(kv.first[k]);
      for (size_t i = 0; i < plan.aggs.size(); ++i) res.cols[nk + i].push_back(kv.second.v[i]);
    }
    res.nrows = (int64_t)all.size();
  }
  res.flags = (overflow || ar.overflow) ? 1 : 0;
  return OK;
}

thread_local std::string g_error;

}  // namespace

extern "C" {

int or_run(const int64_t* words, int64_t nwords, const void* const* ptrs, const int32_t* types,
           const int64_t* lens, int32_t ncols, int64_t fact_rows, int32_t nthreads, void** out) {
  *out = nullptr;
  auto res = std::make_unique<Result>();
  try {
    int rc = run(words, nwords, ptrs, types, lens, ncols, fact_rows, nthreads, *res);
    if (rc != OK) return rc;
  } catch (const std::exception& e) {
    g_error = e.what();
    return ERR_PLAN;
  }
  *out = res.release();
  return OK;
}

int64_t or_result_rows(const void* r) { return static_cast<const Result*>(r)->nrows; }
int32_t or_result_cols(const void* r) { return (int32_t) static_cast<const Result*>(r)->cols.size(); }
int32_t or_result_kind(const void* r) { return static_cast<const Result*>(r)->kind; }
int32_t or_result_flags(const void* r) { return static_cast<const Result*>(r)->flags; }
void or_result_copy_col(const void* r, int32_t c, int64_t* dst) {
  const auto& v = static_cast<const Result*>(r)->cols.at(c);
  if (!v.empty()) std::memcpy(dst, v.data(), v.size() * sizeof(int64_t));
}
void or_result_free(void* r) { delete static_cast<Result*>(r); }
const char* or_last_error(void) { return g_error.c_str(); }
int32_t or_hardware_threads(void) { return (int32_t)std::thread::hardware_concurrency(); }

}  // extern "C"
