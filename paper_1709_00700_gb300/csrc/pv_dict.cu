// Dictionary-coded string columns: host translation of string predicates
// into predicates on the codes (plan compilation; no device work).
//
// A string column is stored as int32 codes into a dictionary of distinct
// strings sorted in byte order, the code of a string being its rank.  Codes
// then order like the strings, so a comparison with a constant (present in
// the dictionary or not) and a prefix match each select one contiguous code
// range: the FILTER of Table 1 on the code column.  A LIKE pattern with
// inner wildcards selects an arbitrary set of codes, which pv_dict_match
// lists for a semi-join probe.  (Section 9.2.1: the missing LIKE operator is
// why the paper's prototype left some SSB and TPC-H queries out.)
#include <cstring>

#include "pv.h"

namespace {

// First code whose string is >= s (strict = false) or > s (strict = true).
int64_t bound(const char* const* d, int64_t n, const char* s, bool strict) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = lo + (hi - lo) / 2;
    const int c = std::strcmp(d[mid], s);
    if (c < 0 || (strict && c == 0)) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// First code whose first m bytes compare >= p (strict = false) or > p
// (strict = true) under strncmp: monotone over a sorted dictionary.
int64_t prefix_bound(const char* const* d, int64_t n, const char* p, size_t m, bool strict) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = lo + (hi - lo) / 2;
    const int c = std::strncmp(d[mid], p, m);
    if (c < 0 || (strict && c == 0)) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// SQL LIKE without an escape character: '%' matches any run of bytes
// (possibly empty), '_' exactly one byte, every other byte itself.  Greedy
// scan that, on a mismatch, lets the most recent '%' absorb one more byte.
bool like(const char* s, const char* p) {
  const char* star = nullptr;  // pattern position just after the last '%'
  const char* mark = nullptr;  // string position that '%' is absorbing up to
  while (*s) {
    if (*p == '%') {
      star = ++p;
      mark = s;
    } else if (*p != '\0' && (*p == '_' || *p == *s)) {
      ++p;
      ++s;
    } else if (star) {
      p = star;
      s = ++mark;
    } else {
      return false;
    }
  }
  while (*p == '%') ++p;
  return *p == '\0';
}

pv_status check_dict(const char* const* d, int64_t n) {
  if (n < 0 || n > INT32_MAX || (n > 0 && d == nullptr)) return PV_ERR_INVALID_ARG;
  for (int64_t i = 0; i < n; ++i) {
    if (d[i] == nullptr) return PV_ERR_INVALID_ARG;
    if (i > 0 && std::strcmp(d[i - 1], d[i]) >= 0) return PV_ERR_INVALID_ARG;  // not strictly ascending
  }
  return PV_OK;
}

}  // namespace

extern "C" {

pv_status pv_dict_range(const char* const* dict, int64_t n_entries, int32_t op, const char* s0, const char* s1,
                        int64_t* lo, int64_t* hi) {
  if (!lo || !hi || !s0 || (op == PV_BETWEEN && !s1)) return PV_ERR_INVALID_ARG;
  const pv_status st = check_dict(dict, n_entries);
  if (st != PV_OK) return st;
  const int64_t n = n_entries;
  int64_t a, b;  // half-open code range [a, b)
  switch (op) {
    case PV_LT: a = 0; b = bound(dict, n, s0, false); break;
    case PV_LE: a = 0; b = bound(dict, n, s0, true); break;
    case PV_GT: a = bound(dict, n, s0, true); b = n; break;
    case PV_GE: a = bound(dict, n, s0, false); b = n; break;
    case PV_EQ: a = bound(dict, n, s0, false); b = bound(dict, n, s0, true); break;
    case PV_BETWEEN: a = bound(dict, n, s0, false); b = bound(dict, n, s1, true); break;
    case PV_PREFIX: {
      const size_t m = std::strlen(s0);
      a = prefix_bound(dict, n, s0, m, false);
      b = prefix_bound(dict, n, s0, m, true);
      break;
    }
    default: return PV_ERR_INVALID_ARG;
  }
  if (a >= b) {
    *lo = 1;
    *hi = 0;
  } else {
    *lo = a;
    *hi = b - 1;
  }
  return PV_OK;
}

pv_status pv_dict_match(const char* const* dict, int64_t n_entries, const char* pattern, int32_t* codes,
                        int64_t capacity, int64_t* n_match) {
  if (!pattern || !n_match || capacity < 0 || (capacity > 0 && !codes)) return PV_ERR_INVALID_ARG;
  const pv_status st = check_dict(dict, n_entries);
  if (st != PV_OK) return st;
  int64_t k = 0;
  for (int64_t i = 0; i < n_entries; ++i) {
    if (!like(dict[i], pattern)) continue;
    if (k < capacity) codes[k] = static_cast<int32_t>(i);
    ++k;
  }
  *n_match = k;
  return PV_OK;
}

}  // extern "C"
