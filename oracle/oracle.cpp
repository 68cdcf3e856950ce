// CPU oracle for in-memory aggregation. TEST INFRASTRUCTURE ONLY: the test
// suite, the smoke check and the benchmark's CPU-baseline leg load it; the
// library under test never does.
//
// What it computes is the plain definition of aggregation: every item of a
// column is folded into one accumulator with the aggregation function
// (Fig. 1, Sec. 1 and Sec. 2.1; the fold r = aggregate(r, input[i]) of the
// TornadoVM kernel in Fig. 4). GROUP BY applies the same fold per distinct
// key (the hash- and sort-based group-by of Sec. 7) with one accumulator per
// key held in an ordered std::map, so that groups come out in ascending key
// order.
//
// Readings where the paper is silent (it sums one integer column, Sec. 4):
//  * integer SUM: int64 accumulation, two's-complement wrap mod 2^64; uint32
//    values are zero-extended.
//  * floating-point SUM: the exact real sum of the inputs, rounded once to
//    float64 (round to nearest, ties to even). It is kept exactly in an
//    integer fixed-point accumulator whose least significant bit is the
//    smallest subnormal of the input type.
//  * MIN/MAX of floats: total order with -0.0 < +0.0 (inputs hold no NaN).
//  * AVG = (double)SUM / (double)COUNT; NaN when COUNT = 0.
//  * COUNT = number of items.
//
// Single-threaded on purpose; no blocking, no fusion, no reordering.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <map>
#include <vector>

// Result of one aggregation: integer fields are used for integer columns,
// floating-point fields for float columns; avg for both.
struct oracle_scalar {
  int64_t count;
  int64_t sum_i;
  double sum_f;
  double avg;
  int64_t min_i;
  int64_t max_i;
  double min_f;
  double max_f;
};

namespace {

// ---------------------------------------------------------------------------
// Exact sum of binary floating-point numbers.
//
// The running sum is an integer N (in units of 2^LSB) held as NDIG signed
// base-2^32 digits in int64 words. One add touches at most three digits, each
// by less than 2^32 in magnitude, so the words cannot overflow before 2^31
// adds; carries are propagated every 2^30 adds and before rounding.
// ---------------------------------------------------------------------------
template <int NDIG, int LSB>
struct ExactSum {
  int64_t d[NDIG];
  int64_t pending = 0;
  ExactSum() { std::memset(d, 0, sizeof(d)); }

  void add_parts(bool neg, uint64_t mant, int lsb_exp) {
    if (mant == 0) return;
    int p = lsb_exp - LSB;  // bit position of mant's least significant bit
    int q = p >> 5, r = p & 31;
    unsigned __int128 v = (unsigned __int128)mant << r;
    int64_t c0 = (int64_t)(uint64_t)(v & 0xFFFFFFFFu);
    int64_t c1 = (int64_t)(uint64_t)((v >> 32) & 0xFFFFFFFFu);
    int64_t c2 = (int64_t)(uint64_t)(v >> 64);
    if (neg) { c0 = -c0; c1 = -c1; c2 = -c2; }
    d[q] += c0;
    d[q + 1] += c1;
    d[q + 2] += c2;
    if (++pending == (int64_t(1) << 30)) normalize();
  }

  void add(double x) {
    uint64_t b;
    std::memcpy(&b, &x, 8);
    bool neg = b >> 63;
    int e = (int)((b >> 52) & 0x7FF);
    uint64_t f = b & ((uint64_t(1) << 52) - 1);
    if (e == 0) add_parts(neg, f, -1074);
    else add_parts(neg, f | (uint64_t(1) << 52), e - 1075);
  }

  void add(float x) {
    uint32_t b;
    std::memcpy(&b, &x, 4);
    bool neg = b >> 31;
    int e = (int)((b >> 23) & 0xFF);
    uint64_t f = b & ((1u << 23) - 1);
    if (e == 0) add_parts(neg, f, -149);
    else add_parts(neg, f | (uint64_t(1) << 23), e - 150);
  }

  // After this, d[i] is in [0, 2^32) for i < NDIG-1 and d[NDIG-1] carries the sign.
  static void carry(int64_t* a) {
    for (int i = 0; i < NDIG - 1; ++i) {
      int64_t c = a[i] >> 32;  // floor division by 2^32
      a[i] -= c * (int64_t(1) << 32);
      a[i + 1] += c;
    }
  }
  void normalize() { carry(d); pending = 0; }

  // Round N * 2^LSB to the nearest double, ties to even.
  double value() const {
    int64_t a[NDIG];
    std::memcpy(a, d, sizeof(a));
    carry(a);
    bool neg = a[NDIG - 1] < 0;
    if (neg) {
      for (int i = 0; i < NDIG; ++i) a[i] = -a[i];
      carry(a);
    }
    int top = NDIG - 1;
    while (top >= 0 && a[top] == 0) --top;
    if (top < 0) return 0.0;
    int hb = 63 - __builtin_clzll((uint64_t)a[top]);
    int H = top * 32 + hb;  // index of the highest set bit of |N|
    auto bit = [&](int i) -> uint64_t {
      if (i < 0) return 0;
      return ((uint64_t)a[i >> 5] >> (i & 31)) & 1u;
    };
    // 53 significant bits, then the round bit and a sticky bit.
    uint64_t mant = 0;
    for (int i = H; i > H - 53; --i) mant = (mant << 1) | bit(i);
    uint64_t round = bit(H - 53);
    bool sticky = false;
    for (int i = H - 54; i >= 0 && !sticky; --i) sticky = bit(i) != 0;
    if (round && (sticky || (mant & 1))) {
      ++mant;
      if (mant == (uint64_t(1) << 53)) { mant >>= 1; ++H; }
    }
    double v = std::ldexp((double)mant, H - 52 + LSB);
    return neg ? -v : v;
  }
};

using ExactF32 = ExactSum<11, -149>;   // |sum| < 2^128 * 2^63
using ExactF64 = ExactSum<68, -1074>;  // |sum| < 2^1024 * 2^63

enum { D_I32 = 0, D_I64 = 1, D_U32 = 2, D_F32 = 3, D_F64 = 4 };

// -0.0 < +0.0 total order on NaN-free values.
inline bool fless(double a, double b) {
  if (a < b) return true;
  if (a == b) return std::signbit(a) && !std::signbit(b);
  return false;
}

inline int64_t int_at(const void* col, int dt, int64_t i) {
  switch (dt) {
    case D_I32: return ((const int32_t*)col)[i];
    case D_I64: return ((const int64_t*)col)[i];
    default: return (int64_t)((const uint32_t*)col)[i];
  }
}

// One aggregate state: the fold of Fig. 4 for SUM, MIN, MAX and COUNT.
template <class Acc>
struct State {
  int64_t count = 0;
  uint64_t isum = 0;  // integer SUM, wraps mod 2^64
  Acc fsum;           // exact floating-point SUM
  int64_t imin = std::numeric_limits<int64_t>::max();
  int64_t imax = std::numeric_limits<int64_t>::min();
  double fmin = std::numeric_limits<double>::infinity();
  double fmax = -std::numeric_limits<double>::infinity();

  void fold_int(int64_t v) {
    ++count;
    isum += (uint64_t)v;
    if (v < imin) imin = v;
    if (v > imax) imax = v;
  }
  template <class F>
  void fold_fp(F v) {
    ++count;
    fsum.add(v);
    double x = (double)v;
    if (fless(x, fmin)) fmin = x;
    if (fless(fmax, x)) fmax = x;
  }
};

struct Dummy {
  void add(double) {}
  void add(float) {}
  double value() const { return 0.0; }
};

template <class S>
static void emit(const S& st, int dt, oracle_scalar* o) {
  o->count = st.count;
  o->sum_i = (int64_t)st.isum;
  o->min_i = st.imin;
  o->max_i = st.imax;
  o->min_f = st.fmin;
  o->max_f = st.fmax;
  if (dt == D_F32 || dt == D_F64) {
    o->sum_f = st.fsum.value();
  } else {
    o->sum_f = (double)(int64_t)st.isum;
  }
  o->avg = st.count ? o->sum_f / (double)st.count : std::numeric_limits<double>::quiet_NaN();
}

// ---------------------------------------------------------------------------
// GROUP BY: one State per distinct key in an ordered map (Sec. 7's group-by
// semantics); output rows in ascending key order.
// ---------------------------------------------------------------------------

struct GroupsBase {
  virtual ~GroupsBase() {}
  virtual int64_t size() const = 0;
  virtual void fetch(uint32_t* keys, oracle_scalar* rows) const = 0;
};

template <class Acc>
struct Groups : GroupsBase {
  int dt;
  std::map<uint32_t, State<Acc>> m;
  int64_t size() const override { return (int64_t)m.size(); }
  void fetch(uint32_t* keys, oracle_scalar* rows) const override {
    int64_t j = 0;
    for (const auto& kv : m) {
      if (keys) keys[j] = kv.first;
      if (rows) emit(kv.second, dt, &rows[j]);
      ++j;
    }
  }
};

template <class Acc>
static GroupsBase* build_groups(const uint32_t* keys, const void* vals, int64_t n, int dt,
                                const uint32_t* sel, int64_t m) {
  auto* g = new Groups<Acc>();
  g->dt = dt;
  if (sel) {
    for (int64_t j = 0; j < m; ++j) g->m[sel[j]];  // selected keys only, count may stay 0
  }
  for (int64_t i = 0; i < n; ++i) {
    uint32_t k = keys[i];
    State<Acc>* st;
    if (sel) {
      auto it = g->m.find(k);
      if (it == g->m.end()) continue;
      st = &it->second;
    } else {
      st = &g->m[k];
    }
    if (dt == D_F32) st->fold_fp(((const float*)vals)[i]);
    else if (dt == D_F64) st->fold_fp(((const double*)vals)[i]);
    else st->fold_int(int_at(vals, dt, i));
  }
  return g;
}

static GroupsBase* groups_any(const uint32_t* keys, const void* vals, int64_t n, int dt,
                              const uint32_t* sel, int64_t m) {
  if (dt == D_F32) return build_groups<ExactF32>(keys, vals, n, dt, sel, m);
  if (dt == D_F64) return build_groups<ExactF64>(keys, vals, n, dt, sel, m);
  return build_groups<Dummy>(keys, vals, n, dt, sel, m);
}

}  // namespace

extern "C" {

double oracle_exact_sum_f64(const double* x, int64_t n) {
  ExactF64 s;
  for (int64_t i = 0; i < n; ++i) s.add(x[i]);
  return s.value();
}

double oracle_exact_sum_f32(const float* x, int64_t n) {
  ExactF32 s;
  for (int64_t i = 0; i < n; ++i) s.add(x[i]);
  return s.value();
}

// Ungrouped aggregation of col[0..n) (Sec. 2.1, Fig. 4).
int oracle_reduce(const void* col, int64_t n, int dt, oracle_scalar* out) {
  if (n < 0 || (n > 0 && !col) || !out || dt < 0 || dt > 4) return -1;
  if (dt == D_F32) {
    State<ExactF32> st;
    for (int64_t i = 0; i < n; ++i) st.fold_fp(((const float*)col)[i]);
    emit(st, dt, out);
  } else if (dt == D_F64) {
    State<ExactF64> st;
    for (int64_t i = 0; i < n; ++i) st.fold_fp(((const double*)col)[i]);
    emit(st, dt, out);
  } else {
    State<Dummy> st;
    for (int64_t i = 0; i < n; ++i) st.fold_int(int_at(col, dt, i));
    emit(st, dt, out);
  }
  return 0;
}

// Full GROUP BY. Returns a handle; *d receives the number of distinct keys.
void* oracle_groupby(const uint32_t* keys, const void* vals, int64_t n, int dt, int64_t* d) {
  if (n < 0 || dt < 0 || dt > 4 || (n > 0 && (!keys || !vals))) return nullptr;
  GroupsBase* g = groups_any(keys, vals, n, dt, nullptr, 0);
  if (d) *d = g->size();
  return g;
}

// GROUP BY restricted to the m distinct keys in sel (for sampled checks of
// inputs too large for the full map). Rows are returned in ascending key order.
void* oracle_groupby_selected(const uint32_t* keys, const void* vals, int64_t n, int dt,
                              const uint32_t* sel, int64_t m, int64_t* d) {
  if (n < 0 || dt < 0 || dt > 4 || m < 0 || (n > 0 && (!keys || !vals))) return nullptr;
  GroupsBase* g = groups_any(keys, vals, n, dt, sel, m);
  if (d) *d = g->size();
  return g;
}

// ---------------------------------------------------------------------------
// GROUP BY over a composite key with several value columns and a range filter
// (the operator fusion the paper names as future work, Sec. 8: a selection
// feeding an aggregation). A row takes part iff flo <= f[i] <= fhi in the
// filter column's own type (integers compared as int64, uint32 zero-extended;
// floats as float64, float32 widened exactly); with no filter column every row
// does. Its group is the 64-bit key (key_hi[i] << 32) | key_lo[i] (key_hi[i] = 0
// when there is no second key column). Each value column is folded per group
// exactly as in oracle_groupby; COUNT is the number of rows that took part.
// Groups come out in ascending 64-bit key order; a group exists iff at least
// one of its rows passed the filter.
// ---------------------------------------------------------------------------
struct MultiState {
  State<ExactF32> f32;
  State<ExactF64> f64;
  State<Dummy> i;
};

struct MultiGroups {
  int ncols;
  std::vector<int> dts;
  std::map<uint64_t, std::vector<MultiState>> m;
};

static bool passes(const void* f, int fdt, int64_t i, int64_t lo_i, int64_t hi_i, double lo_f, double hi_f) {
  if (!f) return true;
  if (fdt == D_F32 || fdt == D_F64) {
    const double x = fdt == D_F32 ? (double)((const float*)f)[i] : ((const double*)f)[i];
    return lo_f <= x && x <= hi_f;
  }
  const int64_t x = int_at(f, fdt, i);
  return lo_i <= x && x <= hi_i;
}

void* oracle_groupby_multi(const uint32_t* key_lo, const uint32_t* key_hi, int64_t n, const void* const* cols,
                           const int* dts, int ncols, const void* fcol, int fdt, int64_t flo_i, int64_t fhi_i,
                           double flo_f, double fhi_f, int64_t* d) {
  if (n < 0 || ncols < 1 || (n > 0 && !key_lo)) return nullptr;
  for (int c = 0; c < ncols; ++c)
    if (dts[c] < 0 || dts[c] > 4 || (n > 0 && !cols[c])) return nullptr;
  if (fcol && (fdt < 0 || fdt > 4)) return nullptr;
  auto* g = new MultiGroups();
  g->ncols = ncols;
  g->dts.assign(dts, dts + ncols);
  for (int64_t i = 0; i < n; ++i) {
    if (!passes(fcol, fdt, i, flo_i, fhi_i, flo_f, fhi_f)) continue;
    const uint64_t key = ((uint64_t)(key_hi ? key_hi[i] : 0u) << 32) | key_lo[i];
    std::vector<MultiState>& st = g->m[key];
    if (st.empty()) st.resize(ncols);
    for (int c = 0; c < ncols; ++c) {
      if (dts[c] == D_F32) st[c].f32.fold_fp(((const float*)cols[c])[i]);
      else if (dts[c] == D_F64) st[c].f64.fold_fp(((const double*)cols[c])[i]);
      else st[c].i.fold_int(int_at(cols[c], dts[c], i));
    }
  }
  if (d) *d = (int64_t)g->m.size();
  return g;
}

// keys[d]; rows[d * ncols] (group-major: rows[j * ncols + c]).
void oracle_multi_fetch(void* h, uint64_t* keys, oracle_scalar* rows) {
  const MultiGroups* g = static_cast<const MultiGroups*>(h);
  int64_t j = 0;
  for (const auto& kv : g->m) {
    keys[j] = kv.first;
    for (int c = 0; c < g->ncols; ++c) {
      oracle_scalar* o = &rows[j * g->ncols + c];
      if (g->dts[c] == D_F32) emit(kv.second[c].f32, g->dts[c], o);
      else if (g->dts[c] == D_F64) emit(kv.second[c].f64, g->dts[c], o);
      else emit(kv.second[c].i, g->dts[c], o);
    }
    ++j;
  }
}

void oracle_multi_free(void* h) { delete static_cast<MultiGroups*>(h); }

void oracle_groups_fetch(void* h, uint32_t* keys, oracle_scalar* rows) {
  static_cast<GroupsBase*>(h)->fetch(keys, rows);
}

void oracle_groups_free(void* h) { delete static_cast<GroupsBase*>(h); }

}  // extern "C"
