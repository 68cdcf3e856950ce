// Shared parts of the ungrouped scans (plain, host-fed, allocation-free and
// bit-packed columns): the per-thread accumulators (the fold of Fig. 4), the
// block partials with their error bound, the fixed-order warp and block
// reduction and the merge of block partials into one result.
#pragma once

#include <cfloat>
#include <climits>
#include <cmath>

#include "common.cuh"

namespace agg {

struct Partial {  // one block's partial aggregate
  int64_t si;     // integer sum
  double hi, lo;  // float sum, unevaluated hi + lo
  uint64_t mn, mx;  // order-preserving images of min / max
  double eb;      // bound on |hi + lo - exact sum of the rows| (float columns)
};

template <int DT> struct Traits;
template <> struct Traits<AGG_I32> { using T = int32_t; static constexpr bool FP = false; };
template <> struct Traits<AGG_I64> { using T = int64_t; static constexpr bool FP = false; };
template <> struct Traits<AGG_U32> { using T = uint32_t; static constexpr bool FP = false; };
template <> struct Traits<AGG_F32> { using T = float; static constexpr bool FP = true; };
template <> struct Traits<AGG_F64> { using T = double; static constexpr bool FP = true; };

// ---------------------------------------------------------------------------
// Per-thread accumulators. fold() is the aggregate() of Fig. 4.
// ---------------------------------------------------------------------------
template <int DT, bool SUM, bool MM, bool FP = Traits<DT>::FP>
struct Acc;

template <int DT, bool SUM, bool MM>
struct Acc<DT, SUM, MM, false> {
  using T = typename Traits<DT>::T;
  int64_t s;
  T mn, mx;
  __device__ void init() {
    s = 0;
    if (DT == AGG_I32) { mn = (T)INT_MAX; mx = (T)INT_MIN; }
    if (DT == AGG_U32) { mn = (T)UINT_MAX; mx = (T)0; }
    if (DT == AGG_I64) { mn = (T)LLONG_MAX; mx = (T)LLONG_MIN; }
  }
  __device__ __forceinline__ void fold(T v) {
    if (SUM) s += (int64_t)v;
    if (MM) { mn = min(mn, v); mx = max(mx, v); }
  }
  __device__ __forceinline__ void fold_vec(const uint4& r) {
    if (sizeof(T) == 4) {
      fold((T)r.x); fold((T)r.y); fold((T)r.z); fold((T)r.w);
    } else {
      fold((T)(((uint64_t)r.y << 32) | r.x));
      fold((T)(((uint64_t)r.w << 32) | r.z));
    }
  }
  __device__ void to_partial(Partial& p, uint32_t) const {
    p.si = s;
    p.hi = 0.0;
    p.lo = 0.0;
    p.mn = img_i64((int64_t)mn);
    p.mx = img_i64((int64_t)mx);
    p.eb = 0.0;
  }
};

template <class F> struct FpImg;
template <> struct FpImg<float> {
  using U = uint32_t;
  __device__ static U img(float x) { return img_f32(x); }
  __device__ static uint64_t widen(U m) {  // f32 image -> image of the same value as f64
    if (m == 0xFFFFFFFFu) return ~0ull;    // identity of min
    if (m == 0u) return 0ull;              // identity of max
    return img_f64((double)f32_of_img(m));
  }
};
template <> struct FpImg<double> {
  using U = uint64_t;
  __device__ static U img(double x) { return img_f64(x); }
  __device__ static uint64_t widen(U m) { return m; }
};

// float64 SUM on the integer pipes: a 128-bit two's-complement fixed-point
// number (hi:lo) scaled to the largest exponent field E seen so far, worth
// (hi:lo) x 2^(E - 1075 - kFixGuard). A row with significand m (53 bits,
// implicit bit included) and exponent field e >= 1 is worth m x 2^(e - 1075),
// i.e. m shifted left by kFixGuard - (E - e) units. Rows more than kFixGuard
// binades below E keep their bits above the unit (each loses less than
// 2^(E - 1075 - kFixGuard), 2^-83 of the largest row); a row with a larger
// exponent shifts the sum right (again less than a unit lost). Sums of up to
// 2^43 rows per thread cannot overflow (|m x 2^kFixGuard| < 2^84). A guard of
// 31 bits keeps the fast path's shift below one word. Infinities and NaNs are added in
// float64 on the side, so that a column holding one sums to a non-finite
// value (which one is unspecified, as for the other float paths).
// GB300 issues few float64 operations per clock (a TwoSum per row held the
// float64 scan to 0.6 TB/s); this takes only integer operations per row.
constexpr int kFixGuard = 31;

struct Fix128 {
  uint64_t lo, hi;
  uint32_t nneg;  // negative rows added on the fast path as ~v, each still owing +1
  int E;
  int base;       // E - kFixGuard: a row of exponent field e sits e - base bits up
  double special;
  __device__ void init() {
    lo = 0;
    hi = 0;
    nneg = 0;
    E = 0;
    base = -kFixGuard;
    special = 0.0;
  }
  // -v = ~v + 1: the fast path adds ~v and counts the +1s, added here.
  __device__ __forceinline__ void fold_neg() {
    lo += nneg;
    hi += lo < nneg ? 1ull : 0ull;
    nneg = 0;
  }
  __device__ __forceinline__ void rescale(int e) {  // e > E
    fold_neg();
    const int k = e - E;
    if (k >= 127) {
      lo = (int64_t)hi < 0 ? ~0ull : 0ull;
      hi = lo;
    } else if (k >= 64) {
      lo = (uint64_t)((int64_t)hi >> (k - 64));
      hi = (uint64_t)((int64_t)hi >> 63);
    } else {
      lo = (lo >> k) | (hi << (64 - k));
      hi = (uint64_t)((int64_t)hi >> k);
    }
    E = e;
    base = e - kFixGuard;
  }
  __device__ __forceinline__ void add(uint64_t u) {
    const uint32_t uh = (uint32_t)(u >> 32), ul = (uint32_t)u;
    const int ef = (int)((uh >> 20) & 0x7FFu);
    const int sh = ef - base;  // E - ef binades below E: sh = kFixGuard - (E - ef)
    if ((unsigned)sh <= (unsigned)kFixGuard && ef != 0) {
      // fast path: a normal value within kFixGuard binades of E. Its 53-bit
      // significand m shifted left by sh (< 32) on 32-bit words (three funnel
      // shifts), in one's complement when negative (the +1 counted in nneg),
      // added with one carry chain.
      static_assert(kFixGuard < 32, "the fast path shifts by less than one word");
      const uint32_t mh = (uh & 0x000FFFFFu) | 0x00100000u;  // m's high 21 bits (implicit bit included)
      const uint32_t s = (uint32_t)((int32_t)uh >> 31);      // all ones for a negative row
      const uint32_t x0 = __funnelshift_l(0u, ul, (unsigned)sh) ^ s;
      const uint32_t x1 = __funnelshift_l(ul, mh, (unsigned)sh) ^ s;
      const uint32_t x2 = __funnelshift_l(mh, 0u, (unsigned)sh) ^ s;  // m >> (32 - sh), 0 when sh = 0
      const uint32_t x3 = s;
      asm("{\n\t.reg .u32 a0, a1, a2, a3;\n\t"
          "mov.b64 {a0, a1}, %0;\n\t"
          "mov.b64 {a2, a3}, %1;\n\t"
          "add.cc.u32 a0, a0, %2;\n\t"
          "addc.cc.u32 a1, a1, %3;\n\t"
          "addc.cc.u32 a2, a2, %4;\n\t"
          "addc.u32 a3, a3, %5;\n\t"
          "mov.b64 %0, {a0, a1};\n\t"
          "mov.b64 %1, {a2, a3};\n\t}"
          : "+l"(lo), "+l"(hi)
          : "r"(x0), "r"(x1), "r"(x2), "r"(x3));
      nneg -= s;
      return;
    }
    fold_neg();
    if (ef == 0x7FF) {  // infinity or NaN
      special += __longlong_as_double((long long)u);
      return;
    }
    const int e = ef > 0 ? ef : 1;  // subnormals: exponent 1, no implicit bit
    const uint64_t m = (u & 0x000FFFFFFFFFFFFFull) | ((uint64_t)(ef > 0) << 52);
    if (e > E) rescale(e);
    const int d = E - e;
    uint64_t vlo, vhi;
    if (d <= kFixGuard) {
      const int sh = kFixGuard - d;  // 0 .. kFixGuard
      vlo = m << sh;
      vhi = sh > 0 ? m >> (64 - sh) : 0ull;
    } else {
      const int r = d - kFixGuard;
      vlo = r < 64 ? m >> r : 0ull;
      vhi = 0ull;
    }
    if ((int64_t)u < 0) {  // two's-complement negation of vhi:vlo
      vlo = ~vlo + 1ull;
      vhi = ~vhi + (vlo == 0ull ? 1ull : 0ull);
    }
    lo += vlo;
    hi += vhi + (lo < vlo ? 1ull : 0ull);
  }
  // The sum as an unevaluated float64 pair (rel. error about 2^-106 before
  // scaling): the 128-bit integer in three chunks that float64 holds exactly,
  // added with TwoSum, then scaled by 2^(E - 1075 - kFixGuard).
  __device__ void to_pair(double& h, double& l) const {
    const uint64_t m43 = (1ull << 43) - 1ull;
    const double q0 = (double)(lo & m43);
    const double q1 = (double)(((lo >> 43) | (hi << 21)) & m43);
    const double q2 = (double)((int64_t)hi >> 22);
    double s1, e1, s2, e2;
    two_sum(ldexp(q2, 86), ldexp(q1, 43), s1, e1);
    two_sum(s1, q0, s2, e2);
    double t, f;
    two_sum(s2, e1 + e2, t, f);
    const int sc = E - 1075 - kFixGuard;
    h = ldexp(t, sc) + special;
    l = special == 0.0 ? ldexp(f, sc) : 0.0;
  }
  // Bound on |h + l - exact sum| after `rows` adds: each add loses less than
  // one unit 2^(E - 1075 - kFixGuard) (a row far below E), each rescale less
  // than one unit of the new scale; to_pair rounds e1 + e2 (under 2^-104 of
  // the sum) and may round h and l into the subnormal range.
  __device__ double error_bound(uint32_t rows, double h, double l) const {
    if (special != 0.0) return __longlong_as_double(0x7ff0000000000000ll);
    if (E == 0) return 0.0;
    return ldexp(2.0 * (double)rows, E - 1075 - kFixGuard) + (fabs(h) + fabs(l)) * 0x1p-100 + 0x1p-1072;
  }
};

template <int DT, bool SUM, bool MM>
struct Acc<DT, SUM, MM, true> {
  using T = typename Traits<DT>::T;
  using U = typename FpImg<T>::U;
  static constexpr bool F64 = sizeof(T) == 8;
  T s, c;       // float32: TwoSum-compensated pair
  T cmax;       // float32: largest |c| so far (bounds the roundings of c)
  Fix128 fx;    // float64
  U mn, mx;
  __device__ void init() {
    s = 0; c = 0; cmax = 0;
    if (F64) fx.init();
    mn = (U)~(U)0; mx = 0;
  }
  __device__ __forceinline__ void fold(T v) {
    if (SUM) {
      if (F64) {
        fx.add((uint64_t)__double_as_longlong((double)v));
      } else {
        T t, e;
        two_sum(s, v, t, e);
        s = t;
        c += e;
        cmax = fmaxf(cmax, fabsf(c));
      }
    }
    if (MM) {
      if (F64) {
        // the image's high word decides unless it ties with an extreme's:
        // the 64-bit compares run only for a row that may move min or max
        const uint64_t b = (uint64_t)__double_as_longlong((double)v);
        const uint32_t s = (uint32_t)((int32_t)(b >> 32) >> 31);
        const uint32_t ih = (uint32_t)(b >> 32) ^ (s | 0x80000000u);
        if (ih <= (uint32_t)((uint64_t)mn >> 32) || ih >= (uint32_t)((uint64_t)mx >> 32)) {
          const U m = (U)(((uint64_t)ih << 32) | ((uint32_t)b ^ s));
          mn = min(mn, m);
          mx = max(mx, m);
        }
      } else {
        U m = FpImg<T>::img(v);
        mn = min(mn, m);
        mx = max(mx, m);
      }
    }
  }
  __device__ __forceinline__ void fold_vec(const uint4& r) {
    if (sizeof(T) == 4) {
      fold(__uint_as_float(r.x)); fold(__uint_as_float(r.y));
      fold(__uint_as_float(r.z)); fold(__uint_as_float(r.w));
    } else {
      fold(__longlong_as_double((long long)(((uint64_t)r.y << 32) | r.x)));
      fold(__longlong_as_double((long long)(((uint64_t)r.w << 32) | r.z)));
    }
  }
  // rows: the number of values this thread folded.
  __device__ void to_partial(Partial& p, uint32_t rows) const {
    p.si = 0;
    p.eb = 0.0;
    if (F64 && SUM) {
      Fix128 f = fx;
      f.fold_neg();
      f.to_pair(p.hi, p.lo);
      p.eb = f.error_bound(rows, p.hi, p.lo);
    } else {
      p.hi = (double)s;
      p.lo = (double)c;
      // TwoSum leaves s + c short only by the roundings of c: each at most
      // 2^-24 of |c| after the add (2^-150 when c is subnormal)
      if (SUM && !F64) {
        p.eb = (isfinite(p.hi) && isfinite(p.lo))
                   ? (double)rows * ((double)cmax * (0x1p-24 * (1.0 + 0x1p-23)) + 0x1p-150)
                   : __longlong_as_double(0x7ff0000000000000ll);
      }
    }
    p.mn = FpImg<T>::widen(mn);
    p.mx = FpImg<T>::widen(mx);
  }
};

// ---------------------------------------------------------------------------
// Warp / block reduction of Partial values (fixed shuffle tree).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void combine(Partial& a, const Partial& b) {
  a.si += b.si;
  double s, e;
  two_sum(a.hi, b.hi, s, e);
  a.hi = s;
  const double r1 = e + b.lo;  // rounded: at most 2^-53 |r1| (+ 2^-1075)
  a.lo += r1;                  // rounded: at most 2^-53 |a.lo| (+ 2^-1075)
  a.eb = a.eb + b.eb + (fabs(r1) + fabs(a.lo)) * 0x1p-53 + 0x1p-1074;
  a.mn = min(a.mn, b.mn);
  a.mx = max(a.mx, b.mx);
}

__device__ __forceinline__ Partial shfl_xor(const Partial& p, int m) {
  Partial q;
  q.si = __shfl_xor_sync(0xffffffffu, p.si, m);
  q.hi = __shfl_xor_sync(0xffffffffu, p.hi, m);
  q.lo = __shfl_xor_sync(0xffffffffu, p.lo, m);
  q.mn = __shfl_xor_sync(0xffffffffu, p.mn, m);
  q.mx = __shfl_xor_sync(0xffffffffu, p.mx, m);
  q.eb = __shfl_xor_sync(0xffffffffu, p.eb, m);
  return q;
}

// Block-wide reduction; the result is valid in thread 0.
template <int BLOCK>
__device__ Partial block_reduce(Partial p) {
  __shared__ Partial sm[BLOCK / 32];
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) combine(p, shfl_xor(p, m));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sm[w] = p;
  __syncthreads();
  if (w == 0) {
    if (l < BLOCK / 32) p = sm[l];
    else p = Partial{0, 0.0, 0.0, ~0ull, 0ull, 0.0};
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) combine(p, shfl_xor(p, m));
  }
  return p;
}

// Merge np partials (written by other blocks or launches) into *out.
// Called by one whole block; thread 0 writes.
template <int DT, int BLOCK>
__device__ void merge_partials(const Partial* parts, int np, agg_scalar* out, uint32_t ops,
                               int64_t count) {
  Partial acc{0, 0.0, 0.0, ~0ull, 0ull, 0.0};
  for (int i = threadIdx.x; i < np; i += BLOCK) {
    Partial q;
    q.si = __ldcg(&parts[i].si);
    q.hi = __ldcg(&parts[i].hi);
    q.lo = __ldcg(&parts[i].lo);
    q.mn = __ldcg(&parts[i].mn);
    q.mx = __ldcg(&parts[i].mx);
    q.eb = __ldcg(&parts[i].eb);
    combine(acc, q);
  }
  __syncthreads();
  acc = block_reduce<BLOCK>(acc);
  if (threadIdx.x != 0) return;
  agg_scalar r;
  r.count = count;
  r.dtype = DT;
  r.ops = ops;
  r.err_bound = 0.0;
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  if (Traits<DT>::FP) {
    double s = acc.hi + acc.lo;
    r.sum_i = 0;
    r.sum_f = s;
    // the partials' bound, plus the rounding of hi + lo and the oracle's own
    // rounding of the exact sum (each at most 2^-53 of the value), plus a
    // margin for the roundings of the bound's own sums
    if (ops & (AGG_SUM | AGG_AVG)) {
      r.err_bound = (acc.eb + fabs(s) * 0x1p-52 + 0x1p-1073) * (1.0 + 0x1p-40);
      // a column holding an infinity or a NaN has no finite bound
      if (!isfinite(s) || !isfinite(r.err_bound)) r.err_bound = __longlong_as_double(0x7ff0000000000000ll);
    }
    r.avg = count ? s / (double)count : nan;
    r.min_f = count ? f64_of_img(acc.mn) : __longlong_as_double(0x7ff0000000000000ll);
    r.max_f = count ? f64_of_img(acc.mx) : __longlong_as_double((long long)0xfff0000000000000ull);
    r.min_i = 0;
    r.max_i = 0;
  } else {
    r.sum_i = acc.si;
    r.sum_f = (double)acc.si;
    r.avg = count ? (double)acc.si / (double)count : nan;
    r.min_i = count ? i64_of_img(acc.mn) : LLONG_MAX;
    r.max_i = count ? i64_of_img(acc.mx) : LLONG_MIN;
    r.min_f = 0.0;
    r.max_f = 0.0;
  }
  *out = r;
}

constexpr int kBlock = 256;
constexpr int kUnroll = 4;

}  // namespace agg
