// Host build of the exact-sum arithmetic of the GPU's exact float GROUP BY
// mode (csrc/exact.cuh), driven by tests/test_exact_host.py: the rows of one
// group are added into digits exactly as the device kernels do (plain adds in
// place of atomics) and rounded once.
#include <climits>
#include <cstring>

#include "../paper_2606_10030_gb300/csrc/exact.cuh"

using namespace agg;

template <class F>
static double run(const F* x, int64_t n, bool f32, int* digits_out) {
  int lo = INT_MAX, hi = INT_MIN;
  for (int64_t i = 0; i < n; ++i) {
    ExactParts p;
    if (f32) {
      uint32_t b;
      std::memcpy(&b, &x[i], 4);
      p = exact_parts_f32(b);
    } else {
      uint64_t b;
      std::memcpy(&b, &x[i], 8);
      p = exact_parts_f64(b);
    }
    if (p.mant == 0) continue;
    lo = lo < p.lsb ? lo : p.lsb;
    hi = hi > p.lsb ? hi : p.lsb;
  }
  int base = 0, D = 1;
  if (lo != INT_MAX) {
    base = lo;
    D = (hi - lo + (f32 ? 24 : 53) + 33 + kDigitBits - 1) / kDigitBits + 2;
  }
  *digits_out = D;
  if (D > kMaxDigits) return 0.0;
  int64_t a[kMaxDigits] = {0};
  for (int64_t i = 0; i < n; ++i) {
    ExactParts p;
    if (f32) {
      uint32_t b;
      std::memcpy(&b, &x[i], 4);
      p = exact_parts_f32(b);
    } else {
      uint64_t b;
      std::memcpy(&b, &x[i], 8);
      p = exact_parts_f64(b);
    }
    if (p.mant == 0) continue;
    const int pos = p.lsb - base;
    const int q = pos / kDigitBits;
    int64_t c[3];
    exact_chunks(p.mant, pos - q * kDigitBits, c);
    for (int k = 0; k < 3; ++k)
      a[q + k] = (int64_t)((uint64_t)a[q + k] + (uint64_t)(p.neg ? -c[k] : c[k]));
  }
  return exact_round(a, D, base);
}

extern "C" double exact_host_sum_f64(const double* x, int64_t n, int* digits) { return run(x, n, false, digits); }
extern "C" double exact_host_sum_f32(const float* x, int64_t n, int* digits) { return run(x, n, true, digits); }
