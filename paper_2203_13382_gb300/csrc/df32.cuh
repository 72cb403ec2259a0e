// FP32-pair ("double-float") arithmetic for the level-0 residual of the FP32-bulk cycle.
//
// A value is carried as an unevaluated sum h + l of two FP32 numbers, |l| at most a few units in the last
// place of h, which gives about 48 significant bits from the FP32 pipes (GB300 runs FP64 at 1/64 of the
// FP32 rate).  The building blocks are the classical error-free transformations:
//  - the exact product of two FP32 numbers a * b = p + e with p = fl(a b), e = fma(a, b, -p)
//    (Dekker 1971, "A floating-point technique for extending the available precision", in its fused
//    multiply-add form);
//  - the exact sum a + b = s + e of Knuth's TwoSum (The Art of Computer Programming, vol. 2, 4.2.2), and
//    Dekker's Fast2Sum when |a| >= |b| is known.
// Every operation below uses the round-to-nearest intrinsics, so the compiler never contracts or
// reassociates them.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace mgrit {

struct df32 {
  float h, l;
};

// The FP64 value x as a pair (h = x rounded to FP32, l = the rest rounded to FP32).
MGRIT_D df32 df_from_double(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(__dsub_rn(x, (double)h))};
}

MGRIT_D double df_to_double(df32 a) { return __dadd_rn((double)a.h, (double)a.l); }

// (double)x for an FP32 x by moving its bits (exact: rebiased exponent, significand shifted into place);
// zero keeps its sign, subnormal, infinite and NaN inputs take the conversion instruction.
MGRIT_D double float_to_double_bits(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
  if ((u & 0x7fffffffu) == 0) return __longlong_as_double((long long)sign);
  if (e == 0 || e == 0xffu) return (double)x;
  return __longlong_as_double((long long)(sign | ((unsigned long long)(e + 896u) << 52) |
                                          ((unsigned long long)(u & 0x7fffffu) << 29)));
}

// df_to_double with the two conversions done by float_to_double_bits (one FP64 instruction, the add).
MGRIT_D double df_to_double_bits(df32 a) { return __dadd_rn(float_to_double_bits(a.h), float_to_double_bits(a.l)); }

// c - e for an integer c with |c| >= 1 and 0 <= e.h < 1 (so |c| >= |e.h|: Fast2Sum), not renormalised.
MGRIT_D df32 df_int_minus(float c, df32 e) {
  const float s = __fsub_rn(c, e.h);
  const float err = __fsub_rn(__fsub_rn(c, s), e.h);
  return {s, __fsub_rn(err, e.l)};
}

// a * b, not renormalised: the exact product of the high parts plus the two cross terms (the product of
// the low parts is below 2^-44 of the result and dropped).
MGRIT_D df32 df_mul(df32 a, df32 b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return {p, e};
}

// a * k for a small integer k (exact in FP32).
MGRIT_D df32 df_mul_int(df32 a, float k) {
  const float p = __fmul_rn(a.h, k);
  return {p, __fmaf_rn(a.l, k, __fmaf_rn(a.h, k, -p))};
}

// Accumulates t into the running sum (sh exact by TwoSum, the rounding errors and low parts into sl).
MGRIT_D void df_acc(float& sh, float& sl, df32 t) {
  const float s = __fadd_rn(sh, t.h);
  const float bb = __fsub_rn(s, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(t.h, bb));
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(err, t.l));
}

// (h, l) with |l| <= half an ulp of h (Fast2Sum; valid when |h| >= |l|).
MGRIT_D df32 df_norm(float h, float l) {
  const float s = __fadd_rn(h, l);
  return {s, __fsub_rn(l, __fsub_rn(s, h))};
}

// (-1)^{P-a} C(P, a): the integer numerators of the Lagrange basis coefficients 1 / prod_{b != a} (a - b)
// once they are scaled by P!.
template <int P>
constexpr float signed_binomial(int a) {
  int c = 1;
  for (int t = 1; t <= a; ++t) c = c * (P - a + t) / t;
  return ((P - a) & 1) ? -(float)c : (float)c;
}

// 1 / P! as a pair (high part and the rest), formed at compile time in FP64.
template <int P>
struct InvFactorial {
  float h, l;
  constexpr InvFactorial() : h(0.f), l(0.f) {
    double f = 1.0;
    for (int t = 2; t <= P; ++t) f *= t;
    const double v = 1.0 / f;
    h = (float)v;
    l = (float)(v - (double)h);
  }
};

// The SL interpolation sum_a w_a(eps) u_a (Sec. 2.1: nodes j = a - (P+1)/2 around the east node, the
// departure point at -eps) in FP32 pairs.  w_a = c_a prod_{b != a} f_b with the factors f_b = -eps - j_b
// = ((P+1)/2 - b) - eps and c_a = (-1)^{P-a} C(P, a) / P!: the products by prefix and suffix products
// (3 (P - 1) pair products), the integers C(P, a) exactly, the sum by TwoSum, then one product by 1/P!.
// FP32 operations: 4 P (factors) + 12 (P - 1) (products) + 3 (P - 1) (integers, P > 1) + 12 (P + 1) - 8
// (gather and sum) + 10 (scaling; 3 for P = 1): 31, 92 and 153 for P = 1, 3, 5.
template <int P>
MGRIT_D df32 df_interp(df32 eps, const float2* __restrict__ u) {
  constexpr int L = (P + 1) / 2;
  df32 f[P + 1];
#pragma unroll
  for (int b = 0; b <= P; ++b)
    f[b] = (b == L) ? df32{-eps.h, -eps.l} : df_int_minus((float)(L - b), eps);
  df32 pre[P + 1], suf[P + 1];  // pre[a] = prod_{b < a} f_b (a >= 1), suf[a] = prod_{b > a} f_b (a <= P - 1)
  pre[1] = f[0];
#pragma unroll
  for (int a = 2; a <= P; ++a) pre[a] = df_mul(pre[a - 1], f[a - 1]);
  suf[P - 1] = f[P];
#pragma unroll
  for (int a = P - 2; a >= 0; --a) suf[a] = df_mul(suf[a + 1], f[a + 1]);
  float sh = 0.f, sl = 0.f;
#pragma unroll
  for (int a = 0; a <= P; ++a) {
    df32 w = (a == 0) ? suf[0] : (a == P ? pre[P] : df_mul(pre[a], suf[a]));
    const float k = signed_binomial<P>(a);
    if (k == -1.f) w = df32{-w.h, -w.l};
    else if (k != 1.f) w = df_mul_int(w, k);
    const float2 ua = u[a];
    const df32 t = df_mul(w, df32{ua.x, ua.y});
    if (a == 0) {
      sh = t.h;
      sl = t.l;
    } else {
      df_acc(sh, sl, t);
    }
  }
  constexpr InvFactorial<P> inv{};
  const df32 s = df_norm(sh, sl);
  if constexpr (P == 1) return s;  // 1 / 1! = 1
  const df32 r = df_mul(s, df32{inv.h, inv.l});
  return df_norm(r.h, r.l);
}

}  // namespace mgrit
