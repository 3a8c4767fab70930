// Double-float ("df32") arithmetic on the FP32 pipe.
//
// A df32 value is the unevaluated sum h + l of two floats with |l| <= ulp(h)/2,
// about 48 significant bits. On GB300 the FP32 pipe issues 64x more operations per
// clock than the FP64 pipe, so FP64-accurate sums and products that are dominated
// by multiply-adds run faster in df32 than in native FP64.
//
// Error-free transformations: TwoSum (Knuth), Fast2Sum (Dekker, |a| >= |b|),
// TwoProd with a fused multiply-add. Files that include this header are compiled
// with -fmad=false, so every FMA below is an explicit fmaf.
#pragma once
#include <cuda_runtime.h>

struct f2 {
  float h, l;
};

__device__ __forceinline__ f2 two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}

__device__ __forceinline__ f2 fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}

__device__ __forceinline__ f2 two_prod(float a, float b) {
  const float p = a * b;
  return {p, fmaf(a, b, -p)};
}

// Product of two df32 values (relative error about 2^-46).
__device__ __forceinline__ f2 df_mul(f2 a, f2 b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return fast_two_sum(p, e);
}

// df32 times a float.
__device__ __forceinline__ f2 df_mulf(f2 a, float b) {
  const float p = a.h * b;
  float e = fmaf(a.h, b, -p);
  e = fmaf(a.l, b, e);
  return fast_two_sum(p, e);
}

// Sum of two df32 values with both parts combined by TwoSum (accurate for any signs).
__device__ __forceinline__ f2 df_add(f2 a, f2 b) {
  f2 s = two_sum(a.h, b.h);
  const f2 t = two_sum(a.l, b.l);
  s.l += t.h;
  s = fast_two_sum(s.h, s.l);
  s.l += t.l;
  return fast_two_sum(s.h, s.l);
}

__device__ __forceinline__ f2 df_neg(f2 a) { return {-a.h, -a.l}; }

// 1 / b by one Newton step on the float reciprocal: x1 = x0 + x0 (1 - b x0).
__device__ __forceinline__ f2 df_recip(f2 b) {
  const float x0 = 1.0f / b.h;
  // residual 1 - b*x0 in df32
  const f2 bx = df_mulf(b, x0);
  const f2 res = df_add({1.0f, 0.0f}, df_neg(bx));
  const f2 corr = two_prod(x0, res.h);
  return df_add({x0, 0.0f}, {corr.h, corr.l + x0 * res.l});
}

// Split a double into a df32 pair (runs on the FP64/convert units: use per particle, not per node).
__device__ __forceinline__ f2 df_from_double(double d) {
  const float h = (float)d;
  return {h, (float)(d - (double)h)};
}

__device__ __forceinline__ double df_to_double(f2 a) { return (double)a.h + (double)a.l; }

// A normalised df32 pair (|l| <= ulp(h)/2) as the double h + l, truncated to 53 bits,
// by integer operations only (no conversion or FP64 instruction, which on GB300 run at
// the FP64 rate even when a branch around them is never taken): a subnormal h gives a
// signed zero, an infinite or NaN h the double infinity or NaN.
__device__ __forceinline__ double df_to_f64(f2 a) {
  const unsigned hb = __float_as_uint(a.h), lb = __float_as_uint(a.l);
  const unsigned long long sgn = (unsigned long long)(hb >> 31) << 63;
  const int eh = (int)((hb >> 23) & 0xFF);
  if (eh == 0) return __longlong_as_double((long long)sgn);
  if (eh == 0xFF)
    return __longlong_as_double((long long)(sgn | 0x7FF0000000000000ull | ((hb & 0x7FFFFFu) ? (1ull << 51) : 0ull)));
  unsigned long long S = (unsigned long long)((hb & 0x7FFFFFu) | 0x800000u) << 29;  // unit 2^(eh - 179)
  if (lb & 0x7FFFFFFFu) {
    const int el = (int)((lb >> 23) & 0xFF);
    const unsigned ml = (lb & 0x7FFFFFu) | (el ? 0x800000u : 0u);
    const int k = min((el ? el : 1) - eh + 29, 5);  // l = ml 2^(el - 150) = ml 2^k units (k <= 5 when normalised)
    const unsigned long long L = k >= 0 ? ((unsigned long long)ml << k) : (k > -32 ? (unsigned long long)(ml >> -k) : 0ull);
    S = ((hb ^ lb) >> 31) ? S - L : S + L;
  }
  int e = eh;
  if (S >> 53) {
    S >>= 1;
    ++e;
  } else if (!(S >> 52)) {
    S <<= 1;
    --e;
  }
  return __longlong_as_double((long long)(sgn | ((unsigned long long)(e + 896) << 52) | (S & ((1ull << 52) - 1))));
}

// Constants of exp2(j/64) and the split of ln(2)/64, computed on the host in
// double precision and passed to the kernels.
struct DfExpTable {
  float th[64], tl[64];  // 2^(j/64) = th[j] + tl[j]
  float L1, L2, L3;      // ln(2)/64 = L1 + L2 + L3, L1 with 11 significant bits
  float inv;             // 64 / ln(2)
};

// exp(u) for u in [-80, 0] to about 2^-46 relative, by the table-driven method of
// P. T. P. Tang (ACM TOMS 15, 1989): u = (64 m + j) ln2/64 + r with |r| <= ln2/128,
// exp(u) = 2^m 2^(j/64) exp(r), exp(r) = 1 + r + r^2/2 + r^3 (1/6 + r/24 + r^2/120 + r^3/720),
// the cubic tail (below 3e-8) in plain float, the rest in df32.
// The table entries th[j], tl[j] are read from th / tl: pass a copy of T.th / T.tl in
// shared memory, since lanes index them with different j (from the constant bank the
// reads would be serialised).
__device__ __forceinline__ f2 df_exp_neg(f2 u, const DfExpTable& T, const float* th, const float* tl) {
  const float kf = rintf(u.h * T.inv);
  const int k = (int)kf;
  // r = u - k (L1 + L2 + L3); k L1 is exact and u.h - k L1 cancels exactly (Sterbenz)
  const float a = fmaf(-kf, T.L1, u.h);
  const f2 b = two_prod(kf, T.L2);
  f2 r = two_sum(a, -b.h);
  r.l += (u.l - b.l) - kf * T.L3;
  r = fast_two_sum(r.h, r.l);
  const float rh = r.h;
  f2 r2 = two_prod(rh, rh);
  r2.l = fmaf(2.0f * rh, r.l, r2.l);
  const float tail = rh * r2.h * (1.0f / 6.0f + rh * (1.0f / 24.0f + rh * (1.0f / 120.0f + rh * (1.0f / 720.0f))));
  f2 s = df_add(r, {0.5f * r2.h, 0.5f * r2.l});
  s = df_add(s, {tail, 0.0f});
  const f2 e = df_add({1.0f, 0.0f}, s);
  const int m = (k >= 0) ? (k >> 6) : -((-k + 63) >> 6);
  const int j = k - 64 * m;
  f2 res = df_mul({th[j], tl[j]}, e);
  const float sc = ldexpf(1.0f, m);
  return {res.h * sc, res.l * sc};
}
