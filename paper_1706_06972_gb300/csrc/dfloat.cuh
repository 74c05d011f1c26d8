// Double-float arithmetic on the FP32 pipe: a real number is an unevaluated
// sum hi + lo of two floats (about 48 significant bits).  Products are split
// exactly with an FMA (p = fl(a b), fma(a, b, -p) = a b - p) and sums by
// Knuth's TwoSum (s = fl(a + b), the exact error from four more additions),
// so the per-frequency FP64 work of the dictionary step (Cholesky factor,
// Sherman-Morrison recursion, Hermitian products) runs at FP32 issue rate.
// Complex entries are stored as float4 (re hi, im hi, re lo, im lo).
#pragma once
#include <cuda_runtime.h>

namespace ocsc {

// a + b = s + e exactly (no ordering condition on a, b).
__device__ __forceinline__ float2 two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return make_float2(s, (a - (s - bb)) + (b - bb));
}

// (S, E) += a b for a = ah + al, b = bh + bl: S takes fl(ah bh) by TwoSum, E
// gathers the rounding errors and the cross terms (al bl is below the pair's
// precision).  __fmul_rn keeps the product from being contracted into the sum.
// The pair (S, E) is unnormalised: its value is S + E.
__device__ __forceinline__ void df_mac(float ah, float al, float bh, float bl, float &S, float &E) {
  const float p = __fmul_rn(ah, bh);
  const float corr = fmaf(ah, bl, fmaf(al, bh, fmaf(ah, bh, -p)));
  const float s = S + p;
  const float bb = s - S;
  const float e = (S - (s - bb)) + (p - bb);
  S = s;
  E += e + corr;
}

// (ah + al)(bh + bl) as an unnormalised pair (S, E).
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float &S, float &E) {
  S = __fmul_rn(ah, bh);
  E = fmaf(ah, bl, fmaf(al, bh, fmaf(ah, bh, -S)));
}

// (S, E) + (S2, E2) as an unnormalised pair.
__device__ __forceinline__ void df_acc(float &S, float &E, float S2, float E2) {
  const float2 s = two_sum(S, S2);
  S = s.x;
  E = (E + E2) + s.y;
}

// v += w for complex unnormalised pairs (re S, im S, re E, im E).
__device__ __forceinline__ void df_acc2(float4 &v, const float4 &w) {
  df_acc(v.x, v.z, w.x, w.z);
  df_acc(v.y, v.w, w.y, w.w);
}

// S + E as a normalised pair (hi, lo), valid for any S, E.
__device__ __forceinline__ float2 df_norm(float S, float E) { return two_sum(S, E); }

// Normalised pair of a double.
__device__ __forceinline__ float2 df_of(double x) {
  const float h = (float)x;
  return make_float2(h, (float)(x - (double)h));
}

__device__ __forceinline__ float4 df_split2(double x, double y) {
  const float hx = (float)x, hy = (float)y;
  return make_float4(hx, hy, (float)(x - (double)hx), (float)(y - (double)hy));
}

__device__ __forceinline__ double df_val(float h, float l) { return (double)h + (double)l; }

}  // namespace ocsc
