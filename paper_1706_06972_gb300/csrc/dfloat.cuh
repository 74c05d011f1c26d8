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

// 1 / sqrt(p) for p = ph + pl > 0 as a pair: the FP32 estimate r0 (a few
// ulp) refined by one Newton step r0 (1 + e / 2), e = 1 - p r0^2 formed in
// double-float, which squares the relative error.
__device__ __forceinline__ float2 df_rsqrt(float ph, float pl) {
  const float r0 = rsqrtf(ph);
  float S, E;
  df_mul(r0, 0.f, r0, 0.f, S, E);
  const float2 q = two_sum(S, E);
  df_mul(ph, pl, q.x, q.y, S, E);
  const float2 pr = two_sum(S, E);
  const float2 e1 = two_sum(1.f, -pr.x);
  const float e = e1.x + (e1.y - pr.y);
  return two_sum(r0, 0.5f * r0 * e);
}

// Normalised pair product (v re, v im) x r for a complex pair v (possibly
// unnormalised) and a real pair r.
__device__ __forceinline__ float4 df_scale(float4 v, float2 r) {
  const float2 vr = two_sum(v.x, v.z), vi = two_sum(v.y, v.w);
  float Sr, Er, Si, Ei;
  df_mul(vr.x, vr.y, r.x, r.y, Sr, Er);
  df_mul(vi.x, vi.y, r.x, r.y, Si, Ei);
  const float2 a = two_sum(Sr, Er), b = two_sum(Si, Ei);
  return make_float4(a.x, b.x, a.y, b.y);
}

// v -= l conj(m) (complex pairs; v unnormalised).
__device__ __forceinline__ void df_sub_lconjm(float4 &v, const float4 &l, const float4 &m) {
  df_mac(-l.x, -l.z, m.x, m.z, v.x, v.z);  // Re: - Re l Re m - Im l Im m
  df_mac(-l.y, -l.w, m.y, m.w, v.x, v.z);
  df_mac(-l.y, -l.w, m.x, m.z, v.y, v.w);  // Im: - Im l Re m + Re l Im m
  df_mac(l.x, l.z, m.y, m.w, v.y, v.w);
}

// w = -l conj(m) (complex pairs, unnormalised): the first product of each
// part needs no TwoSum.
__device__ __forceinline__ void df_neg_lconjm(float4 &w, const float4 &l, const float4 &m) {
  df_mul(-l.x, -l.z, m.x, m.z, w.x, w.z);  // Re: - Re l Re m
  df_mac(-l.y, -l.w, m.y, m.w, w.x, w.z);  //     - Im l Im m
  df_mul(-l.y, -l.w, m.x, m.z, w.y, w.w);  // Im: - Im l Re m
  df_mac(l.x, l.z, m.y, m.w, w.y, w.w);    //     + Re l Im m
}

// v -= l m (complex pairs; v unnormalised).
__device__ __forceinline__ void df_sub_lm(float4 &v, const float4 &l, const float4 &m) {
  df_mac(-l.x, -l.z, m.x, m.z, v.x, v.z);  // Re: - Re l Re m + Im l Im m
  df_mac(l.y, l.w, m.y, m.w, v.x, v.z);
  df_mac(-l.x, -l.z, m.y, m.w, v.y, v.w);  // Im: - Re l Im m - Im l Re m
  df_mac(-l.y, -l.w, m.x, m.z, v.y, v.w);
}

}  // namespace ocsc
