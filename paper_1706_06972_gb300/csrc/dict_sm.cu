// Recursion variant of the history (eq. (C_update), reading R3): instead of
// factoring w A^p + rho I at every update, keep C^p itself and apply, for every
// folded sample t = n + 1, n + 2, ... in arrival order, the printed
// Sherman-Morrison recursion
//   t = 1:  C = I / r - conj(z) z^T / (r (r + z^T conj(z)))
//   t > 1:  C = t/(t-1) [C - u u^H / ((t-1) + z^T u)],   u = C conj(z)
// (z = Z~_t(p, :)^T, r = rho or rho P; C Hermitian, so C conj(z) z^T C = u u^H).
// This is exact for C_t = (A_t + (r / t) I)^-1 (a ridge decaying as 1/t), and
// costs two O(K^2) passes per sample instead of an O(K^3) factorisation.  That
// C_t is eq. (sub_d_sol)'s inverse for the penalty rho / t, so the D-row step
// is d = C (b + (r / t) (v^ - theta^)) (reading R23: with r itself on the right
// the iteration grows by about t - 1 per step in the null space of A_t).
//
// C is kept in double-float (an FP32 pair hi + lo per real number: 16 bytes per
// complex entry, about 48 significant bits) and all O(K^2) work runs on the
// FP32 pipe with error-free products (FMA) and sums (Knuth's TwoSum); the
// per-sample scalars (z^T C conj(z), the scale factors) are FP64.
// Both kernels take one CTA per frequency with the packed triangle in shared
// memory, and split every row of the Hermitian product C x over kRowLanes
// adjacent lanes (columns j = q mod kRowLanes), merged by shuffles in FP64.
// sm_fold:  C for the whole batch; b folded as the running mean in FP32.
// dstep_sm: the caller passes r / t.
#include "common.cuh"
#include "dfloat.cuh"
#include "launch.h"

namespace ocsc {

namespace {

constexpr int kSmThreads = 256;
constexpr int kRowLanes = 2;  // lanes per row of a Hermitian product (divides 32)

// Block-wide sum of an unnormalised pair, in a fixed order, returned to every
// thread normalised.
__device__ __forceinline__ float2 block_sum_df(float S, float E, float2 *red) {
  for (int o = 16; o > 0; o >>= 1)
    df_acc(S, E, __shfl_xor_sync(0xffffffffu, S, o), __shfl_xor_sync(0xffffffffu, E, o));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = make_float2(S, E);
  __syncthreads();
  float tS = 0.f, tE = 0.f;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) df_acc(tS, tE, red[w].x, red[w].y);
  return two_sum(tS, tE);
}

// Row i of C w over the columns j = q, q + kRowLanes, ... (C Hermitian, packed
// lower, double-float [re hi, im hi, re lo, im lo]; w double-float likewise):
// lower entries C_ij (j <= i) sit at tri_off(j) + i - j, upper ones
// C_ij = conj(C_ji) at tri_off(i) + j - i, and both offsets advance by a fixed
// rule per step.  Returns the partial as unnormalised pairs (S re, E re, S im,
// E im).
__device__ __forceinline__ float4 herm_row_part(const float4 *sC, const float4 *sw, int K, int i, int q) {
  constexpr int L = kRowLanes;
  int lo = tri_off(q, K) + i - q, up = tri_off(i, K) + q - i;
  float S0 = 0.f, S1 = 0.f, S2 = 0.f, S3 = 0.f, E0 = 0.f, E1 = 0.f, E2 = 0.f, E3 = 0.f;
#pragma unroll 2
  for (int j = q; j < K; j += L) {
    const bool low = j <= i;
    const float4 c = sC[low ? lo : up];
    const float4 w = sw[j];
    const float yh = low ? c.y : -c.y, yl = low ? c.w : -c.w;
    df_mac(c.x, c.z, w.x, w.z, S0, E0);    // Re C Re w
    df_mac(-yh, -yl, w.y, w.w, S1, E1);    // -Im C Im w
    df_mac(c.x, c.z, w.y, w.w, S2, E2);    // Re C Im w
    df_mac(yh, yl, w.x, w.z, S3, E3);      // Im C Re w
    lo += L * (K - j) - L * (L + 1) / 2;   // tri_off(j + L) - tri_off(j) - L
    up += L;
  }
  df_acc(S0, E0, S1, E1);
  df_acc(S2, E2, S3, E3);
  return make_float4(S0, E0, S2, E2);
}

// Sum of a row's kRowLanes partials (adjacent lanes of one warp), normalised:
// (re hi, im hi, re lo, im lo).
__device__ __forceinline__ float4 row_merge(float4 v) {
#pragma unroll
  for (int o = 1; o < kRowLanes; o <<= 1) {
    const float a = __shfl_xor_sync(0xffffffffu, v.x, o), b = __shfl_xor_sync(0xffffffffu, v.y, o);
    const float c = __shfl_xor_sync(0xffffffffu, v.z, o), d = __shfl_xor_sync(0xffffffffu, v.w, o);
    df_acc(v.x, v.y, a, b);
    df_acc(v.z, v.w, c, d);
  }
  const float2 re = two_sum(v.x, v.y), im = two_sum(v.z, v.w);
  return make_float4(re.x, im.x, re.y, im.y);
}

}  // namespace

// Shared memory: C [T] float4 (double-float), conj(z) as double-float [K]
// float4, v = g u [K] float4, u [K] float4 (double-float), red [32] float2,
// scalars [4] float2.
__global__ void __launch_bounds__(kSmThreads) sm_fold_kernel(SmArgs a) {
  extern __shared__ __align__(16) unsigned char smm[];
  const int K = a.K, F = a.F, T = tri_size(K), TS = tri_stride(K);
  float4 *Cs = reinterpret_cast<float4 *>(smm);
  float4 *zc = Cs + T;
  float4 *vv = zc + K;
  float4 *u = vv + K;
  float2 *red = reinterpret_cast<float2 *>(u + K);
  float2 *scal = red + 32;  // g, sc (double-float), set by thread 0
  const int p = blockIdx.x, tid = threadIdx.x;
  const int row = tid / kRowLanes, q = tid % kRowLanes, ii = row < K ? row : K - 1;
  float4 *Cg = a.C + (size_t)p * TS;
  if (a.n > 0)
    for (int t = tid; t < T; t += kSmThreads) Cs[t] = Cg[t];
  float2 bacc = make_float2(0.f, 0.f);
  for (int s = 0; s < a.B; ++s) {
    const bool first = a.n + s == 0;
    __syncthreads();
    if (tid < K) {
      const float2 v = a.Zp[((size_t)s * K + tid) * F + p];
      zc[tid] = make_float4(v.x, -v.y, 0.f, 0.f);  // conj(z), exact
      const float2 x = a.xh[(size_t)s * F + p];
      bacc = cadd(bacc, cmulc(x, v));  // x~ conj(z)
    }
    if (first) {  // C_0 = I / r
      const float4 d = make_float4(a.rinv.x, 0.f, a.rinv.y, 0.f);
      for (int e = tid; e < T; e += kSmThreads) {
        int i, j;
        tri_ij(e, K, i, j);
        Cs[e] = i == j ? d : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    __syncthreads();
    // u = C conj(z)
    const float4 ui = row_merge(herm_row_part(Cs, zc, K, ii, q));
    if (row < K && q == 0) u[row] = ui;
    __syncthreads();
    // z^T C conj(z) = sum_i Re(z_i u_i), real.
    float Sz = 0.f, Ez = 0.f;
    if (tid < K) {
      const float4 uz = u[tid], z4 = zc[tid];
      df_mac(z4.x, 0.f, uz.x, uz.z, Sz, Ez);
      df_mac(z4.y, 0.f, uz.y, uz.w, Sz, Ez);
    }
    const float2 zu = block_sum_df(Sz, Ez, red);
    // C <- sc C - v v^H with v = g u, g^2 = sc / den (one thread, FP64).
    if (tid == 0) {
      const double t = (double)(a.n + 1 + s), zud = df_val(zu.x, zu.y);
      const double den = first ? 1.0 + zud : (t - 1.0) + zud;
      const double sc = first ? 1.0 : t / (t - 1.0);
      scal[0] = df_of(sqrt(sc / den));
      scal[1] = df_of(sc);
    }
    __syncthreads();
    const float2 g = scal[0], sc = scal[1];
    if (tid < K) {
      const float4 uz = u[tid];
      float Sr, Er, Si, Ei;
      df_mul(uz.x, uz.z, g.x, g.y, Sr, Er);
      df_mul(uz.y, uz.w, g.x, g.y, Si, Ei);
      const float2 vr = two_sum(Sr, Er), vi = two_sum(Si, Ei);
      vv[tid] = make_float4(vr.x, vi.x, vr.y, vi.y);
    }
    __syncthreads();
    for (int e = tid; e < T; e += kSmThreads) {
      int i, j;
      tri_ij(e, K, i, j);
      const float4 vi = vv[i], vj = vv[j], c = Cs[e];
      // Re: sc Re c - (Re vi Re vj + Im vi Im vj);  Im: sc Im c - (Im vi Re vj - Re vi Im vj)
      float Sr, Er, Si, Ei;
      df_mul(c.x, c.z, sc.x, sc.y, Sr, Er);
      df_mac(-vi.x, -vi.z, vj.x, vj.z, Sr, Er);
      df_mac(-vi.y, -vi.w, vj.y, vj.w, Sr, Er);
      df_mul(c.y, c.w, sc.x, sc.y, Si, Ei);
      df_mac(-vi.y, -vi.w, vj.x, vj.z, Si, Ei);
      df_mac(vi.x, vi.z, vj.y, vj.w, Si, Ei);
      const float2 nr = two_sum(Sr, Er), ni = two_sum(Si, Ei);
      Cs[e] = make_float4(nr.x, ni.x, nr.y, ni.y);
    }
  }
  __syncthreads();
  for (int t = tid; t < T; t += kSmThreads) Cg[t] = Cs[t];
  if (tid < K) {
    float2 *bp = a.b + (size_t)tid * F + p;
    const float2 old = a.n == 0 ? make_float2(0.f, 0.f) : *bp;
    *bp = make_float2(fmaf(a.alpha, old.x, a.beta * bacc.x), fmaf(a.alpha, old.y, a.beta * bacc.y));
  }
}

// d = C (b + r (v^ - theta^)) with C Hermitian (packed lower, double-float);
// w = b + r (v^ - theta^) is formed in double-float from the FP32 inputs and
// r = (r hi, r lo).  C_t's ridge decays as r / t, so its condition number
// grows with t and a plain FP32 product would lose accuracy.  Also
// E = d + theta^; ths != 1 rescales theta^ first (stored back: the scaled dual
// after a change of penalty).
__global__ void __launch_bounds__(kRowLanes * 128) dstep_sm_kernel(int K, int F, float2 r, float ths,
                                                                   const float4 *__restrict__ Cf,
                                                                   const float2 *__restrict__ b,
                                                                   const float2 *__restrict__ Vh,
                                                                   float2 *__restrict__ th,
                                                                   float2 *__restrict__ Dcur,
                                                                   float2 *__restrict__ E) {
  extern __shared__ __align__(16) float4 dsm_s[];
  const int TS = tri_stride(K);
  float4 *sC = dsm_s;
  float4 *sw = sC + TS;
  const int p = blockIdx.x, tid = threadIdx.x;
  const int row = tid / kRowLanes, q = tid % kRowLanes, ii = row < K ? row : K - 1;
  const float4 *g = Cf + (size_t)p * TS;
  for (int c = tid; c < TS; c += blockDim.x) cp_async16(sC + c, g + c);
  cp_async_commit();
  float2 thi = make_float2(0.f, 0.f);
  const size_t o = (size_t)row * F + p;
  if (row < K && q == 0) {
    const float2 v = Vh[o], bb = b[o];
    thi = th[o];
    if (ths != 1.f) {
      thi = make_float2(ths * thi.x, ths * thi.y);
      th[o] = thi;
    }
    // b + r (v - theta), each part exact until the final rounding to a pair.
    const float2 dr = two_sum(v.x, -thi.x), di = two_sum(v.y, -thi.y);
    float Sr, Er, Si, Ei;
    df_mul(dr.x, dr.y, r.x, r.y, Sr, Er);
    df_mul(di.x, di.y, r.x, r.y, Si, Ei);
    df_acc(Sr, Er, bb.x, 0.f);
    df_acc(Si, Ei, bb.y, 0.f);
    const float2 wr = two_sum(Sr, Er), wi = two_sum(Si, Ei);
    sw[row] = make_float4(wr.x, wi.x, wr.y, wi.y);
  }
  cp_async_wait_all();
  __syncthreads();
  const float4 d = row_merge(herm_row_part(sC, sw, K, ii, q));  // idle lanes redo row K - 1
  if (row < K && q == 0) {
    const float2 df = make_float2(d.x + d.z, d.y + d.w);
    Dcur[o] = df;
    E[o] = cadd(df, thi);
  }
}

cudaError_t launch_sm_fold(const SmArgs &a, cudaStream_t s) {
  if (a.K < 1 || a.K > 128) return cudaErrorInvalidValue;
  const int T = tri_size(a.K);
  const size_t sm = ((size_t)T + 3 * a.K) * sizeof(float4) + 36 * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(sm_fold_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  sm_fold_kernel<<<a.F, kSmThreads, sm, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_dstep_sm(int K, int F, double r, double ths, const float4 *Cf, const float2 *b,
                            const float2 *Vh, float2 *th, float2 *Dcur, float2 *E, cudaStream_t s) {
  if (K < 1 || K > 128) return cudaErrorInvalidValue;
  const size_t sm = ((size_t)tri_stride(K) + K) * sizeof(float4);
  cudaError_t e = cudaFuncSetAttribute(dstep_sm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const float rh = (float)r;
  const float2 rf = make_float2(rh, (float)(r - (double)rh));
  dstep_sm_kernel<<<F, (kRowLanes * K + 31) / 32 * 32, sm, s>>>(K, F, rf, (float)ths, Cf, b, Vh, th, Dcur, E);
  return cudaGetLastError();
}

}  // namespace ocsc
