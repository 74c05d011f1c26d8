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
// sm_fold:  one CTA per frequency; C (packed lower, FP64) in shared memory for
//           the whole batch; b folded as the running mean in FP32; stores C.
// dstep_sm: one CTA per frequency, thread i owns row i of the Hermitian product
//           (FP64); the caller passes r / t.
#include "common.cuh"
#include "launch.h"

namespace ocsc {

namespace {

constexpr int kSmThreads = 256;

__device__ __forceinline__ double block_sum_d(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];  // fixed order, every thread
  return t;
}

}  // namespace

// Shared memory: C [T] double2, z [K] double2, u [K] double2, two partial
// halves of u [2][K] double2, red [32] double.
__global__ void __launch_bounds__(kSmThreads) sm_fold_kernel(SmArgs a) {
  extern __shared__ __align__(16) unsigned char smm[];
  const int K = a.K, F = a.F, T = tri_size(K), TS = tri_stride(K);
  double2 *Cs = reinterpret_cast<double2 *>(smm);
  double2 *z = Cs + T;
  double2 *u = z + K;
  double2 *uh = u + K;  // [2][K]
  double *red = reinterpret_cast<double *>(uh + 2 * K);
  const int p = blockIdx.x, tid = threadIdx.x;
  double2 *Cg = a.C + (size_t)p * TS;
  if (a.n > 0)
    for (int t = tid; t < T; t += kSmThreads) Cs[t] = Cg[t];
  float2 bacc = make_float2(0.f, 0.f);
  for (int s = 0; s < a.B; ++s) {
    const double t = (double)(a.n + 1 + s);
    __syncthreads();
    for (int k = tid; k < K; k += kSmThreads) {
      const float2 v = a.Zp[((size_t)s * K + k) * F + p];
      z[k] = make_double2(v.x, v.y);
      if (k == tid) {
        const float2 x = a.xh[(size_t)s * F + p];
        bacc = cadd(bacc, cmulc(x, v));  // x~ conj(z)
      }
    }
    if (a.n + s == 0) {  // C_0 = I / r
      for (int e = tid; e < T; e += kSmThreads) {
        int i, j;
        tri_ij(e, K, i, j);
        Cs[e] = make_double2(i == j ? 1.0 / a.r : 0.0, 0.0);
      }
    }
    __syncthreads();
    // u = C conj(z): row i split over two threads (columns j even / odd).
    for (int e = tid; e < 2 * K; e += kSmThreads) {
      const int i = e >> 1, h = e & 1;
      double2 acc = make_double2(0.0, 0.0);
      for (int j = h; j < K; j += 2) {
        const double2 c = j <= i ? Cs[tri_off(j, K) + i - j] : Cs[tri_off(i, K) + j - i];
        const double cy = j <= i ? c.y : -c.y;  // C_ij = conj(C_ji) above the diagonal
        const double2 zc = make_double2(z[j].x, -z[j].y);
        acc.x = fma(c.x, zc.x, acc.x);
        acc.x = fma(-cy, zc.y, acc.x);
        acc.y = fma(c.x, zc.y, acc.y);
        acc.y = fma(cy, zc.x, acc.y);
      }
      uh[h * K + i] = acc;
    }
    __syncthreads();
    double part = 0.0;
    for (int i = tid; i < K; i += kSmThreads) {
      const double2 ui = make_double2(uh[i].x + uh[K + i].x, uh[i].y + uh[K + i].y);
      u[i] = ui;
      part += z[i].x * ui.x - z[i].y * ui.y;  // Re(z_i u_i): z^T C conj(z) is real
    }
    const double zu = block_sum_d(part, red);
    const bool first = a.n + s == 0;
    const double den = first ? 1.0 + zu : (t - 1.0) + zu;
    const double sc = first ? 1.0 : t / (t - 1.0);
    const double inv = 1.0 / den;
    for (int e = tid; e < T; e += kSmThreads) {
      int i, j;
      tri_ij(e, K, i, j);
      const double2 ui = u[i], uj = u[j];
      double2 c = Cs[e];
      // c - u_i conj(u_j) / den
      c.x -= (ui.x * uj.x + ui.y * uj.y) * inv;
      c.y -= (ui.y * uj.x - ui.x * uj.y) * inv;
      Cs[e] = make_double2(sc * c.x, sc * c.y);
    }
  }
  __syncthreads();
  for (int t = tid; t < T; t += kSmThreads) Cg[t] = Cs[t];
  for (int k = tid; k < K; k += kSmThreads) {
    float2 *bp = a.b + (size_t)k * F + p;
    const float2 old = a.n == 0 ? make_float2(0.f, 0.f) : *bp;
    *bp = make_float2(fmaf(a.alpha, old.x, a.beta * bacc.x), fmaf(a.alpha, old.y, a.beta * bacc.y));
  }
}

// d = C (b + r (v^ - theta^)) with C Hermitian (packed lower, FP64), in FP64:
// C_t's ridge decays as r / t, so its condition number grows with t and an FP32
// product would lose accuracy; also E = d + theta^.  ths != 1 rescales theta^
// first (stored back: the scaled dual after a change of penalty).
__global__ void dstep_sm_kernel(int K, int F, double r, double ths, const double2 *__restrict__ C,
                                const float2 *__restrict__ b, const float2 *__restrict__ Vh,
                                float2 *__restrict__ th, float2 *__restrict__ Dcur,
                                float2 *__restrict__ E) {
  extern __shared__ __align__(16) double2 dsm_s[];
  const int TS = tri_stride(K);
  double2 *sC = dsm_s;
  double2 *sw = sC + TS;
  const int p = blockIdx.x, i = threadIdx.x;
  const double2 *g = C + (size_t)p * TS;
  for (int c = i; c < TS; c += blockDim.x) cp_async16(sC + c, g + c);
  float2 thi = make_float2(0.f, 0.f);
  if (i < K) {
    const size_t o = (size_t)i * F + p;
    const float2 v = Vh[o], bb = b[o];
    thi = th[o];
    if (ths != 1.0) {
      thi = make_float2((float)(ths * thi.x), (float)(ths * thi.y));
      th[o] = thi;
    }
    sw[i] = make_double2((double)bb.x + r * ((double)v.x - thi.x), (double)bb.y + r * ((double)v.y - thi.y));
  }
  cp_async_wait_all();
  __syncthreads();
  if (i < K) {
    double2 acc = make_double2(0.0, 0.0);
    for (int j = 0; j < K; ++j) {
      const bool low = j <= i;
      const double2 c = low ? sC[tri_off(j, K) + i - j] : sC[tri_off(i, K) + j - i];
      const double cy = low ? c.y : -c.y;
      const double2 w = sw[j];
      acc.x = fma(c.x, w.x, acc.x);
      acc.x = fma(-cy, w.y, acc.x);
      acc.y = fma(c.x, w.y, acc.y);
      acc.y = fma(cy, w.x, acc.y);
    }
    const size_t o = (size_t)i * F + p;
    const float2 d = make_float2((float)acc.x, (float)acc.y);
    Dcur[o] = d;
    E[o] = cadd(d, thi);
  }
}

cudaError_t launch_sm_fold(const SmArgs &a, cudaStream_t s) {
  if (a.K < 1 || a.K > 128) return cudaErrorInvalidValue;
  const int T = tri_size(a.K);
  const size_t sm = ((size_t)T + 4 * a.K) * sizeof(double2) + 32 * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(sm_fold_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  sm_fold_kernel<<<a.F, kSmThreads, sm, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_dstep_sm(int K, int F, double r, double ths, const double2 *C, const float2 *b,
                            const float2 *Vh, float2 *th, float2 *Dcur, float2 *E, cudaStream_t s) {
  if (K > 128) return cudaErrorInvalidValue;
  const size_t sm = ((size_t)tri_stride(K) + K) * sizeof(double2);
  cudaError_t e = cudaFuncSetAttribute(dstep_sm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  dstep_sm_kernel<<<F, 128, sm, s>>>(K, F, r, ths, C, b, Vh, th, Dcur, E);
  return cudaGetLastError();
}

}  // namespace ocsc
