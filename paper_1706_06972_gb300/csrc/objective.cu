// Objective of eq. (ocsc0) for one sample: 1/2 ||x - sum_k D_k (*) U_k||^2 +
// lambda ||U||_1 on the padded N x N domain, evaluated against the current
// coding dictionary.
//
// The residual norm is taken in the frequency domain (Parseval, Sec. II-C):
// ||r||^2 = (1/P) sum over the full spectrum of |R^(p)|^2 with
// R^ = x~ - sum_k D~_k U^_k; on the stored half spectrum the columns
// k2 = 0 and k2 = N/2 count once and every other column twice.  All sums are
// FP64 and deterministic: fixed per-block partials, then one block adds them in
// order.
#include "common.cuh"
#include "launch.h"

namespace ocsc {

constexpr int kObjBlock = 256;

__device__ __forceinline__ double block_sum(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    t = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;  // valid in thread 0
}

// Partial sums of w(p) |x~(p) - sum_k D~_k(p) U^_k(p)|^2, one per block.
__global__ void __launch_bounds__(kObjBlock)
    objective_resid_kernel(int K, int N, const float2 *__restrict__ Dh, const float2 *__restrict__ xh,
                           const float2 *__restrict__ Uh, double *__restrict__ partial) {
  __shared__ double red[32];
  const int NH = N / 2 + 1, F = N * NH;
  const int p = blockIdx.x * kObjBlock + threadIdx.x;
  double v = 0.0;
  if (p < F) {
    float2 s = xh[p];
    for (int k = 0; k < K; ++k) {
      const float2 d = Dh[(size_t)k * F + p], u = Uh[(size_t)k * F + p];
      s.x -= d.x * u.x - d.y * u.y;
      s.y -= d.x * u.y + d.y * u.x;
    }
    const int k2 = p % NH;
    const double w = (k2 == 0 || k2 == N / 2) ? 1.0 : 2.0;
    v = w * ((double)s.x * s.x + (double)s.y * s.y);
  }
  const double t = block_sum(v, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// Partial sums of |u|, one per block.
__global__ void __launch_bounds__(kObjBlock)
    l1_partial_kernel(const float *__restrict__ u, size_t count, double *__restrict__ partial) {
  __shared__ double red[32];
  double v = 0.0;
  const size_t stride = (size_t)gridDim.x * kObjBlock;
  for (size_t i = (size_t)blockIdx.x * kObjBlock + threadIdx.x; i < count; i += stride) v += fabs((double)u[i]);
  const double t = block_sum(v, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// out[0] = a sa / 2 + b sb, out[1] = a sa, out[2] = sb with sa = sum(pa[0..na)),
// sb = sum(pb[0..nb)), summed in index order: the objective, the squared
// residual norm ||x - sum_k D_k (*) U_k||^2 and ||U||_1.
__global__ void objective_final_kernel(const double *__restrict__ pa, int na, double a,
                                       const double *__restrict__ pb, int nb, double b,
                                       double *__restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double sa = 0.0, sb = 0.0;
  for (int i = 0; i < na; ++i) sa += pa[i];
  for (int i = 0; i < nb; ++i) sb += pb[i];
  out[0] = 0.5 * a * sa + b * sb;
  out[1] = a * sa;
  out[2] = sb;
}

// Partial sums of (a - b)^2 and a^2, one pair per block.
__global__ void __launch_bounds__(kObjBlock)
    rel_diff_partial_kernel(const float *__restrict__ a, const float *__restrict__ b, size_t count,
                            double *__restrict__ partial) {
  __shared__ double red[32];
  double d = 0.0, n = 0.0;
  const size_t stride = (size_t)gridDim.x * kObjBlock;
  for (size_t i = (size_t)blockIdx.x * kObjBlock + threadIdx.x; i < count; i += stride) {
    const double x = a[i], y = b[i];
    d += (x - y) * (x - y);
    n += x * x;
  }
  const double td = block_sum(d, red);
  __syncthreads();
  const double tn = block_sum(n, red);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = td;
    partial[2 * blockIdx.x + 1] = tn;
  }
}

__global__ void rel_diff_final_kernel(const double *__restrict__ partial, int nb, double *__restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double d = 0.0, n = 0.0;
  for (int i = 0; i < nb; ++i) {
    d += partial[2 * i];
    n += partial[2 * i + 1];
  }
  *out = n > 0.0 ? sqrt(d / n) : (d > 0.0 ? INFINITY : 0.0);
}

cudaError_t launch_rel_diff(const float *a, const float *b, size_t count, double *partial, double *out,
                            cudaStream_t s) {
  rel_diff_partial_kernel<<<kObjL1Blocks, kObjBlock, 0, s>>>(a, b, count, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  rel_diff_final_kernel<<<1, 32, 0, s>>>(partial, kObjL1Blocks, out);
  return cudaGetLastError();
}

// PSNR of Sec. IV per sample from its squared residual norm:
// out[i] = 10 log10(peak^2 P_i / r2_i), r2_i = terms[3 i + 1] (the layout the
// objective kernels write), P_i the pixel count of the sample's padded domain.
__global__ void psnr_kernel(const double *__restrict__ terms, PsnrArgs a, double *__restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  out[i] = 10.0 * log10(a.peak * a.peak * (double)a.P[i] / terms[3 * i + 1]);
}

cudaError_t launch_psnr(const double *terms, const PsnrArgs &a, double *out, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  psnr_kernel<<<1, kMaxPsnr, 0, s>>>(terms, a, out);
  return cudaGetLastError();
}

// Display order of the filters (Sec. IV): ascending sample variance over the
// M x M entries of each filter (divided by the entry count minus one; 0 for
// 1 x 1 filters), ties kept in index order.  One block: thread k forms the
// variance of filter k in FP64, then its rank among all K (a stable counting
// rank), and writes order[rank] = k.
__global__ void filter_order_kernel(int K, int MM, const float *__restrict__ V, int *__restrict__ order) {
  __shared__ double var[kMaxOrderK];
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    const float *f = V + (size_t)k * MM;
    double mu = 0.0;
    for (int e = 0; e < MM; ++e) mu += (double)f[e];
    mu /= (double)MM;
    double ss = 0.0;
    for (int e = 0; e < MM; ++e) {
      const double d = (double)f[e] - mu;
      ss += d * d;
    }
    var[k] = MM > 1 ? ss / (double)(MM - 1) : 0.0;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    int rank = 0;
    for (int j = 0; j < K; ++j) rank += (var[j] < var[k] || (var[j] == var[k] && j < k)) ? 1 : 0;
    order[rank] = k;
  }
}

cudaError_t launch_filter_order(int K, int M, const float *V, int *order, cudaStream_t s) {
  if (K > kMaxOrderK) return cudaErrorInvalidValue;
  filter_order_kernel<<<1, 256, 0, s>>>(K, M * M, V, order);
  return cudaGetLastError();
}

int objective_partials(int N) {
  const int F = N * (N / 2 + 1);
  return (F + kObjBlock - 1) / kObjBlock + kObjL1Blocks;
}

cudaError_t launch_objective(int K, int N, double lam, const float2 *Dh, const float2 *xh,
                             const float2 *Uh, const float *u, double *partial, double *out,
                             cudaStream_t s) {
  const int F = N * (N / 2 + 1);
  const int nr = (F + kObjBlock - 1) / kObjBlock;
  objective_resid_kernel<<<nr, kObjBlock, 0, s>>>(K, N, Dh, xh, Uh, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  l1_partial_kernel<<<kObjL1Blocks, kObjBlock, 0, s>>>(u, (size_t)K * N * N, partial + nr);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  objective_final_kernel<<<1, 32, 0, s>>>(partial, nr, 1.0 / ((double)N * N), partial + nr, kObjL1Blocks, lam,
                                          out);
  return cudaGetLastError();
}

}  // namespace ocsc
