// Online dictionary step: history fold (Sec. III-B, eqs. (A_update),
// (B_update)) and DictOCSC (Algorithm 2).
//
// Per frequency p the history is A^p = mean conj(z) z^T (K x K Hermitian, kept
// as a packed lower triangle in FP32) and b^p = mean x~(p) conj(z).  The D-row
// solve of eq. (sub_d_sol) is d = (w A^p + rho I)^-1 (w b^p + rho (v^ - theta^)).
// Its matrix is fixed during the Jd ADMM iterations, so it is factored once per
// update: fold_factor folds the pending codes into A and b, forms w A + rho I in
// FP64 in shared memory, factors it by Cholesky in FP64 and stores L (FP32,
// reciprocal diagonal) together with g = (w A + rho I)^-1 (w b) computed in
// FP64.  Each ADMM iteration then solves with L in FP32 (dstep), forms the V
// update of Proposition 2 from a pruned inverse DFT restricted to the M x M
// support (vstep_cols, vstep_project), and updates the scaled dual.
#include "common.cuh"
#include "launch.h"

namespace ocsc {

__device__ __forceinline__ double2 dcmul_sub(double2 acc, double2 a, double2 b_conj_src) {
  // acc - a * conj(b)
  acc.x -= a.x * b_conj_src.x + a.y * b_conj_src.y;
  acc.y -= a.y * b_conj_src.x - a.x * b_conj_src.y;
  return acc;
}

constexpr int kFoldThreads = 256;
constexpr int kFoldChunk = 16;  // samples staged in shared memory at once

// One CTA per frequency p.
__global__ void __launch_bounds__(kFoldThreads) fold_factor_kernel(FoldArgs a) {
  extern __shared__ __align__(16) unsigned char fsm[];
  const int K = a.K, F = a.F, B = a.B;
  const int T = tri_size(K);
  double2 *M = reinterpret_cast<double2 *>(fsm);                 // [T]
  double2 *rhs = M + T;                                          // [K]
  float2 *zs = reinterpret_cast<float2 *>(rhs + K);              // [kFoldChunk][K]
  float2 *xs = zs + kFoldChunk * K;                              // [kFoldChunk]
  const int p = blockIdx.x;
  const int tid = threadIdx.x;

  for (int t = tid; t < T; t += kFoldThreads) M[t] = make_double2(0.0, 0.0);
  for (int i = tid; i < K; i += kFoldThreads) rhs[i] = make_double2(0.0, 0.0);

  // 1. Sum over the pending samples of conj(z_i) z_j and x~ conj(z_i).
  for (int c0 = 0; c0 < B; c0 += kFoldChunk) {
    const int nb = min(kFoldChunk, B - c0);
    __syncthreads();
    for (int e = tid; e < nb * K; e += kFoldThreads) {
      const int s = e / K, k = e % K;
      zs[s * K + k] = a.Zp[((size_t)(c0 + s) * K + k) * F + p];
    }
    for (int s = tid; s < nb; s += kFoldThreads) xs[s] = a.xh[(size_t)(c0 + s) * F + p];
    __syncthreads();
    for (int t = tid; t < T; t += kFoldThreads) {
      int i, j;
      tri_ij(t, K, i, j);
      float2 acc = make_float2(0.f, 0.f);
      for (int s = 0; s < nb; ++s) acc = cadd(acc, cconjmul(zs[s * K + i], zs[s * K + j]));
      M[t].x += (double)acc.x;
      M[t].y += (double)acc.y;
    }
    for (int i = tid; i < K; i += kFoldThreads) {
      float2 acc = make_float2(0.f, 0.f);
      for (int s = 0; s < nb; ++s) acc = cadd(acc, cmulc(xs[s], zs[s * K + i]));
      rhs[i].x += (double)acc.x;
      rhs[i].y += (double)acc.y;
    }
  }
  __syncthreads();

  // 2. Running means (FP32 storage) and the FP64 matrix w A + rho I.
  float2 *Ap = a.A + (size_t)p * T;
  for (int t = tid; t < T; t += kFoldThreads) {
    int i, j;
    tri_ij(t, K, i, j);
    const float2 old = a.first ? make_float2(0.f, 0.f) : Ap[t];
    const float2 nw = make_float2((float)(a.alpha * old.x + a.beta * M[t].x),
                                  (float)(a.alpha * old.y + a.beta * M[t].y));
    Ap[t] = nw;
    M[t] = make_double2(a.w * nw.x + (i == j ? a.rho_eff : 0.0), i == j ? 0.0 : a.w * nw.y);
  }
  for (int i = tid; i < K; i += kFoldThreads) {
    const float2 old = a.first ? make_float2(0.f, 0.f) : a.b[(size_t)i * F + p];
    const float2 nw = make_float2((float)(a.alpha * old.x + a.beta * rhs[i].x),
                                  (float)(a.alpha * old.y + a.beta * rhs[i].y));
    a.b[(size_t)i * F + p] = nw;
    rhs[i] = make_double2(a.w * nw.x, a.w * nw.y);
  }
  __syncthreads();

  // 3. Right-looking Cholesky in FP64 on the packed lower triangle.
  for (int j = 0; j < K; ++j) {
    const int oj = tri_off(j, K);
    double piv = M[oj].x;
    if (!(piv > 0.0)) {
      if (tid == 0) atomicOr(a.err, ERR_PIVOT);
      piv = a.rho_eff > 0.0 ? a.rho_eff : 1.0;
    }
    const double ljj = sqrt(piv);
    const double inv = 1.0 / ljj;
    for (int i = j + 1 + tid; i < K; i += kFoldThreads) {
      M[oj + i - j].x *= inv;
      M[oj + i - j].y *= inv;
    }
    __syncthreads();
    if (tid == 0) M[oj] = make_double2(ljj, 0.0);
    const int n = K - j - 1;
    const int nt = tri_size(n);
    for (int u = tid; u < nt; u += kFoldThreads) {
      int ii, kk;
      tri_ij(u, n, ii, kk);
      const int i = j + 1 + ii, k = j + 1 + kk;
      const double2 lij = M[oj + i - j];
      const double2 lkj = M[oj + k - j];
      const int dst = tri_off(k, K) + i - k;
      M[dst] = dcmul_sub(M[dst], lij, lkj);
    }
    __syncthreads();
  }

  // 4. g = L^-H L^-1 (w b) in FP64 by one warp (column-oriented substitutions).
  if (tid < 32) {
    const int lane = tid;
    for (int j = 0; j < K; ++j) {
      const int oj = tri_off(j, K);
      if (lane == 0) {
        const double inv = 1.0 / M[oj].x;
        rhs[j].x *= inv;
        rhs[j].y *= inv;
      }
      __syncwarp();
      const double2 yj = rhs[j];
      for (int i = j + 1 + lane; i < K; i += 32) {
        const double2 l = M[oj + i - j];
        rhs[i].x -= l.x * yj.x - l.y * yj.y;
        rhs[i].y -= l.x * yj.y + l.y * yj.x;
      }
      __syncwarp();
    }
    for (int j = K - 1; j >= 0; --j) {
      const int oj = tri_off(j, K);
      if (lane == 0) {
        const double inv = 1.0 / M[oj].x;
        rhs[j].x *= inv;
        rhs[j].y *= inv;
      }
      __syncwarp();
      const double2 xj = rhs[j];
      for (int i = lane; i < j; i += 32) {
        const double2 l = M[tri_off(i, K) + j - i];   // L_ji; L^H_ij = conj(L_ji)
        rhs[i].x -= l.x * xj.x + l.y * xj.y;
        rhs[i].y -= l.x * xj.y - l.y * xj.x;
      }
      __syncwarp();
    }
  }
  __syncthreads();

  // 5. Store L (FP32, reciprocal diagonal) and g.
  float2 *Lp = a.L + (size_t)p * T;
  for (int t = tid; t < T; t += kFoldThreads) {
    int i, j;
    tri_ij(t, K, i, j);
    const double2 v = M[t];
    Lp[t] = (i == j) ? make_float2((float)(1.0 / v.x), 0.f) : make_float2((float)v.x, (float)v.y);
  }
  for (int i = tid; i < K; i += kFoldThreads)
    a.g[(size_t)i * F + p] = make_float2((float)rhs[i].x, (float)rhs[i].y);
}

// D-row step: d = g + rho L^-H L^-1 (v^ - theta^); one warp per frequency, the
// factor of that frequency staged in shared memory.  Also writes E = d + theta^.
template <int NR>
__global__ void dstep_kernel(int K, int F, float rho_eff, const float2 *__restrict__ L,
                             const float2 *__restrict__ g, const float2 *__restrict__ Vh,
                             const float2 *__restrict__ th, float2 *__restrict__ Dcur,
                             float2 *__restrict__ E) {
  extern __shared__ float2 dsm[];
  const int T = tri_size(K);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  const int p = blockIdx.x * wpb + warp;
  if (p >= F) return;
  float2 *sL = dsm + (size_t)warp * T;
  const float2 *Lp = L + (size_t)p * T;
  for (int t = lane; t < T; t += 32) sL[t] = Lp[t];
  float2 y[NR];
#pragma unroll
  for (int m = 0; m < NR; ++m) {
    const int i = lane + 32 * m;
    if (i < K) {
      const float2 v = Vh[(size_t)i * F + p], t = th[(size_t)i * F + p];
      y[m] = make_float2(rho_eff * (v.x - t.x), rho_eff * (v.y - t.y));
    } else {
      y[m] = make_float2(0.f, 0.f);
    }
  }
  __syncwarp();
  // Forward: L y' = y.
  for (int j = 0; j < K; ++j) {
    const int oj = tri_off(j, K);
    float2 mine = y[0];
#pragma unroll
    for (int m = 1; m < NR; ++m)
      if ((j >> 5) == m) mine = y[m];
    float2 yj;
    yj.x = __shfl_sync(0xffffffffu, mine.x, j & 31);
    yj.y = __shfl_sync(0xffffffffu, mine.y, j & 31);
    const float invd = sL[oj].x;
    yj.x *= invd;
    yj.y *= invd;
#pragma unroll
    for (int m = 0; m < NR; ++m) {
      const int i = lane + 32 * m;
      if (i == j) y[m] = yj;
      if (i > j && i < K) {
        const float2 l = sL[oj + i - j];
        y[m].x -= l.x * yj.x - l.y * yj.y;
        y[m].y -= l.x * yj.y + l.y * yj.x;
      }
    }
  }
  // Backward: L^H x = y'.
  for (int j = K - 1; j >= 0; --j) {
    float2 mine = y[0];
#pragma unroll
    for (int m = 1; m < NR; ++m)
      if ((j >> 5) == m) mine = y[m];
    float2 xj;
    xj.x = __shfl_sync(0xffffffffu, mine.x, j & 31);
    xj.y = __shfl_sync(0xffffffffu, mine.y, j & 31);
    const float invd = sL[tri_off(j, K)].x;
    xj.x *= invd;
    xj.y *= invd;
#pragma unroll
    for (int m = 0; m < NR; ++m) {
      const int i = lane + 32 * m;
      if (i == j) y[m] = xj;
      if (i < j) {
        const float2 l = sL[tri_off(i, K) + j - i];
        y[m].x -= l.x * xj.x + l.y * xj.y;
        y[m].y -= l.x * xj.y - l.y * xj.x;
      }
    }
  }
#pragma unroll
  for (int m = 0; m < NR; ++m) {
    const int i = lane + 32 * m;
    if (i < K) {
      const size_t o = (size_t)i * F + p;
      const float2 d = cadd(g[o], y[m]);
      Dcur[o] = d;
      E[o] = cadd(d, th[o]);
    }
  }
}

// Pruned inverse DFT along k1, restricted to m1 in [0, M):
// Y[k][m1][k2] = sum_k1 E[k][k1][k2] exp(+2 pi i k1 m1 / N).
constexpr int kMaxM = 16;
__global__ void vstep_cols_kernel(int K, int N, int M, const float2 *__restrict__ E,
                                  const float2 *__restrict__ tw, float2 *__restrict__ Y) {
  const int NH = N / 2 + 1, F = N * NH;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= K * NH) return;
  const int k = idx / NH, k2 = idx % NH;
  float2 acc[kMaxM];
#pragma unroll
  for (int m = 0; m < kMaxM; ++m) acc[m] = make_float2(0.f, 0.f);
  const float2 *Ek = E + (size_t)k * F + k2;
  for (int k1 = 0; k1 < N; ++k1) {
    const float2 e = Ek[(size_t)k1 * NH];
#pragma unroll
    for (int m = 0; m < kMaxM; ++m) {
      if (m < M) {
        const float2 w = tw[(k1 * m) & (N - 1)];
        acc[m] = cadd(acc[m], cmulc(e, w));
      }
    }
  }
#pragma unroll
  for (int m = 0; m < kMaxM; ++m)
    if (m < M) Y[((size_t)k * M + m) * NH + k2] = acc[m];
}

// One CTA per filter k.  mode 0: alpha = H(F^-1(E)) from Y, V = alpha /
// max(||alpha||, 1) (Proposition 2), V^ = F(pad V), theta^ += D~ - V^.
// mode 1: V^ = F(pad V) for a given V.
constexpr int kProjThreads = 256;
__global__ void __launch_bounds__(kProjThreads)
    vstep_project_kernel(int mode, int K, int N, int M, const float2 *__restrict__ Y,
                         float *__restrict__ V, float2 *__restrict__ Vh, float2 *__restrict__ th,
                         const float2 *__restrict__ Dcur, const float2 *__restrict__ tw) {
  extern __shared__ __align__(16) unsigned char psm[];
  const int NH = N / 2 + 1, F = N * NH, MM = M * M;
  float *alpha = reinterpret_cast<float *>(psm);          // [M*M]
  float *red = alpha + kMaxM * kMaxM;                      // [32]
  float2 *Tm = reinterpret_cast<float2 *>(red + 32);       // [M][NH]
  const int k = blockIdx.x, tid = threadIdx.x;
  if (mode == 0) {
    const float invP = 1.0f / (float)(N * N);
    float ss = 0.f;
    for (int e = tid; e < MM; e += kProjThreads) {
      const int m1 = e / M, m2 = e % M;
      const float2 *Yr = Y + ((size_t)k * M + m1) * NH;
      float s = 0.f;
      for (int k2 = 0; k2 < NH; ++k2) {
        const float2 y = Yr[k2];
        const float2 w = tw[(k2 * m2) & (N - 1)];
        const float c = (k2 == 0 || k2 == N / 2) ? 1.f : 2.f;
        s += c * (y.x * w.x + y.y * w.y);
      }
      s *= invP;
      alpha[e] = s;
      ss += s * s;
    }
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if ((tid & 31) == 0) red[tid >> 5] = ss;
    __syncthreads();
    if (tid < 32) {
      float v = tid < kProjThreads / 32 ? red[tid] : 0.f;
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (tid == 0) red[0] = v;
    }
    __syncthreads();
    const float scale = 1.0f / fmaxf(sqrtf(red[0]), 1.0f);
    for (int e = tid; e < MM; e += kProjThreads) {
      const float v = alpha[e] * scale;
      alpha[e] = v;
      V[(size_t)k * MM + e] = v;
    }
  } else {
    for (int e = tid; e < MM; e += kProjThreads) alpha[e] = V[(size_t)k * MM + e];
  }
  __syncthreads();
  // Tm(m1, k2) = sum_m2 V(m1, m2) W^(k2 m2)
  for (int e = tid; e < M * NH; e += kProjThreads) {
    const int m1 = e / NH, k2 = e % NH;
    float2 acc = make_float2(0.f, 0.f);
    for (int m2 = 0; m2 < M; ++m2) {
      const float2 w = tw[(k2 * m2) & (N - 1)];
      const float v = alpha[m1 * M + m2];
      acc.x += v * w.x;
      acc.y += v * w.y;
    }
    Tm[e] = acc;
  }
  __syncthreads();
  for (int p = tid; p < F; p += kProjThreads) {
    const int k1 = p / NH, k2 = p % NH;
    float2 acc = make_float2(0.f, 0.f);
    for (int m1 = 0; m1 < M; ++m1) acc = cadd(acc, cmul(Tm[m1 * NH + k2], tw[(k1 * m1) & (N - 1)]));
    const size_t o = (size_t)k * F + p;
    Vh[o] = acc;
    if (mode == 0) {
      const float2 d = Dcur[o];
      const float2 t = th[o];
      th[o] = make_float2(t.x + d.x - acc.x, t.y + d.y - acc.y);
    }
  }
}

__global__ void dict_norms_kernel(int K, int F, const float2 *__restrict__ Dh, float *__restrict__ dn) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= F) return;
  float s = 0.f;
  for (int k = 0; k < K; ++k) {
    const float2 d = Dh[(size_t)k * F + p];
    s += d.x * d.x + d.y * d.y;
  }
  dn[p] = s;
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------

size_t fold_smem_bytes(int K) {
  return (size_t)tri_size(K) * sizeof(double2) + (size_t)K * sizeof(double2) +
         (size_t)kFoldChunk * K * sizeof(float2) + kFoldChunk * sizeof(float2);
}

cudaError_t launch_fold_factor(const FoldArgs &a, cudaStream_t s) {
  const size_t sm = fold_smem_bytes(a.K);
  cudaError_t e = cudaFuncSetAttribute(fold_factor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  fold_factor_kernel<<<a.F, kFoldThreads, sm, s>>>(a);
  return cudaGetLastError();
}

template <int NR>
static cudaError_t dstep_n(int K, int F, float rho_eff, const float2 *L, const float2 *g,
                           const float2 *Vh, const float2 *th, float2 *Dcur, float2 *E, cudaStream_t s) {
  const size_t per = (size_t)tri_size(K) * sizeof(float2);
  int wpb = (int)((200u * 1024u) / per);
  wpb = wpb < 1 ? 1 : (wpb > 8 ? 8 : wpb);
  const size_t sm = per * wpb;
  cudaError_t e = cudaFuncSetAttribute(dstep_kernel<NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  dstep_kernel<NR><<<(F + wpb - 1) / wpb, 32 * wpb, sm, s>>>(K, F, rho_eff, L, g, Vh, th, Dcur, E);
  return cudaGetLastError();
}

cudaError_t launch_dstep(int K, int F, float rho_eff, const float2 *L, const float2 *g,
                         const float2 *Vh, const float2 *th, float2 *Dcur, float2 *E,
                         cudaStream_t s) {
  if (K <= 32) return dstep_n<1>(K, F, rho_eff, L, g, Vh, th, Dcur, E, s);
  if (K <= 64) return dstep_n<2>(K, F, rho_eff, L, g, Vh, th, Dcur, E, s);
  if (K <= 128) return dstep_n<4>(K, F, rho_eff, L, g, Vh, th, Dcur, E, s);
  if (K <= 256) return dstep_n<8>(K, F, rho_eff, L, g, Vh, th, Dcur, E, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_vstep_cols(int K, int N, int M, const float2 *E, const float2 *tw, float2 *Y,
                              cudaStream_t s) {
  if (M > kMaxM) return cudaErrorInvalidValue;
  const int total = K * (N / 2 + 1);
  vstep_cols_kernel<<<(total + 127) / 128, 128, 0, s>>>(K, N, M, E, tw, Y);
  return cudaGetLastError();
}

cudaError_t launch_vstep_project(int mode, int K, int N, int M, const float2 *Y, float *V,
                                 float2 *Vh, float2 *th, const float2 *Dcur, const float2 *tw,
                                 cudaStream_t s) {
  if (M > kMaxM) return cudaErrorInvalidValue;
  const size_t sm = (kMaxM * kMaxM + 32) * sizeof(float) + (size_t)M * (N / 2 + 1) * sizeof(float2);
  vstep_project_kernel<<<K, kProjThreads, sm, s>>>(mode, K, N, M, Y, V, Vh, th, Dcur, tw);
  return cudaGetLastError();
}

cudaError_t launch_dict_norms(int K, int F, const float2 *Dh, float *dn, cudaStream_t s) {
  dict_norms_kernel<<<(F + 255) / 256, 256, 0, s>>>(K, F, Dh, dn);
  return cudaGetLastError();
}

}  // namespace ocsc
