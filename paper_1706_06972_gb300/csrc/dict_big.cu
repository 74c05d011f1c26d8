// Dictionary step for K > 128 filters (up to 256), where one frequency's
// packed K x K double-float matrix (K(K+1)/2 x 16 bytes, 526 KB at K = 256) no
// longer fits a CTA's shared memory.  Same mathematics as dict_update.cu
// (Sec. III-B history fold, eq. (sub_d_sol) D-row solve with the Cholesky
// factor of w A^p + rho I), different blocking:
//
//   fold_big    FP32 fold A <- alpha A + beta sum_i conj(z_i) z_i^T and b on
//               the CUDA cores (the all-FP32 path; the tensor-core fold of
//               history_tc.cu is the other one);
//   factor_big  blocked right-looking Cholesky in double-float (FP32 pairs,
//               ~48 bits, on the FP32 pipe): a persistent CTA keeps the packed
//               matrix of the frequency it works on in a global workspace of
//               its own (16 bytes per entry, L2-resident), factors panels of 32
//               columns in shared memory and applies each panel to the
//               trailing matrix with 2 x 2 register tiles; w b rides along as
//               an extra column, giving y = L^-1 (w b).  Stores L in FP32;
//   dstep_big   one warp per frequency: d = L^-H (y + rho L^-1 (v^ - theta^))
//               by forward and back substitution with the FP32 factor.
#include "common.cuh"
#include "dfloat.cuh"
#include "launch.h"

namespace ocsc {

namespace {

constexpr int kBigThreads = 256;
constexpr int kNB = 32;     // panel width of factor_big
constexpr int kFoldS = 32;  // samples staged per chunk in fold_big

// Micro-tile u of the lower triangle of an R x R matrix tiled by 2 x 2:
// (mi, mk) with mk <= mi, enumerated row by row.
__device__ __forceinline__ void micro_tile(int u, int &mi, int &mk) {
  int i = (int)((sqrtf(8.0f * (float)u + 1.0f) - 1.0f) * 0.5f);
  while ((i + 1) * (i + 2) / 2 <= u) ++i;
  while (i * (i + 1) / 2 > u) --i;
  mi = i;
  mk = u - i * (i + 1) / 2;
}

}  // namespace

// One CTA per frequency.  Chunks of kFoldS samples are staged in shared
// memory; every thread owns 2 x 2 tiles of the lower triangle and updates
// them in global memory once per chunk (the first chunk applies alpha).
__global__ void __launch_bounds__(kBigThreads) fold_big_kernel(FoldArgs a) {
  extern __shared__ __align__(16) unsigned char fbs[];
  const int K = a.K, F = a.F, B = a.B;
  float2 *zs = reinterpret_cast<float2 *>(fbs);  // [kFoldS][K]
  float2 *xs = zs + kFoldS * K;                  // [kFoldS]
  const int p = blockIdx.x, tid = threadIdx.x;
  float2 *Ap = a.A + (size_t)p * tri_stride(K);
  const int h = (K + 1) / 2, tiles = h * (h + 1) / 2;
  const float alpha = (float)a.alpha, beta = (float)a.beta;
  float2 bacc = make_float2(0.f, 0.f);
  for (int c0 = 0; c0 < B; c0 += kFoldS) {
    const int nb = min(kFoldS, B - c0);
    __syncthreads();
    for (int e = tid; e < nb * K; e += kBigThreads) {
      const int s = e / K, k = e % K;
      zs[s * K + k] = a.Zp[((size_t)(c0 + s) * K + k) * F + p];
    }
    for (int s = tid; s < nb; s += kBigThreads) xs[s] = a.xh[(size_t)(c0 + s) * F + p];
    __syncthreads();
    if (tid < K)
      for (int s = 0; s < nb; ++s) bacc = cadd(bacc, cmulc(xs[s], zs[s * K + tid]));
    for (int u = tid; u < tiles; u += kBigThreads) {
      int mi, mk;
      micro_tile(u, mi, mk);
      const int i0 = 2 * mi, k0 = 2 * mk;
      float2 acc[2][2] = {};
      for (int s = 0; s < nb; ++s) {
        const float2 *z = zs + s * K;
        const float2 zi0 = z[i0], zi1 = i0 + 1 < K ? z[i0 + 1] : make_float2(0.f, 0.f);
        const float2 zk0 = z[k0], zk1 = k0 + 1 < K ? z[k0 + 1] : make_float2(0.f, 0.f);
        acc[0][0] = cadd(acc[0][0], cconjmul(zi0, zk0));
        acc[0][1] = cadd(acc[0][1], cconjmul(zi0, zk1));
        acc[1][0] = cadd(acc[1][0], cconjmul(zi1, zk0));
        acc[1][1] = cadd(acc[1][1], cconjmul(zi1, zk1));
      }
#pragma unroll
      for (int di = 0; di < 2; ++di)
#pragma unroll
        for (int dk = 0; dk < 2; ++dk) {
          const int i = i0 + di, k = k0 + dk;
          if (i >= K || k > i) continue;
          float2 *dst = Ap + tri_off(k, K) + i - k;
          const float2 old = c0 == 0 ? (a.first ? make_float2(0.f, 0.f) : *dst) : *dst;
          const float sc = c0 == 0 ? alpha : 1.0f;
          *dst = make_float2(fmaf(sc, old.x, beta * acc[di][dk].x), fmaf(sc, old.y, beta * acc[di][dk].y));
        }
    }
  }
  if (tid < K) {
    float2 *bp = a.b + (size_t)tid * F + p;
    const float2 old = a.first ? make_float2(0.f, 0.f) : *bp;
    *bp = make_float2(fmaf(alpha, old.x, beta * bacc.x), fmaf(alpha, old.y, beta * bacc.y));
  }
}

// Persistent: CTA c factors frequencies c, c + gridDim.x, ...  All of the
// factorisation is in double-float (dfloat.cuh: hi + lo FP32 pairs, complex
// entries as float4 (re hi, im hi, re lo, im lo)), as in fold_factor; the
// global workspace of a CTA holds its frequency's packed matrix in that form
// (16 bytes per entry).  Shared memory: the panel Pn[K][kNB + 1] (rows J0..
// of the current panel columns), y[K], 1 / L_jj of the panel.
__global__ void __launch_bounds__(kBigThreads, 1) factor_big_kernel(FoldArgs a, double2 *work) {
  extern __shared__ __align__(16) unsigned char fks[];
  const int K = a.K, F = a.F, T = tri_size(K), TS = tri_stride(K);
  constexpr int PS = kNB + 1;
  float4 *Pn = reinterpret_cast<float4 *>(fks);        // [K][PS]
  float4 *yv = Pn + (size_t)K * PS;                    // [K]
  float2 *invd = reinterpret_cast<float2 *>(yv + K);   // [kNB]
  float4 *W = reinterpret_cast<float4 *>(work) + (size_t)blockIdx.x * TS;
  const float2 wf = df_of(a.w), rf = df_of(a.rho_eff);
  const float rho_fb = a.rho_eff > 0.0 ? (float)a.rho_eff : 1.f;
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
  const int tid = threadIdx.x;
  for (int p = blockIdx.x; p < F; p += gridDim.x) {
    const float2 *Ap = a.A + (size_t)p * TS;
    const float2 *Lo = a.Alo ? a.Alo + (size_t)p * TS : nullptr;
    // 0. W = w A + rho I, y = w b (A as its FP32 word plus compensation word).
    for (int t = tid; t < T; t += kBigThreads) {
      int i, j;
      tri_ij(t, K, i, j);
      const float2 v = Ap[t];
      const float2 l = Lo ? Lo[t] : make_float2(0.f, 0.f);
      float Sr, Er, Si, Ei;
      df_mul(v.x, l.x, wf.x, wf.y, Sr, Er);
      df_mul(v.y, l.y, wf.x, wf.y, Si, Ei);
      if (i == j) {
        const float2 s2 = two_sum(Sr, rf.x);
        Sr = s2.x;
        Er += s2.y + rf.y;
        Si = 0.f;
        Ei = 0.f;
      }
      W[t] = make_float4(Sr, Si, Er, Ei);
    }
    for (int i = tid; i < K; i += kBigThreads) {
      const float2 bv = a.b[(size_t)i * F + p];
      float Sr, Er, Si, Ei;
      df_mul(bv.x, 0.f, wf.x, wf.y, Sr, Er);
      df_mul(bv.y, 0.f, wf.x, wf.y, Si, Ei);
      yv[i] = make_float4(Sr, Si, Er, Ei);
    }
    __syncthreads();
    float2 *Lp = a.L + (size_t)p * TS;
    for (int J0 = 0; J0 < K; J0 += kNB) {
      const int nbj = min(kNB, K - J0), R0 = K - J0;
      // a. panel columns J0 .. J0 + nbj - 1, rows from the diagonal down.
      for (int c = 0; c < nbj; ++c) {
        const int off = tri_off(J0 + c, K);
        for (int r = c + tid; r < R0; r += kBigThreads) Pn[r * PS + c] = W[off + r - c];
      }
      __syncthreads();
      // b. unblocked right-looking factorisation of the panel; y carried.
      for (int c = 0; c < nbj; ++c) {
        if (tid == 0) {
          const float4 d = Pn[c * PS + c];
          float2 pv = two_sum(d.x, d.z);
          if (!(pv.x > 0.f)) {
            atomicOr(a.err, ERR_PIVOT);
            pv = make_float2(rho_fb, 0.f);
          }
          const float2 r = df_rsqrt(pv.x, pv.y);
          float S, E;
          df_mul(pv.x, pv.y, r.x, r.y, S, E);
          const float2 ljj = two_sum(S, E);  // L_jj = p / sqrt(p)
          Pn[c * PS + c] = make_float4(ljj.x, 0.f, ljj.y, 0.f);
          invd[c] = r;
          yv[J0 + c] = df_scale(yv[J0 + c], r);
        }
        __syncthreads();
        const float2 inv = invd[c];
        for (int r = c + 1 + tid; r < R0; r += kBigThreads) Pn[r * PS + c] = df_scale(Pn[r * PS + c], inv);
        __syncthreads();
        const int ncol = nbj - c - 1;
        for (int e = tid; e < ncol * R0; e += kBigThreads) {
          const int c2 = c + 1 + e / R0, r = e % R0;
          if (r < c2) continue;
          float4 v = Pn[r * PS + c2];
          df_sub_lconjm(v, Pn[r * PS + c], Pn[c2 * PS + c]);
          Pn[r * PS + c2] = v;
        }
        const float4 yc = yv[J0 + c];
        for (int r = c + 1 + tid; r < R0; r += kBigThreads) {
          float4 v = yv[J0 + r];
          df_sub_lm(v, Pn[r * PS + c], yc);
          yv[J0 + r] = v;
        }
        __syncthreads();
      }
      // c. L of the panel in FP32.
      for (int c = 0; c < nbj; ++c) {
        const int off = tri_off(J0 + c, K);
        for (int r = c + tid; r < R0; r += kBigThreads) {
          const float4 v = Pn[r * PS + c];
          Lp[off + r - c] = make_float2(v.x + v.z, v.y + v.w);
        }
      }
      // d. trailing update W[i][k] -= sum_c L[i][c] conj(L[k][c]), J1 <= k <= i:
      //    each 2 x 2 tile sums its panel products in double-float registers,
      //    then adds them to W.
      const int J1 = J0 + nbj, R = K - J1;
      if (R > 0) {
        const int hh = (R + 1) / 2, tiles = hh * (hh + 1) / 2;
        for (int u = tid; u < tiles; u += kBigThreads) {
          int mi, mk;
          micro_tile(u, mi, mk);
          const int i0 = nbj + 2 * mi, k0 = nbj + 2 * mk;  // panel rows (relative to J0)
          const bool i1 = i0 + 1 < R0, k1 = k0 + 1 < R0;
          float4 acc[2][2] = {{zero4, zero4}, {zero4, zero4}};
          for (int c = 0; c < nbj; ++c) {
            const float4 a0 = Pn[i0 * PS + c], b0 = Pn[k0 * PS + c];
            const float4 a1 = i1 ? Pn[(i0 + 1) * PS + c] : zero4;
            const float4 b1 = k1 ? Pn[(k0 + 1) * PS + c] : zero4;
            df_sub_lconjm(acc[0][0], a0, b0);
            df_sub_lconjm(acc[0][1], a0, b1);
            df_sub_lconjm(acc[1][0], a1, b0);
            df_sub_lconjm(acc[1][1], a1, b1);
          }
#pragma unroll
          for (int di = 0; di < 2; ++di)
#pragma unroll
            for (int dk = 0; dk < 2; ++dk) {
              const int i = J0 + i0 + di, k = J0 + k0 + dk;
              if (i >= K || k > i) continue;
              float4 *dst = W + tri_off(k, K) + i - k;
              float4 v = *dst;
              df_acc2(v, acc[di][dk]);
              *dst = v;
            }
        }
      }
      __syncthreads();
    }
    for (int i = tid; i < K; i += kBigThreads)
      a.g[(size_t)i * F + p] = make_float2(yv[i].x + yv[i].z, yv[i].y + yv[i].w);
    __syncthreads();
  }
}

// One warp per frequency; lane l owns rows l, l + 32, ... (at most 8).
__global__ void __launch_bounds__(256) dstep_big_kernel(int K, int F, float rho_eff, const float2 *__restrict__ L,
                                                        const float2 *__restrict__ yb, const float2 *__restrict__ Vh,
                                                        const float2 *__restrict__ th, float2 *__restrict__ Dcur,
                                                        float2 *__restrict__ E) {
  constexpr int MR = 8;
  const int p = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (p >= F) return;
  const float2 *Lp = L + (size_t)p * tri_stride(K);
  float2 u[MR], thv[MR];
#pragma unroll
  for (int m = 0; m < MR; ++m) {
    const int i = lane + 32 * m;
    u[m] = thv[m] = make_float2(0.f, 0.f);
    if (i < K) {
      const size_t o = (size_t)i * F + p;
      thv[m] = th[o];
      u[m] = csub(Vh[o], thv[m]);  // r = v^ - theta^
    }
  }
  // Forward substitution L u = r (column by column).
  for (int j = 0; j < K; ++j) {
    const int mj = j >> 5;
    const float2 *col = Lp + tri_off(j, K) - j;  // col[i] = L_ij
    float2 uj = make_float2(0.f, 0.f);
#pragma unroll
    for (int m = 0; m < MR; ++m)
      if (m == mj) uj = u[m];
    const float ljj = col[j].x;
    uj = make_float2(__shfl_sync(0xffffffffu, uj.x, j & 31) / ljj, __shfl_sync(0xffffffffu, uj.y, j & 31) / ljj);
#pragma unroll
    for (int m = 0; m < MR; ++m) {
      const int i = lane + 32 * m;
      if (m == mj && lane == (j & 31)) u[m] = uj;
      if (i > j && i < K) u[m] = csub(u[m], cmul(col[i], uj));
    }
  }
  // z = y + rho u; back substitution L^H d = z (row j of L^H is column j of L).
#pragma unroll
  for (int m = 0; m < MR; ++m) {
    const int i = lane + 32 * m;
    if (i < K) {
      const float2 yv = yb[(size_t)i * F + p];
      u[m] = make_float2(fmaf(rho_eff, u[m].x, yv.x), fmaf(rho_eff, u[m].y, yv.y));
    }
  }
  for (int j = K - 1; j >= 0; --j) {
    const int mj = j >> 5;
    const float2 *col = Lp + tri_off(j, K) - j;
    float2 s = make_float2(0.f, 0.f);
#pragma unroll
    for (int m = 0; m < MR; ++m) {
      const int i = lane + 32 * m;
      if (i > j && i < K) s = cadd(s, cconjmul(col[i], u[m]));  // conj(L_ij) d_i
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
      s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
    }
    const float ljj = col[j].x;
#pragma unroll
    for (int m = 0; m < MR; ++m)
      if (m == mj && lane == (j & 31)) u[m] = make_float2((u[m].x - s.x) / ljj, (u[m].y - s.y) / ljj);
  }
#pragma unroll
  for (int m = 0; m < MR; ++m) {
    const int i = lane + 32 * m;
    if (i < K) {
      const size_t o = (size_t)i * F + p;
      Dcur[o] = u[m];
      E[o] = cadd(u[m], thv[m]);
    }
  }
}

cudaError_t launch_fold_big(const FoldArgs &a, cudaStream_t s) {
  const size_t sm = ((size_t)kFoldS * a.K + kFoldS) * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(fold_big_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  fold_big_kernel<<<a.F, kBigThreads, sm, s>>>(a);
  return cudaGetLastError();
}

size_t factor_big_workspace(int K, int ctas) { return (size_t)ctas * tri_stride(K); }

cudaError_t launch_factor_big(const FoldArgs &a, double2 *work, int ctas, cudaStream_t s) {
  const size_t sm = ((size_t)a.K * (kNB + 1) + a.K) * sizeof(float4) + kNB * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(factor_big_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  factor_big_kernel<<<ctas, kBigThreads, sm, s>>>(a, work);
  return cudaGetLastError();
}

cudaError_t launch_dstep_big(int K, int F, float rho_eff, const float2 *L, const float2 *yb, const float2 *Vh,
                             const float2 *th, float2 *Dcur, float2 *E, cudaStream_t s) {
  if (K > 256) return cudaErrorInvalidValue;
  const int warps = 8;
  dstep_big_kernel<<<(F + warps - 1) / warps, 32 * warps, 0, s>>>(K, F, rho_eff, L, yb, Vh, th, Dcur, E);
  return cudaGetLastError();
}

}  // namespace ocsc
