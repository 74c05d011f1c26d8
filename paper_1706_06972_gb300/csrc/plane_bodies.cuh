// Device bodies of the N <= 128 coding kernels: the per-frequency residual
// of the Z~-step and the fused plane iteration on the half spectrum.  Each
// body takes its block coordinates explicitly; code_admm.cu wraps them as
// kernels and the persistent coder (persist.cu) runs them as units of one
// cooperative launch.  The design notes are at the top of code_admm.cu.
#pragma once
#include "fft.cuh"
#include "launch.h"

namespace ocsc {

template <int N, int NT>
__device__ __forceinline__ void load_twiddles(float2 *s_tw, const float2 *__restrict__ tw) {
  for (int i = threadIdx.x; i < N; i += NT) s_tw[i] = tw[i];
}

__device__ __forceinline__ float soft_threshold(float v, float t) {
  return v > t ? v - t : (v < -t ? v + t : 0.0f);
}

// Sum kResidTerms values over a block; thread 0 writes them to out.
__device__ __forceinline__ void block_sum_terms(float (&v)[kResidTerms], float *out) {
  __shared__ float red[kResidTerms][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < kResidTerms; ++q) {
    float x = v[q];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) red[q][warp] = x;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < kResidTerms; ++q) {
      float x = lane < nw ? red[q][lane] : 0.f;
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) out[q] = x;
    }
  }
}

// r_p = (x~(p) - sum_k D~_k(p) W^_k(p)) / (rho + |d_p|^2) for 32 bins
// pb * 32 .. of image img; 256 threads as (32 bins) x (8 filter lanes).
__device__ __forceinline__ void code_resid_body(int K, int F, float rho, int first, int serve, const ImgBatch &b,
                                                const float2 *__restrict__ Dh, const float *__restrict__ dn,
                                                const float2 *__restrict__ xh, const float2 *__restrict__ What,
                                                float2 *__restrict__ r, int pb, int img, int tx, int ty) {
  __shared__ float2 part[8][33];
  const int p = pb * 32 + tx;
  const int slot = b.slot[img];
  const bool is_first = serve ? b.iter[img] == 0 : first != 0;
  float2 s = make_float2(0.f, 0.f);
  if (!is_first && p < F) {
    const float2 *w = What + (size_t)slot * K * F;
#pragma unroll 4
    for (int k = ty; k < K; k += 8) s = cadd(s, cmul(Dh[(size_t)k * F + p], w[(size_t)k * F + p]));
  }
  part[ty][tx] = s;
  __syncthreads();
  if (ty == 0 && p < F) {
    float2 t = part[0][tx];
#pragma unroll
    for (int y = 1; y < 8; ++y) t = cadd(t, part[y][tx]);
    const float2 x = xh[(size_t)slot * F + p];
    const float inv = 1.0f / (rho + dn[p]);
    r[(size_t)slot * F + p] = make_float2((x.x - t.x) * inv, (x.y - t.y) * inv);
  }
}

// One fused ADMM iteration for filter k of one sample, on its half spectrum.
//
// The tile holds the N x (N/2 + 1) half spectrum exactly as it lies in global
// memory (pitch N/2 + 1), 67.5 KB at N = 128, so two or three CTAs share an SM
// and one CTA's loads and stores overlap another's transforms.  The real 2D
// inverse runs as N/2 column transforms of length N (the columns k2 = 0 and
// k2 = N/2 are Hermitian in k1, so their inverses are real and travel packed
// as one complex column c0 + i cN/2), then per row the half-length complex
// inverse of the packed row: for a real row x with half spectrum X[0..N/2],
// h[m] = x[2m] + i x[2m+1] has the N/2-point spectrum
//   H[k] = (X[k] + conj X[N/2-k]) + i W_N^-k (X[k] - conj X[N/2-k])
// (times 2 against the 1/N-normalised split, which keeps the scale of an
// unnormalised length-N inverse).  The forward transform reverses the steps:
// half-length row transforms of h, the split
//   X[k] = (H[k] + conj H[N/2-k]) / 2 + W_N^k (H[k] - conj H[N/2-k]) / (2i),
// X[0] and X[N/2] real (packed as one complex column), N/2 column transforms.
//
template <int N>
__device__ __forceinline__ void code_plane_body(const CodeIter &it, const ImgBatch &b, const float2 *__restrict__ tw,
                                                int k, int img, float4 *hsmem) {
  constexpr int NT = HalfPlan<N>::NT, NH = N / 2 + 1, H = N / 2, Q = H / 2 + 1;
  constexpr int F = N * NH, P = N * N;
  float2 *tile = reinterpret_cast<float2 *>(hsmem);  // [N][NH]
  float2 *s_tw = tile + F;                           // [N]
  const int K = it.K;
  const int slot = b.slot[img];
  const int t = b.iter[img];
  const bool first = it.serve ? t == 0 : it.first != 0;
  const bool store_last = it.serve ? (t + 1) % it.check == 0 : it.last != 0;
  const bool store_prev = it.serve && (t + 2) % it.check == 0;
  const bool skip_fwd = !it.serve && it.last;
  load_twiddles<N, NT>(s_tw, tw);

  const float2 *Dk = it.Dh + (size_t)k * F;
  const float2 *rr = it.r + (size_t)slot * F;
  float2 *Wk = it.What + ((size_t)slot * K + k) * F;
  float2 *Zk = it.Zp + ((size_t)slot * K + k) * F;

  // 1. Z~-step z = w^ + conj(d) r_p over the half spectrum.  W^ of this
  //    filter comes into the tile (its global layout) by 16-byte asynchronous
  //    copies, all in flight at once; D~ and r are read two bins per 16-byte
  //    load, four loads deep per thread.  Then columns 0 and N/2 are packed as
  //    z0 + i zN/2 in column 0.
  constexpr int F2 = F / 2;  // bin pairs (F is even)
  if (!first) {
    const float4 *src = reinterpret_cast<const float4 *>(Wk);
    float4 *dst = reinterpret_cast<float4 *>(tile);
    for (int c = threadIdx.x; c < F2; c += NT) cp_async16(dst + c, src + c);
    cp_async_wait_all();
  }
  __syncthreads();
  {
    const float4 *D4 = reinterpret_cast<const float4 *>(Dk);
    const float4 *R4 = reinterpret_cast<const float4 *>(rr);
    float4 *Z4 = reinterpret_cast<float4 *>(Zk);
    float4 *T4 = reinterpret_cast<float4 *>(tile);
    constexpr int U = 4;
    for (int c0 = threadIdx.x; c0 < F2; c0 += U * NT) {
      float4 dv[U], rv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int c = c0 + u * NT;
        if (c < F2) {
          dv[u] = D4[c];
          rv[u] = R4[c];
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int c = c0 + u * NT;
        if (c >= F2) break;
        float2 z0 = cconjmul(make_float2(dv[u].x, dv[u].y), make_float2(rv[u].x, rv[u].y));
        float2 z1 = cconjmul(make_float2(dv[u].z, dv[u].w), make_float2(rv[u].z, rv[u].w));
        if (!first) {
          const float4 w = T4[c];
          z0 = cadd(z0, make_float2(w.x, w.y));
          z1 = cadd(z1, make_float2(w.z, w.w));
        }
        const float4 zz = make_float4(z0.x, z0.y, z1.x, z1.y);
        if (store_last) Z4[c] = zz;
        T4[c] = zz;
      }
    }
  }
  __syncthreads();
  for (int k1 = threadIdx.x; k1 < N; k1 += NT) {
    const float2 z0 = tile[k1 * NH], zh = tile[k1 * NH + H];
    tile[k1 * NH] = make_float2(z0.x - zh.y, z0.y + zh.x);  // z0 + i zN/2
  }
  __syncthreads();

  // 2. Inverse transforms along k1 (length N) of the N/2 columns.
  half_cols<N, true>(tile, s_tw);

  // 3. Per row, the half-length spectrum of the packed real row.
  for (int q = threadIdx.x; q < N * Q; q += NT) {
    const int n1 = q / Q, kk = q - n1 * Q;
    float2 *row = tile + n1 * NH;
    if (kk == 0) {
      const float2 c = row[0];  // (X[0], X[N/2]), both real
      row[0] = make_float2(c.x + c.y, c.x - c.y);
    } else {
      const int kq = H - kk;
      const float2 a = row[kk], c = row[kq];
      const float2 wa = make_float2(s_tw[kk].x, -s_tw[kk].y);  // W_N^-k
      const float2 wc = make_float2(s_tw[kq].x, -s_tw[kq].y);
      // H[k] = (a + conj c) + i W^-k (a - conj c)
      const float2 da = cmul(wa, make_float2(a.x - c.x, a.y + c.y));
      row[kk] = make_float2(a.x + c.x - da.y, a.y - c.y + da.x);
      if (kq != kk) {
        const float2 dc = cmul(wc, make_float2(c.x - a.x, c.y + a.y));
        row[kq] = make_float2(c.x + a.x - dc.y, c.y - a.y + dc.x);
      }
    }
  }
  __syncthreads();

  // 4. Inverse transforms of the packed rows (length N/2): P (z[2m] + i z[2m+1]).
  half_rows<N, true>(tile, s_tw);

  // 5. Spatial step on groups of four pixels 4j .. 4j+3 of row n1 (tile
  //    elements 2j, 2j+1): U = S(Z + Gamma), Gamma += Z - U, W = U - Gamma.
  //    Gamma (and, for the serving residual, the previous U) are read four
  //    16-byte loads deep per thread before use.
  const float invP = 1.0f / (float)P;
  float *Gk = it.Gam + ((size_t)slot * K + k) * P;
  float *Uk = b.u[img] ? b.u[img] + (size_t)k * P : nullptr;
  const bool resid = it.serve && store_last;
  const bool wantu = (store_last || store_prev) && Uk;
  float acc[kResidTerms] = {0.f, 0.f, 0.f, 0.f, 0.f};
  {
    constexpr int Q4 = N * N / 4, J = N / 4, U = 4;
    float4 *G4 = reinterpret_cast<float4 *>(Gk);
    float4 *U4 = reinterpret_cast<float4 *>(Uk);
    for (int q0 = threadIdx.x; q0 < Q4; q0 += U * NT) {
      float4 gv[U], pv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int q = q0 + u * NT;
        gv[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        pv[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (q < Q4) {
          if (!first) gv[u] = G4[q];
          if (resid && !first && Uk) pv[u] = U4[q];
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int q = q0 + u * NT;
        if (q >= Q4) break;
        const int n1 = q / J, j = q - n1 * J;
        float2 *tp = tile + n1 * NH + 2 * j;
        const float2 c0 = tp[0], c1 = tp[1];
        const float z[4] = {c0.x * invP, c0.y * invP, c1.x * invP, c1.y * invP};
        const float g[4] = {gv[u].x, gv[u].y, gv[u].z, gv[u].w};
        const float pu[4] = {pv[u].x, pv[u].y, pv[u].z, pv[u].w};
        float un[4], gn[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float v = z[e] + g[e];
          un[e] = soft_threshold(v, it.thr);
          gn[e] = v - un[e];
          if (resid) {
            acc[0] += (z[e] - un[e]) * (z[e] - un[e]);
            acc[1] += z[e] * z[e];
            acc[2] += un[e] * un[e];
            acc[3] += (un[e] - pu[e]) * (un[e] - pu[e]);
            acc[4] += gn[e] * gn[e];
          }
        }
        G4[q] = make_float4(gn[0], gn[1], gn[2], gn[3]);
        if (wantu) U4[q] = make_float4(un[0], un[1], un[2], un[3]);
        if (!skip_fwd) {
          tp[0] = make_float2(un[0] - gn[0], un[1] - gn[1]);
          tp[1] = make_float2(un[2] - gn[2], un[3] - gn[3]);
        }
      }
    }
  }
  if (resid) block_sum_terms(acc, it.resid + ((size_t)slot * K + k) * kResidTerms);
  if (skip_fwd) return;
  __syncthreads();

  // 6. Forward transforms of the packed rows h[m] = w[2m] + i w[2m+1].
  half_rows<N, false>(tile, s_tw);

  // 7. Split each row's H into the half spectrum X[0..N/2] of its real row;
  //    X[0] and X[N/2] are real and stay packed in element 0.
  for (int q = threadIdx.x; q < N * Q; q += NT) {
    const int n1 = q / Q, kk = q - n1 * Q;
    float2 *row = tile + n1 * NH;
    if (kk == 0) {
      const float2 h = row[0];
      row[0] = make_float2(h.x + h.y, h.x - h.y);  // (X[0], X[N/2])
    } else {
      const int kq = H - kk;
      const float2 a = row[kk], c = row[kq];
      // X[k] = (a + conj c) / 2 + W^k (a - conj c) / (2i)
      const float2 ea = cmul(s_tw[kk], make_float2(a.y + c.y, c.x - a.x));  // W^k (a - conj c) / i
      row[kk] = make_float2(0.5f * (a.x + c.x + ea.x), 0.5f * (a.y - c.y + ea.y));
      if (kq != kk) {
        const float2 ec = cmul(s_tw[kq], make_float2(c.y + a.y, a.x - c.x));
        row[kq] = make_float2(0.5f * (c.x + a.x + ec.x), 0.5f * (c.y - a.y + ec.y));
      }
    }
  }
  __syncthreads();

  // 8. Forward transforms along n1 of the N/2 columns.
  half_cols<N, false>(tile, s_tw);

  // 9. W^ to global memory; columns 0 and N/2 unpacked from element 0:
  //    C = X0^ + i XN/2^ with both columns Hermitian in k1.
  for (int p = threadIdx.x; p < F; p += NT) {
    const int k1 = p / NH, k2 = p - k1 * NH;
    float2 v;
    if (k2 == 0 || k2 == H) {
      const float2 c = tile[k1 * NH], cm = tile[((N - k1) & (N - 1)) * NH];
      v = k2 == 0 ? make_float2(0.5f * (c.x + cm.x), 0.5f * (c.y - cm.y))
                  : make_float2(0.5f * (c.y + cm.y), -0.5f * (c.x - cm.x));
    } else {
      v = tile[p];
    }
    Wk[p] = v;
  }
}

}  // namespace ocsc
