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

// r_p = (x~(p) - sum_k D~_k(p) W^_k(p)) / (rho + |d_p|^2) for the 64 bins
// pb * 64 .. of image img (F is even); 256 threads as (32 bin pairs) x
// (8 filter lanes): lane ty sums the filters k = ty, ty + 8, ... of two
// adjacent bins from 16-byte loads, and the lanes' sums are added in order.
constexpr int kResidBins = 64;

__device__ __forceinline__ void code_resid_body(int K, int F, float rho, int first, int serve, const ImgBatch &b,
                                                const float2 *__restrict__ Dh, const float *__restrict__ dn,
                                                const float2 *__restrict__ xh, const float2 *__restrict__ What,
                                                float2 *__restrict__ r, int pb, int img, int tx, int ty) {
  __shared__ float4 part[8][33];
  const int F2 = F / 2, q = pb * 32 + tx;  // bins 2q, 2q + 1
  const int slot = b.slot[img];
  const bool is_first = serve ? b.iter[img] == 0 : first != 0;
  float2 s0 = make_float2(0.f, 0.f), s1 = make_float2(0.f, 0.f);
  if (!is_first && q < F2) {
    const float4 *w = reinterpret_cast<const float4 *>(What + (size_t)slot * K * F);
    const float4 *D = reinterpret_cast<const float4 *>(Dh);
    constexpr int U = 4;  // loads in flight per operand
    for (int k0 = ty; k0 < K; k0 += 8 * U) {
      float4 d[U], v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int k = k0 + 8 * u;
        if (k < K) {
          d[u] = D[(size_t)k * F2 + q];
          v[u] = w[(size_t)k * F2 + q];
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (k0 + 8 * u >= K) break;
        s0 = cadd(s0, cmul(make_float2(d[u].x, d[u].y), make_float2(v[u].x, v[u].y)));
        s1 = cadd(s1, cmul(make_float2(d[u].z, d[u].w), make_float2(v[u].z, v[u].w)));
      }
    }
  }
  part[ty][tx] = make_float4(s0.x, s0.y, s1.x, s1.y);
  __syncthreads();
  if (ty == 0 && q < F2) {
    float4 t = part[0][tx];
#pragma unroll
    for (int y = 1; y < 8; ++y) {
      const float4 u = part[y][tx];
      t = make_float4(t.x + u.x, t.y + u.y, t.z + u.z, t.w + u.w);
    }
    const float4 x = reinterpret_cast<const float4 *>(xh + (size_t)slot * F)[q];
    const float2 dd = reinterpret_cast<const float2 *>(dn)[q];
    const float i0 = 1.0f / (rho + dd.x), i1 = 1.0f / (rho + dd.y);
    reinterpret_cast<float4 *>(r + (size_t)slot * F)[q] =
        make_float4((x.x - t.x) * i0, (x.y - t.y) * i0, (x.z - t.z) * i1, (x.w - t.w) * i1);
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
// The split of a packed real row and its inverse (the plane kernel's
// header explains them): with a = X[k], c = X[N/2 - k] of a real row's half
// spectrum, the half-length spectrum of h[m] = x[2m] + i x[2m+1] is
// H[k] = (a + conj c) + i W_N^-k (a - conj c); with a = H[k], c = H[N/2 - k],
// X[k] = (a + conj c) / 2 + W_N^k (a - conj c) / (2i).
__device__ __forceinline__ float2 split_c2r(float2 a, float2 c, const float2 *s_tw, int k) {
  const float2 w = make_float2(s_tw[k].x, -s_tw[k].y);
  const float2 d = cmul(w, make_float2(a.x - c.x, a.y + c.y));
  return make_float2(a.x + c.x - d.y, a.y - c.y + d.x);
}
__device__ __forceinline__ float2 split_r2c(float2 a, float2 c, const float2 *s_tw, int k) {
  const float2 e = cmul(s_tw[k], make_float2(a.y + c.y, c.x - a.x));
  return make_float2(0.5f * (a.x + c.x + e.x), 0.5f * (a.y - c.y + e.y));
}

// First inverse column pass (radix C0, no twiddles) over the Z~ tile, with
// columns 0 and N/2 packed as z0 + i zN/2 where the thread of column 0 loads
// them.
template <int N, int NT>
__device__ __forceinline__ void cols_inv_first_packed(float2 *tile) {
  using P = HalfPlan<N>;
  constexpr int NH = N / 2 + 1, H = N / 2, R = P::C0, LINES = N / 2, STEP = N / R;
  constexpr int G = LINES * STEP, PER = G / NT;
  static_assert(G % NT == 0, "threads must divide the butterfly groups");
  float2 v[PER][R];
#pragma unroll
  for (int gi = 0; gi < PER; ++gi) {
    const int g = threadIdx.x + gi * NT, c = g % LINES, j = g / LINES;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int p = (j + r * STEP) * NH + c;
      float2 z = tile[p];
      if (c == 0) {
        const float2 zh = tile[p + H];
        z = make_float2(z.x - zh.y, z.y + zh.x);
      }
      v[gi][r] = z;
    }
    RegDFT<R, true>::run(v[gi]);
  }
  __syncthreads();
#pragma unroll
  for (int gi = 0; gi < PER; ++gi) {
    const int g = threadIdx.x + gi * NT, c = g % LINES, j = g / LINES;
#pragma unroll
    for (int r = 0; r < R; ++r) tile[(j * R + r) * NH + c] = v[gi][r];
  }
  __syncthreads();
}

// N = 128: rows of 64 points by two radix-8 passes.  A thread takes one row
// and whole mirror pairs of its eight butterfly groups (group j holds
// elements j + 8r; element k's mirror 64 - k is group 8 - j, element 7 - r,
// and for group 0 element 8 - r, element 0 the packed pair): pair P = 0 is
// groups (0, 4), each its own mirror, and pairs 1, 2, 3 are (P, 8 - P).  With
// NT threads a CTA has NT / 128 threads per row and each takes 512 / NT
// pairs: threads 128 h .. 128 h + 127 pairs h (512 / NT) onwards.  The first
// inverse pass then applies the c2r split where it loads, and the last
// forward pass the r2c split where it stores.
__device__ __forceinline__ void mirror_pair(int P, int &ga, int &gb) {
  ga = P == 0 ? 0 : P;
  gb = P == 0 ? 4 : 8 - P;
}
template <bool FWD>
__device__ __forceinline__ float2 split_dir(float2 a, float2 c, const float2 *s_tw, int k) {
  return FWD ? split_r2c(a, c, s_tw, k) : split_c2r(a, c, s_tw, k);
}

// The split of two groups a (group ga) and b (group 8 - ga) that mirror each
// other; with self set, a and b are groups 0 and 4, each its own mirror.
template <bool FWD>
__device__ __forceinline__ void rows128_split_pair(float2 (&a)[8], float2 (&b)[8], int ga, int gb, bool self,
                                                   const float2 *s_tw) {
  float2 na[8], nb[8];
  if (self) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      na[r] = r == 0 ? make_float2(a[0].x + a[0].y, a[0].x - a[0].y)  // (X[0], X[N/2]) <-> H[0]
                     : split_dir<FWD>(a[r], a[8 - r], s_tw, 8 * r);
      nb[r] = split_dir<FWD>(b[r], b[7 - r], s_tw, 4 + 8 * r);
    }
  } else {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      na[r] = split_dir<FWD>(a[r], b[7 - r], s_tw, ga + 8 * r);
      nb[r] = split_dir<FWD>(b[r], a[7 - r], s_tw, gb + 8 * r);
    }
  }
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    a[r] = na[r];
    b[r] = nb[r];
  }
}

// First inverse row pass (radix 8, no twiddles) with the c2r split folded in.
template <int NT>
__device__ __forceinline__ void rows128_inv_first(float2 *tile, const float2 *s_tw) {
  constexpr int NH = 65, NPAIR = 512 / NT;
  const int row = threadIdx.x & 127, P0 = (threadIdx.x >> 7) * NPAIR;
  float2 *rw = tile + row * NH;
  float2 a[NPAIR][8], b[NPAIR][8];
#pragma unroll
  for (int pp = 0; pp < NPAIR; ++pp) {
    int ga, gb;
    mirror_pair(P0 + pp, ga, gb);
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      a[pp][r] = rw[ga + 8 * r];
      b[pp][r] = rw[gb + 8 * r];
    }
    rows128_split_pair<false>(a[pp], b[pp], ga, gb, P0 + pp == 0, s_tw);
    RegDFT<8, true>::run(a[pp]);
    RegDFT<8, true>::run(b[pp]);
  }
  __syncthreads();
#pragma unroll
  for (int pp = 0; pp < NPAIR; ++pp) {
    int ga, gb;
    mirror_pair(P0 + pp, ga, gb);
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      rw[8 * ga + r] = a[pp][r];
      rw[8 * gb + r] = b[pp][r];
    }
  }
  __syncthreads();
}

// Second forward row pass (twiddles W_64^(n j)) with the r2c split folded in.
// Group j takes Y_n[j] (n = 0 .. 7), which the first pass left at 8j + n,
// and yields X[j + 8k], stored at 8j + k: the packed rows leave this pass with
// element k of the half spectrum at place 8 (k mod 8) + k / 8 (place 0 still
// holds (X[0], X[N/2])).  Each group's outputs land on its own inputs' places,
// so no barrier separates the loads from the stores and each mirror pair is
// finished before the next is loaded.
template <int NT>
__device__ __forceinline__ void rows128_fwd_last(float2 *tile, const float2 *s_tw) {
  constexpr int NH = 65, NPAIR = 512 / NT;
  const int row = threadIdx.x & 127, P0 = (threadIdx.x >> 7) * NPAIR;
  float2 *rw = tile + row * NH;
#pragma unroll
  for (int pp = 0; pp < NPAIR; ++pp) {
    int ga, gb;
    mirror_pair(P0 + pp, ga, gb);
    float2 a[8], b[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      a[r] = rw[8 * ga + r];
      b[r] = rw[8 * gb + r];
    }
#pragma unroll
    for (int r = 1; r < 8; ++r) {  // W_64^(r j) = W_128^(2 r j)
      a[r] = cmul(a[r], s_tw[((r * ga) % 64) * 2]);
      b[r] = cmul(b[r], s_tw[((r * gb) % 64) * 2]);
    }
    RegDFT<8, false>::run(a);
    RegDFT<8, false>::run(b);
    rows128_split_pair<true>(a, b, ga, gb, P0 + pp == 0, s_tw);
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      rw[8 * ga + r] = a[r];
      rw[8 * gb + r] = b[r];
    }
  }
  __syncthreads();
}

// The spatial step of one pixel: u = S(z + gamma), gamma' = z + gamma - u;
// returns u - gamma' (the next iteration's w) and, for the serving residual,
// adds the five terms of the stopping test (pu: the previous u).
__device__ __forceinline__ float spatial_px(float z, float &g, float pu, float thr, bool resid,
                                            float (&acc)[kResidTerms], float &u) {
  const float v = z + g;
  u = soft_threshold(v, thr);
  g = v - u;
  if (resid) {
    acc[0] += (z - u) * (z - u);
    acc[1] += z * z;
    acc[2] += u * u;
    acc[3] += (u - pu) * (u - pu);
    acc[4] += g * g;
  }
  return u - g;
}

// N = 128: the second inverse row pass (radix 8, twiddles W_64^-(r j)), the
// spatial step and the first forward row pass (radix 8, no twiddles) on one
// thread's registers, in place.  Thread t takes row t mod 128 and the group
// pairs (2P, 2P + 1), P = (t / 128) (512 / NT) .. (one or two pairs), one pair
// at a time; the inverse pass leaves h[m] = (z[2m], z[2m+1]), m = j + 8r, in
// slot r of group j, so slot r of the pair is pixels 16r + 4P .. 16r + 4P + 3
// of the row.  The forward pass transforms the same group (elements j + 8 n1,
// over n1) and writes its outputs Y_j[k1] back to the places j + 8 k1 it read,
// leaving the transposition of the 8 x 8 split to the next pass.  Gamma is
// kept in the matching order, pixels 16r + 4P .. + 3 of row n1 at float4
// (4r + P) 128 + n1, so that a warp's 16-byte loads are 512 contiguous bytes
// (pixel 8c + e of row n1 at ((2c + e / 4) 128 + n1) 4 + e % 4); U keeps the
// image layout.  With 256 threads a pair's eight Gamma loads are issued before
// its inverse pass.  Returns after the spatial step when skip_fwd is set.
template <int NT>
__device__ __forceinline__ void rows128_spatial(float2 *tile, const float2 *s_tw, float *__restrict__ Gk,
                                                float *__restrict__ Uk, float thr, bool first, bool resid,
                                                bool wantu, bool skip_fwd, float (&acc)[kResidTerms]) {
  constexpr int NH = 65, NPAIR = 512 / NT;
  constexpr bool HOIST = NT == 256;
  constexpr float invP = 1.0f / (128.0f * 128.0f);
  const int row = threadIdx.x & 127, P0 = (threadIdx.x >> 7) * NPAIR;
  float2 *rw = tile + row * NH;
  float4 *G4 = reinterpret_cast<float4 *>(Gk);
  float4 *U4 = reinterpret_cast<float4 *>(Uk);
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int pp = 0; pp < NPAIR; ++pp) {
    const int P = P0 + pp, ja = 2 * P, jb = ja + 1;
    float4 g[HOIST ? 8 : 1];
    if constexpr (HOIST) {
#pragma unroll
      for (int r = 0; r < 8; ++r) g[r] = first ? zero : G4[(4 * r + P) * 128 + row];
    }
    float2 a[8], b[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      a[r] = rw[ja + 8 * r];
      b[r] = rw[jb + 8 * r];
    }
#pragma unroll
    for (int r = 1; r < 8; ++r) {
      a[r] = cmul(a[r], cconj(s_tw[((r * ja) % 64) * 2]));
      b[r] = cmul(b[r], cconj(s_tw[((r * jb) % 64) * 2]));
    }
    RegDFT<8, true>::run(a);
    RegDFT<8, true>::run(b);
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int gi = (4 * r + P) * 128 + row;  // pixels 16r + 4P .. + 3
      const int ui = row * 32 + 4 * r + P;
      float4 gr;
      if constexpr (HOIST) gr = g[r];
      else gr = first ? zero : G4[gi];
      const float4 pu = resid && !first && Uk ? U4[ui] : zero;
      float4 u;
      a[r] = make_float2(spatial_px(a[r].x * invP, gr.x, pu.x, thr, resid, acc, u.x),
                         spatial_px(a[r].y * invP, gr.y, pu.y, thr, resid, acc, u.y));
      b[r] = make_float2(spatial_px(b[r].x * invP, gr.z, pu.z, thr, resid, acc, u.z),
                         spatial_px(b[r].y * invP, gr.w, pu.w, thr, resid, acc, u.w));
      G4[gi] = gr;
      if (wantu) U4[ui] = u;
    }
    if (skip_fwd) continue;
    RegDFT<8, false>::run(a);
    RegDFT<8, false>::run(b);
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      rw[ja + 8 * r] = a[r];
      rw[jb + 8 * r] = b[r];
    }
  }
  if (!skip_fwd) __syncthreads();
}

// N = 128: the last forward column pass (radix 8 after radix 16, twiddles
// W_128^(r j)) stores W^ straight from registers.  Group j of a column holds
// rows j + 16r, in natural order, and its mirror rows 128 - k1 are group
// 16 - j, element 7 - r (group 0: element 8 - r).  The eight group pairs
// are (0, 8), (4, 12) and, for q = 1 .. 3, (q, 16 - q), (8 - q, 8 + q): pair
// index 2q + pr, and with NT threads threads 64i .. 64i + 63 take the 512 / NT
// pairs from i (512 / NT) on, so the thread of column 0, which unpacks X0^ and
// XN/2^ from the packed column, holds every row's mirror.  The pass is in
// place and the last, so each pair is transformed and stored before the next
// is loaded.
__device__ __forceinline__ void unpack_cols0(float2 *__restrict__ Wk, float2 c, float2 cm, int k1) {
  constexpr int NH = 65, H = 64;
  Wk[k1 * NH] = make_float2(0.5f * (c.x + cm.x), 0.5f * (c.y - cm.y));
  Wk[k1 * NH + H] = make_float2(0.5f * (c.y + cm.y), -0.5f * (c.x - cm.x));
}

template <int NT>
__device__ __forceinline__ void cols128_fwd_last_store(const float2 *tile, const float2 *s_tw,
                                                       float2 *__restrict__ Wk) {
  constexpr int NH = 65, S = 16, NPAIR = 512 / NT;
  const int c = threadIdx.x & 63;
#pragma unroll
  for (int pp = 0; pp < NPAIR; ++pp) {  // the mirror pairs, one at a time
    const int idx = (threadIdx.x >> 6) * NPAIR + pp, q = idx >> 1, pr = idx & 1;
    const int ja = pr == 0 ? q : (q == 0 ? 4 : 8 - q);
    const int jb = pr == 0 ? (q == 0 ? 8 : 16 - q) : (q == 0 ? 12 : 8 + q);
    float2 a[8], b[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      a[r] = tile[(ja + S * r) * NH + c];
      b[r] = tile[(jb + S * r) * NH + c];
    }
#pragma unroll
    for (int r = 1; r < 8; ++r) {
      a[r] = cmul(a[r], s_tw[(r * ja) % 128]);
      b[r] = cmul(b[r], s_tw[(r * jb) % 128]);
    }
    RegDFT<8, false>::run(a);
    RegDFT<8, false>::run(b);
    if (c != 0) {
      const int k2 = (c >> 3) + 8 * (c & 7);  // the tile's columns are in the rows' pass order
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        Wk[(ja + S * r) * NH + k2] = a[r];
        Wk[(jb + S * r) * NH + k2] = b[r];
      }
    } else if (pr == 0 && q == 0) {  // groups 0 and 8, each its own mirror
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        unpack_cols0(Wk, a[r], a[(8 - r) & 7], S * r);
        unpack_cols0(Wk, b[r], b[7 - r], 8 + S * r);
      }
    } else {
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        unpack_cols0(Wk, a[r], b[7 - r], ja + S * r);
        unpack_cols0(Wk, b[r], a[7 - r], jb + S * r);
      }
    }
  }
}

// L2 prefetch of the W^ and Gamma that the plane step of (filter k, image
// img) will read; nothing on its first iteration (neither is read then).
template <int N, bool SERVE>
__device__ __forceinline__ void plane_prefetch(const CodeIter &it, const ImgBatch &b, int k, int img) {
  constexpr int F = N * (N / 2 + 1), P = N * N, kPre = 16384;
  constexpr int NW = (F * 8 + kPre - 1) / kPre, NG = P * 4 / kPre;
  const int t = threadIdx.x;
  if (t >= NW + NG) return;
  const bool first = SERVE ? b.iter[img] == 0 : it.first != 0;
  if (first) return;
  const size_t unit = (size_t)b.slot[img] * it.K + k;
  if (t < NW) {
    const int bytes = min(kPre, F * 8 - t * kPre);
    prefetch_l2(reinterpret_cast<const char *>(it.What + unit * F) + (size_t)t * kPre, (unsigned)bytes);
  } else {
    prefetch_l2(reinterpret_cast<const char *>(it.Gam + unit * P) + (size_t)(t - NW) * kPre, kPre);
  }
}

// SERVE: the serving form (per-slot iteration counters, the stopping test's
// residual terms every `check` iterations); the batch form has it.serve = 0.
// NT: threads of the CTA (256; N = 128 also 512).  pre: the linear unit
// (img * K + k) whose data to prefetch, or -1.  A persistent caller passes
// its own tile and twiddles (tile_in, s_tw_in: the twiddles already loaded),
// staged = true when this unit's W^ copies into tile_in were committed by the
// previous unit, and next_W / next_tile to have this unit commit the next
// unit's W^ copies (they stay in flight through this unit's work).
template <int N, bool SERVE, int NT = HalfPlan<N>::NT>
__device__ __forceinline__ void code_plane_body(const CodeIter &it, const ImgBatch &b, const float2 *__restrict__ tw,
                                                int k, int img, float4 *hsmem, int pre = -1,
                                                float2 *tile_in = nullptr, float2 *s_tw_in = nullptr,
                                                bool staged = false, const float2 *next_W = nullptr,
                                                float2 *next_tile = nullptr) {
  static_assert(NT == 256 || (N == 128 && NT == 512), "CTA size");
  constexpr int NH = N / 2 + 1, H = N / 2, Q = H / 2 + 1;
  constexpr int F = N * NH, P = N * N;
  float2 *tile = tile_in ? tile_in : reinterpret_cast<float2 *>(hsmem);  // [N][NH]
  float2 *s_tw = s_tw_in ? s_tw_in : tile + F;                           // [N]
  const int K = it.K;
  const int slot = b.slot[img];
  const int t = b.iter[img];
  const bool first = SERVE ? t == 0 : it.first != 0;
  const bool store_last = SERVE ? (t + 1) % it.check == 0 : it.last != 0;
  const bool store_prev = SERVE && (t + 2) % it.check == 0;
  const bool skip_fwd = !SERVE && it.last;
  const float2 *Dk = it.Dh + (size_t)k * F;
  const float2 *rr = it.r + (size_t)slot * F;
  float2 *Wk = it.What + ((size_t)slot * K + k) * F;
  float2 *Zk = it.Zp + ((size_t)slot * K + k) * F;
  float *Gk = it.Gam + ((size_t)slot * K + k) * P;
  // Gamma is first needed after the inverse transforms: ask L2 for it now so
  // that its DRAM reads overlap them (16 KB per request); and for the W^ and
  // Gamma of the unit `pre`, which runs about when this one ends.
  constexpr int kPre = 16384, NPRE = P * 4 / kPre;
  if (!first && threadIdx.x < NPRE) prefetch_l2(reinterpret_cast<const char *>(Gk) + threadIdx.x * kPre, kPre);
  if (pre >= 0) plane_prefetch<N, SERVE>(it, b, pre % K, pre / K);
  if (!s_tw_in) load_twiddles<N, NT>(s_tw, tw);

  // 1. Z~-step z = w^ + conj(d) r_p over the half spectrum.  W^ of this
  //    filter comes into the tile (its global layout) by 16-byte asynchronous
  //    copies, all in flight at once; D~ and r are read two bins per 16-byte
  //    load, four loads deep per thread.
  constexpr int F2 = F / 2;  // bin pairs (F is even)
  if (!first && !staged) {
    const float4 *src = reinterpret_cast<const float4 *>(Wk);
    float4 *dst = reinterpret_cast<float4 *>(tile);
    for (int c = threadIdx.x; c < F2; c += NT) cp_async16(dst + c, src + c);
    cp_async_commit();
  }
  if (next_W) {
    const float4 *src = reinterpret_cast<const float4 *>(next_W);
    float4 *dst = reinterpret_cast<float4 *>(next_tile);
    for (int c = threadIdx.x; c < F2; c += NT) cp_async16(dst + c, src + c);
    cp_async_commit();
  }
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
      if (c0 == (int)threadIdx.x) {  // the first loads are in flight with the copies of W^
        if (next_W) cp_async_wait<1>();  // the next unit's copies stay in flight
        else cp_async_wait<0>();
        __syncthreads();
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

  // 2. Inverse transforms along k1 (length N) of the N/2 columns, columns 0
  //    and N/2 packed into one by the first pass.
  cols_inv_first_packed<N, NT>(tile);
  half_pass<N, N / 2, HalfPlan<N>::C1, HalfPlan<N>::C0, true, 1, NH, NT, 1>(tile, s_tw);

  float *Uk = b.u[img] ? b.u[img] + (size_t)k * P : nullptr;
  const bool resid = SERVE && store_last;
  const bool wantu = (store_last || store_prev) && Uk;
  float acc[kResidTerms] = {0.f, 0.f, 0.f, 0.f, 0.f};

  if constexpr (N == 128) {
    // 3-7. The c2r split with the first inverse row pass; the second inverse
    //    row pass, the spatial step and the first forward row pass on
    //    registers; the r2c split with the second forward row pass.
    rows128_inv_first<NT>(tile, s_tw);
    rows128_spatial<NT>(tile, s_tw, Gk, Uk, it.thr, first, resid, wantu, skip_fwd, acc);
    if (resid) block_sum_terms(acc, it.resid + ((size_t)slot * K + k) * kResidTerms);
    if (skip_fwd) return;
    rows128_fwd_last<NT>(tile, s_tw);
    // 8-9. Forward transforms along n1, the last pass storing W^.
    half_pass<128, 64, 16, 1, false, 1, NH, NT, 1>(tile, s_tw);
    cols128_fwd_last_store<NT>(tile, s_tw, Wk);
    return;
  }

  // 3-4. Per row, the half-length spectrum of the packed real row, then its
  //    inverse transform (length N/2): P (z[2m] + i z[2m+1]).
  for (int q = threadIdx.x; q < N * Q; q += NT) {
    const int n1 = q / Q, kk = q - n1 * Q;
    float2 *row = tile + n1 * NH;
    if (kk == 0) {
      const float2 c = row[0];  // (X[0], X[N/2]), both real
      row[0] = make_float2(c.x + c.y, c.x - c.y);
    } else {
      const int kq = H - kk;
      const float2 a = row[kk], c = row[kq];
      row[kk] = split_c2r(a, c, s_tw, kk);
      if (kq != kk) row[kq] = split_c2r(c, a, s_tw, kq);
    }
  }
  __syncthreads();
  half_rows<N, true>(tile, s_tw);

  // 5. Spatial step on groups of four pixels 4j .. 4j+3 of row n1 (tile
  //    elements 2j, 2j+1): U = S(Z + Gamma), Gamma += Z - U, W = U - Gamma.
  //    Gamma (and, for the serving residual, the previous U) are read four
  //    16-byte loads deep per thread before use.
  const float invP = 1.0f / (float)P;
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
        float4 g = gv[u], un;
        const float2 w0 = make_float2(spatial_px(c0.x * invP, g.x, pv[u].x, it.thr, resid, acc, un.x),
                                      spatial_px(c0.y * invP, g.y, pv[u].y, it.thr, resid, acc, un.y));
        const float2 w1 = make_float2(spatial_px(c1.x * invP, g.z, pv[u].z, it.thr, resid, acc, un.z),
                                      spatial_px(c1.y * invP, g.w, pv[u].w, it.thr, resid, acc, un.w));
        G4[q] = g;
        if (wantu) U4[q] = un;
        if (!skip_fwd) {
          tp[0] = w0;
          tp[1] = w1;
        }
      }
    }
  }
  if (resid) block_sum_terms(acc, it.resid + ((size_t)slot * K + k) * kResidTerms);
  if (skip_fwd) return;
  __syncthreads();

  // 6-7. Forward transforms of the packed rows h[m] = w[2m] + i w[2m+1], then
  //    the split of each row's H into the half spectrum X[0..N/2] of its real
  //    row; X[0] and X[N/2] are real and stay packed in element 0.
  half_rows<N, false>(tile, s_tw);
  for (int q = threadIdx.x; q < N * Q; q += NT) {
    const int n1 = q / Q, kk = q - n1 * Q;
    float2 *row = tile + n1 * NH;
    if (kk == 0) {
      const float2 h = row[0];
      row[0] = make_float2(h.x + h.y, h.x - h.y);  // (X[0], X[N/2])
    } else {
      const int kq = H - kk;
      const float2 a = row[kk], c = row[kq];
      row[kk] = split_r2c(a, c, s_tw, kk);
      if (kq != kk) row[kq] = split_r2c(c, a, s_tw, kq);
    }
  }
  __syncthreads();

  // 8-9. Forward transforms along n1 of the N/2 columns, and W^ to global
  //    memory with columns 0 and N/2 unpacked from element 0 (C = X0^ + i XN/2^,
  //    both columns Hermitian in k1).
  half_cols<N, false>(tile, s_tw);
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
