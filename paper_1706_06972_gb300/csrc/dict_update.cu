// Online dictionary step: history fold (Sec. III-B, eqs. (A_update),
// (B_update)) and DictOCSC (Algorithm 2).
//
// Per frequency p the history is A^p = mean conj(z) z^T (K x K Hermitian, kept
// as a packed lower triangle in FP32) and b^p = mean x~(p) conj(z).  The D-row
// solve of eq. (sub_d_sol) is d = (w A^p + rho I)^-1 (w b^p + rho (v^ - theta^)).
// Its matrix is fixed during the Jd ADMM iterations, so it is factored once per
// update: fold_factor folds the pending codes into A and b, forms w A + rho I in
// double-float (two FP32 words, about 48 bits; dfloat.cuh) in shared memory,
// factors it by Cholesky in that arithmetic (L) on the FP32 pipe, and alongside
// it computes X = L^-1 in FP32 and y = L^-1 (w b) from the same sweep.  Each ADMM
// iteration then applies d = X^H (y + rho X (v^ - theta^)) in FP32 (dstep),
// forms the V update of Proposition 2 from a pruned inverse DFT restricted to
// the M x M support (vstep_cols, vstep_project, vstep_spectrum), and updates
// the scaled dual.
#include "common.cuh"
#include "dfloat.cuh"
#include "launch.h"

namespace ocsc {

constexpr int kFoldChunk = 16;  // samples staged in shared memory at once
constexpr int kPanel = 4;       // columns per Cholesky panel

// Factor panel pb (columns j0 .. j0+nb-1, all rows below) by one warp: pivot,
// scaling of the column (kept in registers and as an FP32 copy in Lb), y, and
// the update of the panel's later columns; lanes take rows j+1+lane+32m.
__device__ __forceinline__ void fold_panel(float4 *M, float4 *y, float2 *invf, float2 *Lb, int K, int pb,
                                           int lane, int *err, float rho_fb) {
  const int j0 = pb * kPanel, nb = min(kPanel, K - j0);
  float2 *Lq = Lb + (pb % 3) * kPanel * K;
  for (int q = 0; q < nb; ++q) {
    const int mrows = (K - j0 - q - 1 + 31) / 32;  // row slots j+1+lane+32m below K
    const int j = j0 + q, oj = tri_off(j, K);
    const float4 d = M[oj];
    float2 pv = two_sum(d.x, d.z);
    if (!(pv.x > 0.f)) {
      if (lane == 0) atomicOr(err, ERR_PIVOT);
      pv = make_float2(rho_fb, 0.f);
    }
    const float2 r = df_rsqrt(pv.x, pv.y);
    float S, E;
    df_mul(pv.x, pv.y, r.x, r.y, S, E);
    const float2 ljj = two_sum(S, E);  // L_jj = p / sqrt(p)
    float4 l[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int i = j + 1 + lane + 32 * m;
      if (m >= mrows) break;
      if (i < K) {
        l[m] = df_scale(M[oj + i - j], r);
        M[oj + i - j] = l[m];
        Lq[q * K + i] = make_float2(l[m].x, l[m].y);
      }
    }
    const float4 yj = df_scale(y[j], r);
    __syncwarp();
    if (lane == 0) {
      M[oj] = make_float4(ljj.x, 0.f, ljj.y, 0.f);
      invf[j] = r;
      y[j] = yj;
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int i = j + 1 + lane + 32 * m;
      if (m >= mrows) break;
      if (i < K) {
        float4 v = y[i];
        df_sub_lm(v, l[m], yj);
        y[i] = v;
      }
    }
    for (int qp = q + 1; qp < nb; ++qp) {
      const int jp = j0 + qp, ojp = tri_off(jp, K);
      const float4 lj = M[oj + jp - j];  // L_{jp, j}, scaled above by its row's lane
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const int i = j + 1 + lane + 32 * m;
        if (m >= mrows) break;
        if (i >= jp && i < K) {
          float4 v = M[ojp + i - jp];
          df_sub_lconjm(v, l[m], lj);
          M[ojp + i - jp] = v;
        }
      }
    }
    __syncwarp();
  }
}

// One trailing entry v - sum_q L_{ii, q} conj(L_{kk, q}) over the panel's nb
// columns (nb >= 1), in two independent chains (q even / odd) merged at the end.
__device__ __forceinline__ float4 trail_entry(float4 v, const float4 *M, const int (&cq)[kPanel], int ii,
                                              const float4 (&lk)[kPanel], int nb) {
  float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
  df_sub_lconjm(v, M[cq[0] + ii], lk[0]);
  if (nb > 1) df_neg_lconjm(w, M[cq[1] + ii], lk[1]);
  if (nb > 2) df_sub_lconjm(v, M[cq[2] + ii], lk[2]);
  if (nb > 3) df_sub_lconjm(w, M[cq[3] + ii], lk[3]);
  df_acc2(v, w);
  return v;
}

// Rank-nb update of the trailing triangle (rows / columns from j1 = j0 + nb)
// by panel columns j0 .. j0+nb-1, over rectangle rows r0, r0 + rs, ... < rend;
// the lanes of the calling warp take the entries.
// second = false: only the first part of each row (column r itself).
__device__ __forceinline__ void fold_trail(float4 *M, int K, int j0, int nb, int r0, int rs, int rend, int lane,
                                           bool second) {
  const int j1 = j0 + nb, n = K - j1;
  int cq[kPanel];  // cq[q] + ii: slot of L_{j1+ii, j0+q}
#pragma unroll
  for (int q = 0; q < kPanel; ++q) cq[q] = q < nb ? tri_off(j0 + q, K) - j0 - q + j1 : 0;
  for (int r = r0; r < rend; r += rs) {
    const int cut = n - r, len = (2 * r + 1 == n) ? cut : n + 1, kb = n - 1 - r;
    const int dsta = tri_off(j1 + r, K), dstb = tri_off(j1 + kb, K) - cut;
    float4 lka[kPanel], lkb[kPanel];
#pragma unroll
    for (int q = 0; q < kPanel; ++q) {
      lka[q] = q < nb ? M[cq[q] + r] : make_float4(0.f, 0.f, 0.f, 0.f);
      lkb[q] = q < nb ? M[cq[q] + kb] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    int c = lane;
    // Column r: entry ii = r + c; then column n-1-r: ii = c - 1.
    for (; c < cut; c += 32) {
      const int dst = dsta + c, ii = r + c;
      M[dst] = trail_entry(M[dst], M, cq, ii, lka, nb);
    }
    if (!second) continue;
    for (; c < len; c += 32) {
      const int dst = dstb + c, ii = c - 1;
      M[dst] = trail_entry(M[dst], M, cq, ii, lkb, nb);
    }
  }
}

// The same rank-nb update over the trailing entries (ii, kk) with
// o <= kk <= ii < n (local coordinates of the trailing triangle, whose first
// row and column are j1 = j0 + nb), by 2 x 2 tiles of that sub-triangle:
// tile (ti, tk), ti >= tk, holds rows o + 2 ti (+1) and columns o + 2 tk (+1),
// numbered in packed lower-triangular order (consecutive tiles: consecutive
// row tiles of one column tile, whose L values they share).  A tile loads the
// nb panel entries of its two rows
// and two columns once for its (up to) four entries, and updates the four in
// independent double-float chains.
//
// The calling warps take the tiles 32 at a time from the shared counter *ctr
// (zero on entry; lane 0 claims, the warp's lanes take consecutive tiles), so
// a warp that finishes its other work of the phase early takes more of them.
__device__ __forceinline__ void fold_trail_tiles(float4 *M, int K, int j0, int nb, int o, int *ctr) {
  const int j1 = j0 + nb, n = K - j1, m = n - o;
  if (m <= 0) return;
  const int mt = (m + 1) / 2, ntiles = mt * (mt + 1) / 2;
  int cq[kPanel];  // cq[q] + ii: slot of L_{j1+ii, j0+q}
#pragma unroll
  for (int q = 0; q < kPanel; ++q) cq[q] = q < nb ? tri_off(j0 + q, K) - j0 - q + j1 : 0;
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  const int lane = threadIdx.x & 31;
  for (;;) {
    int base = 0;
    if (lane == 0) base = atomicAdd(ctr, 32);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= ntiles) break;
    const int u = base + lane;
    if (u >= ntiles) continue;
    int ti, tk;
    tri_ij(u, mt, ti, tk);
    const int r0 = o + 2 * ti, c0 = o + 2 * tk;
    const bool r1 = r0 + 1 < n, c1 = c0 + 1 < n;
    const bool e01 = c1 && ti > tk;  // entry (r0, c0 + 1) lies below the diagonal
    float4 lr0[kPanel], lr1[kPanel], lc0[kPanel], lc1[kPanel];
#pragma unroll
    for (int q = 0; q < kPanel; ++q) {
      const bool ok = q < nb;
      lr0[q] = ok ? M[cq[q] + r0] : zero;
      lr1[q] = ok && r1 ? M[cq[q] + r0 + 1] : zero;
      lc0[q] = ok ? M[cq[q] + c0] : zero;
      lc1[q] = ok && c1 ? M[cq[q] + c0 + 1] : zero;
    }
    const int s0 = tri_off(j1 + c0, K) + r0 - c0;          // (r0, c0); (r0 + 1, c0) follows it
    const int s1 = c1 ? tri_off(j1 + c0 + 1, K) + r0 - c0 - 1 : 0;  // (r0, c0 + 1); (r0 + 1, c0 + 1) follows
    float4 v00 = M[s0];
    float4 v10 = r1 ? M[s0 + 1] : zero;
    float4 v01 = e01 ? M[s1] : zero;
    float4 v11 = r1 && c1 ? M[s1 + 1] : zero;
#pragma unroll
    for (int q = 0; q < kPanel; ++q) {
      if (q >= nb) break;
      df_sub_lconjm(v00, lr0[q], lc0[q]);
      df_sub_lconjm(v10, lr1[q], lc0[q]);
      df_sub_lconjm(v01, lr0[q], lc1[q]);
      df_sub_lconjm(v11, lr1[q], lc1[q]);
    }
    M[s0] = v00;
    if (r1) M[s0 + 1] = v10;
    if (e01) M[s1] = v01;
    if (r1 && c1) M[s1 + 1] = v11;
  }
}

// Barrier `id` (not 0, which __syncthreads uses) among `count` threads (a
// multiple of 32: whole warps), all of which execute it.
__device__ __forceinline__ void named_barrier_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Forward substitution L X = I for the pivots of panel pb (FP32, L from the
// panel's FP32 copy in Lb, 1 / L_ss from invf): for every column c <= j0 + nb
// - 1 and every pivot s of the panel, X_sc *= 1 / L_ss (X_ss = 1 / L_ss when
// c = s), then X_ic -= L_is X_sc for the rows i > s.  X_ic lives in the first
// 8 bytes of slot (i, c) of the factor's storage (XS[2 slot]).  Two steps
// over nt threads (t = 0 .. nt-1; nt a multiple of 32, all executing named
// barrier `bar` between the steps):
//   1. the panel's pivot rows s = j0 .. j0+nb-1 of every column c < j0 + nb,
//      one thread per column, in registers (X_sc *= 1 / L_ss, X_s'c -= L_s's
//      X_sc for the later pivots s' of the panel);
//   2. the rows below the panel, X_ic -= sum_q L_{i,j0+q} X_{j0+q,c}, by 2 x 2
//      tiles (row pair, column pair) of that rectangle: a tile loads the nb
//      L values of its two rows and the nb X values of its two columns once.
__device__ __forceinline__ void fold_xpanel_tiled(float2 *XS, const float2 *Lb, const float2 *invf, int K,
                                                  int pb, int t, int nt, int bar) {
  const int j0 = pb * kPanel, nb = min(kPanel, K - j0), nc = j0 + nb;
  const float2 *Lq = Lb + (pb % 3) * kPanel * K;
  const float2 zero = make_float2(0.f, 0.f);
  for (int c = t; c < nc; c += nt) {
    const int base = tri_off(c, K) - c;  // XS[2 (base + i)]: slot (i, c)
    float2 x[kPanel];
#pragma unroll
    for (int q = 0; q < kPanel; ++q) x[q] = (q < nb && c < j0) ? XS[2 * (base + j0 + q)] : zero;
#pragma unroll
    for (int q = 0; q < kPanel; ++q) {
      const int sq = j0 + q;
      if (q >= nb || c > sq) continue;
      const float is = invf[sq].x;
      const float2 xs = (c == sq) ? make_float2(is, 0.f) : make_float2(x[q].x * is, x[q].y * is);
      x[q] = xs;
#pragma unroll
      for (int q2 = q + 1; q2 < kPanel; ++q2) {
        if (q2 >= nb) break;
        const float2 l = Lq[q * K + j0 + q2];
        x[q2].x -= l.x * xs.x - l.y * xs.y;
        x[q2].y -= l.x * xs.y + l.y * xs.x;
      }
    }
#pragma unroll
    for (int q = 0; q < kPanel; ++q)
      if (q < nb && j0 + q >= c) XS[2 * (base + j0 + q)] = x[q];
  }
  named_barrier_sync(bar, nt);
  const int r0 = j0 + nb, nr = (K - r0 + 1) / 2, ncp = (nc + 1) / 2;
  for (int u = t; u < nr * ncp; u += nt) {
    const int cp = u / nr, rp = u - cp * nr;
    const int i0 = r0 + 2 * rp, c0 = 2 * cp;
    const bool i1 = i0 + 1 < K, c1 = c0 + 1 < nc;
    float2 li0[kPanel], li1[kPanel], xc0[kPanel], xc1[kPanel];
#pragma unroll
    for (int q = 0; q < kPanel; ++q) {
      const bool ok = q < nb;
      const int sq = j0 + q;
      li0[q] = ok ? Lq[q * K + i0] : zero;
      li1[q] = ok && i1 ? Lq[q * K + i0 + 1] : zero;
      xc0[q] = ok && c0 <= sq ? XS[2 * (tri_off(c0, K) + sq - c0)] : zero;
      xc1[q] = ok && c1 && c0 + 1 <= sq ? XS[2 * (tri_off(c0 + 1, K) + sq - c0 - 1)] : zero;
    }
    const int s0 = tri_off(c0, K) + i0 - c0, s1 = c1 ? tri_off(c0 + 1, K) + i0 - c0 - 1 : 0;
    float2 v00 = c0 < j0 ? XS[2 * s0] : zero, v10 = i1 && c0 < j0 ? XS[2 * (s0 + 1)] : zero;
    float2 v01 = c1 && c0 + 1 < j0 ? XS[2 * s1] : zero, v11 = i1 && c1 && c0 + 1 < j0 ? XS[2 * (s1 + 1)] : zero;
#pragma unroll
    for (int q = 0; q < kPanel; ++q) {
      if (q >= nb) break;
      v00.x -= li0[q].x * xc0[q].x - li0[q].y * xc0[q].y;
      v00.y -= li0[q].x * xc0[q].y + li0[q].y * xc0[q].x;
      v10.x -= li1[q].x * xc0[q].x - li1[q].y * xc0[q].y;
      v10.y -= li1[q].x * xc0[q].y + li1[q].y * xc0[q].x;
      v01.x -= li0[q].x * xc1[q].x - li0[q].y * xc1[q].y;
      v01.y -= li0[q].x * xc1[q].y + li0[q].y * xc1[q].x;
      v11.x -= li1[q].x * xc1[q].x - li1[q].y * xc1[q].y;
      v11.y -= li1[q].x * xc1[q].y + li1[q].y * xc1[q].x;
    }
    XS[2 * s0] = v00;
    if (i1) XS[2 * (s0 + 1)] = v10;
    if (c1) XS[2 * s1] = v01;
    if (i1 && c1) XS[2 * (s1 + 1)] = v11;
  }
}

// One CTA per frequency p.
//
// 1-2. Fold the pending codes into the FP32 running means A^p, b^p and form
//      M = w A + rho I, y = w b in double-float.
// 3.   Blocked right-looking double-float Cholesky on the packed lower
//      triangle in panels of kPanel columns, with y carried along (forward
//      substitution y <- L^-1 w b), and X = L^-1 in FP32 one panel behind.
//      Per panel b, in one phase between two barriers:
//        warps 0..kPanel-1 apply panel b's rank-kPanel update to the columns
//                  of panel b+1, one column each (warp 0 alone, with the
//                  columns paired with them, once the trailing triangle is
//                  small), and meet at a named barrier; warp 0 then factors
//                  panel b+1 (fold_panel: pivots 1/sqrt by an FP32 estimate and
//                  one double-float Newton step, column scaling, the update
//                  inside the panel, y);
//        all warps apply panel b's update to the rest of the trailing
//                  triangle (fold_trail_tiles, 2 x 2 register tiles claimed
//                  32 at a time: warp 0 joins after its panel), warps 1.. run the
//                  forward substitution L X = I for the pivots of panel b-1
//                  (fold_xpanel_tiled: the pivot rows a column per thread,
//                  then the rows below by 2 x 2 register tiles).
//      The trailing triangle is folded into a rectangle (row r: column r, then
//      column n-1-r) whose rows go to warps and entries to lanes, so every
//      packed offset is a per-row base plus the lane's index.  X_ic is written
//      into the first 8 bytes of slot (i, c) once column c of L is no longer
//      read; panel b's columns are kept as FP32 copies (three buffers: panels
//      b-1 for X, b and b+1 in flight).
// 4.   Store X (FP32, packed lower) and y (FP32).
//
// Shared memory: M [T] float4, y [K] float4 (double-float), invf [K] float2,
// Lb [3][kPanel][K] float2, zs / xs (a chunk of pending codes).  During the
// fold each M slot first holds the FP32 running sum of conj(z_i) z_j in its
// first 8 bytes.
// DF (history precision 3): the products conj(z_i) z_j and x~ conj(z_i) are
// split exactly and summed in double-float, and the running means of A and b
// are kept as FP32 pairs (A + Alo, b + blo) updated in double-float, so that A
// and b stay exact functions of the same FP32 codes: with separately rounded
// products their rounding differs along directions that only rho damps, a
// forward error of order u cond(w A + rho I).
__device__ __forceinline__ void df_acc_cconjmul(float4 &v, float2 a, float2 b) {  // v += conj(a) b
  df_mac(a.x, 0.f, b.x, 0.f, v.x, v.z);
  df_mac(a.y, 0.f, b.y, 0.f, v.x, v.z);
  df_mac(a.x, 0.f, b.y, 0.f, v.y, v.w);
  df_mac(-a.y, 0.f, b.x, 0.f, v.y, v.w);
}
__device__ __forceinline__ void df_acc_cmulc(float4 &v, float2 a, float2 b) {  // v += a conj(b)
  df_mac(a.x, 0.f, b.x, 0.f, v.x, v.z);
  df_mac(a.y, 0.f, b.y, 0.f, v.x, v.z);
  df_mac(a.y, 0.f, b.x, 0.f, v.y, v.w);
  df_mac(-a.x, 0.f, b.y, 0.f, v.y, v.w);
}
// alpha (oh + ol) + beta (S + E) as a normalised pair, all in double-float.
__device__ __forceinline__ float2 df_blend(float oh, float ol, float S, float E, float2 al, float2 be) {
  const float2 s = two_sum(S, E);
  float P1, E1, P2, E2;
  df_mul(oh, ol, al.x, al.y, P1, E1);
  df_mul(s.x, s.y, be.x, be.y, P2, E2);
  df_acc(P1, E1, P2, E2);
  return two_sum(P1, E1);
}

// acc += conj(a) b by four FMAs (one rounding per FMA).
__device__ __forceinline__ void fold_mac(float2 &acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x));
  acc.y = fmaf(a.x, b.y, fmaf(-a.y, b.x, acc.y));
}

template <int kFoldThreads, bool DF>
__global__ void __launch_bounds__(kFoldThreads, 512 / kFoldThreads) fold_factor_kernel(FoldArgs a) {
  extern __shared__ __align__(16) unsigned char fsm[];
  const int K = a.K, F = a.F, B = a.B;
  const int T = tri_size(K);
  float4 *M = reinterpret_cast<float4 *>(fsm);                   // [T] double-float
  float4 *y = M + T;                                             // [K] double-float
  float2 *invf = reinterpret_cast<float2 *>(y + K);              // [K] 1 / L_jj, double-float
  float2 *Lb = invf + K;                                         // [3][kPanel][K]
  // Staged codes: rows of Kp = K rounded up to even, 16-byte aligned, so that
  // a 2 x 2 fold tile reads each pair of codes with one 16-byte load.
  const int Kp = K + (K & 1);
  float2 *zs = Lb + 3 * kPanel * K + (K & 1);                    // [kFoldChunk][Kp]
  float2 *xs = zs + kFoldChunk * Kp;                             // [kFoldChunk]
  float2 *S = reinterpret_cast<float2 *>(M);                     // FP32 sums, stride 2
  float2 *XS = reinterpret_cast<float2 *>(M);                    // X_ic at slot t: XS[2 t]
  // Frequency p of the class's grid (a band context factors rows p0 .. of
  // its own band; its history and factor arrays hold the band only).
  const int p = blockIdx.x + a.p0, pl = blockIdx.x;
  const int zF = a.zF ? a.zF : F, zp = p - a.zp0;
  const int tid = threadIdx.x;

  constexpr int MR = (128 + kFoldThreads - 1) / kFoldThreads;
  for (int t = tid; t < T; t += kFoldThreads) {
    if (DF) M[t] = make_float4(0.f, 0.f, 0.f, 0.f);
    else S[2 * t] = make_float2(0.f, 0.f);
  }
  float2 sb[MR];
  float4 sbd[DF ? MR : 1];
#pragma unroll
  for (int m = 0; m < MR; ++m) sb[m] = make_float2(0.f, 0.f);
#pragma unroll
  for (int m = 0; m < (DF ? MR : 1); ++m) sbd[m] = make_float4(0.f, 0.f, 0.f, 0.f);

  // 1. FP32 sums over the pending samples of conj(z_i) z_j and x~ conj(z_i).
  //    The codes of frequency p (one 8-byte word per sample and filter, F
  //    apart) come in chunks of kFoldChunk samples, every copy of a chunk in
  //    flight at once (asynchronous copies).
  const int mt = (K + 1) / 2, ntile = mt * (mt + 1) / 2;
  for (int c0 = 0; c0 < (a.prefolded ? 0 : B); c0 += kFoldChunk) {
    const int nb = min(kFoldChunk, B - c0);
    __syncthreads();
    for (int e = tid; e < nb * K; e += kFoldThreads) {
      const int s = e / K, k = e - s * K;
      cp_async8(zs + s * Kp + k, a.Zp + ((size_t)(c0 + s) * K + k) * zF + zp);
    }
    for (int s = tid; s < nb; s += kFoldThreads) cp_async8(xs + s, a.xh + (size_t)(c0 + s) * zF + zp);
    cp_async_wait_all();
    __syncthreads();
    // 2 x 2 tiles of the lower triangle (rows i0, i0 + 1, columns j0, j0 + 1):
    // the four codes of a sample are loaded once for the tile's four entries.
    // Entries outside the triangle (above the diagonal of a diagonal tile,
    // or index K for odd K) are computed from zeros and not stored.
    for (int u = tid; u < ntile; u += kFoldThreads) {
      int ti, tj;
      tri_ij(u, mt, ti, tj);
      const int i0 = 2 * ti, j0 = 2 * tj;
      const bool hi = i0 + 1 < K, hj = j0 + 1 < K, e01 = hj && ti > tj;
      const int t00 = tri_off(j0, K) + i0 - j0;                    // (i0 + 1, j0) follows it
      const int t01 = hj ? tri_off(j0 + 1, K) + i0 - j0 - 1 : 0;   // (i0 + 1, j0 + 1) follows it
      const float2 zero = make_float2(0.f, 0.f);
      if (DF) {
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        float4 a00 = M[t00], a10 = hi ? M[t00 + 1] : z4, a01 = e01 ? M[t01] : z4, a11 = hi && hj ? M[t01 + 1] : z4;
        for (int s = 0; s < nb; ++s) {
          const float4 zi = *reinterpret_cast<const float4 *>(zs + s * Kp + i0);
          const float4 zj = *reinterpret_cast<const float4 *>(zs + s * Kp + j0);
          const float2 zi0 = make_float2(zi.x, zi.y), zi1 = hi ? make_float2(zi.z, zi.w) : zero;
          const float2 zj0 = make_float2(zj.x, zj.y), zj1 = hj ? make_float2(zj.z, zj.w) : zero;
          df_acc_cconjmul(a00, zi0, zj0);
          df_acc_cconjmul(a10, zi1, zj0);
          df_acc_cconjmul(a01, zi0, zj1);
          df_acc_cconjmul(a11, zi1, zj1);
        }
        M[t00] = a00;
        if (hi) M[t00 + 1] = a10;
        if (e01) M[t01] = a01;
        if (hi && hj) M[t01 + 1] = a11;
      } else {
        float2 a00 = S[2 * t00], a10 = hi ? S[2 * (t00 + 1)] : zero, a01 = e01 ? S[2 * t01] : zero;
        float2 a11 = hi && hj ? S[2 * (t01 + 1)] : zero;
        for (int s = 0; s < nb; ++s) {
          const float4 zi = *reinterpret_cast<const float4 *>(zs + s * Kp + i0);
          const float4 zj = *reinterpret_cast<const float4 *>(zs + s * Kp + j0);
          const float2 zi0 = make_float2(zi.x, zi.y), zi1 = hi ? make_float2(zi.z, zi.w) : zero;
          const float2 zj0 = make_float2(zj.x, zj.y), zj1 = hj ? make_float2(zj.z, zj.w) : zero;
          fold_mac(a00, zi0, zj0);
          fold_mac(a10, zi1, zj0);
          fold_mac(a01, zi0, zj1);
          fold_mac(a11, zi1, zj1);
        }
        S[2 * t00] = a00;
        if (hi) S[2 * (t00 + 1)] = a10;
        if (e01) S[2 * t01] = a01;
        if (hi && hj) S[2 * (t01 + 1)] = a11;
      }
    }
#pragma unroll
    for (int m = 0; m < MR; ++m) {
      const int i = tid + m * kFoldThreads;
      if (i < K) {
        if (DF)
          for (int s = 0; s < nb; ++s) df_acc_cmulc(sbd[m], xs[s], zs[s * Kp + i]);
        else
          for (int s = 0; s < nb; ++s) sb[m] = cadd(sb[m], cmulc(xs[s], zs[s * Kp + i]));
      }
    }
  }
  __syncthreads();

  // 2. Running means in FP32 (stored), and M = w A + rho I, y = w b in
  //    double-float.
  float2 *Ap = a.A + (size_t)pl * tri_stride(K);
  const float alpha = (float)a.alpha, beta = (float)a.beta;
  float2 *Lo = a.Alo ? a.Alo + (size_t)pl * tri_stride(K) : nullptr;
  const float2 wf = df_of(a.w), rf = df_of(a.rho_eff);
  const float2 ald = df_of(a.alpha), bed = df_of(a.beta);
  for (int t = tid; t < T; t += kFoldThreads) {
    int i, j;
    tri_ij(t, K, i, j);
    float2 hf, lf = make_float2(0.f, 0.f);
    if (a.prefolded) {  // A (+ its compensation word) already holds the new mean
      hf = Ap[t];
      if (Lo) lf = Lo[t];
    } else if (DF) {
      const float2 oh = a.first ? make_float2(0.f, 0.f) : Ap[t];
      const float2 ol = a.first ? make_float2(0.f, 0.f) : Lo[t];
      const float4 sum = M[t];
      const float2 nr = df_blend(oh.x, ol.x, sum.x, sum.z, ald, bed);
      const float2 ni = df_blend(oh.y, ol.y, sum.y, sum.w, ald, bed);
      hf = make_float2(nr.x, ni.x);
      lf = make_float2(nr.y, ni.y);
      Ap[t] = hf;
      Lo[t] = lf;
    } else {
      const float2 old = a.first ? make_float2(0.f, 0.f) : Ap[t];
      const float2 sum = S[2 * t];
      hf = make_float2(fmaf(alpha, old.x, beta * sum.x), fmaf(alpha, old.y, beta * sum.y));
      Ap[t] = hf;
    }
    // w (h + lo) in FP32 pairs (the FP64 pipe is kept for the pivots).
    float Sr, Er, Si, Ei;
    df_mul(hf.x, lf.x, wf.x, wf.y, Sr, Er);
    df_mul(hf.y, lf.y, wf.x, wf.y, Si, Ei);
    if (i == j) {
      const float2 s2 = two_sum(Sr, rf.x);
      Sr = s2.x;
      Er += s2.y + rf.y;
      Si = 0.f;
      Ei = 0.f;
    }
    M[t] = make_float4(Sr, Si, Er, Ei);
  }
#pragma unroll
  for (int m = 0; m < (128 + kFoldThreads - 1) / kFoldThreads; ++m) {
    const int i = tid + m * kFoldThreads;
    if (i < K) {
      float2 nw, nl = make_float2(0.f, 0.f);
      const size_t o = (size_t)i * F + p;
      if (a.prefolded) {
        nw = a.b[o];
        if (a.blo) nl = a.blo[o];
      } else if (DF) {
        const float2 oh = a.first ? make_float2(0.f, 0.f) : a.b[o];
        const float2 ol = a.first ? make_float2(0.f, 0.f) : a.blo[o];
        const float4 sum = sbd[DF ? m : 0];
        const float2 nr = df_blend(oh.x, ol.x, sum.x, sum.z, ald, bed);
        const float2 ni = df_blend(oh.y, ol.y, sum.y, sum.w, ald, bed);
        nw = make_float2(nr.x, ni.x);
        nl = make_float2(nr.y, ni.y);
        a.b[o] = nw;
        a.blo[o] = nl;
      } else {
        const float2 old = a.first ? make_float2(0.f, 0.f) : a.b[o];
        nw = make_float2(fmaf(alpha, old.x, beta * sb[m].x), fmaf(alpha, old.y, beta * sb[m].y));
        a.b[o] = nw;
      }
      float Sr, Er, Si, Ei;
      df_mul(nw.x, nl.x, wf.x, wf.y, Sr, Er);
      df_mul(nw.y, nl.y, wf.x, wf.y, Si, Ei);
      y[i] = make_float4(Sr, Si, Er, Ei);
    }
  }
  __syncthreads();

  // 3. Blocked Cholesky (double-float), y alongside, X = L^-1 one panel behind.
  const int warp = tid >> 5, lane = tid & 31;
  const float rho_fb = a.rho_eff > 0.0 ? (float)a.rho_eff : 1.f;
  const int nblk = (K + kPanel - 1) / kPanel;
  __shared__ int s_ctr[2];  // tile counters of the trailing update, by phase parity
  if (tid < 2) s_ctr[tid] = 0;
  if (warp == 0) fold_panel(M, y, invf, Lb, K, 0, lane, a.err, rho_fb);
  __syncthreads();
  for (int b = 0; b < nblk; ++b) {
    const int j0 = b * kPanel, nb = min(kPanel, K - j0), n = K - j0 - nb;
    const int nb2 = min(kPanel, n), R = (n + 1) / 2, rw = min(nb2, R);
    // For n >= 2 kPanel the next panel's columns are exactly the first parts
    // of rectangle rows r < kPanel (warp 0) and the flat pool takes the rest;
    // below that warp 0 takes the whole (small) triangle.
    const bool small = n < 2 * kPanel;
    if (small) {
      if (warp == 0) {
        fold_trail(M, K, j0, nb, 0, 1, R, lane, true);
        __syncwarp();
        if (nb2 > 0) fold_panel(M, y, invf, Lb, K, b + 1, lane, a.err, rho_fb);
      } else if (b >= 1) {
        fold_xpanel_tiled(XS, Lb, invf, K, b - 1, tid - 32, kFoldThreads - 32, 2);
      }
    } else {
      // Here nb2 = rw = kPanel: warps 0 .. kPanel-1 update one column of the
      // next panel each and meet at a named barrier before warp 0 factors it.
      if (warp < kPanel) {
        fold_trail(M, K, j0, nb, warp, kPanel, rw, lane, false);
        named_barrier_sync(1, kPanel * 32);
      }
      if (warp == 0) {
        fold_panel(M, y, invf, Lb, K, b + 1, lane, a.err, rho_fb);
        fold_trail_tiles(M, K, j0, nb, rw, &s_ctr[b & 1]);
      } else {
        fold_trail_tiles(M, K, j0, nb, rw, &s_ctr[b & 1]);
        if (b >= 1) fold_xpanel_tiled(XS, Lb, invf, K, b - 1, tid - 32, kFoldThreads - 32, 2);
      }
      if (tid == 0) s_ctr[(b + 1) & 1] = 0;  // the next phase's counter (unused in this one)
    }
    __syncthreads();
  }
  fold_xpanel_tiled(XS, Lb, invf, K, nblk - 1, tid, kFoldThreads, 2);
  __syncthreads();

  // 4. Store X = L^-1 (FP32) and y = L^-1 (w b) (FP32).
  float2 *Xp = a.L + (size_t)pl * tri_stride(K);
  for (int t = tid; t < T; t += kFoldThreads) Xp[t] = XS[2 * t];
  for (int i = tid; i < K; i += kFoldThreads)
    a.g[(size_t)i * F + p] = make_float2(y[i].x + y[i].z, y[i].y + y[i].w);
}

// D-row step of eq. (sub_d_sol): d = (w A + rho I)^-1 (w b + rho (v^ - theta^))
// = X^H (y + rho X r) with X = L^-1, y = L^-1 (w b) and r = v^ - theta^: two
// triangular matrix-vector products per frequency, no sequential dependency.
// One CTA per frequency, thread i owns row i: the first product
// t_i = y_i + rho sum_{j<=i} X_ij r_j takes i+1 terms and the second
// d_i = sum_{k>=i} conj(X_ki) t_k takes K-i, so every thread does K+1 terms.
// X is staged in shared memory with 16-byte cp.async copies (the per-frequency
// stride is even, so sources are 16-byte aligned).  Also writes E = d + theta^.
__global__ void dstep_kernel(int K, int F, float rho_eff, const float2 *__restrict__ X,
                             const float2 *__restrict__ yb, const float2 *__restrict__ Vh,
                             const float2 *__restrict__ th, float2 *__restrict__ Dcur,
                             float2 *__restrict__ E, int p0) {
  extern __shared__ __align__(16) float2 dsm[];
  const int TS = tri_stride(K);
  float2 *sX = dsm;
  float2 *sr = sX + TS;
  float2 *st = sr + K;
  const int p = blockIdx.x + p0, i = threadIdx.x;  // X holds frequencies p0 .. only
  const float4 *g4 = reinterpret_cast<const float4 *>(X + (size_t)blockIdx.x * TS);
  float4 *s4 = reinterpret_cast<float4 *>(sX);
  for (int c = i; c < TS / 2; c += blockDim.x) cp_async16(s4 + c, g4 + c);
  float2 thi = make_float2(0.f, 0.f), yi = make_float2(0.f, 0.f);
  if (i < K) {
    const size_t o = (size_t)i * F + p;
    const float2 v = Vh[o];
    thi = th[o];
    yi = yb[o];
    sr[i] = make_float2(v.x - thi.x, v.y - thi.y);
  }
  cp_async_wait_all();
  __syncthreads();
  if (i < K) {
    float2 acc = make_float2(0.f, 0.f);
    for (int j = 0; j <= i; ++j) {
      const float2 x = sX[tri_off(j, K) + i - j], rj = sr[j];
      acc.x += x.x * rj.x - x.y * rj.y;
      acc.y += x.x * rj.y + x.y * rj.x;
    }
    st[i] = make_float2(yi.x + rho_eff * acc.x, yi.y + rho_eff * acc.y);
  }
  __syncthreads();
  if (i < K) {
    const float2 *col = sX + tri_off(i, K) - i;
    float2 acc = make_float2(0.f, 0.f);
    for (int k = i; k < K; ++k) {
      const float2 x = col[k], tk = st[k];
      acc.x += x.x * tk.x + x.y * tk.y;
      acc.y += x.x * tk.y - x.y * tk.x;
    }
    const size_t o = (size_t)i * F + p;
    Dcur[o] = acc;
    E[o] = cadd(acc, thi);
  }
}

// Pruned inverse DFT along k1, restricted to m1 in [0, M):
// Y[k][m1][k2] = sum_k1 E[k][k1][k2] exp(+2 pi i k1 m1 / N).
// Grid (K, ceil(NH/32)), block (32, M): the block first stages its N x 32
// column block of E in shared memory (coalesced rows of 32 bins), then thread
// (k2, m1) sums over k1 from there.
constexpr int kMaxM = 16;
// Rows k1 in [k1_lo, k1_hi) only (an even count): the whole range, or the
// band of a band context, whose sums over bands add up to the full one.
__global__ void vstep_cols_kernel(int K, int N, int M, const float2 *__restrict__ E,
                                  const float2 *__restrict__ tw, float2 *__restrict__ Y, int k1_lo, int k1_hi) {
  extern __shared__ float2 s_twc[];  // [N] twiddles, then [rows][32] column block
  float2 *s_e = s_twc + N;
  const int NH = N / 2 + 1, F = N * NH, rows = k1_hi - k1_lo;
  const int tid = threadIdx.y * 32 + threadIdx.x, nthr = 32 * blockDim.y;
  for (int i = tid; i < N; i += nthr) s_twc[i] = tw[i];
  const int k = blockIdx.x, k2 = blockIdx.y * 32 + threadIdx.x, m1 = threadIdx.y;
  const float2 *Ek = E + (size_t)k * F + (size_t)k1_lo * NH + blockIdx.y * 32;
  const int ncol = min(32, NH - blockIdx.y * 32);
  for (int e = tid; e < rows * 32; e += nthr) {
    const int k1 = e >> 5, c = e & 31;
    s_e[e] = c < ncol ? Ek[(size_t)k1 * NH + c] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  if (k2 >= NH) return;
  float2 acc0 = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
  int ph = (k1_lo * m1) % N;  // (k1 m1) mod N
  for (int k1 = 0; k1 < rows; k1 += 2) {
    acc0 = cadd(acc0, cmulc(s_e[k1 * 32 + threadIdx.x], s_twc[ph]));
    ph += m1;
    if (ph >= N) ph -= N;
    acc1 = cadd(acc1, cmulc(s_e[(k1 + 1) * 32 + threadIdx.x], s_twc[ph]));
    ph += m1;
    if (ph >= N) ph -= N;
  }
  Y[((size_t)k * M + m1) * NH + k2] = cadd(acc0, acc1);
}

// V-step of Proposition 2 over the active size classes, one CTA per filter k:
// alpha_c = H(F_c^-1(D~_c + theta^_c)) from each class's Y_c, alpha = mean over
// classes (with one class, alpha_c itself), V_k = alpha / max(||alpha||, 1).
// With ac.project = 0 it writes alpha itself (H(F^-1(.)) of what Y was formed
// from), which publishes D~_{t,J} literally.
constexpr int kProjThreads = 256;
__global__ void __launch_bounds__(kProjThreads)
    vstep_project_kernel(int K, int M, AlphaClasses ac, float *__restrict__ V) {
  __shared__ float alpha[kMaxM * kMaxM];
  __shared__ float red[32];
  const int MM = M * M;
  const int k = blockIdx.x, tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31, nwarps = kProjThreads / 32;
  for (int e = tid; e < MM; e += kProjThreads) alpha[e] = 0.f;
  __syncthreads();
  for (int c = 0; c < ac.C; ++c) {
    const int N = ac.N[c], NH = N / 2 + 1;
    const float2 *tw = ac.tw[c];
    const float scale = 1.0f / ((float)(N * N) * (float)ac.C);
    for (int e = warp; e < MM; e += nwarps) {
      const int m1 = e / M, m2 = e % M;
      const float2 *Yr = ac.Y[c] + ((size_t)k * M + m1) * NH;
      float s = 0.f;
      for (int k2 = lane; k2 < NH; k2 += 32) {
        const float2 yv = Yr[k2];
        const float2 w = tw[(k2 * m2) % N];
        const float cw = (k2 == 0 || k2 == N / 2) ? 1.f : 2.f;
        s += cw * (yv.x * w.x + yv.y * w.y);
      }
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) alpha[e] += s * scale;
    }
    __syncthreads();
  }
  float ss = 0.f;
  for (int e = tid; e < MM; e += kProjThreads) ss += alpha[e] * alpha[e];
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  if (lane == 0) red[warp] = ss;
  __syncthreads();
  if (tid < 32) {
    float v = tid < nwarps ? red[tid] : 0.f;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (tid == 0) red[0] = v;
  }
  __syncthreads();
  const float sc = ac.project ? 1.0f / fmaxf(sqrtf(red[0]), 1.0f) : 1.0f;
  for (int e = tid; e < MM; e += kProjThreads) V[(size_t)k * MM + e] = alpha[e] * sc;
}

// Partial forward DFT of the filters for one size class, one CTA per filter:
// Tm(m1, k2) = sum_m2 V(m1, m2) W_N^(k2 m2), k2 in [0, N/2].
__global__ void __launch_bounds__(kProjThreads)
    vstep_partial_dft_kernel(int K, int N, int M, const float *__restrict__ V,
                             const float2 *__restrict__ tw, float2 *__restrict__ Tm) {
  extern __shared__ __align__(16) unsigned char psm[];
  const int NH = N / 2 + 1, MM = M * M;
  float2 *s_tw = reinterpret_cast<float2 *>(psm);
  float *alpha = reinterpret_cast<float *>(s_tw + N);
  const int k = blockIdx.x, tid = threadIdx.x;
  for (int i = tid; i < N; i += kProjThreads) s_tw[i] = tw[i];
  for (int e = tid; e < MM; e += kProjThreads) alpha[e] = V[(size_t)k * MM + e];
  __syncthreads();
  for (int e = tid; e < M * NH; e += kProjThreads) {
    const int m1 = e / NH, k2 = e % NH;
    float2 acc = make_float2(0.f, 0.f);
    for (int m2 = 0; m2 < M; ++m2) {
      const float2 w = s_tw[(k2 * m2) % N];
      const float v = alpha[m1 * M + m2];
      acc.x += v * w.x;
      acc.y += v * w.y;
    }
    Tm[(size_t)k * M * NH + e] = acc;
  }
}

// V^(k1, k2) = sum_m1 Tm(m1, k2) W^(k1 m1) over the half spectrum; mode 0 also
// updates the dual theta^ += D~ - V^.  Grid (K, ceil(F/256)).
__global__ void __launch_bounds__(256)
    vstep_spectrum_kernel(int mode, int K, int N, int M, const float2 *__restrict__ Tm,
                          const float2 *__restrict__ tw, float2 *__restrict__ Vh, float2 *__restrict__ th,
                          const float2 *__restrict__ Dcur, int p0, int p1) {
  __shared__ float2 s_tw[kMaxFFT];
  const int NH = N / 2 + 1, F = N * NH;
  for (int i = threadIdx.x; i < N; i += 256) s_tw[i] = tw[i];
  __syncthreads();
  const int k = blockIdx.x;
  const int p = blockIdx.y * 256 + threadIdx.x;
  if (p >= F) return;
  const int k1 = p / NH, k2 = p % NH;
  const float2 *T = Tm + (size_t)k * M * NH + k2;
  float2 acc = make_float2(0.f, 0.f);
  for (int m1 = 0; m1 < M; ++m1) acc = cadd(acc, cmul(T[(size_t)m1 * NH], s_tw[(k1 * m1) % N]));
  const size_t o = (size_t)k * F + p;
  Vh[o] = acc;
  if (mode == 0 && p >= p0 && p < p1) {  // the dual lives on the frequencies this context solves
    const float2 d = Dcur[o];
    const float2 t = th[o];
    th[o] = make_float2(t.x + d.x - acc.x, t.y + d.y - acc.y);
  }
}

// Proposition 2 on given support sums: V_k = alpha_k / max(||alpha_k||, 1)
// (the band path: alpha is the sum over the bands of their partial crops).
__global__ void __launch_bounds__(kProjThreads)
    project_alpha_kernel(int K, int MM, const float *__restrict__ alpha, float *__restrict__ V) {
  __shared__ float red[32];
  const int k = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarps = kProjThreads / 32;
  const float *a = alpha + (size_t)k * MM;
  float ss = 0.f;
  for (int e = tid; e < MM; e += kProjThreads) ss += a[e] * a[e];
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  if (lane == 0) red[warp] = ss;
  __syncthreads();
  if (tid < 32) {
    float v = tid < nwarps ? red[tid] : 0.f;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (tid == 0) red[0] = v;
  }
  __syncthreads();
  const float sc = 1.0f / fmaxf(sqrtf(red[0]), 1.0f);
  for (int e = tid; e < MM; e += kProjThreads) V[(size_t)k * MM + e] = a[e] * sc;
}

cudaError_t launch_project_alpha(int K, int M, const float *alpha, float *V, cudaStream_t s) {
  project_alpha_kernel<<<K, kProjThreads, 0, s>>>(K, M * M, alpha, V);
  return cudaGetLastError();
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
  return (size_t)(tri_size(K) + K) * sizeof(float4) + (size_t)(1 + 3 * kPanel) * K * sizeof(float2) +
         ((size_t)kFoldChunk * (K + (K & 1)) + (K & 1)) * sizeof(float2) + kFoldChunk * sizeof(float2);
}

// threads: 256 or 512 (CTA size of the per-frequency factorisation; every
// entry sees the same operations in the same order either way).
template <int NTH, bool DF>
static cudaError_t fold_factor_n(const FoldArgs &a, size_t sm, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(fold_factor_kernel<NTH, DF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  fold_factor_kernel<NTH, DF><<<a.nF ? a.nF : a.F, NTH, sm, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_fold_factor(const FoldArgs &a, int threads, cudaStream_t s) {
  const size_t sm = fold_smem_bytes(a.K);
  if (a.dfold && !a.prefolded && (!a.Alo || !a.blo)) return cudaErrorInvalidValue;
  const bool df = a.dfold && !a.prefolded;
  if (threads == 512) return df ? fold_factor_n<512, true>(a, sm, s) : fold_factor_n<512, false>(a, sm, s);
  return df ? fold_factor_n<256, true>(a, sm, s) : fold_factor_n<256, false>(a, sm, s);
}

cudaError_t launch_dstep(int K, int F, float rho_eff, const float2 *X, const float2 *yb,
                         const float2 *Vh, const float2 *th, float2 *Dcur, float2 *E,
                         cudaStream_t s, int p0, int nF) {
  if (K > 256) return cudaErrorInvalidValue;
  const size_t sm = ((size_t)tri_stride(K) + 2 * (size_t)K) * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(dstep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const int threads = (K + 31) / 32 * 32;
  dstep_kernel<<<nF ? nF : F, threads, sm, s>>>(K, F, rho_eff, X, yb, Vh, th, Dcur, E, p0);
  return cudaGetLastError();
}

cudaError_t launch_vstep_cols(int K, int N, int M, const float2 *E, const float2 *tw, float2 *Y,
                              cudaStream_t s, int k1_lo, int k1_hi) {
  if (M > kMaxM || N > kMaxFFT) return cudaErrorInvalidValue;
  if (k1_hi == 0) k1_hi = N;
  if (k1_lo < 0 || k1_hi > N || k1_lo >= k1_hi || (k1_hi - k1_lo) % 2) return cudaErrorInvalidValue;
  dim3 grid(K, (N / 2 + 1 + 31) / 32), block(32, M);
  const size_t sm = (size_t)N * 33 * sizeof(float2);
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(vstep_cols_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  vstep_cols_kernel<<<grid, block, sm, s>>>(K, N, M, E, tw, Y, k1_lo, k1_hi);
  return cudaGetLastError();
}

cudaError_t launch_vstep_project(int K, int M, const AlphaClasses &ac, float *V, cudaStream_t s) {
  if (M > kMaxM || ac.C < 1 || ac.C > kMaxClasses) return cudaErrorInvalidValue;
  vstep_project_kernel<<<K, kProjThreads, 0, s>>>(K, M, ac, V);
  return cudaGetLastError();
}

cudaError_t launch_vstep_partial_dft(int K, int N, int M, const float *V, const float2 *tw, float2 *Tm,
                                     cudaStream_t s) {
  if (M > kMaxM || N > kMaxFFT) return cudaErrorInvalidValue;
  const size_t sm = N * sizeof(float2) + kMaxM * kMaxM * sizeof(float);
  vstep_partial_dft_kernel<<<K, kProjThreads, sm, s>>>(K, N, M, V, tw, Tm);
  return cudaGetLastError();
}

cudaError_t launch_vstep_spectrum(int mode, int K, int N, int M, const float2 *Tm, const float2 *tw,
                                  float2 *Vh, float2 *th, const float2 *Dcur, cudaStream_t s, int p0, int p1) {
  if (M > kMaxM || N > kMaxFFT) return cudaErrorInvalidValue;
  const int F = N * (N / 2 + 1);
  dim3 grid(K, (F + 255) / 256);
  vstep_spectrum_kernel<<<grid, 256, 0, s>>>(mode, K, N, M, Tm, tw, Vh, th, Dcur, p0, p1 ? p1 : F);
  return cudaGetLastError();
}

cudaError_t launch_dict_norms(int K, int F, const float2 *Dh, float *dn, cudaStream_t s) {
  dict_norms_kernel<<<(F + 255) / 256, 256, 0, s>>>(K, F, Dh, dn);
  return cudaGetLastError();
}

}  // namespace ocsc
