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

// One CTA per frequency p.
//
// 1-2. Fold the pending codes into the FP32 running means A^p, b^p and form
//      M = w A + rho I, y = w b in double-float.
// 3.   Right-looking double-float Cholesky on the packed lower triangle, with
//      y carried as an extra column (forward substitution: y <- L^-1 w b); the
//      pivots 1 / sqrt(.) are taken in FP64.  One step behind it, the same
//      threads run the right-looking forward substitution of L X = I in FP32
//      (X = L^-1): after column s of L is final, row s of X is scaled by
//      1/L_ss and every X_ic with i > s, c <= s gets X_ic -= L_is X_sc.  The
//      FP32 update of step s runs in the same phase as the trailing update of
//      step s+1 and writes only slots of columns <= s, whose double-float
//      values are no longer read: the first 8 bytes of such a slot then hold
//      X_ic.  L's column s (FP32 copy) and X's row s are kept in small buffers
//      so those reads are broadcasts.
// 4.   Store X (FP32, packed lower) and y (FP32).
//
// Shared memory: M [T] float4, y [K] float4 (double-float), invf [K] float2,
// Lcol [2][K] float2, Xrow [K] float2, zs / xs (a chunk of pending codes).
// During the fold each M slot first holds the FP32 running sum of
// conj(z_i) z_j in its first 8 bytes.
template <int kFoldThreads>
__global__ void __launch_bounds__(kFoldThreads) fold_factor_kernel(FoldArgs a) {
  extern __shared__ __align__(16) unsigned char fsm[];
  const int K = a.K, F = a.F, B = a.B;
  const int T = tri_size(K);
  float4 *M = reinterpret_cast<float4 *>(fsm);                   // [T] double-float
  float4 *y = M + T;                                             // [K] double-float
  float2 *invf = reinterpret_cast<float2 *>(y + K);              // [K] 1 / L_jj, double-float
  float2 *Lcol = invf + K;                                       // [2][K]
  float2 *Xrow = Lcol + 2 * K;                                   // [K]
  float2 *zs = Xrow + K;                                         // [kFoldChunk][K]
  float2 *xs = zs + kFoldChunk * K;                              // [kFoldChunk]
  float2 *S = reinterpret_cast<float2 *>(M);                     // FP32 sums, stride 2
  float2 *XS = reinterpret_cast<float2 *>(M);                    // X_ic at slot t: XS[2 t]
  const int p = blockIdx.x;
  const int tid = threadIdx.x;

  for (int t = tid; t < T; t += kFoldThreads) S[2 * t] = make_float2(0.f, 0.f);
  float2 sb[(128 + kFoldThreads - 1) / kFoldThreads];
#pragma unroll
  for (int m = 0; m < (128 + kFoldThreads - 1) / kFoldThreads; ++m) sb[m] = make_float2(0.f, 0.f);

  // 1. FP32 sums over the pending samples of conj(z_i) z_j and x~ conj(z_i).
  for (int c0 = 0; c0 < (a.prefolded ? 0 : B); c0 += kFoldChunk) {
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
      float2 acc = S[2 * t];
      for (int s = 0; s < nb; ++s) acc = cadd(acc, cconjmul(zs[s * K + i], zs[s * K + j]));
      S[2 * t] = acc;
    }
#pragma unroll
    for (int m = 0; m < (128 + kFoldThreads - 1) / kFoldThreads; ++m) {
      const int i = tid + m * kFoldThreads;
      if (i < K)
        for (int s = 0; s < nb; ++s) sb[m] = cadd(sb[m], cmulc(xs[s], zs[s * K + i]));
    }
  }
  __syncthreads();

  // 2. Running means in FP32 (stored), and M = w A + rho I, y = w b in
  //    double-float.
  float2 *Ap = a.A + (size_t)p * tri_stride(K);
  const float alpha = (float)a.alpha, beta = (float)a.beta;
  const float2 *Lo = a.Alo ? a.Alo + (size_t)p * tri_stride(K) : nullptr;
  const float2 wf = df_of(a.w), rf = df_of(a.rho_eff);
  for (int t = tid; t < T; t += kFoldThreads) {
    int i, j;
    tri_ij(t, K, i, j);
    float2 hf, lf = make_float2(0.f, 0.f);
    if (a.prefolded) {  // A (+ its compensation word) already holds the new mean
      hf = Ap[t];
      if (Lo) lf = Lo[t];
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
      float2 nw;
      if (a.prefolded) {
        nw = a.b[(size_t)i * F + p];
      } else {
        const float2 old = a.first ? make_float2(0.f, 0.f) : a.b[(size_t)i * F + p];
        nw = make_float2(fmaf(alpha, old.x, beta * sb[m].x), fmaf(alpha, old.y, beta * sb[m].y));
        a.b[(size_t)i * F + p] = nw;
      }
      float Sr, Er, Si, Ei;
      df_mul(nw.x, 0.f, wf.x, wf.y, Sr, Er);
      df_mul(nw.y, 0.f, wf.x, wf.y, Si, Ei);
      y[i] = make_float4(Sr, Si, Er, Ei);
    }
  }
  __syncthreads();

  // 3. Cholesky (double-float) with the FP32 inverse one step behind.  Slots
  //    of M and y hold unnormalised pairs (S, E) while they are being updated
  //    and are normalised when they become entries of L (scale phase).
  if (tid == 0) {
    double piv = df_val(M[0].x, M[0].z);
    if (!(piv > 0.0)) {
      atomicOr(a.err, ERR_PIVOT);
      piv = a.rho_eff > 0.0 ? a.rho_eff : 1.0;
    }
    const double r = rsqrt(piv);  // 1 / L_00; L_00 = piv / sqrt(piv)
    M[0] = df_split2(piv * r, 0.0);
    invf[0] = df_of(r);
  }
  __syncthreads();
  for (int j = 0; j <= K; ++j) {
    // --- scale phase: column j of L (double-float + FP32 copy), row j-1 of X.
    if (j < K) {
      const int oj = tri_off(j, K);
      const float2 inv = invf[j];
      float2 *lc = Lcol + (j & 1) * K;
      for (int i = j + 1 + tid; i < K; i += kFoldThreads) {
        const float4 v = M[oj + i - j];
        const float2 vr = two_sum(v.x, v.z), vi = two_sum(v.y, v.w);
        float Sr, Er, Si, Ei;
        df_mul(vr.x, vr.y, inv.x, inv.y, Sr, Er);
        df_mul(vi.x, vi.y, inv.x, inv.y, Si, Ei);
        const float2 lr = two_sum(Sr, Er), li = two_sum(Si, Ei);
        M[oj + i - j] = make_float4(lr.x, li.x, lr.y, li.y);
        lc[i] = make_float2(lr.x, li.x);
      }
      if (tid == 0) {
        const float4 v = y[j];
        const float2 vr = two_sum(v.x, v.z), vi = two_sum(v.y, v.w);
        float Sr, Er, Si, Ei;
        df_mul(vr.x, vr.y, inv.x, inv.y, Sr, Er);
        df_mul(vi.x, vi.y, inv.x, inv.y, Si, Ei);
        const float2 yr = two_sum(Sr, Er), yi = two_sum(Si, Ei);
        y[j] = make_float4(yr.x, yi.x, yr.y, yi.y);
      }
    }
    if (j >= 1) {
      const int s1 = j - 1;                 // X row s1 is final up to its scaling
      const float is = invf[s1].x;
      for (int c = tid; c <= s1; c += kFoldThreads) {
        const int slot = tri_off(c, K) + s1 - c;
        const float2 xv = (c == s1) ? make_float2(is, 0.f)
                                    : make_float2(XS[2 * slot].x * is, XS[2 * slot].y * is);
        Xrow[c] = xv;
        XS[2 * slot] = xv;
      }
    }
    __syncthreads();
    // --- update phase: trailing update of step j, FP32 X update of step j-1.
    if (j < K) {
      const int oj = tri_off(j, K);
      const int n = K - j - 1;
      const int nt = tri_size(n);
      const float4 yj = y[j];
      if (tid == 0 && nt > 0) {  // element (j+1, j+1) also finishes the next pivot
        const int d1 = tri_off(j + 1, K);
        const float4 l = M[oj + 1], v = M[d1];
        const double lx = df_val(l.x, l.z), ly = df_val(l.y, l.w);
        double piv = df_val(v.x, v.z) - (lx * lx + ly * ly);
        if (!(piv > 0.0)) {
          atomicOr(a.err, ERR_PIVOT);
          piv = a.rho_eff > 0.0 ? a.rho_eff : 1.0;
        }
        const double r = rsqrt(piv);
        M[d1] = df_split2(piv * r, 0.0);
        invf[j + 1] = df_of(r);
      }
      // M_ik -= L_ij conj(L_kj) over the trailing triangle (ii >= kk in [0, n),
      // rows j+1+ii, columns j+1+kk), folded into a rectangle: row r holds
      // column kk = r (c < n - r: ii = r + c) followed by column n - 1 - r
      // (ii = c - 1); for odd n the middle row holds only its first part.  A
      // warp takes a rectangle row, its lanes the entries, so every packed
      // offset is a per-row base plus c.  Element (0, 0), the next pivot, is
      // done above.
      {
        const int warp = tid >> 5, lane = tid & 31, R = (n + 1) / 2;
        for (int r = warp; r < R; r += kFoldThreads / 32) {
          const int cut = n - r, len = (2 * r + 1 == n) ? cut : n + 1, kb = n - 1 - r;
          const int dsta = tri_off(j + 1 + r, K), dstb = tri_off(j + 1 + kb, K) - cut;
          const int lia = oj + 1 + r, lib = oj;  // L row offsets: + c
          for (int c = lane; c < len; c += 32) {
            if (r == 0 && c == 0) continue;
            const bool first = c < cut;
            const float4 lk = M[first ? oj + 1 + r : oj + 1 + kb];
            const float4 li = M[(first ? lia : lib) + c];
            const int dst = (first ? dsta : dstb) + c;
            float4 v = M[dst];
            df_mac(-li.x, -li.z, lk.x, lk.z, v.x, v.z);  // Re: - Re li Re lk - Im li Im lk
            df_mac(-li.y, -li.w, lk.y, lk.w, v.x, v.z);
            df_mac(-li.y, -li.w, lk.x, lk.z, v.y, v.w);  // Im: - Im li Re lk + Re li Im lk
            df_mac(li.x, li.z, lk.y, lk.w, v.y, v.w);
            M[dst] = v;
          }
        }
      }
      // y_i -= L_ij y_j.
      for (int u = tid; u < n; u += kFoldThreads) {
        const int i = j + 1 + u;
        const float4 l = M[oj + i - j];
        float4 v = y[i];
        df_mac(-l.x, -l.z, yj.x, yj.z, v.x, v.z);  // Re: - Re l Re y + Im l Im y
        df_mac(l.y, l.w, yj.y, yj.w, v.x, v.z);
        df_mac(-l.x, -l.z, yj.y, yj.w, v.y, v.w);  // Im: - Re l Im y - Im l Re y
        df_mac(-l.y, -l.w, yj.x, yj.z, v.y, v.w);
        y[i] = v;
      }
    }
    if (j >= 1) {
      // X_ic -= L_i,s1 X_s1,c for i > s1, c <= s1; column s1 of X starts here
      // (its entries below the diagonal were zero).  A warp takes columns c,
      // its lanes the rows i, whose L entries stay in registers.
      const int s1 = j - 1;
      const float2 *lc = Lcol + (s1 & 1) * K;
      const int warp = tid >> 5, lane = tid & 31;
      float2 lreg[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const int i = j + lane + 32 * m;
        lreg[m] = i < K ? lc[i] : make_float2(0.f, 0.f);
      }
      for (int c = warp; c <= s1; c += kFoldThreads / 32) {
        const float2 xs1 = Xrow[c];
        const int base = tri_off(c, K) - c;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const int i = j + lane + 32 * m;
          if (i < K) {
            const float2 l = lreg[m];
            float2 v = (c == s1) ? make_float2(0.f, 0.f) : XS[2 * (base + i)];
            v.x -= l.x * xs1.x - l.y * xs1.y;
            v.y -= l.x * xs1.y + l.y * xs1.x;
            XS[2 * (base + i)] = v;
          }
        }
      }
    }
    __syncthreads();
  }

  // 4. Store X = L^-1 (FP32) and y = L^-1 (w b) (FP32).
  float2 *Xp = a.L + (size_t)p * tri_stride(K);
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
                             float2 *__restrict__ E) {
  extern __shared__ __align__(16) float2 dsm[];
  const int TS = tri_stride(K);
  float2 *sX = dsm;
  float2 *sr = sX + TS;
  float2 *st = sr + K;
  const int p = blockIdx.x, i = threadIdx.x;
  const float4 *g4 = reinterpret_cast<const float4 *>(X + (size_t)p * TS);
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
// Grid (K, ceil(NH/32)), block (32, M): thread (k2, m1).
constexpr int kMaxM = 16;
__global__ void vstep_cols_kernel(int K, int N, int M, const float2 *__restrict__ E,
                                  const float2 *__restrict__ tw, float2 *__restrict__ Y) {
  extern __shared__ float2 s_twc[];
  const int NH = N / 2 + 1, F = N * NH;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  for (int i = tid; i < N; i += 32 * blockDim.y) s_twc[i] = tw[i];
  __syncthreads();
  const int k = blockIdx.x, k2 = blockIdx.y * 32 + threadIdx.x, m1 = threadIdx.y;
  if (k2 >= NH) return;
  const float2 *Ek = E + (size_t)k * F + k2;
  float2 acc0 = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
  for (int k1 = 0; k1 < N; k1 += 2) {
    acc0 = cadd(acc0, cmulc(Ek[(size_t)k1 * NH], s_twc[(k1 * m1) % N]));
    acc1 = cadd(acc1, cmulc(Ek[(size_t)(k1 + 1) * NH], s_twc[((k1 + 1) * m1) % N]));
  }
  Y[((size_t)k * M + m1) * NH + k2] = cadd(acc0, acc1);
}

// V-step of Proposition 2 over the active size classes, one CTA per filter k:
// alpha_c = H(F_c^-1(D~_c + theta^_c)) from each class's Y_c, alpha = mean over
// classes (with one class, alpha_c itself), V_k = alpha / max(||alpha||, 1).
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
  const float sc = 1.0f / fmaxf(sqrtf(red[0]), 1.0f);
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
                          const float2 *__restrict__ Dcur) {
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
  if (mode == 0) {
    const float2 d = Dcur[o];
    const float2 t = th[o];
    th[o] = make_float2(t.x + d.x - acc.x, t.y + d.y - acc.y);
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
  return (size_t)tri_size(K) * sizeof(double2) + (size_t)K * sizeof(double2) + (size_t)K * sizeof(double) +
         (size_t)3 * K * sizeof(float2) + (size_t)kFoldChunk * K * sizeof(float2) + kFoldChunk * sizeof(float2);
}

// threads: 256 or 512 (CTA size of the per-frequency factorisation; every
// entry sees the same operations in the same order either way).
cudaError_t launch_fold_factor(const FoldArgs &a, int threads, cudaStream_t s) {
  const size_t sm = fold_smem_bytes(a.K);
  cudaError_t e;
  if (threads == 512) {
    e = cudaFuncSetAttribute(fold_factor_kernel<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    fold_factor_kernel<512><<<a.F, 512, sm, s>>>(a);
  } else {
    e = cudaFuncSetAttribute(fold_factor_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    fold_factor_kernel<256><<<a.F, 256, sm, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_dstep(int K, int F, float rho_eff, const float2 *X, const float2 *yb,
                         const float2 *Vh, const float2 *th, float2 *Dcur, float2 *E,
                         cudaStream_t s) {
  if (K > 256) return cudaErrorInvalidValue;
  const size_t sm = ((size_t)tri_stride(K) + 2 * (size_t)K) * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(dstep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const int threads = (K + 31) / 32 * 32;
  dstep_kernel<<<F, threads, sm, s>>>(K, F, rho_eff, X, yb, Vh, th, Dcur, E);
  return cudaGetLastError();
}

cudaError_t launch_vstep_cols(int K, int N, int M, const float2 *E, const float2 *tw, float2 *Y,
                              cudaStream_t s) {
  if (M > kMaxM || N > kMaxFFT) return cudaErrorInvalidValue;
  dim3 grid(K, (N / 2 + 1 + 31) / 32), block(32, M);
  vstep_cols_kernel<<<grid, block, N * sizeof(float2), s>>>(K, N, M, E, tw, Y);
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
                                  float2 *Vh, float2 *th, const float2 *Dcur, cudaStream_t s) {
  if (M > kMaxM || N > kMaxFFT) return cudaErrorInvalidValue;
  const int F = N * (N / 2 + 1);
  dim3 grid(K, (F + 255) / 256);
  vstep_spectrum_kernel<<<grid, 256, 0, s>>>(mode, K, N, M, Tm, tw, Vh, th, Dcur);
  return cudaGetLastError();
}

cudaError_t launch_dict_norms(int K, int F, const float2 *Dh, float *dn, cudaStream_t s) {
  dict_norms_kernel<<<(F + 255) / 256, 256, 0, s>>>(K, F, Dh, dn);
  return cudaGetLastError();
}

}  // namespace ocsc
