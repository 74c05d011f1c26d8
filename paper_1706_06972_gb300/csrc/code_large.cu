// Code ADMM for FFT sizes whose packed N x N complex plane does not fit one
// CTA's shared memory (N = 256, 512).  The iteration is the one of
// code_admm.cu (Sec. II-C.1 problem (fcsc_code), ADMM of Sec. II-B) with the 2D
// transforms split by dimension around a per-(sample, filter pair) complex tile
// T[N][N] in global memory:
//   col_in  : per block of CB half-spectrum columns k2 and their mirrors N-k2,
//             the Z~-step z = w^ + conj(d) r for both filters of the pair,
//             packed as z_a + i z_b over the full spectrum, inverse FFT along k1;
//   rows    : per block of RB rows, inverse FFT along k2, the spatial step
//             U = S(Z + Gamma), Gamma += Z - U, W = U - Gamma, forward FFT
//             along the row;
//   col_out : per column block, forward FFT along k1 and the split of the
//             packed spectrum into the two half spectra W^_a, W^_b.
// The same kernels with other modes give the sample spectrum and the batched
// real 2D FFT building blocks.  Every block uses 64 KB of lines plus twiddles.
#include "fft.cuh"
#include "launch.h"

namespace ocsc {

constexpr int kLargeThreads = 256;
template <int N> struct LargeGeom {
  static constexpr int NH = N / 2 + 1, F = N * NH, P = N * N;
  static constexpr int CB = 4096 / N;          // half-spectrum columns per column block
  static constexpr int NL = 2 * CB;            // lines per column block (with mirrors)
  static constexpr int RB = 8192 / N;          // rows per row block
  static constexpr int NBLK = (NH + CB - 1) / CB;
  static constexpr int PITCH = N + 1;
};

template <int N>
size_t large_smem_bytes() {
  using G = LargeGeom<N>;
  const int lines = G::NL > G::RB ? G::NL : G::RB;
  return (size_t)lines * G::PITCH * sizeof(float2) + (size_t)N * sizeof(float2);
}

__device__ __forceinline__ float soft_thr(float v, float t) { return v > t ? v - t : (v < -t ? v + t : 0.0f); }

// Sum kResidTerms values over a block; thread 0 writes them to out.
__device__ __forceinline__ void block_terms(float (&v)[kResidTerms], float *out) {
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

// Column-block source / destination of line l: half-spectrum column c0 + l for
// l < CB, mirror column N - (c0 + l - CB) otherwise; -1 when it does not exist.
template <int N>
__device__ __forceinline__ int line_column(int c0, int l) {
  using G = LargeGeom<N>;
  if (l < G::CB) {
    const int k2 = c0 + l;
    return k2 <= N / 2 ? k2 : -1;
  }
  const int k2 = c0 + l - G::CB;
  return (k2 > 0 && k2 < N / 2) ? N - k2 : -1;
}

// MODE 0: Z~-step of the ADMM; MODE 1: given half spectra Xa, Xb (c2r).
template <int N, int MODE>
__global__ void __launch_bounds__(kLargeThreads)
    large_col_in_kernel(CodeIter it, ImgBatch b, LargeIO io, const float2 *__restrict__ tw) {
  using G = LargeGeom<N>;
  extern __shared__ float2 lsm[];
  float2 *lines = lsm;
  float2 *s_tw = lsm + (G::NL > G::RB ? G::NL : G::RB) * G::PITCH;
  for (int i = threadIdx.x; i < N; i += kLargeThreads) s_tw[i] = tw[i];
  const int c0 = blockIdx.x * G::CB;
  const int pair = blockIdx.y, img = blockIdx.z;
  const int ka = 2 * pair, kb = ka + 1;
  const int npairs = gridDim.y;
  const int K = MODE == 0 ? it.K : io.planes;
  const bool hasb = kb < K;
  const int slot = MODE == 0 ? b.slot[img] : img;
  const int t = MODE == 0 ? b.iter[img] : 0;
  const bool first = it.serve ? t == 0 : it.first != 0;
  const bool store_last = it.serve ? (t + 1) % it.check == 0 : it.last != 0;
  const float2 *Da = nullptr, *Db = nullptr, *rr = nullptr;
  const float2 *Wa = nullptr, *Wb = nullptr;
  float2 *Za = nullptr, *Zb = nullptr;
  const float2 *Xa = nullptr, *Xb = nullptr;
  if (MODE == 0) {
    Da = it.Dh + (size_t)ka * G::F;
    Db = it.Dh + (size_t)(hasb ? kb : ka) * G::F;
    rr = it.r + (size_t)slot * G::F;
    Wa = it.What + ((size_t)slot * K + ka) * G::F;
    Wb = it.What + ((size_t)slot * K + (hasb ? kb : ka)) * G::F;
    Za = it.Zp + ((size_t)slot * K + ka) * G::F;
    Zb = it.Zp + ((size_t)slot * K + (hasb ? kb : ka)) * G::F;
  } else {
    Xa = io.spec_in + (size_t)ka * G::F;
    Xb = io.spec_in + (size_t)(hasb ? kb : ka) * G::F;
  }
  for (int e = threadIdx.x; e < N * G::CB; e += kLargeThreads) {
    const int k1 = e / G::CB, l = e % G::CB;
    const int k2 = c0 + l;
    if (k2 > N / 2) continue;
    const int p = k1 * G::NH + k2;
    float2 za, zb = make_float2(0.f, 0.f);
    if (MODE == 0) {
      const float2 rp = rr[p];
      za = cconjmul(Da[p], rp);
      if (hasb) zb = cconjmul(Db[p], rp);
      if (!first) {
        za = cadd(za, Wa[p]);
        if (hasb) zb = cadd(zb, Wb[p]);
      }
      if (store_last) {
        Za[p] = za;
        if (hasb) Zb[p] = zb;
      }
    } else {
      za = Xa[p];
      if (hasb) zb = Xb[p];
    }
    lines[l * G::PITCH + k1] = make_float2(za.x - zb.y, za.y + zb.x);
    if (k2 > 0 && k2 < N / 2)
      lines[(G::CB + l) * G::PITCH + (N - k1) % N] = make_float2(za.x + zb.y, zb.x - za.y);
  }
  __syncthreads();
  fft_lines<N, G::NL, true, kLargeThreads>(lines, G::PITCH, s_tw);
  float2 *T = io.T + ((size_t)slot * npairs + pair) * G::P;
  for (int e = threadIdx.x; e < N * G::NL; e += kLargeThreads) {
    const int q1 = e / G::NL, l = e % G::NL;
    const int col = line_column<N>(c0, l);
    if (col >= 0) T[(size_t)q1 * N + col] = lines[l * G::PITCH + q1];
  }
}

// MODE 0: spatial ADMM step between the inverse and forward row transforms.
// MODE 1: real planes (or zero-padded images) in, forward row transforms out.
// MODE 2: inverse row transforms, real planes out (c2r).
template <int N, int MODE>
__global__ void __launch_bounds__(kLargeThreads)
    large_rows_kernel(CodeIter it, ImgBatch b, LargeIO io, const float2 *__restrict__ tw) {
  using G = LargeGeom<N>;
  extern __shared__ float2 lsm[];
  float2 *lines = lsm;
  float2 *s_tw = lsm + (G::NL > G::RB ? G::NL : G::RB) * G::PITCH;
  for (int i = threadIdx.x; i < N; i += kLargeThreads) s_tw[i] = tw[i];
  const int q0 = blockIdx.x * G::RB;
  const int pair = blockIdx.y, img = blockIdx.z;
  const int npairs = gridDim.y;
  const int slot = (MODE == 0 || io.images) ? b.slot[img] : img;
  float2 *T = io.T + ((size_t)slot * npairs + pair) * G::P;
  if (MODE == 1) {
    if (io.images) {  // sample spectrum: image img, zero-padded, as the real part
      const float *x = b.x[img];
      const int H = b.H[img], W = b.W[img];
      for (int e = threadIdx.x; e < G::RB * N; e += kLargeThreads) {
        const int rrow = e / N, q2 = e % N, q1 = q0 + rrow;
        const float v = (q1 < H && q2 < W) ? x[(size_t)q1 * W + q2] : 0.f;
        lines[rrow * G::PITCH + q2] = make_float2(v, 0.f);
      }
    } else {          // planes 2 pair and 2 pair + 1 as real and imaginary parts
      const int pa = 2 * pair, pb = pa + 1;
      const bool hasb = pb < io.planes;
      const float *xa = io.real_in + (size_t)pa * G::P;
      const float *xb = io.real_in + (size_t)pb * G::P;
      for (int e = threadIdx.x; e < G::RB * N; e += kLargeThreads) {
        const int rrow = e / N, q2 = e % N;
        const size_t o = (size_t)(q0 + rrow) * N + q2;
        lines[rrow * G::PITCH + q2] = make_float2(xa[o], hasb ? xb[o] : 0.f);
      }
    }
    __syncthreads();
    fft_lines<N, G::RB, false, kLargeThreads>(lines, G::PITCH, s_tw);
  } else {
    for (int e = threadIdx.x; e < G::RB * N; e += kLargeThreads) {
      const int rrow = e / N, q2 = e % N;
      lines[rrow * G::PITCH + q2] = T[(size_t)(q0 + rrow) * N + q2];
    }
    __syncthreads();
    fft_lines<N, G::RB, true, kLargeThreads>(lines, G::PITCH, s_tw);
    const float invP = 1.0f / (float)G::P;
    if (MODE == 2) {
      const int pa = 2 * pair, pb = pa + 1;
      const bool hasb = pb < io.planes;
      float *xa = io.real_out + (size_t)pa * G::P;
      float *xb = io.real_out + (size_t)pb * G::P;
      for (int e = threadIdx.x; e < G::RB * N; e += kLargeThreads) {
        const int rrow = e / N, q2 = e % N;
        const size_t o = (size_t)(q0 + rrow) * N + q2;
        const float2 c = lines[rrow * G::PITCH + q2];
        xa[o] = c.x * invP;
        if (hasb) xb[o] = c.y * invP;
      }
      return;
    }
    const int K = it.K, ka = 2 * pair, kb = ka + 1;
    const bool hasb = kb < K;
    const int t = b.iter[img];
    const bool first = it.serve ? t == 0 : it.first != 0;
    const bool store_last = it.serve ? (t + 1) % it.check == 0 : it.last != 0;
    const bool store_prev = it.serve && (t + 2) % it.check == 0;
    const bool skip_fwd = !it.serve && it.last;
    const bool resid = it.serve && store_last;
    float *Ga = it.Gam + ((size_t)slot * K + ka) * G::P;
    float *Gb = it.Gam + ((size_t)slot * K + (hasb ? kb : ka)) * G::P;
    float *Ua = b.u[img] ? b.u[img] + (size_t)ka * G::P : nullptr;
    float *Ub = (b.u[img] && hasb) ? b.u[img] + (size_t)kb * G::P : nullptr;
    float acc[kResidTerms] = {0.f, 0.f, 0.f, 0.f, 0.f};
    for (int e = threadIdx.x; e < G::RB * N; e += kLargeThreads) {
      const int rrow = e / N, q2 = e % N;
      const size_t o = (size_t)(q0 + rrow) * N + q2;
      const float2 c = lines[rrow * G::PITCH + q2];
      const float ga = first ? 0.f : Ga[o];
      const float gb = (first || !hasb) ? 0.f : Gb[o];
      const float za = c.x * invP, zb = c.y * invP;
      const float va = za + ga, vb = zb + gb;
      const float ua = soft_thr(va, it.thr), ub = soft_thr(vb, it.thr);
      const float ga2 = va - ua, gb2 = vb - ub;
      if (resid) {
        const float pa = (first || !Ua) ? 0.f : Ua[o];
        const float pb = (first || !Ub) ? 0.f : Ub[o];
        acc[0] += (za - ua) * (za - ua) + (hasb ? (zb - ub) * (zb - ub) : 0.f);
        acc[1] += za * za + (hasb ? zb * zb : 0.f);
        acc[2] += ua * ua + (hasb ? ub * ub : 0.f);
        acc[3] += (ua - pa) * (ua - pa) + (hasb ? (ub - pb) * (ub - pb) : 0.f);
        acc[4] += ga2 * ga2 + (hasb ? gb2 * gb2 : 0.f);
      }
      Ga[o] = ga2;
      if (hasb) Gb[o] = gb2;
      if (store_last || store_prev) {
        if (Ua) Ua[o] = ua;
        if (Ub) Ub[o] = ub;
      }
      if (!skip_fwd) lines[rrow * G::PITCH + q2] = make_float2(ua - ga2, hasb ? ub - gb2 : 0.f);
    }
    if (resid)
      block_terms(acc, it.resid + (((size_t)slot * npairs + pair) * gridDim.x + blockIdx.x) * kResidTerms);
    if (skip_fwd) return;
    __syncthreads();
    fft_lines<N, G::RB, false, kLargeThreads>(lines, G::PITCH, s_tw);
  }
  for (int e = threadIdx.x; e < G::RB * N; e += kLargeThreads) {
    const int rrow = e / N, q2 = e % N;
    T[(size_t)(q0 + rrow) * N + q2] = lines[rrow * G::PITCH + q2];
  }
}

// MODE 0: W^_a, W^_b of the ADMM; MODE 1: half spectra of two real planes
// (r2c); MODE 2: the half spectrum of one real plane (sample spectrum).
template <int N, int MODE>
__global__ void __launch_bounds__(kLargeThreads)
    large_col_out_kernel(CodeIter it, ImgBatch b, LargeIO io, const float2 *__restrict__ tw) {
  using G = LargeGeom<N>;
  extern __shared__ float2 lsm[];
  float2 *lines = lsm;
  float2 *s_tw = lsm + (G::NL > G::RB ? G::NL : G::RB) * G::PITCH;
  for (int i = threadIdx.x; i < N; i += kLargeThreads) s_tw[i] = tw[i];
  const int c0 = blockIdx.x * G::CB;
  const int pair = blockIdx.y, img = blockIdx.z;
  const int npairs = gridDim.y;
  const int slot = (MODE == 0 || MODE == 2) ? b.slot[img] : img;
  const float2 *T = io.T + ((size_t)slot * npairs + pair) * G::P;
  constexpr int NLOAD = MODE == 2 ? G::CB : G::NL;
  for (int e = threadIdx.x; e < N * NLOAD; e += kLargeThreads) {
    const int q1 = e / NLOAD, l = e % NLOAD;
    const int col = line_column<N>(c0, l);
    lines[l * G::PITCH + q1] = col >= 0 ? T[(size_t)q1 * N + col] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  fft_lines<N, NLOAD, false, kLargeThreads>(lines, G::PITCH, s_tw);
  if (MODE == 2) {
    float2 *out = io.spec_out + (size_t)slot * G::F;
    for (int e = threadIdx.x; e < N * G::CB; e += kLargeThreads) {
      const int k1 = e / G::CB, l = e % G::CB, k2 = c0 + l;
      if (k2 <= N / 2) out[k1 * G::NH + k2] = lines[l * G::PITCH + k1];
    }
    return;
  }
  const int ka = 2 * pair, kb = ka + 1;
  const int K = MODE == 0 ? it.K : io.planes;
  const bool hasb = kb < K;
  float2 *Oa, *Ob;
  if (MODE == 0) {
    Oa = it.What + ((size_t)slot * K + ka) * G::F;
    Ob = it.What + ((size_t)slot * K + (hasb ? kb : ka)) * G::F;
  } else {
    Oa = io.spec_out + (size_t)ka * G::F;
    Ob = io.spec_out + (size_t)(hasb ? kb : ka) * G::F;
  }
  for (int e = threadIdx.x; e < N * G::CB; e += kLargeThreads) {
    const int k1 = e / G::CB, l = e % G::CB, k2 = c0 + l;
    if (k2 > N / 2) continue;
    const int m1 = (N - k1) % N;
    const float2 c = lines[l * G::PITCH + k1];
    const float2 cm = (k2 > 0 && k2 < N / 2) ? lines[(G::CB + l) * G::PITCH + m1] : lines[l * G::PITCH + m1];
    const int p = k1 * G::NH + k2;
    Oa[p] = make_float2(0.5f * (c.x + cm.x), 0.5f * (c.y - cm.y));
    if (hasb) Ob[p] = make_float2(0.5f * (c.y + cm.y), -0.5f * (c.x - cm.x));
  }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------

template <typename Kern>
static cudaError_t prep(Kern k, size_t sm) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
}

template <int N>
static cudaError_t large_n(int what, const CodeIter &it, const ImgBatch &b, const LargeIO &io, int n,
                           int npairs, const float2 *tw, cudaStream_t s) {
  using G = LargeGeom<N>;
  const size_t sm = large_smem_bytes<N>();
  cudaError_t e = cudaSuccess;
  const dim3 gc(G::NBLK, npairs, n), gr(N / G::RB, npairs, n);
  switch (what) {
    case LARGE_COL_IN_ADMM:
      if ((e = prep(large_col_in_kernel<N, 0>, sm)) != cudaSuccess) return e;
      large_col_in_kernel<N, 0><<<gc, kLargeThreads, sm, s>>>(it, b, io, tw);
      break;
    case LARGE_COL_IN_C2R:
      if ((e = prep(large_col_in_kernel<N, 1>, sm)) != cudaSuccess) return e;
      large_col_in_kernel<N, 1><<<gc, kLargeThreads, sm, s>>>(it, b, io, tw);
      break;
    case LARGE_ROWS_ADMM:
      if ((e = prep(large_rows_kernel<N, 0>, sm)) != cudaSuccess) return e;
      large_rows_kernel<N, 0><<<gr, kLargeThreads, sm, s>>>(it, b, io, tw);
      break;
    case LARGE_ROWS_FWD:
      if ((e = prep(large_rows_kernel<N, 1>, sm)) != cudaSuccess) return e;
      large_rows_kernel<N, 1><<<gr, kLargeThreads, sm, s>>>(it, b, io, tw);
      break;
    case LARGE_ROWS_C2R:
      if ((e = prep(large_rows_kernel<N, 2>, sm)) != cudaSuccess) return e;
      large_rows_kernel<N, 2><<<gr, kLargeThreads, sm, s>>>(it, b, io, tw);
      break;
    case LARGE_COL_OUT_ADMM:
      if ((e = prep(large_col_out_kernel<N, 0>, sm)) != cudaSuccess) return e;
      large_col_out_kernel<N, 0><<<gc, kLargeThreads, sm, s>>>(it, b, io, tw);
      break;
    case LARGE_COL_OUT_R2C:
      if ((e = prep(large_col_out_kernel<N, 1>, sm)) != cudaSuccess) return e;
      large_col_out_kernel<N, 1><<<gc, kLargeThreads, sm, s>>>(it, b, io, tw);
      break;
    case LARGE_COL_OUT_IMAGE:
      if ((e = prep(large_col_out_kernel<N, 2>, sm)) != cudaSuccess) return e;
      large_col_out_kernel<N, 2><<<gc, kLargeThreads, sm, s>>>(it, b, io, tw);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_large(int N, int what, const CodeIter &it, const ImgBatch &b, const LargeIO &io,
                         int n, int npairs, const float2 *tw, cudaStream_t s) {
  if (n <= 0 || npairs <= 0) return cudaSuccess;
  switch (N) {
    case 256: return large_n<256>(what, it, b, io, n, npairs, tw, s);
    case 512: return large_n<512>(what, it, b, io, n, npairs, tw, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ocsc
