// Per-sample code ADMM in the frequency domain (Sec. II-C.1, problem
// (fcsc_code), with the scaled-dual ADMM template of Sec. II-B).
//
// One iteration, with W^ = F(U - Gamma), for every frequency p of the half
// spectrum and d = D~(p,:)^T:
//   Z~-step: (conj(d) d^T + rho I) z = conj(d) x~(p) + rho w^(p).  The matrix
//            is rank one plus rho*I; by Sherman-Morrison the solution is
//            z = w^ + conj(d) r_p  with  r_p = (x~(p) - d^T w^) / (rho + |d|^2).
//   Z       = F^-1(Z~)
//   U       = S_{lambda/rho}(Z + Gamma)          (soft threshold)
//   Gamma   = Gamma + Z - U
// The only coupling across filters is r_p (a reduction over k at each p); the
// only coupling across frequencies is the FFT of each filter plane.  So each
// iteration is two kernels:
//   code_resid  -- r_p for every (sample, p): reduce d_k w^_k over k;
//   code_plane  -- one CTA per (sample, filter): build z on the half
//                  spectrum in shared memory, real inverse 2D FFT (column
//                  transforms, then half-length transforms of the packed
//                  rows), shrink + dual update on pairs of pixels, forward
//                  real 2D FFT of W = U - Gamma back to the half spectrum.
//                  Gamma is the only spatial array that goes to global memory.
//                  Every pass moves the whole tile through registers, so the
//                  kernel is fused to as few passes as the transforms allow:
//                  the column packing rides on the first column pass, the
//                  last pass of each transform is done in place without a
//                  barrier, and for N = 128 the c2r split rides on the first
//                  row pass, the spatial step sits between the last inverse
//                  and the first forward row pass on each thread's registers,
//                  the r2c split rides on the last row pass and the last
//                  column pass stores W^ to global memory itself.
#include "plane_bodies.cuh"

namespace ocsc {

// x~ = F(zero-padded image): one CTA per image.
template <int N>
__global__ void __launch_bounds__(TileThreads<N>::value)
    image_spectrum_kernel(ImgBatch b, const float2 *__restrict__ tw, float2 *__restrict__ xh) {
  constexpr int NT = TileThreads<N>::value, PITCH = tile_pitch<N>(), NH = N / 2 + 1;
  constexpr int F = N * NH;
  extern __shared__ float2 smem[];
  float2 *tile = smem;
  float2 *s_tw = smem + N * PITCH;
  const int img = blockIdx.x;
  const float *x = b.x[img];
  const int H = b.H[img], W = b.W[img];
  load_twiddles<N, NT>(s_tw, tw);
  for (int q = threadIdx.x; q < N * N; q += NT) {
    const int q1 = q / N, q2 = q % N;
    const float v = (q1 < H && q2 < W) ? x[q1 * W + q2] : 0.0f;
    tile[q1 * PITCH + q2] = make_float2(v, 0.0f);
  }
  __syncthreads();
  fft2d_tile<N, NT, false>(tile, s_tw);
  float2 *out = xh + (size_t)b.slot[img] * F;
  for (int p = threadIdx.x; p < F; p += NT) {
    const int k1 = p / NH, k2 = p % NH;
    out[p] = tile[k1 * PITCH + k2];
  }
}

// r_p = (x~(p) - sum_k D~_k(p) W^_k(p)) / (rho + |d_p|^2); block (32, 8).
__global__ void code_resid_kernel(int K, int F, float rho, int first, int serve, ImgBatch b,
                                  const float2 *__restrict__ Dh, const float *__restrict__ dn,
                                  const float2 *__restrict__ xh, const float2 *__restrict__ What,
                                  float2 *__restrict__ r) {
  code_resid_body(K, F, rho, first, serve, b, Dh, dn, xh, What, r, blockIdx.x, blockIdx.y, threadIdx.x, threadIdx.y);
}

// One fused ADMM iteration for filter k of one sample (grid: K x images).
// NT threads per CTA (256; 512 for N = 128), MINB the number of CTAs per SM
// the register budget is sized for (256 threads: 2, no spills, or 3, a few
// spilled registers; 512 threads: 2, with half the values per thread); every
// form performs the same operations in the same order.  SERVE selects the
// serving form of the body.
template <int N, int MINB, bool SERVE, int NT>
__global__ void __launch_bounds__(NT, MINB)
    code_plane_kernel(CodeIter it, ImgBatch b, const float2 *__restrict__ tw) {
  extern __shared__ __align__(16) float4 hsmem[];
  const int pre = it.ahead > 0 ? (int)(blockIdx.y * gridDim.x + blockIdx.x) + it.ahead : -1;
  code_plane_body<N, SERVE, NT>(it, b, tw, blockIdx.x, blockIdx.y, hsmem,
                                pre < (int)(gridDim.x * gridDim.y) ? pre : -1);
}

// N = 128, batch form: persistent CTAs of NT threads, one per SM, each with
// two tiles.  CTA c takes the units (image, filter) c, c + gridDim.x, ...;
// while it works on one unit the W^ copies of its next unit fill the other
// tile (committed at the unit's start, waited for at the next one's).
template <int NT>
__global__ void __launch_bounds__(NT, 1) code_plane_persist_kernel(CodeIter it, ImgBatch b, const float2 *__restrict__ tw) {
  constexpr int N = 128, F = N * (N / 2 + 1), F2 = F / 2;
  extern __shared__ __align__(16) float4 hsmem[];
  float2 *s_tw = reinterpret_cast<float2 *>(hsmem);  // [N], then two [N][N/2+1] tiles
  float2 *tiles[2] = {s_tw + N, s_tw + N + F};
  load_twiddles<N, NT>(s_tw, tw);  // read after the first unit's first barrier
  const int K = it.K, total = K * b.n, G = gridDim.x;
  const bool read_w = it.first == 0;
  auto w_of = [&](int u) { return it.What + ((size_t)b.slot[u / K] * K + u % K) * F; };
  int u = blockIdx.x;
  if (u < total && read_w) {
    const float4 *src = reinterpret_cast<const float4 *>(w_of(u));
    float4 *dst = reinterpret_cast<float4 *>(tiles[0]);
    for (int c = threadIdx.x; c < F2; c += NT) cp_async16(dst + c, src + c);
    cp_async_commit();
  }
  for (int buf = 0; u < total; u += G, buf ^= 1) {
    const int nu = u + G;
    const float2 *nw = read_w && nu < total ? w_of(nu) : nullptr;
    code_plane_body<N, false, NT>(it, b, tw, u % K, u / K, hsmem, -1, tiles[buf], s_tw, read_w, nw,
                                  tiles[buf ^ 1]);
    __syncthreads();  // this tile is the copy target two units on
  }
}

// Building block: batched real 2D FFT (pairs of planes share one complex FFT).
template <int N, bool INV>
__global__ void __launch_bounds__(TileThreads<N>::value)
    fft2_pair_kernel(const float *__restrict__ in, float *__restrict__ out, int planes,
                     const float2 *__restrict__ tw) {
  constexpr int NT = TileThreads<N>::value, PITCH = tile_pitch<N>(), NH = N / 2 + 1;
  constexpr int F = N * NH, P = N * N;
  extern __shared__ float2 smem[];
  float2 *tile = smem;
  float2 *s_tw = smem + N * PITCH;
  const int pa = 2 * blockIdx.x, pb = pa + 1;
  const bool hasb = pb < planes;
  load_twiddles<N, NT>(s_tw, tw);
  if (!INV) {
    const float *xa = in + (size_t)pa * P;
    const float *xb = in + (size_t)pb * P;
    for (int q = threadIdx.x; q < P; q += NT)
      tile[(q / N) * PITCH + (q % N)] = make_float2(xa[q], hasb ? xb[q] : 0.f);
    __syncthreads();
    fft2d_tile<N, NT, false>(tile, s_tw);
    float2 *Xa = reinterpret_cast<float2 *>(out) + (size_t)pa * F;
    float2 *Xb = reinterpret_cast<float2 *>(out) + (size_t)pb * F;
    for (int p = threadIdx.x; p < F; p += NT) {
      const int k1 = p / NH, k2 = p % NH;
      const float2 c = tile[k1 * PITCH + k2];
      const float2 cm = tile[((N - k1) & (N - 1)) * PITCH + ((N - k2) & (N - 1))];
      Xa[p] = make_float2(0.5f * (c.x + cm.x), 0.5f * (c.y - cm.y));
      if (hasb) Xb[p] = make_float2(0.5f * (c.y + cm.y), -0.5f * (c.x - cm.x));
    }
  } else {
    const float2 *Xa = reinterpret_cast<const float2 *>(in) + (size_t)pa * F;
    const float2 *Xb = reinterpret_cast<const float2 *>(in) + (size_t)pb * F;
    for (int p = threadIdx.x; p < F; p += NT) {
      const int k1 = p / NH, k2 = p % NH;
      const float2 za = Xa[p];
      const float2 zb = hasb ? Xb[p] : make_float2(0.f, 0.f);
      tile[k1 * PITCH + k2] = make_float2(za.x - zb.y, za.y + zb.x);
      if (k2 > 0 && k2 < N / 2)
        tile[((N - k1) & (N - 1)) * PITCH + (N - k2)] = make_float2(za.x + zb.y, zb.x - za.y);
    }
    __syncthreads();
    fft2d_tile<N, NT, true>(tile, s_tw);
    const float invP = 1.0f / (float)P;
    float *xa = out + (size_t)pa * P;
    float *xb = out + (size_t)pb * P;
    for (int q = threadIdx.x; q < P; q += NT) {
      const float2 c = tile[(q / N) * PITCH + (q % N)];
      xa[q] = c.x * invP;
      if (hasb) xb[q] = c.y * invP;
    }
  }
}

// Per-slot residual sums in double, in a fixed order: out[i][q] = sum over the
// slot's partial groups of partials[slot][g][q].
__global__ void resid_reduce_kernel(const int *__restrict__ slots, int n, int groups,
                                    const float *__restrict__ partials, double *__restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * kResidTerms) return;
  const int img = i / kResidTerms, q = i % kResidTerms;
  const float *p = partials + (size_t)slots[img] * groups * kResidTerms + q;
  double s = 0.0;
  for (int g = 0; g < groups; ++g) s += (double)p[(size_t)g * kResidTerms];
  out[i] = s;
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------

cudaError_t launch_resid_reduce(const int *slots_dev, int n, int groups, const float *partials,
                                double *out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int total = n * kResidTerms;
  resid_reduce_kernel<<<(total + 127) / 128, 128, 0, s>>>(slots_dev, n, groups, partials, out);
  return cudaGetLastError();
}

template <typename Kern>
static cudaError_t set_smem(Kern k, size_t bytes) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int N>
static cudaError_t image_spectrum_n(const ImgBatch &b, const float2 *tw, float2 *xh, cudaStream_t s) {
  const size_t sm = tile_smem_bytes<N>();
  cudaError_t e = set_smem(image_spectrum_kernel<N>, sm);
  if (e != cudaSuccess) return e;
  image_spectrum_kernel<N><<<b.n, TileThreads<N>::value, sm, s>>>(b, tw, xh);
  return cudaGetLastError();
}

cudaError_t launch_image_spectrum(int N, const ImgBatch &b, const float2 *tw, float2 *xh,
                                  cudaStream_t s) {
  if (b.n <= 0) return cudaSuccess;
  switch (N) {
    case 64: return image_spectrum_n<64>(b, tw, xh, s);
    case 128: return image_spectrum_n<128>(b, tw, xh, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_code_resid(int N, const ImgBatch &b, const CodeIter &it, float rho, const float *dn,
                              const float2 *xh, cudaStream_t s) {
  if (b.n <= 0) return cudaSuccess;
  const int F = N * (N / 2 + 1);
  dim3 grid((F + kResidBins - 1) / kResidBins, b.n), block(32, 8);
  code_resid_kernel<<<grid, block, 0, s>>>(it.K, F, rho, it.first, it.serve, b, it.Dh, dn, xh, it.What, it.r);
  return cudaGetLastError();
}

template <int N, int MINB, bool SERVE, int NT>
static cudaError_t code_plane_nms(const CodeIter &it, const ImgBatch &b, const float2 *tw, cudaStream_t s) {
  const size_t sm = half_smem_bytes<N>();
  cudaError_t e = set_smem(code_plane_kernel<N, MINB, SERVE, NT>, sm);
  if (e != cudaSuccess) return e;
  dim3 grid(it.K, b.n);
  code_plane_kernel<N, MINB, SERVE, NT><<<grid, NT, sm, s>>>(it, b, tw);
  return cudaGetLastError();
}

// CTAs of the plane kernel resident at once with MINB per SM: the distance
// of its L2 prefetch.
static int plane_resident(int minb) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  return sms * minb;
}

template <int N, int MINB, int NT = 256>
static cudaError_t code_plane_n(const CodeIter &it, const ImgBatch &b, const float2 *tw, cudaStream_t s) {
  return it.serve ? code_plane_nms<N, MINB, true, NT>(it, b, tw, s) : code_plane_nms<N, MINB, false, NT>(it, b, tw, s);
}

int plane_resid_groups(int K) { return K; }

bool plane_shape_ok(int N, int threads, int ctas) {
  if (N != 64 && N != 128) return false;
  if (threads == 256) return ctas == 2 || ctas == 3;
  return N == 128 && threads == 512 && (ctas == 2 || ctas == 1);
}

// The persistent two-tile form (512 threads, one CTA per SM), batch form only.
static cudaError_t code_plane_persist(const CodeIter &it, const ImgBatch &b, const float2 *tw, cudaStream_t s) {
  constexpr int N = 128, F = N * (N / 2 + 1);
  const size_t sm = (size_t)(N + 2 * F) * sizeof(float2);
  cudaError_t e = set_smem(code_plane_persist_kernel<512>, sm);
  if (e != cudaSuccess) return e;
  int per_sm = 0, dev = 0, sms = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, code_plane_persist_kernel<512>, 512, sm);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int total = it.K * b.n, grid = total < per_sm * sms ? total : per_sm * sms;
  code_plane_persist_kernel<512><<<grid, 512, sm, s>>>(it, b, tw);
  return cudaGetLastError();
}

cudaError_t launch_code_plane(int N, const CodeIter &it, const ImgBatch &b, const float2 *tw,
                              cudaStream_t s, int ctas, bool ahead, int threads) {
  if (b.n <= 0) return cudaSuccess;
  if (!plane_shape_ok(N, threads, ctas)) return cudaErrorInvalidValue;
  CodeIter ia = it;
  if (threads == 512 && ctas == 1) {
    ia.ahead = 0;
    if (!it.serve) return code_plane_persist(ia, b, tw, s);
    ctas = 2;  // the serving form has no persistent variant
  }
  ia.ahead = ahead ? plane_resident(ctas) : 0;
  if (threads == 512) return code_plane_n<128, 2, 512>(ia, b, tw, s);
  const bool three = ctas == 3;
  if (N == 64) return three ? code_plane_n<64, 3>(ia, b, tw, s) : code_plane_n<64, 2>(ia, b, tw, s);
  return three ? code_plane_n<128, 3>(ia, b, tw, s) : code_plane_n<128, 2>(ia, b, tw, s);
}

template <int N, bool INV>
static cudaError_t fft2_n(const float *in, float *out, int planes, const float2 *tw, cudaStream_t s) {
  const size_t sm = tile_smem_bytes<N>();
  cudaError_t e = set_smem(fft2_pair_kernel<N, INV>, sm);
  if (e != cudaSuccess) return e;
  fft2_pair_kernel<N, INV><<<(planes + 1) / 2, TileThreads<N>::value, sm, s>>>(in, out, planes, tw);
  return cudaGetLastError();
}

cudaError_t launch_fft2(int N, int inverse, const float *in, float *out, int planes,
                        const float2 *tw, cudaStream_t s) {
  if (planes <= 0) return cudaSuccess;
  if (N == 64) return inverse ? fft2_n<64, true>(in, out, planes, tw, s) : fft2_n<64, false>(in, out, planes, tw, s);
  if (N == 128) return inverse ? fft2_n<128, true>(in, out, planes, tw, s) : fft2_n<128, false>(in, out, planes, tw, s);
  return cudaErrorInvalidValue;
}

}  // namespace ocsc
