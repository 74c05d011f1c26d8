// Allocation-free coding entry point (ocsc_code_noalloc).
//
// Some callers cannot allocate device memory when they code an image: a plug-in
// whose host application has already reserved the whole device through its own
// allocator, a latency-sensitive pipeline that cannot afford the device-wide
// synchronisation that cudaMalloc / cudaFree can imply while other streams run,
// or a deployment that must not fail at run time for lack of memory and so
// takes everything it needs at start-up.  For them this file keeps the scratch
// of one coding call in a fixed file-scope device array and runs the same
// kernels as ocsc_code on it.  The caller still provides the image, the filters
// and the output buffer.
//
// The array below is part of this file's module.  Under CUDA's default lazy
// module loading the module (with the array) and the coding kernels are loaded
// on the first call on each device, and loading can itself take device memory;
// after that, the array stays resident on that device until the process exits.
// A caller that must never allocate after start-up therefore makes one call at
// start-up (or runs with CUDA_MODULE_LOADING=EAGER).  All calls share the array
// and it keeps whatever the last call left there; nothing has to start at zero
// because the twiddles are rewritten by every call and the first ADMM
// iteration reads no earlier state.  Two calls whose work overlaps on the GPU
// (other streams, other host threads) overwrite each other's scratch:
// serialise them.
#include <cmath>
#include <cstdarg>
#include <cstdio>

#include "../../include/ocsc.h"
#include "common.cuh"
#include "launch.h"

using namespace ocsc;

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[OCSC_NOALLOC_SCRATCH_BYTES];

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Carve {
  size_t tw, Tm, Dh, dn, xh, r, What, Zp, Gam, total;
};

Carve carve(int K, int N) {
  const size_t F = (size_t)N * (N / 2 + 1), P = (size_t)N * N;
  Carve c{};
  size_t o = 0;
  c.tw = o;   o += up256(N * sizeof(float2));
  c.Tm = o;   o += up256((size_t)K * 16 * (N / 2 + 1) * sizeof(float2));
  c.Dh = o;   o += up256(K * F * sizeof(float2));
  c.dn = o;   o += up256(F * sizeof(float));
  c.xh = o;   o += up256(F * sizeof(float2));
  c.r = o;    o += up256(F * sizeof(float2));
  c.What = o; o += up256(K * F * sizeof(float2));
  c.Zp = o;   o += up256(K * F * sizeof(float2));
  c.Gam = o;  o += up256(K * P * sizeof(float));
  c.total = o;
  return c;
}

// W_N^m = exp(-2 pi i m / N) for m < N, evaluated in double and rounded once
// to float, as the context path's host table is.
__global__ void noalloc_twiddles_kernel(int N, float2 *tw) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= N) return;
  const double a = -2.0 * 3.14159265358979323846 * (double)m / (double)N;
  tw[m] = make_float2((float)cos(a), (float)sin(a));
}

ocsc_status say(char *err, size_t len, ocsc_status s, const char *fmt, ...) {
  if (err && len > 0) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(err, len, fmt, ap);
    va_end(ap);
  }
  return s;
}

}  // namespace

extern "C" ocsc_status ocsc_code_noalloc(const float *x, int H, int W, const float *D, int K, int M,
                                         int N, double lambda, double rho, int Jz, float *u,
                                         void *cuda_stream, char *err, size_t err_len) {
  if (err && err_len > 0) err[0] = '\0';
  if (!x || !D || !u) return say(err, err_len, OCSC_EINVAL, "null image, filter or output pointer");
  if (reinterpret_cast<uintptr_t>(u) % 16 != 0)
    return say(err, err_len, OCSC_EINVAL, "the code buffer must be 16-byte aligned");
  if (N != 64 && N != 128) return say(err, err_len, OCSC_EUNSUPPORTED, "N=%d: only 64 or 128", N);
  if (H <= 0 || W <= 0 || H > N || W > N)
    return say(err, err_len, OCSC_EINVAL, "image %dx%d does not fit the %dx%d domain", H, W, N, N);
  if (K <= 0 || K > 128 || M <= 0 || M > 16 || M > N)
    return say(err, err_len, OCSC_EUNSUPPORTED, "K=%d, M=%d outside 1..128 and 1..16", K, M);
  if (!(lambda >= 0) || !(rho > 0) || Jz < 1)
    return say(err, err_len, OCSC_EINVAL, "need lambda >= 0, rho > 0, Jz >= 1");
  const Carve cv = carve(K, N);
  if (cv.total > (size_t)OCSC_NOALLOC_SCRATCH_BYTES)
    return say(err, err_len, OCSC_EUNSUPPORTED,
               "K=%d at N=%d needs %zu bytes of scratch; the fixed array holds %zu", K, N, cv.total,
               (size_t)OCSC_NOALLOC_SCRATCH_BYTES);

  // The array's device address, looked up on every call with the caller's
  // device current: host code only sees a host-side stand-in for the symbol,
  // and the address belongs to the current context (a context created anew,
  // for instance after cudaDeviceReset, may place the module elsewhere).
  void *p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return say(err, err_len, OCSC_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
  unsigned char *base = static_cast<unsigned char *>(p);

  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int F = N * (N / 2 + 1);
  float2 *tw = reinterpret_cast<float2 *>(base + cv.tw);
  float2 *Dh = reinterpret_cast<float2 *>(base + cv.Dh);
  float *dn = reinterpret_cast<float *>(base + cv.dn);
  float2 *xh = reinterpret_cast<float2 *>(base + cv.xh);
  float2 *r = reinterpret_cast<float2 *>(base + cv.r);

  noalloc_twiddles_kernel<<<(N + 127) / 128, 128, 0, s>>>(N, tw);
  e = cudaGetLastError();
  // D~ = F(pad D) and |D~(p,:)|^2, then the same code-ADMM launches as ocsc_code.
  float2 *Tm = reinterpret_cast<float2 *>(base + cv.Tm);
  if (e == cudaSuccess) e = launch_vstep_partial_dft(K, N, M, D, tw, Tm, s);
  if (e == cudaSuccess) e = launch_vstep_spectrum(1, K, N, M, Tm, tw, Dh, nullptr, nullptr, s);
  if (e == cudaSuccess) e = launch_dict_norms(K, F, Dh, dn, s);
  ImgBatch b{};
  b.n = 1;
  b.x[0] = x;
  b.u[0] = u;
  b.H[0] = H;
  b.W[0] = W;
  b.slot[0] = 0;
  b.iter[0] = 0;
  if (e == cudaSuccess) e = launch_image_spectrum(N, b, tw, xh, s);
  CodeIter it{};
  it.K = K;
  it.F = F;
  it.thr = (float)(lambda / rho);
  it.Dh = Dh;
  it.r = r;
  it.What = reinterpret_cast<float2 *>(base + cv.What);
  it.Gam = reinterpret_cast<float *>(base + cv.Gam);
  it.Zp = reinterpret_cast<float2 *>(base + cv.Zp);
  for (int t = 0; t < Jz && e == cudaSuccess; ++t) {
    it.first = t == 0;
    it.last = t == Jz - 1;
    e = launch_code_resid(N, b, it, (float)rho, dn, xh, s);
    if (e == cudaSuccess) e = launch_code_plane(N, it, b, tw, s);
  }
  if (e != cudaSuccess) return say(err, err_len, OCSC_ECUDA, "launch: %s", cudaGetErrorString(e));
  return OCSC_OK;
}
