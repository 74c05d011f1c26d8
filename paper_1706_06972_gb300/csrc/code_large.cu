// Code ADMM for FFT sizes whose packed N x N complex plane does not fit one
// CTA's shared memory, and for the sizes with a factor 3 (N = 96, 144, 192,
// 256, 288, 384, 512, 576).  The iteration is the one of
// code_admm.cu (Sec. II-C.1 problem (fcsc_code), ADMM of Sec. II-B):
//   W^ = F(U - Gamma),  z = w^ + conj(d) r,  r = (x~ - d^T w^) / (rho + |d|^2),
//   U' = S(Z + Gamma),  Gamma' = Gamma + Z - U'.
// With g = F^-1(conj(d) r) this is Z = U - Gamma + g, so V := Z + Gamma = U + g,
// U' = S(V), Gamma' = V - U' and the next W = U' - Gamma' = 2U' - V: the spatial
// state is U alone, and the spectral side only needs F(W) and produces g.
// The 2D transforms are split by dimension around a per-(sample, filter pair)
// complex tile M[k1][q2] in global memory.  Two kernels per iteration:
//
//   spectral (one CTA per row pair k1, -k1 of one sample, all filters):
//     pass 1: M holds the column transform of the packed pair w_a + i w_b;
//             its forward FFT along q2, split into the two half spectra,
//             gives s(p) = sum_k D~_k(p) W^_k(p) and
//             r(p) = (x~(p) - s(p)) / (rho + |d(p)|^2);
//     pass 2: M <- row inverse of the packed conj(d_a) r + i conj(d_b) r.  On
//             the iteration whose Z~ is kept, z = w^ + conj(d) r is also
//             written to the pending spectra.
//   spatial (one CTA per block of CB columns q2 of one pair of one sample):
//             the inverse FFT along k1 gives g; V = U + g, U' = S(V),
//             W = 2U' - V, and the forward FFT along q1 writes M for the next
//             iteration.  U is stored tiled by column block, so a CTA reads
//             and writes one contiguous chunk.
//
// Rows of spectral CTA i: (i, N - i) for 0 < i < N/2 and (0, N/2) for i = 0;
// either way the Hermitian mirror (-k1, -k2) of every bin of a row lies in
// one of the CTA's two rows.  The same kernels in other modes give the sample
// spectrum and the batched real 2D FFT building blocks.
#include "large_bodies.cuh"

namespace ocsc {

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------

template <typename Kern>
static cudaError_t prep(Kern k, size_t sm) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
}

template <typename Kern>
static cudaError_t go(Kern k, dim3 grid, size_t sm, const CodeIter &it, const ImgBatch &b, const LargeIO &io,
                      const float2 *tw, cudaStream_t s) {
  cudaError_t e = prep(k, sm);
  if (e != cudaSuccess) return e;
  k<<<grid, kLargeThreads, sm, s>>>(it, b, io, tw);
  return cudaGetLastError();
}

template <int N, int CB>
static cudaError_t spat_n(int what, const CodeIter &it, const ImgBatch &b, const LargeIO &io, int n, int npairs,
                          const float2 *tw, cudaStream_t s) {
  constexpr int NCB = N / CB;
  const size_t ss = spat_smem_bytes<N, CB>();
  switch (what) {
    case LARGE_SPAT_ADMM: return go(large_spat_kernel<N, CB, 0>, dim3(NCB, npairs, n), ss, it, b, io, tw, s);
    case LARGE_SPAT_IMAGE: return go(large_spat_kernel<N, CB, 1>, dim3(NCB, 1, n), ss, it, b, io, tw, s);
    case LARGE_SPAT_R2C: return go(large_spat_kernel<N, CB, 2>, dim3(NCB, npairs, 1), ss, it, b, io, tw, s);
    case LARGE_SPAT_C2R: return go(large_spat_kernel<N, CB, 3>, dim3(NCB, npairs, 1), ss, it, b, io, tw, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int N>
static cudaError_t large_n(int what, const CodeIter &it, const ImgBatch &b, const LargeIO &io, int n,
                           int npairs, const float2 *tw, cudaStream_t s) {
  using G = LargeGeom<N>;
  if (what >= LARGE_SPAT_ADMM) {
    const int cb = io.spat_cb ? io.spat_cb : G::CB;
    if (cb == 8) {
      if constexpr (spat_ok<N, 8>()) return spat_n<N, 8>(what, it, b, io, n, npairs, tw, s);
    }
    if (cb == 16) {
      if constexpr (spat_ok<N, 16>()) return spat_n<N, 16>(what, it, b, io, n, npairs, tw, s);
    }
    return cudaErrorInvalidValue;
  }
  const size_t sp = spec_smem_bytes<N>();
  const int S = (npairs + G::GP - 1) / G::GP;
  const dim3 gs(n, N / 2), gz(n, N / 2, S), gp(1, N / 2, S);
  switch (what) {
    case LARGE_SPEC_DOT: return go(large_spec_kernel<N, 0>, gz, sp, it, b, io, tw, s);
    case LARGE_SPEC_Z: return go(large_spec_kernel<N, 4>, gz, sp, it, b, io, tw, s);
    case LARGE_SPEC_IMAGE: return go(large_spec_kernel<N, 1>, gs, sp, it, b, io, tw, s);
    case LARGE_SPEC_R2C: return go(large_spec_kernel<N, 2>, gp, sp, it, b, io, tw, s);
    case LARGE_SPEC_C2R: return go(large_spec_kernel<N, 3>, gp, sp, it, b, io, tw, s);
    default: return cudaErrorInvalidValue;
  }
}

// Calls f(std::integral_constant<int, N>) for the supported sizes.
template <typename Fn, typename R>
static R with_size(int N, R fallback, Fn &&f) {
  switch (N) {
    case 96: return f(std::integral_constant<int, 96>());
    case 144: return f(std::integral_constant<int, 144>());
    case 192: return f(std::integral_constant<int, 192>());
    case 256: return f(std::integral_constant<int, 256>());
    case 288: return f(std::integral_constant<int, 288>());
    case 384: return f(std::integral_constant<int, 384>());
    case 512: return f(std::integral_constant<int, 512>());
    case 576: return f(std::integral_constant<int, 576>());
    default: return fallback;
  }
}

cudaError_t launch_large(int N, int what, const CodeIter &it, const ImgBatch &b, const LargeIO &io,
                         int n, int npairs, const float2 *tw, cudaStream_t s) {
  if (n <= 0 || npairs <= 0) return cudaSuccess;
  return with_size(N, cudaErrorInvalidValue, [&](auto nc) {
    return large_n<decltype(nc)::value>(what, it, b, io, n, npairs, tw, s);
  });
}

int large_default_cb(int N) {
  return with_size(N, 0, [](auto nc) { return LargeGeom<decltype(nc)::value>::CB; });
}

bool large_cb_ok(int N, int cb) {
  return with_size(N, false, [cb](auto nc) {
    constexpr int n = decltype(nc)::value;
    return (cb == 8 && spat_ok<n, 8>()) || (cb == 16 && spat_ok<n, 16>());
  });
}

int large_stages(int N, int npairs) {
  return with_size(N, 0, [npairs](auto nc) {
    constexpr int gp = LargeGeom<decltype(nc)::value>::GP;
    return (npairs + gp - 1) / gp;
  });
}

int large_resid_groups(int N, int npairs) {
  return with_size(N, 0, [npairs](auto nc) { return npairs * LargeGeom<decltype(nc)::value>::NCB; });
}

}  // namespace ocsc
