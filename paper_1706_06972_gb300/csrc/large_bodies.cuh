// Device bodies of the N >= 256 coding kernels (row / column split through a
// per-pair tile in global memory).  Each body takes its block coordinates
// explicitly; code_large.cu wraps them as kernels and the persistent coder
// (persist.cu) runs them as units of one cooperative launch.  The design notes
// are at the top of code_large.cu.
#pragma once
#include <type_traits>

#include "fft.cuh"
#include "launch.h"

namespace ocsc {

constexpr int kLargeThreads = 256;

// Columns per spatial CTA (CB, even, dividing N) and filter pairs per spectral
// stage (GP) for each size.
template <int N> struct LargeTile;
template <> struct LargeTile<96> { static constexpr int CB = 8, GP = 8; };
template <> struct LargeTile<144> { static constexpr int CB = 16, GP = 8; };
template <> struct LargeTile<192> { static constexpr int CB = 16, GP = 8; };
template <> struct LargeTile<256> { static constexpr int CB = 16, GP = 8; };
template <> struct LargeTile<288> { static constexpr int CB = 16, GP = 4; };
template <> struct LargeTile<384> { static constexpr int CB = 8, GP = 4; };
template <> struct LargeTile<512> { static constexpr int CB = 8, GP = 4; };
template <> struct LargeTile<576> { static constexpr int CB = 8, GP = 4; };

// Spatial tile widths a size admits: CB even, dividing N, N * CB a multiple of
// the CTA's thread count.
template <int N, int CB>
constexpr bool spat_ok() {
  return N % CB == 0 && CB % 2 == 0 && (N * CB) % kLargeThreads == 0;
}

template <int N>
struct LargeGeom {
  static constexpr int NH = N / 2 + 1, F = N * NH, P = N * N;
  static constexpr int PITCH = N + 2;          // complex elements per shared-memory line
  static constexpr int CB = LargeTile<N>::CB;  // spatial CTA: columns per block
  static constexpr int NCB = N / CB;
  static constexpr int GP = LargeTile<N>::GP;  // spectral CTA: filter pairs per stage
  static constexpr int NL = 2 * GP;            // spectral CTA: lines per stage
  static constexpr int EPT = (2 * NH + kLargeThreads - 1) / kLargeThreads;  // row bins per thread
  static constexpr int SPT = N * CB / kLargeThreads;                        // spatial elements per thread
  static constexpr int CH = SPT % 4 == 0 ? 4 : (SPT % 3 == 0 ? 3 : (SPT % 2 == 0 ? 2 : 1));
};

// Spectral CTA: two stage buffers of NL lines (pass 1 is double-buffered)
// and the twiddles; spatial CTA: its N x CB block and the twiddles.
template <int N>
__host__ __device__ constexpr int spec_lines() { return 2 * LargeGeom<N>::NL; }
// Spatial CTA geometry for a block of CB columns (CB even, dividing N).
template <int N, int CB_>
struct SpatGeom {
  static constexpr int CB = CB_, NCB = N / CB, P = N * N;
  static constexpr int SPT = N * CB / kLargeThreads;  // elements per thread
  static constexpr int CH = SPT % 4 == 0 ? 4 : (SPT % 3 == 0 ? 3 : (SPT % 2 == 0 ? 2 : 1));
  static_assert(N % CB == 0 && CB % 2 == 0 && N * CB % kLargeThreads == 0, "spatial tiling");
};

template <int N>
size_t spec_smem_bytes() {
  return (size_t)spec_lines<N>() * LargeGeom<N>::PITCH * sizeof(float2) + (size_t)N * sizeof(float2);
}
template <int N, int CB>
size_t spat_smem_bytes() {
  return (size_t)N * CB * sizeof(float2) + (size_t)N * sizeof(float2);
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

// ---------------------------------------------------------------------------
// Spectral kernel
// ---------------------------------------------------------------------------

// Row r (0 or 1) of spectral CTA i.
template <int N>
__device__ __forceinline__ int spec_row(int i, int r) {
  return r == 0 ? i : (i == 0 ? N / 2 : N - i);
}

// Lines 2g + r <- row r of tile j0 + g, for g < ng (16-byte copies).
template <int N>
__device__ __forceinline__ void load_rows(float2 *lines, const float2 *tiles, int j0, int ng, int row0,
                                          int row1) {
  using G = LargeGeom<N>;
  constexpr int V = N / 2;  // float4 per row
  constexpr int TRIPS = (G::NL * V + kLargeThreads - 1) / kLargeThreads;
#pragma unroll
  for (int s = 0; s < TRIPS; ++s) {
    const int e = threadIdx.x + s * kLargeThreads;
    const int line = e / V, c = e % V;
    if (line < 2 * ng) {
      const int g = line >> 1, row = (line & 1) ? row1 : row0;
      const float4 v = *reinterpret_cast<const float4 *>(tiles + (size_t)(j0 + g) * G::P + (size_t)row * N + 2 * c);
      *reinterpret_cast<float4 *>(lines + line * G::PITCH + 2 * c) = v;
    }
  }
}

// load_rows with asynchronous copies (the caller commits and waits).
template <int N>
__device__ __forceinline__ void load_rows_async(float2 *lines, const float2 *tiles, int j0, int ng, int row0,
                                                int row1) {
  using G = LargeGeom<N>;
  constexpr int V = N / 2;
  constexpr int TRIPS = (G::NL * V + kLargeThreads - 1) / kLargeThreads;
#pragma unroll
  for (int s = 0; s < TRIPS; ++s) {
    const int e = threadIdx.x + s * kLargeThreads;
    const int line = e / V, c = e % V;
    if (line < 2 * ng) {
      const int g = line >> 1, row = (line & 1) ? row1 : row0;
      cp_async16(lines + line * G::PITCH + 2 * c, tiles + (size_t)(j0 + g) * G::P + (size_t)row * N + 2 * c);
    }
  }
}

// Rows of tiles j0 + g <- lines 2g + r.
template <int N>
__device__ __forceinline__ void store_rows(const float2 *lines, float2 *tiles, int j0, int ng, int row0, int row1) {
  using G = LargeGeom<N>;
  constexpr int V = N / 2;
  constexpr int TRIPS = (G::NL * V + kLargeThreads - 1) / kLargeThreads;
#pragma unroll
  for (int s = 0; s < TRIPS; ++s) {
    const int e = threadIdx.x + s * kLargeThreads;
    const int line = e / V, c = e % V;
    if (line < 2 * ng) {
      const int g = line >> 1, row = (line & 1) ? row1 : row0;
      *reinterpret_cast<float4 *>(tiles + (size_t)(j0 + g) * G::P + (size_t)row * N + 2 * c) =
          *reinterpret_cast<const float4 *>(lines + line * G::PITCH + 2 * c);
    }
  }
}

// Half spectra wa, wb of the two real planes packed as a + i b, from the
// packed value P at a bin and Pm at its Hermitian mirror.
__device__ __forceinline__ void split_pair(float2 P, float2 Pm, float2 &wa, float2 &wb) {
  wa = make_float2(0.5f * (P.x + Pm.x), 0.5f * (P.y - Pm.y));
  wb = make_float2(0.5f * (P.y + Pm.y), -0.5f * (P.x - Pm.x));
}

// Packed za + i zb at (line own, k2) and, for 0 < k2 < N/2, its Hermitian
// partner conj(za) + i conj(zb) at (line mir, N - k2).
template <int N>
__device__ __forceinline__ void put_pair(float2 *lines, int own, int mir, int k2, float2 za, float2 zb) {
  using G = LargeGeom<N>;
  lines[own * G::PITCH + k2] = make_float2(za.x - zb.y, za.y + zb.x);
  if (k2 > 0 && k2 < N / 2) lines[mir * G::PITCH + (N - k2)] = make_float2(za.x + zb.y, zb.x - za.y);
}

// MODE 0: ADMM partial sums D^T w^ and r (grid: images x N/2 x stages);
// MODE 4: ADMM row inverse of conj(d) r, and the kept Z~ (grid: images x N/2 x stages);
// MODE 1: sample spectra from the column-transformed images (grid: images x N/2);
// MODE 2: half spectra of planes 2j, 2j+1 (r2c; grid: 1 x N/2 x pair stages);
// MODE 3: packed row inverse of half spectra (c2r; grid: 1 x N/2 x pair stages).
// The body takes the CTA's block coordinates (bid) and grid size (gdim)
// explicitly, so that the persistent coder can run it as a unit of its own.
template <int N, int MODE>
__device__ __forceinline__ void large_spec_body(const CodeIter &it, const ImgBatch &b, const LargeIO &io,
                                                const float2 *__restrict__ tw, dim3 bid, dim3 gdim, float2 *lsm) {
  using G = LargeGeom<N>;
  float2 *lines = lsm;
  float2 *s_tw = lsm + spec_lines<N>() * G::PITCH;
  for (int i = threadIdx.x; i < N; i += kLargeThreads) s_tw[i] = tw[i];
  const int i = bid.y;
  const int row0 = spec_row<N>(i, 0), row1 = spec_row<N>(i, 1);
  const bool selfm = i == 0;  // rows 0 and N/2 are their own mirrors

  if (MODE == 1) {
    const int slot = b.slot[bid.x];
    const float2 *tiles = io.T + (size_t)slot * io.tile_pairs * G::P;
    load_rows<N>(lines, tiles, 0, 1, row0, row1);
    __syncthreads();
    fft_lines<N, G::NL, false, kLargeThreads>(lines, G::PITCH, 1, s_tw);
    float2 *out = io.spec_out + (size_t)slot * G::F;
    for (int e = threadIdx.x; e < 2 * G::NH; e += kLargeThreads) {
      const int r = e / G::NH, k2 = e % G::NH;
      out[(size_t)(r ? row1 : row0) * G::NH + k2] = lines[r * G::PITCH + k2];
    }
    return;
  }

  if (MODE == 2 || MODE == 3) {
    const int npairs = (io.planes + 1) / 2;
    const int j0 = bid.z * G::GP;
    const int ng = npairs - j0 < G::GP ? npairs - j0 : G::GP;
    if (MODE == 2) {
      load_rows<N>(lines, io.T, j0, ng, row0, row1);
      __syncthreads();
      fft_lines<N, G::NL, false, kLargeThreads>(lines, G::PITCH, 1, s_tw);
      for (int e = threadIdx.x; e < 2 * G::NH; e += kLargeThreads) {
        const int r = e / G::NH, k2 = e % G::NH, mr = selfm ? r : 1 - r;
        const size_t p = (size_t)(r ? row1 : row0) * G::NH + k2;
        for (int g = 0; g < ng; ++g) {
          const int a = 2 * (j0 + g);
          float2 wa, wb;
          split_pair(lines[(2 * g + r) * G::PITCH + k2], lines[(2 * g + mr) * G::PITCH + (N - k2) % N], wa, wb);
          io.spec_out[(size_t)a * G::F + p] = wa;
          if (a + 1 < io.planes) io.spec_out[(size_t)(a + 1) * G::F + p] = wb;
        }
      }
    } else {
      for (int e = threadIdx.x; e < 2 * G::NH; e += kLargeThreads) {
        const int r = e / G::NH, k2 = e % G::NH, mr = selfm ? r : 1 - r;
        const size_t p = (size_t)(r ? row1 : row0) * G::NH + k2;
        for (int g = 0; g < ng; ++g) {
          const int a = 2 * (j0 + g);
          const float2 za = io.spec_in[(size_t)a * G::F + p];
          const float2 zb = a + 1 < io.planes ? io.spec_in[(size_t)(a + 1) * G::F + p] : make_float2(0.f, 0.f);
          put_pair<N>(lines, 2 * g + r, 2 * g + mr, k2, za, zb);
        }
      }
      __syncthreads();
      fft_lines<N, G::NL, true, kLargeThreads>(lines, G::PITCH, 1, s_tw);
      store_rows<N>(lines, io.T, j0, ng, row0, row1);
    }
    return;
  }

  // MODE 0 (s = D^T w^ partial sums and r) and MODE 4 (row inverse of
  // conj(d) r): one CTA per (sample, row pair, stage of GP filter pairs).
  const int img = bid.x, st = bid.z, S = gdim.z;
  const int slot = b.slot[img], t = b.iter[img];
  const bool first = it.serve ? t == 0 : it.first != 0;
  const bool keep_z = it.serve ? (t + 1) % it.check == 0 : it.last != 0;
  const int K = it.K, npairs = (K + 1) / 2;
  const int j0 = st * G::GP, ng = npairs - j0 < G::GP ? npairs - j0 : G::GP;
  float2 *tiles = io.T + (size_t)slot * io.tile_pairs * G::P;
  // D rows of the stage, line ((g * 2 + f) * 2 + r) = row r of filter 2(j0 + g) + f.
  float2 *dsm = lines + G::NL * G::PITCH;
  constexpr int DL = 4 * G::NH;  // complex values per filter pair in dsm

  const bool need_w = MODE == 0 ? !first : (keep_z && !first);
  if (need_w) load_rows_async<N>(lines, tiles, j0, ng, row0, row1);
  {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int line = warp; line < 4 * ng; line += kLargeThreads / 32) {
      const int a = 2 * j0 + (line >> 1);
      if (a >= K) continue;
      const float2 *src = it.Dh + (size_t)a * G::F + (size_t)((line & 1) ? row1 : row0) * G::NH;
      float2 *dst = dsm + line * G::NH;
      for (int k2 = lane; k2 < G::NH; k2 += 32) cp_async8(dst + k2, src + k2);
    }
  }
  cp_async_wait_all();

  // Per bin of this thread: global index pe, shared offsets of the bin (lo)
  // and of its mirror (lm) in the lines of pair 0, and of the bin in dsm (ld).
  int pe[G::EPT], lo[G::EPT], lm[G::EPT], ld[G::EPT], kk[G::EPT];
#pragma unroll
  for (int q = 0; q < G::EPT; ++q) {
    const int e = threadIdx.x + q * kLargeThreads;
    const bool ok = e < 2 * G::NH;
    const int r = ok ? (e >= G::NH) : 0, k2 = ok ? e - r * G::NH : 0;
    const int mr = selfm ? r : 1 - r;
    kk[q] = k2;
    lo[q] = r * G::PITCH + k2;
    lm[q] = mr * G::PITCH + (k2 == 0 ? 0 : N - k2);
    ld[q] = r * G::NH + k2;
    pe[q] = ok ? (r ? row1 : row0) * G::NH + k2 : -1;
  }
  __syncthreads();
  if (need_w) fft_lines<N, G::NL, false, kLargeThreads>(lines, G::PITCH, 1, s_tw);

  if (MODE == 0) {
    // Partial sums of this stage, then the last CTA of the row pair adds the
    // S partials in stage order and forms r (no CTA waits for another).
    float2 *part = it.part + (size_t)slot * S * G::F;
#pragma unroll
    for (int q = 0; q < G::EPT; ++q) {
      if (pe[q] < 0) continue;
      float2 acc = make_float2(0.f, 0.f);
      if (!first) {
        for (int g = 0; g < ng; ++g) {
          const bool hasb = 2 * (j0 + g) + 1 < K;
          float2 wa, wb;
          split_pair(lines[2 * g * G::PITCH + lo[q]], lines[2 * g * G::PITCH + lm[q]], wa, wb);
          acc = cadd(acc, cmul(dsm[g * DL + ld[q]], wa));
          if (hasb) acc = cadd(acc, cmul(dsm[g * DL + 2 * G::NH + ld[q]], wb));
        }
      }
      part[(size_t)st * G::F + pe[q]] = acc;
    }
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      int *cnt = it.cnt + (size_t)slot * (N / 2) + i;
      const int old = atomicAdd(cnt, 1);
      s_last = old == S - 1;
      if (s_last) *cnt = 0;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
#pragma unroll
    for (int q = 0; q < G::EPT; ++q) {
      if (pe[q] < 0) continue;
      float2 sum = make_float2(0.f, 0.f);
      for (int u = 0; u < S; ++u) sum = cadd(sum, __ldcg(part + (size_t)u * G::F + pe[q]));
      const float2 x = it.xh[(size_t)slot * G::F + pe[q]];
      const float inv = 1.0f / (it.rho + it.dn[pe[q]]);
      it.r[(size_t)slot * G::F + pe[q]] = make_float2((x.x - sum.x) * inv, (x.y - sum.y) * inv);
    }
    return;
  }

  // MODE 4: r (from MODE 0, or x~ / (rho + |d|^2) on the first iteration).
  float2 rr[G::EPT];
#pragma unroll
  for (int q = 0; q < G::EPT; ++q) {
    rr[q] = make_float2(0.f, 0.f);
    if (pe[q] < 0) continue;
    if (first) {
      const float2 x = it.xh[(size_t)slot * G::F + pe[q]];
      const float inv = 1.0f / (it.rho + it.dn[pe[q]]);
      rr[q] = make_float2(x.x * inv, x.y * inv);
    } else {
      rr[q] = it.r[(size_t)slot * G::F + pe[q]];
    }
  }
  if (keep_z) {
#pragma unroll
    for (int q = 0; q < G::EPT; ++q) {
      if (pe[q] < 0) continue;
      for (int g = 0; g < ng; ++g) {
        const int a = 2 * (j0 + g);
        float2 wa = make_float2(0.f, 0.f), wb = wa;
        if (!first) split_pair(lines[2 * g * G::PITCH + lo[q]], lines[2 * g * G::PITCH + lm[q]], wa, wb);
        it.Zp[((size_t)slot * K + a) * G::F + pe[q]] = cadd(wa, cconjmul(dsm[g * DL + ld[q]], rr[q]));
        if (a + 1 < K)
          it.Zp[((size_t)slot * K + a + 1) * G::F + pe[q]] =
              cadd(wb, cconjmul(dsm[g * DL + 2 * G::NH + ld[q]], rr[q]));
      }
    }
    // the bins k2 = 0, N/2 of one row are read above as mirrors by the
    // thread owning the other row
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < G::EPT; ++q) {
    if (pe[q] < 0) continue;
    const bool mirrored = kk[q] > 0 && kk[q] < N / 2;
    for (int g = 0; g < ng; ++g) {
      const bool hasb = 2 * (j0 + g) + 1 < K;
      const float2 ca = cconjmul(dsm[g * DL + ld[q]], rr[q]);
      const float2 cb = hasb ? cconjmul(dsm[g * DL + 2 * G::NH + ld[q]], rr[q]) : make_float2(0.f, 0.f);
      lines[2 * g * G::PITCH + lo[q]] = make_float2(ca.x - cb.y, ca.y + cb.x);
      if (mirrored) lines[2 * g * G::PITCH + lm[q]] = make_float2(ca.x + cb.y, cb.x - ca.y);
    }
  }
  __syncthreads();
  fft_lines<N, G::NL, true, kLargeThreads>(lines, G::PITCH, 1, s_tw);
  store_rows<N>(lines, tiles, j0, ng, row0, row1);
}

template <int N, int MODE>
__global__ void __launch_bounds__(kLargeThreads, 3)
    large_spec_kernel(CodeIter it, ImgBatch b,
                      LargeIO io, const float2 *__restrict__ tw) {
  extern __shared__ float2 lsm[];
  large_spec_body<N, MODE>(it, b, io, tw, blockIdx, gridDim, lsm);
}

// ---------------------------------------------------------------------------
// Spatial kernel
// ---------------------------------------------------------------------------

// The spatial CTA keeps its block as [q1][l] (CB contiguous complex values
// per row of the tile), so that a tile row segment is one 16-byte-aligned run
// in both memories; its column transforms see element q1 of line l at
// q1 * CB + l.
// Block <- columns c0 .. c0 + CB - 1 of a tile (asynchronous 16-byte copies;
// the caller commits and waits).
template <int N, int CB>
__device__ __forceinline__ void load_cols_async(float2 *blk, const float2 *tile, int c0) {
  using G = LargeGeom<N>;
  using S = SpatGeom<N, CB>;
  constexpr int V = S::CB / 2;
  constexpr int TRIPS = (N * V + kLargeThreads - 1) / kLargeThreads;
#pragma unroll
  for (int s = 0; s < TRIPS; ++s) {
    const int e = threadIdx.x + s * kLargeThreads;
    const int k1 = e / V, c = e % V;
    if (N * V % kLargeThreads == 0 || e < N * V) cp_async16(blk + k1 * S::CB + 2 * c, tile + (size_t)k1 * N + c0 + 2 * c);
  }
}

template <int N, int CB>
__device__ __forceinline__ void store_cols(const float2 *blk, float2 *tile, int c0) {
  using G = LargeGeom<N>;
  using S = SpatGeom<N, CB>;
  constexpr int V = S::CB / 2;
  constexpr int TRIPS = (N * V + kLargeThreads - 1) / kLargeThreads;
#pragma unroll
  for (int s = 0; s < TRIPS; ++s) {
    const int e = threadIdx.x + s * kLargeThreads;
    const int k1 = e / V, c = e % V;
    if (N * V % kLargeThreads == 0 || e < N * V) *reinterpret_cast<float4 *>(tile + (size_t)k1 * N + c0 + 2 * c) =
        *reinterpret_cast<const float4 *>(blk + k1 * S::CB + 2 * c);
  }
}

// MODE 0: spatial ADMM step between the inverse and forward column transforms
//         (grid: NCB x pairs x images);
// MODE 1: zero-padded images in, forward column transforms out (grid: NCB x 1 x images);
// MODE 2: real planes 2j, 2j+1 in, forward column transforms out (grid: NCB x pairs);
// MODE 3: inverse column transforms, real planes out (c2r; grid: NCB x pairs).
template <int N, int CB, int MODE>
__device__ __forceinline__ void large_spat_body(const CodeIter &it, const ImgBatch &b, const LargeIO &io,
                                                const float2 *__restrict__ tw, dim3 bid, dim3 gdim, float2 *lsm) {
  using G = LargeGeom<N>;
  using S = SpatGeom<N, CB>;
  float2 *blk = lsm;  // [N][CB]
  float2 *s_tw = lsm + N * S::CB;
  for (int i = threadIdx.x; i < N; i += kLargeThreads) s_tw[i] = tw[i];
  const int cb = bid.x, c0 = cb * S::CB;
  const int pair = bid.y, img = bid.z;

  if (MODE == 1) {
    const int slot = b.slot[img];
    float2 *tile = io.T + (size_t)slot * io.tile_pairs * G::P;
    const float *x = b.x[img];
    const int H = b.H[img], W = b.W[img];
#pragma unroll 4
    for (int s = 0; s < S::SPT; ++s) {
      const int e = threadIdx.x + s * kLargeThreads;
      const int q1 = e / S::CB, q2 = c0 + e % S::CB;
      blk[e] = make_float2((q1 < H && q2 < W) ? x[(size_t)q1 * W + q2] : 0.f, 0.f);
    }
    __syncthreads();
    fft_lines<N, S::CB, false, kLargeThreads>(blk, 1, S::CB, s_tw);
    store_cols<N, CB>(blk, tile, c0);
    return;
  }
  if (MODE == 2) {
    const int pa = 2 * pair, pb = pa + 1;
    const bool hasb = pb < io.planes;
    const float *xa = io.real_in + (size_t)pa * G::P;
    const float *xb = io.real_in + (size_t)pb * G::P;
#pragma unroll 4
    for (int s = 0; s < S::SPT; ++s) {
      const int e = threadIdx.x + s * kLargeThreads;
      const size_t o = (size_t)(e / S::CB) * N + c0 + e % S::CB;
      blk[e] = make_float2(xa[o], hasb ? xb[o] : 0.f);
    }
    __syncthreads();
    fft_lines<N, S::CB, false, kLargeThreads>(blk, 1, S::CB, s_tw);
    store_cols<N, CB>(blk, io.T + (size_t)pair * G::P, c0);
    return;
  }
  if (MODE == 3) {
    load_cols_async<N, CB>(blk, io.T + (size_t)pair * G::P, c0);
    cp_async_wait_all();
    __syncthreads();
    fft_lines<N, S::CB, true, kLargeThreads>(blk, 1, S::CB, s_tw);
    const int pa = 2 * pair, pb = pa + 1;
    const bool hasb = pb < io.planes;
    float *xa = io.real_out + (size_t)pa * G::P;
    float *xb = io.real_out + (size_t)pb * G::P;
    const float invP = 1.0f / (float)G::P;
#pragma unroll 4
    for (int s = 0; s < S::SPT; ++s) {
      const int e = threadIdx.x + s * kLargeThreads;
      const size_t o = (size_t)(e / S::CB) * N + c0 + e % S::CB;
      const float2 c = blk[e];
      xa[o] = c.x * invP;
      if (hasb) xb[o] = c.y * invP;
    }
    return;
  }

  // MODE 0
  const int K = it.K, npairs = gdim.y, ka = 2 * pair, kb = ka + 1;
  const bool hasb = kb < K;
  const int slot = b.slot[img], t = b.iter[img];
  const bool first = it.serve ? t == 0 : it.first != 0;
  const bool store_last = it.serve ? (t + 1) % it.check == 0 : it.last != 0;
  const bool store_prev = it.serve && (t + 2) % it.check == 0;
  const bool skip_fwd = !it.serve && it.last;
  const bool resid = it.serve && store_last;
  float2 *tile = io.T + ((size_t)slot * io.tile_pairs + pair) * G::P;
  load_cols_async<N, CB>(blk, tile, c0);
  cp_async_wait_all();
  // U of this column block, [q1][l] like blk, contiguous.
  float *Sa = it.Gam + ((size_t)slot * K + ka) * G::P + (size_t)cb * N * S::CB;
  float *Sb = it.Gam + ((size_t)slot * K + (hasb ? kb : ka)) * G::P + (size_t)cb * N * S::CB;
  __syncthreads();
  fft_lines<N, S::CB, true, kLargeThreads>(blk, 1, S::CB, s_tw);
  // The code output doubles as the store of Gamma from the iteration before
  // a residual check (serving), where Z = V - Gamma_prev is needed.
  float *Ua = b.u[img] ? b.u[img] + (size_t)ka * G::P : nullptr;
  float *Ub = (b.u[img] && hasb) ? b.u[img] + (size_t)kb * G::P : nullptr;
  const float invP = 1.0f / (float)G::P;
  float acc[kResidTerms] = {0.f, 0.f, 0.f, 0.f, 0.f};
  constexpr int CH = S::CH;  // state loads in flight per thread
#pragma unroll 1
  for (int s0 = 0; s0 < S::SPT; s0 += CH) {
    float pa[CH], pb[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      const int e = threadIdx.x + (s0 + u) * kLargeThreads;
      pa[u] = first ? 0.f : Sa[e];
      pb[u] = (first || !hasb) ? 0.f : Sb[e];
    }
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      const int e = threadIdx.x + (s0 + u) * kLargeThreads;
      const size_t o = (size_t)(e / S::CB) * N + c0 + e % S::CB;
      const float2 c = blk[e];
      const float va = pa[u] + c.x * invP, vb = pb[u] + c.y * invP;
      const float ua = soft_thr(va, it.thr), ub = soft_thr(vb, it.thr);
      const float ga = va - ua, gb = vb - ub;
      if (resid) {
        const float qa = (first || !Ua) ? 0.f : Ua[o];  // Gamma of the previous iteration
        const float qb = (first || !Ub) ? 0.f : Ub[o];
        const float za = va - qa, zb = vb - qb;
        acc[0] += (za - ua) * (za - ua) + (hasb ? (zb - ub) * (zb - ub) : 0.f);
        acc[1] += za * za + (hasb ? zb * zb : 0.f);
        acc[2] += ua * ua + (hasb ? ub * ub : 0.f);
        acc[3] += (ua - pa[u]) * (ua - pa[u]) + (hasb ? (ub - pb[u]) * (ub - pb[u]) : 0.f);
        acc[4] += ga * ga + (hasb ? gb * gb : 0.f);
      }
      Sa[e] = ua;
      if (hasb) Sb[e] = ub;
      if (store_last || store_prev) {
        if (Ua) Ua[o] = store_last ? ua : ga;
        if (Ub) Ub[o] = store_last ? ub : gb;
      }
      blk[e] = make_float2(2.f * ua - va, hasb ? 2.f * ub - vb : 0.f);
    }
  }
  if (resid)
    block_terms(acc, it.resid + (((size_t)slot * npairs + pair) * S::NCB + cb) * kResidTerms);
  if (skip_fwd) return;
  __syncthreads();
  fft_lines<N, S::CB, false, kLargeThreads>(blk, 1, S::CB, s_tw);
  store_cols<N, CB>(blk, tile, c0);
}

template <int N, int CB, int MODE>
__global__ void __launch_bounds__(kLargeThreads, N * CB > 4608 ? 2 : 4)
    large_spat_kernel(CodeIter it, ImgBatch b,
                      LargeIO io, const float2 *__restrict__ tw) {
  extern __shared__ float2 lsm[];
  large_spat_body<N, CB, MODE>(it, b, io, tw, blockIdx, gridDim, lsm);
}


}  // namespace ocsc
