// Shared-memory 2D complex FFT on an N x N tile for one CTA.
//
// The 2D DFT of Sec. II-C (convolution theorem) is computed as 1D transforms
// along columns and rows.  Each 1D transform is a Stockham auto-sort
// decimation-in-time sequence of radix-R passes (Stockham; see Govindaraju et
// al., SC'08, for the GPU formulation): a pass reads R elements at stride N/R,
// multiplies by twiddles W_N^(r*(j mod Ns)*N/(Ns*R)), applies an R-point DFT in
// registers and writes them at stride Ns, so the output comes out in natural
// order with no bit reversal.  All N lines of the tile are transformed in the
// same pass; consecutive threads take consecutive lines, which with a row pitch
// of N+1 complex elements keeps 64-bit shared-memory accesses conflict-free for
// both row and column passes.
//
// Twiddles W_N^m = exp(-2 pi i m / N) come from a table computed on the host in
// double precision and rounded once to float.
#pragma once
#include "common.cuh"

namespace ocsc {

// exp(-+ 2 pi i k / 16) for k in [0, 8): cos(k pi/8) and sin(k pi/8).
template <int K16, bool INV>
__device__ __forceinline__ float2 tw_mul16(float2 o) {
  if constexpr (K16 == 0) {
    return o;
  } else if constexpr (K16 == 4) {  // -i (forward) / +i (inverse)
    return INV ? make_float2(-o.y, o.x) : make_float2(o.y, -o.x);
  } else {
    constexpr float c = K16 == 1 ? 0.92387953251128674f
                      : K16 == 2 ? 0.70710678118654752f
                      : K16 == 3 ? 0.38268343236508978f
                      : K16 == 5 ? -0.38268343236508978f
                      : K16 == 6 ? -0.70710678118654752f
                                 : -0.92387953251128674f;
    constexpr float s0 = K16 == 1 ? 0.38268343236508978f
                       : K16 == 2 ? 0.70710678118654752f
                       : K16 == 3 ? 0.92387953251128674f
                       : K16 == 5 ? 0.92387953251128674f
                       : K16 == 6 ? 0.70710678118654752f
                                  : 0.38268343236508978f;
    constexpr float s = INV ? s0 : -s0;
    return make_float2(o.x * c - o.y * s, o.x * s + o.y * c);
  }
}

// In-register R-point DFT (R = 2, 4, 8, 16), natural order in and out,
// by even/odd splitting.
template <int R, bool INV>
struct RegDFT {
  template <int K>
  static __device__ __forceinline__ void combine(float2 *v, const float2 *e, const float2 *o) {
    if constexpr (K < R / 2) {
      const float2 t = tw_mul16<K * (16 / R), INV>(o[K]);
      v[K] = make_float2(e[K].x + t.x, e[K].y + t.y);
      v[K + R / 2] = make_float2(e[K].x - t.x, e[K].y - t.y);
      combine<K + 1>(v, e, o);
    }
  }
  static __device__ __forceinline__ void run(float2 *v) {
    float2 e[R / 2], o[R / 2];
#pragma unroll
    for (int n = 0; n < R / 2; ++n) {
      e[n] = v[2 * n];
      o[n] = v[2 * n + 1];
    }
    RegDFT<R / 2, INV>::run(e);
    RegDFT<R / 2, INV>::run(o);
    combine<0>(v, e, o);
  }
};
template <bool INV>
struct RegDFT<1, INV> {
  static __device__ __forceinline__ void run(float2 *) {}
};

// 3-point DFT: X0 = a + b + c, X1,2 = a - (b + c)/2 -+ i sqrt(3)/2 (b - c)
// (forward; the signs of the sine terms flip for the inverse).
template <bool INV>
struct RegDFT<3, INV> {
  static __device__ __forceinline__ void run(float2 *v) {
    constexpr float h = 0.86602540378443865f;  // sqrt(3) / 2
    const float2 a = v[0], s = make_float2(v[1].x + v[2].x, v[1].y + v[2].y);
    const float2 d = make_float2(v[1].x - v[2].x, v[1].y - v[2].y);
    const float2 t = make_float2(a.x - 0.5f * s.x, a.y - 0.5f * s.y);
    const float2 r = INV ? make_float2(-h * d.y, h * d.x) : make_float2(h * d.y, -h * d.x);  // -+ i h d
    v[0] = make_float2(a.x + s.x, a.y + s.y);
    v[1] = make_float2(t.x + r.x, t.y + r.y);
    v[2] = make_float2(t.x - r.x, t.y - r.y);
  }
};

// 9-point DFT as 3 x 3 (n = n1 + 3 n2, k = k1 + 3 k2): 3-point DFTs over n2,
// twiddles W9^(n1 k1), 3-point DFTs over n1.  cos and sin of 2 pi m / 9 for
// m = 1, 2, 4.
template <bool INV>
struct RegDFT<9, INV> {
  static __device__ __forceinline__ float2 tw9(float2 o, float c, float s0) {
    const float s = INV ? s0 : -s0;  // W9^m = cos - i sin (forward)
    return make_float2(o.x * c - o.y * s, o.x * s + o.y * c);
  }
  static __device__ __forceinline__ void run(float2 *v) {
    constexpr float c1 = 0.76604444311897804f, s1 = 0.64278760968653933f;
    constexpr float c2 = 0.17364817766693041f, s2 = 0.98480775301220802f;
    constexpr float c4 = -0.93969262078590832f, s4 = 0.34202014332566888f;
    float2 y[3][3];
#pragma unroll
    for (int n1 = 0; n1 < 3; ++n1) {
      y[n1][0] = v[n1];
      y[n1][1] = v[n1 + 3];
      y[n1][2] = v[n1 + 6];
      RegDFT<3, INV>::run(y[n1]);
    }
    y[1][1] = tw9(y[1][1], c1, s1);
    y[1][2] = tw9(y[1][2], c2, s2);
    y[2][1] = tw9(y[2][1], c2, s2);
    y[2][2] = tw9(y[2][2], c4, s4);
#pragma unroll
    for (int k1 = 0; k1 < 3; ++k1) {
      float2 w[3] = {y[0][k1], y[1][k1], y[2][k1]};
      RegDFT<3, INV>::run(w);
      v[k1] = w[0];
      v[k1 + 3] = w[1];
      v[k1 + 6] = w[2];
    }
  }
};

// Radix plan per transform length.
template <int N> struct FFTPlan;
template <> struct FFTPlan<64> { static constexpr int R0 = 8, R1 = 8; };
template <> struct FFTPlan<128> { static constexpr int R0 = 16, R1 = 8; };

template <int N>
__host__ __device__ constexpr int tile_pitch() { return N + 1; }

// One Stockham radix-R pass over all N lines of the tile.  ROWS: transform
// along the second index (contiguous); otherwise along the first index.
template <int N, int R, int NS, bool INV, bool ROWS, int NT>
__device__ __forceinline__ void fft_pass(float2 *__restrict__ tile, const float2 *__restrict__ tw) {
  constexpr int PITCH = tile_pitch<N>();
  constexpr int G = N * (N / R);
  static_assert(G % NT == 0, "threads must divide the butterfly groups");
  constexpr int PER = G / NT;
  float2 v[PER][R];
  const int tid = threadIdx.x;
#pragma unroll
  for (int gi = 0; gi < PER; ++gi) {
    const int g = tid + gi * NT;
    const int line = g % N;
    const int j = g / N;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int e = j + r * (N / R);
      v[gi][r] = ROWS ? tile[line * PITCH + e] : tile[e * PITCH + line];
    }
    if constexpr (NS > 1) {
      const int jm = j % NS;
#pragma unroll
      for (int r = 1; r < R; ++r) {
        float2 w = tw[(r * jm * (N / (NS * R))) & (N - 1)];
        if (INV) w.y = -w.y;
        v[gi][r] = cmul(v[gi][r], w);
      }
    }
    RegDFT<R, INV>::run(v[gi]);
  }
  __syncthreads();
#pragma unroll
  for (int gi = 0; gi < PER; ++gi) {
    const int g = tid + gi * NT;
    const int line = g % N;
    const int j = g / N;
    const int base = (j / NS) * NS * R + (j % NS);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int e = base + r * NS;
      if (ROWS)
        tile[line * PITCH + e] = v[gi][r];
      else
        tile[e * PITCH + line] = v[gi][r];
    }
  }
  __syncthreads();
}

// Full 2D transform of the tile (columns, then rows).  The caller must have
// synchronised after writing the tile; the tile is complete on return.
template <int N, int NT, bool INV>
__device__ __forceinline__ void fft2d_tile(float2 *tile, const float2 *tw) {
  constexpr int R0 = FFTPlan<N>::R0, R1 = FFTPlan<N>::R1;
  static_assert(R0 * R1 == N, "two-pass plan");
  fft_pass<N, R0, 1, INV, false, NT>(tile, tw);
  fft_pass<N, R1, R0, INV, false, NT>(tile, tw);
  fft_pass<N, R0, 1, INV, true, NT>(tile, tw);
  fft_pass<N, R1, R0, INV, true, NT>(tile, tw);
}

// ---------------------------------------------------------------------------
// Line transforms for sizes whose full tile does not fit one CTA (N = 256,
// 512): NL lines of N contiguous complex elements at a runtime pitch.
// ---------------------------------------------------------------------------
template <int N> struct LinePlan;
template <> struct LinePlan<256> { static constexpr int NP = 2, R0 = 16, R1 = 16, R2 = 1; };
template <> struct LinePlan<512> { static constexpr int NP = 3, R0 = 8, R1 = 8, R2 = 8; };
template <> struct LinePlan<288> { static constexpr int NP = 3, R0 = 8, R1 = 4, R2 = 9; };
template <> struct LinePlan<96> { static constexpr int NP = 3, R0 = 8, R1 = 4, R2 = 3; };
template <> struct LinePlan<144> { static constexpr int NP = 2, R0 = 16, R1 = 9, R2 = 1; };
template <> struct LinePlan<192> { static constexpr int NP = 3, R0 = 8, R1 = 8, R2 = 3; };
template <> struct LinePlan<384> { static constexpr int NP = 3, R0 = 8, R1 = 16, R2 = 3; };
template <> struct LinePlan<576> { static constexpr int NP = 3, R0 = 8, R1 = 8, R2 = 9; };

// One Stockham radix-R pass over NL lines; element m of line l is at
// buf[l * ls + m * es].  Consecutive threads take consecutive lines of the
// same butterfly index.
template <int N, int NL, int R, int NS, bool INV, int NT>
__device__ __forceinline__ void line_pass(float2 *__restrict__ buf, int ls, int es, const float2 *__restrict__ tw) {
  constexpr int G = NL * (N / R);
  constexpr int PER = (G + NT - 1) / NT;
  float2 v[PER][R];
  const int tid = threadIdx.x;
#pragma unroll
  for (int gi = 0; gi < PER; ++gi) {
    const int g = tid + gi * NT;
    if (G % NT == 0 || g < G) {
      const int line = g % NL;
      const int j = g / NL;
#pragma unroll
      for (int r = 0; r < R; ++r) v[gi][r] = buf[line * ls + (j + r * (N / R)) * es];
      if constexpr (NS > 1) {
        const int jm = j % NS;
#pragma unroll
        for (int r = 1; r < R; ++r) {
          float2 w = tw[(r * jm * (N / (NS * R))) % N];
          if (INV) w.y = -w.y;
          v[gi][r] = cmul(v[gi][r], w);
        }
      }
      RegDFT<R, INV>::run(v[gi]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int gi = 0; gi < PER; ++gi) {
    const int g = tid + gi * NT;
    if (G % NT == 0 || g < G) {
      const int line = g % NL;
      const int j = g / NL;
      const int base = (j / NS) * NS * R + (j % NS);
#pragma unroll
      for (int r = 0; r < R; ++r) buf[line * ls + (base + r * NS) * es] = v[gi][r];
    }
  }
  __syncthreads();
}

// Full 1D transform of NL lines of length N (unnormalised), element m of
// line l at buf[l * ls + m * es].  The caller must have synchronised after
// filling the lines.
template <int N, int NL, bool INV, int NT>
__device__ __forceinline__ void fft_lines(float2 *buf, int ls, int es, const float2 *tw) {
  using P = LinePlan<N>;
  line_pass<N, NL, P::R0, 1, INV, NT>(buf, ls, es, tw);
  line_pass<N, NL, P::R1, P::R0, INV, NT>(buf, ls, es, tw);
  if constexpr (P::NP == 3) line_pass<N, NL, P::R2, P::R0 * P::R1, INV, NT>(buf, ls, es, tw);
}

// ---------------------------------------------------------------------------
// Half-spectrum tile of one real N x N plane: N rows of NH = N/2 + 1 complex
// elements at pitch NH (element (k1, k2) at k1 * NH + k2 -- the global layout
// of a half spectrum).  Columns are transformed with length N, rows (the
// packed real row of the r2c / c2r step) with length N/2.  A pitch of NH
// (= 1 mod 16 for N = 64, 128) keeps 64-bit accesses conflict-free both when
// consecutive threads take consecutive columns of one row and when they take
// consecutive rows of one column.
// ---------------------------------------------------------------------------

// One Stockham radix-R pass of length LEN over LINES lines: element m of line
// l at buf[l * LS + m * ES]; twiddles W_LEN^x = tw[x * TWS] from the table of
// size LEN * TWS.  Consecutive threads take consecutive lines of the same
// butterfly index.  Every group is held in registers across the barrier
// between the reads and the in-place writes.
template <int LEN, int LINES, int R, int NS, bool INV, int LS, int ES, int NT, int TWS>
__device__ __forceinline__ void half_pass(float2 *__restrict__ buf, const float2 *__restrict__ tw) {
  constexpr int G = LINES * (LEN / R);
  static_assert(G % NT == 0, "threads must divide the butterfly groups");
  constexpr int PER = G / NT;
  const int tid = threadIdx.x;
  if constexpr (NS * R == LEN) {
    // The last pass writes each group's outputs onto its own inputs
    // (j + r LEN / R), so a group is finished before the next is loaded and
    // no barrier separates the loads from the stores.
#pragma unroll
    for (int gi = 0; gi < PER; ++gi) {
      const int g = tid + gi * NT;
      const int line = g % LINES;
      const int j = g / LINES;
      float2 u[R];
#pragma unroll
      for (int r = 0; r < R; ++r) u[r] = buf[line * LS + (j + r * NS) * ES];
      if constexpr (NS > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          float2 w = tw[((r * j) % LEN) * TWS];
          if (INV) w.y = -w.y;
          u[r] = cmul(u[r], w);
        }
      }
      RegDFT<R, INV>::run(u);
#pragma unroll
      for (int r = 0; r < R; ++r) buf[line * LS + (j + r * NS) * ES] = u[r];
    }
    __syncthreads();
    return;
  }
  float2 v[PER][R];
#pragma unroll
  for (int gi = 0; gi < PER; ++gi) {
    const int g = tid + gi * NT;
    const int line = g % LINES;
    const int j = g / LINES;
#pragma unroll
    for (int r = 0; r < R; ++r) v[gi][r] = buf[line * LS + (j + r * (LEN / R)) * ES];
    if constexpr (NS > 1) {
      const int jm = j % NS;
#pragma unroll
      for (int r = 1; r < R; ++r) {
        float2 w = tw[((r * jm * (LEN / (NS * R))) % LEN) * TWS];
        if (INV) w.y = -w.y;
        v[gi][r] = cmul(v[gi][r], w);
      }
    }
    RegDFT<R, INV>::run(v[gi]);
  }
  __syncthreads();
#pragma unroll
  for (int gi = 0; gi < PER; ++gi) {
    const int g = tid + gi * NT;
    const int line = g % LINES;
    const int j = g / LINES;
    const int base = (j / NS) * NS * R + (j % NS);
#pragma unroll
    for (int r = 0; r < R; ++r) buf[line * LS + (base + r * NS) * ES] = v[gi][r];
  }
  __syncthreads();
}

// Radix plans of the half-spectrum tile: columns (length N) and rows (N/2).
template <int N> struct HalfPlan;
template <> struct HalfPlan<64> { static constexpr int C0 = 8, C1 = 8, R0 = 8, R1 = 4, NT = 256; };
template <> struct HalfPlan<128> { static constexpr int C0 = 16, C1 = 8, R0 = 8, R1 = 8, NT = 256; };

// Transform of the N/2 columns k2 < N/2 (length N, along k1); column N/2 is
// carried packed in column 0 by the caller.
template <int N, bool INV>
__device__ __forceinline__ void half_cols(float2 *tile, const float2 *tw) {
  using P = HalfPlan<N>;
  constexpr int NH = N / 2 + 1;
  half_pass<N, N / 2, P::C0, 1, INV, 1, NH, P::NT, 1>(tile, tw);
  half_pass<N, N / 2, P::C1, P::C0, INV, 1, NH, P::NT, 1>(tile, tw);
}

// Transform of the N rows (length N/2, elements 0 .. N/2 - 1 of each row).
template <int N, bool INV>
__device__ __forceinline__ void half_rows(float2 *tile, const float2 *tw) {
  using P = HalfPlan<N>;
  constexpr int NH = N / 2 + 1;
  half_pass<N / 2, N, P::R0, 1, INV, NH, 1, P::NT, 2>(tile, tw);
  half_pass<N / 2, N, P::R1, P::R0, INV, NH, 1, P::NT, 2>(tile, tw);
}

template <int N>
__host__ __device__ constexpr size_t half_smem_bytes() {
  return (size_t)N * (N / 2 + 1) * sizeof(float2) + (size_t)N * sizeof(float2);
}

// Threads per CTA used with an N x N tile.
template <int N> struct TileThreads;
template <> struct TileThreads<64> { static constexpr int value = 256; };
template <> struct TileThreads<128> { static constexpr int value = 512; };

template <int N>
__host__ __device__ constexpr size_t tile_smem_bytes() {
  return (size_t)N * tile_pitch<N>() * sizeof(float2) + (size_t)N * sizeof(float2);
}

}  // namespace ocsc
