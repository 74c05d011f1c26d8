// History contraction on the tensor cores (the Precision variant of the fold
// of Sec. III-B, eqs. (A_update), (B_update)).
//
// Per frequency p the pending codes z_i (i < B, K filters) enter the history as
// A^p <- alpha A^p + beta G,  G = sum_i conj(z_i) z_i^T  (K x K Hermitian).
// With z = zr + i zi:  Re G = zr^T zr + zi^T zi,  Im G = zr^T zi - zi^T zr.  Each
// is a sum of real products D[m][n] = sum_s X[s][m] Y[s][n] over the samples s,
// which one tcgen05.mma (kind::f16: BF16 operands, FP32 accumulation in tensor
// memory) computes for 16 samples, 128 rows m and N columns n at a time.  The
// operands are the codes rounded to BF16 (terms = 1) or split as z = hi + lo,
// both BF16, with the products hi hi + hi lo + lo hi (terms = 3).
//
// Across the stream the history is kept as two FP32 words per entry (A, Alo)
// and every update is added with a compensated (Fast2Sum) step:
//   delta = beta G - (1 - alpha)(A + Alo),  s = A + (Alo + delta),
//   Alo <- (Alo + delta) - (s - A),  A <- s,
// so the stored pair carries the running mean to about twice FP32 precision.
// b^p = alpha b^p + beta sum_i x~_i conj(z_i) is formed in FP32 from the
// unrounded codes.
//
// One CTA per frequency, 256 threads.  Shared memory holds a chunk of SC
// samples of every operand plane in the canonical K-major layout without
// swizzle: 8 x 8 BF16 core matrices of 128 contiguous bytes, adjacent along
// the samples at LBO = 128 bytes and along the rows at SBO = SC / 8 * 128
// bytes.  Rows are padded with zeros to a multiple of 128 (the MMA's M) and
// samples to a multiple of 16.  For K > 128 the row blocks of 128 are done one
// after the other (each needs up to 2 x 256 tensor-memory columns).
#include <cuda_bf16.h>

#include "common.cuh"
#include "launch.h"

namespace ocsc {

namespace {

constexpr int kTcThreads = 256;
constexpr unsigned kWaitLimit = 1u << 24;  // mbarrier polls of the drain wait after a timeout

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory matrix descriptor: start address, leading and stride
// byte offsets (all >> 4), descriptor version 1 at bit 46, no swizzle.
__device__ __forceinline__ uint64_t mat_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24,
// optional negation of A (bit 13).
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, bool negA) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (negA ? (1u << 13) : 0u) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(mbar), "r"(count) : "memory");
}

// Bounded wait for the phase with the given parity (at most `polls` polls);
// false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, unsigned polls) {
  for (unsigned it = 0; it < polls; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// 8 consecutive FP32 columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t *>(&h);
}

}  // namespace

// Plane q of the chunk: BF16 [rows][SC] in the canonical layout.  Planes:
// 0 = Re hi, 1 = Im hi, 2 = Re lo, 3 = Im lo.
__global__ void __launch_bounds__(kTcThreads, 1) gram_fold_tc_kernel(GramArgs a) {
  extern __shared__ __align__(128) unsigned char gsm[];
  const int K = a.K, F = a.F, B = a.B, SC = a.SC;
  const int ROWS = (K + 127) / 128 * 128;  // 128 or 256
  const int TPR = kTcThreads / ROWS;       // threads per row: 2 or 1
  const int planes = a.terms == 3 ? 4 : 2;
  const uint32_t LBO = 128, SBO = (uint32_t)(SC / 8) * 128;
  const uint32_t plane_bytes = (uint32_t)ROWS * SC * 2;
  unsigned char *ops = gsm;
  float2 *bpart = reinterpret_cast<float2 *>(ops + planes * plane_bytes);  // [TPR][ROWS]
  float2 *xs = bpart + 2 * ROWS;                                            // [SC]
  uint64_t *mbar = reinterpret_cast<uint64_t *>(xs + SC);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);
  const int p = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t mb_addr = smem_u32(mbar);
  const int KN = (K + 15) / 16 * 16;

  // Tensor memory: a Re and an Im tile of up to KN columns each.
  const uint32_t ncols = 2 * KN <= 32 ? 32 : 2 * KN <= 64 ? 64 : 2 * KN <= 128 ? 128 : 2 * KN <= 256 ? 256 : 512;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(mb_addr, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tbase = *tslot;
  uint32_t phase = 0;
  bool ok = true;

  const int row = tid % ROWS, g0 = tid / ROWS;  // this thread's row; sample groups g0, g0 + TPR, ...
  const int nblk = ROWS / 128;
  float2 bacc = make_float2(0.f, 0.f);

  for (int mb = nblk - 1; mb >= 0; --mb) {
    const int N = mb == nblk - 1 ? KN : (mb + 1) * 128;  // columns j <= the block's last row
    const uint32_t d_re = tbase, d_im = tbase + (uint32_t)N;
    const bool first_pass = mb == nblk - 1;
    for (int c0 = 0; c0 < B; c0 += SC) {
      const int nb = B - c0 < SC ? B - c0 : SC;
      // (a) stage the chunk: x~, then the codes as BF16 planes.
      for (int s = tid; s < SC; s += kTcThreads)
        xs[s] = s < nb ? a.xh[(size_t)(c0 + s) * F + p] : make_float2(0.f, 0.f);
      __syncthreads();
      for (int g8 = g0; g8 < SC / 8; g8 += TPR) {
        float zr[8], zi[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int s = g8 * 8 + e;
          float2 z = make_float2(0.f, 0.f);
          if (row < K && s < nb) z = a.Zp[((size_t)(c0 + s) * K + row) * F + p];
          zr[e] = z.x;
          zi[e] = z.y;
        }
        if (first_pass) {
#pragma unroll
          for (int e = 0; e < 8; ++e) {  // x~ conj(z)
            const float2 x = xs[g8 * 8 + e];
            bacc.x += x.x * zr[e] + x.y * zi[e];
            bacc.y += x.y * zr[e] - x.x * zi[e];
          }
        }
        const uint32_t off = (uint32_t)(row / 8) * SBO + (uint32_t)g8 * LBO + (uint32_t)(row % 8) * 16;
        uint32_t hr[4], hi[4], lr[4], li[4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
          const __nv_bfloat162 r2 = __floats2bfloat162_rn(zr[e], zr[e + 1]);
          const __nv_bfloat162 i2 = __floats2bfloat162_rn(zi[e], zi[e + 1]);
          hr[e / 2] = *reinterpret_cast<const uint32_t *>(&r2);
          hi[e / 2] = *reinterpret_cast<const uint32_t *>(&i2);
          lr[e / 2] = pack_bf16(zr[e] - __low2float(r2), zr[e + 1] - __high2float(r2));
          li[e / 2] = pack_bf16(zi[e] - __low2float(i2), zi[e + 1] - __high2float(i2));
        }
        *reinterpret_cast<uint4 *>(ops + 0 * plane_bytes + off) = make_uint4(hr[0], hr[1], hr[2], hr[3]);
        *reinterpret_cast<uint4 *>(ops + 1 * plane_bytes + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        if (planes == 4) {
          *reinterpret_cast<uint4 *>(ops + 2 * plane_bytes + off) = make_uint4(lr[0], lr[1], lr[2], lr[3]);
          *reinterpret_cast<uint4 *>(ops + 3 * plane_bytes + off) = make_uint4(li[0], li[1], li[2], li[3]);
        }
      }
      fence_async_smem();
      fence_before();
      __syncthreads();
      fence_after();
      // (b) one thread issues the chunk's MMAs and commits them to the barrier.
      if (tid == 0) {
        const uint32_t base = smem_u32(ops);
        const uint32_t id_pos = idesc_bf16(128, N, false), id_neg = idesc_bf16(128, N, true);
        for (int t = 0; t < (nb + 15) / 16; ++t) {
          const uint32_t ka = base + (uint32_t)(mb * 16) * SBO + (uint32_t)t * 2 * LBO;  // rows of the block
          const uint32_t kb = base + (uint32_t)t * 2 * LBO;                              // rows 0 .. N-1
          const uint64_t A0 = mat_desc(ka, LBO, SBO), A1 = mat_desc(ka + plane_bytes, LBO, SBO);
          const uint64_t B0 = mat_desc(kb, LBO, SBO), B1 = mat_desc(kb + plane_bytes, LBO, SBO);
          const uint32_t acc = (c0 > 0 || t > 0) ? 1u : 0u;
          mma_bf16(d_re, A0, B0, id_pos, acc);   // Re G += zr^T zr
          mma_bf16(d_re, A1, B1, id_pos, 1u);    //       + zi^T zi
          mma_bf16(d_im, A0, B1, id_pos, acc);   // Im G += zr^T zi
          mma_bf16(d_im, A1, B0, id_neg, 1u);    //       - zi^T zr
          if (planes == 4) {
            const uint64_t A2 = mat_desc(ka + 2 * plane_bytes, LBO, SBO), A3 = mat_desc(ka + 3 * plane_bytes, LBO, SBO);
            const uint64_t B2 = mat_desc(kb + 2 * plane_bytes, LBO, SBO), B3 = mat_desc(kb + 3 * plane_bytes, LBO, SBO);
            mma_bf16(d_re, A0, B2, id_pos, 1u);
            mma_bf16(d_re, A2, B0, id_pos, 1u);
            mma_bf16(d_re, A1, B3, id_pos, 1u);
            mma_bf16(d_re, A3, B1, id_pos, 1u);
            mma_bf16(d_im, A0, B3, id_pos, 1u);
            mma_bf16(d_im, A2, B1, id_pos, 1u);
            mma_bf16(d_im, A1, B2, id_neg, 1u);
            mma_bf16(d_im, A3, B0, id_neg, 1u);
          }
        }
        mma_commit(mb_addr);
      }
      // (c) the MMAs have read the chunk and written the tiles.
      if (!mbar_wait(mb_addr, phase, a.wait_polls)) ok = false;
      phase ^= 1u;
      fence_after();
      if (__syncthreads_or(!ok)) {
        ok = false;
        break;
      }
    }
    if (!ok) break;

    // (d) b, on the first pass: per-row partial sums added in a fixed order.
    if (first_pass && !a.dry) {
      bpart[g0 * ROWS + row] = bacc;
      __syncthreads();
      for (int r = tid; r < K; r += kTcThreads) {
        float2 sum = bpart[r];
        for (int q = 1; q < TPR; ++q) sum = cadd(sum, bpart[q * ROWS + r]);
        float2 *bp = a.b + (size_t)r * F + p;
        const float2 old = a.first ? make_float2(0.f, 0.f) : *bp;
        *bp = make_float2(fmaf(a.alpha, old.x, a.beta * sum.x), fmaf(a.alpha, old.y, a.beta * sum.y));
      }
    }

    // (e) epilogue: warp w reads lanes 32 (w % 4) .. + 31 (rows) and one half
    // of the column chunks; compensated fold into A, Alo.
    const int m = mb * 128 + 32 * (warp & 3) + lane;
    float2 *Ap = a.A + (size_t)p * tri_stride(K);
    float2 *Lp = a.Alo + (size_t)p * tri_stride(K);
    const int nch = N / 8, half = (nch + 1) / 2;
    const int cbeg = (warp >> 2) * half, cend = min(nch, cbeg + half);
    const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
    for (int cc = cbeg; cc < cend; ++cc) {
      float re[8], im[8];
      tmem_ld8(d_re + lane_off + (uint32_t)cc * 8, re);
      tmem_ld8(d_im + lane_off + (uint32_t)cc * 8, im);
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int j = cc * 8 + e;
        if (m >= K || j > m || a.dry) continue;
        const size_t t = (size_t)tri_off(j, K) + m - j;
        if (a.first) {
          const float2 h = make_float2(a.beta * re[e], a.beta * im[e]);
          Ap[t] = h;
          Lp[t] = make_float2(fmaf(a.beta, re[e], -h.x), fmaf(a.beta, im[e], -h.y));
        } else {
          const float2 hi = Ap[t], lo = Lp[t];
          const float2 d = make_float2(fmaf(a.beta, re[e], -a.keep * (hi.x + lo.x)),
                                       fmaf(a.beta, im[e], -a.keep * (hi.y + lo.y)));
          const float2 y = make_float2(lo.x + d.x, lo.y + d.y);
          const float2 sum = make_float2(hi.x + y.x, hi.y + y.y);
          Lp[t] = make_float2(y.x - (sum.x - hi.x), y.y - (sum.y - hi.y));
          Ap[t] = sum;
        }
      }
    }
    fence_before();
    __syncthreads();
    fence_after();
  }

  // On a timeout, record it and wait once more, with the full poll budget
  // whatever the caller's limit, so that no MMA is still writing tensor memory
  // when it is released.
  if (!ok) {
    if (tid == 0) atomicOr(a.err, ERR_TIMEOUT);
    (void)mbar_wait(mb_addr, phase ^ 1u, kWaitLimit);
  }
  fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tbase), "r"(ncols) : "memory");
}

size_t gram_smem_bytes(int K, int terms, int SC) {
  const int ROWS = (K + 127) / 128 * 128;
  const int planes = terms == 3 ? 4 : 2;
  return (size_t)planes * ROWS * SC * 2 + 2 * (size_t)ROWS * sizeof(float2) + (size_t)SC * sizeof(float2) + 16;
}

int gram_chunk(int K, int B, int terms) {
  const int ROWS = (K + 127) / 128 * 128;
  const int planes = terms == 3 ? 4 : 2;
  const size_t budget = 200 * 1024;
  int sc = ((B + 15) / 16) * 16;
  if (sc > 128) sc = 128;
  while (sc > 16 && (size_t)planes * ROWS * sc * 2 > budget) sc -= 16;
  return sc;
}

cudaError_t launch_gram_fold(const GramArgs &a, cudaStream_t s) {
  if (a.K < 1 || a.K > 256 || a.B < 1 || (a.terms != 1 && a.terms != 3) || a.SC % 16 || a.SC < 16)
    return cudaErrorInvalidValue;
  const size_t sm = gram_smem_bytes(a.K, a.terms, a.SC);
  cudaError_t e = cudaFuncSetAttribute(gram_fold_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  gram_fold_tc_kernel<<<a.F, kTcThreads, sm, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ocsc
