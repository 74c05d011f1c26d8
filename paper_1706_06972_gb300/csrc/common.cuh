// Shared device helpers: complex arithmetic on float2/double2 and the packed
// lower-triangular layout of the per-frequency K x K Hermitian matrices.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ocsc {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// conj(a) * b
__device__ __forceinline__ float2 cconjmul(float2 a, float2 b) {
  return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// 16-byte asynchronous global -> shared copy (cp.async.cg: through L2 only),
// its group commit and the wait for all but PENDING committed groups.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
// 8-byte variant (through L1), for sources that are only 8-byte aligned.
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(PENDING) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  cp_async_commit();
  cp_async_wait<0>();
}

// Hint that `bytes` (a multiple of 16) from the 16-byte aligned gmem be
// brought into L2 (cp.async.bulk.prefetch: no completion, no ordering).
__device__ __forceinline__ void prefetch_l2(const void *gmem, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(gmem), "r"(bytes) : "memory");
}

// Packed lower triangle, column-major: column j holds rows j..K-1.
// Offset of column j: j*K - j*(j-1)/2.
__host__ __device__ __forceinline__ int tri_off(int j, int K) { return j * (2 * K - j + 1) / 2; }
__host__ __device__ __forceinline__ int tri_size(int K) { return K * (K + 1) / 2; }
// Per-frequency stride of packed complex-FP32 matrices in global memory: the
// triangle rounded up to an even element count, so every frequency starts on a
// 16-byte boundary.
__host__ __device__ __forceinline__ int tri_stride(int K) { return (tri_size(K) + 1) & ~1; }

// Inverse of tri_off: packed index t -> (i, j) with i >= j.
__device__ __forceinline__ void tri_ij(int t, int K, int &i, int &j) {
  const float kf = 2.0f * K + 1.0f;
  int jj = (int)floorf(0.5f * (kf - sqrtf(fmaxf(kf * kf - 8.0f * (float)t, 0.0f))));
  jj = max(0, min(jj, K - 1));
  // The float estimate is off by at most one column (all operands are exact
  // integers below 2^24 and sqrtf is correctly rounded).
  if (jj < K - 1 && tri_off(jj + 1, K) <= t) ++jj;
  else if (jj > 0 && tri_off(jj, K) > t) --jj;
  j = jj;
  i = t - tri_off(jj, K) + jj;
}

// Device error word bits.
enum : int { ERR_PIVOT = 1, ERR_TIMEOUT = 2 };

// Largest FFT side of any size class.
constexpr int kMaxFFT = 576;

}  // namespace ocsc
