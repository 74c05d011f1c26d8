// Persistent coder: the Jz code-ADMM iterations of a mini-batch (Sec. II-C.1,
// per sample as Sec. III-B.2 prescribes) in one cooperative launch.
//
// Each iteration of the per-kernel path is two launches for N <= 128
// (code_resid, code_plane) and three for N >= 256 (spectral partial sums,
// spectral row inverse, spatial column step).  Here every CTA of one
// co-resident grid walks the units of those launches -- the same bodies, on
// block coordinates it computes itself -- in three intervals per iteration,
// separated by a grid barrier: the only dependencies are that an interval
// reads what the one before wrote.  Images of several FFT sizes (64, 128, 256,
// 512) share each interval.
//
// The grid barrier counts arrivals in a global word and waits for a
// generation word to change.  Every wait is bounded (PersistArgs::polls): a
// CTA that gives up records ERR_TIMEOUT in the device error word and returns,
// and a CTA that finds the word set at a barrier returns too, so a launch in
// which one CTA fails ends in every CTA within the same bound.
#include <algorithm>

#include "large_bodies.cuh"
#include "plane_bodies.cuh"

namespace ocsc {

namespace {

__device__ __forceinline__ bool grid_sync(unsigned *bar, unsigned nblocks, unsigned polls, int *err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *vgen = bar + 1;
    volatile int *verr = err;
    int ok = *verr == 0;
    if (ok) {
      const unsigned gen = *vgen;
      __threadfence();
      const unsigned arrived = atomicAdd(bar, 1u) + 1u;
      if (arrived == nblocks) {
        atomicExch(bar, 0u);
        __threadfence();
        atomicAdd(bar + 1, 1u);
      } else {
        unsigned it = 0;
        while (*vgen == gen) {
          if (it++ >= polls || *verr != 0) {
            ok = 0;
            break;
          }
          __nanosleep(64);
        }
      }
      __threadfence();
    }
    if (!ok) atomicOr(err, ERR_TIMEOUT);
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Units of interval `phase` of iteration t for class c.
__device__ __forceinline__ int units_of(const PersistClass &c, int phase, int t, int K) {
  const int npairs = (K + 1) / 2;
  if (c.N <= 128) {
    const int F = c.N * (c.N / 2 + 1);
    if (phase == 0) return c.n * ((F + kResidBins - 1) / kResidBins);
    if (phase == 1) return c.n * K;
    return 0;
  }
  if (phase == 0) return t > 0 ? c.n * (c.N / 2) * c.S : 0;
  if (phase == 1) return c.n * (c.N / 2) * c.S;
  return (c.N / c.cb) * npairs * c.n;
}

// Each unit kind is compiled as a function of its own (not inlined), so that
// its registers are allocated for it alone and not for the union of all bodies.
template <int N>
__device__ __noinline__ void small_unit(const PersistArgs &a, const PersistClass &c, const CodeIter &it,
                                           int phase, int v, float4 *psm) {
  constexpr int F = N * (N / 2 + 1), NB = (F + kResidBins - 1) / kResidBins;
  if (phase == 0) {
    code_resid_body(it.K, F, it.rho, it.first, 0, a.b, it.Dh, it.dn, it.xh, it.What, it.r, v % NB, c.n0 + v / NB,
                    threadIdx.x & 31, threadIdx.x >> 5);
  } else {
    code_plane_body<N, false, 256>(it, a.b, c.tw, v % it.K, c.n0 + v / it.K, psm);
  }
}

template <int N>
__device__ __noinline__ void large_unit(const PersistArgs &a, const PersistClass &c, const CodeIter &it,
                                           int phase, int v, float4 *psm) {
  float2 *lsm = reinterpret_cast<float2 *>(psm);
  const int npairs = (it.K + 1) / 2;
  if (phase < 2) {
    const int st = v % c.S, rest = v / c.S, i = rest % (N / 2), img = c.n0 + rest / (N / 2);
    const dim3 bid(img, i, st), gdim(a.b.n, N / 2, c.S);
    if (phase == 0) large_spec_body<N, 0>(it, a.b, c.io, c.tw, bid, gdim, lsm);
    else large_spec_body<N, 4>(it, a.b, c.io, c.tw, bid, gdim, lsm);
    return;
  }
  const int ncb = N / c.cb, cbk = v % ncb, rest = v / ncb, pair = rest % npairs, img = c.n0 + rest / npairs;
  const dim3 bid(cbk, pair, img), gdim(ncb, npairs, a.b.n);
  if (c.cb == 16) large_spat_body<N, 16, 0>(it, a.b, c.io, c.tw, bid, gdim, lsm);
  else large_spat_body<N, 8, 0>(it, a.b, c.io, c.tw, bid, gdim, lsm);
}

__global__ void __launch_bounds__(kPersistThreads, 2) code_persist_kernel(const __grid_constant__ PersistArgs a) {
  extern __shared__ __align__(16) float4 psm[];
  const unsigned G = gridDim.x;
  for (int t = 0; t < a.Jz; ++t) {
    for (int phase = 0; phase < 3; ++phase) {
      int cnt[kMaxPersistClasses];
      int total = 0;
      for (int c = 0; c < a.ncls; ++c) {
        cnt[c] = units_of(a.c[c], phase, t, a.K);
        total += cnt[c];
      }
      if (total == 0) continue;
      for (int u = blockIdx.x; u < total; u += G) {
        int c = 0, v = u;
        while (v >= cnt[c]) v -= cnt[c++];
        const PersistClass &pc = a.c[c];
        const CodeIter &it = pc.it[t == 0 ? 0 : (t == a.Jz - 1 ? 2 : 1)];
        __syncthreads();  // the previous unit's shared memory is free
        switch (pc.N) {
          case 64: small_unit<64>(a, pc, it, phase, v, psm); break;
          case 128: small_unit<128>(a, pc, it, phase, v, psm); break;
          case 256: large_unit<256>(a, pc, it, phase, v, psm); break;
          case 512: large_unit<512>(a, pc, it, phase, v, psm); break;
          default: break;
        }
      }
      if (!grid_sync(a.bar, G, a.polls, a.err)) return;
    }
  }
}

}  // namespace

bool persist_size_ok(int N) { return N == 64 || N == 128 || N == 256 || N == 512; }

size_t persist_smem_bytes(const PersistArgs &a) {
  size_t sm = 0;
  for (int i = 0; i < a.ncls; ++i) {
    const PersistClass &c = a.c[i];
    size_t need = 0;
    switch (c.N) {
      case 64: need = half_smem_bytes<64>(); break;
      case 128: need = half_smem_bytes<128>(); break;
      case 256:
        need = spec_smem_bytes<256>();
        need = std::max(need, c.cb == 16 ? spat_smem_bytes<256, 16>() : spat_smem_bytes<256, 8>());
        break;
      case 512:
        need = spec_smem_bytes<512>();
        need = std::max(need, c.cb == 16 ? spat_smem_bytes<512, 16>() : spat_smem_bytes<512, 8>());
        break;
      default: break;
    }
    sm = std::max(sm, need);
  }
  return sm;
}

int persist_grid(size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(code_persist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return -(int)e;
  int per_sm = 0, dev = 0, sms = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, code_persist_kernel, kPersistThreads, smem);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return -(int)e;
  return per_sm * sms;
}

cudaError_t launch_persist(const PersistArgs &a, int grid, size_t smem, cudaStream_t s) {
  if (grid <= 0 || a.ncls < 1 || a.ncls > kMaxPersistClasses) return cudaErrorInvalidValue;
  for (int i = 0; i < a.ncls; ++i) {
    if (!persist_size_ok(a.c[i].N) || (a.c[i].N > 128 && a.c[i].cb != 8 && a.c[i].cb != 16))
      return cudaErrorInvalidValue;
    for (const CodeIter &it : a.c[i].it)
      if (it.serve) return cudaErrorInvalidValue;  // batch coding only
  }
  cudaError_t e = cudaFuncSetAttribute(code_persist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(a.bar, 0, 2 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kPersistThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, code_persist_kernel, a);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace ocsc
