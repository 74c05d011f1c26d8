// Internal context state shared by the runtime files (not part of the ABI).
#pragma once
#include <cstdarg>
#include <cstdio>
#include <set>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/ocsc.h"
#include "common.cuh"
#include "launch.h"

namespace ocsc {

struct SizeClass {
  int N = 0, NH = 0, F = 0, P = 0;
  int p0 = 0, Fb = 0;       // frequencies p0 .. p0 + Fb - 1 of the history (a band context: its band)
  float2 *tw = nullptr;     // [N] twiddles
  // dictionary state in this class's frequency grid
  float2 *Vh = nullptr;     // [K][F] F(pad V)
  float2 *th = nullptr;     // [K][F] scaled dual of DictOCSC
  float2 *Dcur = nullptr;   // [K][F] D~_{t,tau}
  float2 *E = nullptr;      // [K][F] D~ + theta^
  float2 *Y = nullptr;      // [K][M][NH] pruned inverse DFT along k1
  float2 *Tm = nullptr;     // [K][M][NH] partial DFT of V
  float *dn = nullptr;      // [F] |D~(p,:)|^2 of the coding dictionary
  // history and factor
  float2 *A = nullptr;      // [F][stride] packed FP32 history
  float2 *Alo = nullptr;    // [F][stride] its compensation word (precision > 0)
  float4 *Csf = nullptr;    // [F][stride] C^p of the recursion variant (history = 1), double-float
  float2 *b = nullptr;      // [K][F]
  float2 *blo = nullptr;    // [K][F] its compensation word (precision 3)
  float2 *X = nullptr;      // [F][stride] X = L^-1 (FP32) of the FP64 factor
  float2 *y = nullptr;      // [K][F] y = L^-1 (w b)
  // pending samples
  float2 *Zp = nullptr;     // [max_batch][K][F]
  float2 *xhp = nullptr;    // [max_batch][F]
  // code workspace
  float2 *What = nullptr;   // [max_batch][K][F]
  float *Gam = nullptr;     // [max_batch][K][P] spatial ADMM state (see CodeIter::Gam)
  float2 *r = nullptr;      // [max_batch][F]
  float2 *tiles = nullptr;  // [max_batch][ceil(K/2)][N][N] for N >= 256
  float2 *part = nullptr;   // [max_batch][stages][F] for N >= 256
  int *cnt = nullptr;       // [max_batch][N/2] for N >= 256
  float2 *obj_xh = nullptr; // [F]
  long long n_seen = 0;
  int pending = 0;
  // tile shapes picked by the autotuner (0 = not tuned yet)
  int fold_threads = 0, spat_cb = 0, gram_sc = 0, plane_ctas = 0, plane_ahead = 1, plane_threads = 256;
  // graph path of ocsc_code: image and code staging per slot (lazily allocated)
  float *xstage = nullptr;  // [max_batch][N*N]
  float *ustage = nullptr;  // [max_batch][K][N*N]
};

// A captured coding graph of one chunk shape.
struct GraphEntry {
  std::string key;
  cudaGraphExec_t exec = nullptr;
  size_t kernels = 0;  // kernel nodes per replay
};
constexpr size_t kMaxGraphs = 32;
// Default poll count of the bounded device waits (tensor-core fold, persistent coder).
constexpr unsigned kWaitPolls = 1u << 24;

}  // namespace ocsc

struct ocsc_ctx {
  int K = 0, M = 0, T = 0;
  double lam = 0, rho = 0;
  ocsc_opts opts{};
  cudaStream_t stream = nullptr;
  float *V = nullptr;       // [K][M][M] the spatial filters
  float *Dpub = nullptr;    // [K][M][M] H(F^-1(D~_{t,J})) when return_feasible = 0
  std::vector<ocsc::SizeClass> cls;
  double *obj_part = nullptr;
  double *obj_out = nullptr;
  int *err = nullptr;       // device error word
  unsigned *bar = nullptr;  // [2] grid barrier of the persistent coder
  int *order = nullptr;     // [K] filter order (ocsc_filter_order)
  unsigned wait_polls = ocsc::kWaitPolls;  // polls of a bounded device wait before it gives up
  double2 *work = nullptr;  // K > 128: FP64 factorisation workspace, one matrix per persistent CTA
  int work_ctas = 0;
  long long n_seen = 0;     // samples folded over all classes
  uint64_t version = 0;
  std::string msg;
  std::vector<void *> allocs;
  std::vector<ocsc::GraphEntry> graphs;
  cudaStream_t cap_stream = nullptr;  // capture stream of the graph path
  std::set<std::string> graph_seen;
  ocsc_counters counters{};
  unsigned prof_mask = 0;
  std::vector<cudaEvent_t> prof_ev[OCSC_K_COUNT];  // start/stop pairs
  size_t prof_used[OCSC_K_COUNT] = {};
};

namespace ocsc {

// NVTX range over one library call (visible in Nsight timelines; a no-op
// unless a tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

inline ocsc_status fail(ocsc_ctx *c, ocsc_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->msg = buf;
  return s;
}

inline ocsc_status cuda_fail(ocsc_ctx *c, cudaError_t e, const char *where) {
  return fail(c, OCSC_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

// Device allocation owned by the context (freed in ocsc_destroy).
template <typename T>
ocsc_status dalloc(ocsc_ctx *c, T **p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    *p = nullptr;
    return fail(c, OCSC_ENOMEM, "cudaMalloc of %zu bytes failed: %s", count * sizeof(T),
                cudaGetErrorString(e));
  }
  c->allocs.push_back(*p);
  return OCSC_OK;
}

// FFT sides: 2^a 3^b with b <= 2.  64 and 128 run the whole-plane kernels of
// code_admm.cu; every other size the row / column kernels of code_large.cu.
inline bool supported_fft(int n) {
  for (int m : {64, 96, 128, 144, 192, 256, 288, 384, 512, 576})
    if (n == m) return true;
  return false;
}
inline bool large_fft(int n) { return n != 64 && n != 128; }

// Class of an H x W image: the smallest FFT size of the context that holds
// max(H, W) + pad, or -1.
inline int class_of(const ocsc_ctx *c, int H, int W) {
  const int need = (H > W ? H : W) + c->opts.pad;
  int best = -1;
  for (size_t i = 0; i < c->cls.size(); ++i)
    if (c->cls[i].N >= need && (best < 0 || c->cls[i].N < c->cls[best].N)) best = (int)i;
  return best;
}

// Launch one kernel through `fn`, counting it and, when its class is being
// profiled, bracketing it with events on the context's stream.
template <typename Fn>
cudaError_t timed(ocsc_ctx *c, int id, Fn &&fn) {
  c->counters.kernel_launches++;
  if (id >= OCSC_K_COUNT || !(c->prof_mask & (1u << id))) return fn();
  auto &ev = c->prof_ev[id];
  size_t &used = c->prof_used[id];
  while (used + 2 > ev.size()) {
    cudaEvent_t e;
    cudaError_t err = cudaEventCreate(&e);
    if (err != cudaSuccess) return err;
    ev.push_back(e);
  }
  cudaError_t err = cudaEventRecord(ev[used], c->stream);
  if (err != cudaSuccess) return err;
  err = fn();
  if (err != cudaSuccess) return err;
  err = cudaEventRecord(ev[used + 1], c->stream);
  used += 2;
  return err;
}

// K above this uses the dict_big.cu kernels (matrix outside shared memory).
constexpr int kSmallK = 128;
inline bool big_k(const ocsc_ctx *c) { return c->K > kSmallK; }

// Mean duration in ms of reps runs of fn (which enqueues on the context's
// stream); negative on a launch error.  Used by the autotuner.
template <typename Fn>
float time_runs(ocsc_ctx *c, int reps, Fn &&fn) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return -1.f;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return -1.f;
  }
  float ms = -1.f;
  // One untimed run first: a kernel's first launch also loads its module.
  bool ok = fn() == cudaSuccess;
  c->counters.kernel_launches++;
  ok = ok && cudaEventRecord(e0, c->stream) == cudaSuccess;
  for (int r = 0; ok && r < reps; ++r) {
    ok = fn() == cudaSuccess;
    c->counters.kernel_launches++;
  }
  if (ok && cudaEventRecord(e1, c->stream) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
      cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
    ms /= (float)reps;
  else
    ms = -1.f;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms;
}

inline const float2 *coding_spectrum(const ocsc_ctx *c, const SizeClass &s) {
  return c->opts.return_feasible ? s.Vh : s.Dcur;
}

}  // namespace ocsc
