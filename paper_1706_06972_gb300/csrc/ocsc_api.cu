// C-ABI runtime: context state, allocation and the launch sequences of
// Algorithm 3 (code, fold, DictOCSC).  All method arithmetic runs in the
// kernels of code_admm.cu and dict_update.cu; this file only sequences them.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ocsc.h"
#include "common.cuh"
#include "launch.h"

using namespace ocsc;

struct ocsc_ctx {
  int K = 0, M = 0, N = 0, NH = 0, F = 0, P = 0, T = 0;
  double lam = 0, rho = 0;
  ocsc_opts opts{};
  cudaStream_t stream = nullptr;
  // dictionary state
  float *V = nullptr;       // [K][M][M]
  float2 *Vh = nullptr;     // [K][F] F(pad V)
  float2 *th = nullptr;     // [K][F] scaled dual of DictOCSC
  float2 *Dcur = nullptr;   // [K][F] D~_{t,tau}
  float2 *E = nullptr;      // [K][F] D~ + theta^
  float2 *Y = nullptr;      // [K][M][NH]
  float2 *Tm = nullptr;     // [K][M][NH] partial DFT of V
  float *dn = nullptr;      // [F] |D~(p,:)|^2 of the coding dictionary
  // history and factor
  float2 *A = nullptr;      // [F][T]
  float2 *b = nullptr;      // [K][F]
  float2 *L = nullptr;      // [F][T] X = L^-1 (FP32) of the FP64 factor
  float2 *g = nullptr;      // [K][F] y = L^-1 (w b)
  // pending samples
  float2 *Zp = nullptr;     // [max_batch][K][F]
  float2 *xhp = nullptr;    // [max_batch][F]
  // code workspace
  float2 *What = nullptr;   // [max_batch][K][F]
  float *Gam = nullptr;     // [max_batch][K][P]
  float2 *r = nullptr;      // [max_batch][F]
  float2 *tiles = nullptr;  // [max_batch][ceil(K/2)][N][N] tiles for N >= 256
  float2 *tw = nullptr;     // [N] twiddles
  // objective evaluation scratch
  float2 *obj_xh = nullptr;  // [F]
  double *obj_part = nullptr;
  double *obj_out = nullptr; // [kObjChunk]
  int *err = nullptr;       // device error word
  long long n_seen = 0;
  int pending = 0;
  uint64_t version = 0;
  std::string msg;
  std::vector<void *> allocs;
  // bookkeeping and optional per-kernel event timing
  ocsc_counters counters{};
  unsigned prof_mask = 0;
  std::vector<cudaEvent_t> prof_ev[OCSC_K_COUNT];  // start/stop pairs
  size_t prof_used[OCSC_K_COUNT] = {};
};

namespace {

constexpr int kObjChunk = 64;
thread_local std::string g_init_error = "no error";

ocsc_status fail(ocsc_ctx *c, ocsc_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->msg = buf;
  return s;
}

ocsc_status cuda_fail(ocsc_ctx *c, cudaError_t e, const char *where) {
  return fail(c, OCSC_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

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

bool supported_fft(int n) { return n == 64 || n == 128 || n == 256 || n == 512; }
bool large_fft(int n) { return n >= 256; }

int padded_side(int side, int pad) {
  const int need = side + pad;
  for (int n : {64, 128, 256, 512})
    if (n >= need) return n;
  return -1;
}

// splitmix64 (Steele, Lea & Flood 2014) and Box-Muller for the Gaussian
// initial filters of Algorithm 3.
uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

double uniform01(uint64_t seed, uint64_t i) {
  return ((double)(splitmix64(seed ^ splitmix64(i)) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

// Launch one kernel through `fn`, counting it and, when its class is being
// profiled, bracketing it with events on the context's stream.
template <typename Fn>
cudaError_t timed(ocsc_ctx *c, int id, Fn &&fn) {
  c->counters.kernel_launches++;
  if (!(c->prof_mask & (1u << id))) return fn();
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

ocsc_status upload_dict(ocsc_ctx *c, const float *D_host, int normalize) {
  const int MM = c->M * c->M;
  std::vector<float> Dn((size_t)c->K * MM);
  for (int k = 0; k < c->K; ++k) {
    double s = 0;
    for (int e = 0; e < MM; ++e) s += (double)D_host[(size_t)k * MM + e] * D_host[(size_t)k * MM + e];
    const double nrm = std::sqrt(s);
    if (normalize && !(nrm > 0)) return fail(c, OCSC_EINVAL, "filter %d has zero norm", k);
    if (!normalize && nrm > 1.0 + 1e-5) return fail(c, OCSC_EINVAL, "filter %d has norm %.6f > 1", k, nrm);
    const double sc = normalize ? 1.0 / nrm : 1.0;
    for (int e = 0; e < MM; ++e) Dn[(size_t)k * MM + e] = (float)(D_host[(size_t)k * MM + e] * sc);
  }
  cudaError_t e = cudaMemcpyAsync(c->V, Dn.data(), Dn.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "upload filters");
  e = timed(c, OCSC_K_VSTEP_PROJECT, [&] { return launch_vstep_project(1, c->K, c->N, c->M, nullptr, c->V, c->tw, c->Tm, c->stream); });
  if (e == cudaSuccess)
    e = timed(c, OCSC_K_VSTEP_SPECTRUM, [&] { return launch_vstep_spectrum(1, c->K, c->N, c->M, c->Tm, c->tw, c->Vh, nullptr, nullptr, c->stream); });
  if (e != cudaSuccess) return cuda_fail(c, e, "filter spectrum");
  e = cudaMemsetAsync(c->th, 0, (size_t)c->K * c->F * sizeof(float2), c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "reset dual");
  // D~ = F(pad D) also seeds D~_{t,tau}, the coding dictionary when
  // return_feasible = 0.
  e = cudaMemcpyAsync(c->Dcur, c->Vh, (size_t)c->K * c->F * sizeof(float2), cudaMemcpyDeviceToDevice, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "seed D~");
  e = timed(c, OCSC_K_DICT_NORMS, [&] { return launch_dict_norms(c->K, c->F, c->Vh, c->dn, c->stream); });
  if (e != cudaSuccess) return cuda_fail(c, e, "dictionary norms");
  e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "set_dict sync");
  return OCSC_OK;
}

ocsc_status check_device(ocsc_ctx *c) {
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronize");
  int h = 0;
  e = cudaMemcpy(&h, c->err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "read device error word");
  if (h & ERR_PIVOT) {
    cudaMemset(c->err, 0, sizeof(int));
    return fail(c, OCSC_ENUMERIC, "non-positive pivot in the per-frequency Cholesky factorisation");
  }
  return OCSC_OK;
}

}  // namespace

extern "C" {

void ocsc_default_opts(ocsc_opts *o) {
  if (!o) return;
  o->Jz = 50;
  o->Jd = 10;
  o->pad = -1;
  o->max_batch = 1;
  o->fft_size = 128;
  o->warm_start = 1;
  o->return_feasible = 1;
  o->rho_convention = 0;
  o->seed = 0x5EEDull;
}

const char *ocsc_last_error(const ocsc_ctx *ctx) { return ctx ? ctx->msg.c_str() : g_init_error.c_str(); }

void ocsc_destroy(ocsc_ctx *ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  for (void *p : ctx->allocs) cudaFree(p);
  for (auto &v : ctx->prof_ev)
    for (cudaEvent_t e : v) cudaEventDestroy(e);
  delete ctx;
}

ocsc_status ocsc_init(ocsc_ctx **out, int K, int filter_h, int filter_w, double lambda, double rho,
                      const ocsc_opts *opts, void *cuda_stream) {
  if (!out) return OCSC_EINVAL;
  *out = nullptr;
  ocsc_ctx *c = new ocsc_ctx();
  ocsc_default_opts(&c->opts);
  if (opts) c->opts = *opts;
  ocsc_status st = OCSC_OK;
  auto bail = [&](ocsc_status s) {
    g_init_error = c->msg;  // reachable through ocsc_last_error(NULL)
    ocsc_destroy(c);
    return s;
  };
  if (K <= 0 || K > 128) { fail(c, OCSC_EUNSUPPORTED, "K=%d outside 1..128", K); return bail(OCSC_EUNSUPPORTED); }
  if (filter_h != filter_w || filter_h <= 0 || filter_h > 16) {
    fail(c, OCSC_EUNSUPPORTED, "filters must be square with side 1..16");
    return bail(OCSC_EUNSUPPORTED);
  }
  if (!(lambda >= 0) || !(rho > 0)) { fail(c, OCSC_EINVAL, "need lambda >= 0 and rho > 0"); return bail(OCSC_EINVAL); }
  if (!supported_fft(c->opts.fft_size) || c->opts.fft_size < filter_h) {
    fail(c, OCSC_EUNSUPPORTED, "fft_size %d not supported (64, 128, 256 or 512)", c->opts.fft_size);
    return bail(OCSC_EUNSUPPORTED);
  }
  if (c->opts.Jz < 1 || c->opts.Jd < 1 || c->opts.max_batch < 1) {
    fail(c, OCSC_EINVAL, "Jz, Jd and max_batch must be positive");
    return bail(OCSC_EINVAL);
  }
  if (c->opts.pad < 0) c->opts.pad = filter_h - 1;
  c->K = K;
  c->M = filter_h;
  c->N = c->opts.fft_size;
  c->NH = c->N / 2 + 1;
  c->F = c->N * c->NH;
  c->P = c->N * c->N;
  c->T = tri_size(K);
  c->lam = lambda;
  c->rho = rho;
  c->stream = (cudaStream_t)cuda_stream;
  const size_t KF = (size_t)K * c->F, B = (size_t)c->opts.max_batch;
  if ((st = dalloc(c, &c->V, (size_t)K * c->M * c->M)) ||
      (st = dalloc(c, &c->Vh, KF)) || (st = dalloc(c, &c->th, KF)) || (st = dalloc(c, &c->Dcur, KF)) ||
      (st = dalloc(c, &c->E, KF)) || (st = dalloc(c, &c->Y, (size_t)K * c->M * c->NH)) ||
      (st = dalloc(c, &c->Tm, (size_t)K * c->M * c->NH)) ||
      (st = dalloc(c, &c->dn, (size_t)c->F)) || (st = dalloc(c, &c->A, (size_t)c->F * tri_stride(K))) ||
      (st = dalloc(c, &c->b, KF)) || (st = dalloc(c, &c->L, (size_t)c->F * tri_stride(K))) ||
      (st = dalloc(c, &c->g, KF)) || (st = dalloc(c, &c->Zp, B * KF)) ||
      (st = dalloc(c, &c->xhp, B * c->F)) || (st = dalloc(c, &c->What, B * KF)) ||
      (st = dalloc(c, &c->Gam, B * K * c->P)) || (st = dalloc(c, &c->r, B * c->F)) ||
      (st = dalloc(c, &c->tw, (size_t)c->N)) || (st = dalloc(c, &c->err, 1)) ||
      (st = dalloc(c, &c->obj_xh, (size_t)c->F)) ||
      (st = dalloc(c, &c->obj_part, (size_t)objective_partials(c->N))) ||
      (st = dalloc(c, &c->obj_out, (size_t)kObjChunk)))
    return bail(st);
  if (large_fft(c->N) && (st = dalloc(c, &c->tiles, B * ((K + 1) / 2) * (size_t)c->P)))
    return bail(st);
  std::vector<float2> tw(c->N);
  for (int m = 0; m < c->N; ++m) {
    const double a = -2.0 * M_PI * (double)m / (double)c->N;
    tw[m] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  cudaError_t e = cudaMemcpy(c->tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) { cuda_fail(c, e, "upload twiddles"); return bail(OCSC_ECUDA); }
  e = cudaMemset(c->err, 0, sizeof(int));
  if (e != cudaSuccess) { cuda_fail(c, e, "clear error word"); return bail(OCSC_ECUDA); }
  // Algorithm 3: Gaussian random initial filters (normalised in upload_dict).
  std::vector<float> D0((size_t)K * c->M * c->M);
  for (size_t i = 0; i < D0.size(); ++i) {
    const double u1 = uniform01(c->opts.seed, 2 * i), u2 = uniform01(c->opts.seed, 2 * i + 1);
    D0[i] = (float)(std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * M_PI * u2));
  }
  if ((st = upload_dict(c, D0.data(), 1)) != OCSC_OK) return bail(st);
  *out = c;
  return OCSC_OK;
}

ocsc_status ocsc_padded_size(const ocsc_ctx *ctx, int H, int W, int *N) {
  if (!ctx || !N || H <= 0 || W <= 0) return OCSC_EINVAL;
  const int n = padded_side(H > W ? H : W, ctx->opts.pad);
  if (n < 0) return OCSC_EUNSUPPORTED;
  *N = n;
  return OCSC_OK;
}

ocsc_status ocsc_code(ocsc_ctx *c, int n, const float *const *x, const int *H, const int *W,
                      float *const *u) {
  if (!c) return OCSC_EINVAL;
  if (n <= 0 || !x || !H || !W) return fail(c, OCSC_EINVAL, "ocsc_code: bad arguments");
  if (c->pending + n > c->opts.max_batch)
    return fail(c, OCSC_ESTATE, "ocsc_code: %d pending + %d new exceeds max_batch %d; call ocsc_update_dict",
                c->pending, n, c->opts.max_batch);
  for (int i = 0; i < n; ++i) {
    if (!x[i] || H[i] <= 0 || W[i] <= 0) return fail(c, OCSC_EINVAL, "ocsc_code: image %d invalid", i);
    const int side = H[i] > W[i] ? H[i] : W[i];
    if (padded_side(side, c->opts.pad) != c->N)
      return fail(c, OCSC_EUNSUPPORTED, "image %d (%dx%d, pad %d) does not map to FFT size %d", i, H[i], W[i],
                  c->opts.pad, c->N);
  }
  for (int s0 = 0; s0 < n; s0 += kMaxCallImages) {
    ImgBatch bt{};
    bt.n = n - s0 < kMaxCallImages ? n - s0 : kMaxCallImages;
    for (int i = 0; i < bt.n; ++i) {
      bt.x[i] = x[s0 + i];
      bt.u[i] = u ? u[s0 + i] : nullptr;
      bt.H[i] = H[s0 + i];
      bt.W[i] = W[s0 + i];
    }
    const int slot = c->pending + s0;
    float2 *xh = c->xhp + (size_t)slot * c->F;
    const int npairs = (c->K + 1) / 2;
    LargeIO io{};
    io.T = c->tiles ? c->tiles + (size_t)slot * npairs * c->P : nullptr;
    cudaError_t e;
    if (large_fft(c->N)) {
      io.spec_out = xh;
      io.images = 1;
      CodeIter none{};
      e = timed(c, OCSC_K_IMAGE_SPECTRUM, [&] { return launch_large(c->N, LARGE_ROWS_FWD, none, bt, io, bt.n, 1, c->tw, c->stream); });
      if (e == cudaSuccess)
        e = timed(c, OCSC_K_IMAGE_SPECTRUM, [&] { return launch_large(c->N, LARGE_COL_OUT_IMAGE, none, bt, io, bt.n, 1, c->tw, c->stream); });
    } else {
      e = timed(c, OCSC_K_IMAGE_SPECTRUM, [&] { return launch_image_spectrum(c->N, bt, c->tw, xh, c->stream); });
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "image spectrum");
    CodeIter it{};
    it.K = c->K;
    it.F = c->F;
    it.thr = (float)(c->lam / c->rho);
    it.Dh = c->opts.return_feasible ? c->Vh : c->Dcur;
    it.r = c->r + (size_t)slot * c->F;
    it.What = c->What + (size_t)slot * c->K * c->F;
    it.Gam = c->Gam + (size_t)slot * c->K * c->P;
    it.Zp = c->Zp + (size_t)slot * c->K * c->F;
    for (int t = 0; t < c->opts.Jz; ++t) {
      it.first = t == 0;
      it.last = t == c->opts.Jz - 1;
      e = timed(c, OCSC_K_CODE_RESID, [&] {
        return launch_code_resid(c->N, bt.n, c->K, (float)c->rho, it.first, it.Dh, c->dn, xh, it.What,
                                 c->r + (size_t)slot * c->F, c->stream);
      });
      if (e != cudaSuccess) return cuda_fail(c, e, "code_resid");
      if (large_fft(c->N)) {
        e = timed(c, OCSC_K_CODE_PLANE, [&] { return launch_large(c->N, LARGE_COL_IN_ADMM, it, bt, io, bt.n, npairs, c->tw, c->stream); });
        if (e == cudaSuccess)
          e = timed(c, OCSC_K_CODE_PLANE, [&] { return launch_large(c->N, LARGE_ROWS_ADMM, it, bt, io, bt.n, npairs, c->tw, c->stream); });
        if (e == cudaSuccess && !it.last)
          e = timed(c, OCSC_K_CODE_PLANE, [&] { return launch_large(c->N, LARGE_COL_OUT_ADMM, it, bt, io, bt.n, npairs, c->tw, c->stream); });
      } else {
        e = timed(c, OCSC_K_CODE_PLANE, [&] { return launch_code_plane(c->N, it, bt, c->tw, c->stream); });
      }
      if (e != cudaSuccess) return cuda_fail(c, e, "code_plane");
    }
  }
  c->pending += n;
  c->counters.samples_coded += n;
  return OCSC_OK;
}

ocsc_status ocsc_update_dict(ocsc_ctx *c) {
  if (!c) return OCSC_EINVAL;
  if (c->pending == 0) return OCSC_OK;
  const int B = c->pending;
  const double rho_eff = c->opts.rho_convention == 1 ? c->rho * c->P : c->rho;
  cudaError_t e;
  if (!c->opts.warm_start) {
    e = cudaMemsetAsync(c->V, 0, (size_t)c->K * c->M * c->M * sizeof(float), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->Vh, 0, (size_t)c->K * c->F * sizeof(float2), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->th, 0, (size_t)c->K * c->F * sizeof(float2), c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "cold start reset");
  }
  FoldArgs fa{};
  fa.K = c->K;
  fa.F = c->F;
  fa.B = B;
  fa.first = c->n_seen == 0;
  fa.alpha = (double)c->n_seen / (double)(c->n_seen + B);
  fa.beta = 1.0 / (double)(c->n_seen + B);
  fa.w = 1.0;
  fa.rho_eff = rho_eff;
  fa.A = c->A;
  fa.b = c->b;
  fa.Zp = c->Zp;
  fa.xh = c->xhp;
  fa.L = c->L;
  fa.g = c->g;
  fa.err = c->err;
  e = timed(c, OCSC_K_FOLD_FACTOR, [&] { return launch_fold_factor(fa, c->stream); });
  if (e != cudaSuccess) return cuda_fail(c, e, "fold_factor");
  for (int t = 0; t < c->opts.Jd; ++t) {
    e = timed(c, OCSC_K_DSTEP, [&] { return launch_dstep(c->K, c->F, (float)rho_eff, c->L, c->g, c->Vh, c->th, c->Dcur, c->E, c->stream); });
    if (e != cudaSuccess) return cuda_fail(c, e, "dstep");
    e = timed(c, OCSC_K_VSTEP_COLS, [&] { return launch_vstep_cols(c->K, c->N, c->M, c->E, c->tw, c->Y, c->stream); });
    if (e != cudaSuccess) return cuda_fail(c, e, "vstep_cols");
    e = timed(c, OCSC_K_VSTEP_PROJECT, [&] { return launch_vstep_project(0, c->K, c->N, c->M, c->Y, c->V, c->tw, c->Tm, c->stream); });
    if (e != cudaSuccess) return cuda_fail(c, e, "vstep_project");
    e = timed(c, OCSC_K_VSTEP_SPECTRUM, [&] { return launch_vstep_spectrum(0, c->K, c->N, c->M, c->Tm, c->tw, c->Vh, c->th, c->Dcur, c->stream); });
    if (e != cudaSuccess) return cuda_fail(c, e, "vstep_spectrum");
  }
  e = timed(c, OCSC_K_DICT_NORMS, [&] { return launch_dict_norms(c->K, c->F, c->opts.return_feasible ? c->Vh : c->Dcur, c->dn, c->stream); });
  if (e != cudaSuccess) return cuda_fail(c, e, "dict_norms");
  c->n_seen += B;
  c->pending = 0;
  c->version += 1;
  c->counters.dict_updates += 1;
  return OCSC_OK;
}

ocsc_status ocsc_get_dict(ocsc_ctx *c, float *D_host, uint64_t *version) {
  if (!c || !D_host) return c ? fail(c, OCSC_EINVAL, "null output") : OCSC_EINVAL;
  ocsc_status st = check_device(c);
  if (st != OCSC_OK) return st;
  const size_t bytes = (size_t)c->K * c->M * c->M * sizeof(float);
  if (c->opts.return_feasible) {
    cudaError_t e = cudaMemcpy(D_host, c->V, bytes, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "copy filters");
  } else {
    // D_t = H(F^-1(D~_t)) with D~_t = D~_{t,J}: the pruned inverse DFT of the
    // V-step applied to D~ alone, read back without projection.
    return fail(c, OCSC_EUNSUPPORTED, "get_dict with return_feasible=0 is not implemented");
  }
  if (version) *version = c->version;
  return OCSC_OK;
}

ocsc_status ocsc_set_dict(ocsc_ctx *c, const float *D_host, int normalize) {
  if (!c || !D_host) return c ? fail(c, OCSC_EINVAL, "null input") : OCSC_EINVAL;
  return upload_dict(c, D_host, normalize);
}

ocsc_status ocsc_sync(ocsc_ctx *c) {
  if (!c) return OCSC_EINVAL;
  return check_device(c);
}

// Real 2D FFT building blocks; for N >= 256 they run in chunks of pairs that
// fit the context's tile buffer.
static ocsc_status fft2_any(ocsc_ctx *c, int inverse, const float *in, float *out, int planes, const char *name) {
  if (!large_fft(c->N)) {
    cudaError_t e = timed(c, OCSC_K_COUNT, [&] { return launch_fft2(c->N, inverse, in, out, planes, c->tw, c->stream); });
    return e == cudaSuccess ? OCSC_OK : cuda_fail(c, e, name);
  }
  const int cap_pairs = c->opts.max_batch * ((c->K + 1) / 2);
  const size_t spec = (size_t)c->F * 2, real = (size_t)c->P;  // floats per plane
  for (int p0 = 0; p0 < planes; p0 += 2 * cap_pairs) {
    const int np = planes - p0 < 2 * cap_pairs ? planes - p0 : 2 * cap_pairs;
    LargeIO io{};
    io.T = c->tiles;
    io.planes = np;
    CodeIter none{};
    ImgBatch b{};
    cudaError_t e;
    if (!inverse) {
      io.real_in = in + (size_t)p0 * real;
      io.spec_out = reinterpret_cast<float2 *>(out + (size_t)p0 * spec);
      e = timed(c, OCSC_K_COUNT, [&] { return launch_large(c->N, LARGE_ROWS_FWD, none, b, io, 1, (np + 1) / 2, c->tw, c->stream); });
      if (e == cudaSuccess)
        e = timed(c, OCSC_K_COUNT, [&] { return launch_large(c->N, LARGE_COL_OUT_R2C, none, b, io, 1, (np + 1) / 2, c->tw, c->stream); });
    } else {
      io.spec_in = reinterpret_cast<const float2 *>(in + (size_t)p0 * spec);
      io.real_out = out + (size_t)p0 * real;
      e = timed(c, OCSC_K_COUNT, [&] { return launch_large(c->N, LARGE_COL_IN_C2R, none, b, io, 1, (np + 1) / 2, c->tw, c->stream); });
      if (e == cudaSuccess)
        e = timed(c, OCSC_K_COUNT, [&] { return launch_large(c->N, LARGE_ROWS_C2R, none, b, io, 1, (np + 1) / 2, c->tw, c->stream); });
    }
    if (e != cudaSuccess) return cuda_fail(c, e, name);
  }
  return OCSC_OK;
}

ocsc_status ocsc_fft2_r2c(ocsc_ctx *c, const float *x, float *X, int planes) {
  if (!c) return OCSC_EINVAL;
  if (!x || !X || planes < 0) return fail(c, OCSC_EINVAL, "fft2_r2c: bad arguments");
  return fft2_any(c, 0, x, X, planes, "fft2_r2c");
}

ocsc_status ocsc_fft2_c2r(ocsc_ctx *c, const float *X, float *x, int planes) {
  if (!c) return OCSC_EINVAL;
  if (!x || !X || planes < 0) return fail(c, OCSC_EINVAL, "fft2_c2r: bad arguments");
  return fft2_any(c, 1, X, x, planes, "fft2_c2r");
}

ocsc_status ocsc_drop_pending(ocsc_ctx *c) {
  if (!c) return OCSC_EINVAL;
  c->pending = 0;
  return OCSC_OK;
}

ocsc_status ocsc_objective(ocsc_ctx *c, int n, const float *const *x, const int *H, const int *W,
                           const float *const *u, double *out_host) {
  if (!c) return OCSC_EINVAL;
  if (n < 0 || (n > 0 && (!x || !H || !W || !u || !out_host)))
    return fail(c, OCSC_EINVAL, "ocsc_objective: bad arguments");
  for (int i = 0; i < n; ++i) {
    if (!x[i] || !u[i] || H[i] <= 0 || W[i] <= 0) return fail(c, OCSC_EINVAL, "ocsc_objective: sample %d invalid", i);
    if (padded_side(H[i] > W[i] ? H[i] : W[i], c->opts.pad) != c->N)
      return fail(c, OCSC_EUNSUPPORTED, "sample %d does not map to FFT size %d", i, c->N);
  }
  const float2 *Dh = c->opts.return_feasible ? c->Vh : c->Dcur;
  float2 *Uh = c->What;  // coding workspace of slot 0, idle between ocsc_code calls
  for (int s0 = 0; s0 < n; s0 += kObjChunk) {
    const int m = n - s0 < kObjChunk ? n - s0 : kObjChunk;
    for (int i = 0; i < m; ++i) {
      ImgBatch bt{};
      bt.n = 1;
      bt.x[0] = x[s0 + i];
      bt.u[0] = nullptr;
      bt.H[0] = H[s0 + i];
      bt.W[0] = W[s0 + i];
      cudaError_t e = cudaSuccess;
      if (large_fft(c->N)) {
        CodeIter none{};
        LargeIO io{};
        io.T = c->tiles;
        io.spec_out = c->obj_xh;
        io.images = 1;
        e = timed(c, OCSC_K_COUNT, [&] { return launch_large(c->N, LARGE_ROWS_FWD, none, bt, io, 1, 1, c->tw, c->stream); });
        if (e == cudaSuccess)
          e = timed(c, OCSC_K_COUNT, [&] { return launch_large(c->N, LARGE_COL_OUT_IMAGE, none, bt, io, 1, 1, c->tw, c->stream); });
        LargeIO jo{};
        jo.T = c->tiles;
        jo.real_in = u[s0 + i];
        jo.spec_out = Uh;
        jo.planes = c->K;
        const int np = (c->K + 1) / 2;
        if (e == cudaSuccess)
          e = timed(c, OCSC_K_COUNT, [&] { return launch_large(c->N, LARGE_ROWS_FWD, none, bt, jo, 1, np, c->tw, c->stream); });
        if (e == cudaSuccess)
          e = timed(c, OCSC_K_COUNT, [&] { return launch_large(c->N, LARGE_COL_OUT_R2C, none, bt, jo, 1, np, c->tw, c->stream); });
      } else {
        e = timed(c, OCSC_K_COUNT, [&] { return launch_image_spectrum(c->N, bt, c->tw, c->obj_xh, c->stream); });
        if (e == cudaSuccess)
          e = timed(c, OCSC_K_COUNT, [&] { return launch_fft2(c->N, 0, u[s0 + i], reinterpret_cast<float *>(Uh), c->K, c->tw, c->stream); });
      }
      if (e == cudaSuccess) {
        c->counters.kernel_launches += 2;  // three kernels in launch_objective
        e = timed(c, OCSC_K_COUNT, [&] {
          return launch_objective(c->K, c->N, c->lam, Dh, c->obj_xh, Uh, u[s0 + i], c->obj_part, c->obj_out + i,
                                  c->stream);
        });
      }
      if (e != cudaSuccess) return cuda_fail(c, e, "objective");
    }
    cudaError_t e = cudaMemcpyAsync(out_host + s0, c->obj_out, m * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "objective readback");
  }
  return OCSC_OK;
}

ocsc_status ocsc_get_counters(const ocsc_ctx *c, ocsc_counters *out) {
  if (!c || !out) return OCSC_EINVAL;
  *out = c->counters;
  return OCSC_OK;
}

ocsc_status ocsc_profile(ocsc_ctx *c, unsigned mask) {
  if (!c) return OCSC_EINVAL;
  c->prof_mask = mask & ((1u << OCSC_K_COUNT) - 1u);
  return OCSC_OK;
}

ocsc_status ocsc_profile_read(ocsc_ctx *c, int kernel, double *total_ms, uint64_t *launches) {
  if (!c) return OCSC_EINVAL;
  if (kernel < 0 || kernel >= OCSC_K_COUNT || !total_ms || !launches)
    return fail(c, OCSC_EINVAL, "profile_read: bad arguments");
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "profile_read sync");
  double ms = 0;
  auto &ev = c->prof_ev[kernel];
  const size_t used = c->prof_used[kernel];
  for (size_t i = 0; i + 1 < used; i += 2) {
    float t = 0;
    e = cudaEventElapsedTime(&t, ev[i], ev[i + 1]);
    if (e != cudaSuccess) return cuda_fail(c, e, "profile_read elapsed");
    ms += t;
  }
  *total_ms = ms;
  *launches = used / 2;
  c->prof_used[kernel] = 0;
  return OCSC_OK;
}

}  // extern "C"
