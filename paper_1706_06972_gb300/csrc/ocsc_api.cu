// C-ABI runtime: context state, allocation and the launch sequences of
// Algorithm 3 (code, fold, DictOCSC).  All method arithmetic runs in the
// kernels of code_admm.cu, code_large.cu, dict_update.cu and objective.cu;
// this file only sequences them.
//
// A context holds one spatial dictionary V and one or more size classes, one
// per FFT side N.  Each class keeps its own frequency-domain state (history,
// factor, dual, coding spectrum) and coding workspaces; the dictionary step is
// the consensus form of DictOCSC over the classes that have seen samples
// (with a single class it is Algorithm 2 as is).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ctx.h"

using namespace ocsc;

namespace {

constexpr int kObjChunk = 64;
thread_local std::string g_init_error = "no error";

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

// V^_c = F_c(pad V) for one class, without touching its dual.
cudaError_t class_spectrum(ocsc_ctx *c, SizeClass &s) {
  cudaError_t e = timed(c, OCSC_K_VSTEP_SPECTRUM, [&] { return launch_vstep_partial_dft(c->K, s.N, c->M, c->V, s.tw, s.Tm, c->stream); });
  if (e == cudaSuccess)
    e = timed(c, OCSC_K_VSTEP_SPECTRUM, [&] { return launch_vstep_spectrum(1, c->K, s.N, c->M, s.Tm, s.tw, s.Vh, nullptr, nullptr, c->stream); });
  return e;
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
  for (SizeClass &s : c->cls) {
    const size_t kf = (size_t)c->K * s.F * sizeof(float2);
    e = class_spectrum(c, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.th, 0, kf, c->stream);
    // D~ = F(pad D) also seeds D~_{t,tau}, the coding dictionary when
    // return_feasible = 0.
    if (e == cudaSuccess) e = cudaMemcpyAsync(s.Dcur, s.Vh, kf, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess)
      e = timed(c, OCSC_K_DICT_NORMS, [&] { return launch_dict_norms(c->K, s.F, s.Vh, s.dn, c->stream); });
    if (e != cudaSuccess) return cuda_fail(c, e, "set dictionary");
  }
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
  if (h & ERR_TIMEOUT) {
    cudaMemset(c->err, 0, sizeof(int));
    // A persistent launch that gave up may have left the arrival counters of
    // the N >= 256 spectral units part-way; they must start at zero.
    for (SizeClass &s : c->cls)
      if (s.cnt) cudaMemset(s.cnt, 0, (size_t)c->opts.max_batch * (s.N / 2) * sizeof(int));
    return fail(c, OCSC_ETIMEOUT, "a bounded device wait gave up (tensor-core history fold or persistent coder barrier)");
  }
  return OCSC_OK;
}

ocsc_status alloc_class(ocsc_ctx *c, SizeClass &s, int N) {
  s.N = N;
  s.NH = N / 2 + 1;
  s.F = N * s.NH;
  s.P = N * N;
  // A band context keeps the history and factor of its own rows only.
  s.p0 = c->opts.band_hi > 0 ? c->opts.band_lo * s.NH : 0;
  s.Fb = c->opts.band_hi > 0 ? (c->opts.band_hi - c->opts.band_lo) * s.NH : s.F;
  const int K = c->K, M = c->M;
  const size_t KF = (size_t)K * s.F, B = (size_t)c->opts.max_batch, TS = (size_t)tri_stride(K);
  const size_t FT = (size_t)s.Fb * TS;
  ocsc_status st;
  if ((st = dalloc(c, &s.tw, (size_t)N)) || (st = dalloc(c, &s.Vh, KF)) || (st = dalloc(c, &s.th, KF)) ||
      (st = dalloc(c, &s.Dcur, KF)) || (st = dalloc(c, &s.E, KF)) ||
      (st = dalloc(c, &s.Y, (size_t)K * M * s.NH)) || (st = dalloc(c, &s.Tm, (size_t)K * M * s.NH)) ||
      (st = dalloc(c, &s.dn, (size_t)s.F)) || (st = dalloc(c, &s.A, FT)) ||
      (st = dalloc(c, &s.b, KF)) || (st = dalloc(c, &s.X, FT)) || (st = dalloc(c, &s.y, KF)) ||
      (st = dalloc(c, &s.Zp, B * KF)) || (st = dalloc(c, &s.xhp, B * s.F)) ||
      (st = dalloc(c, &s.obj_xh, (size_t)s.F)))
    return st;
  if (c->opts.history == 1 && (st = dalloc(c, &s.Csf, (size_t)s.F * TS))) return st;
  if (c->opts.precision > 0) {
    if ((st = dalloc(c, &s.Alo, FT))) return st;
    cudaError_t e = cudaMemset(s.Alo, 0, FT * sizeof(float2));
    if (e != cudaSuccess) return cuda_fail(c, e, "clear history compensation");
  }
  if (c->opts.precision == 3) {
    if ((st = dalloc(c, &s.blo, KF))) return st;
    cudaError_t e = cudaMemset(s.blo, 0, KF * sizeof(float2));
    if (e != cudaSuccess) return cuda_fail(c, e, "clear history compensation");
  }
  std::vector<float2> tw(N);
  for (int m = 0; m < N; ++m) {
    const double a = -2.0 * M_PI * (double)m / (double)N;
    tw[m] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  cudaError_t e = cudaMemcpy(s.tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(c, e, "upload twiddles");
  return OCSC_OK;
}

// The coding workspace of a class (per slot: W^ and r, or the pair tiles and
// partial sums; the spatial state), allocated at the class's first coding,
// objective or FFT call, so that a context used only through the server never
// holds it.
ocsc_status ensure_code_ws(ocsc_ctx *c, SizeClass &s) {
  if (s.Gam) return OCSC_OK;
  const int K = c->K, N = s.N;
  const size_t KF = (size_t)K * s.F, B = (size_t)c->opts.max_batch;
  ocsc_status st;
  if ((st = dalloc(c, &s.What, (large_fft(N) ? 1 : B) * KF)) || (st = dalloc(c, &s.r, B * s.F)))
    return st;
  if (large_fft(N)) {
    const int npairs = (K + 1) / 2;
    if ((st = dalloc(c, &s.tiles, B * npairs * (size_t)s.P)) ||
        (st = dalloc(c, &s.part, B * large_stages(N, npairs) * (size_t)s.F)) ||
        (st = dalloc(c, &s.cnt, B * (size_t)(N / 2))))
      return st;
    cudaError_t e = cudaMemset(s.cnt, 0, B * (size_t)(N / 2) * sizeof(int));
    if (e != cudaSuccess) return cuda_fail(c, e, "clear counters");
  }
  return dalloc(c, &s.Gam, B * K * (size_t)s.P);  // last: marks the workspace complete
}

}  // namespace

extern "C" {

void ocsc_default_opts(ocsc_opts *o) {
  if (!o) return;
  o->Jz = 50;
  o->Jd = 10;
  o->pad = -1;
  o->max_batch = 1;
  for (int i = 0; i < OCSC_MAX_FFT_SIZES; ++i) o->fft_sizes[i] = 0;
  o->fft_sizes[0] = 128;
  o->warm_start = 1;
  o->return_feasible = 1;
  o->rho_convention = 0;
  o->precision = 0;
  o->autotune = 1;
  o->graphs = 0;
  o->history = 0;
  o->persistent = 0;
  o->band_lo = 0;
  o->band_hi = 0;
  o->seed = 0x5EEDull;
}

const char *ocsc_last_error(const ocsc_ctx *ctx) { return ctx ? ctx->msg.c_str() : g_init_error.c_str(); }

void ocsc_destroy(ocsc_ctx *ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  for (ocsc::GraphEntry &g : ctx->graphs) cudaGraphExecDestroy(g.exec);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
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
  if (K <= 0 || K > 256) { fail(c, OCSC_EUNSUPPORTED, "K=%d outside 1..256", K); return bail(OCSC_EUNSUPPORTED); }
  if (filter_h != filter_w || filter_h <= 0 || filter_h > 16) {
    fail(c, OCSC_EUNSUPPORTED, "filters must be square with side 1..16");
    return bail(OCSC_EUNSUPPORTED);
  }
  if (!(lambda >= 0) || !(rho > 0)) { fail(c, OCSC_EINVAL, "need lambda >= 0 and rho > 0"); return bail(OCSC_EINVAL); }
  if (c->opts.history < 0 || c->opts.history > 1) {
    fail(c, OCSC_EINVAL, "history must be 0 or 1");
    return bail(OCSC_EINVAL);
  }
  if (c->opts.history == 1 &&
      (c->opts.precision != 0 || K > 128 || c->opts.fft_sizes[1] != 0 || c->opts.rho_convention != 1)) {
    fail(c, OCSC_EUNSUPPORTED, "history = 1 needs rho_convention 1, precision 0, K <= 128 and one FFT size");
    return bail(OCSC_EUNSUPPORTED);
  }
  if (c->opts.precision < 0 || c->opts.precision > 3) {
    fail(c, OCSC_EINVAL, "precision must be 0, 1, 2 or 3");
    return bail(OCSC_EINVAL);
  }
  if (c->opts.precision == 3 && K > kSmallK) {
    fail(c, OCSC_EUNSUPPORTED, "precision 3 (double-float history) needs K <= %d", kSmallK);
    return bail(OCSC_EUNSUPPORTED);
  }
  if (c->opts.Jz < 1 || c->opts.Jd < 1 || c->opts.max_batch < 1) {
    fail(c, OCSC_EINVAL, "Jz, Jd and max_batch must be positive");
    return bail(OCSC_EINVAL);
  }
  std::vector<int> sizes;
  for (int i = 0; i < OCSC_MAX_FFT_SIZES && c->opts.fft_sizes[i] != 0; ++i) {
    const int n = c->opts.fft_sizes[i];
    if (!supported_fft(n) || n < filter_h) {
      fail(c, OCSC_EUNSUPPORTED, "fft size %d not supported (64, 96, 128, 144, 192, 256, 288, 384, 512, 576)", n);
      return bail(OCSC_EUNSUPPORTED);
    }
    for (int m : sizes)
      if (m == n) { fail(c, OCSC_EINVAL, "fft size %d listed twice", n); return bail(OCSC_EINVAL); }
    sizes.push_back(n);
  }
  if (sizes.empty()) { fail(c, OCSC_EINVAL, "no fft size given"); return bail(OCSC_EINVAL); }
  if (c->opts.band_hi != 0) {
    const int N = sizes[0], lo = c->opts.band_lo, hi = c->opts.band_hi;
    if (sizes.size() != 1 || lo < 0 || hi > N || lo >= hi || (hi - lo) % 2 || c->opts.history != 0 ||
        (c->opts.precision != 0 && c->opts.precision != 3) || K > kSmallK || !c->opts.return_feasible) {
      fail(c, OCSC_EUNSUPPORTED, "a band context needs one FFT size N, 0 <= band_lo < band_hi <= N with an "
           "even row count, history 0, precision 0 or 3, K <= %d and return_feasible 1", kSmallK);
      return bail(OCSC_EUNSUPPORTED);
    }
  }
  if (sizes.size() > 1 && (c->opts.rho_convention != 0 || !c->opts.return_feasible)) {
    fail(c, OCSC_EUNSUPPORTED, "several size classes need rho_convention = 0 and return_feasible = 1");
    return bail(OCSC_EUNSUPPORTED);
  }
  if (c->opts.pad < 0) c->opts.pad = filter_h - 1;
  c->K = K;
  c->M = filter_h;
  c->T = tri_size(K);
  c->lam = lambda;
  c->rho = rho;
  c->stream = (cudaStream_t)cuda_stream;
  int max_partials = 0;
  c->cls.resize(sizes.size());
  for (size_t i = 0; i < sizes.size(); ++i) {
    if ((st = alloc_class(c, c->cls[i], sizes[i])) != OCSC_OK) return bail(st);
    max_partials = std::max(max_partials, objective_partials(sizes[i]));
  }
  if (K > kSmallK) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 1;
    c->work_ctas = sms;
    if ((st = dalloc(c, &c->work, factor_big_workspace(K, sms)))) return bail(st);
  }
  if ((st = dalloc(c, &c->V, (size_t)K * c->M * c->M)) || (st = dalloc(c, &c->Dpub, (size_t)K * c->M * c->M)) || (st = dalloc(c, &c->err, 1)) || (st = dalloc(c, &c->bar, 2)) ||
      (st = dalloc(c, &c->obj_part, (size_t)std::max(max_partials, 2 * kObjL1Blocks))) ||
      (st = dalloc(c, &c->obj_out, (size_t)4 * kObjChunk)) || (st = dalloc(c, &c->order, (size_t)K)))
    return bail(st);
  cudaError_t e = cudaMemset(c->err, 0, sizeof(int));
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
  const int k = class_of(ctx, H, W);
  if (k < 0) return OCSC_EUNSUPPORTED;
  *N = ctx->cls[k].N;
  return OCSC_OK;
}

// Enqueue the coding of one chunk of images of one class (sample spectra and
// Jz ADMM iterations) for the images, outputs and slots in bt.
// Sample spectra x~ = F(pad x) of the images in bt into their slots.
static ocsc_status enqueue_spectra(ocsc_ctx *c, SizeClass &s, const ImgBatch &bt) {
  LargeIO io{};
  io.T = s.tiles;
  io.tile_pairs = (c->K + 1) / 2;
  cudaError_t e;
  if (large_fft(s.N)) {
    io.spec_out = s.xhp;
    CodeIter none{};
    e = timed(c, OCSC_K_IMAGE_SPECTRUM, [&] { return launch_large(s.N, LARGE_SPAT_IMAGE, none, bt, io, bt.n, 1, s.tw, c->stream); });
    if (e == cudaSuccess)
      e = timed(c, OCSC_K_IMAGE_SPECTRUM, [&] { return launch_large(s.N, LARGE_SPEC_IMAGE, none, bt, io, bt.n, 1, s.tw, c->stream); });
  } else {
    e = timed(c, OCSC_K_IMAGE_SPECTRUM, [&] { return launch_image_spectrum(s.N, bt, s.tw, s.xhp, c->stream); });
  }
  return e == cudaSuccess ? OCSC_OK : cuda_fail(c, e, "image spectrum");
}

// Code-ADMM parameters and workspaces of a class (batch mode).
static CodeIter class_iter(const ocsc_ctx *c, const SizeClass &s) {
  CodeIter it{};
  it.K = c->K;
  it.F = s.F;
  it.thr = (float)(c->lam / c->rho);
  it.Dh = coding_spectrum(c, s);
  it.r = s.r;
  it.What = s.What;
  it.Gam = s.Gam;
  it.Zp = s.Zp;
  it.serve = 0;
  it.check = 1;
  it.rho = (float)c->rho;
  it.dn = s.dn;
  it.xh = s.xhp;
  it.part = s.part;
  it.cnt = s.cnt;
  return it;
}

static ocsc_status enqueue_chunk(ocsc_ctx *c, SizeClass &s, const ImgBatch &bt) {
  const int npairs = (c->K + 1) / 2;
  LargeIO io{};
  io.T = s.tiles;
  io.tile_pairs = npairs;
  cudaError_t e;
  ocsc_status sst = enqueue_spectra(c, s, bt);
  if (sst != OCSC_OK) return sst;
  CodeIter it = class_iter(c, s);
  if (large_fft(s.N)) {
    if (s.spat_cb == 0) {
      s.spat_cb = large_default_cb(s.N);
      if (c->opts.autotune) {
        // Time both spatial tile widths on this call's slots before the first
        // iteration (which rewrites every tile row and all U it touches).
        CodeIter tt = it;
        tt.first = 1;
        tt.last = 0;
        float best = -1.f;
        for (int cb : {8, 16}) {
          if (!large_cb_ok(s.N, cb)) continue;
          LargeIO tio = io;
          tio.spat_cb = cb;
          const float ms = time_runs(c, 2, [&] {
            return launch_large(s.N, LARGE_SPAT_ADMM, tt, bt, tio, bt.n, npairs, s.tw, c->stream);
          });
          if (ms < 0.f) return cuda_fail(c, cudaGetLastError(), "autotune spatial tile");
          if (best < 0.f || ms < best) {
            best = ms;
            s.spat_cb = cb;
          }
        }
      }
    }
    io.spat_cb = s.spat_cb;
  } else if (s.plane_ctas == 0) {
    s.plane_ctas = 2;
    s.plane_ahead = 1;
    s.plane_threads = 256;
    if (c->opts.autotune) {
      // Time the plane kernel's CTA shapes (256 threads at 2 or 3 CTAs per
      // SM, 512 threads at 2, and 512 threads at 1 as persistent CTAs with
      // two tiles), each with and without the L2 prefetch one
      // residency ahead, as a middle iteration (W^ and Gamma read and
      // written) on this call's slots before its first iteration, which
      // rewrites all of W^ and Gamma it touches: the timing runs read stale
      // state and multipliers, harmlessly.
      CodeIter tt = it;
      tt.first = 0;
      tt.last = 0;
      float best = -1.f;
      const int shapes[4][2] = {{256, 2}, {256, 3}, {512, 2}, {512, 1}};
      for (const auto &sh : shapes) {
        if (!plane_shape_ok(s.N, sh[0], sh[1])) continue;
        for (int ahead : {0, 1}) {
          if (sh[1] == 1 && ahead) continue;  // the persistent form has no look-ahead
          const float ms = time_runs(
              c, 2, [&] { return launch_code_plane(s.N, tt, bt, s.tw, c->stream, sh[1], ahead != 0, sh[0]); });
          if (ms < 0.f) return cuda_fail(c, cudaGetLastError(), "autotune coding plane");
          if (best < 0.f || ms < best) {
            best = ms;
            s.plane_threads = sh[0];
            s.plane_ctas = sh[1];
            s.plane_ahead = ahead;
          }
        }
      }
    }
  }
  for (int t = 0; t < c->opts.Jz; ++t) {
    it.first = t == 0;
    it.last = t == c->opts.Jz - 1;
    if (large_fft(s.N)) {
      e = cudaSuccess;
      if (!it.first)
        e = timed(c, OCSC_K_CODE_RESID, [&] { return launch_large(s.N, LARGE_SPEC_DOT, it, bt, io, bt.n, npairs, s.tw, c->stream); });
      if (e == cudaSuccess)
        e = timed(c, OCSC_K_CODE_RESID, [&] { return launch_large(s.N, LARGE_SPEC_Z, it, bt, io, bt.n, npairs, s.tw, c->stream); });
      if (e == cudaSuccess)
        e = timed(c, OCSC_K_CODE_PLANE, [&] { return launch_large(s.N, LARGE_SPAT_ADMM, it, bt, io, bt.n, npairs, s.tw, c->stream); });
    } else {
      e = timed(c, OCSC_K_CODE_RESID, [&] { return launch_code_resid(s.N, bt, it, (float)c->rho, s.dn, s.xhp, c->stream); });
      if (e == cudaSuccess)
        e = timed(c, OCSC_K_CODE_PLANE, [&] {
          return launch_code_plane(s.N, it, bt, s.tw, c->stream, s.plane_ctas, s.plane_ahead != 0, s.plane_threads);
        });
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "code iteration");
  }
  return OCSC_OK;
}

// Graph path of one chunk: images copied into the class's staging slots, the
// captured coding graph of this chunk shape replayed, codes copied out.  A
// shape is captured at its second occurrence (the first runs eagerly, which
// also autotunes); false = not handled here (caller runs it eagerly).
static bool graph_chunk(ocsc_ctx *c, SizeClass &s, const ImgBatch &user, ocsc_status *st) {
  *st = OCSC_OK;
  constexpr unsigned coding_kinds =
      (1u << OCSC_K_IMAGE_SPECTRUM) | (1u << OCSC_K_CODE_RESID) | (1u << OCSC_K_CODE_PLANE);
  if (!c->opts.graphs || (c->prof_mask & coding_kinds)) return false;
  bool want_u = false;
  std::string key = std::to_string(s.N) + ":" + std::to_string(user.n) + ":" + std::to_string(user.slot[0]);
  for (int i = 0; i < user.n; ++i) {
    key += ":" + std::to_string(user.H[i]) + "x" + std::to_string(user.W[i]) + (user.u[i] ? "u" : "-");
    want_u = want_u || user.u[i];
  }
  GraphEntry *g = nullptr;
  for (GraphEntry &ge : c->graphs)
    if (ge.key == key) g = &ge;
  if (!g) {
    if (c->graph_seen.insert(key).second) return false;  // first occurrence: eager
    if (c->graphs.size() >= kMaxGraphs) return false;
  }
  const size_t P = (size_t)s.P, KP = (size_t)c->K * s.P;
  if (!s.xstage && dalloc(c, &s.xstage, (size_t)c->opts.max_batch * P) != OCSC_OK) return false;
  if (want_u && !s.ustage && dalloc(c, &s.ustage, (size_t)c->opts.max_batch * KP) != OCSC_OK) return false;
  ImgBatch st_b = user;
  for (int i = 0; i < user.n; ++i) {
    st_b.x[i] = s.xstage + (size_t)user.slot[i] * P;
    st_b.u[i] = user.u[i] ? s.ustage + (size_t)user.slot[i] * KP : nullptr;
  }
  if (!g) {
    // Capture on a library stream (the context's stream may be the legacy
    // default stream, which cannot capture); nothing executes during capture.
    cudaError_t e = cudaSuccess;
    if (!c->cap_stream) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    cudaGraph_t graph = nullptr;
    if (e == cudaSuccess) e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
      *st = cuda_fail(c, e, "graph capture");
      return true;
    }
    const uint64_t counted = c->counters.kernel_launches;
    cudaStream_t user_stream = c->stream;
    c->stream = c->cap_stream;
    const ocsc_status es = enqueue_chunk(c, s, st_b);
    c->stream = user_stream;
    c->counters.kernel_launches = counted;  // the replay below counts them
    e = cudaStreamEndCapture(c->cap_stream, &graph);
    if (es != OCSC_OK || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      *st = es != OCSC_OK ? es : cuda_fail(c, e, "graph capture");
      return true;
    }
    GraphEntry ne;
    ne.key = key;
    cudaGraphGetNodes(graph, nullptr, &ne.kernels);
    e = cudaGraphInstantiate(&ne.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      *st = cuda_fail(c, e, "graph instantiate");
      return true;
    }
    c->graphs.push_back(ne);
    g = &c->graphs.back();
  }
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < user.n && e == cudaSuccess; ++i)
    e = cudaMemcpyAsync(s.xstage + (size_t)user.slot[i] * P, user.x[i], (size_t)user.H[i] * user.W[i] * sizeof(float),
                        cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess) e = cudaGraphLaunch(g->exec, c->stream);
  for (int i = 0; i < user.n && e == cudaSuccess; ++i)
    if (user.u[i]) e = cudaMemcpyAsync(user.u[i], st_b.u[i], KP * sizeof(float), cudaMemcpyDeviceToDevice, c->stream);
  if (e != cudaSuccess) *st = cuda_fail(c, e, "graph launch");
  c->counters.graph_launches++;
  c->counters.kernel_launches += g->kernels;
  return true;
}

// Code the images of one class (all of the same padded size).
static ocsc_status code_class(ocsc_ctx *c, SizeClass &s, const std::vector<int> &idx, const float *const *x,
                              const int *H, const int *W, float *const *u) {
  const int n = (int)idx.size();
  ocsc_status wst = ensure_code_ws(c, s);
  if (wst != OCSC_OK) return wst;
  for (int s0 = 0; s0 < n; s0 += kMaxCallImages) {
    ImgBatch bt{};
    bt.n = n - s0 < kMaxCallImages ? n - s0 : kMaxCallImages;
    for (int i = 0; i < bt.n; ++i) {
      const int j = idx[s0 + i];
      bt.x[i] = x[j];
      bt.u[i] = u ? u[j] : nullptr;
      bt.H[i] = H[j];
      bt.W[i] = W[j];
      bt.slot[i] = s.pending + s0 + i;
      bt.iter[i] = 0;
    }
    ocsc_status st;
    if (!graph_chunk(c, s, bt, &st)) st = enqueue_chunk(c, s, bt);
    if (st != OCSC_OK) return st;
  }
  s.pending += n;
  return OCSC_OK;
}

// Persistent path: the images of the classes in pcls (each of FFT size 64,
// 128, 256 or 512), in chunks of at most kMaxCallImages ordered by class; per
// chunk the sample spectra of each class, then one cooperative launch running
// all Jz iterations of every image of the chunk.
static ocsc_status code_persistent(ocsc_ctx *c, const std::vector<int> &pcls,
                                   const std::vector<std::vector<int>> &groups, const float *const *x,
                                   const int *H, const int *W, float *const *u) {
  std::vector<std::pair<int, int>> all;  // (class, image index)
  for (int k : pcls) {
    SizeClass &s = c->cls[k];
    ocsc_status st = ensure_code_ws(c, s);
    if (st != OCSC_OK) return st;
    if (large_fft(s.N) && s.spat_cb == 0) s.spat_cb = large_default_cb(s.N);
    for (int j : groups[k]) all.emplace_back(k, j);
  }
  std::vector<int> used(c->cls.size(), 0);
  for (size_t s0 = 0; s0 < all.size(); s0 += kMaxCallImages) {
    const int m = (int)std::min<size_t>(kMaxCallImages, all.size() - s0);
    PersistArgs pa{};
    pa.b.n = m;
    pa.Jz = c->opts.Jz;
    pa.K = c->K;
    pa.bar = c->bar;
    pa.err = c->err;
    pa.polls = c->wait_polls;
    for (int i = 0; i < m; ++i) {
      const int k = all[s0 + i].first, j = all[s0 + i].second;
      SizeClass &s = c->cls[k];
      pa.b.x[i] = x[j];
      pa.b.u[i] = u ? u[j] : nullptr;
      pa.b.H[i] = H[j];
      pa.b.W[i] = W[j];
      pa.b.slot[i] = s.pending + used[k]++;
      pa.b.iter[i] = 0;
      if (pa.ncls == 0 || pa.c[pa.ncls - 1].N != s.N) {
        PersistClass &pc = pa.c[pa.ncls++];
        pc.N = s.N;
        pc.n0 = i;
        pc.n = 0;
        for (int v = 0; v < 3; ++v) {
          pc.it[v] = class_iter(c, s);
          pc.it[v].first = v == 0;
          pc.it[v].last = v == 2 || c->opts.Jz == 1;
        }
        pc.tw = s.tw;
        pc.io.T = s.tiles;
        pc.io.tile_pairs = (c->K + 1) / 2;
        pc.io.spat_cb = s.spat_cb;
        pc.cb = s.spat_cb;
        pc.S = large_fft(s.N) ? large_stages(s.N, (c->K + 1) / 2) : 0;
      }
      pa.c[pa.ncls - 1].n++;
    }
    for (int q = 0; q < pa.ncls; ++q) {
      const PersistClass &pc = pa.c[q];
      ImgBatch bt{};
      bt.n = pc.n;
      for (int i = 0; i < pc.n; ++i) {
        bt.x[i] = pa.b.x[pc.n0 + i];
        bt.u[i] = pa.b.u[pc.n0 + i];
        bt.H[i] = pa.b.H[pc.n0 + i];
        bt.W[i] = pa.b.W[pc.n0 + i];
        bt.slot[i] = pa.b.slot[pc.n0 + i];
      }
      SizeClass *sp = nullptr;
      for (SizeClass &sc : c->cls)
        if (sc.N == pc.N) sp = &sc;
      ocsc_status st = enqueue_spectra(c, *sp, bt);
      if (st != OCSC_OK) return st;
    }
    const size_t smem = persist_smem_bytes(pa);
    const int grid = persist_grid(smem);
    if (grid <= 0) return cuda_fail(c, grid < 0 ? (cudaError_t)(-grid) : cudaErrorInvalidConfiguration, "persistent coder occupancy");
    cudaError_t e = timed(c, OCSC_K_PERSIST, [&] { return launch_persist(pa, grid, smem, c->stream); });
    if (e != cudaSuccess) return cuda_fail(c, e, "persistent coder launch");
  }
  for (int k : pcls) c->cls[k].pending += (int)groups[k].size();
  return OCSC_OK;
}

ocsc_status ocsc_code(ocsc_ctx *c, int n, const float *const *x, const int *H, const int *W,
                      float *const *u) {
  if (!c) return OCSC_EINVAL;
  NvtxRange range("ocsc_code");
  if (n <= 0 || !x || !H || !W) return fail(c, OCSC_EINVAL, "ocsc_code: bad arguments");
  std::vector<std::vector<int>> groups(c->cls.size());
  for (int i = 0; i < n; ++i) {
    if (!x[i] || H[i] <= 0 || W[i] <= 0) return fail(c, OCSC_EINVAL, "ocsc_code: image %d invalid", i);
    if (u && u[i] && reinterpret_cast<uintptr_t>(u[i]) % 16 != 0)
      return fail(c, OCSC_EINVAL, "ocsc_code: code buffer %d is not 16-byte aligned", i);
    const int k = class_of(c, H[i], W[i]);
    if (k < 0)
      return fail(c, OCSC_EUNSUPPORTED, "image %d (%dx%d, pad %d) maps to no FFT size of this context", i, H[i],
                  W[i], c->opts.pad);
    groups[k].push_back(i);
  }
  for (size_t k = 0; k < groups.size(); ++k)
    if (c->cls[k].pending + (int)groups[k].size() > c->opts.max_batch)
      return fail(c, OCSC_ESTATE, "ocsc_code: %d pending + %d new samples of size %d exceed max_batch %d; "
                  "call ocsc_update_dict", c->cls[k].pending, (int)groups[k].size(), c->cls[k].N, c->opts.max_batch);
  std::vector<int> pcls;  // classes coded by the persistent launch
  for (size_t k = 0; k < groups.size(); ++k) {
    if (groups[k].empty()) continue;
    if (c->opts.persistent && persist_size_ok(c->cls[k].N)) {
      pcls.push_back((int)k);
      continue;
    }
    ocsc_status st = code_class(c, c->cls[k], groups[k], x, H, W, u);
    if (st != OCSC_OK) return st;
  }
  if (!pcls.empty()) {
    ocsc_status st = code_persistent(c, pcls, groups, x, H, W, u);
    if (st != OCSC_OK) return st;
  }
  c->counters.samples_coded += n;
  return OCSC_OK;
}

ocsc_status ocsc_update_dict(ocsc_ctx *c) {
  if (!c) return OCSC_EINVAL;
  NvtxRange range("ocsc_update_dict");
  if (c->opts.band_hi != 0)
    return fail(c, OCSC_ESTATE, "a band context updates its dictionary through the ocsc_band_* calls");
  long long fresh = 0;
  for (const SizeClass &s : c->cls) fresh += s.pending;
  if (fresh == 0) return OCSC_OK;
  const long long n_total = c->n_seen + fresh;
  cudaError_t e = cudaSuccess;
  if (!c->opts.warm_start) {
    e = cudaMemsetAsync(c->V, 0, (size_t)c->K * c->M * c->M * sizeof(float), c->stream);
    for (SizeClass &s : c->cls) {
      const size_t kf = (size_t)c->K * s.F * sizeof(float2);
      if (e == cudaSuccess) e = cudaMemsetAsync(s.Vh, 0, kf, c->stream);
      if (e == cudaSuccess) e = cudaMemsetAsync(s.th, 0, kf, c->stream);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "cold start reset");
  }
  // Fold and factor every class that has samples (its weight w_c changed).
  std::vector<SizeClass *> active;
  for (SizeClass &s : c->cls) {
    const long long nc = s.n_seen + s.pending;
    if (nc == 0) continue;
    active.push_back(&s);
    FoldArgs fa{};
    fa.K = c->K;
    fa.F = s.F;
    fa.B = s.pending;
    fa.first = s.n_seen == 0;
    fa.alpha = (double)s.n_seen / (double)nc;
    fa.beta = 1.0 / (double)nc;
    fa.w = (double)nc / (double)n_total;
    fa.rho_eff = c->opts.rho_convention == 1 ? c->rho * s.P : c->rho;
    fa.A = s.A;
    fa.b = s.b;
    fa.Zp = s.Zp;
    fa.xh = s.xhp;
    fa.L = s.X;
    fa.g = s.y;
    fa.err = c->err;
    if (c->opts.history == 1) {
      SmArgs sa{};
      sa.K = c->K;
      sa.F = s.F;
      sa.B = s.pending;
      sa.n = (int)s.n_seen;
      sa.r = fa.rho_eff;
      {
        const double ri = 1.0 / fa.rho_eff;
        const float rh = (float)ri;
        sa.rinv = make_float2(rh, (float)(ri - (double)rh));
      }
      sa.alpha = (float)fa.alpha;
      sa.beta = (float)fa.beta;
      sa.Zp = s.Zp;
      sa.xh = s.xhp;
      sa.C = s.Csf;
      sa.b = s.b;
      if (s.pending > 0) {
        e = timed(c, OCSC_K_FOLD_FACTOR, [&] { return launch_sm_fold(sa, c->stream); });
        if (e != cudaSuccess) return cuda_fail(c, e, "history recursion");
      }
      continue;
    }
    if (big_k(c) && c->opts.precision == 0 && s.pending > 0) {
      e = timed(c, OCSC_K_FOLD_FACTOR, [&] { return launch_fold_big(fa, c->stream); });
      if (e != cudaSuccess) return cuda_fail(c, e, "history fold (K > 128)");
    }
    if (c->opts.precision == 3) {
      // Double-float fold inside the factorisation kernel.
      fa.dfold = 1;
      fa.Alo = s.Alo;
      fa.blo = s.blo;
    }
    if (c->opts.precision == 1 || c->opts.precision == 2) {
      // Tensor-core fold of the pending codes (compensated), then factor only.
      if (s.pending > 0) {
        GramArgs ga{};
        ga.K = c->K;
        ga.F = s.F;
        ga.B = s.pending;
        ga.first = s.n_seen == 0;
        ga.terms = c->opts.precision == 2 ? 3 : 1;
        if (s.gram_sc == 0) {
          s.gram_sc = gram_chunk(c->K, c->opts.max_batch, ga.terms);
          if (c->opts.autotune) {
            // Dry runs (sums without stores) of each chunk size that fits.
            float best = -1.f;
            for (int sc : {32, 64, 128}) {
              if (sc > gram_chunk(c->K, 128, ga.terms)) continue;
              GramArgs gd = ga;
              gd.SC = sc;
              gd.dry = 1;
              gd.Zp = s.Zp;
              gd.xh = s.xhp;
              gd.A = s.A;
              gd.Alo = s.Alo;
              gd.b = s.b;
              gd.err = c->err;
              gd.wait_polls = ocsc::kWaitPolls;
              gd.F = s.F;
              gd.K = c->K;
              gd.B = s.pending;
              const float t = time_runs(c, 2, [&] { return launch_gram_fold(gd, c->stream); });
              if (t < 0.f) return cuda_fail(c, cudaGetLastError(), "autotune history fold");
              if (best < 0.f || t < best) {
                best = t;
                s.gram_sc = sc;
              }
            }
          }
        }
        ga.SC = s.gram_sc;
        ga.alpha = (float)fa.alpha;
        ga.beta = (float)fa.beta;
        ga.keep = (float)((double)s.pending / (double)nc);
        ga.Zp = s.Zp;
        ga.xh = s.xhp;
        ga.A = s.A;
        ga.Alo = s.Alo;
        ga.b = s.b;
        ga.err = c->err;
        ga.wait_polls = c->wait_polls;
        e = timed(c, OCSC_K_HISTORY_TC, [&] { return launch_gram_fold(ga, c->stream); });
        if (e != cudaSuccess) return cuda_fail(c, e, "history fold (tensor cores)");
      }
      fa.prefolded = 1;
      fa.Alo = s.Alo;
    }
    if (big_k(c)) {
      e = timed(c, OCSC_K_FOLD_FACTOR, [&] { return launch_factor_big(fa, c->work, c->work_ctas, c->stream); });
    } else {
      const int nt = s.fold_threads ? s.fold_threads : 256;
      e = timed(c, OCSC_K_FOLD_FACTOR, [&] { return launch_fold_factor(fa, nt, c->stream); });
      if (e == cudaSuccess && s.fold_threads == 0) {
        // Autotune the CTA size on this class's own history: factor-only
        // reruns recompute the same X and y from the folded A and b.
        s.fold_threads = 256;
        if (c->opts.autotune) {
          FoldArgs fp = fa;
          fp.prefolded = 1;
          fp.Alo = s.Alo;
          fp.blo = s.blo;
          const float t256 = time_runs(c, 2, [&] { return launch_fold_factor(fp, 256, c->stream); });
          const float t512 = time_runs(c, 2, [&] { return launch_fold_factor(fp, 512, c->stream); });
          if (t256 < 0.f || t512 < 0.f) return cuda_fail(c, cudaGetLastError(), "autotune fold_factor");
          s.fold_threads = t512 < t256 ? 512 : 256;
        }
      }
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "fold_factor");
  }
  AlphaClasses ac{};
  ac.project = 1;
  ac.C = (int)active.size();
  for (int i = 0; i < ac.C; ++i) {
    ac.N[i] = active[i]->N;
    ac.Y[i] = active[i]->Y;
    ac.tw[i] = active[i]->tw;
  }
  for (int t = 0; t < c->opts.Jd; ++t) {
    for (SizeClass *s : active) {
      const float rho_eff = (float)(c->opts.rho_convention == 1 ? c->rho * s->P : c->rho);
      e = timed(c, OCSC_K_DSTEP, [&] {
        if (c->opts.history == 1) {
          // Reading R23: penalty r / n after n folded samples; the scaled dual
          // keeps rho Theta, so it grows by n / n_before at the first step.
          const double nc = (double)(s->n_seen + s->pending);
          const double ths = (t == 0 && s->n_seen > 0) ? nc / (double)s->n_seen : 1.0;
          return launch_dstep_sm(c->K, s->F, (c->opts.rho_convention == 1 ? c->rho * s->P : c->rho) / nc, ths,
                                 s->Csf, s->b, s->Vh, s->th, s->Dcur, s->E, c->stream);
        }
        return big_k(c) ? launch_dstep_big(c->K, s->F, rho_eff, s->X, s->y, s->Vh, s->th, s->Dcur, s->E, c->stream)
                        : launch_dstep(c->K, s->F, rho_eff, s->X, s->y, s->Vh, s->th, s->Dcur, s->E, c->stream);
      });
      if (e != cudaSuccess) return cuda_fail(c, e, "dstep");
      e = timed(c, OCSC_K_VSTEP_COLS, [&] { return launch_vstep_cols(c->K, s->N, c->M, s->E, s->tw, s->Y, c->stream); });
      if (e != cudaSuccess) return cuda_fail(c, e, "vstep_cols");
    }
    e = timed(c, OCSC_K_VSTEP_PROJECT, [&] { return launch_vstep_project(c->K, c->M, ac, c->V, c->stream); });
    if (e != cudaSuccess) return cuda_fail(c, e, "vstep_project");
    for (SizeClass *s : active) {
      e = timed(c, OCSC_K_VSTEP_SPECTRUM, [&] { return launch_vstep_partial_dft(c->K, s->N, c->M, c->V, s->tw, s->Tm, c->stream); });
      if (e == cudaSuccess)
        e = timed(c, OCSC_K_VSTEP_SPECTRUM, [&] { return launch_vstep_spectrum(0, c->K, s->N, c->M, s->Tm, s->tw, s->Vh, s->th, s->Dcur, c->stream); });
      if (e != cudaSuccess) return cuda_fail(c, e, "vstep_spectrum");
    }
  }
  for (SizeClass &s : c->cls) {
    const bool is_active = std::find(active.begin(), active.end(), &s) != active.end();
    if (!is_active && (e = class_spectrum(c, s)) != cudaSuccess) return cuda_fail(c, e, "class spectrum");
    e = timed(c, OCSC_K_DICT_NORMS, [&] { return launch_dict_norms(c->K, s.F, coding_spectrum(c, s), s.dn, c->stream); });
    if (e != cudaSuccess) return cuda_fail(c, e, "dict_norms");
    s.n_seen += s.pending;
    s.pending = 0;
  }
  c->n_seen = n_total;
  c->version += 1;
  c->counters.dict_updates += 1;
  return OCSC_OK;
}

ocsc_status ocsc_get_dict(ocsc_ctx *c, float *D_host, uint64_t *version) {
  if (!c || !D_host) return c ? fail(c, OCSC_EINVAL, "null output") : OCSC_EINVAL;
  ocsc_status st = check_device(c);
  if (st != OCSC_OK) return st;
  const size_t bytes = (size_t)c->K * c->M * c->M * sizeof(float);
  const float *src = c->V;
  if (!c->opts.return_feasible) {
    // Algorithm 3 publishes H(F^-1(D~_t)) with D~_t = D~_{t,J} as Algorithm 2
    // returns it (one size class): the support crop of its inverse DFT.
    SizeClass &s = c->cls[0];
    AlphaClasses ac{};
    ac.project = 0;
    ac.C = 1;
    ac.N[0] = s.N;
    ac.Y[0] = s.Y;
    ac.tw[0] = s.tw;
    cudaError_t e = timed(c, OCSC_K_VSTEP_COLS, [&] { return launch_vstep_cols(c->K, s.N, c->M, s.Dcur, s.tw, s.Y, c->stream); });
    if (e == cudaSuccess)
      e = timed(c, OCSC_K_VSTEP_PROJECT, [&] { return launch_vstep_project(c->K, c->M, ac, c->Dpub, c->stream); });
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "publish D~_{t,J}");
    src = c->Dpub;
  }
  cudaError_t e = cudaMemcpy(D_host, src, bytes, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "copy filters");
  if (version) *version = c->version;
  return OCSC_OK;
}

ocsc_status ocsc_set_dict(ocsc_ctx *c, const float *D_host, int normalize) {
  if (!c || !D_host) return c ? fail(c, OCSC_EINVAL, "null input") : OCSC_EINVAL;
  return upload_dict(c, D_host, normalize);
}

// ---------------------------------------------------------------------------
// Checkpoint: the learner state between updates (no pending samples).
// ---------------------------------------------------------------------------
namespace {

constexpr uint32_t kStateMagic = 0x4353434Fu;  // "OCSC"
constexpr uint32_t kStateFormat = 2;

struct StateHeader {
  uint32_t magic, format;
  int32_t K, M, ncls, N[OCSC_MAX_FFT_SIZES];
  int32_t rho_convention, return_feasible, warm_start, precision, history;
  double lam, rho;
  int64_t n_seen;
  uint64_t version;
  int64_t class_seen[OCSC_MAX_FFT_SIZES];
};

// Device regions of the state, in file order.
std::vector<std::pair<void *, size_t>> state_regions(ocsc_ctx *c) {
  std::vector<std::pair<void *, size_t>> r;
  const size_t K = (size_t)c->K;
  r.emplace_back(c->V, K * c->M * c->M * sizeof(float));
  for (SizeClass &s : c->cls) {
    const size_t kf = K * s.F * sizeof(float2);
    r.emplace_back(s.Vh, kf);
    r.emplace_back(s.th, kf);
    r.emplace_back(s.Dcur, kf);
    r.emplace_back(s.b, kf);
    r.emplace_back(s.A, (size_t)s.Fb * tri_stride(c->K) * sizeof(float2));
    if (s.Alo) r.emplace_back(s.Alo, (size_t)s.Fb * tri_stride(c->K) * sizeof(float2));
    if (s.blo) r.emplace_back(s.blo, kf);
    if (s.Csf) r.emplace_back(s.Csf, (size_t)s.F * tri_stride(c->K) * sizeof(float4));
    r.emplace_back(s.dn, (size_t)s.F * sizeof(float));
  }
  return r;
}

size_t state_bytes(ocsc_ctx *c) {
  size_t n = sizeof(StateHeader);
  for (auto &p : state_regions(c)) n += p.second;
  return n;
}

StateHeader make_header(const ocsc_ctx *c) {
  StateHeader h{};
  h.magic = kStateMagic;
  h.format = kStateFormat;
  h.K = c->K;
  h.M = c->M;
  h.ncls = (int32_t)c->cls.size();
  for (size_t i = 0; i < c->cls.size(); ++i) {
    h.N[i] = c->cls[i].N;
    h.class_seen[i] = c->cls[i].n_seen;
  }
  h.rho_convention = c->opts.rho_convention;
  h.return_feasible = c->opts.return_feasible;
  h.warm_start = c->opts.warm_start;
  h.precision = c->opts.precision;
  h.history = c->opts.history;
  h.lam = c->lam;
  h.rho = c->rho;
  h.n_seen = c->n_seen;
  h.version = c->version;
  return h;
}

}  // namespace

ocsc_status ocsc_get_state(ocsc_ctx *c, void *buf, size_t *len) {
  if (!c) return OCSC_EINVAL;
  if (!len) return fail(c, OCSC_EINVAL, "get_state: null length");
  const size_t need = state_bytes(c);
  if (!buf) {
    *len = need;
    return OCSC_OK;
  }
  if (*len < need) return fail(c, OCSC_EINVAL, "get_state: buffer of %zu bytes, need %zu", *len, need);
  for (const SizeClass &s : c->cls)
    if (s.pending) return fail(c, OCSC_ESTATE, "get_state: %d samples of size %d are pending", s.pending, s.N);
  ocsc_status st = check_device(c);
  if (st != OCSC_OK) return st;
  const StateHeader h = make_header(c);
  char *o = static_cast<char *>(buf);
  std::memcpy(o, &h, sizeof h);
  o += sizeof h;
  for (auto &p : state_regions(c)) {
    cudaError_t e = cudaMemcpy(o, p.first, p.second, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "get_state copy");
    o += p.second;
  }
  *len = need;
  return OCSC_OK;
}

ocsc_status ocsc_set_state(ocsc_ctx *c, const void *buf, size_t len) {
  if (!c) return OCSC_EINVAL;
  if (!buf) return fail(c, OCSC_EINVAL, "set_state: null buffer");
  const size_t need = state_bytes(c);
  if (len != need) return fail(c, OCSC_EINVAL, "set_state: %zu bytes, this context's state has %zu", len, need);
  StateHeader h;
  std::memcpy(&h, buf, sizeof h);
  const StateHeader mine = make_header(c);
  bool same = h.magic == kStateMagic && h.format == kStateFormat && h.K == mine.K && h.M == mine.M &&
              h.ncls == mine.ncls && h.rho_convention == mine.rho_convention &&
              h.return_feasible == mine.return_feasible && h.warm_start == mine.warm_start &&
              h.precision == mine.precision && h.history == mine.history &&
              h.lam == mine.lam && h.rho == mine.rho;
  for (int i = 0; same && i < h.ncls; ++i) same = h.N[i] == mine.N[i];
  if (!same) return fail(c, OCSC_EINVAL, "set_state: the state was saved by a context of another shape or parameters");
  ocsc_status st = check_device(c);
  if (st != OCSC_OK) return st;
  const char *o = static_cast<const char *>(buf) + sizeof h;
  for (auto &p : state_regions(c)) {
    cudaError_t e = cudaMemcpy(p.first, o, p.second, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e, "set_state copy");
    o += p.second;
  }
  for (size_t i = 0; i < c->cls.size(); ++i) {
    c->cls[i].n_seen = h.class_seen[i];
    c->cls[i].pending = 0;
  }
  c->n_seen = h.n_seen;
  c->version = h.version;
  return OCSC_OK;
}

ocsc_status ocsc_get_tuning(const ocsc_ctx *c, int N, ocsc_tuning *out) {
  if (!c || !out) return OCSC_EINVAL;
  for (const SizeClass &s : c->cls)
    if (s.N == N) {
      out->fold_threads = s.fold_threads;
      out->spat_cb = s.spat_cb;
      out->plane_ctas = s.plane_ctas;
      out->plane_ahead = s.plane_ahead;
      out->plane_threads = s.plane_threads;
      out->gram_sc = s.gram_sc;
      return OCSC_OK;
    }
  return OCSC_EUNSUPPORTED;
}

ocsc_status ocsc_set_tuning(ocsc_ctx *c, int N, const ocsc_tuning *in) {
  if (!c || !in) return OCSC_EINVAL;
  for (SizeClass &s : c->cls)
    if (s.N == N) {
      const bool plane = in->plane_ctas != 0;
      if (plane && (large_fft(N) || !plane_shape_ok(N, in->plane_threads, in->plane_ctas) ||
                    (in->plane_ahead != 0 && in->plane_ahead != 1)))
        return fail(c, OCSC_EINVAL, "ocsc_set_tuning: unsupported plane kernel shape");
      if (in->fold_threads != 0 && in->fold_threads != 256 && in->fold_threads != 512)
        return fail(c, OCSC_EINVAL, "ocsc_set_tuning: fold_threads must be 256 or 512");
      if (in->spat_cb != 0 && (!large_fft(N) || !large_cb_ok(N, in->spat_cb)))
        return fail(c, OCSC_EINVAL, "ocsc_set_tuning: unsupported spat_cb");
      if (in->gram_sc != 0)
        return fail(c, OCSC_EINVAL, "ocsc_set_tuning: gram_sc is chosen by the library (pass 0)");
      if (plane) {
        s.plane_ctas = in->plane_ctas;
        s.plane_threads = in->plane_threads;
        s.plane_ahead = in->plane_ahead;
      }
      if (in->fold_threads) s.fold_threads = in->fold_threads;
      if (in->spat_cb) s.spat_cb = in->spat_cb;
      return OCSC_OK;
    }
  return fail(c, OCSC_EUNSUPPORTED, "ocsc_set_tuning: no size class of that FFT side");
}

ocsc_status ocsc_sync(ocsc_ctx *c) {
  if (!c) return OCSC_EINVAL;
  return check_device(c);
}

// Real 2D FFT building blocks on one class size; for N >= 256 they run in
// chunks of pairs that fit the class's tile buffer.
static ocsc_status fft2_any(ocsc_ctx *c, int N, int inverse, const float *in, float *out, int planes,
                            const char *name) {
  SizeClass *s = nullptr;
  for (SizeClass &k : c->cls)
    if (k.N == N) s = &k;
  if (!s) return fail(c, OCSC_EUNSUPPORTED, "%s: N=%d is not a size of this context", name, N);
  ocsc_status wst = ensure_code_ws(c, *s);
  if (wst != OCSC_OK) return wst;
  if (!large_fft(N)) {
    cudaError_t e = timed(c, OCSC_K_COUNT, [&] { return launch_fft2(N, inverse, in, out, planes, s->tw, c->stream); });
    return e == cudaSuccess ? OCSC_OK : cuda_fail(c, e, name);
  }
  const int cap_pairs = c->opts.max_batch * ((c->K + 1) / 2);
  const size_t spec = (size_t)s->F * 2, real = (size_t)s->P;  // floats per plane
  for (int p0 = 0; p0 < planes; p0 += 2 * cap_pairs) {
    const int np = planes - p0 < 2 * cap_pairs ? planes - p0 : 2 * cap_pairs;
    LargeIO io{};
    io.T = s->tiles;
    io.planes = np;
    CodeIter none{};
    ImgBatch b{};
    cudaError_t e;
    if (!inverse) {
      io.real_in = in + (size_t)p0 * real;
      io.spec_out = reinterpret_cast<float2 *>(out + (size_t)p0 * spec);
      e = timed(c, OCSC_K_COUNT, [&] { return launch_large(N, LARGE_SPAT_R2C, none, b, io, 1, (np + 1) / 2, s->tw, c->stream); });
      if (e == cudaSuccess)
        e = timed(c, OCSC_K_COUNT, [&] { return launch_large(N, LARGE_SPEC_R2C, none, b, io, 1, (np + 1) / 2, s->tw, c->stream); });
    } else {
      io.spec_in = reinterpret_cast<const float2 *>(in + (size_t)p0 * spec);
      io.real_out = out + (size_t)p0 * real;
      e = timed(c, OCSC_K_COUNT, [&] { return launch_large(N, LARGE_SPEC_C2R, none, b, io, 1, (np + 1) / 2, s->tw, c->stream); });
      if (e == cudaSuccess)
        e = timed(c, OCSC_K_COUNT, [&] { return launch_large(N, LARGE_SPAT_C2R, none, b, io, 1, (np + 1) / 2, s->tw, c->stream); });
    }
    if (e != cudaSuccess) return cuda_fail(c, e, name);
  }
  return OCSC_OK;
}

ocsc_status ocsc_fft2_r2c(ocsc_ctx *c, int N, const float *x, float *X, int planes) {
  if (!c) return OCSC_EINVAL;
  if (!x || !X || planes < 0) return fail(c, OCSC_EINVAL, "fft2_r2c: bad arguments");
  return fft2_any(c, N, 0, x, X, planes, "fft2_r2c");
}

ocsc_status ocsc_fft2_c2r(ocsc_ctx *c, int N, const float *X, float *x, int planes) {
  if (!c) return OCSC_EINVAL;
  if (!x || !X || planes < 0) return fail(c, OCSC_EINVAL, "fft2_c2r: bad arguments");
  return fft2_any(c, N, 1, X, x, planes, "fft2_c2r");
}

ocsc_status ocsc_drop_pending(ocsc_ctx *c) {
  if (!c) return OCSC_EINVAL;
  for (SizeClass &s : c->cls) s.pending = 0;
  return OCSC_OK;
}

static ocsc_status objective_terms(ocsc_ctx *c, int n, const float *const *x, const int *H, const int *W,
                                   const float *const *u, double *f_host, double *r2_host, double *l1_host,
                                   double *psnr_host = nullptr, double peak = 0.0) {
  if (!c) return OCSC_EINVAL;
  if (n < 0 || (n > 0 && (!x || !H || !W || !u || !(f_host || r2_host || l1_host || psnr_host))))
    return fail(c, OCSC_EINVAL, "ocsc_objective: bad arguments");
  std::vector<int> cl(n);
  for (int i = 0; i < n; ++i) {
    if (!x[i] || !u[i] || H[i] <= 0 || W[i] <= 0) return fail(c, OCSC_EINVAL, "ocsc_objective: sample %d invalid", i);
    cl[i] = class_of(c, H[i], W[i]);
    if (cl[i] < 0) return fail(c, OCSC_EUNSUPPORTED, "sample %d maps to no FFT size of this context", i);
  }
  for (int s0 = 0; s0 < n; s0 += kObjChunk) {
    const int m = n - s0 < kObjChunk ? n - s0 : kObjChunk;
    for (int i = 0; i < m; ++i) {
      SizeClass &s = c->cls[cl[s0 + i]];
      ocsc_status wst = ensure_code_ws(c, s);
      if (wst != OCSC_OK) return wst;
      float2 *Uh = s.What;  // coding workspace of slot 0, idle between ocsc_code calls
      ImgBatch bt{};
      bt.n = 1;
      bt.x[0] = x[s0 + i];
      bt.u[0] = nullptr;
      bt.H[0] = H[s0 + i];
      bt.W[0] = W[s0 + i];
      cudaError_t e = cudaSuccess;
      if (large_fft(s.N)) {
        CodeIter none{};
        LargeIO io{};
        io.T = s.tiles;
        io.spec_out = s.obj_xh;
        io.tile_pairs = 1;
        e = timed(c, OCSC_K_COUNT, [&] { return launch_large(s.N, LARGE_SPAT_IMAGE, none, bt, io, 1, 1, s.tw, c->stream); });
        if (e == cudaSuccess)
          e = timed(c, OCSC_K_COUNT, [&] { return launch_large(s.N, LARGE_SPEC_IMAGE, none, bt, io, 1, 1, s.tw, c->stream); });
        LargeIO jo{};
        jo.T = s.tiles;
        jo.real_in = u[s0 + i];
        jo.spec_out = Uh;
        jo.planes = c->K;
        const int np = (c->K + 1) / 2;
        if (e == cudaSuccess)
          e = timed(c, OCSC_K_COUNT, [&] { return launch_large(s.N, LARGE_SPAT_R2C, none, bt, jo, 1, np, s.tw, c->stream); });
        if (e == cudaSuccess)
          e = timed(c, OCSC_K_COUNT, [&] { return launch_large(s.N, LARGE_SPEC_R2C, none, bt, jo, 1, np, s.tw, c->stream); });
      } else {
        e = timed(c, OCSC_K_COUNT, [&] { return launch_image_spectrum(s.N, bt, s.tw, s.obj_xh, c->stream); });
        if (e == cudaSuccess)
          e = timed(c, OCSC_K_COUNT, [&] { return launch_fft2(s.N, 0, u[s0 + i], reinterpret_cast<float *>(Uh), c->K, s.tw, c->stream); });
      }
      if (e == cudaSuccess) {
        c->counters.kernel_launches += 2;  // three kernels in launch_objective
        e = timed(c, OCSC_K_COUNT, [&] {
          return launch_objective(c->K, s.N, c->lam, coding_spectrum(c, s), s.obj_xh, Uh, u[s0 + i], c->obj_part,
                                  c->obj_out + 3 * i, c->stream);
        });
      }
      if (e != cudaSuccess) return cuda_fail(c, e, "objective");
    }
    std::vector<double> h((size_t)4 * kObjChunk);
    cudaError_t e = cudaSuccess;
    if (psnr_host) {
      PsnrArgs pa{};
      pa.n = m;
      pa.peak = peak;
      for (int i = 0; i < m; ++i) pa.P[i] = c->cls[cl[s0 + i]].P;
      c->counters.kernel_launches += 1;
      e = launch_psnr(c->obj_out, pa, c->obj_out + 3 * kObjChunk, c->stream);
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h.data(), c->obj_out, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "objective readback");
    for (int i = 0; i < m; ++i) {
      if (f_host) f_host[s0 + i] = h[3 * i];
      if (r2_host) r2_host[s0 + i] = h[3 * i + 1];
      if (l1_host) l1_host[s0 + i] = h[3 * i + 2];
      if (psnr_host) psnr_host[s0 + i] = h[3 * kObjChunk + i];
    }
  }
  return OCSC_OK;
}

ocsc_status ocsc_objective(ocsc_ctx *c, int n, const float *const *x, const int *H, const int *W,
                           const float *const *u, double *out_host) {
  if (!c) return OCSC_EINVAL;
  if (n > 0 && !out_host) return fail(c, OCSC_EINVAL, "ocsc_objective: bad arguments");
  return objective_terms(c, n, x, H, W, u, out_host, nullptr, nullptr);
}

ocsc_status ocsc_objective_terms(ocsc_ctx *c, int n, const float *const *x, const int *H, const int *W,
                                 const float *const *u, double *resid2_host, double *l1_host) {
  if (!c) return OCSC_EINVAL;
  if (n > 0 && (!resid2_host || !l1_host)) return fail(c, OCSC_EINVAL, "ocsc_objective_terms: bad arguments");
  return objective_terms(c, n, x, H, W, u, nullptr, resid2_host, l1_host);
}

ocsc_status ocsc_psnr(ocsc_ctx *c, int n, const float *const *x, const int *H, const int *W,
                      const float *const *u, double peak, double *psnr_host) {
  if (!c) return OCSC_EINVAL;
  if (n > 0 && (!psnr_host || !(peak > 0))) return fail(c, OCSC_EINVAL, "ocsc_psnr: bad arguments");
  return objective_terms(c, n, x, H, W, u, nullptr, nullptr, nullptr, psnr_host, peak);
}

ocsc_status ocsc_filter_order(ocsc_ctx *c, int *order_host) {
  if (!c) return OCSC_EINVAL;
  if (!order_host) return fail(c, OCSC_EINVAL, "ocsc_filter_order: null output");
  c->counters.kernel_launches += 1;
  cudaError_t e = launch_filter_order(c->K, c->M, c->V, c->order, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(order_host, c->order, (size_t)c->K * sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return e == cudaSuccess ? OCSC_OK : cuda_fail(c, e, "filter_order");
}

ocsc_status ocsc_copy_dict(ocsc_ctx *c, float *D_dev) {
  if (!c) return OCSC_EINVAL;
  if (!D_dev) return fail(c, OCSC_EINVAL, "ocsc_copy_dict: null output");
  const size_t bytes = (size_t)c->K * c->M * c->M * sizeof(float);
  cudaError_t e = cudaMemcpyAsync(D_dev, c->V, bytes, cudaMemcpyDeviceToDevice, c->stream);
  return e == cudaSuccess ? OCSC_OK : cuda_fail(c, e, "copy_dict");
}

ocsc_status ocsc_set_wait_limit(ocsc_ctx *c, uint64_t polls) {
  if (!c) return OCSC_EINVAL;
  c->wait_polls = polls > 0xffffffffull ? 0xffffffffu : (unsigned)polls;
  return OCSC_OK;
}

ocsc_status ocsc_rel_diff(ocsc_ctx *c, const float *a, const float *b, size_t count, double *out_host) {
  if (!c) return OCSC_EINVAL;
  if (!a || !b || !out_host) return fail(c, OCSC_EINVAL, "ocsc_rel_diff: bad arguments");
  if (count == 0) {
    *out_host = 0.0;
    return OCSC_OK;
  }
  c->counters.kernel_launches += 2;
  cudaError_t e = launch_rel_diff(a, b, count, c->obj_part, c->obj_out, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out_host, c->obj_out, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return e == cudaSuccess ? OCSC_OK : cuda_fail(c, e, "rel_diff");
}

// ---------------------------------------------------------------------------
// Frequency-band sharding of the dictionary step (Prop. 1 decouples the
// D-row systems per frequency): a band context folds, factors and solves the
// frequencies of its k1 rows only; the caller moves the codes' band rows to
// their owners and sums the support crops over the bands.
// ---------------------------------------------------------------------------

static ocsc_status band_ctx(ocsc_ctx *c, const char *what) {
  if (c->opts.band_hi == 0) return fail(c, OCSC_ESTATE, "%s: not a band context (opts.band_hi = 0)", what);
  return OCSC_OK;
}

ocsc_status ocsc_band_export(ocsc_ctx *c, int k1_lo, int k1_hi, float *Z_dev, float *x_dev) {
  if (!c) return OCSC_EINVAL;
  SizeClass &s = c->cls[0];
  if (c->cls.size() != 1 || k1_lo < 0 || k1_hi > s.N || k1_lo >= k1_hi || !Z_dev || !x_dev)
    return fail(c, OCSC_EINVAL, "band_export: bad arguments");
  const size_t row = (size_t)s.NH * sizeof(float2), w = (size_t)(k1_hi - k1_lo) * row, F8 = (size_t)s.F * sizeof(float2);
  if (s.pending == 0) return OCSC_OK;
  cudaError_t e = cudaMemcpy2DAsync(Z_dev, w, s.Zp + (size_t)k1_lo * s.NH, F8, w, (size_t)s.pending * c->K,
                                    cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(x_dev, w, s.xhp + (size_t)k1_lo * s.NH, F8, w, (size_t)s.pending, cudaMemcpyDeviceToDevice,
                          c->stream);
  return e == cudaSuccess ? OCSC_OK : cuda_fail(c, e, "band_export");
}

ocsc_status ocsc_band_fold(ocsc_ctx *c, int B, const float *Z_dev, const float *x_dev) {
  if (!c) return OCSC_EINVAL;
  ocsc_status st = band_ctx(c, "band_fold");
  if (st != OCSC_OK) return st;
  if (B < 1 || !Z_dev || !x_dev) return fail(c, OCSC_EINVAL, "band_fold: bad arguments");
  SizeClass &s = c->cls[0];
  cudaError_t e = cudaSuccess;
  if (!c->opts.warm_start) {
    e = cudaMemsetAsync(c->V, 0, (size_t)c->K * c->M * c->M * sizeof(float), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.Vh, 0, (size_t)c->K * s.F * sizeof(float2), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.th, 0, (size_t)c->K * s.F * sizeof(float2), c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "band cold start");
  }
  const long long nc = s.n_seen + B;
  FoldArgs fa{};
  fa.K = c->K;
  fa.F = s.F;
  fa.B = B;
  fa.first = s.n_seen == 0;
  fa.alpha = (double)s.n_seen / (double)nc;
  fa.beta = 1.0 / (double)nc;
  fa.w = 1.0;
  fa.rho_eff = c->opts.rho_convention == 1 ? c->rho * s.P : c->rho;
  fa.A = s.A;
  fa.b = s.b;
  fa.Zp = reinterpret_cast<const float2 *>(Z_dev);
  fa.xh = reinterpret_cast<const float2 *>(x_dev);
  fa.L = s.X;
  fa.g = s.y;
  fa.err = c->err;
  fa.p0 = s.p0;
  fa.nF = s.Fb;
  fa.zF = s.Fb;
  fa.zp0 = s.p0;
  if (c->opts.precision == 3) {
    fa.dfold = 1;
    fa.Alo = s.Alo;
    fa.blo = s.blo;
  }
  const int nt = s.fold_threads ? s.fold_threads : 256;
  e = timed(c, OCSC_K_FOLD_FACTOR, [&] { return launch_fold_factor(fa, nt, c->stream); });
  if (e != cudaSuccess) return cuda_fail(c, e, "band fold_factor");
  s.n_seen = nc;
  c->n_seen += B;
  return OCSC_OK;
}

ocsc_status ocsc_band_dict_step(ocsc_ctx *c, float *alpha_dev) {
  if (!c) return OCSC_EINVAL;
  ocsc_status st = band_ctx(c, "band_dict_step");
  if (st != OCSC_OK) return st;
  if (!alpha_dev) return fail(c, OCSC_EINVAL, "band_dict_step: null output");
  if (c->cls[0].n_seen == 0) return fail(c, OCSC_ESTATE, "band_dict_step: nothing folded yet");
  SizeClass &s = c->cls[0];
  const float rho_eff = (float)(c->opts.rho_convention == 1 ? c->rho * s.P : c->rho);
  cudaError_t e = timed(c, OCSC_K_DSTEP, [&] {
    return launch_dstep(c->K, s.F, rho_eff, s.X, s.y, s.Vh, s.th, s.Dcur, s.E, c->stream, s.p0, s.Fb);
  });
  if (e == cudaSuccess)
    e = timed(c, OCSC_K_VSTEP_COLS, [&] {
      return launch_vstep_cols(c->K, s.N, c->M, s.E, s.tw, s.Y, c->stream, c->opts.band_lo, c->opts.band_hi);
    });
  AlphaClasses ac{};
  ac.project = 0;
  ac.C = 1;
  ac.N[0] = s.N;
  ac.Y[0] = s.Y;
  ac.tw[0] = s.tw;
  if (e == cudaSuccess)
    e = timed(c, OCSC_K_VSTEP_PROJECT, [&] { return launch_vstep_project(c->K, c->M, ac, alpha_dev, c->stream); });
  return e == cudaSuccess ? OCSC_OK : cuda_fail(c, e, "band_dict_step");
}

ocsc_status ocsc_band_project(ocsc_ctx *c, const float *alpha_dev, int last) {
  if (!c) return OCSC_EINVAL;
  ocsc_status st = band_ctx(c, "band_project");
  if (st != OCSC_OK) return st;
  if (!alpha_dev) return fail(c, OCSC_EINVAL, "band_project: null input");
  SizeClass &s = c->cls[0];
  cudaError_t e = timed(c, OCSC_K_VSTEP_PROJECT, [&] { return launch_project_alpha(c->K, c->M, alpha_dev, c->V, c->stream); });
  if (e == cudaSuccess)
    e = timed(c, OCSC_K_VSTEP_SPECTRUM, [&] { return launch_vstep_partial_dft(c->K, s.N, c->M, c->V, s.tw, s.Tm, c->stream); });
  if (e == cudaSuccess)
    e = timed(c, OCSC_K_VSTEP_SPECTRUM, [&] {
      return launch_vstep_spectrum(0, c->K, s.N, c->M, s.Tm, s.tw, s.Vh, s.th, s.Dcur, c->stream, s.p0, s.p0 + s.Fb);
    });
  if (e == cudaSuccess && last) {
    e = timed(c, OCSC_K_DICT_NORMS, [&] { return launch_dict_norms(c->K, s.F, s.Vh, s.dn, c->stream); });
    if (e == cudaSuccess) {
      c->version += 1;
      c->counters.dict_updates += 1;
    }
  }
  return e == cudaSuccess ? OCSC_OK : cuda_fail(c, e, "band_project");
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
