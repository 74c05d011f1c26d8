// Serving engine: continuous batching of coding requests over one context.
//
// A request is one image coded by the ADMM of Sec. II-C.1 until its relative
// primal and dual residuals fall below tol (checked every check_every
// iterations, capped at max_iters).  Each size class owns a fixed set of
// workspace slots.  A scheduling round (ocsc_server_step):
//   1. admits queued requests in arrival order while a slot of their class is
//      free and their working set fits the memory budget;
//   2. runs check_every ADMM iterations for every admitted request, whatever
//      its iteration count (the kernels take a slot and an iteration index per
//      image), grouped by class and dictionary version;
//   3. reduces each request's residual sums in a fixed order, completes the
//      requests that converged or hit the cap, and frees their slots;
//   4. with learning on, folds completed requests into the history and runs
//      DictOCSC after every update_every completions (Algorithm 3).
// Request work runs on a stream of the server; the dictionary update runs on
// the context's stream, ordered after the staging of the completed requests
// only, so it overlaps the coding of the requests in flight.  A request is
// coded against the dictionary current when it was admitted: the engine keeps
// two coding spectra per class, starts an update only when no request still
// uses the older one, and makes the new one current once its copies are done.  Every per-request computation reads only
// that request's slot and its dictionary version, so a result does not depend
// on the other requests in flight.
#include <algorithm>
#include <cmath>
#include <deque>
#include <vector>

#include "ctx.h"

using namespace ocsc;

namespace {

struct Request {
  uint64_t id = 0;
  const float *x = nullptr;
  float *u = nullptr;
  int H = 0, W = 0, cls = 0;
};

struct Slot {
  bool used = false;
  Request req;
  int iter = 0;
  int ver = 0;
};

struct ServeClass {
  int nslots = 0;
  size_t ws = 0;  // bytes of one request's working set
  std::vector<Slot> slots;
  float2 *What = nullptr, *r = nullptr, *xh = nullptr, *Zp = nullptr, *tiles = nullptr, *part = nullptr;
  int *cnt = nullptr;
  float *Gam = nullptr;
  float *resid = nullptr;     // [nslots][groups][kResidTerms]
  int groups = 0;
  int *d_slots = nullptr;     // [nslots]
  double *d_res = nullptr;    // [nslots][kResidTerms]
  float2 *D[2] = {nullptr, nullptr};  // coding spectra of two dictionary versions
  float *dn[2] = {nullptr, nullptr};
};

}  // namespace

struct ocsc_server {
  ocsc_ctx *ctx = nullptr;
  ocsc_server_opts o{};
  std::vector<ServeClass> sc;
  std::deque<Request> queue;
  std::vector<ocsc_served> done;
  size_t mem_used = 0;
  int cur = 0;                // dictionary version slot new requests use
  int refs[2] = {0, 0};       // requests in flight per version slot
  uint64_t ver_id[2] = {0, 0};
  int since_update = 0;
  double *h_res = nullptr;    // pinned [max slots][kResidTerms]
  int *h_slots = nullptr;     // pinned [max slots]
  std::vector<void *> allocs;
  // Streams: request work runs on `stream`; dictionary updates on the
  // context's stream (ctx_stream), so an update overlaps the coding of the
  // requests in flight.  Completed requests are staged into one of two pending
  // sets per class (set 0 = the context's own buffers) while an update reads
  // the other; ev_read[set] marks the end of the last update that read it.
  cudaStream_t stream = nullptr, ctx_stream = nullptr;
  cudaEvent_t ev_stage = nullptr, ev_pub = nullptr, ev_read[2] = {nullptr, nullptr};
  int pend_set = 0;
  std::vector<float2 *> pend_Zp[2], pend_xh[2];
  bool pub_pending = false;   // a published version is waiting for its event
  int pub_slot = 0;
};

namespace {

template <typename T>
ocsc_status salloc(ocsc_server *s, T **p, size_t count) {
  *p = nullptr;
  cudaError_t e = cudaMalloc((void **)p, (count ? count : 1) * sizeof(T));
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return fail(s->ctx, OCSC_ENOMEM, "server: cudaMalloc of %zu bytes failed", count * sizeof(T));
  }
  s->allocs.push_back(*p);
  return OCSC_OK;
}

// Publish the context's current coding spectra into version slot v.
cudaError_t publish(ocsc_server *s, int v) {
  ocsc_ctx *c = s->ctx;
  for (size_t k = 0; k < c->cls.size(); ++k) {
    const SizeClass &cl = c->cls[k];
    cudaError_t e = cudaMemcpyAsync(s->sc[k].D[v], coding_spectrum(c, cl), (size_t)c->K * cl.F * sizeof(float2),
                                    cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(s->sc[k].dn[v], cl.dn, (size_t)cl.F * sizeof(float), cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) return e;
  }
  s->ver_id[v] = c->version;
  return cudaSuccess;
}

// Launch the sample spectra of newly admitted requests of one class.
cudaError_t launch_spectra(ocsc_server *s, int k, const std::vector<int> &slots) {
  ocsc_ctx *c = s->ctx;
  const SizeClass &cl = c->cls[k];
  ServeClass &q = s->sc[k];
  for (size_t s0 = 0; s0 < slots.size(); s0 += kMaxCallImages) {
    ImgBatch b{};
    b.n = (int)std::min<size_t>(kMaxCallImages, slots.size() - s0);
    for (int i = 0; i < b.n; ++i) {
      const Slot &sl = q.slots[slots[s0 + i]];
      b.x[i] = sl.req.x;
      b.u[i] = sl.req.u;
      b.H[i] = sl.req.H;
      b.W[i] = sl.req.W;
      b.slot[i] = slots[s0 + i];
      b.iter[i] = 0;
    }
    cudaError_t e;
    if (large_fft(cl.N)) {
      LargeIO io{};
      io.T = q.tiles;
      io.spec_out = q.xh;
      io.tile_pairs = (c->K + 1) / 2;
      CodeIter none{};
      e = timed(c, OCSC_K_IMAGE_SPECTRUM, [&] { return launch_large(cl.N, LARGE_SPAT_IMAGE, none, b, io, b.n, 1, cl.tw, c->stream); });
      if (e == cudaSuccess)
        e = timed(c, OCSC_K_IMAGE_SPECTRUM, [&] { return launch_large(cl.N, LARGE_SPEC_IMAGE, none, b, io, b.n, 1, cl.tw, c->stream); });
    } else {
      e = timed(c, OCSC_K_IMAGE_SPECTRUM, [&] { return launch_image_spectrum(cl.N, b, cl.tw, q.xh, c->stream); });
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// One ADMM iteration for the given slots of one class and dictionary version.
cudaError_t launch_iteration(ocsc_server *s, int k, int v, const std::vector<int> &slots) {
  ocsc_ctx *c = s->ctx;
  const SizeClass &cl = c->cls[k];
  ServeClass &q = s->sc[k];
  const int npairs = (c->K + 1) / 2;
  CodeIter it{};
  it.K = c->K;
  it.F = cl.F;
  it.thr = (float)(c->lam / c->rho);
  it.Dh = q.D[v];
  it.r = q.r;
  it.What = q.What;
  it.Gam = q.Gam;
  it.Zp = q.Zp;
  it.serve = 1;
  it.check = s->o.check_every;
  it.resid = q.resid;
  it.rho = (float)c->rho;
  it.dn = q.dn[v];
  it.xh = q.xh;
  it.part = q.part;
  it.cnt = q.cnt;
  for (size_t s0 = 0; s0 < slots.size(); s0 += kMaxCallImages) {
    ImgBatch b{};
    b.n = (int)std::min<size_t>(kMaxCallImages, slots.size() - s0);
    for (int i = 0; i < b.n; ++i) {
      const Slot &sl = q.slots[slots[s0 + i]];
      b.x[i] = sl.req.x;
      b.u[i] = sl.req.u;
      b.H[i] = sl.req.H;
      b.W[i] = sl.req.W;
      b.slot[i] = slots[s0 + i];
      b.iter[i] = sl.iter;
    }
    cudaError_t e;
    if (large_fft(cl.N)) {
      LargeIO io{};
      io.T = q.tiles;
      io.tile_pairs = npairs;
      e = timed(c, OCSC_K_CODE_RESID, [&] { return launch_large(cl.N, LARGE_SPEC_DOT, it, b, io, b.n, npairs, cl.tw, c->stream); });
      if (e == cudaSuccess)
        e = timed(c, OCSC_K_CODE_RESID, [&] { return launch_large(cl.N, LARGE_SPEC_Z, it, b, io, b.n, npairs, cl.tw, c->stream); });
      if (e == cudaSuccess)
        e = timed(c, OCSC_K_CODE_PLANE, [&] { return launch_large(cl.N, LARGE_SPAT_ADMM, it, b, io, b.n, npairs, cl.tw, c->stream); });
    } else {
      e = timed(c, OCSC_K_CODE_RESID, [&] { return launch_code_resid(cl.N, b, it, (float)c->rho, q.dn[v], q.xh, c->stream); });
      if (e == cudaSuccess)
        e = timed(c, OCSC_K_CODE_PLANE, [&] { return launch_code_plane(cl.N, it, b, cl.tw, c->stream, cl.plane_ctas ? cl.plane_ctas : 2, cl.plane_ahead != 0, cl.plane_threads); });
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

extern "C" {

void ocsc_server_default_opts(ocsc_server_opts *o) {
  if (!o) return;
  o->tol = 1e-4;
  o->check_every = 5;
  o->max_iters = 500;
  o->mem_budget = (size_t)8 << 30;
  o->update_every = 64;
  o->learn = 1;
}

void ocsc_server_destroy(ocsc_server *s) {
  if (!s) return;
  ocsc_ctx *c = s->ctx;
  if (s->stream) cudaStreamSynchronize(s->stream);
  if (s->ctx_stream) c->stream = s->ctx_stream;
  cudaStreamSynchronize(c->stream);
  // Give the context back its own pending buffers (with the samples staged in
  // the server's set, if that one is current).
  if (!s->pend_Zp[0].empty()) {
    for (size_t k = 0; k < c->cls.size(); ++k) {
      SizeClass &cl = c->cls[k];
      if (s->pend_set == 1 && cl.pending > 0) {
        cudaMemcpy(s->pend_Zp[0][k], s->pend_Zp[1][k], (size_t)cl.pending * c->K * cl.F * sizeof(float2),
                   cudaMemcpyDeviceToDevice);
        cudaMemcpy(s->pend_xh[0][k], s->pend_xh[1][k], (size_t)cl.pending * cl.F * sizeof(float2),
                   cudaMemcpyDeviceToDevice);
      }
      cl.Zp = s->pend_Zp[0][k];
      cl.xhp = s->pend_xh[0][k];
    }
  }
  for (cudaEvent_t ev : {s->ev_stage, s->ev_pub, s->ev_read[0], s->ev_read[1]})
    if (ev) cudaEventDestroy(ev);
  if (s->stream) cudaStreamDestroy(s->stream);
  for (void *p : s->allocs) cudaFree(p);
  if (s->h_res) cudaFreeHost(s->h_res);
  if (s->h_slots) cudaFreeHost(s->h_slots);
  delete s;
}

ocsc_status ocsc_server_create(ocsc_server **out, ocsc_ctx *c, const ocsc_server_opts *opts) {
  if (!out || !c) return OCSC_EINVAL;
  *out = nullptr;
  ocsc_server *s = new ocsc_server();
  s->ctx = c;
  ocsc_server_default_opts(&s->o);
  if (opts) s->o = *opts;
  auto bail = [&](ocsc_status st) {
    ocsc_server_destroy(s);
    return st;
  };
  if (!(s->o.tol > 0) || s->o.check_every < 2 || s->o.max_iters < s->o.check_every || s->o.update_every < 0)
    return bail(fail(c, OCSC_EINVAL, "server: need tol > 0, check_every >= 2, max_iters >= check_every"));
  if (s->o.learn && s->o.update_every > c->opts.max_batch)
    return bail(fail(c, OCSC_EINVAL, "server: update_every %d exceeds the context's max_batch %d",
                     s->o.update_every, c->opts.max_batch));
  const int K = c->K, npairs = (K + 1) / 2;
  int max_slots = 0;
  s->sc.resize(c->cls.size());
  for (size_t k = 0; k < c->cls.size(); ++k) {
    const SizeClass &cl = c->cls[k];
    ServeClass &q = s->sc[k];
    const size_t KF = (size_t)K * cl.F;
    // Per request: Z~, the spatial state, the code U it writes, the sample
    // spectrum, r, and W^ (N <= 128) or the pair tiles and partial sums (N >= 256).
    const bool big = large_fft(cl.N);
    const int stages = big ? large_stages(cl.N, npairs) : 0;
    q.ws = KF * sizeof(float2) + (size_t)K * cl.P * sizeof(float) * 2 + (size_t)cl.F * sizeof(float2) * 2 +
           (big ? ((size_t)npairs * cl.P + (size_t)stages * cl.F) * sizeof(float2) : KF * sizeof(float2));
    q.nslots = (int)std::max<size_t>(1, std::min<size_t>(kMaxCallImages, s->o.mem_budget / q.ws));
    q.slots.resize(q.nslots);
    q.groups = big ? large_resid_groups(cl.N, npairs) : plane_resid_groups(c->K);
    const size_t ns = (size_t)q.nslots, nw = big ? 1 : ns;
    ocsc_status st;
    if ((st = salloc(s, &q.What, nw * KF)) || (st = salloc(s, &q.Zp, ns * KF)) ||
        (st = salloc(s, &q.Gam, ns * K * (size_t)cl.P)) || (st = salloc(s, &q.r, ns * cl.F)) ||
        (st = salloc(s, &q.xh, ns * cl.F)) || (st = salloc(s, &q.resid, ns * q.groups * kResidTerms)) ||
        (st = salloc(s, &q.d_slots, ns)) || (st = salloc(s, &q.d_res, ns * kResidTerms)) ||
        (st = salloc(s, &q.D[0], KF)) || (st = salloc(s, &q.D[1], KF)) || (st = salloc(s, &q.dn[0], (size_t)cl.F)) ||
        (st = salloc(s, &q.dn[1], (size_t)cl.F)))
      return bail(st);
    if (big) {
      if ((st = salloc(s, &q.tiles, ns * npairs * (size_t)cl.P)) || (st = salloc(s, &q.part, ns * stages * (size_t)cl.F)) ||
          (st = salloc(s, &q.cnt, ns * (size_t)(cl.N / 2))))
        return bail(st);
      cudaError_t e = cudaMemset(q.cnt, 0, ns * (size_t)(cl.N / 2) * sizeof(int));
      if (e != cudaSuccess) return bail(cuda_fail(c, e, "server: clear counters"));
    }
    max_slots = std::max(max_slots, q.nslots);
  }
  if (cudaMallocHost((void **)&s->h_res, (size_t)max_slots * kResidTerms * sizeof(double)) != cudaSuccess ||
      cudaMallocHost((void **)&s->h_slots, (size_t)max_slots * sizeof(int)) != cudaSuccess)
    return bail(fail(c, OCSC_ENOMEM, "server: pinned host buffers"));
  if (s->o.learn) {
    s->pend_Zp[0].resize(c->cls.size());
    s->pend_Zp[1].resize(c->cls.size());
    s->pend_xh[0].resize(c->cls.size());
    s->pend_xh[1].resize(c->cls.size());
    for (size_t k = 0; k < c->cls.size(); ++k) {
      SizeClass &cl = c->cls[k];
      s->pend_Zp[0][k] = cl.Zp;
      s->pend_xh[0][k] = cl.xhp;
      ocsc_status st;
      if ((st = salloc(s, &s->pend_Zp[1][k], (size_t)c->opts.max_batch * K * cl.F)) ||
          (st = salloc(s, &s->pend_xh[1][k], (size_t)c->opts.max_batch * cl.F)))
        return bail(st);
    }
  }
  // Request work gets the highest stream priority: while an update's long
  // FP64 CTAs hold the SMs, freed SMs go to request kernels first.
  int prio_least = 0, prio_greatest = 0;
  cudaError_t e = cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s->stream, cudaStreamNonBlocking, prio_greatest);
  for (cudaEvent_t *ev : {&s->ev_stage, &s->ev_pub, &s->ev_read[0], &s->ev_read[1]})
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "server: stream and events"));
  s->ctx_stream = c->stream;
  e = publish(s, 0);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventRecord(s->ev_read[i], c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "server: publish dictionary"));
  *out = s;
  return OCSC_OK;
}

ocsc_status ocsc_server_submit(ocsc_server *s, uint64_t id, const float *x, int H, int W, float *u) {
  if (!s) return OCSC_EINVAL;
  if (!x || !u || H <= 0 || W <= 0) return fail(s->ctx, OCSC_EINVAL, "server_submit: bad arguments");
  if (reinterpret_cast<uintptr_t>(u) % 16 != 0)
    return fail(s->ctx, OCSC_EINVAL, "server_submit: the code buffer must be 16-byte aligned");
  const int k = class_of(s->ctx, H, W);
  if (k < 0) return fail(s->ctx, OCSC_EUNSUPPORTED, "server_submit: %dx%d maps to no FFT size of this context", H, W);
  Request r;
  r.id = id;
  r.x = x;
  r.u = u;
  r.H = H;
  r.W = W;
  r.cls = k;
  s->queue.push_back(r);
  return OCSC_OK;
}

namespace {

// Enqueue a dictionary update on the context's stream after the staging copies
// of the serving stream, switch the pending set, and (publish) copy the new
// coding spectra into version slot 1 - cur, marked by ev_pub.
ocsc_status start_update(ocsc_server *s, bool publish_new) {
  ocsc_ctx *c = s->ctx;
  cudaError_t e = cudaEventRecord(s->ev_stage, s->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s->ctx_stream, s->ev_stage, 0);
  if (e != cudaSuccess) return cuda_fail(c, e, "server: order the update after staging");
  c->stream = s->ctx_stream;
  ocsc_status st = ocsc_update_dict(c);
  if (st == OCSC_OK && publish_new) {
    if ((e = publish(s, 1 - s->cur)) == cudaSuccess) e = cudaEventRecord(s->ev_pub, c->stream);
    if (e != cudaSuccess) st = cuda_fail(c, e, "server: publish dictionary");
    s->pub_pending = true;
    s->pub_slot = 1 - s->cur;
  }
  if (st == OCSC_OK && !s->pend_Zp[0].empty()) {
    // The update read the current pending set; further samples go to the other
    // one once the update that last read it has finished.
    if ((e = cudaEventRecord(s->ev_read[s->pend_set], c->stream)) != cudaSuccess)
      st = cuda_fail(c, e, "server: pending set event");
    s->pend_set = 1 - s->pend_set;
    for (size_t k = 0; k < c->cls.size(); ++k) {
      c->cls[k].Zp = s->pend_Zp[s->pend_set][k];
      c->cls[k].xhp = s->pend_xh[s->pend_set][k];
    }
    if (st == OCSC_OK && (e = cudaStreamWaitEvent(s->stream, s->ev_read[s->pend_set], 0)) != cudaSuccess)
      st = cuda_fail(c, e, "server: wait for the pending set");
  }
  c->stream = s->stream;
  return st;
}

}  // namespace

static ocsc_status step_body(ocsc_server *s, int *n_active, int *n_queued);

ocsc_status ocsc_server_step(ocsc_server *s, int *n_active, int *n_queued) {
  if (!s) return OCSC_EINVAL;
  NvtxRange range("ocsc_server_step");
  ocsc_ctx *c = s->ctx;
  // Request work runs on the server's stream for the whole step.
  struct StreamSwap {
    ocsc_ctx *c;
    cudaStream_t saved;
    ~StreamSwap() { c->stream = saved; }
  } swap{c, c->stream};
  c->stream = s->stream;
  return step_body(s, n_active, n_queued);
}

static ocsc_status step_body(ocsc_server *s, int *n_active, int *n_queued) {
  ocsc_ctx *c = s->ctx;
  cudaError_t e = cudaSuccess;
  // 0. A published dictionary becomes current once its copies are done.
  if (s->pub_pending && cudaEventQuery(s->ev_pub) == cudaSuccess) {
    s->cur = s->pub_slot;
    s->pub_pending = false;
  }
  // 1. Admission in arrival order.
  std::vector<std::vector<int>> admitted(s->sc.size());
  auto active_count = [&]() {
    int n = 0;
    for (auto &q : s->sc)
      for (auto &sl : q.slots) n += sl.used;
    return n;
  };
  while (!s->queue.empty()) {
    const Request &r = s->queue.front();
    ServeClass &q = s->sc[r.cls];
    int free_slot = -1;
    for (int i = 0; i < q.nslots; ++i)
      if (!q.slots[i].used) { free_slot = i; break; }
    const bool fits = s->mem_used + q.ws <= s->o.mem_budget || active_count() == 0;
    if (free_slot < 0 || !fits) break;
    Slot &sl = q.slots[free_slot];
    sl.used = true;
    sl.req = r;
    sl.iter = 0;
    sl.ver = s->cur;
    s->refs[s->cur]++;
    s->mem_used += q.ws;
    admitted[r.cls].push_back(free_slot);
    s->queue.pop_front();
  }
  for (size_t k = 0; k < s->sc.size(); ++k)
    if (!admitted[k].empty() && (e = launch_spectra(s, (int)k, admitted[k])) != cudaSuccess)
      return cuda_fail(c, e, "server: sample spectra");
  // 2. check_every iterations for every active request.
  for (int t = 0; t < s->o.check_every; ++t) {
    for (size_t k = 0; k < s->sc.size(); ++k) {
      ServeClass &q = s->sc[k];
      for (int v = 0; v < 2; ++v) {
        std::vector<int> slots;
        for (int i = 0; i < q.nslots; ++i)
          if (q.slots[i].used && q.slots[i].ver == v) slots.push_back(i);
        if (slots.empty()) continue;
        if ((e = launch_iteration(s, (int)k, v, slots)) != cudaSuccess) return cuda_fail(c, e, "server: iteration");
        for (int i : slots) q.slots[i].iter++;
      }
    }
  }
  // 3. Residuals (fixed-order reduction per request), completion.
  std::vector<std::pair<int, int>> order;  // (class, slot) in h_res order
  for (size_t k = 0; k < s->sc.size(); ++k) {
    ServeClass &q = s->sc[k];
    int n = 0;
    for (int i = 0; i < q.nslots; ++i)
      if (q.slots[i].used) s->h_slots[n++] = i;
    if (n == 0) continue;
    e = cudaMemcpyAsync(q.d_slots, s->h_slots, n * sizeof(int), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = launch_resid_reduce(q.d_slots, n, q.groups, q.resid, q.d_res, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->h_res, q.d_res, (size_t)n * kResidTerms * sizeof(double),
                                              cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "server: residuals");
    for (int j = 0; j < n; ++j) {
      Slot &sl = q.slots[s->h_slots[j]];
      const double *rs = s->h_res + (size_t)j * kResidTerms;
      const double zu = std::sqrt(rs[0]), zn = std::sqrt(rs[1]), un = std::sqrt(rs[2]);
      const double du = std::sqrt(rs[3]), gn = std::sqrt(rs[4]);
      const double scale_p = std::max(zn, un), scale_d = gn;  // dual: rho |U - U_prev| vs rho |Gamma|
      const double rp = scale_p > 0 ? zu / scale_p : 0.0;
      const double rd = scale_d > 0 ? du / scale_d : (du > 0 ? 1.0 : 0.0);
      if ((rp <= s->o.tol && rd <= s->o.tol) || sl.iter >= s->o.max_iters) {
        ocsc_served d;
        d.id = sl.req.id;
        d.iters = sl.iter;
        d.primal = rp;
        d.dual = rd;
        d.dict_version = s->ver_id[sl.ver];
        s->done.push_back(d);
        if (s->o.learn) {
          SizeClass &cl = c->cls[k];
          if (cl.pending >= c->opts.max_batch) {
            ocsc_status st = start_update(s, false);
            if (st != OCSC_OK) return st;
          }
          const size_t KF = (size_t)c->K * cl.F;
          e = cudaMemcpyAsync(cl.Zp + (size_t)cl.pending * KF, q.Zp + (size_t)s->h_slots[j] * KF, KF * sizeof(float2),
                              cudaMemcpyDeviceToDevice, c->stream);
          if (e == cudaSuccess)
            e = cudaMemcpyAsync(cl.xhp + (size_t)cl.pending * cl.F, q.xh + (size_t)s->h_slots[j] * cl.F,
                                cl.F * sizeof(float2), cudaMemcpyDeviceToDevice, c->stream);
          if (e != cudaSuccess) return cuda_fail(c, e, "server: stage for the update");
          cl.pending++;
          s->since_update++;
        }
        s->refs[sl.ver]--;
        s->mem_used -= q.ws;
        sl.used = false;
      }
    }
  }
  // 4. Dictionary update once enough requests completed and no request still
  //    uses the version slot the new dictionary goes to.
  if (s->o.learn && s->o.update_every > 0 && s->since_update >= s->o.update_every && s->refs[1 - s->cur] == 0 &&
      !s->pub_pending) {
    ocsc_status st = start_update(s, true);
    if (st != OCSC_OK) return st;
    s->since_update = 0;
  }
  if (n_active) *n_active = active_count();
  if (n_queued) *n_queued = (int)s->queue.size();
  return OCSC_OK;
}

ocsc_status ocsc_server_poll(ocsc_server *s, ocsc_served *out, int max, int *n) {
  if (!s || !n || (max > 0 && !out)) return OCSC_EINVAL;
  const int m = std::min<int>(max, (int)s->done.size());
  for (int i = 0; i < m; ++i) out[i] = s->done[i];
  s->done.erase(s->done.begin(), s->done.begin() + m);
  *n = m;
  return OCSC_OK;
}

}  // extern "C"
