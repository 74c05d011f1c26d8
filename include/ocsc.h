/*
 * ocsc.h -- C ABI of the GB300 (sm_103a) online convolutional sparse coding
 * library (Wang, Yao, Kwok & Ni, "Scalable Online Convolutional Sparse Coding").
 *
 * The library runs the method's hot path on one GPU:
 *   ocsc_code        -- per-sample code ADMM in the frequency domain
 *                       (Sec. II-C.1 problem (fcsc_code); Sec. III-B.2 says
 *                       codes are updated per sample as in batch CSC; ADMM
 *                       template of Sec. II-B, eqs. (admm_aux), (admm_dual)).
 *   ocsc_update_dict -- the online dictionary step of Algorithm 3: fold the
 *                       new codes into the per-frequency history A^p, b^p
 *                       (Sec. III-B, eqs. (A_update), (B_update)), then
 *                       DictOCSC (Algorithm 2): the D-row solve of eq.
 *                       (sub_d_sol) with C^p = (A^p + rho I)^-1 = X^H X, X the
 *                       inverse of the Cholesky factor (computed in
 *                       double-float, FP32 hi + lo pairs, ~48 significant
 *                       bits; for K > 128 the factor L itself), the support +
 *                       unit-ball projection of Proposition 2 and the scaled
 *                       dual update.
 *   ocsc_get_dict    -- the filters D_t (Algorithm 3, last loop).
 *
 * Conventions (shared by every call):
 *  - All image, code and filter arrays are float32, row-major.
 *  - Images are square or rectangular H x W; each is zero-padded at the end of
 *    both axes to an N x N FFT domain, N = the smallest FFT size of the context
 *    >= max(H, W) + pad.  Convolution is circular on that domain and filters
 *    occupy its top-left M x M corner.  Supported N: 64, 96, 128, 144, 192,
 *    256, 288, 384, 512, 576 (2^a 3^b); an image goes to the smallest size of
 *    the context that holds it.
 *  - lambda is the l1 weight (beta in the paper); rho is a spatial-domain
 *    ADMM penalty used by both ADMMs (the paper's frequency-domain penalty
 *    rho' of eq. (sub_d_sol) equals rho / P; opts.rho_convention = 1 uses the
 *    printed A + rho*P*I instead).
 *  - Device work is enqueued on the CUDA stream given to ocsc_init and is
 *    asynchronous with respect to the host unless a call says it synchronises.
 *  - Every call returns an ocsc_status; on failure ocsc_last_error() gives a
 *    message.  Nothing aborts the process.  A context is not thread-safe.
 *  - Ownership: the caller owns the images and code buffers it passes (they
 *    must stay valid until the stream has finished the work); the library owns
 *    all method state (dictionary spectra, duals, histories, factors,
 *    workspaces) and frees it in ocsc_destroy.
 */
#ifndef OCSC_H
#define OCSC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ocsc_ctx ocsc_ctx;

typedef enum {
  OCSC_OK = 0,
  OCSC_EINVAL = 1,       /* bad argument (null pointer, non-positive size ...) */
  OCSC_ENOMEM = 2,       /* device allocation failed */
  OCSC_ECUDA = 3,        /* a CUDA runtime call or kernel launch failed */
  OCSC_ETIMEOUT = 4,     /* a bounded device wait gave up */
  OCSC_ESTATE = 5,       /* call not valid in the current state */
  OCSC_EUNSUPPORTED = 6, /* size or option outside what this build supports */
  OCSC_ENUMERIC = 7      /* a factorisation met a non-positive pivot */
} ocsc_status;

#define OCSC_MAX_FFT_SIZES 12

typedef struct {
  int Jz;             /* code-ADMM iterations per sample (default 50) */
  int Jd;             /* dictionary-ADMM iterations per update (default 10) */
  int pad;            /* zeros appended per axis before the FFT; -1 (default)
                         means filter side - 1, so that the circular model has
                         no wrap-around across the image boundary */
  int max_batch;      /* most samples that may be pending between two
                         ocsc_update_dict calls (default 1) */
  int fft_sizes[OCSC_MAX_FFT_SIZES]; /* the FFT sides N this context serves,
                         zero-terminated, each of 64, 96, 128, 144, 192, 256,
                         288, 384, 512, 576 (default {128, 0, ...}).
                         Each size is a class with its own history, factor,
                         dual and coding spectrum of the one shared
                         dictionary; with several classes the dictionary step
                         is the consensus DictOCSC over the classes that have
                         seen samples (class weights n_c / n).  An image goes
                         to the class of its padded size. */
  int warm_start;     /* 1 (default): V and the dual theta of DictOCSC carry
                         over between updates; 0: restart at 0 each update as
                         Algorithm 2 prints its initialisation */
  int return_feasible;/* 1 (default): code against F(V_{t,J}) (feasible);
                         0: against D~_{t,J} as Algorithm 2 returns it */
  int rho_convention; /* 0 (default): D-row matrix A + rho I; 1: A + rho P I */
  uint64_t seed;      /* seed of the Gaussian initial filters */
  int precision;      /* history fold (eqs. (A_update), (B_update)):
                         0 (default): FP32 on the CUDA cores;
                         1: the K x K sums of conj(z) z^T per frequency on the
                            tensor cores with BF16 operands and FP32
                            accumulation, the history kept as a compensated
                            pair of FP32 words (A + Alo) across the stream;
                         2: as 1 with each code split into two BF16 words
                            (hi + lo; products hi hi + hi lo + lo hi);
                         3: the products conj(z_i) z_j and x~ conj(z_i) split
                            exactly and summed in double-float (FP32 pairs),
                            the running means A + Alo and b + blo kept as
                            pairs (K <= 128).  A and b then stay exact
                            functions of the same FP32 codes; with the
                            separately rounded FP32 products of 0 the solve's
                            forward error grows like u cond(w A + rho I)
                            (u = 2^-24), which matters at small rho. */
  int autotune;       /* 1 (default): at a size class's first use, time the
                         candidate tile shapes on its own buffers and keep the
                         fastest: threads per CTA of the factorisation
                         (256 or 512), columns per CTA of the N >= 256 spatial
                         FFT kernel in ocsc_code (8 or 16), CTAs per SM of the
                         N <= 128 coding plane kernel (256 threads at 2 or 3,
                         512 threads at 2, each with and without the L2
                         look-ahead, or 512-thread persistent CTAs with two
                         tiles), samples per
                         chunk of the tensor-core contraction (32, 64, 128).  Every
                         candidate performs the same operations in the same
                         order, so results do not depend on the choice.
                         0: fixed defaults (256, the size's default, largest
                         chunk that fits). */
  int graphs;         /* 1: ocsc_code replays a CUDA graph per chunk shape
                         (class, image count, first slot, image sizes, codes
                         requested or not): the second call with a shape
                         captures the sample spectra and the Jz iterations,
                         later calls copy their images into library staging
                         slots and launch the graph (codes are copied out).
                         Not used while coding kernels are profiled.  0
                         (default): every launch is issued directly. */
  int history;        /* 0 (default): keep A^p and factor w A^p + rho I at
                         every update (the C^p definition of eq. (sub_d_sol)).
                         1: keep C^p itself (double-float) and apply the
                         printed Sherman-Morrison recursion of eq. (C_update)
                         per folded sample (O(K^2)); it yields
                         C_t = (A_t + (rho P / t) I)^-1, a ridge that decays
                         with the sample count t, and DictOCSC then runs with
                         the matching penalty rho / t (the scaled dual carried
                         as rho Theta across updates).  Needs rho_convention 1 (the
                         printed rho P: with the spatial rho the first C
                         already has a condition number near |z|^2 / rho and
                         the rank-one downdates diverge, in FP64 too), one FFT
                         size, precision 0 and K <= 128. */
  int persistent;     /* 1: ocsc_code runs all Jz iterations of the images of
                         FFT sizes 64, 128, 256 and 512 in one cooperative
                         launch per chunk of up to 64 images (sizes may be
                         mixed in one launch), after their sample spectra:
                         every CTA of a co-resident grid walks the units of
                         the per-iteration kernels, three intervals per
                         iteration separated by a bounded grid barrier.  Codes
                         are identical to those of the per-iteration launches.
                         Other sizes take the per-iteration path.  0 (default):
                         per-iteration launches. */
  int band_lo, band_hi; /* 0, 0 (default): the context solves every frequency.
                         0 <= band_lo < band_hi <= N (one FFT size, an even row
                         count): a band context, which keeps the history and
                         factor of the frequencies of rows k1 in
                         [band_lo, band_hi) only and updates its dictionary
                         through the ocsc_band_* calls (frequency-band
                         sharding of the dictionary step).  Needs history 0,
                         precision 0 or 3, K <= 128, return_feasible 1. */
} ocsc_opts;

/* Fill *o with the defaults listed above. */
void ocsc_default_opts(ocsc_opts *o);

/*
 * Create a context for K filters of filter_h x filter_w (square only:
 * filter_h == filter_w = M, M <= 16; K <= 256; above 128 the factor is
 * blocked through a global FP64 workspace of one matrix per SM), l1 weight lambda >= 0 and
 * penalty rho > 0.  opts may be NULL (defaults).  cuda_stream is a
 * cudaStream_t (NULL = legacy default stream).  The initial dictionary is
 * Algorithm 3's Gaussian random initialisation: K x M x M N(0,1) draws from a
 * splitmix64/Box-Muller generator seeded by opts->seed, each filter scaled to
 * unit l2 norm; ocsc_set_dict replaces it.
 * Allocates all device state per size class (history and factor:
 * 2 * F * K(K+1)/2 * 8 bytes with F = N * (N/2 + 1); coding workspaces of
 * about max_batch * K * N^2 * 24 bytes, plus for N >= 256 a complex N x N tile
 * per pending sample and filter pair).  On failure *out is NULL and
 * ocsc_last_error(NULL) gives the reason.
 */
ocsc_status ocsc_init(ocsc_ctx **out, int K, int filter_h, int filter_w, double lambda,
                      double rho, const ocsc_opts *opts, void *cuda_stream);

/* Release every device and host resource of ctx (NULL is a no-op).
 * Synchronises ctx's stream first. */
void ocsc_destroy(ocsc_ctx *ctx);

/* Padded FFT side N for an H x W image: the smallest FFT size of ctx that
 * holds max(H, W) + pad (OCSC_EUNSUPPORTED if none does). */
ocsc_status ocsc_padded_size(const ocsc_ctx *ctx, int H, int W, int *N);

/*
 * Code n samples against the current dictionary (Algorithm 3, FFT and code
 * steps).  x[i] is a DEVICE pointer to an H[i] x W[i] float image; u[i] is a
 * DEVICE pointer to a caller-owned K x N x N float buffer that receives the
 * sparse code U_i after the last U-step, or NULL to skip writing it (16-byte
 * aligned, as cudaMalloc and torch allocations are; OCSC_EINVAL otherwise).  x, H, W
 * and u are HOST arrays of length n.  Every image must map to one of the
 * context's FFT sizes; images of different sizes may be mixed in one call.
 * The last Z~-step of each sample and its spectrum stay pending inside the
 * library for the next ocsc_update_dict; per size class, pending + new must
 * not exceed opts.max_batch (OCSC_ESTATE otherwise).  Asynchronous.
 */
ocsc_status ocsc_code(ocsc_ctx *ctx, int n, const float *const *x, const int *H,
                      const int *W, float *const *u);

/*
 * Fold every pending sample into the history (running mean over all samples
 * seen) and run DictOCSC for Jd iterations.  No pending samples: no-op.
 * Asynchronous; errors found on the device (non-positive pivot) are reported
 * by the next synchronising call.
 */
ocsc_status ocsc_update_dict(ocsc_ctx *ctx);

/*
 * Copy the filters D_t (K x M x M floats) to HOST memory D_host and the
 * dictionary version (number of completed updates) to *version (nullable).
 * With return_feasible = 1, D_t = V_{t,J} (feasible); with return_feasible = 0,
 * D_t = H(F^-1(D~_{t,J})), the support crop of the D~ that Algorithm 2 returns
 * (Algorithm 3, last loop), formed on the device.  Synchronises ctx's stream
 * and reports pending device-side errors.
 */
ocsc_status ocsc_get_dict(ocsc_ctx *ctx, float *D_host, uint64_t *version);

/*
 * Replace the dictionary with K x M x M floats from HOST memory.  normalize=1
 * scales each filter to unit l2 norm (the initialisation of Algorithm 3);
 * normalize=0 takes them as given (they must satisfy ||D_k|| <= 1).  Resets
 * the DictOCSC dual to 0; the history is kept.  Synchronises.
 */
ocsc_status ocsc_set_dict(ocsc_ctx *ctx, const float *D_host, int normalize);

/*
 * Checkpoint of the learner between dictionary updates (the paper has no
 * counterpart; it keeps the state of Algorithm 3 across a restart): the
 * filters V, and per size class the coding and DictOCSC spectra (V^, theta^,
 * D~), the history A (packed) and b, |d|^2 and the sample counts.
 * ocsc_get_state with buf == NULL stores the byte count in *len; otherwise it
 * copies the state into HOST buf (*len >= that count, set to it on return).
 * OCSC_ESTATE if samples are pending (call ocsc_update_dict or
 * ocsc_drop_pending first).  ocsc_set_state loads a state saved by a context
 * with the same K, filter size, lambda, rho, conventions and FFT sizes
 * (OCSC_EINVAL otherwise; nothing is changed then).  Both synchronise.
 */
ocsc_status ocsc_get_state(ocsc_ctx *ctx, void *buf, size_t *len);
ocsc_status ocsc_set_state(ocsc_ctx *ctx, const void *buf, size_t len);

/* Tile shapes in use for FFT size N (0 where not tuned yet or not used). */
typedef struct {
  int fold_threads; /* CTA size of the K <= 128 fold + factorisation */
  int spat_cb;      /* columns per CTA of the N >= 256 spatial kernel in ocsc_code */
  int gram_sc;      /* samples per chunk of the tensor-core contraction */
  int plane_ctas;   /* CTAs per SM the N <= 128 coding plane kernel's register
                       budget is sized for (2 or 3) */
  int plane_ahead;  /* 1: each plane CTA asks L2 for the data of the CTA that
                       runs one residency later (N <= 128); 0: it does not */
  int plane_threads; /* CTA size of the N <= 128 coding plane kernel (256, or
                        512 at N = 128: 2 CTAs per SM, or 1 persistent CTA
                        per SM with two tiles) */
} ocsc_tuning;
ocsc_status ocsc_get_tuning(const ocsc_ctx *ctx, int N, ocsc_tuning *out);
/* Pin tile shapes of FFT size N before (or instead of) the autotuner: every
 * nonzero field is checked and kept, and the autotuner leaves a pinned knob
 * alone.  plane_ctas != 0 sets the plane kernel's shape (plane_threads 256
 * with plane_ctas 2 or 3, or at N = 128 512 with 2, or 512 with 1: persistent
 * CTAs with two tiles, batch coding only; plane_ahead 0 or 1);
 * fold_threads 256 or 512; spat_cb 8 or 16 for N >= 256 where supported;
 * gram_sc must be 0.  No tile shape changes any result (each performs the
 * same operations in the same order).  OCSC_EINVAL on a bad value (nothing
 * is changed), OCSC_EUNSUPPORTED if the context has no class of side N. */
ocsc_status ocsc_set_tuning(ocsc_ctx *ctx, int N, const ocsc_tuning *in);

/* Block until all work queued on ctx's stream is done; reports device errors. */
ocsc_status ocsc_sync(ocsc_ctx *ctx);

/* Message of the last failed call on ctx, or of the last failed ocsc_init on
 * this thread when ctx is NULL (never NULL). */
const char *ocsc_last_error(const ocsc_ctx *ctx);

/*
 * Forget the samples coded since the last ocsc_update_dict without folding them
 * into the history (for coding held-out or served samples against a fixed
 * dictionary).  Host-side bookkeeping only.
 */
ocsc_status ocsc_drop_pending(ocsc_ctx *ctx);

/*
 * Objective of eq. (ocsc0) per sample against the current coding dictionary:
 * out_host[i] = 1/2 ||x_i - sum_k D_k (*) U_i,k||^2 + lambda ||U_i||_1, with the
 * convolution circular on the padded N x N domain and x_i zero-padded as in
 * ocsc_code.  x, H, W are as in ocsc_code; u[i] is a DEVICE pointer to the
 * K x N x N codes (for instance those ocsc_code wrote).  The residual norm is
 * taken in the frequency domain by Parseval's identity (Sec. II-C); sums are
 * FP64 and deterministic.  out_host is a HOST array of n doubles.
 * Synchronises.
 */
ocsc_status ocsc_objective(ocsc_ctx *ctx, int n, const float *const *x, const int *H, const int *W,
                           const float *const *u, double *out_host);

/*
 * The two terms of the objective separately (evaluation of Sec. IV: the test
 * set objective and the PSNR of the reconstruction sum_k D_k (*) U_k):
 * resid2_host[i] = ||x_i - sum_k D_k (*) U_ik||^2 over the padded N x N domain,
 * l1_host[i] = ||U_i||_1.  Same arguments and rules as ocsc_objective.
 */
ocsc_status ocsc_objective_terms(ocsc_ctx *ctx, int n, const float *const *x, const int *H, const int *W,
                                 const float *const *u, double *resid2_host, double *l1_host);

/*
 * ||a - b||_2 / ||a||_2 over count floats of two DEVICE arrays (FP64, fixed
 * summation order; the relative changes of the stopping rule of Sec. IV).
 * Result in *out_host (0 for count = 0, +inf if a = 0 and b != 0).  Synchronises.
 */
ocsc_status ocsc_rel_diff(ocsc_ctx *ctx, const float *a, const float *b, size_t count, double *out_host);

/*
 * PSNR of the reconstruction sum_k D_k (*) U_ik against x_i, the test-set
 * measure of Sec. IV: psnr_host[i] = 10 log10(peak^2 P_i / ||x_i - sum_k D_k (*)
 * U_ik||^2) with P_i the pixel count of the sample's padded N x N domain (the
 * domain the model is defined on) and peak > 0 the signal peak (255 for the
 * paper's 8-bit images).  Same arguments and rules as ocsc_objective; the
 * logarithm is taken on the device in FP64.  Synchronises.
 */
ocsc_status ocsc_psnr(ocsc_ctx *ctx, int n, const float *const *x, const int *H, const int *W,
                      const float *const *u, double peak, double *psnr_host);

/*
 * Display order of the filters (Sec. IV, the learned filters shown sorted by
 * variance): order_host[r] (HOST, K ints) = the index of the filter with the
 * r-th smallest sample variance over its M x M entries (sum of squared
 * deviations divided by M*M - 1; 0 when M = 1), ties in index order.  Computed
 * on the device from the current filters D_t.  Synchronises.
 */
ocsc_status ocsc_filter_order(ocsc_ctx *ctx, int *order_host);

/*
 * Copy the filters D_t (K x M x M floats) into the DEVICE buffer D_dev
 * (caller-owned), on ctx's stream; asynchronous.  With ocsc_rel_diff this gives
 * the dictionary change of the stopping rule of Sec. IV without a host copy.
 */
ocsc_status ocsc_copy_dict(ocsc_ctx *ctx, float *D_dev);

/*
 * Poll budget of the bounded device waits of ctx (the tensor-core history
 * fold's wait for its MMAs; the persistent coder's grid barrier): a wait that
 * has polled this many times gives up, the kernel records OCSC_ETIMEOUT in the
 * context's device error word, finishes or releases what it holds (a timed-out
 * tensor-core fold still waits, with the full default budget, for the MMAs it
 * issued before it frees tensor memory) and returns; the next synchronising
 * call reports OCSC_ETIMEOUT and clears the word.  The paper has no
 * counterpart: the hook exists so that the failure path can be exercised
 * (polls = 0 makes every such wait give up at once).  Default 2^24.  The
 * history of an update that timed out is left as it was before the update.
 */
ocsc_status ocsc_set_wait_limit(ocsc_ctx *ctx, uint64_t polls);

/*
 * Frequency-band sharding of the dictionary step.  Proposition 1 (Sec. III-B)
 * decouples the D-row systems of eq. (sub_d_sol) per frequency, so the
 * history, its factorisation and the D~-step split by frequency band; only the
 * V-step of Proposition 2 couples the bands, through the support crop
 * H(F^-1(D~ + theta^)), which is a sum over frequencies.  With G contexts (one
 * per GPU, each a band context owning rows [band_lo, band_hi) of k1; the bands
 * cover 0 .. N once) one update of Algorithm 2 is:
 *   1. every context codes its own samples (ocsc_code) and exports each band's
 *      rows of their Z~ and x~ (ocsc_band_export); the caller moves them to the
 *      band owners (an all-to-all) and concatenates them in one global sample
 *      order (the order of the fold);
 *   2. every context folds the B samples of the mini-batch into its band and
 *      factors it (ocsc_band_fold);
 *   3. Jd times: ocsc_band_dict_step writes the band's share of the support
 *      sums alpha (K x M x M floats); the caller adds the G shares in a fixed
 *      order (an all-reduce of K M^2 floats) and passes the sum to every
 *      context's ocsc_band_project (last = 1 on the last iteration, which also
 *      publishes the new dictionary and its coding spectrum);
 *   4. every context drops its pending samples (ocsc_drop_pending).
 * All contexts then hold the same filters D_t.  All calls are asynchronous on
 * the context's stream; Z_dev, x_dev, alpha_dev are DEVICE buffers owned by the
 * caller.  Errors: OCSC_ESTATE when ctx is not a band context (band_fold,
 * band_dict_step, band_project) or nothing has been folded yet
 * (band_dict_step); OCSC_EINVAL for bad arguments.
 *
 * ocsc_band_export: the pending samples' Z~ rows k1 in [k1_lo, k1_hi) as
 *   [pending][K][(k1_hi - k1_lo)(N/2 + 1)] complex floats (interleaved) into
 *   Z_dev, their x~ rows as [pending][(k1_hi - k1_lo)(N/2 + 1)] into x_dev.
 *   Any context may export any band.
 * ocsc_band_fold: fold B samples, given in that layout for this context's
 *   band, in order (eqs. (A_update), (B_update), the running mean over all
 *   samples seen), then factor the band (eq. (sub_d_sol)).
 * ocsc_band_dict_step: the D~-step of the band, then alpha_dev[k][m1][m2] =
 *   (1/P) sum over the band's frequencies of the inverse-DFT terms of
 *   D~ + theta^ on the M x M support.
 * ocsc_band_project: V = Proposition 2 of alpha_dev, then V^ = F(pad V) and
 *   the scaled dual on the band.
 */
ocsc_status ocsc_band_export(ocsc_ctx *ctx, int k1_lo, int k1_hi, float *Z_dev, float *x_dev);
ocsc_status ocsc_band_fold(ocsc_ctx *ctx, int B, const float *Z_dev, const float *x_dev);
ocsc_status ocsc_band_dict_step(ocsc_ctx *ctx, float *alpha_dev);
ocsc_status ocsc_band_project(ocsc_ctx *ctx, const float *alpha_dev, int last);

/*
 * Serving: continuous batching of coding requests over one context
 * (spec serving pattern; each request runs the code ADMM of
 * Sec. II-C.1 to a residual tolerance instead of a fixed iteration count).
 *
 * Requests are admitted in arrival order while a workspace slot of their size
 * class is free and the sum of the admitted requests' working sets stays within
 * mem_budget bytes.  Each ocsc_server_step advances every admitted request by
 * check_every ADMM iterations (requests at different iteration counts share the
 * same launches), then reduces each request's relative primal residual
 * |Z - U| / max(|Z|, |U|) and dual residual |U - U_prev| / |Gamma| in a fixed
 * order and completes the requests whose both residuals are <= tol, or that
 * reached max_iters.  A completed request's code U is in its output buffer.
 * With learn = 1 completed requests are folded into the history and DictOCSC
 * runs after every update_every completions (Algorithm 3 with mini-batches);
 * a request is coded against the dictionary current at its admission, so its
 * result does not depend on the other requests in flight.
 */
typedef struct ocsc_server ocsc_server;

typedef struct {
  double tol;          /* relative residual target (default 1e-4) */
  int check_every;     /* iterations per step and between checks (default 5, >= 2) */
  int max_iters;       /* iteration cap (default 500) */
  size_t mem_budget;   /* bytes of in-flight working sets (default 8 GiB) */
  int update_every;    /* completions between dictionary updates (default 64;
                          must not exceed the context's max_batch) */
  int learn;           /* 1 (default): fold completed requests, update the dictionary */
} ocsc_server_opts;

typedef struct {
  uint64_t id;           /* the id given at submission */
  int iters;             /* ADMM iterations run */
  double primal, dual;   /* relative residuals at completion */
  uint64_t dict_version; /* dictionary version (ocsc_get_dict) it was coded with */
} ocsc_served;

void ocsc_server_default_opts(ocsc_server_opts *o);

/* Create a server on ctx (which must outlive it); allocates the slot
 * workspaces of every size class (at most 64 slots per class, as many as fit
 * mem_budget). */
ocsc_status ocsc_server_create(ocsc_server **out, ocsc_ctx *ctx, const ocsc_server_opts *opts);
void ocsc_server_destroy(ocsc_server *s);

/* Queue one request: x (DEVICE, H x W floats) is coded into u (DEVICE,
 * K x N x N floats, N its padded size, 16-byte aligned).  Both stay owned by the caller and must
 * remain valid until the request is reported by ocsc_server_poll. */
ocsc_status ocsc_server_submit(ocsc_server *s, uint64_t id, const float *x, int H, int W, float *u);

/* One scheduling round (admission, check_every iterations, residual checks,
 * completions, a due dictionary update).  Synchronises ctx's stream.  Reports
 * the requests in flight and still queued. */
ocsc_status ocsc_server_step(ocsc_server *s, int *n_active, int *n_queued);

/* Copy up to max completed requests (completion order) to out; *n = count. */
ocsc_status ocsc_server_poll(ocsc_server *s, ocsc_served *out, int max, int *n);

/* Kernel classes for ocsc_profile / ocsc_profile_read. */
typedef enum {
  OCSC_K_IMAGE_SPECTRUM = 0, /* x~ = F(pad x) */
  OCSC_K_CODE_RESID = 1,     /* per-frequency residual of the Z~-step (N >= 256:
                                the spectral row kernels) */
  OCSC_K_CODE_PLANE = 2,     /* fused code-ADMM iteration per filter pair (N >= 256:
                                the spatial column kernel) */
  OCSC_K_FOLD_FACTOR = 3,    /* history fold + Cholesky (double-float)
                                + FP32 L^-1 per frequency; with history = 1 the
                                Sherman-Morrison fold */
  OCSC_K_DSTEP = 4,          /* D-row solve of eq. (sub_d_sol) */
  OCSC_K_VSTEP_COLS = 5,     /* pruned inverse DFT along the first axis */
  OCSC_K_VSTEP_PROJECT = 6,  /* Proposition 2 projection of the support */
  OCSC_K_DICT_NORMS = 7,     /* |D~(p,:)|^2 of the coding dictionary */
  OCSC_K_VSTEP_SPECTRUM = 8, /* V^ = F(pad V) and the dual update */
  OCSC_K_HISTORY_TC = 9,     /* tensor-core history fold (opts.precision 1 or 2) */
  OCSC_K_PERSIST = 10,       /* persistent coder: all Jz iterations of a chunk (opts.persistent) */
  OCSC_K_COUNT = 11
} ocsc_kernel;

typedef struct {
  uint64_t kernel_launches; /* kernels launched by this context so far */
  uint64_t samples_coded;   /* samples passed to ocsc_code */
  uint64_t dict_updates;    /* completed ocsc_update_dict calls that folded samples */
  uint64_t graph_launches;  /* CUDA graph replays of ocsc_code (opts.graphs); their
                               kernels are included in kernel_launches */
} ocsc_counters;

/* Counters of ctx (host-side bookkeeping; no synchronisation). */
ocsc_status ocsc_get_counters(const ocsc_ctx *ctx, ocsc_counters *out);

/*
 * Enable CUDA-event timing of every launch of the kernel classes whose bit
 * (1 << ocsc_kernel) is set in mask (0 disables).  Events are recorded on
 * ctx's stream immediately before and after each launch.
 */
ocsc_status ocsc_profile(ocsc_ctx *ctx, unsigned mask);

/*
 * Total device time (ms) and number of timed launches of one kernel class
 * since the last read; clears that class's records.  Synchronises.
 */
ocsc_status ocsc_profile_read(ocsc_ctx *ctx, int kernel, double *total_ms, uint64_t *launches);

/*
 * Building block: forward 2D DFT (the F of Sec. II-C, unnormalised) of
 * `planes` real N x N float planes x (DEVICE, contiguous) into half spectra
 * N x (N/2+1) of interleaved complex float X (DEVICE).  N must be one of the
 * context's FFT sizes.  Enqueued on ctx's stream.
 */
ocsc_status ocsc_fft2_r2c(ocsc_ctx *ctx, int N, const float *x, float *X, int planes);

/* Building block: inverse of ocsc_fft2_r2c, including the 1/P factor.  The
 * input half spectra must be those of real planes (Hermitian symmetric). */
ocsc_status ocsc_fft2_c2r(ocsc_ctx *ctx, int N, const float *X, float *x, int planes);

/* Size of the fixed device array used by ocsc_code_noalloc (32 MiB). */
#define OCSC_NOALLOC_SCRATCH_BYTES (32u << 20)

/*
 * Allocation-free coding of one image.  The paper has no counterpart: this is
 * a deployment variant of ocsc_code for callers that must not allocate device
 * memory while they run -- for instance a plug-in whose host application has
 * reserved all device memory through its own allocator, a latency-critical
 * pipeline that cannot absorb the device-wide synchronisation cudaMalloc and
 * cudaFree may cause, or a service that must not fail at run time for lack of
 * memory.  It calls no cudaMalloc, cudaFree or allocating library routine.
 *
 * It codes the H x W image x (DEVICE floats, zero-padded at the end of both
 * axes to N x N, N in {64, 128}, H, W <= N) against the K filters D (DEVICE,
 * K x M x M floats, M <= 16, used as given) with Jz code-ADMM iterations of
 * ocsc_code's kernels, and writes the sparse code U (DEVICE, K x N x N floats,
 * 16-byte aligned, caller-owned) -- the same result ocsc_code gives for that image and
 * dictionary.  Work is enqueued on cuda_stream (a cudaStream_t; NULL = legacy
 * default stream); the call is asynchronous.  err (nullable, err_len bytes)
 * receives a message on failure.
 *
 * Scratch lives in one file-scope device array of OCSC_NOALLOC_SCRATCH_BYTES.
 * The scratch needed is about K * ((3 N + 16) (N/2+1) * 8 + N * N * 4) bytes
 * (K <= 122 at N = 128, K <= 128 at N = 64); larger requests return
 * OCSC_EUNSUPPORTED without touching the device.  Every call looks up the
 * array's device address (cudaGetSymbolAddress) with the caller's device
 * current.  Under CUDA's default lazy module loading the array and the coding
 * kernels are loaded on a device by the first call there, and that loading can
 * take device memory; from then on the array stays resident on that device
 * until the process exits and calls allocate nothing.  A caller that must not
 * allocate after start-up makes one valid call at start-up, or runs with
 * CUDA_MODULE_LOADING=EAGER (the array is then loaded with the library).  All
 * calls share the array and it keeps the last call's contents (every call
 * rewrites what it reads before reading it); calls whose work overlaps on the
 * GPU -- on different streams or from different host threads -- race on it and
 * must be serialised by the caller.
 */
ocsc_status ocsc_code_noalloc(const float *x, int H, int W, const float *D, int K, int M, int N,
                              double lambda, double rho, int Jz, float *u, void *cuda_stream,
                              char *err, size_t err_len);

#ifdef __cplusplus
}
#endif

#endif /* OCSC_H */
