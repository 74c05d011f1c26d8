// Internal launch interface between the C-ABI runtime and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ocsc {

constexpr int kMaxCallImages = 64;  // images per kernel-parameter batch

// Per-call image table, passed by value as a kernel parameter.  Image i of a
// launch uses workspace slot slot[i] (its spectrum, W^, Gamma, r, Z~ and, for
// N >= 256, its tiles); iter[i] is its ADMM iteration index when the launch
// runs in serving mode.
struct ImgBatch {
  const float *x[kMaxCallImages];  // device images, H x W row-major
  float *u[kMaxCallImages];        // device code outputs K x N x N (or null)
  int H[kMaxCallImages];
  int W[kMaxCallImages];
  int slot[kMaxCallImages];
  int iter[kMaxCallImages];
  int n;
};

// Code-ADMM iteration parameters.  Workspace pointers are slot 0 of arrays
// indexed by ImgBatch::slot.
struct CodeIter {
  int K, F;
  int first, last;     // batch mode: first / last ADMM iteration of this call
  float thr;           // lambda / rho
  const float2 *Dh;    // [K][F] dictionary spectrum used for coding
  float2 *r;           // [slots][F] per-frequency residual multipliers
  float2 *What;        // [slots][K][F] F(U - Gamma)
  float *Gam;          // [slots][K][N*N] spatial state: Gamma (N <= 128); U tiled by column block (N >= 256)
  float2 *Zp;          // [slots][K][F] last Z~ (written on the last iteration)
  // Serving mode (serve = 1): every image has its own iteration index; at
  // iterations t with (t + 1) % check == 0 the kernel stores Z~ and U and
  // writes its share of the residual sums, at (t + 2) % check == 0 it stores U
  // (the U_prev of the next check).  The forward transform always runs.
  int serve, check;
  float *resid;        // [slots][groups][kResidTerms] partial sums
  // N >= 256 only: the spectral kernels form r (into `r`) from these.
  float rho;
  const float *dn;     // [F] |D~(p,:)|^2 of Dh
  const float2 *xh;    // [slots][F] sample spectra
  float2 *part;        // [slots][stages][F] partial sums of D^T w^
  int *cnt;            // [slots][N/2] arrival counters (zero between launches)
  // N <= 128: the plane kernel's CTA i asks L2 for the W^ and Gamma of CTA
  // i + ahead (about the CTAs resident at once, so the data arrives while
  // this CTA computes); 0 turns it off.
  int ahead;
};
constexpr int kResidTerms = 5;  // |Z-U|^2, |Z|^2, |U|^2, |U-U_prev|^2, |Gamma|^2

cudaError_t launch_image_spectrum(int N, const ImgBatch &b, const float2 *tw, float2 *xh,
                                  cudaStream_t s);
cudaError_t launch_code_resid(int N, const ImgBatch &b, const CodeIter &it, float rho, const float *dn,
                              const float2 *xh, cudaStream_t s);
// Per-slot residual sums (double, fixed order) from `groups` partials per slot.
cudaError_t launch_resid_reduce(const int *slots_dev, int n, int groups, const float *partials,
                                double *out, cudaStream_t s);
// threads: CTA size (256; 512 for N = 128); ctas: CTAs per SM the kernel's
// register budget is sized for (2 or 3 with 256 threads, 2 with 512); ahead:
// L2 prefetch of the data of the CTA one residency later (CodeIter::ahead).
// None of them changes the results; an unsupported shape returns
// cudaErrorInvalidValue.
cudaError_t launch_code_plane(int N, const CodeIter &it, const ImgBatch &b, const float2 *tw,
                              cudaStream_t s, int ctas = 2, bool ahead = true, int threads = 256);
bool plane_shape_ok(int N, int threads, int ctas);
// Residual partial sums per slot written by code_plane in serving mode (one per CTA).
int plane_resid_groups(int K);
cudaError_t launch_fft2(int N, int inverse, const float *in, float *out, int planes,
                        const float2 *tw, cudaStream_t s);

// FFT sizes 256 and 512 (code_large.cu): per (sample, filter pair) a complex
// tile M[N][N] in global memory holds the column-transformed packed pair
// between the spectral (row) and spatial (column) kernels of an iteration.
struct LargeIO {
  float2 *T;              // tiles [slots][tile_pairs][N][N] (r2c / c2r: [pairs][N][N])
  const float2 *spec_in;  // c2r input half spectra [planes][F]
  float2 *spec_out;       // r2c output [planes][F], or sample spectra [slots][F]
  const float *real_in;   // r2c input planes [planes][N][N]
  float *real_out;        // c2r output planes [planes][N][N]
  int planes;             // planes of an r2c / c2r call
  int tile_pairs;         // tiles per slot (ceil(K / 2)) for the ADMM and sample-spectrum modes
  int spat_cb;            // columns per spatial CTA, 8 or 16 (0: the size's default; serving
                          // residual partials assume the default)
};
enum {
  LARGE_SPEC_DOT, LARGE_SPEC_Z, LARGE_SPEC_IMAGE, LARGE_SPEC_R2C, LARGE_SPEC_C2R,
  LARGE_SPAT_ADMM, LARGE_SPAT_IMAGE, LARGE_SPAT_R2C, LARGE_SPAT_C2R
};
// n: images (ADMM, IMAGE modes); npairs: filter pairs (ADMM) or plane pairs (R2C, C2R).
// An iteration is SPEC_DOT (skipped on a batch's first iteration), SPEC_Z,
// SPAT_ADMM; a sample spectrum SPAT_IMAGE then
// SPEC_IMAGE; r2c SPAT_R2C then SPEC_R2C; c2r SPEC_C2R then SPAT_C2R.
cudaError_t launch_large(int N, int what, const CodeIter &it, const ImgBatch &b, const LargeIO &io,
                         int n, int npairs, const float2 *tw, cudaStream_t s);
// Default columns per spatial CTA (the serving residual partials assume it).
int large_default_cb(int N);
bool large_cb_ok(int N, int cb);
// Stages of filter pairs per spectral CTA row (sizes CodeIter::part).
int large_stages(int N, int npairs);
// Residual partial sums per slot written by SPAT_ADMM in serving mode.
int large_resid_groups(int N, int npairs);

// Dictionary step.
struct FoldArgs {
  int K, F, B, first;
  double alpha, beta, w, rho_eff;
  float2 *A;            // [F][K(K+1)/2] history, packed lower, FP32
  float2 *b;            // [K][F]
  const float2 *Zp;     // [B][K][F]
  const float2 *xh;     // [B][F]
  float2 *L;            // [F][stride] X = L^-1 of the double-float Cholesky factor, FP32 (K > 128: L)
  float2 *g;            // [K][F]  y = L^-1 (w b)
  int *err;
  // prefolded = 1: A (+ Alo when not null) and b (+ blo when not null) already
  // hold the new means (tensor-core fold); the kernel only factors.
  int prefolded;
  float2 *Alo;          // [F][stride] compensation word of A (precision > 0)
  // dfold = 1 (history precision 3): products and running means in
  // double-float, A + Alo and b + blo kept as FP32 pairs.
  int dfold;
  float2 *blo;          // [K][F] compensation word of b (precision 3)
  // Band contexts: frequencies p0 .. p0 + nF - 1 (nF = 0: all F); A, Alo and
  // L hold these frequencies only; Zp and xh have row stride zF (0: F) and
  // start at frequency zp0.
  int p0, nF, zF, zp0;
};
cudaError_t launch_fold_factor(const FoldArgs &a, int threads, cudaStream_t s);

// Tensor-core history fold (history_tc.cu): A, Alo <- compensated
// alpha (A + Alo) + beta sum_i conj(z_i) z_i^T with BF16 operands (terms = 1)
// or split BF16 hi + lo (terms = 3) and FP32 accumulation; b in FP32.
struct GramArgs {
  int K, F, B, first, terms, SC;
  int dry;                  // 1: compute the sums but store nothing (timing runs)
  float alpha, beta, keep;  // keep = 1 - alpha = B beta
  const float2 *Zp;         // [B][K][F]
  const float2 *xh;         // [B][F]
  float2 *A, *Alo;          // [F][stride]
  float2 *b;                // [K][F]
  int *err;
  unsigned wait_polls;      // polls of the MMA-completion wait before it reports ERR_TIMEOUT
};
int gram_chunk(int K, int B, int terms);

// Recursion variant of the history (dict_sm.cu, eq. (C_update)).
struct SmArgs {
  int K, F, B, n;       // pending samples B folded after n earlier ones
  double r;             // ridge of the first sample: rho (rho P under the paper's convention)
  float2 rinv;          // 1 / r as a double-float pair
  float alpha, beta;    // running mean of b: n/(n+B), 1/(n+B)
  const float2 *Zp;     // [B][K][F]
  const float2 *xh;     // [B][F]
  float4 *C;            // [F][stride] C = (A + (r/t) I)^-1, packed lower, double-float
                        // (re hi, im hi, re lo, im lo)
  float2 *b;            // [K][F]
};
cudaError_t launch_sm_fold(const SmArgs &a, cudaStream_t s);
// r is the penalty matching C's ridge; ths != 1 first rescales theta^ in place
// (the scaled dual carried across a change of penalty).
cudaError_t launch_dstep_sm(int K, int F, double r, double ths, const float4 *Cf, const float2 *b,
                            const float2 *Vh, float2 *th, float2 *Dcur, float2 *E, cudaStream_t s);

// K > 128 (dict_big.cu): FP32 fold into A, b; blocked double-float Cholesky of
// w (A + Alo) + rho I storing L (FP32, in FoldArgs::L) and y = L^-1 (w b);
// D-step by substitution with L.
cudaError_t launch_fold_big(const FoldArgs &a, cudaStream_t s);
size_t factor_big_workspace(int K, int ctas);
cudaError_t launch_factor_big(const FoldArgs &a, double2 *work, int ctas, cudaStream_t s);
cudaError_t launch_dstep_big(int K, int F, float rho_eff, const float2 *L, const float2 *yb, const float2 *Vh,
                             const float2 *th, float2 *Dcur, float2 *E, cudaStream_t s);
cudaError_t launch_gram_fold(const GramArgs &a, cudaStream_t s);
// d = X^H (y + rho X (v^ - theta^)) with X = L^-1, y = L^-1 (w b).
// p0, nF: the frequencies solved (a band context; X holds them only); nF = 0: all.
cudaError_t launch_dstep(int K, int F, float rho_eff, const float2 *X, const float2 *yb,
                         const float2 *Vh, const float2 *th, float2 *Dcur, float2 *E,
                         cudaStream_t s, int p0 = 0, int nF = 0);
// Rows k1 in [k1_lo, k1_hi) (k1_hi = 0: all N; an even count).
cudaError_t launch_vstep_cols(int K, int N, int M, const float2 *E, const float2 *tw, float2 *Y,
                              cudaStream_t s, int k1_lo = 0, int k1_hi = 0);
// Size classes that take part in one V-step (reading R16).
constexpr int kMaxClasses = 12;
struct AlphaClasses {
  int project;                      // 1: Proposition 2 projection; 0: the mean crop as is
  int C;                            // active classes
  int N[kMaxClasses];               // FFT side of each
  const float2 *Y[kMaxClasses];     // [K][M][N/2+1] pruned inverse DFT along k1
  const float2 *tw[kMaxClasses];    // twiddles of each size
};
// Proposition 2 on the mean over classes of the support crops: writes V
// (ac.project = 0: the mean crop itself, for the literal return of Algorithm 2).
cudaError_t launch_vstep_project(int K, int M, const AlphaClasses &ac, float *V, cudaStream_t s);
// Partial DFT Tm [K][M][N/2+1] of the filters V for one class size.
cudaError_t launch_vstep_partial_dft(int K, int N, int M, const float *V, const float2 *tw, float2 *Tm,
                                     cudaStream_t s);
// V^ = F(pad V) from Tm; mode 0 also theta^ += D~ - V^.
// The dual is updated on frequencies [p0, p1) only (p1 = 0: all).
cudaError_t launch_vstep_spectrum(int mode, int K, int N, int M, const float2 *Tm, const float2 *tw,
                                  float2 *Vh, float2 *th, const float2 *Dcur, cudaStream_t s, int p0 = 0,
                                  int p1 = 0);
// Proposition 2 on the support sums alpha [K][M][M] (writes V).
cudaError_t launch_project_alpha(int K, int M, const float *alpha, float *V, cudaStream_t s);
cudaError_t launch_dict_norms(int K, int F, const float2 *Dh, float *dn, cudaStream_t s);

// Objective of one sample: out = 1/2 ||x - sum_k D_k (*) U_k||^2 + lam ||U||_1
// from its spectrum xh, the code spectra Uh [K][F] and the codes u [K][N][N].
// `partial` holds objective_partials(N) doubles of scratch.
constexpr int kObjL1Blocks = 256;
int objective_partials(int N);
cudaError_t launch_objective(int K, int N, double lam, const float2 *Dh, const float2 *xh,
                             const float2 *Uh, const float *u, double *partial, double *out,
                             cudaStream_t s);
// ||a - b|| / ||a|| over count floats (FP64, fixed order); partial holds
// 2 kObjL1Blocks doubles.
cudaError_t launch_rel_diff(const float *a, const float *b, size_t count, double *partial, double *out,
                            cudaStream_t s);

// Persistent coder (persist.cu): all Jz code-ADMM iterations of up to
// kMaxCallImages images of FFT sizes 64, 128, 256 and 512 in one cooperative
// launch.  Per iteration three intervals of units separated by a grid
// barrier: (A) the residual r of the Z~-step (N <= 128) and the partial sums
// D^T w^ (N >= 256, not on the first iteration); (B) the plane iteration
// (N <= 128) and the row inverse of conj(d) r (N >= 256); (C) the spatial
// column step (N >= 256).  Every unit is the body of the corresponding
// per-iteration kernel, so the results are those of the launches it replaces.
constexpr int kMaxPersistClasses = 4;
constexpr int kPersistThreads = 256;
struct PersistClass {
  int N;           // FFT side (64, 128, 256 or 512)
  int n0, n;       // images n0 .. n0 + n - 1 of PersistArgs::b
  int S;           // N >= 256: stages of filter pairs of the spectral units
  int cb;          // N >= 256: columns per spatial unit (8 or 16)
  CodeIter it[3];  // the class's workspaces, for the first, a middle and the last iteration
  LargeIO io;      // N >= 256: the pair tiles
  const float2 *tw;
};
struct PersistArgs {
  ImgBatch b;
  int ncls, Jz, K;
  PersistClass c[kMaxPersistClasses];
  unsigned *bar;   // [2] arrivals and generation of the grid barrier, zero at launch
  int *err;        // device error word: ERR_TIMEOUT when a barrier wait gave up
  unsigned polls;  // polls of one barrier wait
};
bool persist_size_ok(int N);
size_t persist_smem_bytes(const PersistArgs &a);
// CTAs of one cooperative launch with `smem` bytes of dynamic shared memory
// (all co-resident), or a negative CUDA error.
int persist_grid(size_t smem);
cudaError_t launch_persist(const PersistArgs &a, int grid, size_t smem, cudaStream_t s);

// PSNR of Sec. IV from the objective terms of n samples (terms [n][3], the
// squared residual norm at [3 i + 1]).
constexpr int kMaxPsnr = 64;
struct PsnrArgs {
  int n;
  double peak;
  int P[kMaxPsnr];  // pixel count of each sample's padded domain
};
cudaError_t launch_psnr(const double *terms, const PsnrArgs &a, double *out, cudaStream_t s);
// Filters in ascending order of their sample variance (K <= kMaxOrderK).
constexpr int kMaxOrderK = 256;
cudaError_t launch_filter_order(int K, int M, const float *V, int *order, cudaStream_t s);

}  // namespace ocsc
