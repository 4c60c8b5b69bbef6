/*
 * hotrg.h - C ABI of the GB300 HOTRG coarse-graining library (libhotrg.so).
 *
 * The library computes the higher-order tensor renormalisation group flow of the
 * d-dimensional Ising model (d = 1..4) as used in arXiv:1906.06060:
 *   Sec. 2, Eq. (pf)        partition function Z_N = sum_s prod_<ij> e^{b s_i s_j} prod_i e^{b h s_i}
 *   Sec. 2, after Eq. (pf)  initial site tensor T^(0) = sum_s V_s prod_{2d legs} W[s, leg], W = U sqrt(L)
 *   Sec. 2, Eqs. (SS),(ST) with S -> T   one coarse-graining step (isometries + squeeze)
 *   Sec. 2, Eq. (tTr)       periodic trace of the coarse-grained tensor
 *   Sec. 3, Eqs. (matA),(x) the degeneracy indicator X^(n)
 * Normalisation (not written in the paper): c_n = ||T^(n)||_F, T <- T / c_n and
 *   ln Z_N / N = sum_{k=0}^{n} 2^{-k} ln c_k + 2^{-n} ln Tr T^(n),   N = 2^n sites.
 *
 * Tensor layout used everywhere in this ABI ("natural layout"): a site tensor of a
 * d-dimensional lattice is a row-major array T[u_0..u_{d-1}, p_0..p_{d-1}], where u_b is the
 * leg towards the lower neighbour along axis b (x=0, y=1, z=2, t=3) and p_b the leg towards the
 * upper one. Both legs of axis b have the same bond dimension D_b. P = prod_b D_b.
 *
 * Conventions
 *  - Every int-returning function returns 0 (HOTRG_OK) or a negative hotrg_status; none aborts.
 *  - A context's first error is sticky: later calls on it return the same code.
 *  - Calls are ordered on the context's CUDA stream. hotrg_step only enqueues work; query
 *    functions (free energy, observables, spectra, get_tensor) synchronise that stream.
 *  - The library never allocates device memory: the caller passes one device workspace of at
 *    least hotrg_workspace_size() bytes (256-byte aligned) and keeps it alive until
 *    hotrg_destroy. Host pointers passed in are only accessed during the call.
 *  - One context must not be used from two host threads at once.
 */
#ifndef HOTRG_H_
#define HOTRG_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum hotrg_status {
  HOTRG_OK = 0,
  HOTRG_EINVAL = -1,   /* bad argument: d, beta, Dcut, axis, sizes, null pointer */
  HOTRG_ENOMEM = -2,   /* workspace smaller than hotrg_workspace_size() */
  HOTRG_ENUMERIC = -3, /* NaN/Inf or zero norm, or Tr T <= 0 */
  HOTRG_ENOCONV = -4,  /* eigensolver did not converge within its sweep limit */
  HOTRG_ETIMEOUT = -5, /* a bounded device-side wait gave up */
  HOTRG_EDEVICE = -6,  /* CUDA runtime/driver error, or no sm_103 device */
  HOTRG_ESTATE = -7,   /* call not valid in the context's state (e.g. step log full) */
  HOTRG_ENOTSUP = -8   /* valid request that this library does not provide */
} hotrg_status;

typedef enum hotrg_precision {
  HOTRG_FP64 = 0,   /* every contraction in FP64 on the CUDA cores */
  HOTRG_BF16X3 = 1, /* squeeze GEMM on tcgen05 tensor cores with split operands x = hi + lo
                       (bf16 each); products hi*hi + hi*lo + lo*hi accumulate in FP32 (TMEM):
                       O(2^-16) relative error per product. Gram matrices, eigensolver, norms
                       and ln sums stay FP64; other intermediates are FP32. */
  HOTRG_BF16X6 = 2, /* as BF16X3 with three planes x = hi + mid + lo and the six products
                       hh, hm, mh, hl, mm, lh: O(2^-24) per product, twice the tensor work */
  HOTRG_BF16X4 = 3, /* two planes and all four products (adds lo*lo): no systematic
                       truncation of the product, O(2^-17) unbiased per product */
  HOTRG_FP16X3 = 4, /* as BF16X3 with fp16 planes: each operand is first scaled by an exact power
                       of two 2^e (from its largest magnitude, measured on the device, so that it
                       lies below 2^15), then split x 2^e = hi + lo in fp16 (11 significant bits
                       each); hi*hi + hi*lo + lo*hi accumulate in FP32 and the result is scaled
                       back by 2^-(eA + eB): O(2^-22) relative error per product (entries more than
                       2^-18 below their operand's largest lose the lo part's low bits, an absolute
                       error below 2^-39 of that largest), at the tensor cost of BF16X3. With
                       opts.derivatives the squeezes that carry tangents use bf16 planes (BF16X3) */
  HOTRG_FP16X4 = 5  /* FP16X3 plus lo*lo: no systematic truncation of the product */
} hotrg_precision;

typedef struct hotrg_opts {
  int precision;          /* hotrg_precision (default HOTRG_FP64) */
  int fp64_steps;         /* in the split modes the first fp64_steps steps run in FP64 (default 2) */
  int x6_steps;           /* in the two-plane split modes (BF16X3/X4, FP16X3/X4), steps
                             fp64_steps+1 .. x6_steps use the 6-pass BF16X6 GEMM (the early steps
                             weigh 2^-n in ln Z/N; default 0) */
  int batch;              /* independent (beta, h) instances in the context (default 1) */
  const double *beta;     /* [batch] host array; NULL: all instances use the beta argument */
  const double *h;        /* [batch] host array; NULL: all instances use the h argument */
  void *stream;           /* cudaStream_t for all work; NULL = legacy default stream */
  void *workspace;        /* device pointer, >= hotrg_workspace_size() bytes, 256-B aligned */
  size_t workspace_bytes;
  int max_steps;          /* capacity of the per-step logs, 1..64 (default 64) */
  int kblock;             /* split modes: K width of a pipeline stage, 32 or 64 (0 = 64) */
  int fold_group;         /* split modes: stages per accumulator fold, 1 or 2 (0 = 1): the tensor
                             cores' FP32 accumulator restarts every fold_group * kblock K */
  int derivatives;        /* also propagate d/d beta and d/d h of the flow (forward-mode tangents;
                             each step adds two squeeze GEMMs over a doubled k range):
                             0 none; 1 with the isometries of every step held fixed;
                             2 exact derivative of the truncated flow, differentiating the
                               isometries through the Gram eigendecomposition (first-order
                               eigenvector perturbation; NaN where a cut splits a degenerate
                               eigenvalue, where no derivative exists). EINVAL otherwise. */
  int impurities;         /* 1: also coarse-grain the impure tensors of Sec. 2 (Eqs. (impTN),
                             (SS), (ST)) with the pure flow's isometries and report the
                             estimates of Eqs. (energy) and (spin): two extra squeezes per step */
  int z2;                 /* 1: zero-field block-sparse squeeze: at h = 0 every tensor entry whose
                             legs' spin-flip parities add up to odd vanishes, and the squeeze
                             (split-precision and FP64 steps alike) computes only the two
                             nonzero GEMM blocks per chunk (a quarter of the dense flops); bond
                             indices are then ordered even-parity first. Needs h = 0 for every
                             instance, d >= 2, no derivatives and no impurities (EINVAL
                             otherwise); set_tensor turns it off, set_tensor_z2 keeps it. */
  int graphs;             /* 1: capture a steady-state step (bond dimensions unchanged) once per
                             axis as a CUDA graph and replay it (default 1; off while timing and
                             on the legacy default stream, which cannot be captured) */
  double wait_timeout_s;  /* bound on any device-side spin wait, seconds (default 4) */
  int max_sweeps;         /* Jacobi sweep limit of the eigensolver (default 40; 0 = default, at most
                             1000); a Gram matrix not diagonalised within it sets HOTRG_ENOCONV */
  int group;              /* instances squeezed together: the squeeze GEMM of a chunk is one persistent
                             launch over a group (its tile list spans the group's instances), and the
                             workspace holds that many copies of the per-step buffers. 1..256, capped
                             at batch; 0 (default) = 8; with derivatives or impurities always 1 */
  int cta_group;          /* split modes: CTAs per squeeze-GEMM output tile. 2 = a pair of CTAs (a
                             thread-block cluster of two SMs) per 256 x 256 tile, whose tcgen05
                             MMAs read A rows from both CTAs and half of the B rows from each;
                             1 = one CTA per 128 x 256 tile. Both give identical results. 0 =
                             default: 2 with opts.z2, else 1 (the faster at the Dcut = 10
                             shapes); the autotuner may change it. 1 or 2 fix it; EINVAL
                             otherwise */
} hotrg_opts;

typedef struct hotrg_obs {
  int steps;              /* coarse-graining steps done */
  int last_axis;          /* axis of the last step (-1 if none) */
  double lnz_per_site;    /* ln Z_N / N estimate after the last step, N = 2^steps */
  double last_ln_c;       /* ln c_n of the last step */
  double x_indicator;     /* X^(n) of Eq. (x) along the last axis (1 for steps == 0) */
  /* with opts.derivatives (NaN otherwise), derivatives of the ln Z_N / N estimate (isometries
   * held fixed, or differentiated, per opts.derivatives) and what they give
   * (H = -sum s s' - h sum s):
   *   d(lnZ/N)/d beta = -<H>/N = d <s s'> + h <s>,   d(lnZ/N)/d h = beta <s>   */
  double dlnz_dbeta;
  double dlnz_dh;
  double internal_energy; /* <H>/N = -d(lnZ/N)/d beta */
  double magnetization;   /* <s> = (1/beta) d(lnZ/N)/d h */
  /* with opts.impurities (NaN otherwise), the impure-tensor estimates Tr S^(n) / Tr T^(n):
   * <s_i s_j> for a nearest-neighbour pair along the first step's axis (Eq. (energy); NaN
   * before the first step) and <s_i> (Eq. (spin)) */
  double nn_correlation;
  double spin;
} hotrg_obs;

typedef struct hotrg_ctx hotrg_ctx;

/* Fill *o with the defaults listed in hotrg_opts. */
void hotrg_opts_default(hotrg_opts *o);

/* Bytes of device workspace for a context of dimension d (1..4) and bond cut Dcut (2..16) with
 * the given options (precision, batch and max_steps are read; NULL means defaults).
 * Errors: EINVAL for d or Dcut out of range, batch < 1, or bytes == NULL. */
int hotrg_workspace_size(int d, int Dcut, const hotrg_opts *opt, size_t *bytes);

/* Create a context (Sec. 2): builds T^(0) = sum_s V_s prod W[s, leg] for every instance on the
 * device, normalises it (c_0) and starts the ln Z accumulator at ln c_0.
 * beta > 0 and finite, h finite (per instance when opt->beta / opt->h are given).
 * *out receives a host object freed by hotrg_destroy; the workspace stays caller-owned.
 * Errors: EINVAL (d not in 1..4, Dcut not in 2..16, bad beta/h, batch < 1, opt NULL),
 * ENOMEM (workspace too small or misaligned), EDEVICE (no sm_103 device / CUDA error). */
int hotrg_init(hotrg_ctx **out, int d, double beta, double h, int Dcut, const hotrg_opts *opt);

/* One coarse-graining step along `axis` (0..d-1), or the next axis of the cycle t,z,y,x
 * (d-1 .. 0) when axis == -1 (Sec. 2, Eqs. (SS),(ST) with S -> T, for every instance):
 *   1. Gram matrices G_b of the two-site unfolding for each transverse axis b (FP64),
 *   2. symmetric eigendecomposition, keep chi_b = min(D_b^2, Dcut) leading eigenvectors,
 *      each sign-fixed so that its largest-magnitude component is positive,
 *   3. squeeze T' = U..U (T T) U..U (the O(Dcut^15) contraction),
 *   4. c_n = ||T'||_F, T <- T'/c_n, ln Z accumulator += 2^{-n} ln c_n.
 * Enqueues work on the stream and returns. Errors: EINVAL (axis), ESTATE (log full). */
int hotrg_step(hotrg_ctx *c, int axis);

/* ln Z_N / N = accumulator + 2^{-n} ln Tr T^(n) (Eq. (tTr)) and f = -(ln Z_N / N) / beta, one
 * value per instance written to the caller's host arrays (either may be NULL). Synchronises.
 * Errors: ENUMERIC (Tr T <= 0), and any sticky device error. */
int hotrg_free_energy(hotrg_ctx *c, double *lnz_per_site, double *f_per_site);

/* Observables of instance `instance` after the last step (see hotrg_obs). Synchronises. */
int hotrg_observables(hotrg_ctx *c, int instance, hotrg_obs *out);

/* Eigenvalues (descending, all D_b^2 of them) of the Gram matrix G_axis of step `step`
 * (1-based) of instance `instance`, copied to buf[0..cap). *n_out = number available (0 if
 * `axis` was the step's own axis). Synchronises. Errors: EINVAL (step/axis/instance). */
int hotrg_spectra(hotrg_ctx *c, int step, int axis, int instance, double *buf, int cap, int *n_out);

/* ln c_n of steps 0..steps of `instance` (n_out = steps + 1 values). Synchronises. */
int hotrg_ln_norms(hotrg_ctx *c, int instance, double *buf, int cap, int *n_out);

/* Current bond dimensions (d ints) and the normalised tensor of `instance` in natural layout
 * (P^2 doubles) copied to host memory; `host` may be NULL to query dims only. Synchronises.
 * Errors: EINVAL (cap < P^2 when host != NULL). */
int hotrg_get_tensor(hotrg_ctx *c, int instance, int *dims, double *host, size_t cap);

/* Replace the tensor of `instance` by a host array in natural layout with bond dimensions
 * dims[0..d) (each 1..Dcut). Used to coarse-grain arbitrary tensors. It does not normalise and
 * does not touch the ln Z accumulator; with opts.derivatives it zeroes the instance's tangents
 * (the supplied tensor does not depend on beta or h), with opts.impurities its impure tensors.
 * With opts.z2 it switches the context to the dense squeeze for all instances (the tensor's block
 * structure is unknown; hotrg_set_tensor_z2 keeps it). Errors: EINVAL (also when prod dims exceeds the
 * largest P of the workspace plan, i.e. of the states reachable from T^(0) within
 * opts.max_steps steps). */
int hotrg_set_tensor(hotrg_ctx *c, int instance, const int *dims, const double *host);

/* The same for a context created with opts.z2, keeping the block-sparse squeeze: the tensor
 * must have the zero-field block structure (Sec. 2's T^(0) at h = 0 and every coarse-grained
 * tensor of that flow), with the values of leg b ordered even-parity first and evens[b] of
 * them even (d ints, 0..dims[b]): every entry whose legs' parities add up to odd must be exactly
 * zero, which is checked on the host. The block-sparse squeeze applies again only once every
 * instance of the context holds such a tensor: one given a dense tensor by hotrg_set_tensor, and
 * every instance after a step taken with the dense squeeze, needs its own hotrg_set_tensor_z2
 * first (until then the context squeezes densely, which is correct for any tensor).
 * Errors: EINVAL (bad sizes, structure violated), ESTATE (context created without opts.z2).
 * Synchronises. */
int hotrg_set_tensor_z2(hotrg_ctx *c, int instance, const int *dims, const int *evens, const double *host);

/* Checkpoint: size of, save to and restore from a host buffer holding the full flow state
 * (tensors, dims, accumulators, step logs). load requires a context created with the same
 * d, Dcut, batch and precision. Synchronise. Errors: EINVAL (size/format mismatch). */
int hotrg_state_size(hotrg_ctx *c, size_t *bytes);
int hotrg_state_save(hotrg_ctx *c, void *host, size_t cap);
int hotrg_state_load(hotrg_ctx *c, const void *host, size_t size);

/* Phase timing, for benchmarks: after hotrg_timing_start, every phase the context enqueues is
 * bracketed by CUDA events on its stream; hotrg_timing_stop synchronises and returns the summed
 * event durations (ms) and work counters since the start. Timing adds two event records per
 * phase and per GEMM launch. */
typedef struct hotrg_timing {
  double ms_step;           /* whole steps */
  double ms_isometry;       /* Gram matrices and eigensolver */
  double ms_operands;       /* GEMM operand construction: transposes, mode products, splits */
  double ms_gemm;           /* squeeze GEMM launches */
  double ms_epilogue;       /* primed-side isometry contractions into the new tensor */
  double ms_norm;           /* norm, scale, trace, X^(n) */
  long long steps;          /* steps taken (per instance count: batch x steps in step_flops) */
  long long gemm_launches;  /* squeeze GEMM kernels launched */
  long long kernel_launches;/* all library kernels launched in this process since start */
  double gemm_flops;        /* algorithmic flops of those GEMMs, 2 M N K each */
  double gemm_tensor_flops; /* flops the tensor pipe executed (x 3 or x 6 split passes) */
  double step_flops;        /* algorithmic squeeze flops of the steps, 2 prod(chi_b) P^3; with
                               opts.z2, what the parity blocks compute (about a quarter) */
  double dense_step_flops;  /* 2 prod(chi_b) P^3 per step, also with opts.z2 */
} hotrg_timing;

int hotrg_timing_start(hotrg_ctx *c);
int hotrg_timing_stop(hotrg_ctx *c, hotrg_timing *out);

/* Autotuner of the squeeze GEMM's tile configuration: times the split-precision GEMM of the
 * last step's shape (M = P, N = chi P, K = P, on the operands that step left in the workspace;
 * with opts.z2 the two-block GEMM of the last chunk, on its block descriptor) for each candidate -
 * k-block 64 or 32 (unless opts.kblock fixed it; 32 only for 6 passes), one or two k-blocks per
 * accumulator fold at k-block 32, tile-raster groups of 4, 8, 16, 32 or 64 M-tiles, and CTA pairs or
 * single CTAs per output tile (unless opts.cta_group fixed it) - keeps the
 * fastest for the following steps and drops captured step graphs (tuned on a six-product GEMM, it
 * keeps the k-block of the two-plane steps). Call it after a steady-state split-precision step
 * (its operands must still be in the workspace). Synchronises.
 * Errors: ESTATE (no split-precision step yet), EDEVICE. */
typedef struct hotrg_tuning {
  int kblock;
  int group_m;
  int fold_group;
  double ms;  /* best GEMM time of the timed shape */
  int cta_group;
} hotrg_tuning;
int hotrg_autotune(hotrg_ctx *c, hotrg_tuning *out);

/* Release the context's host object. The workspace is not touched. NULL is a no-op. */
void hotrg_destroy(hotrg_ctx *c);

/* Static description of a status code. */
const char *hotrg_strerror(int code);

/* ---------------------------------------------------------------------------------------
 * Kernel-level entry point: the squeeze GEMM of the split-precision paths on its own (Sec. 2
 * cost statement: the O(Dcut^15) contraction is this GEMM), for tests and benchmarks.
 *   C[m][n] = sum_k A[m][k] * Bt[n][k],  m < M, n < N, k < K   (M >= 128, N >= 256, K >= 64)
 * A (M x lda floats, row-major) and Bt (N x ldb floats, row-major) are device FP32 arrays that
 * are split into bf16 planes in `scratch` (device, >= hotrg_gemm_scratch_bytes(M,N,K) bytes,
 * 256-B aligned) before the tcgen05 GEMM; C is device FP32 with leading dimension ldc.
 * npass: 1 = hi*hi only, 3 / 4 / 6 = BF16X3 / BF16X4 / BF16X6 products. kblock: 64 or 32, the K
 * width of a pipeline stage (0 = 64; the 6-pass GEMM always uses 32). fold_group: stages whose
 * products share one tensor-core accumulator before it is folded into FP32 registers with
 * round-to-nearest adds (0 = 1; larger values are clamped to what the kernel variant's ring
 * allows, at most 2). The launch uses one CTA per 128 x 256 output tile (the flow contexts can
 * also run CTA pairs: opts.cta_group).
 * Enqueued on `stream`; not synchronised. Errors: EINVAL (sizes, npass, kblock, alignment),
 * EDEVICE. */
size_t hotrg_gemm_scratch_bytes(long long M, long long N, long long K);
int hotrg_gemm_split(const float *A, long long lda, const float *Bt, long long ldb, float *C,
                     long long ldc, long long M, long long N, long long K, int npass, int kblock,
                     int fold_group, void *scratch, size_t scratch_bytes, void *stream);

/* The same GEMM for callers that cannot allocate device memory (the paper has no counterpart:
 * this is a service of the library). hotrg_gemm_split needs a scratch buffer from its caller;
 * some callers have none to give, e.g. a process whose device memory is already reserved in
 * full by another framework's pool, or a latency-critical loop that must not call cudaMalloc
 * (it may synchronise the device). This variant allocates nothing: the bf16 planes and the
 * status word live in a fixed device array inside the library (about 12 MiB, held on every GPU
 * where this entry point is used until the process exits).
 *   Sizes: M >= 128, N >= 256, K >= 64 (as hotrg_gemm_split) and
 *          (M + N) * round_up(K, 64) <= HOTRG_GEMM_NOALLOC_MAX_ELEMS (2^21), else HOTRG_EINVAL.
 *   Set-up: the first call on a device (made while it is current) looks up the array's device
 *   address.
 *   Capture: every call synchronises `stream` and reads the status word back to the host, so the
 *   entry point cannot be used inside a CUDA stream capture.
 *   Sharing: every call uses the same array. Calls whose GPU work overlaps (other streams or
 *   host threads) race on it. Returns the GEMM's status (0, HOTRG_ETIMEOUT if a pipeline wait
 *   gave up, HOTRG_EDEVICE). Other errors: EINVAL. */
#define HOTRG_GEMM_NOALLOC_MAX_ELEMS 2097152LL
int hotrg_gemm_split_noalloc(const float *A, long long lda, const float *Bt, long long ldb, float *C,
                             long long ldc, long long M, long long N, long long K, int npass,
                             void *stream);

/* The same GEMM with fp16 planes (the FP16X3 / FP16X4 products of the flow): A and Bt are each
 * scaled by an exact power of two 2^e from their largest magnitude (measured on the device) so
 * that they lie below 2^15, split x 2^e = hi + lo in fp16, multiplied on the tensor cores
 * (npass 1: hi*hi; 3: + hi*lo + lo*hi; 4: + lo*lo) with FP32 accumulation, and the result is
 * scaled back by 2^-(eA + eB). Per product O(2^-22) relative error, plus an absolute error below
 * 2^-39 x max|A| |b| (resp. max|Bt| |a|) for entries far below their operand's largest. Same
 * arguments, sizes, scratch (hotrg_gemm_scratch_bytes) and errors as hotrg_gemm_split. */
int hotrg_gemm_split_f16(const float *A, long long lda, const float *Bt, long long ldb, float *C,
                         long long ldc, long long M, long long N, long long K, int npass, int kblock,
                         int fold_group, void *scratch, size_t scratch_bytes, void *stream);

/* Failure-detection probe of the bounded device-side waits (the paper has no counterpart): two
 * launches of the tensor-core GEMM (BF16X3, one output tile: first on one CTA, then on a CTA pair)
 * whose copy-issuing thread issues no copies, so that the first wait for operand data can never
 * be satisfied. The waits give up after timeout_s (0 < timeout_s <= 10), each kernel records the
 * timeout, frees its tensor memory and returns; nothing is left in flight. `scratch` (device,
 * 256-B aligned) holds at least hotrg_gemm_wait_probe_bytes() bytes. Synchronises `stream`;
 * returns HOTRG_ETIMEOUT when both launches timed out as intended, else the first other status.
 * Other errors: EINVAL, EDEVICE. */
size_t hotrg_gemm_wait_probe_bytes(void);
int hotrg_gemm_wait_probe(double timeout_s, void *scratch, size_t scratch_bytes, void *stream);

/* Status of the last hotrg_gemm_split or hotrg_gemm_split_f16 call that used `scratch` (0 = ok,
 * HOTRG_ETIMEOUT if a pipeline wait of the GEMM kernel gave up). The word lives in the first bytes
 * of scratch and is cleared by each GEMM call. Synchronises `stream`. */
int hotrg_gemm_status(const void *scratch, void *stream);

/* Benchmark support (the paper has no counterpart): the GPU's FP64 FMA rate, measured with
 * independent FMA chains on every SM (8, 16 and 32 chains per thread, and a 4 x 4 outer-product
 * accumulation; each as two launches of `iters` loop iterations of which the second is timed with
 * CUDA events on `stream`; the best rate is returned). It is the roofline denominator of the FP64 squeeze, whose cost is
 * fixed by Sec. 2's O(Dcut^15) statement. `sink` is a device array of at least 8 x (SM count)
 * doubles that the kernel may write (in practice it writes nothing); *tflops receives the rate.
 * Synchronises `stream`. Errors: EINVAL (iters outside 1..2^32, null pointers), EDEVICE. */
int hotrg_bench_fp64_fma(long long iters, double *sink, double *tflops, void *stream);

#ifdef __cplusplus
}
#endif
#endif
