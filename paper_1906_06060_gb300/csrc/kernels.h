// Host-side launchers of the libhotrg kernels. All launch on the given stream and return
// immediately; errors surface through cudaGetLastError() and the device status word.
#pragma once
#include "common.cuh"

namespace hotrg {

// Number of kernels the launchers below have enqueued in this process (diagnostics: lets a
// caller count the library's launches inside a timed region).
void count_launches(int n);
long long launches_total();

// ---- kernels_tensor.cu --------------------------------------------------------------------
// T^(0) (Sec. 2) for `batch` instances: T + i*stride gets beta[i], h[i] (device arrays). With
// spin_insertion, the impure tensor S^(0) (the summand carries the spin s).
void launch_init_tensor(double* T, long long inst_stride, int batch, int d, const double* beta,
                        const double* h, cudaStream_t s, int spin_insertion = 0);
// *dstep += 1 (device-side step counter read by the kernels below, so that a captured step
// can be replayed for any step number).
void launch_step_advance(int* dstep, cudaStream_t s);
// c = ||x||_F (deterministic), lnc_log[n] = ln c, L += 2^-n ln c with n = *dstep; status on a bad
// norm.
void launch_norm_log(const double* x, long long n, double* partial, double* c_out,
                     double* lnc_log, double* L, const int* dstep, int* status, cudaStream_t s);
// Tangents of the flow (fixed isometries). dT = d T^(0) / d beta (which = 0) or d / d h (which = 1).
void launch_init_tangent(double* dT, long long inst_stride, int batch, int d, const double* beta, const double* h,
                         int which, cudaStream_t s);
// For an unnormalised tensor T with norm *c and tangent D = D1 + D2 (D2 may be null):
// dlnc = <T, D> / c^2, dL += 2^-n dlnc (n = *dstep), dTn = (D - dlnc T) / c (tangent of T / c).
void launch_tangent_norm(const double* T, const double* D1, const double* D2, double* dTn, long long n,
                         const double* c, double* partial, double* dlnc, double* dL, const int* dstep,
                         cudaStream_t s);
// out[i] = dL[i] + 2^-n Tr dT_i / Tr T_i for every instance.
void launch_trace_tangent(const double* T, const double* dT, long long t_stride, int batch, long long P,
                          const double* dL, const int* dstep, double* out, cudaStream_t s);
// out[i] = Tr S_i / Tr T_i (Eqs. (energy), (spin)) for every instance.
void launch_trace_ratio(const double* S, const double* T, long long t_stride, int batch, long long P, double* out,
                        cudaStream_t s);
// *out = max |x| over a rows x cols array with row stride ld (upper bound as a float; the bits
// of that non-negative float are written, after zeroing *out on the stream).
template <class T>
void launch_absmax(const T* x, long long rows, long long cols, long long ld, unsigned* out, cudaStream_t s);
// dst = src / *c
void launch_scale(const double* src, double* dst, long long n, const double* c, cudaStream_t s);
// Tr T (Eq. (tTr)) and ln Z/N = L + 2^-n ln Tr (n = *dstep); X^(n) along `axis` (Eq. (x)).
// One CTA per instance: T + i*t_stride, L + i, out3 + 3 i.
void launch_trace_x(const double* T, long long t_stride, int batch, Geom g, int axis, const double* L,
                    const int* dstep, double* out3, cudaStream_t s);
// out[..u_b=j..] = sum_i U[kk][i][j] in[..u_b=i..] on unprimed leg b (U: [chi][Db][Db] fp64);
// with in2, plus the same product of in2 with U2. With amax, *amax = max |out| (the bits of a
// non-negative float, as launch_absmax writes them).
template <class Tin, class Tout>
void launch_mode_unprimed(const Tin* in, Tout* out, Geom g, int b, const double* U, int kk,
                          cudaStream_t s, const Tin* in2 = nullptr, const double* U2 = nullptr,
                          unsigned* amax = nullptr);
// Tt[p][u] = T[u][p] (P x P), converted to Tout.
template <class Tout>
void launch_transpose(const double* T, Tout* Tt, long long P, cudaStream_t s);
// B operand, K-major: Bt[(j*P + n)][k] = sum_x U3[j][k_c3][x] Tt[n][k | c3 := x], j < chi3.
// c3 < 0: Bt = Tt. Mixed: 2 or 3 bf16 planes; FP64: one double plane. With Tt2 (c3 >= 0), plus
// the same sum over Tt2 with U3b.
template <class Tin, class Tout>
void launch_build_bt(const Tin* Tt, const Planes<Tout>& out, long long ld, Geom g, int c3,
                     const double* U3, int chi3, cudaStream_t s, const Tin* Tt2 = nullptr,
                     const double* U3b = nullptr);
// A operand, K-major: Y[m][k] = X[u = (k_b, m_a)][p = (m_b, k_a)] for a step along `a`.
template <class Tin, class Tout>
void launch_build_y(const Tin* X, const Planes<Tout>& out, long long ld, Geom g, int a,
                    cudaStream_t s);
// Generic pair contraction / strided copy (see View): out[o] = sum_{i,j} U[k'][i][j] in[...].
template <class Tin, class Tout>
void launch_pair_contract(const Tin* in, Tout* out, const View& v, int kaxis, int Di, int Dj,
                          long long si, long long sj, const double* U, int chi, long long in_base,
                          long long out_base, cudaStream_t s);
// Same contraction with one thread per index of `rest` (the output axes without k'), computing
// all chi outputs out[o + k' sk]; every input element is read once. With in2 (same layout), plus
// the same contraction of in2 with U2.
template <class Tin, class Tout>
void launch_pair_contract_all(const Tin* in, Tout* out, const View& rest, int Di, int Dj, long long si,
                              long long sj, long long sk, const double* U, int chi, long long in_base,
                              long long out_base, cudaStream_t s, const Tin* in2 = nullptr,
                              const double* U2 = nullptr);
// Raise the dynamic shared-memory limit of the two-input kernels (call once, before any capture).
void prepare_kernel_attributes();

// ---- gram.cu -------------------------------------------------------------------------------
// Q[(i,al)][(i~,al~)] = sum over all other legs of T[..i..al..] T[..i~..al~..]; legs l1, l2 are
// positions 0..2d-1 in the natural layout. partial: nsplit * nr^2 doubles scratch.
// Instance i reads T + i*t_stride and writes Q + i*q_stride.
size_t gram_partial_doubles(int nr_max, int batch);  // scratch for `partial`
// With TA: rows from TA (same layout and strides as T), columns from T: Q(TA, T).
// With z2ev ([batch][kMaxD] even-value counts, values ordered even-parity first), the zero-field
// block structure is used: a quarter of the work (see gram.cu).
void launch_half_gram(const double* T, long long t_stride, int batch, Geom g, int l1, int l2,
                      double* partial, double* Q, long long q_stride, cudaStream_t s,
                      const double* TA = nullptr, const int* z2ev = nullptr);
// G[(b1 b2)][(b1~ b2~)] = sum_{al,al~} Q1[(b1,al)][(b1~,al~)] Q2[(b2,al)][(b2~,al~)] per instance
void launch_gram_combine(const double* Q1, const double* Q2, long long q_stride, int batch, int Db,
                         int Da, double* G, long long g_stride, cudaStream_t s);
// dG = sum (H1 + H1^T) Q2 + Q1 (H2 + H2^T), H = Q(dT, T): the tangent of the Gram matrix.
void launch_gram_combine_tangent(const double* Q1, const double* Q2, const double* H1, const double* H2,
                                 long long q_stride, int batch, int Db, int Da, double* dG, long long g_stride,
                                 cudaStream_t s);

// ---- eig.cu --------------------------------------------------------------------------------
// Where the sorted eigenvalues go: base + i*inst_stride + (*step - 1)*step_stride for instance
// i (nothing is written when the step is outside 1..max_steps).
struct EigOut {
  double* base;
  long long inst_stride, step_stride;
  const int* step;
  int max_steps;
};
// Symmetric eigendecomposition of G (n x n, n <= 256) by cyclic Jacobi, one CTA per instance;
// eigenvalues sorted descending, the leading chi eigenvectors, sign-fixed, into U[k][0..n).
// work: batch * 2*n*n doubles. Sets ST_NOCONV on the sweep limit.
// Several axes in one launch (blockIdx.y = axis): per axis its Gram matrices G (+ instance x
// g_stride), size n, kept count chi, the axis and Db for the zero-field ordering, the eigenvalue
// log base (+ instance x out.inst_stride + (step - 1) x out.step_stride), U (+ instance x u_stride)
// and a work area of batch x 2 n^2 doubles.
struct EigAxis {
  const double* G;
  int n, chi, z2_axis, Db;
  double* evals;
  double* U;
  double* work;
};
struct EigAxes {
  int nt;
  int max_sweeps;  // sweep limit (ST_NOCONV when reached)
  long long g_stride, u_stride;
  EigOut out;  // strides, step counter and step limit (its base is unused here)
  EigAxis ax[kMaxD];
};
void launch_eig_axes(const EigAxes& ea, int batch, int* status, cudaStream_t s, const int* z2_ev = nullptr,
                     int* z2_ev_new = nullptr);
// z2_ev (non-null): zero-field flow: [batch][kMaxD] even counts of the legs; the kept vectors of
// axis z2_axis (Db x Db fused index) are written even-parity first (each group in descending
// eigenvalue order), z2_ev_new[i][z2_axis] = number of even ones; a vector that is not
// parity-pure sets ST_Z2.
void launch_eig(const double* G, long long g_stride, int batch, int n, int chi, const EigOut& o,
                double* U, long long u_stride, double* work, int* status, cudaStream_t s,
                const int* z2_ev = nullptr, int* z2_ev_new = nullptr, int z2_axis = 0, int Db = 0,
                int max_sweeps = 40);
// First-order change of the kept eigenvectors for a change dG of G, from the eigensystem that
// launch_eig left in `work` (call before the next launch_eig reuses it):
//   dU_k = sign_k sum_{j >= chi} V_j (V_j^T dG V_k) / (lambda_k - lambda_j),  k < chi,
// with sign_k the sign convention applied to U_k. Rotations inside the kept space are left out:
// they are a gauge change of the new bond under which the flow's ln Z is invariant. A cut with
// lambda_k == lambda_j (k < chi <= j) has no derivative: dU gets NaN.
void launch_eig_tangent(const double* work, const double* U, long long u_stride, const double* dG,
                        long long g_stride, int batch, int n, int chi, double* dU, cudaStream_t s);
void prepare_eig_attributes();  // shared-memory limit of the tangent kernel (once, before any capture)

// ---- gemm_simt.cu --------------------------------------------------------------------------
// C[m][n] = sum_k A[m][k] Bt[n][k] in FP64 (CUDA cores).
// With blk (device memory, see GemmBlocks below), only the listed output blocks are computed, each
// over its own k range; M, N are then the extents of A's and Bt's rows.
// With bat (a batched launch, see GemmBatch), `batch` such products, instance i at A + i a_inst,
// Bt + i b_inst, C + i c_inst with blocks blk[i].
struct GemmBlocks;
struct GemmBatch;
void launch_gemm_f64(const double* A, long long lda, const double* Bt, long long ldb, double* C,
                     long long ldc, long long M, long long N, long long K, cudaStream_t s,
                     const GemmBlocks* blk = nullptr, const GemmBatch* bat = nullptr);

// ---- gemm_tc.cu ----------------------------------------------------------------------------
// C[m][n] = sum over passes p of sum_k A_{a(p)}[m][k] Bt_{b(p)}[n][k], bf16 operand planes on
// tcgen05, FP32 accumulation in TMEM. npass = 1: (hi,hi); 3: + (hi,lo), (lo,hi) with 2 planes;
// 4: + (lo,lo); 6: (hi,hi), (hi,mid), (mid,hi), (hi,lo), (mid,mid), (lo,hi) with 3 planes.
// bk = 64 or 32: the k-block width (the accumulator restarts and is folded once per k-block);
// group_m: output tiles are visited in groups of group_m M-tiles (L2 reuse); fold_group: k-blocks
// per accumulator fold (at most ring stages - 1 when > 1).
// Returns 0 or a hotrg_status (tensor-map encode failure, bad alignment or sizes).
// Block-sparse form (blk != null, device memory read by the kernel at start): only the output
// blocks listed are computed. Block b: rows [m0, m0+mc) of A and C, rows [n0, n0+nc) of Bt
// (columns of C), k range [k0, k0+kc), where both operands must hold zeros from k0+kc up to the
// next multiple of bk. M, N, K are then the operands' extents (rows of A, rows of Bt, row
// length) and bound every copy; nothing outside the blocks is written.
struct GemmBlocks {
  int nb;
  int m0[2], mc[2], n0[2], nc[2], k0[2], kc[2];
};
// Largest number of instances one batched GEMM launch takes (its tile prefix lives in shared memory).
constexpr int kMaxGemmBatch = 256;
// Batched launch (up to kMaxGemmBatch instances): `batch` independent products of the same shape in one
// persistent launch; plane k of instance i starts at A.p[k] + i a_inst (elements, multiple of 8,
// at least M lda), likewise B (b_inst) and C (c_inst); with blk, instance i's blocks are blk[i];
// fp16 scale bounds at A.amax + i amax_inst and B.amax + i amax_inst.
struct GemmBatch {
  int batch = 1;
  long long a_inst = 0, b_inst = 0, c_inst = 0;
  int amax_inst = 0;
};
int launch_gemm_split(const Planes<__nv_bfloat16>& A, long long lda, const Planes<__nv_bfloat16>& B,
                      long long ldb, float* C, long long ldc, long long M, long long N, long long K,
                      int npass, int* status, double timeout_s, cudaStream_t s, int bk = 64,
                      int group_m = 16, int fold_group = 1, const GemmBlocks* blk = nullptr,
                      const GemmBatch* bat = nullptr, bool stall = false, int cta_group = 0);
// stall (test of the bounded waits): the kernel's producer issues no copies, so every CTA's first
// wait for a stage runs out after timeout_s and the launch ends with ST_TIMEOUT in *status.
// cta_group: 1 = one CTA per 128 x 256 output tile, 2 = a CTA pair (cluster of two) per 256 x 256
// tile with tcgen05 cta_group::2 MMAs, each CTA staging half the B rows; 0 = kDefaultCtaGroup.
constexpr int kDefaultCtaGroup = 1;
// Largest fold group the kernel variant for (npass, bk) accepts.
int max_fold_group(int npass, int bk);
void launch_split_rows(const float* X, long long ldx, long long rows, long long cols,
                       const Planes<__nv_bfloat16>& out, long long ld, cudaStream_t s);

// ---- z2.cu ---------------------------------------------------------------------------------
// Parity-blocked layout of the zero-field squeeze's operands for one instance (see z2.cu).
struct Z2Layout {
  int d;
  int D[kMaxD], e[kMaxD];      // bond dimensions and even-value counts of the current legs
  int ncls[2];                 // natural P-indices of even / odd total parity
  int kstart[2];               // operand column where each parity class starts (64-aligned)
  int patoff[16];              // rank of the first index of each leg-parity pattern
  int bs[16][kMaxD];           // row-major strides inside each pattern's box
  int chi3, e3;                // the new c3 index: range and number of even values
  int goff[2];                 // first output column of each group (parity of (j, n))
  int jstart[2][kMaxBond + 1]; // offset of new index j inside each group
};
// Layouts of every instance (ev, ev_new: [batch][kMaxD] even counts before / after the step).
void launch_z2_layout(const int* ev, const int* ev_new, int batch, Geom g, int c3, int chi3, Z2Layout* out,
                      cudaStream_t s);
// rank_tab[P], kcol_tab[P], colpos_tab[chi3 * P] of one instance's layout.
void launch_z2_tables(const Z2Layout* L, long long P, int chi3, int* rank_tab, int* kcol_tab, int* colpos_tab,
                      cudaStream_t s);
// The chunk's parity (fixed new indices k0 of axis b0, k1 of b1; nfix of them) and its two GEMM
// blocks; flops[0] += their 2 M N K, flops[1] += that times npass.
void launch_z2_chunk(const Z2Layout* L, const int* ev_new, int nfix, int b0, int k0, int b1, int k1, long long ldO,
                     GemmBlocks* blk, int* pi, double* flops, int npass, cudaStream_t s);
// ev[i][b] = ev_new[i][b] for the axes b in trans_mask (end of a step).
void launch_z2_advance(int* ev, const int* ev_new, int batch, unsigned trans_mask, cudaStream_t s);
template <class Tin, class Tout>
void launch_build_y_z2(const Tin* X, const Planes<Tout>& out, long long ld, Geom g, int a,
                       const int* rank_tab, const int* kcol_tab, const Z2Layout* L, const int* pi, cudaStream_t s);
template <class Tin, class Tout>
void launch_build_bt_z2(const Tin* Tt, const Planes<Tout>& out, long long ld, Geom g, int c3, const double* U3,
                        int chi3, const int* rank_tab, const int* kcol_tab, const int* colpos_tab, const Z2Layout* L,
                        cudaStream_t s);
// First epilogue contraction (over slot t0, Dt x Dt -> chi) from the parity-blocked GEMM output;
// rest / sk / out_base as for launch_pair_contract_all.
template <class Tin, class Tout>
void launch_epi_z2(const Tin* O, long long ldO, Tout* out, const View& rest, long long sk, long long out_base,
                   int t0, int Dt, const double* U, int chi, const Z2Layout* L, const int* pi, cudaStream_t s);

}  // namespace hotrg
