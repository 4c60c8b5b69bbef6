// Host side of libhotrg: context, workspace plan, the coarse-graining step sequence and the
// C ABI declared in include/hotrg.h (arXiv:1906.06060 Sec. 2).
//
// One step along axis a, for each instance (b runs over the transverse axes, c3 = the last one,
// "others" = the rest; T1 = T2 = T by translation invariance):
//   1. Q1_b, Q2_b, G_b (gram.cu), eigendecomposition -> U_b[k][b1 b2] (eig.cu)
//   2. B operand once per step:  Bt[(j, n)][k] = sum_x U_c3[j][k_c3][x] T[k | c3 := x][n]
//      (the c3 isometry of site 1's unprimed leg, moved onto site 2)
//   3. per chunk (k_o for the other transverse axes):
//        X = T with U_o[k_o] applied to u_o (mode products)
//        A operand Y[m][k] = X[u = (k_b.., m_a)][p = (m_b.., k_a)]       (m: site-1 primed legs)
//        O[m][(j, n)] = sum_k Y[m][k] Bt[(j, n)][k]                       (the O(D^15) GEMM)
//        T'[(k_o, j, m_a)][(k'_b, n_a)] = sum prod_b U_b[k'_b][m_b n_b] O[m][(j, n)]  (epilogue)
//   4. c_n = ||T'||_F, T <- T'/c_n, L += 2^-n ln c_n, Tr T, X^(n).
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "kernels.h"

using namespace hotrg;

struct hotrg_ctx {
  int d = 0, Dcut = 0, batch = 1, precision = HOTRG_FP64, fp64_steps = 2, x6_steps = 0, max_steps = 64;
  int kblock = 64;
  bool kblock_fixed = false;  // the caller fixed the k-block (else the autotuner may change it)
  int cta_group = 1;          // CTAs per squeeze-GEMM output tile (1 or 2)
  bool cta_group_fixed = false;
  int group_m = 16;
  int fold_group = 0;  // k-blocks per accumulator fold (0: one)
  // shape of the last split-precision GEMM launched (what the autotuner times)
  struct LastGemm {
    long long M = 0, N = 0, K = 0, ldk = 0;
    int npass = 0, nparts = 0, fmt = 0;
    float mult_b = 1.f;
    const GemmBlocks* blk = nullptr;  // block-sparse: the descriptor of the last chunk (slot 0)
  } last_gemm;
  double timeout_s = 4.0;
  int max_sweeps = 40;  // Jacobi sweep limit of the eigensolver
  cudaStream_t stream = nullptr;
  int dims[kMaxD] = {1, 1, 1, 1};
  int steps = 0, last_axis = -1, sticky = 0;
  int hist_dims[64][kMaxD] = {};  // bond dimensions before step n+1
  int hist_axis[64] = {};
  long long Pmax = 1;
  std::vector<double> beta, h;
  // device buffers carved from the workspace
  double *T = nullptr, *Tnext = nullptr, *dbeta = nullptr, *dh = nullptr, *L = nullptr;
  double *lnc_log = nullptr, *spec_log = nullptr, *out3 = nullptr, *cval = nullptr;
  double *norm_partial = nullptr, *gpartial = nullptr, *Q1 = nullptr, *Q2 = nullptr;
  double *G = nullptr, *U = nullptr, *ework = nullptr;
  long long ework_axis = 0;  // doubles of ework per axis (batch x 2 n_max^2)
  int* status = nullptr;
  int* dstep = nullptr;       // device-side step counter (steps done)
  unsigned* amax = nullptr;   // [0] max |B source|, [1] max |A source| of the fp16 split GEMM
  // tangents d/d beta (0) and d/d h (1) of the flow: deriv_mode 1 holds the isometries fixed,
  // 2 also differentiates them through the eigendecomposition
  bool deriv = false;
  int deriv_mode = 0;
  double *dT = nullptr;       // [2][batch][Pmax^2] tangents of the normalised tensors
  double *D1 = nullptr, *D2 = nullptr;  // tangent squeeze outputs (one instance at a time)
  double *dL = nullptr, *dlnc = nullptr, *dout = nullptr;  // [2][batch]
  double *dU = nullptr;       // [2][batch][u_stride] isometry tangents (mode 2)
  double *H1 = nullptr, *H2 = nullptr, *dG = nullptr;  // half-Gram and Gram tangents (mode 2)
  long long dg_stride = 0;
  void *Tt2 = nullptr, *dX1[2] = {nullptr, nullptr}, *dX2 = nullptr, *dO = nullptr;  // tangent squeeze scratch
  void *dR1 = nullptr, *dR2 = nullptr;
  // zero-field block structure (z2.cu): even-value counts of every leg, before / after a step,
  // the per-instance layouts, index tables and the current chunk's GEMM blocks and parity
  bool z2 = false;      // the block-sparse squeeze is in use
  bool z2_opt = false;  // requested at init (set_tensor turns z2 off, set_tensor_z2 back on)
  // per instance: its tensor is known to have the block structure, with even-first bonds and the
  // even counts in z2ev (z2 is on only while every instance is)
  std::vector<char> z2_inst;
  int *z2ev = nullptr, *z2ev_new = nullptr;
  Z2Layout* z2L = nullptr;
  int *z2rank = nullptr, *z2kcol = nullptr, *z2colpos = nullptr, *z2pi = nullptr;
  double* z2flops = nullptr;  // [2] flops of the GEMM blocks since hotrg_timing_start
  bool t_z2 = false;          // a parity-blocked squeeze ran while timing
  GemmBlocks* z2blk = nullptr;
  // impure tensors (Eqs. (SS), (ST)): [0] the nearest-neighbour pair, [1] the single spin
  bool impure = false;
  double *SI = nullptr;       // [2][batch][Pmax^2], normalised by the pure flow's c_n
  double *Stmp = nullptr;     // [2][Pmax^2] unnormalised squeeze outputs (one instance at a time)
  double *imp_out = nullptr;  // [2][batch] Tr S / Tr T
  long long q_stride = 0, g_stride = 0, u_stride = 0;  // per-instance strides (doubles)
  void *Tt = nullptr, *Bt = nullptr, *X1 = nullptr, *X2 = nullptr, *Y = nullptr, *O = nullptr;
  void *R1 = nullptr, *R2 = nullptr;
  size_t sz_Tt = 0, sz_Bt = 0, sz_X = 0, sz_Y = 0, sz_O = 0, sz_R1 = 0, sz_R2 = 0;
  // instances squeezed together (one GEMM launch per chunk for all of them): every per-step buffer
  // holds `group` slots, st_* bytes apart
  int group = 1;
  size_t st_Tt = 0, st_Bt = 0, st_X = 0, st_Y = 0, st_O = 0, st_R1 = 0, st_R2 = 0, st_Tnext = 0;
  long long spec_stride = 0;  // doubles per instance in spec_log
  // phase timing (hotrg_timing_start/stop): CUDA events recorded on `stream`
  struct Ev {
    int phase;
    cudaEvent_t a, b;
  };
  bool timing = false;
  std::vector<Ev> evs;
  // captured steady-state steps, one per axis (replayed while the bond dimensions do not change)
  bool graphs = true;
  cudaGraphExec_t graph_exec[kMaxD] = {nullptr, nullptr, nullptr, nullptr};
  int graph_dims[kMaxD][kMaxD] = {};
  int graph_planes[kMaxD] = {-1, -1, -1, -1};
  long long launch0 = 0, t_gemm_launches = 0, t_steps = 0;
  double t_gemm_flops = 0, t_gemm_tflops = 0, t_step_flops = 0, t_dense_step_flops = 0;
};

namespace {
enum Phase { PH_STEP = 0, PH_ISO, PH_OPERANDS, PH_GEMM, PH_EPILOGUE, PH_NORM, PH_COUNT };
const char* const kPhaseName[PH_COUNT] = {"hotrg step", "isometries", "operands", "squeeze gemm", "epilogue",
                                          "norm"};

// Marks the phase as an NVTX range on the host thread that enqueues it (visible to profilers that
// attach to NVTX; without one the calls do nothing), and with timing enabled records a start event
// now and an end event when it goes out of scope.
struct PhaseScope {
  hotrg_ctx* c;
  int phase;
  cudaEvent_t a = nullptr;
  PhaseScope(hotrg_ctx* ctx, int ph) : c(ctx), phase(ph) {
    nvtxRangePushA(kPhaseName[ph]);
    if (c->timing && cudaEventCreate(&a) == cudaSuccess) cudaEventRecord(a, c->stream);
  }
  ~PhaseScope() {
    nvtxRangePop();
    cudaEvent_t b = nullptr;
    if (a && cudaEventCreate(&b) == cudaSuccess) {
      cudaEventRecord(b, c->stream);
      c->evs.push_back({phase, a, b});
    }
  }
};
}  // namespace

namespace {

constexpr long long kAlign = 256;
// shape of the wait probe's GEMM launch: one output tile, one k-block
constexpr long long TC_PROBE_M = 128, TC_PROBE_N = 256, TC_PROBE_K = 64;
constexpr int kSpecCap = kMaxGram;  // eigenvalues stored per (step, axis)

long long round_up(long long x, long long m) { return (x + m - 1) / m * m; }

// Sizes (bytes) of the per-step scratch buffers for one configuration.
struct StepNeeds {
  size_t Tt, Bt, X, Y, O, R1, R2;
};

// mixed: 0 = FP64 path, 2 or 3 = tensor-core path with that many bf16 planes per operand
StepNeeds needs_for(int d, const int* dims, int a, int Dcut, int planes) {
  const bool mixed = planes > 0;
  Geom g = make_geom(d, dims);
  const long long P = g.P;
  // operand rows: P rounded up to 64, plus one more 64-column block for the zero-field
  // (parity-blocked) layout, whose two k classes start at 64-aligned columns
  const long long ldk = round_up(P, 64) + 64;
  int chi[kMaxD];
  int trans[kMaxD], nt = 0;
  for (int b = 0; b < d; ++b) {
    chi[b] = dims[b];
    if (b != a) {
      const long long sq = (long long)dims[b] * dims[b];
      chi[b] = (int)(sq < Dcut ? sq : Dcut);
      trans[nt++] = b;
    }
  }
  const int c3 = nt ? trans[nt - 1] : -1;
  const long long chi3 = c3 >= 0 ? chi[c3] : 1;
  const size_t es = mixed ? 4 : 8;  // intermediate element size (float / double)
  StepNeeds n;
  n.Tt = (size_t)(P * P) * es;
  n.Bt = (size_t)(chi3 * P * ldk) * (mixed ? 2 * planes : 8);  // bf16 planes, or double
  n.X = (size_t)(P * P) * es;
  n.Y = (size_t)(P * ldk) * (mixed ? 2 * planes : 8);
  n.O = (size_t)(P * chi3 * P) * es;
  // epilogue intermediates: contract the other transverse axes in order
  long long cur = P * chi3 * P;
  size_t r[2] = {0, 0};
  for (int i = 0; i < nt - 1 && i < 2; ++i) {
    const int b = trans[i];
    cur = cur / ((long long)dims[b] * dims[b]) * chi[b];
    r[i] = (size_t)cur * es;
  }
  n.R1 = r[0];
  n.R2 = r[1];
  return n;
}

void max_into(StepNeeds& acc, const StepNeeds& n) {
  acc.Tt = std::max(acc.Tt, n.Tt);
  acc.Bt = std::max(acc.Bt, n.Bt);
  acc.X = std::max(acc.X, n.X);
  acc.Y = std::max(acc.Y, n.Y);
  acc.O = std::max(acc.O, n.O);
  acc.R1 = std::max(acc.R1, n.R1);
  acc.R2 = std::max(acc.R2, n.R2);
}

// Workspace plan: the per-step buffers must hold every step a context can take. The bond
// dimensions reachable within max_steps steps (any axis sequence, starting from all 2) are
// enumerated breadth-first; each D_b is 2, min(4, Dcut) or min(16, Dcut). Path of a step: FP64
// for P < 256 or (in split modes) for steps <= fp64_steps, tensor cores otherwise with 3 planes
// if the step may run the 6-pass GEMM.
int planes_for_step(int precision, int step, int fp64_steps, int x6_steps, long long P) {
  if (precision == HOTRG_FP64 || P < 256 || step <= fp64_steps) return 0;
  if (precision == HOTRG_BF16X6 || step <= x6_steps) return 3;
  return 2;
}

// Instances squeezed together (opts.group; 0: up to 8, whose per-step buffers are 8 copies), one
// with tangents or impurities (those squeezes run instance by instance).
int group_for(const hotrg_opts* o) {
  if (o->derivatives || o->impurities) return 1;
  const int g = o->group > 0 ? o->group : 8;
  return std::max(1, std::min(std::min(g, o->batch), kMaxGemmBatch));
}

// k-blocks per accumulator fold: one unless the caller chose otherwise, within what the kernel
// variant's ring allows
int fold_group_for(const hotrg_ctx* c, int npass) {
  const int bk = npass == 6 ? 32 : c->kblock;
  const int g = c->fold_group > 0 ? c->fold_group : 1;
  return std::max(1, std::min(g, max_fold_group(npass, bk)));
}

// passes of the split GEMM for a step (0 = FP64 path)
int passes_for_step(int precision, int step, int fp64_steps, int x6_steps, long long P) {
  const int pl = planes_for_step(precision, step, fp64_steps, x6_steps, P);
  if (pl == 0) return 0;
  if (pl == 3) return 6;
  return (precision == HOTRG_BF16X4 || precision == HOTRG_FP16X4) ? 4 : 3;
}

// the two-plane split steps of the FP16 modes use fp16 planes with power-of-two operand scales
bool f16_planes(int precision, int planes) {
  return planes == 2 && (precision == HOTRG_FP16X3 || precision == HOTRG_FP16X4);
}

StepNeeds plan(int d, int Dcut, int precision, int fp64_steps, int x6_steps, int max_steps,
               long long* Pmax_out) {
  // breadth-first: minimal number of steps after which each bond-dimension state is reached
  std::vector<std::vector<int>> states{std::vector<int>(d, 2)};
  std::vector<int> depth{0};
  for (size_t i = 0; i < states.size(); ++i) {
    if (depth[i] >= max_steps) continue;
    for (int a = 0; a < d; ++a) {
      std::vector<int> nd(states[i]);
      for (int b = 0; b < d; ++b)
        if (b != a) nd[b] = std::min(nd[b] * nd[b], Dcut);
      if (std::find(states.begin(), states.end(), nd) == states.end()) {
        states.push_back(nd);
        depth.push_back(depth[i] + 1);
      }
    }
  }
  StepNeeds acc{0, 0, 0, 0, 0, 0, 0};
  long long Pmax = 1;
  for (size_t i = 0; i < states.size(); ++i) {
    long long P = 1;
    for (int b = 0; b < d; ++b) P *= states[i][b];
    Pmax = std::max(Pmax, P);
    const int first = depth[i] + 1;  // earliest step number taken from this state
    if (first > max_steps) continue;
    for (int a = 0; a < d; ++a)
      for (int step : {first, fp64_steps + 1, x6_steps + 1, max_steps})
        if (step >= first && step <= max_steps)
          max_into(acc, needs_for(d, states[i].data(), a, Dcut,
                                  planes_for_step(precision, step, fp64_steps, x6_steps, P)));
  }
  *Pmax_out = Pmax;
  return acc;
}

struct Carver {
  char* base;
  size_t off = 0;
  template <class T>
  T* take(size_t bytes) {
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += (size_t)round_up((long long)bytes, kAlign);
    return p;
  }
};

// Lay out every buffer; with base == nullptr only the total size is computed.
size_t carve(hotrg_ctx* c, char* base) {
  long long Pmax = 1;
  StepNeeds n = plan(c->d, c->Dcut, c->precision, c->fp64_steps, c->x6_steps, c->max_steps, &Pmax);
  c->Pmax = Pmax;
  const long long P2 = Pmax * Pmax;
  const int nr_max = kMaxGram;
  Carver k{base};
  const int G = c->group;
  c->T = k.take<double>(sizeof(double) * P2 * c->batch);
  c->st_Tnext = (size_t)round_up((long long)(sizeof(double) * P2), kAlign);
  c->Tnext = k.take<double>(c->st_Tnext * G);
  c->dbeta = k.take<double>(sizeof(double) * c->batch);
  c->dh = k.take<double>(sizeof(double) * c->batch);
  c->L = k.take<double>(sizeof(double) * c->batch);
  c->lnc_log = k.take<double>(sizeof(double) * c->batch * (c->max_steps + 1));
  c->spec_stride = (long long)c->max_steps * c->d * kSpecCap;
  c->spec_log = k.take<double>(sizeof(double) * c->batch * c->spec_stride);
  c->out3 = k.take<double>(sizeof(double) * 3 * c->batch);
  c->cval = k.take<double>(sizeof(double) * c->batch);
  c->status = k.take<int>(sizeof(int) * 32);
  c->dstep = k.take<int>(sizeof(int) * 32);
  c->amax = k.take<unsigned>(sizeof(unsigned) * 2 * G);
  c->norm_partial = k.take<double>(sizeof(double) * 1024);
  // Gram matrices and isometries: sized for the largest Gram this Dcut produces (n <= Dcut^2... 256)
  const int nmax = std::min(kMaxGram, std::max(16, c->Dcut * c->Dcut));
  const int nrm = std::min(kMaxGram, std::max(16, c->Dcut * c->Dcut));
  c->q_stride = (long long)nrm * nrm;
  c->g_stride = (long long)kMaxD * nmax * nmax;
  c->u_stride = (long long)kMaxD * kMaxBond * kMaxGram;
  c->gpartial = k.take<double>(sizeof(double) * gram_partial_doubles(nrm, c->batch));
  c->Q1 = k.take<double>(sizeof(double) * c->q_stride * c->batch);
  c->Q2 = k.take<double>(sizeof(double) * c->q_stride * c->batch);
  c->G = k.take<double>(sizeof(double) * c->g_stride * c->batch);
  c->U = k.take<double>(sizeof(double) * c->u_stride * c->batch);
  c->ework_axis = 2LL * nmax * nmax * c->batch;
  c->ework = k.take<double>(sizeof(double) * c->ework_axis * kMaxD);  // one area per axis
  (void)nr_max;
  if (c->deriv) {
    c->dT = k.take<double>(sizeof(double) * 2 * P2 * c->batch);
    c->D1 = k.take<double>(sizeof(double) * P2);
    c->D2 = k.take<double>(sizeof(double) * P2);
    c->dL = k.take<double>(sizeof(double) * 2 * c->batch);
    c->dlnc = k.take<double>(sizeof(double) * 2 * c->batch);
    c->dout = k.take<double>(sizeof(double) * 2 * c->batch);
  }
  if (c->deriv_mode == 2) {
    c->dU = k.take<double>(sizeof(double) * 2 * c->u_stride * c->batch);
    c->H1 = k.take<double>(sizeof(double) * c->q_stride * c->batch);
    c->H2 = k.take<double>(sizeof(double) * c->q_stride * c->batch);
    c->dg_stride = (long long)nmax * nmax;
    c->dG = k.take<double>(sizeof(double) * c->dg_stride * c->batch);
  }
  if (c->z2) {
    c->z2ev = k.take<int>(sizeof(int) * kMaxD * c->batch);
    c->z2ev_new = k.take<int>(sizeof(int) * kMaxD * c->batch);
    c->z2L = k.take<Z2Layout>(sizeof(Z2Layout) * c->batch);
    c->z2rank = k.take<int>(sizeof(int) * Pmax * G);
    c->z2kcol = k.take<int>(sizeof(int) * Pmax * G);
    c->z2colpos = k.take<int>(sizeof(int) * Pmax * kMaxBond * G);
    c->z2blk = k.take<GemmBlocks>(sizeof(GemmBlocks) * G);  // contiguous: the batched GEMM reads blk[j]
    c->z2pi = k.take<int>(sizeof(int) * G);
    c->z2flops = k.take<double>(sizeof(double) * 4);
  }
  if (c->impure) {
    c->SI = k.take<double>(sizeof(double) * 2 * P2 * c->batch);
    c->Stmp = k.take<double>(sizeof(double) * 2 * P2);
    c->imp_out = k.take<double>(sizeof(double) * 2 * c->batch);
  }
  // with tangents the operands hold three column blocks per row (see squeeze)
  const size_t blk = c->deriv ? 3 : 1;
  // per-step buffers: `group` slots of each (slot strides 256-byte aligned: TMA plane starts)
  auto slots = [&](size_t bytes, size_t& sz, size_t& st) {
    sz = bytes;
    st = (size_t)round_up((long long)(bytes ? bytes : 256), kAlign);
    return k.take<char>(st * G);
  };
  size_t st_x2 = 0;
  c->Tt = slots(n.Tt, c->sz_Tt, c->st_Tt);
  c->Bt = slots(n.Bt * blk, c->sz_Bt, c->st_Bt);
  c->X1 = slots(n.X, c->sz_X, c->st_X);
  c->X2 = slots(n.X, c->sz_X, st_x2);
  c->Y = slots(n.Y * blk, c->sz_Y, c->st_Y);
  c->O = slots(n.O, c->sz_O, c->st_O);
  c->R1 = slots(n.R1, c->sz_R1, c->st_R1);
  c->R2 = slots(n.R2, c->sz_R2, c->st_R2);
  if (c->deriv) {
    c->Tt2 = k.take<char>(n.Tt);
    c->dX1[0] = k.take<char>(n.X);
    c->dX1[1] = k.take<char>(n.X);
    c->dX2 = k.take<char>(n.X);
    c->dO = k.take<char>(n.O);
    c->dR1 = k.take<char>(n.R1 ? n.R1 : 256);
    c->dR2 = k.take<char>(n.R2 ? n.R2 : 256);
  }
  return k.off;
}

int cuda_err(hotrg_ctx* c) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    if (c && !c->sticky) c->sticky = HOTRG_EDEVICE;
    return HOTRG_EDEVICE;
  }
  return HOTRG_OK;
}

int status_to_code(int bits) {
  if (bits & ST_TIMEOUT) return HOTRG_ETIMEOUT;
  if (bits & ST_NOCONV) return HOTRG_ENOCONV;
  if (bits & (ST_NUMERIC | ST_Z2)) return HOTRG_ENUMERIC;
  if (bits) return HOTRG_EDEVICE;
  return HOTRG_OK;
}

// Synchronise and fold the device status word into the sticky error.
int sync_check(hotrg_ctx* c) {
  if (c->sticky) return c->sticky;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
    cudaGetLastError();
    return c->sticky = HOTRG_EDEVICE;
  }
  int bits = 0;
  if (cudaMemcpy(&bits, c->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return c->sticky = HOTRG_EDEVICE;
  const int code = status_to_code(bits);
  if (code) c->sticky = code;
  return code;
}

// Forget the captured steady-state steps (after the tensor, its bond order or the squeeze
// path changed from outside the flow).
void drop_graphs(hotrg_ctx* c) {
  for (int a = 0; a < kMaxD; ++a)
    if (c->graph_exec[a]) {
      cudaGraphExecDestroy(c->graph_exec[a]);
      c->graph_exec[a] = nullptr;
      c->graph_planes[a] = -1;
    }
}

// ----------------------------------------------------------------- epilogue axis bookkeeping
struct Ax {
  int dim;
  long long stride;
  int kind;  // 0 = m (site-1 primed / a1), 1 = j (c3 isometry index), 2 = n (site-2 primed)
  int slot;
};

// Contract (m_b, n_b) with U_b into k'_b; output dense row-major unless out_strides given.
// Output description of contracting (m_b, n_b) into k'_b: the output view without k' (rest),
// the stride of k', the contracted input axes and the dense output axes.
struct Contraction {
  View rest;
  long long sk;
  int im, in_;
  std::vector<Ax> out_axes;
};

Contraction plan_contraction(const std::vector<Ax>& axes, int b, int chi_b, const long long* final_out_stride) {
  Contraction r;
  int im = -1, in_ = -1;
  for (int i = 0; i < (int)axes.size(); ++i) {
    if (axes[i].kind == 0 && axes[i].slot == b) im = i;
    if (axes[i].kind == 2 && axes[i].slot == b) in_ = i;
  }
  View v{};
  int kaxis = -1;
  for (int i = 0; i < (int)axes.size(); ++i) {
    if (i == im) continue;
    Ax ax = axes[i];
    if (i == in_) {
      kaxis = v.ndim;
      ax.dim = chi_b;
      ax.stride = 0;
    }
    v.shape[v.ndim] = ax.dim;
    v.in_stride[v.ndim] = ax.stride;
    r.out_axes.push_back(ax);
    ++v.ndim;
  }
  long long st = 1;
  for (int i = v.ndim - 1; i >= 0; --i) {
    v.out_stride[i] = final_out_stride ? final_out_stride[i] : st;
    st *= v.shape[i];
  }
  r.rest.ndim = 0;
  for (int i = 0; i < v.ndim; ++i) {
    if (i == kaxis) continue;
    r.rest.shape[r.rest.ndim] = v.shape[i];
    r.rest.in_stride[r.rest.ndim] = v.in_stride[i];
    r.rest.out_stride[r.rest.ndim] = v.out_stride[i];
    ++r.rest.ndim;
  }
  r.sk = v.out_stride[kaxis];
  r.im = im;
  r.in_ = in_;
  st = 1;
  for (int i = v.ndim - 1; i >= 0; --i) {
    r.out_axes[i].stride = st;
    st *= r.out_axes[i].dim;
  }
  return r;
}

// The first contraction of a chunk's epilogue from the parity-blocked GEMM output (z2.cu).
template <class Tin, class Tout>
void contract_axes_z2(std::vector<Ax>& axes, const Tin* O, long long ldO, Tout* out, int b, int chi_b,
                      const double* Ub, const long long* final_out_stride, long long out_base,
                      const Z2Layout* L, const int* pi, cudaStream_t s) {
  Contraction r = plan_contraction(axes, b, chi_b, final_out_stride);
  launch_epi_z2<Tin, Tout>(O, ldO, out, r.rest, r.sk, out_base, b, axes[r.im].dim, Ub, chi_b, L, pi, s);
  axes = r.out_axes;
}

// With in2 (laid out like in), the same contraction of in2 with U2 is added.
template <class Tin, class Tout>
void contract_axes(std::vector<Ax>& axes, const Tin* in, Tout* out, int b, int chi_b, const double* Ub,
                   const long long* final_out_stride, long long out_base, cudaStream_t s,
                   const Tin* in2 = nullptr, const double* U2 = nullptr) {
  int im = -1, in_ = -1;
  for (int i = 0; i < (int)axes.size(); ++i) {
    if (axes[i].kind == 0 && axes[i].slot == b) im = i;
    if (axes[i].kind == 2 && axes[i].slot == b) in_ = i;
  }
  std::vector<Ax> out_axes;
  View v{};
  int kaxis = -1;
  for (int i = 0; i < (int)axes.size(); ++i) {
    if (i == im) continue;
    Ax ax = axes[i];
    if (i == in_) {
      kaxis = v.ndim;
      ax.dim = chi_b;
      ax.stride = 0;
    }
    v.shape[v.ndim] = ax.dim;
    v.in_stride[v.ndim] = ax.stride;
    out_axes.push_back(ax);
    ++v.ndim;
  }
  // output strides
  long long st = 1;
  for (int i = v.ndim - 1; i >= 0; --i) {
    v.out_stride[i] = final_out_stride ? final_out_stride[i] : st;
    st *= v.shape[i];
  }
  // rest view: the output axes without k'
  View rest;
  rest.ndim = 0;
  for (int i = 0; i < v.ndim; ++i) {
    if (i == kaxis) continue;
    rest.shape[rest.ndim] = v.shape[i];
    rest.in_stride[rest.ndim] = v.in_stride[i];
    rest.out_stride[rest.ndim] = v.out_stride[i];
    ++rest.ndim;
  }
  launch_pair_contract_all<Tin, Tout>(in, out, rest, axes[im].dim, axes[in_].dim, axes[im].stride,
                                      axes[in_].stride, v.out_stride[kaxis], Ub, chi_b, 0, out_base, s, in2, U2);
  // new axes describe the dense output (only meaningful when not final)
  st = 1;
  for (int i = v.ndim - 1; i >= 0; --i) {
    out_axes[i].stride = st;
    st *= out_axes[i].dim;
  }
  axes = out_axes;
}

// Strides of the final output (Tnext in the new geometry) for an axes list.
void final_strides(const std::vector<Ax>& axes, int skip_m_slot, int kslot, const Geom& gn, int c3,
                   long long* out) {
  int v = 0;
  for (const Ax& ax : axes) {
    if (ax.kind == 0 && ax.slot == skip_m_slot) continue;  // contracted away
    long long s = 0;
    if (ax.kind == 0) s = gn.Sn[ax.slot] * gn.P;          // m_a -> u'_a
    else if (ax.kind == 1) s = c3 >= 0 ? gn.Sn[c3] * gn.P : 0;  // j -> u'_c3
    else s = gn.Sn[ax.slot];                                // n_b / k'_b -> p'_b
    (void)kslot;
    out[v++] = s;
  }
}

// d = 1: no transverse axes, the GEMM output O[m][n] is the new tensor Tnext[u'][p'].
template <class TC>
void copy_final(const std::vector<Ax>& axes, const TC* in, double* out, const Geom& gn, cudaStream_t s) {
  long long fs[kMaxAxes];
  final_strides(axes, -2, -1, gn, -1, fs);
  View v;
  v.ndim = (int)axes.size();
  for (int i = 0; i < v.ndim; ++i) {
    v.shape[i] = axes[i].dim;
    v.in_stride[i] = axes[i].stride;
    v.out_stride[i] = fs[i];
  }
  launch_pair_contract<TC, double>(in, out, v, -1, 1, 1, 0, 0, nullptr, 1, 0, 0, s);
}

template <class TC>
struct Ops;  // operand element types of a path

template <>
struct Ops<double> {
  using Op = double;
};
template <>
struct Ops<float> {
  using Op = __nv_bfloat16;
};

// Tangent inputs of a squeeze of T with itself: for each of n parameters the tangent dT (same
// layout as T), the output tangent (new geometry, before normalisation) and the isometry
// tangents dU (null: isometries held fixed).
struct Tangents {
  int n = 0;
  const double* dT[2] = {nullptr, nullptr};
  double* dout[2] = {nullptr, nullptr};
  const double* dU[2] = {nullptr, nullptr};
};

// Per-step scratch of one instance of a squeeze group: slot j of every per-step buffer (the plan
// holds opts.group slots of each).
struct Slot {
  void *Tt, *Bt, *X1, *X2, *Y, *O, *R1, *R2;
  double* Tnext;
  unsigned* amax;  // [0] bound of the B operand's source, [1] of the A operand's (fp16 planes)
  int *z2rank, *z2kcol, *z2colpos, *z2pi;
  GemmBlocks* z2blk;
};

Slot slot(const hotrg_ctx* c, int j) {
  auto at = [j](void* base, size_t stride) -> void* {
    return base ? static_cast<void*>(static_cast<char*>(base) + stride * (size_t)j) : nullptr;
  };
  Slot q;
  q.Tt = at(c->Tt, c->st_Tt);
  q.Bt = at(c->Bt, c->st_Bt);
  q.X1 = at(c->X1, c->st_X);
  q.X2 = at(c->X2, c->st_X);
  q.Y = at(c->Y, c->st_Y);
  q.O = at(c->O, c->st_O);
  q.R1 = at(c->R1, c->st_R1);
  q.R2 = at(c->R2, c->st_R2);
  q.Tnext = static_cast<double*>(at(c->Tnext, c->st_Tnext));
  q.amax = c->amax + 2 * j;
  q.z2rank = c->z2rank ? c->z2rank + c->Pmax * j : nullptr;
  q.z2kcol = c->z2kcol ? c->z2kcol + c->Pmax * j : nullptr;
  q.z2colpos = c->z2colpos ? c->z2colpos + c->Pmax * kMaxBond * j : nullptr;
  q.z2pi = c->z2pi ? c->z2pi + j : nullptr;
  q.z2blk = c->z2blk ? c->z2blk + j : nullptr;
  return q;
}

// The instances squeezed together: instance j reads T1[j] (lower site, A operand) and T2[j] (upper
// site, B operand) with isometries U[j], writes out[j] and works in per-step slot j; inst[j] is its
// index in the context (zero-field layouts). One GEMM launch per chunk covers all of them.
struct Group {
  int n = 0;
  std::vector<const double*> T1, T2, U;
  std::vector<double*> out;
  std::vector<int> inst;
  void add(const double* t1, const double* t2, const double* u, double* o, int i) {
    T1.push_back(t1);
    T2.push_back(t2);
    U.push_back(u);
    out.push_back(o);
    inst.push_back(i);
    ++n;
  }
};

// planes: 0 = FP64 path (TC = double), 2 / 3 = tensor-core path (TC = float) with 3 / 6 passes.
template <class TC>
// Coarse-grained tensor of the pair (T1 lower site, T2 upper site along a) into `out` (new
// geometry gn) for every instance of the group: T1 feeds the A operand, T2 the B operand. The
// small operand and epilogue kernels run instance by instance; the squeeze GEMM of a chunk is one
// batched launch over the group. With tangents (a group of one, T1 = T2 = T), also
//   dT' = S(dT, T) + S(T, dT) + sum over the six places of an isometry of S with dU there,
// computed as a dual-number pass: every producer and epilogue stage propagates (x, dx), and the
// O(D^15) contraction of a tangent is one GEMM over the concatenated k range,
//   dO = [dY | Y] . [Bt | dBt]^T,
// with the operand blocks laid out side by side in one row: Y' = [dY_0 | Y | dY_1] and
// Bt' = [dBt_1 | Bt | dBt_0] (row stride 3 ldk), so that [dY_0 | Y] pairs with [Bt | dBt_0] and
// [Y | dY_1] with [dBt_1 | Bt].
int squeeze(hotrg_ctx* c, const Group& G, const Geom& g, const Geom& gn, int a, const int* chi, const int* trans,
            int nt, int planes, int npass, const Tangents& tg = Tangents()) {
  using Op = typename Ops<TC>::Op;
  constexpr bool mixed = std::is_same<TC, float>::value;
  cudaStream_t s = c->stream;
  const int ng = G.n;
  if (ng < 1 || ng > c->group || (tg.n && ng != 1)) return HOTRG_ESTATE;
  const long long P = g.P;
  const long long ldk = mixed ? round_up(P, 64) : P;
  const int nblk = tg.n ? 3 : 1;
  const long long ld = nblk * ldk;
  const int fwd_blk = tg.n ? 1 : 0;
  const int c3 = nt ? trans[nt - 1] : -1;
  const int chi3 = c3 >= 0 ? chi[c3] : 1;
  auto Ub = [&](const double* base, int b) { return base + (long long)b * kMaxBond * kMaxGram; };
  // bounds of this step's buffers against the plan
  StepNeeds need = needs_for(c->d, g.D, a, c->Dcut, planes);
  if (need.Tt > c->sz_Tt || need.Bt * nblk > c->sz_Bt || need.X > c->sz_X || need.Y * nblk > c->sz_Y ||
      need.O > c->sz_O || need.R1 > c->sz_R1 || need.R2 > c->sz_R2)
    return HOTRG_ENOMEM;
  if (tg.n && (!c->Tt2 || !c->dO || tg.n > 2)) return HOTRG_ESTATE;
  const int nparts = mixed ? planes : 1;
  const long long bt_plane = (long long)chi3 * P * ld, y_plane = P * ld;
  // fp16 planes (FP16 modes; the forward squeeze only, tangents keep bf16): each operand's scale
  // comes from the largest entry of its source, measured on the device. |Bt| <= sqrt(D_c3) max|Tt|
  // (each Bt entry contracts a fibre of D_c3 entries with part of a unit isometry vector); Y's
  // entries are the source's own.
  const bool f16 = mixed && tg.n == 0 && f16_planes(c->precision, planes);
  const float bt_mult = c3 >= 0 ? (float)std::sqrt((double)g.D[c3]) : 1.f;
  // which: 0 = B operand, 1 = A operand (fp16 scale bound amax[which])
  auto blocks = [&](void* base, long long plane_elems, int blk, int which = -1, const unsigned* amax = nullptr) {
    Planes<Op> pl;
    pl.nparts = nparts;
    for (int k = 0; k < 3; ++k)
      pl.p[k] = static_cast<Op*>(base) + (size_t)(k < nparts ? k : 0) * plane_elems + blk * ldk;
    if (f16 && which >= 0) {
      pl.fmt = 1;
      pl.amax = amax + which;
      pl.amax_mult = which == 0 ? bt_mult : 1.f;
    }
    return pl;
  };
  // tangent p: A operand block, B operand block written by its build, and the GEMM's first blocks
  auto dy_blk = [](int p) { return p == 0 ? 0 : 2; };
  auto dbt_blk = [](int p) { return p == 0 ? 2 : 0; };
  auto gemm_a_blk = [](int p) { return p == 0 ? 0 : 1; };
  auto gemm_b_blk = [](int p) { return p == 0 ? 1 : 0; };
  const Slot S0 = slot(c, 0);
  // B operand(s), one per instance
  PhaseScope* ops_scope = new PhaseScope(c, PH_OPERANDS);
  if (tg.n && mixed && ldk != P) {
    // the concatenated k range runs over the zero padding between blocks
    cudaMemsetAsync(S0.Bt, 0, sizeof(Op) * nparts * bt_plane, s);
    cudaMemsetAsync(S0.Y, 0, sizeof(Op) * nparts * y_plane, s);
  }
  for (int j = 0; j < ng; ++j) {
    const Slot S = slot(c, j);
    TC* Tt = static_cast<TC*>(S.Tt);
    launch_transpose<TC>(G.T2[j], Tt, P, s);
    if (f16) launch_absmax<TC>(Tt, P, P, P, S.amax + 0, s);
    launch_build_bt<TC, Op>(Tt, blocks(S.Bt, bt_plane, fwd_blk, 0, S.amax), ld, g, c3,
                            c3 >= 0 ? Ub(G.U[j], c3) : nullptr, chi3, s);
  }
  for (int p = 0; p < tg.n; ++p) {
    TC* dTt = static_cast<TC*>(c->Tt2);
    launch_transpose<TC>(tg.dT[p], dTt, P, s);
    const bool two = tg.dU[p] && c3 >= 0;
    launch_build_bt<TC, Op>(dTt, blocks(S0.Bt, bt_plane, dbt_blk(p)), ld, g, c3, c3 >= 0 ? Ub(G.U[0], c3) : nullptr,
                            chi3, s, two ? static_cast<TC*>(S0.Tt) : nullptr, two ? Ub(tg.dU[p], c3) : nullptr);
  }
  delete ops_scope;
  TC* O = static_cast<TC*>(S0.O);
  TC* dO = static_cast<TC*>(c->dO);
  const long long ldO = (long long)chi3 * P;
  // chunks over the other transverse axes
  const int no = nt > 0 ? nt - 1 : 0;
  int kcnt[kMaxD] = {0, 0, 0, 0};
  long long nchunks = 1;
  for (int i = 0; i < no; ++i) nchunks *= chi[trans[i]];
  int prev_k0 = -1;
  // instance j's operand planes and output are slot j's: one launch for the group
  GemmBatch bat;
  bat.batch = ng;
  bat.a_inst = (long long)(c->st_Y / sizeof(Op));
  bat.b_inst = (long long)(c->st_Bt / sizeof(Op));
  bat.c_inst = (long long)(c->st_O / sizeof(TC));
  bat.amax_inst = 2;
  const GemmBatch* batp = ng > 1 ? &bat : nullptr;
  auto gemm = [&](int ablk, int bblk, TC* C, long long K) -> int {
    PhaseScope gemm_scope(c, PH_GEMM);
    if constexpr (mixed) {
      const int rc = launch_gemm_split(blocks(S0.Y, y_plane, ablk, 1, S0.amax), ld,
                                       blocks(S0.Bt, bt_plane, bblk, 0, S0.amax), ld, reinterpret_cast<float*>(C),
                                       ldO, P, ldO, K, npass, c->status, c->timeout_s, s, c->kblock, c->group_m,
                                       fold_group_for(c, npass), nullptr, batp, false, c->cta_group);
      if (rc) return rc;
      if (c->timing) c->t_gemm_tflops += 2.0 * P * (double)ldO * K * npass * ng;
    } else {
      launch_gemm_f64(blocks(S0.Y, y_plane, ablk).p[0], ld, blocks(S0.Bt, bt_plane, bblk).p[0], ld, C, ldO, P, ldO,
                      K, s, nullptr, batp);
      if (c->timing) c->t_gemm_tflops += 2.0 * P * (double)ldO * K * ng;
    }
    if (c->timing) {
      c->t_gemm_flops += 2.0 * P * (double)ldO * K * ng;
      ++c->t_gemm_launches;
    }
    return HOTRG_OK;
  };
  for (long long ch = 0; ch < nchunks; ++ch) {
    long long r = ch;
    for (int i = no - 1; i >= 0; --i) {
      kcnt[i] = (int)(r % chi[trans[i]]);
      r /= chi[trans[i]];
    }
    // producer: mode products on the unprimed legs of the other transverse axes
    ops_scope = new PhaseScope(c, PH_OPERANDS);
    for (int j = 0; j < ng; ++j) {
      const Slot S = slot(c, j);
      const double* T1 = G.T1[j];
      const double* U = G.U[j];
      if (no == 0) {
        if (f16) launch_absmax<double>(T1, P, P, P, S.amax + 1, s);
        launch_build_y<double, Op>(T1, blocks(S.Y, y_plane, fwd_blk, 1, S.amax), ld, g, a, s);
        for (int p = 0; p < tg.n; ++p)
          launch_build_y<double, Op>(tg.dT[p], blocks(S.Y, y_plane, dy_blk(p)), ld, g, a, s);
      } else {
        TC* X1 = static_cast<TC*>(S.X1);
        TC* X2 = static_cast<TC*>(S.X2);
        const int b0 = trans[0];
        // the mode product that writes X also measures max |X|, the fp16 scale bound of Y
        if (kcnt[0] != prev_k0) {
          launch_mode_unprimed<double, TC>(T1, X1, g, b0, Ub(U, b0), kcnt[0], s, nullptr, nullptr,
                                           (f16 && no == 1) ? S.amax + 1 : nullptr);
          for (int p = 0; p < tg.n; ++p)
            launch_mode_unprimed<double, TC>(tg.dT[p], static_cast<TC*>(c->dX1[p]), g, b0, Ub(U, b0), kcnt[0], s,
                                             tg.dU[p] ? T1 : nullptr, tg.dU[p] ? Ub(tg.dU[p], b0) : nullptr);
        }
        const TC* X = X1;
        if (no >= 2) {
          launch_mode_unprimed<TC, TC>(X1, X2, g, trans[1], Ub(U, trans[1]), kcnt[1], s, nullptr, nullptr,
                                       f16 ? S.amax + 1 : nullptr);
          X = X2;
        }
        launch_build_y<TC, Op>(X, blocks(S.Y, y_plane, fwd_blk, 1, S.amax), ld, g, a, s);
        for (int p = 0; p < tg.n; ++p) {
          const TC* dX = static_cast<TC*>(c->dX1[p]);
          if (no >= 2) {
            TC* dX2 = static_cast<TC*>(c->dX2);
            launch_mode_unprimed<TC, TC>(dX, dX2, g, trans[1], Ub(U, trans[1]), kcnt[1], s,
                                         tg.dU[p] ? X1 : nullptr, tg.dU[p] ? Ub(tg.dU[p], trans[1]) : nullptr);
            dX = dX2;
          }
          launch_build_y<TC, Op>(dX, blocks(S.Y, y_plane, dy_blk(p)), ld, g, a, s);
        }
      }
    }
    if (no > 0) prev_k0 = kcnt[0];
    delete ops_scope;
    // the O(D^15) GEMM, all instances of the group in one launch
    {
      const int rc = gemm(fwd_blk, fwd_blk, O, P);
      if (rc) return rc;
      c->last_gemm.M = P;
      c->last_gemm.N = ldO;
      c->last_gemm.K = P;
      c->last_gemm.ldk = ld;
      c->last_gemm.npass = npass;
      c->last_gemm.nparts = planes;
      c->last_gemm.fmt = f16 ? 1 : 0;
      c->last_gemm.mult_b = bt_mult;
      c->last_gemm.blk = nullptr;
    }
    // epilogue: O axes [m_0..m_{d-1}, j, n_0..n_{d-1}]
    std::vector<Ax> hist[kMaxD];  // axes of the input of each contraction of the chain
    TC* dbufs[2] = {static_cast<TC*>(c->dR1), static_cast<TC*>(c->dR2)};
    long long out_base = 0;
    for (int i = 0; i < no; ++i) out_base += (long long)kcnt[i] * gn.Sn[trans[i]] * gn.P;
    {
      PhaseScope epi_scope(c, PH_EPILOGUE);
      for (int j = 0; j < ng; ++j) {
        const Slot S = slot(c, j);
        TC* bufs[2] = {static_cast<TC*>(S.R1), static_cast<TC*>(S.R2)};
        std::vector<Ax> axes;
        for (int b = 0; b < c->d; ++b) axes.push_back({g.D[b], g.Sn[b] * ldO, 0, b});
        axes.push_back({chi3, P, 1, -1});
        for (int b = 0; b < c->d; ++b) axes.push_back({g.D[b], g.Sn[b], 2, b});
        const TC* cur = static_cast<TC*>(S.O);
        for (int i = 0; i < no; ++i) {
          hist[i] = axes;
          contract_axes<TC, TC>(axes, cur, bufs[i], trans[i], chi[trans[i]], Ub(G.U[j], trans[i]), nullptr, 0, s);
          cur = bufs[i];
        }
        hist[no] = axes;
        long long fs[kMaxAxes];
        if (c3 >= 0) {
          // final axes after contracting c3 (m_c3 removed, n_c3 -> k'_c3)
          final_strides(axes, c3, c3, gn, c3, fs);
          contract_axes<TC, double>(axes, cur, G.out[j], c3, chi3, Ub(G.U[j], c3), fs, out_base, s);
        } else {
          copy_final<TC>(axes, cur, G.out[j], gn, s);
        }
      }
    }
    // tangents (a group of one): dO by one GEMM over the concatenated k range, then the epilogue
    // chain in dual numbers (dR' = C_U(dR) + C_dU(R))
    for (int p = 0; p < tg.n; ++p) {
      const int rc = gemm(gemm_a_blk(p), gemm_b_blk(p), dO, ldk + P);
      if (rc) return rc;
      PhaseScope epi_scope(c, PH_EPILOGUE);
      const double* U = G.U[0];
      TC* bufs[2] = {static_cast<TC*>(S0.R1), static_cast<TC*>(S0.R2)};
      const TC* cur = dO;
      const TC* curF = O;
      for (int i = 0; i < no; ++i) {
        std::vector<Ax> ax = hist[i];
        contract_axes<TC, TC>(ax, cur, dbufs[i], trans[i], chi[trans[i]], Ub(U, trans[i]), nullptr, 0, s,
                              tg.dU[p] ? curF : nullptr, tg.dU[p] ? Ub(tg.dU[p], trans[i]) : nullptr);
        cur = dbufs[i];
        curF = bufs[i];
      }
      std::vector<Ax> ax = hist[no];
      long long fs[kMaxAxes];
      if (c3 >= 0) {
        final_strides(ax, c3, c3, gn, c3, fs);
        contract_axes<TC, double>(ax, cur, tg.dout[p], c3, chi3, Ub(U, c3), fs, out_base, s,
                                  tg.dU[p] ? curF : nullptr, tg.dU[p] ? Ub(tg.dU[p], c3) : nullptr);
      } else {
        copy_final<TC>(ax, cur, tg.dout[p], gn, s);
      }
    }
  }
  return HOTRG_OK;
}

// The zero-field squeeze of T with itself (z2.cu) for every instance of the group: parity-blocked
// operands, two dense GEMM blocks per chunk and instance (one batched launch over the group, each
// instance with its own block descriptor), the first epilogue contraction reading the blocked
// output. TC = float: the tensor-core path (bf16 or fp16 planes, npass split products); TC = double:
// the FP64 path. Same output as squeeze<TC> up to the order of summation.
template <class TC>
int squeeze_z2(hotrg_ctx* c, const Group& G, const Geom& g, const Geom& gn, int a, const int* chi, const int* trans,
               int nt, int planes, int npass) {
  using Op = typename Ops<TC>::Op;
  constexpr bool mixed = std::is_same<TC, float>::value;
  cudaStream_t s = c->stream;
  const int ng = G.n;
  if (ng < 1 || ng > c->group) return HOTRG_ESTATE;
  const long long P = g.P;
  const long long ldz = round_up(P, 64) + 64;
  const int c3 = trans[nt - 1];
  const int chi3 = chi[c3];
  auto Ub = [&](int j, int b) { return G.U[j] + (long long)b * kMaxBond * kMaxGram; };
  StepNeeds need = needs_for(c->d, g.D, a, c->Dcut, planes);
  if (need.Tt > c->sz_Tt || need.Bt > c->sz_Bt || need.X > c->sz_X || need.Y > c->sz_Y || need.O > c->sz_O ||
      need.R1 > c->sz_R1 || need.R2 > c->sz_R2 || P > c->Pmax)
    return HOTRG_ENOMEM;
  const int nparts = mixed ? planes : 1;
  const long long bt_plane = (long long)chi3 * P * ldz, y_plane = P * ldz;
  // fp16 planes in the FP16 modes, with the scale bounds of squeeze<TC> (B: sqrt(D_c3) max|Tt|)
  const bool f16 = mixed && f16_planes(c->precision, planes);
  const float bt_mult = (float)std::sqrt((double)g.D[c3]);
  auto pl = [&](void* base, long long plane_elems, int which, const unsigned* amax) {  // which: 0 = B, 1 = A
    Planes<Op> q;
    q.nparts = nparts;
    for (int k = 0; k < 3; ++k) q.p[k] = static_cast<Op*>(base) + (size_t)(k < nparts ? k : 0) * plane_elems;
    if (f16) {
      q.fmt = 1;
      q.amax = amax + which;
      q.amax_mult = which == 0 ? bt_mult : 1.f;
    }
    return q;
  };
  const long long ldO = (long long)chi3 * P;
  const Slot S0 = slot(c, 0);
  PhaseScope* ops_scope = new PhaseScope(c, PH_OPERANDS);
  for (int j = 0; j < ng; ++j) {
    const Slot S = slot(c, j);
    const int inst = G.inst[j];
    Z2Layout* L = c->z2L + inst;
    launch_z2_layout(c->z2ev + inst * kMaxD, c->z2ev_new + inst * kMaxD, 1, g, c3, chi3, L, s);
    launch_z2_tables(L, P, chi3, S.z2rank, S.z2kcol, S.z2colpos, s);
    // zeros between and after the k classes (the GEMM's k-blocks run over them)
    cudaMemsetAsync(S.Bt, 0, sizeof(Op) * nparts * bt_plane, s);
    cudaMemsetAsync(S.Y, 0, sizeof(Op) * nparts * y_plane, s);
    TC* Tt = static_cast<TC*>(S.Tt);
    launch_transpose<TC>(G.T2[j], Tt, P, s);
    if (f16) launch_absmax<TC>(Tt, P, P, P, S.amax + 0, s);
    launch_build_bt_z2<TC, Op>(Tt, pl(S.Bt, bt_plane, 0, S.amax), ldz, g, c3, Ub(j, c3), chi3, S.z2rank, S.z2kcol,
                               S.z2colpos, L, s);
  }
  delete ops_scope;
  const int no = nt - 1;
  int kcnt[kMaxD] = {0, 0, 0, 0};
  long long nchunks = 1;
  for (int i = 0; i < no; ++i) nchunks *= chi[trans[i]];
  int prev_k0 = -1;
  GemmBatch bat;
  bat.batch = ng;
  bat.a_inst = (long long)(c->st_Y / sizeof(Op));
  bat.b_inst = (long long)(c->st_Bt / sizeof(Op));
  bat.c_inst = (long long)(c->st_O / sizeof(TC));
  bat.amax_inst = 2;
  const GemmBatch* batp = ng > 1 ? &bat : nullptr;
  for (long long ch = 0; ch < nchunks; ++ch) {
    long long r = ch;
    for (int i = no - 1; i >= 0; --i) {
      kcnt[i] = (int)(r % chi[trans[i]]);
      r /= chi[trans[i]];
    }
    ops_scope = new PhaseScope(c, PH_OPERANDS);
    for (int j = 0; j < ng; ++j) {
      const Slot S = slot(c, j);
      const int inst = G.inst[j];
      const Z2Layout* L = c->z2L + inst;
      launch_z2_chunk(L, c->z2ev_new + inst * kMaxD, no, no > 0 ? trans[0] : 0, kcnt[0], no > 1 ? trans[1] : 0,
                      kcnt[1], ldO, S.z2blk, S.z2pi, c->z2flops, mixed ? npass : 1, s);
      if (no == 0) {
        if (f16) launch_absmax<double>(G.T1[j], P, P, P, S.amax + 1, s);
        launch_build_y_z2<double, Op>(G.T1[j], pl(S.Y, y_plane, 1, S.amax), ldz, g, a, S.z2rank, S.z2kcol, L,
                                      S.z2pi, s);
      } else {
        TC* X1 = static_cast<TC*>(S.X1);
        TC* X2 = static_cast<TC*>(S.X2);
        // the mode product that writes X also measures max |X|, the fp16 scale bound of Y
        if (kcnt[0] != prev_k0)
          launch_mode_unprimed<double, TC>(G.T1[j], X1, g, trans[0], Ub(j, trans[0]), kcnt[0], s, nullptr, nullptr,
                                           (f16 && no == 1) ? S.amax + 1 : nullptr);
        const TC* X = X1;
        if (no >= 2) {
          launch_mode_unprimed<TC, TC>(X1, X2, g, trans[1], Ub(j, trans[1]), kcnt[1], s, nullptr, nullptr,
                                       f16 ? S.amax + 1 : nullptr);
          X = X2;
        }
        launch_build_y_z2<TC, Op>(X, pl(S.Y, y_plane, 1, S.amax), ldz, g, a, S.z2rank, S.z2kcol, L, S.z2pi, s);
      }
    }
    if (no > 0) prev_k0 = kcnt[0];
    delete ops_scope;
    {
      PhaseScope gemm_scope(c, PH_GEMM);
      if constexpr (mixed) {
        const int rc = launch_gemm_split(pl(S0.Y, y_plane, 1, S0.amax), ldz, pl(S0.Bt, bt_plane, 0, S0.amax), ldz,
                                         static_cast<float*>(S0.O), ldO, P, ldO, ldz, npass, c->status, c->timeout_s,
                                         s, c->kblock, c->group_m, fold_group_for(c, npass), S0.z2blk, batp, false,
                                         c->cta_group);
        if (rc) return rc;
        // what the autotuner replays: slot 0's operands and block descriptor of this chunk
        c->last_gemm.M = P;
        c->last_gemm.N = ldO;
        c->last_gemm.K = ldz;
        c->last_gemm.ldk = ldz;
        c->last_gemm.npass = npass;
        c->last_gemm.nparts = planes;
        c->last_gemm.fmt = f16 ? 1 : 0;
        c->last_gemm.mult_b = bt_mult;
        c->last_gemm.blk = S0.z2blk;
      } else {
        launch_gemm_f64(pl(S0.Y, y_plane, 1, S0.amax).p[0], ldz, pl(S0.Bt, bt_plane, 0, S0.amax).p[0], ldz,
                        static_cast<double*>(S0.O), ldO, P, ldO, ldz, s, S0.z2blk, batp);
      }
      // the blocks' flops are counted on the device (k_z2_chunk)
      if (c->timing) {
        ++c->t_gemm_launches;
        c->t_z2 = true;
      }
    }
    PhaseScope epi_scope(c, PH_EPILOGUE);
    long long out_base = 0;
    for (int i = 0; i < no; ++i) out_base += (long long)kcnt[i] * gn.Sn[trans[i]] * gn.P;
    for (int j = 0; j < ng; ++j) {
      const Slot S = slot(c, j);
      const Z2Layout* L = c->z2L + G.inst[j];
      const TC* O = static_cast<TC*>(S.O);
      std::vector<Ax> axes;
      for (int b = 0; b < c->d; ++b) axes.push_back({g.D[b], g.Sn[b] * ldO, 0, b});
      axes.push_back({chi3, P, 1, -1});
      for (int b = 0; b < c->d; ++b) axes.push_back({g.D[b], g.Sn[b], 2, b});
      TC* bufs[2] = {static_cast<TC*>(S.R1), static_cast<TC*>(S.R2)};
      long long fs[kMaxAxes];
      if (no == 0) {
        final_strides(axes, c3, c3, gn, c3, fs);
        contract_axes_z2<TC, double>(axes, O, ldO, G.out[j], c3, chi3, Ub(j, c3), fs, out_base, L, S.z2pi, s);
        continue;
      }
      contract_axes_z2<TC, TC>(axes, O, ldO, bufs[0], trans[0], chi[trans[0]], Ub(j, trans[0]), nullptr, 0, L,
                               S.z2pi, s);
      const TC* cur = bufs[0];
      for (int i = 1; i < no; ++i) {
        contract_axes<TC, TC>(axes, cur, bufs[i], trans[i], chi[trans[i]], Ub(j, trans[i]), nullptr, 0, s);
        cur = bufs[i];
      }
      final_strides(axes, c3, c3, gn, c3, fs);
      contract_axes<TC, double>(axes, cur, G.out[j], c3, chi3, Ub(j, c3), fs, out_base, s);
    }
  }
  return HOTRG_OK;
}

}  // namespace

// ================================================================= C ABI
extern "C" {

void hotrg_opts_default(hotrg_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = HOTRG_FP64;
  o->fp64_steps = 2;
  o->x6_steps = 0;
  o->batch = 1;
  o->max_steps = 64;
  o->kblock = 64;
  o->graphs = 1;
  o->wait_timeout_s = 4.0;
  o->max_sweeps = 40;
}

int hotrg_workspace_size(int d, int Dcut, const hotrg_opts* opt, size_t* bytes) {
  if (!bytes || d < 1 || d > kMaxD || Dcut < 2 || Dcut > kMaxBond) return HOTRG_EINVAL;
  hotrg_opts def;
  hotrg_opts_default(&def);
  if (!opt) opt = &def;
  if (opt->batch < 1 || opt->max_steps < 1 || opt->max_steps > 64 || opt->group < 0) return HOTRG_EINVAL;
  if (opt->precision < HOTRG_FP64 || opt->precision > HOTRG_FP16X4) return HOTRG_EINVAL;
  if (opt->derivatives < 0 || opt->derivatives > 2) return HOTRG_EINVAL;
  hotrg_ctx c;
  c.d = d;
  c.Dcut = Dcut;
  c.batch = opt->batch;
  c.precision = opt->precision;
  c.fp64_steps = opt->fp64_steps;
  c.x6_steps = opt->x6_steps;
  c.max_steps = opt->max_steps;
  c.deriv = opt->derivatives != 0;
  c.deriv_mode = opt->derivatives;
  c.impure = opt->impurities != 0;
  c.z2 = opt->z2 != 0;
  c.group = group_for(opt);
  *bytes = carve(&c, nullptr);
  return HOTRG_OK;
}

int hotrg_init(hotrg_ctx** out, int d, double beta, double h, int Dcut, const hotrg_opts* opt) {
  if (!out || !opt) return HOTRG_EINVAL;
  *out = nullptr;
  if (d < 1 || d > kMaxD || Dcut < 2 || Dcut > kMaxBond || opt->batch < 1) return HOTRG_EINVAL;
  if (opt->max_steps < 1 || opt->max_steps > 64 || opt->fp64_steps < 0) return HOTRG_EINVAL;
  if (opt->kblock != 0 && opt->kblock != 32 && opt->kblock != 64) return HOTRG_EINVAL;
  if (opt->fold_group < 0) return HOTRG_EINVAL;
  if (opt->precision < HOTRG_FP64 || opt->precision > HOTRG_FP16X4) return HOTRG_EINVAL;
  if (opt->derivatives < 0 || opt->derivatives > 2) return HOTRG_EINVAL;
  if (opt->max_sweeps < 0 || opt->max_sweeps > 1000) return HOTRG_EINVAL;
  if (opt->cta_group < 0 || opt->cta_group > 2) return HOTRG_EINVAL;
  if (opt->group < 0) return HOTRG_EINVAL;
  std::vector<double> vb(opt->batch), vh(opt->batch);
  for (int i = 0; i < opt->batch; ++i) {
    vb[i] = opt->beta ? opt->beta[i] : beta;
    vh[i] = opt->h ? opt->h[i] : h;
    if (!(vb[i] > 0.0) || !std::isfinite(vb[i]) || !std::isfinite(vh[i])) return HOTRG_EINVAL;
    // the block structure holds only at zero field, and not for tangents or impurities in h
    if (opt->z2 && vh[i] != 0.0) return HOTRG_EINVAL;
  }
  if (opt->z2 && (opt->derivatives || opt->impurities || d < 2)) return HOTRG_EINVAL;
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    cudaGetLastError();
    return HOTRG_EDEVICE;
  }
  if (!(prop.major == 10 && prop.minor == 3)) return HOTRG_EDEVICE;
  prepare_kernel_attributes();
  prepare_eig_attributes();
  hotrg_ctx* c = new hotrg_ctx();
  c->d = d;
  c->Dcut = Dcut;
  c->batch = opt->batch;
  c->precision = opt->precision;
  c->fp64_steps = opt->fp64_steps;
  c->x6_steps = opt->x6_steps;
  c->max_steps = opt->max_steps;
  c->kblock = opt->kblock ? opt->kblock : 64;
  c->kblock_fixed = opt->kblock != 0;
  c->fold_group = opt->fold_group;
  c->graphs = opt->graphs != 0;
  c->deriv = opt->derivatives != 0;
  c->deriv_mode = opt->derivatives;
  c->impure = opt->impurities != 0;
  c->z2 = opt->z2 != 0;
  c->z2_opt = c->z2;
  c->z2_inst.assign(opt->batch, c->z2 ? 1 : 0);
  c->group = group_for(opt);
  c->timeout_s = opt->wait_timeout_s > 0 ? opt->wait_timeout_s : 4.0;
  c->max_sweeps = opt->max_sweeps > 0 ? opt->max_sweeps : 40;
  // the faster of the two at the Dcut = 10 shapes: pairs for the two-block squeeze (A rows of a block
  // fit L2), single CTAs for the dense one
  c->cta_group = opt->cta_group ? opt->cta_group : (c->z2 ? 2 : 1);
  c->cta_group_fixed = opt->cta_group != 0;
  c->stream = static_cast<cudaStream_t>(opt->stream);
  c->beta = vb;
  c->h = vh;
  const size_t need = carve(c, nullptr);
  if (!opt->workspace || opt->workspace_bytes < need ||
      (reinterpret_cast<uintptr_t>(opt->workspace) % kAlign)) {
    delete c;
    return HOTRG_ENOMEM;
  }
  carve(c, static_cast<char*>(opt->workspace));
  for (int b = 0; b < d; ++b) c->dims[b] = 2;
  cudaStream_t s = c->stream;
  cudaMemsetAsync(c->status, 0, sizeof(int) * 32, s);
  cudaMemsetAsync(c->dstep, 0, sizeof(int) * 32, s);
  cudaMemsetAsync(c->L, 0, sizeof(double) * c->batch, s);
  cudaMemsetAsync(c->lnc_log, 0, sizeof(double) * c->batch * (c->max_steps + 1), s);
  cudaMemsetAsync(c->spec_log, 0, sizeof(double) * c->batch * c->spec_stride, s);
  cudaMemcpyAsync(c->dbeta, vb.data(), sizeof(double) * c->batch, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(c->dh, vh.data(), sizeof(double) * c->batch, cudaMemcpyHostToDevice, s);
  const long long P2 = c->Pmax * c->Pmax;
  if (c->z2) {
    // every initial leg: index 0 even, index 1 odd
    std::vector<int> ones((size_t)kMaxD * c->batch, 1);
    cudaMemcpyAsync(c->z2ev, ones.data(), sizeof(int) * ones.size(), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(c->z2ev_new, ones.data(), sizeof(int) * ones.size(), cudaMemcpyHostToDevice, s);
    cudaStreamSynchronize(s);
  }
  launch_init_tensor(c->T, P2, c->batch, d, c->dbeta, c->dh, s);
  if (c->impure)
    for (int w = 0; w < 2; ++w) launch_init_tensor(c->SI + w * P2 * c->batch, P2, c->batch, d, c->dbeta, c->dh, s, 1);
  const long long n0 = 1LL << (2 * d);
  Geom g = make_geom(d, c->dims);
  if (c->deriv) {
    cudaMemsetAsync(c->dL, 0, sizeof(double) * 2 * c->batch, s);
    for (int w = 0; w < 2; ++w) launch_init_tangent(c->dT + w * P2 * c->batch, P2, c->batch, d, c->dbeta, c->dh, w, s);
  }
  for (int i = 0; i < c->batch; ++i) {
    double* Ti = c->T + i * P2;
    launch_norm_log(Ti, n0, c->norm_partial, c->cval + i, c->lnc_log + (long long)i * (c->max_steps + 1),
                    c->L + i, c->dstep, c->status, s);
    if (c->deriv)
      for (int w = 0; w < 2; ++w) {
        double* dTi = c->dT + (w * c->batch + i) * P2;
        launch_tangent_norm(Ti, dTi, nullptr, dTi, n0, c->cval + i, c->norm_partial, c->dlnc + w * c->batch + i,
                            c->dL + w * c->batch + i, c->dstep, s);
      }
    launch_scale(Ti, Ti, n0, c->cval + i, s);
    for (int w = 0; c->impure && w < 2; ++w) {
      double* Si = c->SI + (w * c->batch + i) * P2;
      launch_scale(Si, Si, n0, c->cval + i, s);
    }
  }
  launch_trace_x(c->T, P2, c->batch, g, d - 1, c->L, c->dstep, c->out3, s);
  for (int w = 0; c->impure && w < 2; ++w)
    launch_trace_ratio(c->SI + w * P2 * c->batch, c->T, P2, c->batch, g.P, c->imp_out + w * c->batch, s);
  if (c->deriv)
    for (int w = 0; w < 2; ++w)
      launch_trace_tangent(c->T, c->dT + w * P2 * c->batch, P2, c->batch, g.P, c->dL + w * c->batch, c->dstep,
                           c->dout + w * c->batch, s);
  if (cuda_err(c)) {
    delete c;
    return HOTRG_EDEVICE;
  }
  *out = c;
  return HOTRG_OK;
}

// Enqueue one step along axis a on the context's stream (all instances).
static int enqueue_step(hotrg_ctx* c, int a, int step) {
  Geom g = make_geom(c->d, c->dims);
  int chi[kMaxD], trans[kMaxD], nt = 0, nd[kMaxD];
  for (int b = 0; b < c->d; ++b) {
    nd[b] = c->dims[b];
    chi[b] = c->dims[b];
    if (b != a) {
      const long long sq = (long long)c->dims[b] * c->dims[b];
      chi[b] = (int)(sq < c->Dcut ? sq : c->Dcut);
      nd[b] = chi[b];
      trans[nt++] = b;
    }
  }
  Geom gn = make_geom(c->d, nd);
  const int planes = planes_for_step(c->precision, step, c->fp64_steps, c->x6_steps, g.P);
  const int npass = passes_for_step(c->precision, step, c->fp64_steps, c->x6_steps, g.P);
  cudaStream_t s = c->stream;
  const long long P2max = c->Pmax * c->Pmax;
  PhaseScope step_scope(c, PH_STEP);
  launch_step_advance(c->dstep, s);
  // 1. isometries of every instance (batched launches: one CTA group per instance)
  {
    PhaseScope iso_scope(c, PH_ISO);
    const int* zev = c->z2 ? c->z2ev : nullptr;
    if (c->deriv_mode != 2 && nt > 0) {
      // every transverse axis' Gram matrix, then one eigensolver launch for all of them
      EigAxes ea;
      ea.nt = nt;
      ea.max_sweeps = c->max_sweeps;
      ea.g_stride = c->g_stride;
      ea.u_stride = c->u_stride;
      ea.out = EigOut{nullptr, c->spec_stride, (long long)c->d * kSpecCap, c->dstep, c->max_steps};
      for (int t = 0; t < nt; ++t) {
        const int b = trans[t];
        double* Gb = c->G + (long long)b * (c->g_stride / kMaxD);
        launch_half_gram(c->T, P2max, c->batch, g, b, c->d + a, c->gpartial, c->Q1, c->q_stride, s, nullptr, zev);
        launch_half_gram(c->T, P2max, c->batch, g, b, a, c->gpartial, c->Q2, c->q_stride, s, nullptr, zev);
        launch_gram_combine(c->Q1, c->Q2, c->q_stride, c->batch, g.D[b], g.D[a], Gb, c->g_stride, s);
        ea.ax[t] = EigAxis{Gb, g.D[b] * g.D[b], chi[b], b, g.D[b], c->spec_log + (long long)b * kSpecCap,
                           c->U + (long long)b * kMaxBond * kMaxGram, c->ework + t * c->ework_axis};
      }
      launch_eig_axes(ea, c->batch, c->status, s, zev, c->z2ev_new);
    }
    for (int t = 0; t < nt && c->deriv_mode == 2; ++t) {
      const int b = trans[t];
      const int n = g.D[b] * g.D[b];
      double* Gb = c->G + (long long)b * (c->g_stride / kMaxD);
      double* Ub = c->U + (long long)b * kMaxBond * kMaxGram;
      launch_half_gram(c->T, P2max, c->batch, g, b, c->d + a, c->gpartial, c->Q1, c->q_stride, s, nullptr, zev);
      launch_half_gram(c->T, P2max, c->batch, g, b, a, c->gpartial, c->Q2, c->q_stride, s, nullptr, zev);
      launch_gram_combine(c->Q1, c->Q2, c->q_stride, c->batch, g.D[b], g.D[a], Gb, c->g_stride, s);
      EigOut eo{c->spec_log + (long long)b * kSpecCap, c->spec_stride, (long long)c->d * kSpecCap, c->dstep,
                c->max_steps};
      launch_eig(Gb, c->g_stride, c->batch, n, chi[b], eo, Ub, c->u_stride, c->ework, c->status, s,
                 c->z2 ? c->z2ev : nullptr, c->z2ev_new, b, g.D[b], c->max_sweeps);
      if (c->deriv_mode == 2)
        for (int w = 0; w < 2; ++w) {
          // dG from the half-Gram tangents, then dU from the eigensystem still in ework
          const double* dTw = c->dT + w * P2max * c->batch;
          launch_half_gram(c->T, P2max, c->batch, g, b, c->d + a, c->gpartial, c->H1, c->q_stride, s, dTw);
          launch_half_gram(c->T, P2max, c->batch, g, b, a, c->gpartial, c->H2, c->q_stride, s, dTw);
          launch_gram_combine_tangent(c->Q1, c->Q2, c->H1, c->H2, c->q_stride, c->batch, g.D[b], g.D[a], c->dG,
                                      c->dg_stride, s);
          launch_eig_tangent(c->ework, Ub, c->u_stride, c->dG, c->dg_stride, c->batch, n, chi[b],
                             c->dU + w * c->u_stride * c->batch + (long long)b * kMaxBond * kMaxGram, s);
        }
    }
  }
  // 2-4. squeeze (groups of instances: one GEMM launch per chunk for the whole group), normalise
  // and accumulate instance by instance
  for (int i0 = 0; i0 < c->batch; i0 += c->group) {
    const int ng = std::min(c->group, c->batch - i0);
    Group grp;
    for (int j = 0; j < ng; ++j) {
      const double* Ti = c->T + (i0 + j) * P2max;
      grp.add(Ti, Ti, c->U + (i0 + j) * c->u_stride, slot(c, j).Tnext, i0 + j);
    }
    Tangents tg;  // the group is a single instance when there are tangents (group_for)
    if (c->deriv) {
      tg.n = 2;
      for (int w = 0; w < 2; ++w) {
        tg.dT[w] = c->dT + (w * c->batch + i0) * P2max;
        tg.dout[w] = w ? c->D2 : c->D1;
        tg.dU[w] = c->deriv_mode == 2 ? c->dU + (w * c->batch + i0) * c->u_stride : nullptr;
      }
    }
    int rc = (c->z2 && nt > 0)
                 ? (planes ? squeeze_z2<float>(c, grp, g, gn, a, chi, trans, nt, planes, npass)
                           : squeeze_z2<double>(c, grp, g, gn, a, chi, trans, nt, 0, 0))
             : planes ? squeeze<float>(c, grp, g, gn, a, chi, trans, nt, planes, npass, tg)
                      : squeeze<double>(c, grp, g, gn, a, chi, trans, nt, 0, 0, tg);
    if (rc) return rc;
    // impure tensors with the pure flow's isometries (a group of one): the pair merges with itself
    // at step 1 (Eq. (SS)) and with a pure site after (Eq. (ST)); the single spin always with a pure
    // site
    for (int w = 0; c->impure && w < 2; ++w) {
      const double* Si = c->SI + (w * c->batch + i0) * P2max;
      const double* partner = (w == 0 && step == 1) ? Si : grp.T1[0];
      Group imp;
      imp.add(Si, partner, grp.U[0], c->Stmp + w * P2max, i0);
      rc = planes ? squeeze<float>(c, imp, g, gn, a, chi, trans, nt, planes, npass)
                  : squeeze<double>(c, imp, g, gn, a, chi, trans, nt, 0, 0);
      if (rc) return rc;
    }
    for (int j = 0; j < ng; ++j) {
      const int i = i0 + j;
      const double* Tn = grp.out[j];
      double* Tw = c->T + i * P2max;
      {
        PhaseScope norm_scope(c, PH_NORM);
        launch_norm_log(Tn, gn.P * gn.P, c->norm_partial, c->cval + i, c->lnc_log + (long long)i * (c->max_steps + 1),
                        c->L + i, c->dstep, c->status, s);
      }
      // tangent of T' / ||T'||
      for (int w = 0; w < tg.n; ++w) {
        double* dTi = c->dT + (w * c->batch + i) * P2max;
        launch_tangent_norm(Tn, tg.dout[w], nullptr, dTi, gn.P * gn.P, c->cval + i, c->norm_partial,
                            c->dlnc + w * c->batch + i, c->dL + w * c->batch + i, c->dstep, s);
      }
      launch_scale(Tn, Tw, gn.P * gn.P, c->cval + i, s);
      for (int w = 0; c->impure && w < 2; ++w)
        launch_scale(c->Stmp + w * P2max, c->SI + (w * c->batch + i) * P2max, gn.P * gn.P, c->cval + i, s);
    }
  }
  launch_trace_x(c->T, P2max, c->batch, gn, a, c->L, c->dstep, c->out3, s);
  for (int w = 0; c->impure && w < 2; ++w)
    launch_trace_ratio(c->SI + w * P2max * c->batch, c->T, P2max, c->batch, gn.P, c->imp_out + w * c->batch, s);
  if (c->z2) {
    unsigned mask = 0;
    for (int t = 0; t < nt; ++t) mask |= 1u << trans[t];
    launch_z2_advance(c->z2ev, c->z2ev_new, c->batch, mask, s);
  }
  if (c->deriv)
    for (int w = 0; w < 2; ++w)
      launch_trace_tangent(c->T, c->dT + w * P2max * c->batch, P2max, c->batch, gn.P, c->dL + w * c->batch,
                           c->dstep, c->dout + w * c->batch, s);
  if (c->timing) {
    double f = 2.0 * (double)g.P * (double)g.P * (double)g.P * c->batch;
    for (int t = 0; t < nt; ++t) f *= chi[trans[t]];
    c->t_dense_step_flops += f;
    // parity-blocked steps add what their GEMM blocks computed, counted on the device
    if (!(c->z2 && nt > 0)) c->t_step_flops += f;
    ++c->t_steps;
  }
  return HOTRG_OK;
}

int hotrg_step(hotrg_ctx* c, int axis) {
  if (!c) return HOTRG_EINVAL;
  if (c->sticky) return c->sticky;
  if (axis < -1 || axis >= c->d) return HOTRG_EINVAL;
  if (c->steps >= c->max_steps) return HOTRG_ESTATE;
  const int a = axis >= 0 ? axis : c->d - 1 - (c->steps % c->d);
  const int step = c->steps + 1;
  int nd[kMaxD];
  bool steady = true;
  long long P = 1;
  for (int b = 0; b < c->d; ++b) {
    nd[b] = c->dims[b];
    P *= c->dims[b];
    if (b != a) {
      const long long sq = (long long)c->dims[b] * c->dims[b];
      nd[b] = (int)(sq < c->Dcut ? sq : c->Dcut);
      if (nd[b] != c->dims[b]) steady = false;
    }
  }
  const int pl = passes_for_step(c->precision, step, c->fp64_steps, c->x6_steps, P);
  int rc = HOTRG_OK;
  // graphs need a capturable stream: not the legacy default stream
  if (c->graphs && steady && !c->timing && c->stream != nullptr) {
    // a steady-state step is the same launch sequence every time: capture it once per axis
    bool hit = c->graph_exec[a] && c->graph_planes[a] == pl;
    for (int b = 0; hit && b < c->d; ++b) hit = c->graph_dims[a][b] == c->dims[b];
    if (!hit) {
      if (c->graph_exec[a]) cudaGraphExecDestroy(c->graph_exec[a]);
      c->graph_exec[a] = nullptr;
      cudaGraph_t graph = nullptr;
      if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return c->sticky = HOTRG_EDEVICE;
      }
      rc = enqueue_step(c, a, step);
      const cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
      if (rc) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return c->sticky = rc;
      }
      if (e != cudaSuccess || cudaGraphInstantiate(&c->graph_exec[a], graph, 0) != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return c->sticky = HOTRG_EDEVICE;
      }
      cudaGraphDestroy(graph);
      c->graph_planes[a] = pl;
      for (int b = 0; b < c->d; ++b) c->graph_dims[a][b] = c->dims[b];
    }
    if (cudaGraphLaunch(c->graph_exec[a], c->stream) != cudaSuccess) {
      cudaGetLastError();
      return c->sticky = HOTRG_EDEVICE;
    }
  } else {
    rc = enqueue_step(c, a, step);
    if (rc) {
      cudaGetLastError();
      return c->sticky = rc;
    }
  }
  if (cuda_err(c)) return HOTRG_EDEVICE;
  // a dense step writes its bonds in plain descending order and no even counts: no instance keeps
  // a known block layout after it
  if (!c->z2) std::fill(c->z2_inst.begin(), c->z2_inst.end(), 0);
  for (int b = 0; b < c->d; ++b) c->hist_dims[step - 1][b] = c->dims[b];
  c->hist_axis[step - 1] = a;
  for (int b = 0; b < c->d; ++b) c->dims[b] = nd[b];
  c->steps = step;
  c->last_axis = a;
  return HOTRG_OK;
}

int hotrg_free_energy(hotrg_ctx* c, double* lnz, double* f) {
  if (!c) return HOTRG_EINVAL;
  const int rc = sync_check(c);
  if (rc) return rc;
  std::vector<double> o3(3 * c->batch);
  if (cudaMemcpy(o3.data(), c->out3, sizeof(double) * 3 * c->batch, cudaMemcpyDeviceToHost) != cudaSuccess)
    return c->sticky = HOTRG_EDEVICE;
  for (int i = 0; i < c->batch; ++i) {
    if (!(o3[3 * i] > 0.0)) return HOTRG_ENUMERIC;  // the flow state itself stays valid
    if (lnz) lnz[i] = o3[3 * i + 1];
    if (f) f[i] = -o3[3 * i + 1] / c->beta[i];
  }
  return HOTRG_OK;
}

int hotrg_observables(hotrg_ctx* c, int instance, hotrg_obs* out) {
  if (!c || !out || instance < 0 || instance >= c->batch) return HOTRG_EINVAL;
  const int rc = sync_check(c);
  if (rc) return rc;
  double o3[3], lc = 0.0;
  if (cudaMemcpy(o3, c->out3 + 3 * instance, sizeof(o3), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(&lc, c->lnc_log + (long long)instance * (c->max_steps + 1) + c->steps, sizeof(double),
                 cudaMemcpyDeviceToHost) != cudaSuccess)
    return c->sticky = HOTRG_EDEVICE;
  out->steps = c->steps;
  out->last_axis = c->last_axis;
  out->lnz_per_site = o3[1];
  out->last_ln_c = lc;
  out->x_indicator = c->steps ? o3[2] : 1.0;
  out->dlnz_dbeta = out->dlnz_dh = out->internal_energy = out->magnetization = std::nan("");
  if (c->deriv) {
    double db = 0.0, dh = 0.0;
    if (cudaMemcpy(&db, c->dout + instance, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&dh, c->dout + c->batch + instance, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
      return c->sticky = HOTRG_EDEVICE;
    out->dlnz_dbeta = db;
    out->dlnz_dh = dh;
    out->internal_energy = -db;                 // <H>/N with H = -sum s s' - h sum s
    out->magnetization = dh / c->beta[instance];  // <s>
  }
  out->nn_correlation = out->spin = std::nan("");
  if (c->impure) {
    double r[2] = {0.0, 0.0};
    for (int w = 0; w < 2; ++w)
      if (cudaMemcpy(r + w, c->imp_out + w * c->batch + instance, sizeof(double), cudaMemcpyDeviceToHost) !=
          cudaSuccess)
        return c->sticky = HOTRG_EDEVICE;
    if (c->steps > 0) out->nn_correlation = r[0];  // the pair exists only after the first merge
    out->spin = r[1];
  }
  return HOTRG_OK;
}

int hotrg_spectra(hotrg_ctx* c, int step, int axis, int instance, double* buf, int cap, int* n_out) {
  if (!c || !n_out || step < 1 || step > c->steps || axis < 0 || axis >= c->d || instance < 0 ||
      instance >= c->batch || cap < 0 || (cap > 0 && !buf))
    return HOTRG_EINVAL;
  const int rc = sync_check(c);
  if (rc) return rc;
  const int n = (axis == c->hist_axis[step - 1]) ? 0 : c->hist_dims[step - 1][axis] * c->hist_dims[step - 1][axis];
  std::vector<double> tmp(kSpecCap);
  const double* src = c->spec_log + instance * c->spec_stride + ((long long)(step - 1) * c->d + axis) * kSpecCap;
  if (n > 0 && cudaMemcpy(tmp.data(), src, sizeof(double) * n, cudaMemcpyDeviceToHost) != cudaSuccess)
    return c->sticky = HOTRG_EDEVICE;
  *n_out = n;
  for (int i = 0; i < n && i < cap; ++i) buf[i] = tmp[i];
  return HOTRG_OK;
}

int hotrg_ln_norms(hotrg_ctx* c, int instance, double* buf, int cap, int* n_out) {
  if (!c || !n_out || instance < 0 || instance >= c->batch || cap < 0 || (cap > 0 && !buf))
    return HOTRG_EINVAL;
  const int rc = sync_check(c);
  if (rc) return rc;
  const int n = c->steps + 1;
  std::vector<double> tmp(n);
  if (cudaMemcpy(tmp.data(), c->lnc_log + (long long)instance * (c->max_steps + 1), sizeof(double) * n,
                 cudaMemcpyDeviceToHost) != cudaSuccess)
    return c->sticky = HOTRG_EDEVICE;
  *n_out = n;
  for (int i = 0; i < n && i < cap; ++i) buf[i] = tmp[i];
  return HOTRG_OK;
}

int hotrg_get_tensor(hotrg_ctx* c, int instance, int* dims, double* host, size_t cap) {
  if (!c || instance < 0 || instance >= c->batch) return HOTRG_EINVAL;
  if (dims)
    for (int b = 0; b < c->d; ++b) dims[b] = c->dims[b];
  if (!host) return HOTRG_OK;
  Geom g = make_geom(c->d, c->dims);
  if (cap < (size_t)(g.P * g.P)) return HOTRG_EINVAL;
  const int rc = sync_check(c);
  if (rc) return rc;
  if (cudaMemcpy(host, c->T + instance * c->Pmax * c->Pmax, sizeof(double) * g.P * g.P,
                 cudaMemcpyDeviceToHost) != cudaSuccess)
    return c->sticky = HOTRG_EDEVICE;
  return HOTRG_OK;
}

int hotrg_set_tensor(hotrg_ctx* c, int instance, const int* dims, const double* host) {
  if (!c || !dims || !host || instance < 0 || instance >= c->batch) return HOTRG_EINVAL;
  if (c->sticky) return c->sticky;
  for (int b = 0; b < c->d; ++b)
    if (dims[b] < 1 || dims[b] > c->Dcut) return HOTRG_EINVAL;
  // all instances share the bond dimensions
  if (c->batch > 1)
    for (int b = 0; b < c->d; ++b)
      if (dims[b] != c->dims[b]) return HOTRG_EINVAL;
  Geom g = make_geom(c->d, dims);
  // the tensor slot holds Pmax^2 entries (the largest state the workspace plan reaches)
  if (g.P > c->Pmax) return HOTRG_EINVAL;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess ||
      cudaMemcpy(c->T + instance * c->Pmax * c->Pmax, host, sizeof(double) * g.P * g.P,
                 cudaMemcpyHostToDevice) != cudaSuccess)
    return c->sticky = HOTRG_EDEVICE;
  // a tensor supplied from outside does not depend on (beta, h): its tangents are zero
  for (int w = 0; c->deriv && w < 2; ++w)
    if (cudaMemsetAsync(c->dT + (w * c->batch + instance) * c->Pmax * c->Pmax, 0, sizeof(double) * g.P * g.P,
                        c->stream) != cudaSuccess)
      return c->sticky = HOTRG_EDEVICE;
  // an arbitrary tensor need not have the zero-field block structure: use the dense squeeze
  // (for every instance: they share the launches)
  if (c->z2_opt) c->z2_inst[instance] = 0;
  c->z2 = false;
  drop_graphs(c);
  // nor does it carry impurities: the impure estimates restart from zero
  for (int w = 0; c->impure && w < 2; ++w)
    if (cudaMemsetAsync(c->SI + (w * c->batch + instance) * c->Pmax * c->Pmax, 0, sizeof(double) * g.P * g.P,
                        c->stream) != cudaSuccess)
      return c->sticky = HOTRG_EDEVICE;
  for (int b = 0; b < c->d; ++b) c->dims[b] = dims[b];
  return HOTRG_OK;
}

int hotrg_set_tensor_z2(hotrg_ctx* c, int instance, const int* dims, const int* evens, const double* host) {
  if (!c || !dims || !evens || !host || instance < 0 || instance >= c->batch) return HOTRG_EINVAL;
  if (c->sticky) return c->sticky;
  if (!c->z2_opt) return HOTRG_ESTATE;
  for (int b = 0; b < c->d; ++b)
    if (dims[b] < 1 || dims[b] > c->Dcut || evens[b] < 0 || evens[b] > dims[b]) return HOTRG_EINVAL;
  if (c->batch > 1)
    for (int b = 0; b < c->d; ++b)
      if (dims[b] != c->dims[b]) return HOTRG_EINVAL;
  Geom g = make_geom(c->d, dims);
  if (g.P > c->Pmax) return HOTRG_EINVAL;
  // the block structure must hold exactly: every entry with odd total leg parity is zero
  std::vector<int> upar(g.P);
  for (long long u = 0; u < g.P; ++u) {
    int par = 0;
    for (int b = 0; b < c->d; ++b) par ^= ((u / g.Sn[b]) % g.D[b]) >= evens[b] ? 1 : 0;
    upar[u] = par;
  }
  for (long long u = 0; u < g.P; ++u)
    for (long long q = 0; q < g.P; ++q)
      if ((upar[u] ^ upar[q]) && host[u * g.P + q] != 0.0) return HOTRG_EINVAL;
  int ev[kMaxD] = {1, 1, 1, 1};
  for (int b = 0; b < c->d; ++b) ev[b] = evens[b];
  if (cudaStreamSynchronize(c->stream) != cudaSuccess ||
      cudaMemcpy(c->T + instance * c->Pmax * c->Pmax, host, sizeof(double) * g.P * g.P,
                 cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->z2ev + instance * kMaxD, ev, sizeof(ev), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->z2ev_new + instance * kMaxD, ev, sizeof(ev), cudaMemcpyHostToDevice) != cudaSuccess)
    return c->sticky = HOTRG_EDEVICE;
  // the block-sparse squeeze resumes only once every instance is known to be structured (an
  // instance given a dense tensor by hotrg_set_tensor, or stepped densely since, is not)
  c->z2_inst[instance] = 1;
  c->z2 = std::all_of(c->z2_inst.begin(), c->z2_inst.end(), [](char v) { return v != 0; });
  drop_graphs(c);
  for (int b = 0; b < c->d; ++b) c->dims[b] = dims[b];
  return HOTRG_OK;
}

// ---- checkpoint format: header, then per instance T (P^2), L, lnc_log, spec_log, out3
struct StateHeader {
  char magic[8];
  int version, d, Dcut, batch, precision, max_steps, steps, last_axis, deriv, impure, z2;
  int dims[kMaxD];
  long long P;
  int hist_dims[64][kMaxD];
  int hist_axis[64];
};

// Bytes saved per instance: T, L, the ln c log, the spectra, out3 and, with tangents, for each
// of the two parameters dT, dL and the derivative of ln Z / N.
size_t state_per_instance(const hotrg_ctx* c, long long P) {
  size_t n = (size_t)P * P + 1 + (c->max_steps + 1) + c->spec_stride + 3;
  if (c->deriv) n += 2 * ((size_t)P * P + 2);
  if (c->impure) n += 2 * ((size_t)P * P + 1);
  // with the block-sparse squeeze: the legs' even-value counts
  return sizeof(double) * n + (c->z2_opt ? sizeof(int) * kMaxD : 0);
}

int hotrg_state_size(hotrg_ctx* c, size_t* bytes) {
  if (!c || !bytes) return HOTRG_EINVAL;
  Geom g = make_geom(c->d, c->dims);
  *bytes = sizeof(StateHeader) + state_per_instance(c, g.P) * c->batch;
  return HOTRG_OK;
}

int hotrg_state_save(hotrg_ctx* c, void* host, size_t cap) {
  size_t need = 0;
  if (hotrg_state_size(c, &need) || !host || cap < need) return HOTRG_EINVAL;
  const int rc = sync_check(c);
  if (rc) return rc;
  StateHeader h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, "HOTRGST", 8);
  h.version = 3;
  h.z2 = c->z2 ? 1 : 0;
  h.deriv = c->deriv ? c->deriv_mode : 0;
  h.impure = c->impure ? 1 : 0;
  h.d = c->d; h.Dcut = c->Dcut; h.batch = c->batch; h.precision = c->precision;
  h.max_steps = c->max_steps; h.steps = c->steps; h.last_axis = c->last_axis;
  for (int b = 0; b < kMaxD; ++b) h.dims[b] = c->dims[b];
  std::memcpy(h.hist_dims, c->hist_dims, sizeof(h.hist_dims));
  std::memcpy(h.hist_axis, c->hist_axis, sizeof(h.hist_axis));
  Geom g = make_geom(c->d, c->dims);
  h.P = g.P;
  char* p = static_cast<char*>(host);
  std::memcpy(p, &h, sizeof(h));
  p += sizeof(h);
  for (int i = 0; i < c->batch; ++i) {
    bool ok = cudaMemcpy(p, c->T + i * c->Pmax * c->Pmax, sizeof(double) * g.P * g.P, cudaMemcpyDeviceToHost) == cudaSuccess;
    p += sizeof(double) * g.P * g.P;
    ok = ok && cudaMemcpy(p, c->L + i, sizeof(double), cudaMemcpyDeviceToHost) == cudaSuccess;
    p += sizeof(double);
    ok = ok && cudaMemcpy(p, c->lnc_log + (long long)i * (c->max_steps + 1), sizeof(double) * (c->max_steps + 1),
                          cudaMemcpyDeviceToHost) == cudaSuccess;
    p += sizeof(double) * (c->max_steps + 1);
    ok = ok && cudaMemcpy(p, c->spec_log + i * c->spec_stride, sizeof(double) * c->spec_stride,
                          cudaMemcpyDeviceToHost) == cudaSuccess;
    p += sizeof(double) * c->spec_stride;
    ok = ok && cudaMemcpy(p, c->out3 + 3 * i, sizeof(double) * 3, cudaMemcpyDeviceToHost) == cudaSuccess;
    p += sizeof(double) * 3;
    for (int w = 0; c->deriv && w < 2; ++w) {
      const long long j = w * c->batch + i;
      ok = ok && cudaMemcpy(p, c->dT + j * c->Pmax * c->Pmax, sizeof(double) * g.P * g.P,
                            cudaMemcpyDeviceToHost) == cudaSuccess;
      p += sizeof(double) * g.P * g.P;
      ok = ok && cudaMemcpy(p, c->dL + j, sizeof(double), cudaMemcpyDeviceToHost) == cudaSuccess;
      p += sizeof(double);
      ok = ok && cudaMemcpy(p, c->dout + j, sizeof(double), cudaMemcpyDeviceToHost) == cudaSuccess;
      p += sizeof(double);
    }
    for (int w = 0; c->impure && w < 2; ++w) {
      const long long j = w * c->batch + i;
      ok = ok && cudaMemcpy(p, c->SI + j * c->Pmax * c->Pmax, sizeof(double) * g.P * g.P,
                            cudaMemcpyDeviceToHost) == cudaSuccess;
      p += sizeof(double) * g.P * g.P;
      ok = ok && cudaMemcpy(p, c->imp_out + j, sizeof(double), cudaMemcpyDeviceToHost) == cudaSuccess;
      p += sizeof(double);
    }
    if (c->z2_opt) {
      ok = ok && cudaMemcpy(p, c->z2ev + i * kMaxD, sizeof(int) * kMaxD, cudaMemcpyDeviceToHost) == cudaSuccess;
      p += sizeof(int) * kMaxD;
    }
    if (!ok) return c->sticky = HOTRG_EDEVICE;
  }
  return HOTRG_OK;
}

int hotrg_state_load(hotrg_ctx* c, const void* host, size_t size) {
  if (!c || !host || size < sizeof(StateHeader)) return HOTRG_EINVAL;
  StateHeader h;
  std::memcpy(&h, host, sizeof(h));
  if (std::memcmp(h.magic, "HOTRGST", 8) || h.version != 3 || h.d != c->d || h.Dcut != c->Dcut ||
      h.batch != c->batch || h.precision != c->precision || h.max_steps != c->max_steps ||
      h.deriv != (c->deriv ? c->deriv_mode : 0) || h.impure != (c->impure ? 1 : 0) || (h.z2 && !c->z2_opt))
    return HOTRG_EINVAL;
  Geom g = make_geom(h.d, h.dims);
  if (g.P != h.P || g.P > c->Pmax) return HOTRG_EINVAL;
  if (size < sizeof(StateHeader) + state_per_instance(c, g.P) * c->batch) return HOTRG_EINVAL;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return c->sticky = HOTRG_EDEVICE;
  const char* p = static_cast<const char*>(host) + sizeof(h);
  for (int i = 0; i < c->batch; ++i) {
    bool ok = cudaMemcpy(c->T + i * c->Pmax * c->Pmax, p, sizeof(double) * g.P * g.P, cudaMemcpyHostToDevice) == cudaSuccess;
    p += sizeof(double) * g.P * g.P;
    ok = ok && cudaMemcpy(c->L + i, p, sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess;
    p += sizeof(double);
    ok = ok && cudaMemcpy(c->lnc_log + (long long)i * (c->max_steps + 1), p, sizeof(double) * (c->max_steps + 1),
                          cudaMemcpyHostToDevice) == cudaSuccess;
    p += sizeof(double) * (c->max_steps + 1);
    ok = ok && cudaMemcpy(c->spec_log + i * c->spec_stride, p, sizeof(double) * c->spec_stride,
                          cudaMemcpyHostToDevice) == cudaSuccess;
    p += sizeof(double) * c->spec_stride;
    ok = ok && cudaMemcpy(c->out3 + 3 * i, p, sizeof(double) * 3, cudaMemcpyHostToDevice) == cudaSuccess;
    p += sizeof(double) * 3;
    for (int w = 0; c->deriv && w < 2; ++w) {
      const long long j = w * c->batch + i;
      ok = ok && cudaMemcpy(c->dT + j * c->Pmax * c->Pmax, p, sizeof(double) * g.P * g.P,
                            cudaMemcpyHostToDevice) == cudaSuccess;
      p += sizeof(double) * g.P * g.P;
      ok = ok && cudaMemcpy(c->dL + j, p, sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess;
      p += sizeof(double);
      ok = ok && cudaMemcpy(c->dout + j, p, sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess;
      p += sizeof(double);
    }
    for (int w = 0; c->impure && w < 2; ++w) {
      const long long j = w * c->batch + i;
      ok = ok && cudaMemcpy(c->SI + j * c->Pmax * c->Pmax, p, sizeof(double) * g.P * g.P,
                            cudaMemcpyHostToDevice) == cudaSuccess;
      p += sizeof(double) * g.P * g.P;
      ok = ok && cudaMemcpy(c->imp_out + j, p, sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess;
      p += sizeof(double);
    }
    if (c->z2_opt) {
      ok = ok && cudaMemcpy(c->z2ev + i * kMaxD, p, sizeof(int) * kMaxD, cudaMemcpyHostToDevice) == cudaSuccess;
      ok = ok && cudaMemcpy(c->z2ev_new + i * kMaxD, p, sizeof(int) * kMaxD, cudaMemcpyHostToDevice) == cudaSuccess;
      p += sizeof(int) * kMaxD;
    }
    if (!ok) return c->sticky = HOTRG_EDEVICE;
  }
  if (cudaMemcpy(c->dstep, &h.steps, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
    return c->sticky = HOTRG_EDEVICE;
  for (int b = 0; b < kMaxD; ++b) c->dims[b] = h.dims[b];
  std::memcpy(c->hist_dims, h.hist_dims, sizeof(h.hist_dims));
  std::memcpy(c->hist_axis, h.hist_axis, sizeof(h.hist_axis));
  c->steps = h.steps;
  c->last_axis = h.last_axis;
  c->z2 = h.z2 != 0;
  std::fill(c->z2_inst.begin(), c->z2_inst.end(), c->z2 ? 1 : 0);
  drop_graphs(c);
  return HOTRG_OK;
}

int hotrg_timing_start(hotrg_ctx* c) {
  if (!c) return HOTRG_EINVAL;
  if (c->sticky) return c->sticky;
  for (auto& e : c->evs) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  c->evs.clear();
  c->timing = true;
  c->launch0 = launches_total();
  c->t_gemm_launches = c->t_steps = 0;
  c->t_gemm_flops = c->t_gemm_tflops = c->t_step_flops = c->t_dense_step_flops = 0;
  c->t_z2 = false;
  if (c->z2flops && cudaMemsetAsync(c->z2flops, 0, sizeof(double) * 2, c->stream) != cudaSuccess)
    return c->sticky = HOTRG_EDEVICE;
  return HOTRG_OK;
}

int hotrg_timing_stop(hotrg_ctx* c, hotrg_timing* out) {
  if (!c || !out) return HOTRG_EINVAL;
  const int rc = sync_check(c);
  c->timing = false;
  if (rc) return rc;
  double ms[PH_COUNT] = {0, 0, 0, 0, 0, 0};
  for (auto& e : c->evs) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, e.a, e.b) == cudaSuccess) ms[e.phase] += t;
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  c->evs.clear();
  std::memset(out, 0, sizeof(*out));
  out->ms_step = ms[PH_STEP];
  out->ms_isometry = ms[PH_ISO];
  out->ms_operands = ms[PH_OPERANDS];
  out->ms_gemm = ms[PH_GEMM];
  out->ms_epilogue = ms[PH_EPILOGUE];
  out->ms_norm = ms[PH_NORM];
  out->steps = c->t_steps;
  out->gemm_launches = c->t_gemm_launches;
  out->kernel_launches = launches_total() - c->launch0;
  out->gemm_flops = c->t_gemm_flops;
  out->gemm_tensor_flops = c->t_gemm_tflops;
  out->step_flops = c->t_step_flops;
  out->dense_step_flops = c->t_dense_step_flops;
  if (c->t_z2 && c->z2flops) {
    double zf[2] = {0.0, 0.0};
    if (cudaMemcpy(zf, c->z2flops, sizeof(zf), cudaMemcpyDeviceToHost) != cudaSuccess)
      return c->sticky = HOTRG_EDEVICE;
    out->gemm_flops += zf[0];
    out->gemm_tensor_flops += zf[1];
    out->step_flops += zf[0];
  }
  cudaGetLastError();
  return HOTRG_OK;
}

int hotrg_autotune(hotrg_ctx* c, hotrg_tuning* out) {
  if (!c) return HOTRG_EINVAL;
  const int rc = sync_check(c);
  if (rc) return rc;
  const auto& lg = c->last_gemm;
  if (lg.npass == 0) return HOTRG_ESTATE;  // no split-precision step has run yet
  Planes<__nv_bfloat16> Y, Bt;
  Y.nparts = Bt.nparts = lg.nparts;
  if (lg.fmt == 1) {  // the fp16 planes and scale bounds the last step's GEMM used
    Y.fmt = Bt.fmt = 1;
    Y.amax = c->amax + 1;
    Bt.amax = c->amax + 0;
    Bt.amax_mult = lg.mult_b;
  }
  for (int k = 0; k < 3; ++k) {
    const int kk = k < lg.nparts ? k : 0;
    Y.p[k] = static_cast<__nv_bfloat16*>(c->Y) + (size_t)kk * lg.M * lg.ldk;
    Bt.p[k] = static_cast<__nv_bfloat16*>(c->Bt) + (size_t)kk * lg.N * lg.ldk;
  }
  // candidates keep the hi*hi chain between folds at most 64 K: (k-block 64, 1 per fold),
  // (32, 1) or (32, 2)
  std::vector<int> kbs;
  if (lg.npass == 6) kbs = {32};
  else if (c->kblock_fixed) kbs = {c->kblock};
  else kbs = {64, 32};
  const int groups[5] = {4, 8, 16, 32, 64};
  std::vector<int> cgs;
  if (c->cta_group_fixed) cgs = {c->cta_group};
  else cgs = {2, 1};
  struct Cand {
    int kb, fg, gm, cg;
  };
  std::vector<Cand> cands;
  for (int cg : cgs)
    for (int kb : kbs)
      for (int fg = 1; fg <= (kb == 32 ? 2 : 1); ++fg)
        for (int gm : groups) cands.push_back({kb, fg, gm, cg});
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return HOTRG_EDEVICE;
  double best = 1e300;
  int best_kb = c->kblock, best_g = c->group_m, best_fg = std::max(1, c->fold_group), best_cg = c->cta_group;
  for (const Cand& cd : cands) {
    double t_min = 1e300;
    for (int rep = 0; rep < 2; ++rep) {
      cudaEventRecord(e0, c->stream);
      const int r = launch_gemm_split(Y, lg.ldk, Bt, lg.ldk, static_cast<float*>(c->O), lg.N, lg.M, lg.N, lg.K,
                                      lg.npass, c->status, c->timeout_s, c->stream, cd.kb, cd.gm, cd.fg, lg.blk,
                                      nullptr, false, cd.cg);
      cudaEventRecord(e1, c->stream);
      float ms = 0.f;
      if (r || cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaGetLastError();
        return r ? r : (c->sticky = HOTRG_EDEVICE);
      }
      t_min = std::min(t_min, (double)ms);
    }
    if (t_min < best) {
      best = t_min;
      best_kb = cd.kb;
      best_g = cd.gm;
      best_fg = cd.fg;
      best_cg = cd.cg;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const int rc2 = sync_check(c);
  if (rc2) return rc2;
  // a six-product GEMM always runs 32-wide k-blocks: tuning it must not change the k-block of the
  // two-plane steps that follow
  if (lg.npass != 6) c->kblock = best_kb;
  c->group_m = best_g;
  c->fold_group = best_fg;
  c->cta_group = best_cg;
  for (int a = 0; a < kMaxD; ++a)
    if (c->graph_exec[a]) {
      cudaGraphExecDestroy(c->graph_exec[a]);  // captured with the previous choice
      c->graph_exec[a] = nullptr;
    }
  if (out) {
    out->kblock = best_kb;
    out->group_m = best_g;
    out->fold_group = best_fg;
    out->ms = best;
    out->cta_group = best_cg;
  }
  return HOTRG_OK;
}

void hotrg_destroy(hotrg_ctx* c) {
  if (!c) return;
  for (int a = 0; a < kMaxD; ++a)
    if (c->graph_exec[a]) cudaGraphExecDestroy(c->graph_exec[a]);
  for (auto& e : c->evs) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  delete c;
}

const char* hotrg_strerror(int code) {
  switch (code) {
    case HOTRG_OK: return "ok";
    case HOTRG_EINVAL: return "invalid argument";
    case HOTRG_ENOMEM: return "workspace too small or misaligned";
    case HOTRG_ENUMERIC: return "numerical failure (NaN/Inf, zero norm or non-positive trace)";
    case HOTRG_ENOCONV: return "eigensolver did not converge";
    case HOTRG_ETIMEOUT: return "a bounded device-side wait gave up";
    case HOTRG_EDEVICE: return "CUDA device error or no sm_103 device";
    case HOTRG_ESTATE: return "call not valid in the current state";
    case HOTRG_ENOTSUP: return "not supported by this library";
    default: return "unknown error";
  }
}

// ---- kernel-level GEMM entry point
size_t hotrg_gemm_scratch_bytes(long long M, long long N, long long K) {
  if (M <= 0 || N <= 0 || K <= 0) return 0;
  const long long ld = round_up(K, 64);
  return (size_t)kAlign + 3 * (size_t)round_up(M * ld * 2, kAlign) + 3 * (size_t)round_up(N * ld * 2, kAlign);
}

int hotrg_gemm_split(const float* A, long long lda, const float* Bt, long long ldb, float* C, long long ldc,
                     long long M, long long N, long long K, int npass, int kblock, int fold_group, void* scratch,
                     size_t scratch_bytes, void* stream) {
  if (fold_group < 0) return HOTRG_EINVAL;
  if (!A || !Bt || !C || !scratch || lda < K || ldb < K || ldc < N) return HOTRG_EINVAL;
  if (kblock == 0) kblock = 64;
  if (kblock != 32 && kblock != 64) return HOTRG_EINVAL;
  if (npass != 1 && npass != 3 && npass != 4 && npass != 6) return HOTRG_EINVAL;
  if (scratch_bytes < hotrg_gemm_scratch_bytes(M, N, K) || (reinterpret_cast<uintptr_t>(scratch) % kAlign))
    return HOTRG_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long ld = round_up(K, 64);
  char* p = static_cast<char*>(scratch);
  int* status = reinterpret_cast<int*>(p);
  p += kAlign;
  const int nparts = npass == 1 ? 1 : (npass == 6 ? 3 : 2);
  Planes<__nv_bfloat16> Ap, Bp;
  Ap.nparts = Bp.nparts = nparts;
  for (int k = 0; k < 3; ++k) {
    Ap.p[k] = reinterpret_cast<__nv_bfloat16*>(p);
    p += round_up(M * ld * 2, kAlign);
  }
  for (int k = 0; k < 3; ++k) {
    Bp.p[k] = reinterpret_cast<__nv_bfloat16*>(p);
    p += round_up(N * ld * 2, kAlign);
  }
  cudaMemsetAsync(status, 0, sizeof(int), s);
  launch_split_rows(A, lda, M, K, Ap, ld, s);
  launch_split_rows(Bt, ldb, N, K, Bp, ld, s);
  const int fg = fold_group > 0 ? fold_group : 1;
  const int rc = launch_gemm_split(Ap, ld, Bp, ld, C, ldc, M, N, K, npass, status, 4.0, s, kblock, 16, fg);
  if (rc) return rc;
  return cudaGetLastError() == cudaSuccess ? HOTRG_OK : HOTRG_EDEVICE;
}

int hotrg_gemm_split_f16(const float* A, long long lda, const float* Bt, long long ldb, float* C, long long ldc,
                         long long M, long long N, long long K, int npass, int kblock, int fold_group, void* scratch,
                         size_t scratch_bytes, void* stream) {
  if (fold_group < 0) return HOTRG_EINVAL;
  if (!A || !Bt || !C || !scratch || lda < K || ldb < K || ldc < N) return HOTRG_EINVAL;
  if (kblock == 0) kblock = 64;
  if (kblock != 32 && kblock != 64) return HOTRG_EINVAL;
  if (npass != 1 && npass != 3 && npass != 4) return HOTRG_EINVAL;
  if (scratch_bytes < hotrg_gemm_scratch_bytes(M, N, K) || (reinterpret_cast<uintptr_t>(scratch) % kAlign))
    return HOTRG_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long ld = round_up(K, 64);
  char* p = static_cast<char*>(scratch);
  int* status = reinterpret_cast<int*>(p);
  unsigned* amax = reinterpret_cast<unsigned*>(p + 64);  // [0] max |A|, [1] max |Bt|
  p += kAlign;
  const int nparts = npass == 1 ? 1 : 2;
  Planes<__nv_bfloat16> Ap, Bp;
  Ap.nparts = Bp.nparts = nparts;
  Ap.fmt = Bp.fmt = 1;
  Ap.amax = amax;
  Bp.amax = amax + 1;
  for (int k = 0; k < 3; ++k) {
    Ap.p[k] = reinterpret_cast<__nv_bfloat16*>(p);
    p += round_up(M * ld * 2, kAlign);
  }
  for (int k = 0; k < 3; ++k) {
    Bp.p[k] = reinterpret_cast<__nv_bfloat16*>(p);
    p += round_up(N * ld * 2, kAlign);
  }
  cudaMemsetAsync(status, 0, sizeof(int), s);
  launch_absmax<float>(A, M, K, lda, amax, s);
  launch_absmax<float>(Bt, N, K, ldb, amax + 1, s);
  launch_split_rows(A, lda, M, K, Ap, ld, s);
  launch_split_rows(Bt, ldb, N, K, Bp, ld, s);
  const int fg = fold_group > 0 ? fold_group : 1;
  const int rc = launch_gemm_split(Ap, ld, Bp, ld, C, ldc, M, N, K, npass, status, 4.0, s, kblock, 16, fg);
  if (rc) return rc;
  return cudaGetLastError() == cudaSuccess ? HOTRG_OK : HOTRG_EDEVICE;
}

size_t hotrg_gemm_wait_probe_bytes(void) {
  return hotrg_gemm_scratch_bytes(TC_PROBE_M, TC_PROBE_N, TC_PROBE_K) + sizeof(float) * TC_PROBE_M * TC_PROBE_N;
}

int hotrg_gemm_wait_probe(double timeout_s, void* scratch, size_t scratch_bytes, void* stream) {
  if (!scratch || !(timeout_s > 0.0) || timeout_s > 10.0) return HOTRG_EINVAL;
  if (scratch_bytes < hotrg_gemm_wait_probe_bytes() || (reinterpret_cast<uintptr_t>(scratch) % kAlign))
    return HOTRG_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long M = TC_PROBE_M, N = TC_PROBE_N, K = TC_PROBE_K;
  char* p = static_cast<char*>(scratch);
  int* status = reinterpret_cast<int*>(p);
  p += kAlign;
  Planes<__nv_bfloat16> Ap, Bp;
  Ap.nparts = Bp.nparts = 2;
  for (int k = 0; k < 3; ++k) {
    Ap.p[k] = reinterpret_cast<__nv_bfloat16*>(p);
    p += round_up(M * K * 2, kAlign);
  }
  for (int k = 0; k < 3; ++k) {
    Bp.p[k] = reinterpret_cast<__nv_bfloat16*>(p);
    p += round_up(N * K * 2, kAlign);
  }
  float* C = reinterpret_cast<float*>(p);
  // one CTA per tile, then a CTA pair (whose waits span both CTAs and end at a cluster barrier)
  for (int cg = 1; cg <= 2; ++cg) {
    if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) return HOTRG_EDEVICE;
    const int rc = launch_gemm_split(Ap, K, Bp, K, C, N, M, N, K, 3, status, timeout_s, s, 64, 16, 1, nullptr,
                                     nullptr, true, cg);
    if (rc) return rc;
    const int st = hotrg_gemm_status(scratch, stream);
    if (st != HOTRG_ETIMEOUT) return st;
  }
  return HOTRG_ETIMEOUT;
}

int hotrg_gemm_status(const void* scratch, void* stream) {
  if (!scratch) return HOTRG_EINVAL;
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return HOTRG_EDEVICE;
  int bits = 0;
  if (cudaMemcpy(&bits, scratch, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return HOTRG_EDEVICE;
  return status_to_code(bits);
}

}  // extern "C"
