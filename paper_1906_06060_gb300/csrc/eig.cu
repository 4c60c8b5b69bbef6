// FP64 symmetric eigensolver for the Gram matrices (n = D_b^2 <= 256), one CTA per matrix.
//
// Method: cyclic two-sided Jacobi with the round-robin (tournament) parallel ordering of
// Brent & Luk (1985): each round rotates n/2 disjoint (p, q) pairs at once, n - 1 rounds make a
// sweep. Rotation angle as in Rutishauser's formulation (tan of the angle from
// theta = (a_qq - a_pp) / (2 a_pq)), so that a'_pq = 0, a'_pp = a_pp - t a_pq, a'_qq = a_qq + t a_pq.
// Converged when a whole sweep finds no off-diagonal entry above the rotation threshold
// (|a_pq| > 1e-18 sqrt|a_pp a_qq| and > 2^-53 ||A||_F: below that an entry is rounding noise of
// the matrix and rotating it changes no eigenvector beyond working precision).
// Then (arXiv:1906.06060 Sec. 2 / HOTRG truncation): eigenvalues sorted descending (stable),
// the first chi eigenvectors kept, each sign-fixed so its largest-magnitude component is
// positive (lowest index on a tie).
#include "kernels.h"

namespace hotrg {

namespace {

constexpr int kEigThreads = 512;

// Sort key of an eigenvalue: NaN (a Gram matrix of a tensor holding NaN) orders below every number,
// so that the ranks computed from it always form a permutation of 0..n-1 (ties by index).
__device__ __forceinline__ double order_key(double x) { return isnan(x) ? -INFINITY : x; }

__device__ void sm_red_sum(double* sred, double v, int tid) {
  sred[tid] = v;
  __syncthreads();
  for (int w = kEigThreads / 2; w > 0; w >>= 1) {
    if (tid < w) sred[tid] += sred[tid + w];
    __syncthreads();
  }
}

// One CTA per (instance = blockIdx.x, axis = blockIdx.y): the Gram matrices of all transverse
// axes of a step are diagonalised in one launch.
__global__ void __launch_bounds__(kEigThreads) k_jacobi(EigAxes ea, int* status, const int* z2_ev, int* z2_ev_new) {
  extern __shared__ double sm[];
  const EigAxis& ax = ea.ax[blockIdx.y];
  const int n = ax.n, chi = ax.chi, z2_axis = ax.z2_axis, Db = ax.Db > 0 ? ax.Db : 1;
  const double* G = ax.G + (long long)blockIdx.x * ea.g_stride;
  double* Uout = ax.U + (long long)blockIdx.x * ea.u_stride;
  double* work = ax.work + (long long)blockIdx.x * 2 * n * n;
  const EigOut& o = ea.out;
  // eigenvalue log slot of this instance for the current step (device step counter, 1-based)
  const int step = o.step ? *o.step : 1;
  double* evals = (step >= 1 && step <= o.max_steps)
                      ? ax.evals + (long long)blockIdx.x * o.inst_stride + (long long)(step - 1) * o.step_stride
                      : nullptr;
  const int tid = threadIdx.x;
  const int np = n + (n & 1);          // padded to even (index n is a dummy)
  const int npairs = np / 2;
  // shared: per-pair data
  int* sp = reinterpret_cast<int*>(sm);                   // [128] p
  int* sq = sp + 128;                                     // [128] q
  double* sc = sm + 128;                                  // [128] c
  double* ss = sc + 128;                                  // [128] s
  double* st = ss + 128;                                  // [128] t
  double* sred = st + 128;                                // [kEigThreads] reduction

  double* A = work;                    // n x n
  double* V = work + (long long)n * n; // n x n
  for (int e = tid; e < n * n; e += kEigThreads) {
    A[e] = G[e];
    V[e] = (e / n == e % n) ? 1.0 : 0.0;
  }
  __syncthreads();

  // matrix scale for the absolute rotation threshold
  {
    double f = 0.0;
    for (int e = tid; e < n * n; e += kEigThreads) f += A[e] * A[e];
    sm_red_sum(sred, f, tid);
  }
  const double floor_abs = 0x1p-53 * sqrt(sred[0]);
  __syncthreads();
  __shared__ int s_rot;
  int sweep = 0;
  for (;; ++sweep) {
    if (tid == 0) s_rot = 0;
    if (sweep >= ea.max_sweeps) {
      if (tid == 0) atomic_status(status, ST_NOCONV);
      break;
    }
    __syncthreads();
    for (int round = 0; round < np - 1; ++round) {
      if (tid < npairs) {
        auto player = [&](int pos) { return pos == 0 ? 0 : ((pos - 1 + round) % (np - 1)) + 1; };
        int p = player(tid), q = player(np - 1 - tid);
        if (p > q) { int x = p; p = q; q = x; }
        double c = 1.0, s = 0.0, t = 0.0;
        if (q < n) {
          const double apq = A[(long long)p * n + q];
          const double app = A[(long long)p * n + p], aqq = A[(long long)q * n + q];
          if (fabs(apq) > floor_abs && fabs(apq) > 1e-18 * sqrt(fabs(app * aqq))) {
            s_rot = 1;
            const double theta = (aqq - app) / (2.0 * apq);
            t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(1.0 + theta * theta));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
          }
        } else {
          p = q = -1;
        }
        sp[tid] = p; sq[tid] = q; sc[tid] = c; ss[tid] = s; st[tid] = t;
      }
      __syncthreads();
      // columns: A <- A J, V <- V J
      for (int e = tid; e < npairs * n; e += kEigThreads) {
        const int k = e / n, r = e % n;
        const int p = sp[k], q = sq[k];
        if (p < 0 || ss[k] == 0.0) continue;
        const double c = sc[k], s = ss[k];
        const double arp = A[(long long)r * n + p], arq = A[(long long)r * n + q];
        A[(long long)r * n + p] = c * arp - s * arq;
        A[(long long)r * n + q] = s * arp + c * arq;
        const double vrp = V[(long long)r * n + p], vrq = V[(long long)r * n + q];
        V[(long long)r * n + p] = c * vrp - s * vrq;
        V[(long long)r * n + q] = s * vrp + c * vrq;
      }
      __syncthreads();
      // rows: A <- J^T A
      for (int e = tid; e < npairs * n; e += kEigThreads) {
        const int k = e / n, r = e % n;
        const int p = sp[k], q = sq[k];
        if (p < 0 || ss[k] == 0.0) continue;
        const double c = sc[k], s = ss[k];
        const double apr = A[(long long)p * n + r], aqr = A[(long long)q * n + r];
        A[(long long)p * n + r] = c * apr - s * aqr;
        A[(long long)q * n + r] = s * apr + c * aqr;
      }
      __syncthreads();
    }
    const int rotated = s_rot;
    __syncthreads();  // every thread has read the flag before it is reset
    if (!rotated) break;  // a full sweep without a rotation: converged
  }
  // eigenvalues and ranks (descending, stable in the index)
  double* lam = sred;  // reuse: n <= 256 <= kEigThreads
  for (int i = tid; i < n; i += kEigThreads) {
    lam[i] = A[(long long)i * n + i];
    if (isnan(lam[i])) atomic_status(status, ST_NUMERIC);
  }
  __syncthreads();
  int* perm = sp;      // reuse 256 ints (sp and sq are contiguous)
  for (int i = tid; i < n; i += kEigThreads) {
    const double li = order_key(lam[i]);
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const double lj = order_key(lam[j]);
      rank += (lj > li) || (lj == li && j < i);
    }
    perm[rank] = i;
  }
  __syncthreads();
  if (evals)
    for (int k = tid; k < n; k += kEigThreads) evals[k] = lam[perm[k]];
  // sign-fixed eigenvectors: one warp per kept vector
  const int warp = tid / 32, lane = tid % 32;
  // zero-field block structure: parity of fused index r = (b1, b2) of this axis
  const int ez = z2_ev ? z2_ev[blockIdx.x * kMaxD + z2_axis] : 0;
  auto rpar = [&](int r) { return ((r / Db) >= ez ? 1 : 0) ^ ((r % Db) >= ez ? 1 : 0); };
  int* kpar = reinterpret_cast<int*>(sc);       // [chi] parity of kept vector k (sc, ss, st are free)
  int* kpos = reinterpret_cast<int*>(ss);       // [chi] its output row
  for (int k = warp; k < chi; k += kEigThreads / 32) {
    const int col = perm[k];
    double best = -1.0;
    int bidx = 0;  // stays a valid row when every entry is NaN (no comparison succeeds)
    for (int r = lane; r < n; r += 32) {
      const double a = fabs(V[(long long)r * n + col]);
      if (a > best) { best = a; bidx = r; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
      if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; }
    }
    if (z2_ev) {
      // the vector must live in one parity sector: the other sector's weight is exactly zero
      const int pk = rpar(bidx);
      double bad = 0.0;
      for (int r = lane; r < n; r += 32)
        if (rpar(r) != pk) bad += V[(long long)r * n + col] * V[(long long)r * n + col];
      for (int o = 16; o > 0; o >>= 1) bad += __shfl_xor_sync(0xffffffffu, bad, o);
      if (lane == 0) {
        kpar[k] = pk;
        if (bad > 1e-24) atomic_status(status, ST_Z2);
      }
    }
  }
  __syncthreads();
  if (z2_ev && tid == 0) {
    // even vectors first, each group in descending eigenvalue order
    int ne = 0;
    for (int k = 0; k < chi; ++k) ne += kpar[k] == 0;
    int ie = 0, io = ne;
    for (int k = 0; k < chi; ++k) kpos[k] = kpar[k] == 0 ? ie++ : io++;
    z2_ev_new[blockIdx.x * kMaxD + z2_axis] = ne;
  }
  __syncthreads();
  for (int k = warp; k < chi; k += kEigThreads / 32) {
    const int col = perm[k];
    double best = -1.0;
    int bidx = 0;  // stays a valid row when every entry is NaN (no comparison succeeds)
    for (int r = lane; r < n; r += 32) {
      const double a = fabs(V[(long long)r * n + col]);
      if (a > best) { best = a; bidx = r; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
      if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; }
    }
    const double sgn = V[(long long)bidx * n + col] < 0 ? -1.0 : 1.0;
    const int row = z2_ev ? kpos[k] : k;
    for (int r = lane; r < n; r += 32) Uout[(long long)row * n + r] = sgn * V[(long long)r * n + col];
  }
}

// First-order perturbation of the kept eigenvectors (one CTA per instance). work holds the
// Jacobi result of launch_eig: A (diagonal = eigenvalues, unsorted) and V (columns = eigenvectors).
// Shared memory: lambda[n], perm[n], sign[chi], Z = dG V_kept [n][chi], W [(n - chi)][chi].
__global__ void __launch_bounds__(256) k_eig_tangent(const double* __restrict__ work, const double* __restrict__ U,
                                                     long long u_stride, const double* __restrict__ dG,
                                                     long long g_stride, int n, int chi,
                                                     double* __restrict__ dU) {
  extern __shared__ double sm[];
  work += (long long)blockIdx.x * 2 * n * n;
  U += (long long)blockIdx.x * u_stride;
  dU += (long long)blockIdx.x * u_stride;
  dG += (long long)blockIdx.x * g_stride;
  const double* A = work;
  const double* V = work + (long long)n * n;
  double* lam = sm;                                   // [n]
  double* sgn = lam + n;                              // [chi]
  double* Z = sgn + kMaxBond;                         // [n][chi]
  double* W = Z + (long long)n * chi;                 // [n - chi][chi]
  int* perm = reinterpret_cast<int*>(W + (long long)(n - chi) * chi);  // [n]
  const int tid = threadIdx.x;
  for (int i = tid; i < n; i += blockDim.x) lam[i] = A[(long long)i * n + i];
  __syncthreads();
  // the same descending, index-stable order as launch_eig
  for (int i = tid; i < n; i += blockDim.x) {
    const double li = order_key(lam[i]);
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const double lj = order_key(lam[j]);
      rank += (lj > li) || (lj == li && j < i);
    }
    perm[rank] = i;
  }
  __syncthreads();
  // sign convention of U_k relative to column perm[k] of V: U_k = sign_k V[:, perm[k]]
  const int warp = tid / 32, lane = tid % 32;
  for (int k = warp; k < chi; k += blockDim.x / 32) {
    double dot = 0.0;
    for (int r = lane; r < n; r += 32) dot += U[(long long)k * n + r] * V[(long long)r * n + perm[k]];
    for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
    if (lane == 0) sgn[k] = dot < 0 ? -1.0 : 1.0;
  }
  // Z[r][k] = sum_c dG[r][c] V[c][perm[k]]
  for (int e = tid; e < n * chi; e += blockDim.x) {
    const int r = e / chi, k = e % chi;
    const int col = perm[k];
    double acc = 0.0;
    for (int c2 = 0; c2 < n; ++c2) acc = fma(dG[(long long)r * n + c2], V[(long long)c2 * n + col], acc);
    Z[e] = acc;
  }
  __syncthreads();
  // W[j - chi][k] = (V_j^T Z_k) / (lambda_k - lambda_j)
  for (int e = tid; e < (n - chi) * chi; e += blockDim.x) {
    const int jj = e / chi, k = e % chi;
    const int colj = perm[chi + jj];
    double acc = 0.0;
    for (int r = 0; r < n; ++r) acc = fma(V[(long long)r * n + colj], Z[r * chi + k], acc);
    const double gap = lam[perm[k]] - lam[colj];
    W[e] = gap != 0.0 ? acc / gap : nan("");
  }
  __syncthreads();
  // dU[k][r] = sign_k sum_j V[r][perm[j]] W[j][k]
  for (int e = tid; e < chi * n; e += blockDim.x) {
    const int k = e / n, r = e % n;
    double acc = 0.0;
    for (int jj = 0; jj < n - chi; ++jj) acc = fma(V[(long long)r * n + perm[chi + jj]], W[jj * chi + k], acc);
    dU[(long long)k * n + r] = sgn[k] * acc;
  }
}

}  // namespace

void launch_eig_tangent(const double* work, const double* U, long long u_stride, const double* dG,
                        long long g_stride, int batch, int n, int chi, double* dU, cudaStream_t s) {
  const size_t smem = sizeof(double) * ((size_t)n + kMaxBond + (size_t)n * chi + (size_t)(n - chi) * chi) +
                      sizeof(int) * (size_t)n;
  k_eig_tangent<<<batch, 256, smem, s>>>(work, U, u_stride, dG, g_stride, n, chi, dU);
  count_launches(1);
}

void prepare_eig_attributes() {
  const int big = (int)(sizeof(double) * (kMaxGram + kMaxBond + 2 * kMaxGram * kMaxBond) + sizeof(int) * kMaxGram);
  cudaFuncSetAttribute(k_eig_tangent, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
}

void launch_eig_axes(const EigAxes& ea, int batch, int* status, cudaStream_t s, const int* z2_ev, int* z2_ev_new) {
  if (ea.nt < 1) return;
  const size_t smem = sizeof(double) * (128 + 128 + 128 + 128 + kEigThreads);
  k_jacobi<<<dim3(batch, ea.nt), kEigThreads, smem, s>>>(ea, status, z2_ev, z2_ev_new);
  count_launches(1);
}

void launch_eig(const double* G, long long g_stride, int batch, int n, int chi, const EigOut& o, double* U,
                long long u_stride, double* work, int* status, cudaStream_t s, const int* z2_ev, int* z2_ev_new,
                int z2_axis, int Db, int max_sweeps) {
  EigAxes ea;
  ea.nt = 1;
  ea.max_sweeps = max_sweeps;
  ea.g_stride = g_stride;
  ea.u_stride = u_stride;
  ea.out = o;
  ea.ax[0] = EigAxis{G, n, chi, z2_axis, Db, o.base, U, work};
  const size_t smem = sizeof(double) * (128 + 128 + 128 + 128 + kEigThreads);
  k_jacobi<<<dim3(batch, 1), kEigThreads, smem, s>>>(ea, status, z2_ev, z2_ev_new);
  count_launches(1);
}

}  // namespace hotrg
