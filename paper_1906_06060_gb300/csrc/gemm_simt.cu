// FP64 squeeze GEMM on the CUDA cores: C[m][n] = sum_k A[m][k] Bt[n][k] (both operands K-major).
// This is the plain FP64 path of the O(Dcut^15) contraction (arXiv:1906.06060 Sec. 2 cost
// statement). 64 x 64 output tiles, K chunks of 16, 4 x 4 register blocking per thread.
#include "kernels.h"

namespace hotrg {

namespace {

constexpr int BM = 64, BN = 64, BK = 16;

// With blk (block-sparse product), blockIdx.z picks the block: its rows [m0, m0+mc), columns
// [n0, n0+nc) and k range [k0, k0+kc); CTAs whose tile lies outside the block return at once.
// Batched launch: blockIdx.z / nbz is the instance (operands and output at its strides, its own
// blocks blk[instance]), blockIdx.z % nbz the block (nbz = 2 with blocks, else 1).
__global__ void __launch_bounds__(256) k_gemm_f64(const double* __restrict__ A, long long lda,
                                                  const double* __restrict__ Bt, long long ldb,
                                                  double* __restrict__ C, long long ldc, long long M,
                                                  long long N, long long K, const GemmBlocks* __restrict__ blk,
                                                  long long a_inst, long long b_inst, long long c_inst) {
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int nbz = blk ? 2 : 1;
  const int inst = blockIdx.z / nbz;
  A += inst * a_inst;
  Bt += inst * b_inst;
  C += inst * c_inst;
  if (blk) blk += inst;
  long long mb = 0, nb = 0, kb = 0;
  if (blk) {
    const int b = blockIdx.z % nbz;
    if (b >= blk->nb) return;
    mb = min((long long)max(blk->m0[b], 0), M);
    nb = min((long long)max(blk->n0[b], 0), N);
    kb = min((long long)max(blk->k0[b], 0), K);
    const long long mc = min((long long)max(blk->mc[b], 0), M - mb);
    const long long nc = min((long long)max(blk->nc[b], 0), N - nb);
    const long long kc = min((long long)max(blk->kc[b], 0), K - kb);
    if ((long long)blockIdx.y * BM >= mc || (long long)blockIdx.x * BN >= nc) return;
    M = mb + mc;
    N = nb + nc;
    K = kb + kc;
  }
  const long long m0 = mb + (long long)blockIdx.y * BM, n0 = nb + (long long)blockIdx.x * BN;
  const int tx = tid % 16, ty = tid / 16;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (long long k0 = kb; k0 < K; k0 += BK) {
#pragma unroll
    for (int q = 0; q < (BM * BK) / 256; ++q) {
      const int e = tid + 256 * q;
      const int kk = e % BK, rr = e / BK;
      const long long k = k0 + kk;
      const long long m = m0 + rr, n = n0 + rr;
      As[kk][rr] = (m < M && k < K) ? A[m * lda + k] : 0.0;
      Bs[kk][rr] = (n < N && k < K) ? Bt[n * ldb + k] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const long long m = m0 + ty * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const long long n = n0 + tx * 4 + j;
      if (n < N) C[m * ldc + n] = acc[i][j];
    }
  }
}

}  // namespace

void launch_gemm_f64(const double* A, long long lda, const double* Bt, long long ldb, double* C,
                     long long ldc, long long M, long long N, long long K, cudaStream_t s, const GemmBlocks* blk,
                     const GemmBatch* bat) {
  // block-sparse: enough tiles for a block as large as the whole product, two blocks; batched:
  // that for every instance
  const int batch = bat ? bat->batch : 1;
  dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((M + BM - 1) / BM), (unsigned)(batch * (blk ? 2 : 1)));
  k_gemm_f64<<<grid, 256, 0, s>>>(A, lda, Bt, ldb, C, ldc, M, N, K, blk, bat ? bat->a_inst : 0,
                                  bat ? bat->b_inst : 0, bat ? bat->c_inst : 0);
  count_launches(1);
}

}  // namespace hotrg
