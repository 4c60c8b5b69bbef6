// Gram matrices of the two-site unfolding (arXiv:1906.06060 Sec. 2: the isometry U of Eq. (SS)
// comes from the HOSVD of the merged pair; its left factor is the eigenbasis of this Gram matrix).
//
// G_b[(b1 b2), (b1~ b2~)] = sum over every other leg of the merged pair M
//                         = sum_{al, al~} Q1[(b1,al)][(b1~,al~)] Q2[(b2,al)][(b2~,al~)]
// Q1 contracts site 1 over all legs except (u_b, p_a); Q2 site 2 over all except (u_b, u_a).
// Both are X X^T of an unfolding of T with nr = D_b D_a rows and P^2 / nr columns, computed in
// FP64 on the CUDA cores by split-K tiles (edge chosen per nr to waste the least padding; only
// the upper tiles of a symmetric product) and a fixed-order reduction (deterministic).
#include "kernels.h"

namespace hotrg {

namespace {

constexpr int GK = 16;               // column chunk
constexpr int kGramWarps = 152 * 24;  // warps the split-K grid aims at (latency hiding on the FP64 pipe)

struct LegInfo {
  int nrest;                     // number of remaining legs (2d - 2)
  int dim[kMaxLegs];             // remaining legs, natural order
  long long stride[kMaxLegs];
  int ax[kMaxLegs];              // lattice axis of each remaining leg
  int ax1, ax2;                  // axes of the two row legs
};

// Zero-field block structure (ev: the instance's even-value counts per axis, values ordered
// even-parity first): row r = (i1, i2) has parity [i1 >= e1] ^ [i2 >= e2], and a column the
// parity of its legs. Q vanishes between rows of different parity, and a row meets only the
// columns of its own parity: with the rows in parity order (even rows first) each of the two
// diagonal blocks is tiled on its own and sums over its parity's columns only, a quarter of
// the dense work. The class sizes are known on the device only: the grid holds enough tiles for
// a class of nr rows, and tiles beyond the actual class exit at once.
__device__ __forceinline__ int gram_row_par(int r, int Da, int e1, int e2) {
  return ((r / Da) >= e1 ? 1 : 0) ^ ((r % Da) >= e2 ? 1 : 0);
}
// natural row of the s-th row in parity order
__device__ int gram_row_sorted(int s, int nr, int Da, int e1, int e2, int neven) {
  const int want = s < neven ? 0 : 1;
  int k = s < neven ? s : s - neven;
  for (int r = 0; r < nr; ++r)
    if (gram_row_par(r, Da, e1, e2) == want && k-- == 0) return r;
  return 0;
}

// Output tiles of edge GT ((GT/4)^2 threads, 4 x 4 outputs each). With sym (TA = TB: Q is
// symmetric) only the tiles on and above the diagonal are computed; the reduction mirrors the
// rest. Rows of a tile come from TA, columns from TB (both T for the Gram itself; the tangent dT
// and T for its derivative).
template <int GT>
__global__ void __launch_bounds__((GT / 4) * (GT / 4)) k_half_gram(const double* __restrict__ TA,
                                                                   const double* __restrict__ TB, long long t_stride,
                                                                   LegInfo li, long long S1, long long S2, int Da,
                                                                   int nr, long long K, int ntile, int sym,
                                                                   int nsplit, double* __restrict__ partial,
                                                                   const int* __restrict__ ev) {
  constexpr int NT = (GT / 4) * (GT / 4);
  TA += (long long)blockIdx.z * t_stride;
  TB += (long long)blockIdx.z * t_stride;
  partial += (long long)blockIdx.z * nsplit * nr * nr;
  __shared__ double As[GK][GT + 1];
  __shared__ double Bs[GK][GT + 1];
  __shared__ long long coloff[GK];
  __shared__ long long rowoffA[GT], rowoffB[GT];
  // zero-field blocks: per-leg even counts and the column layout of each parity pattern
  __shared__ int e_rest[kMaxLegs];
  __shared__ long long patsz[64];
  const int tid = threadIdx.x;
  int e1 = 0, e2 = 0, neven = nr;
  long long K0 = K;
  int cls = 0, base = 0, ncls = nr;   // parity class of this tile (zero-field) and its row range
  if (ev) {
    ev += blockIdx.z * kMaxD;
    e1 = ev[li.ax1];
    e2 = ev[li.ax2];
    neven = 0;
    for (int r = 0; r < nr; ++r) neven += gram_row_par(r, Da, e1, e2) == 0;
    if (tid < li.nrest) e_rest[tid] = ev[li.ax[tid]];
    __syncthreads();
    const int npat = 1 << li.nrest;
    for (int pat = tid; pat < npat; pat += NT) {
      long long sz = 1;
      for (int l = 0; l < li.nrest; ++l) sz *= ((pat >> l) & 1) ? li.dim[l] - e_rest[l] : e_rest[l];
      patsz[pat] = sz;
    }
    __syncthreads();
    K0 = 0;
    for (int pat = 0; pat < npat; ++pat)
      if ((__popc(pat) & 1) == 0) K0 += patsz[pat];
  }
  const int split = blockIdx.y;
  const int tiles_per_cls = sym ? ntile * (ntile + 1) / 2 : ntile * ntile;
  int t = blockIdx.x;
  if (ev) {
    cls = t / tiles_per_cls;
    t %= tiles_per_cls;
    base = cls ? neven : 0;
    ncls = cls ? nr - neven : neven;
  }
  int tr = 0, tc = 0;
  if (sym) {
    while (t >= ntile - tr) { t -= ntile - tr; ++tr; }
    tc = tr + t;
  } else {
    tr = t / ntile;
    tc = t % ntile;
  }
  // tile rows / columns in class-local sorted order (the whole range without the block structure)
  const int r0 = tr * GT, c0 = tc * GT;
  if (r0 >= ncls || c0 >= ncls) return;  // beyond this instance's class: no output (uniform per CTA)
  long long cs = 0, ce = K;
  const int colcls = ev ? cls : -1;
  if (ev) {
    cs = cls ? K0 : 0;
    ce = cls ? K : K0;
  }
  const long long kper = (ce - cs + nsplit - 1) / nsplit;
  const long long kb = cs + (long long)split * kper;
  const long long ke = min(ce, kb + kper);
  for (int q = tid; q < GT; q += NT) {
    int ra = r0 + q, rb = c0 + q;
    if (ev) {
      ra = ra < ncls ? gram_row_sorted(base + ra, nr, Da, e1, e2, neven) : nr;
      rb = rb < ncls ? gram_row_sorted(base + rb, nr, Da, e1, e2, neven) : nr;
    }
    rowoffA[q] = ra < nr ? (long long)(ra / Da) * S1 + (long long)(ra % Da) * S2 : -1;
    rowoffB[q] = rb < nr ? (long long)(rb / Da) * S1 + (long long)(rb % Da) * S2 : -1;
  }
  const int tx = tid % (GT / 4), ty = tid / (GT / 4);
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  for (long long kc = kb; kc < ke; kc += GK) {
    if (tid < GK) {
      long long col = kc + tid;
      long long off = -1;
      if (col < ke) {
        off = 0;
        if (colcls < 0) {
          for (int l = li.nrest - 1; l >= 0; --l) {
            const long long c = col % li.dim[l];
            col /= li.dim[l];
            off += c * li.stride[l];
          }
        } else {
          // blocked order inside the class: patterns of that parity in increasing order, then
          // row-major inside the pattern's box
          long long local = col - (colcls ? K0 : 0);
          int pat = 0;
          for (; pat < (1 << li.nrest); ++pat) {
            if ((__popc(pat) & 1) != colcls) continue;
            if (local < patsz[pat]) break;
            local -= patsz[pat];
          }
          for (int l = li.nrest - 1; l >= 0; --l) {
            const int bit = (pat >> l) & 1;
            const int dl = bit ? li.dim[l] - e_rest[l] : e_rest[l];
            const long long c = local % dl;
            local /= dl;
            off += (c + (bit ? e_rest[l] : 0)) * li.stride[l];
          }
        }
      }
      coloff[tid] = off;
    }
    __syncthreads();
    for (int e = tid; e < GT * GK; e += NT) {
      const int kk = e % GK, rr = e / GK;
      const long long co = coloff[kk];
      const long long ra = rowoffA[rr], rb = rowoffB[rr];
      As[kk][rr] = (co >= 0 && ra >= 0) ? TA[ra + co] : 0.0;
      Bs[kk][rr] = (co >= 0 && rb >= 0) ? TB[rb + co] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
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
  // partial sums at the rows' positions in parity order (base + class-local index)
  double* out = partial + (long long)split * nr * nr;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = r0 + ty * 4 + i;
    if (r >= ncls) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + tx * 4 + j;
      if (c < ncls) out[(long long)(base + r) * nr + base + c] = acc[i][j];
    }
  }
}

// Q[e] = sum over the splits in a fixed order; with sym, entries below the diagonal tiles read
// their mirror; with ev, the partial sums are in parity row order.
__global__ void k_reduce_splits(const double* __restrict__ partial, int nsplit, int nr, int gt, int sym,
                                double* __restrict__ Q, long long q_stride, const int* __restrict__ ev,
                                int ax1, int ax2, int Da) {
  const int nn = nr * nr;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nn) return;
  partial += (long long)blockIdx.y * nsplit * nn;
  Q += (long long)blockIdx.y * q_stride;
  int r = e / nr, c = e % nr;
  int base = 0;
  if (ev) {
    // rows of different parity: zero; otherwise the class-local positions in parity order
    const int e1 = ev[blockIdx.y * kMaxD + ax1], e2 = ev[blockIdx.y * kMaxD + ax2];
    int neven = 0, br = 0, bc = 0;
    const int pr = gram_row_par(r, Da, e1, e2), pc = gram_row_par(c, Da, e1, e2);
    if (pr != pc) {
      Q[e] = 0.0;
      return;
    }
    for (int q = 0; q < nr; ++q) {
      const int pq = gram_row_par(q, Da, e1, e2);
      neven += pq == 0;
      if (q < r && pq == pr) ++br;
      if (q < c && pq == pc) ++bc;
    }
    base = pr ? neven : 0;
    r = br;
    c = bc;
  }
  const int src = (sym && r / gt > c / gt) ? (base + c) * nr + base + r : (base + r) * nr + base + c;
  double s = 0.0;
  for (int k = 0; k < nsplit; ++k) s += partial[(long long)k * nn + src];
  Q[e] = s;
}

__global__ void k_gram_combine(const double* __restrict__ Q1, const double* __restrict__ Q2, long long q_stride,
                               int Db, int Da, double* __restrict__ G, long long g_stride) {
  const int n = Db * Db, nr = Db * Da;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * n) return;
  Q1 += (long long)blockIdx.y * q_stride;
  Q2 += (long long)blockIdx.y * q_stride;
  G += (long long)blockIdx.y * g_stride;
  const int row = e / n, col = e % n;
  const int b1 = row / Db, b2 = row % Db, c1 = col / Db, c2 = col % Db;
  double s = 0.0;
  for (int al = 0; al < Da; ++al) {
    const double* q1 = Q1 + (long long)(b1 * Da + al) * nr + c1 * Da;
    const double* q2 = Q2 + (long long)(b2 * Da + al) * nr + c2 * Da;
    for (int at = 0; at < Da; ++at) s = fma(q1[at], q2[at], s);
  }
  G[e] = s;
}

// Tangent of G from the tangents of the half-Grams: with H1 = Q1(dT, T) and H2 = Q2(dT, T)
// (rows from dT), dQ = H + H^T and dG = sum dQ1 Q2 + Q1 dQ2.
__global__ void k_gram_combine_tangent(const double* __restrict__ Q1, const double* __restrict__ Q2,
                                       const double* __restrict__ H1, const double* __restrict__ H2,
                                       long long q_stride, int Db, int Da, double* __restrict__ dG,
                                       long long g_stride) {
  const int n = Db * Db, nr = Db * Da;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * n) return;
  const long long qo = (long long)blockIdx.y * q_stride;
  Q1 += qo; Q2 += qo; H1 += qo; H2 += qo;
  dG += (long long)blockIdx.y * g_stride;
  const int row = e / n, col = e % n;
  const int b1 = row / Db, b2 = row % Db, c1 = col / Db, c2 = col % Db;
  double s = 0.0;
  for (int al = 0; al < Da; ++al)
    for (int at = 0; at < Da; ++at) {
      const long long i1 = (long long)(b1 * Da + al) * nr + c1 * Da + at;   // Q1[(b1,al)][(c1,at)]
      const long long t1 = (long long)(c1 * Da + at) * nr + b1 * Da + al;   // transposed entry
      const long long i2 = (long long)(b2 * Da + al) * nr + c2 * Da + at;
      const long long t2 = (long long)(c2 * Da + at) * nr + b2 * Da + al;
      s = fma(H1[i1] + H1[t1], Q2[i2], s);
      s = fma(Q1[i1], H2[i2] + H2[t2], s);
    }
  dG[e] = s;
}

}  // namespace

// Tile edge for nr x nr outputs: the candidate that computes the fewest padded entries.
static int gram_tile(int nr, bool sym) {
  const int cand[5] = {36, 44, 52, 60, 64};
  int best = 64;
  long long best_area = -1;
  for (int gt : cand) {
    const long long n = (nr + gt - 1) / gt;
    const long long area = (sym ? n * (n + 1) / 2 : n * n) * gt * gt;
    if (best_area < 0 || area < best_area) { best_area = area; best = gt; }
  }
  return best;
}

static int gram_tiles(int nr, bool sym, int gt) {
  const int n = (nr + gt - 1) / gt;
  return sym ? n * (n + 1) / 2 : n * n;
}

// split-K factor for nr x nr outputs over `batch` instances (about kGramWarps warps in total)
static int nsplit_for(int nr, long long K, int batch, bool sym) {
  const int gt = gram_tile(nr, sym);
  const int wpc = ((gt / 4) * (gt / 4) + 31) / 32;
  int nsplit = kGramWarps / (gram_tiles(nr, sym, gt) * wpc * batch);
  if (nsplit < 1) nsplit = 1;
  if (nsplit > K) nsplit = (int)K;
  return nsplit;
}

size_t gram_partial_doubles(int nr_max, int batch) {
  size_t best = 0;
  for (int nr = 1; nr <= nr_max; ++nr)
    for (int sym = 0; sym < 2; ++sym)
      for (int z2 = 0; z2 < 2; ++z2) {
        // the zero-field launch splits as for half the rows but writes at full nr x nr positions
        const int ns = z2 ? nsplit_for((nr + 1) / 2, 1LL << 40, batch, sym != 0)
                          : nsplit_for(nr, 1LL << 40, batch, sym != 0);
        const size_t v = (size_t)batch * ns * nr * nr;
        if (v > best) best = v;
      }
  return best;
}

void launch_half_gram(const double* T, long long t_stride, int batch, Geom g, int l1, int l2, double* partial,
                      double* Q, long long q_stride, cudaStream_t s, const double* TA, const int* z2ev) {
  const int d = g.d;
  auto leg_dim = [&](int l) { return g.D[l % d]; };
  auto leg_stride = [&](int l) { return l < d ? g.Sn[l] * g.P : g.Sn[l - d]; };
  LegInfo li;
  li.nrest = 0;
  for (int l = 0; l < 2 * d; ++l) {
    if (l == l1 || l == l2) continue;
    li.dim[li.nrest] = leg_dim(l);
    li.stride[li.nrest] = leg_stride(l);
    li.ax[li.nrest] = l % d;
    ++li.nrest;
  }
  li.ax1 = l1 % d;
  li.ax2 = l2 % d;
  const int Da = leg_dim(l2);
  const int nr = leg_dim(l1) * Da;
  const long long K = g.P * g.P / nr;
  const bool sym = TA == nullptr || TA == T;
  // zero-field: each parity class is tiled on its own, for about half the rows (a class may
  // hold up to nr rows: ntile covers that, the tiles beyond the actual class exit)
  const int gt = z2ev ? gram_tile((nr + 1) / 2, sym) : gram_tile(nr, sym);
  const int ntile = (nr + gt - 1) / gt;
  const int nsplit = z2ev ? nsplit_for((nr + 1) / 2, K / 2, batch, sym) : nsplit_for(nr, K, batch, sym);
  dim3 grid((z2ev ? 2 : 1) * (sym ? ntile * (ntile + 1) / 2 : ntile * ntile), nsplit, batch);
  const double* A = TA ? TA : T;
  switch (gt) {
#define HOTRG_GRAM(GT_)                                                                                        \
  case GT_:                                                                                                    \
    k_half_gram<GT_><<<grid, (GT_ / 4) * (GT_ / 4), 0, s>>>(A, T, t_stride, li, leg_stride(l1), leg_stride(l2), \
                                                            Da, nr, K, ntile, sym ? 1 : 0, nsplit, partial,      \
                                                            z2ev);                                               \
    break;
    HOTRG_GRAM(36) HOTRG_GRAM(44) HOTRG_GRAM(52) HOTRG_GRAM(60) HOTRG_GRAM(64)
#undef HOTRG_GRAM
  }
  count_launches(1);
  const int nn = nr * nr;
  k_reduce_splits<<<dim3((nn + 255) / 256, batch), 256, 0, s>>>(partial, nsplit, nr, gt, sym ? 1 : 0, Q, q_stride,
                                                                 z2ev, li.ax1, li.ax2, Da);
  count_launches(1);
}

void launch_gram_combine(const double* Q1, const double* Q2, long long q_stride, int batch, int Db, int Da,
                         double* G, long long g_stride, cudaStream_t s) {
  const int n = Db * Db;
  k_gram_combine<<<dim3((n * n + 255) / 256, batch), 256, 0, s>>>(Q1, Q2, q_stride, Db, Da, G, g_stride);
  count_launches(1);
}

void launch_gram_combine_tangent(const double* Q1, const double* Q2, const double* H1, const double* H2,
                                 long long q_stride, int batch, int Db, int Da, double* dG, long long g_stride,
                                 cudaStream_t s) {
  const int n = Db * Db;
  k_gram_combine_tangent<<<dim3((n * n + 255) / 256, batch), 256, 0, s>>>(Q1, Q2, H1, H2, q_stride, Db, Da, dG,
                                                                          g_stride);
  count_launches(1);
}

}  // namespace hotrg
