// Spin-flip (Z2) block structure of the zero-field flow, used to skip the squeeze's zero blocks.
//
// At h = 0 the site weight is even in the spin, so T^(0) vanishes unless an even number of its
// legs carry the odd bond index (Sec. 2's T^(0): the odd-n1 terms of the sum over s cancel
// exactly). Every step keeps this: the Gram matrices commute with the parity of the fused
// index, the eigenvectors are parity-pure (Jacobi never rotates an entry that is exactly zero),
// so every new bond index has a parity and every tensor entry whose legs' parities add up to
// odd is exactly zero. Here each bond index is kept parity-sorted (even values first; a
// relabelling of the bond, under which ln Z/N and the spectra are invariant), and the squeeze
// works on parity-blocked operands:
//   rows m and columns k of the A operand, and the columns n of B, are ordered by total parity
//   (even class first), inside a class by the parity pattern of the legs and then row-major
//   inside the pattern's box; the two k classes start at 64-aligned columns with zeros between;
//   the rows (j, n) of B (columns of the GEMM output) are grouped by parity(j) + parity(n).
// In a chunk with isometry-index parity pi, A[m][k] vanishes unless parity(m) + parity(k) = pi
// and B[(j, n)][k] unless parity(j) + parity(n) = parity(k): the product is two dense blocks,
// a quarter of the dense flops.
#include "kernels.h"

namespace hotrg {

namespace {

__device__ __forceinline__ int popc4(int x) { return __popc(x & 15); }

// arithmetic type of a path: FP64 path in double, tensor-core path (bf16 planes, FP32 output) in float
template <class T>
using ZAcc = typename std::conditional<std::is_same<T, double>::value, double, float>::type;

// natural P-index -> digits (slot 0 slowest) and leg-parity pattern (bit b = digit_b >= e_b)
__device__ __forceinline__ int z2_digits(const Z2Layout& L, int idx, int* dig) {
  int pat = 0;
  for (int b = L.d - 1; b >= 0; --b) {
    dig[b] = idx % L.D[b];
    idx /= L.D[b];
    if (dig[b] >= L.e[b]) pat |= 1 << b;
  }
  return pat;
}

__device__ __forceinline__ int z2_rank(const Z2Layout& L, const int* dig, int pat) {
  int r = L.patoff[pat];
  for (int b = 0; b < L.d; ++b) r += (dig[b] - (((pat >> b) & 1) ? L.e[b] : 0)) * L.bs[pat][b];
  return r;
}

__global__ void k_z2_layout(const int* ev, const int* ev_new, Geom g, int c3, int chi3, Z2Layout* out) {
  if (threadIdx.x != 0) return;
  const int inst = blockIdx.x;
  ev += inst * kMaxD;
  ev_new += inst * kMaxD;
  Z2Layout L;
  L.d = g.d;
  for (int b = 0; b < kMaxD; ++b) {
    L.D[b] = b < g.d ? g.D[b] : 1;
    L.e[b] = b < g.d ? min(max(ev[b], 0), L.D[b]) : 1;
  }
  const int npat = 1 << g.d;
  int off = 0;
  L.ncls[0] = L.ncls[1] = 0;
  for (int cls = 0; cls < 2; ++cls)
    for (int pat = 0; pat < 16; ++pat) {
      if (pat >= npat || (popc4(pat) & 1) != cls) {
        if (cls == 0) {
          L.patoff[pat] = 0;
          for (int b = 0; b < kMaxD; ++b) L.bs[pat][b] = 0;
        }
        continue;
      }
      int box = 1;
      for (int b = g.d - 1; b >= 0; --b) {
        L.bs[pat][b] = box;
        box *= ((pat >> b) & 1) ? L.D[b] - L.e[b] : L.e[b];
      }
      for (int b = g.d; b < kMaxD; ++b) L.bs[pat][b] = 0;
      L.patoff[pat] = off;
      off += box;
      L.ncls[cls] += box;
    }
  L.kstart[0] = 0;
  L.kstart[1] = (L.ncls[0] + 63) / 64 * 64;
  L.chi3 = chi3;
  L.e3 = c3 >= 0 ? min(max(ev_new[c3], 0), chi3) : chi3;
  for (int t = 0; t < 2; ++t) {
    int acc = 0;
    for (int j = 0; j <= kMaxBond; ++j) {
      L.jstart[t][j] = acc;
      if (j < chi3) acc += L.ncls[t ^ (j >= L.e3 ? 1 : 0)];
    }
  }
  L.goff[0] = 0;
  L.goff[1] = L.jstart[0][chi3];
  out[inst] = L;
}

// rank_tab[i] = rank of natural index i (even class first); kcol_tab[i] = its operand column;
// colpos_tab[j * P + n] = GEMM-output column of (j, n).
__global__ void k_z2_tables(const Z2Layout* Lp, int P, int chi3, int* rank_tab, int* kcol_tab, int* colpos_tab) {
  const Z2Layout L = *Lp;
  const long long total = (long long)chi3 * P;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(t / P), n = (int)(t % P);
    int dig[kMaxD];
    const int pat = z2_digits(L, n, dig);
    const int par = popc4(pat) & 1;
    const int r = z2_rank(L, dig, pat);
    const int within = r - (par ? L.ncls[0] : 0);
    if (j == 0) {
      rank_tab[n] = r;
      kcol_tab[n] = L.kstart[par] + within;
    }
    const int grp = par ^ (j >= L.e3 ? 1 : 0);
    colpos_tab[t] = L.goff[grp] + L.jstart[grp][j] + within;
  }
}

// pi = parity of the chunk's fixed new indices; the GEMM's two blocks (row class cm, k class
// and column group cm ^ pi).
__global__ void k_z2_chunk(const Z2Layout* Lp, const int* ev_new, int nfix, int b0, int k0, int b1, int k1,
                           long long ldO, GemmBlocks* blk, int* pi_out, double* flops, int npass) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const Z2Layout& L = *Lp;
  int pi = 0;
  if (nfix > 0) pi ^= k0 >= ev_new[b0] ? 1 : 0;
  if (nfix > 1) pi ^= k1 >= ev_new[b1] ? 1 : 0;
  GemmBlocks g;
  g.nb = 2;
  for (int cm = 0; cm < 2; ++cm) {
    const int ck = cm ^ pi;
    g.m0[cm] = cm ? L.ncls[0] : 0;
    g.mc[cm] = L.ncls[cm];
    g.k0[cm] = L.kstart[ck];
    g.kc[cm] = L.ncls[ck];
    g.n0[cm] = L.goff[ck];
    g.nc[cm] = ck ? (int)(ldO - L.goff[1]) : L.goff[1];
  }
  *blk = g;
  *pi_out = pi;
  // algorithmic flops of the two blocks: [0] 2 M N K, [1] times the split passes
  double f = 0.0;
  for (int b = 0; b < 2; ++b) f += 2.0 * g.mc[b] * (double)g.nc[b] * g.kc[b];
  flops[0] += f;
  flops[1] += f * npass;
}

__global__ void k_z2_advance(int* ev, const int* ev_new, int batch, unsigned trans_mask) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= batch * kMaxD) return;
  if ((trans_mask >> (t % kMaxD)) & 1) ev[t] = ev_new[t];
}

// A operand of one chunk, parity-blocked: Y[rank(m)][kcol(k)] = X[R(k) + C(m)] where
// parity(m) + parity(k) = pi (the other entries of X are zero and not stored). A block covers 32
// columns k and Y_MT x 32 rows m: warp 0 decomposes its 32 k (offset R(k), operand column, parity),
// warps 1..Y_MT its rows (offset C(m), rank, parity) at the same time, in 32-bit index arithmetic
// (P < 2^31); then every thread issues its 4 Y_MT loads before its stores (the tile's rows share
// L1 sectors where X is contiguous along m).
constexpr int Y_MT = 4;
template <class Tin, class Tout>
__global__ void __launch_bounds__(256) k_build_y_z2(const Tin* __restrict__ X, Planes<Tout> out,
                                                    long long ld, Geom g, int a, const int* __restrict__ rank_tab,
                                                    const int* __restrict__ kcol_tab, const Z2Layout* Lp,
                                                    const int* pi_ptr) {
  __shared__ long long Rk[32], Cm[32 * Y_MT];
  __shared__ int rowr[32 * Y_MT], colk[32], parm[32 * Y_MT], park[32];
  const int P = (int)g.P;
  const long long PP = g.P;
  const int ncls0 = Lp->ncls[0];
  const int pi = *pi_ptr;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int m0 = blockIdx.y * 32 * Y_MT, k0 = blockIdx.x * 32;
  if (ty == 0) {
    const int k = k0 + tx;
    long long rk = 0;
    for (int b = 0; b < g.d; ++b) {
      const int sb = (int)g.Sn[b];
      const long long kb = (k / sb) % g.D[b];
      rk += b == a ? kb * sb : kb * sb * PP;
    }
    Rk[tx] = rk;
    colk[tx] = k < P ? kcol_tab[k] : 0;
    park[tx] = k < P ? (rank_tab[k] >= ncls0 ? 1 : 0) : 0;
  } else if (ty <= Y_MT) {
    const int r = (ty - 1) * 32 + tx;
    const int m = m0 + r;
    long long cm = 0;
    for (int b = 0; b < g.d; ++b) {
      const int sb = (int)g.Sn[b];
      const long long mb = (m / sb) % g.D[b];
      cm += b == a ? mb * sb * PP : mb * sb;
    }
    Cm[r] = cm;
    const int rm = m < P ? rank_tab[m] : 0;
    rowr[r] = rm;
    parm[r] = rm >= ncls0 ? 1 : 0;
  }
  __syncthreads();
  ZAcc<Tout> v[4 * Y_MT];
  bool w[4 * Y_MT];
  const int k = k0 + tx;
  const float sc = plane_scale(out);
#pragma unroll
  for (int q = 0; q < 4 * Y_MT; ++q) {
    const int r = ty + 8 * q;
    w[q] = m0 + r < P && k < P && (parm[r] ^ park[tx]) == pi;
    v[q] = w[q] ? (ZAcc<Tout>)X[Rk[tx] + Cm[r]] : (ZAcc<Tout>)0;
  }
#pragma unroll
  for (int q = 0; q < 4 * Y_MT; ++q)
    if (w[q]) store_planes_sc(out, (long long)rowr[ty + 8 * q] * ld + colk[tx], v[q], sc);
}

// B operand, parity-blocked: Bt[colpos(j, n)][kcol(k)] = sum_x U3[j][k_c3][x] Tt[n][k | c3 := x]
// where parity(j) + parity(n) = parity(k).
template <class Tin, class Tout>
__global__ void __launch_bounds__(256) k_build_bt_z2(const Tin* __restrict__ Tt, Planes<Tout> out,
                                                     long long ld, long long P, long long Sc, int Dc,
                                                     const double* __restrict__ U3, int chi3,
                                                     const int* __restrict__ rank_tab, const int* __restrict__ kcol_tab,
                                                     const int* __restrict__ colpos_tab, const Z2Layout* Lp) {
  using Acc = ZAcc<Tout>;
  extern __shared__ unsigned char smraw_bt[];
  Acc* W = reinterpret_cast<Acc*>(smraw_bt);  // [chi3][Dc][Dc]
  const int nW = chi3 * Dc * Dc;
  for (int t = threadIdx.x; t < nW; t += blockDim.x) W[t] = (Acc)U3[t];
  __syncthreads();
  const int ncls0 = Lp->ncls[0];
  const int goff1 = Lp->goff[1];
  const long long total = (long long)chi3 * P * P;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long k = idx % P;
    const long long row = idx / P;  // j*P + n
    const int cp = colpos_tab[row];
    const int grp = cp >= goff1 ? 1 : 0;
    const int park = rank_tab[k] >= ncls0 ? 1 : 0;
    if (grp != park) continue;
    const long long n = row % P;
    const int j = (int)(row / P);
    const int kc = (int)((k / Sc) % Dc);
    const long long base = n * P + k - (long long)kc * Sc;
    const Acc* w = W + ((long long)j * Dc + kc) * Dc;
    Acc acc = 0;
    for (int x = 0; x < Dc; ++x) acc += w[x] * (Acc)Tt[base + x * Sc];
    store_planes(out, (long long)cp * ld + kcol_tab[k], acc);
  }
}

// First epilogue contraction of a chunk from the parity-blocked GEMM output:
//   R[rest, k'] = sum_{i, jj} U_t0[k'][i][jj] O[m = (rest_m, m_t0 = i)][(j, n = (rest_n, n_t0 = jj))]
// with O stored as O[rank(m)][colpos(j, n)]. rest = (m_b for b != t0, j, n_b for b != t0) in that
// order, shaped and strided by `rest` (out_stride) and sk (stride of k'). Only the (i, jj)
// parity combinations of the chunk's two computed blocks are read; the rest of O is zero.
// CHI = chi (compile-time: exact accumulator count, no predicated FMAs).
// W rows padded to a multiple of 4 entries (16-byte shared-memory loads)
template <int CHI>
constexpr int chi_pad() {
  return (CHI + 3) / 4 * 4;
}

// Rows of one parity class with a compile-time column count NC: acc[k] += sum over the nrow
// rows r and the NC columns u of w[r * wrow + u * CHIP + k] * src[r * rstep + u * cs]. The
// loads of max(1, 8 / NC) rows are issued before their FMAs (few registers: the kernel is
// latency-bound and gains more from resident warps than from loads in flight per thread).
template <class Tin, class Acc, int CHI, int NC>
__device__ __forceinline__ void epi_class_rows(const Tin* __restrict__ src, long long rstep, long long cs,
                                               int nrow, const Acc* __restrict__ w, int wrow, Acc* acc) {
  constexpr int CHIP = chi_pad<CHI>();
  constexpr int R = NC >= 8 ? 1 : 8 / NC;
  for (int r0 = 0; r0 < nrow; r0 += R) {
    Acc x[R][NC];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const bool ok = r0 + r < nrow;
      const Tin* p = src + (long long)(r0 + r) * rstep;
#pragma unroll
      for (int u = 0; u < NC; ++u) x[r][u] = ok ? (Acc)p[u * cs] : (Acc)0;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (r0 + r >= nrow) break;
      const Acc* wr = w + (r0 + r) * wrow;
#pragma unroll
      for (int u = 0; u < NC; ++u)
#pragma unroll
        for (int k = 0; k < CHI; ++k) acc[k] += wr[u * CHIP + k] * x[r][u];
    }
  }
}

// Same for any column count (runtime ncol), two rows' loads (up to 8 each) before the FMAs.
template <class Tin, class Acc, int CHI>
__device__ __forceinline__ void epi_class_rows_any(const Tin* __restrict__ src, long long rstep, long long cs,
                                                   int nrow, int ncol, const Acc* __restrict__ w, int wrow,
                                                   Acc* acc) {
  constexpr int CHIP = chi_pad<CHI>();
  for (int i = 0; i < nrow; i += 2) {
    const bool two = i + 1 < nrow;
    const Tin* src0 = src + (long long)i * rstep;
    const Tin* src1 = src0 + rstep;
    for (int u0 = 0; u0 < ncol; u0 += 8) {
      Acc x0[8], x1[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const bool ok = u0 + u < ncol;
        x0[u] = ok ? (Acc)src0[(long long)(u0 + u) * cs] : (Acc)0;
        x1[u] = (ok && two) ? (Acc)src1[(long long)(u0 + u) * cs] : (Acc)0;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (u0 + u >= ncol) break;
        const Acc* w0 = w + i * wrow + (u0 + u) * CHIP;
        const Acc* w1 = w0 + wrow;
#pragma unroll
        for (int k = 0; k < CHI; ++k) acc[k] += w0[k] * x0[u];
        if (two) {
#pragma unroll
          for (int k = 0; k < CHI; ++k) acc[k] += w1[k] * x1[u];
        }
      }
    }
  }
}

// CTAs per SM the register budget targets: four for the FP32 path; two for FP64 (its
// accumulators take twice the registers)
template <class Tin>
constexpr int epi_min_blocks() {
  return std::is_same<Tin, float>::value ? 4 : 2;
}

template <class Tin, class Tout, int CHI>
__global__ void __launch_bounds__(256, epi_min_blocks<Tin>()) k_epi_z2(const Tin* __restrict__ O, long long ldO, Tout* __restrict__ out,
                                                View rest, int total, long long sk, long long out_base,
                                                int t0, const double* __restrict__ U,
                                                const Z2Layout* Lp, const int* pi_ptr) {
  using Acc = ZAcc<Tin>;
  constexpr int CHIP = chi_pad<CHI>();
  extern __shared__ __align__(16) unsigned char smraw_epi[];
  Acc* W = reinterpret_cast<Acc*>(smraw_epi);  // [D*D][CHIP]
  __shared__ Z2Layout L;
  __shared__ int shape[2 * kMaxD + 1];
  __shared__ long long ostr[2 * kMaxD + 1];
  if (threadIdx.x == 0) L = *Lp;
  if (threadIdx.x < rest.ndim) {
    shape[threadIdx.x] = rest.shape[threadIdx.x];
    ostr[threadIdx.x] = rest.out_stride[threadIdx.x];
  }
  const int Dt = Lp->D[t0];
  const int nij = Dt * Dt;
  for (int t = threadIdx.x; t < CHIP * nij; t += blockDim.x) {
    const int k = t / nij, ij = t % nij;
    W[ij * CHIP + k] = k < CHI ? (Acc)U[t] : (Acc)0;
  }
  __syncthreads();
  const int pi = *pi_ptr;
  const int d = L.d, et = L.e[t0], nd = rest.ndim;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    // decode rest coordinates, last axis first: the d-1 n digits, j, the d-1 m digits (32-bit:
    // rest has < 2^31 entries); unrolled over the slots so that the digits stay in registers
    int rem = idx;
    long long ooff = out_base;
    int ax = nd - 1;
    int dm[kMaxD], dn[kMaxD];
    int pm = 0, pn = 0;
#pragma unroll
    for (int b = kMaxD - 1; b >= 0; --b) {
      dn[b] = 0;
      if (b >= d || b == t0) continue;
      const int sh = shape[ax];
      const int qq = rem / sh;
      dn[b] = rem - qq * sh;
      rem = qq;
      ooff += (long long)dn[b] * ostr[ax--];
      if (dn[b] >= L.e[b]) pn |= 1 << b;
    }
    int j;
    {
      const int sh = shape[ax];
      const int qq = rem / sh;
      j = rem - qq * sh;
      rem = qq;
      ooff += (long long)j * ostr[ax--];
    }
#pragma unroll
    for (int b = kMaxD - 1; b >= 0; --b) {
      dm[b] = 0;
      if (b >= d || b == t0) continue;
      const int sh = shape[ax];
      const int qq = rem / sh;
      dm[b] = rem - qq * sh;
      rem = qq;
      ooff += (long long)dm[b] * ostr[ax--];
      if (dm[b] >= L.e[b]) pm |= 1 << b;
    }
    const int pj = j >= L.e3 ? 1 : 0;
    const int tau = pi ^ pj ^ (popc4(pm) & 1) ^ (popc4(pn) & 1);
    Acc acc[CHI];
#pragma unroll
    for (int k = 0; k < CHI; ++k) acc[k] = 0;
    // loop over the column class: its width is the same in every lane of a warp (the row class
    // ci = cj ^ tau varies with the lane's parities, only as a row count)
    for (int cj = 0; cj < 2; ++cj) {
      const int ci = cj ^ tau;
      const int patm = pm | (ci << t0), patn = pn | (cj << t0);
      const int parn = popc4(patn) & 1;
      long long rb = L.patoff[patm];
      long long cb = L.patoff[patn] - (parn ? L.ncls[0] : 0);
#pragma unroll
      for (int b = 0; b < kMaxD; ++b) {
        if (b >= d || b == t0) continue;
        rb += (long long)(dm[b] - (((patm >> b) & 1) ? L.e[b] : 0)) * L.bs[patm][b];
        cb += (long long)(dn[b] - (((patn >> b) & 1) ? L.e[b] : 0)) * L.bs[patn][b];
      }
      const int grp = parn ^ pj;
      cb += L.goff[grp] + L.jstart[grp][j];
      const long long rstep = L.bs[patm][t0] * ldO, cs = L.bs[patn][t0];
      const int i0 = ci ? et : 0, nrow = ci ? Dt - et : et;
      const int j0 = cj ? et : 0, ncol = cj ? Dt - et : et;
      const Tin* src = O + rb * ldO + cb;
      const Acc* w = W + (i0 * Dt + j0) * CHIP;
      const int wrow = Dt * CHIP;
      if constexpr (std::is_same<Tin, float>::value && CHI >= 6) {
        switch (ncol) {
#define HOTRG_EPI_NC(NC) \
  case NC:               \
    epi_class_rows<Tin, Acc, CHI, NC>(src, rstep, cs, nrow, w, wrow, acc); \
    break;
          HOTRG_EPI_NC(1) HOTRG_EPI_NC(2) HOTRG_EPI_NC(3) HOTRG_EPI_NC(4)
          HOTRG_EPI_NC(5) HOTRG_EPI_NC(6) HOTRG_EPI_NC(7) HOTRG_EPI_NC(8)
#undef HOTRG_EPI_NC
          default:
            epi_class_rows_any<Tin, Acc, CHI>(src, rstep, cs, nrow, ncol, w, wrow, acc);
        }
      } else {
        epi_class_rows_any<Tin, Acc, CHI>(src, rstep, cs, nrow, ncol, w, wrow, acc);
      }
    }
#pragma unroll
    for (int k = 0; k < CHI; ++k) out[ooff + k * sk] = (Tout)acc[k];
  }
}

inline int grid_cap(long long n) {
  long long g = (n + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

void launch_z2_layout(const int* ev, const int* ev_new, int batch, Geom g, int c3, int chi3, Z2Layout* out,
                      cudaStream_t s) {
  k_z2_layout<<<batch, 32, 0, s>>>(ev, ev_new, g, c3, chi3, out);
  count_launches(1);
}

void launch_z2_tables(const Z2Layout* L, long long P, int chi3, int* rank_tab, int* kcol_tab, int* colpos_tab,
                      cudaStream_t s) {
  k_z2_tables<<<grid_cap((long long)chi3 * P), 256, 0, s>>>(L, (int)P, chi3, rank_tab, kcol_tab, colpos_tab);
  count_launches(1);
}

void launch_z2_chunk(const Z2Layout* L, const int* ev_new, int nfix, int b0, int k0, int b1, int k1, long long ldO,
                     GemmBlocks* blk, int* pi, double* flops, int npass, cudaStream_t s) {
  k_z2_chunk<<<1, 32, 0, s>>>(L, ev_new, nfix, b0, k0, b1, k1, ldO, blk, pi, flops, npass);
  count_launches(1);
}

void launch_z2_advance(int* ev, const int* ev_new, int batch, unsigned trans_mask, cudaStream_t s) {
  k_z2_advance<<<(batch * kMaxD + 127) / 128, 128, 0, s>>>(ev, ev_new, batch, trans_mask);
  count_launches(1);
}

template <class Tin, class Tout>
void launch_build_y_z2(const Tin* X, const Planes<Tout>& out, long long ld, Geom g, int a,
                       const int* rank_tab, const int* kcol_tab, const Z2Layout* L, const int* pi, cudaStream_t s) {
  dim3 grid((unsigned)((g.P + 31) / 32), (unsigned)((g.P + 32 * Y_MT - 1) / (32 * Y_MT)));
  k_build_y_z2<Tin, Tout><<<grid, dim3(32, 8), 0, s>>>(X, out, ld, g, a, rank_tab, kcol_tab, L, pi);
  count_launches(1);
}

template <class Tin, class Tout>
void launch_build_bt_z2(const Tin* Tt, const Planes<Tout>& out, long long ld, Geom g, int c3, const double* U3,
                        int chi3, const int* rank_tab, const int* kcol_tab, const int* colpos_tab, const Z2Layout* L,
                        cudaStream_t s) {
  const size_t smem = sizeof(ZAcc<Tout>) * (size_t)chi3 * g.D[c3] * g.D[c3];
  const long long total = (long long)chi3 * g.P * g.P;
  k_build_bt_z2<Tin, Tout><<<grid_cap(total), 256, smem, s>>>(Tt, out, ld, g.P, g.Sn[c3], g.D[c3], U3, chi3, rank_tab,
                                                               kcol_tab, colpos_tab, L);
  count_launches(1);
}

template <class Tin, class Tout>
void launch_epi_z2(const Tin* O, long long ldO, Tout* out, const View& rest, long long sk, long long out_base,
                   int t0, int Dt, const double* U, int chi, const Z2Layout* L, const int* pi, cudaStream_t s) {
  long long total = 1;
  for (int i = 0; i < rest.ndim; ++i) total *= rest.shape[i];
  const size_t smem = sizeof(ZAcc<Tin>) * (size_t)((chi + 3) / 4 * 4) * Dt * Dt;
  const int n = (int)total;  // rest < 2^31 entries (P^2 chi3 / Dt^2 <= 2.3e9 / 4 for Dcut <= 14)
  switch (chi) {
#define HOTRG_EPI_Z2(C)                                                                                        \
  case C:                                                                                                      \
    k_epi_z2<Tin, Tout, C><<<grid_cap(total), 256, smem, s>>>(O, ldO, out, rest, n, sk, out_base, t0, U, L, pi); \
    break;
    HOTRG_EPI_Z2(1) HOTRG_EPI_Z2(2) HOTRG_EPI_Z2(3) HOTRG_EPI_Z2(4) HOTRG_EPI_Z2(5) HOTRG_EPI_Z2(6)
    HOTRG_EPI_Z2(7) HOTRG_EPI_Z2(8) HOTRG_EPI_Z2(9) HOTRG_EPI_Z2(10) HOTRG_EPI_Z2(11) HOTRG_EPI_Z2(12)
    HOTRG_EPI_Z2(13) HOTRG_EPI_Z2(14) HOTRG_EPI_Z2(15) HOTRG_EPI_Z2(16)
#undef HOTRG_EPI_Z2
    default:
      return;
  }
  count_launches(1);
}

using bf16 = __nv_bfloat16;
template void launch_build_y_z2<float, bf16>(const float*, const Planes<bf16>&, long long, Geom, int, const int*,
                                             const int*, const Z2Layout*, const int*, cudaStream_t);
template void launch_build_y_z2<double, bf16>(const double*, const Planes<bf16>&, long long, Geom, int, const int*,
                                              const int*, const Z2Layout*, const int*, cudaStream_t);
template void launch_build_y_z2<double, double>(const double*, const Planes<double>&, long long, Geom, int,
                                                const int*, const int*, const Z2Layout*, const int*, cudaStream_t);
template void launch_build_bt_z2<float, bf16>(const float*, const Planes<bf16>&, long long, Geom, int, const double*,
                                              int, const int*, const int*, const int*, const Z2Layout*, cudaStream_t);
template void launch_build_bt_z2<double, double>(const double*, const Planes<double>&, long long, Geom, int,
                                                 const double*, int, const int*, const int*, const int*,
                                                 const Z2Layout*, cudaStream_t);
template void launch_epi_z2<float, float>(const float*, long long, float*, const View&, long long, long long, int,
                                          int, const double*, int, const Z2Layout*, const int*, cudaStream_t);
template void launch_epi_z2<float, double>(const float*, long long, double*, const View&, long long, long long, int,
                                           int, const double*, int, const Z2Layout*, const int*, cudaStream_t);
template void launch_epi_z2<double, double>(const double*, long long, double*, const View&, long long, long long,
                                            int, int, const double*, int, const Z2Layout*, const int*, cudaStream_t);

}  // namespace hotrg
