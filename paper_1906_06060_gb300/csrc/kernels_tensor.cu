// Element-wise, reduction and re-layout kernels of one HOTRG step (arXiv:1906.06060, Sec. 2).
// The squeeze GEMM itself lives in gemm_tc.cu (tensor cores) and gemm_simt.cu (FP64).
#include <atomic>
#include <type_traits>

#include "kernels.h"

namespace hotrg {

static std::atomic<long long> g_launches{0};
void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launches_total() { return g_launches.load(std::memory_order_relaxed); }

namespace {

template <class Tout>
using AccT = typename std::conditional<std::is_same<Tout, double>::value, double, float>::type;


inline int grid_for(long long n, int block, int cap = 152 * 16) {
  long long g = (n + block - 1) / block;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

constexpr int kNormBlocks = 1024;

// ---------------------------------------------------------------------------- max |x|
// Upper bound of |x| as a float (rounded up from double).
__device__ __forceinline__ float abs_up(double x) { return __double2float_ru(fabs(x)); }
__device__ __forceinline__ float abs_up(float x) { return fabsf(x); }

// *out = max(*out, max |x|) over rows x cols entries with row stride ld, as the bits of a
// non-negative float (their unsigned order is the order of the values). NaN entries are skipped.
template <class T>
__global__ void __launch_bounds__(256) k_absmax(const T* __restrict__ x, long long rows, long long cols,
                                                long long ld, unsigned* out) {
  float m = 0.f;
  const long long total = rows * cols;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / cols, c = i - r * cols;
    m = fmaxf(m, abs_up(x[r * ld + c]));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// ---------------------------------------------------------------------------- T^(0)
// T[idx] = sum_s V_s prod_{legs} W[s, leg]; W[s,0] = sqrt(cosh b), W[s,1] = s sqrt(sinh b),
// V_s = e^{b h s}; bit l of idx (from the most significant) is the index of leg l.
__global__ void k_init_tensor(double* T, long long inst_stride, int d, const double* beta,
                              const double* hfield, int spin_insertion) {
  const int nlegs = 2 * d;
  const int total = 1 << nlegs;
  const int inst = blockIdx.y;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const double b = beta[inst], h = hfield[inst];
  const double wc = sqrt(cosh(b)), ws = sqrt(sinh(b));
  double acc = 0.0;
  for (int si = 0; si < 2; ++si) {
    const double s = si ? -1.0 : 1.0;
    double v = exp(s * b * h);
    for (int l = 0; l < nlegs; ++l) {
      const int bit = (idx >> (nlegs - 1 - l)) & 1;
      v *= bit ? s * ws : wc;
    }
    acc += spin_insertion ? s * v : v;
  }
  T[inst * inst_stride + idx] = acc;
}

// ---------------------------------------------------------------------------- T^(0) tangents
// dT[idx] = d T^(0)[idx] / d beta (which = 0) or d / d h (which = 1). With n1 legs at index 1 and
// n0 = 2d - n1 at index 0, prod W = cosh^{n0/2} (s sinh^{1/2})^{n1} and
//   d/d beta [V_s prod W] = V_s prod W (h s + n0 tanh(b)/2 + n1 coth(b)/2),
//   d/d h    [V_s prod W] = V_s prod W (b s).
__global__ void k_init_tangent(double* dT, long long inst_stride, int d, const double* beta, const double* hfield,
                               int which) {
  const int nlegs = 2 * d;
  const int total = 1 << nlegs;
  const int inst = blockIdx.y;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const double b = beta[inst], h = hfield[inst];
  const double wc = sqrt(cosh(b)), ws = sqrt(sinh(b));
  const int n1 = __popc(idx);
  const int n0 = nlegs - n1;
  double acc = 0.0;
  for (int si = 0; si < 2; ++si) {
    const double s = si ? -1.0 : 1.0;
    double v = exp(s * b * h);
    for (int l = 0; l < nlegs; ++l) {
      const int bit = (idx >> (nlegs - 1 - l)) & 1;
      v *= bit ? s * ws : wc;
    }
    const double f = which == 0 ? h * s + 0.5 * n0 * tanh(b) + 0.5 * n1 / tanh(b) : b * s;
    acc += v * f;
  }
  dT[inst * inst_stride + idx] = acc;
}

// ---------------------------------------------------------------------------- norms
template <int BS>
__device__ double block_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int w = BS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  double r = sh[0];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(256) k_sumsq_partial(const double* __restrict__ x, long long n,
                                                       double* __restrict__ partial) {
  __shared__ double sh[256];
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < n; i += (long long)kNormBlocks * 256) {
    const double v = x[i];
    s = fma(v, v, s);
  }
  const double t = block_sum<256>(s, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

__global__ void k_step_advance(int* dstep) { *dstep += 1; }

__global__ void __launch_bounds__(256) k_norm_finish(const double* __restrict__ partial, double* c_out,
                                                     double* lnc_log, double* L, const int* dstep, int* status) {
  const int step = *dstep;
  __shared__ double sh[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < kNormBlocks; i += 256) s += partial[i];
  const double t = block_sum<256>(s, sh);
  if (threadIdx.x == 0) {
    const double c = sqrt(t);
    if (!(c > 0.0) || !isfinite(c)) atomic_status(status, ST_NUMERIC);
    const double lc = log(c);
    *c_out = c;
    lnc_log[step] = lc;
    *L += ldexp(lc, -step);
  }
}

// partial[b] = sum over this block's share of x[i] (y1[i] + y2[i]) (y2 may be null): fixed grid.
__global__ void __launch_bounds__(256) k_dot_partial(const double* __restrict__ x, const double* __restrict__ y1,
                                                     const double* __restrict__ y2, long long n,
                                                     double* __restrict__ partial) {
  __shared__ double sh[256];
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < n; i += (long long)kNormBlocks * 256) {
    const double y = y2 ? y1[i] + y2[i] : y1[i];
    s = fma(x[i], y, s);
  }
  const double t = block_sum<256>(s, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// dlnc = <T, D> / c^2 for the tangent D of an unnormalised tensor T with norm c; dL += 2^-n dlnc.
__global__ void __launch_bounds__(256) k_tangent_finish(const double* __restrict__ partial, const double* c,
                                                        double* dlnc, double* dL, const int* dstep) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < kNormBlocks; i += 256) s += partial[i];
  const double t = block_sum<256>(s, sh);
  if (threadIdx.x == 0) {
    const double cv = *c;
    const double v = t / (cv * cv);
    *dlnc = v;
    *dL += ldexp(v, -*dstep);
  }
}

// dTn = (D1 + D2) / c - dlnc T / c : the tangent of T / ||T||.
// D1 and dTn may be the same buffer (each element is read before it is written, by one thread).
__global__ void k_tangent_update(const double* __restrict__ T, const double* D1,
                                 const double* __restrict__ D2, double* dTn, long long n,
                                 const double* c, const double* dlnc) {
  const double inv = 1.0 / *c, g = *dlnc;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double d = D2 ? D1[i] + D2[i] : D1[i];
    dTn[i] = (d - g * T[i]) * inv;
  }
}

// d(ln Z/N) = dL + 2^-n Tr dT / Tr T for every instance (one CTA each).
__global__ void __launch_bounds__(256) k_trace_tangent(const double* __restrict__ T, const double* __restrict__ dT,
                                                       long long t_stride, long long P, const double* dL,
                                                       const int* dstep, double* out) {
  __shared__ double sh[256];
  T += (long long)blockIdx.x * t_stride;
  dT += (long long)blockIdx.x * t_stride;
  double a = 0.0, b = 0.0;
  for (long long u = threadIdx.x; u < P; u += 256) {
    a += T[u * P + u];
    b += dT[u * P + u];
  }
  const double ta = block_sum<256>(a, sh);
  const double tb = block_sum<256>(b, sh);
  if (threadIdx.x == 0) out[blockIdx.x] = dL[blockIdx.x] + ldexp(tb / ta, -*dstep);
}

// out[i] = Tr S_i / Tr T_i for every instance (one CTA each): Eqs. (energy), (spin).
__global__ void __launch_bounds__(256) k_trace_ratio(const double* __restrict__ S, const double* __restrict__ T,
                                                     long long t_stride, long long P, double* out) {
  __shared__ double sh[256];
  S += (long long)blockIdx.x * t_stride;
  T += (long long)blockIdx.x * t_stride;
  double a = 0.0, b = 0.0;
  for (long long u = threadIdx.x; u < P; u += 256) {
    a += S[u * P + u];
    b += T[u * P + u];
  }
  const double ta = block_sum<256>(a, sh);
  const double tb = block_sum<256>(b, sh);
  if (threadIdx.x == 0) out[blockIdx.x] = ta / tb;
}

__global__ void k_scale(const double* __restrict__ src, double* __restrict__ dst, long long n,
                        const double* __restrict__ c) {
  const double cv = *c;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = src[i] / cv;
}

// ---------------------------------------------------------------------------- trace, X^(n)
// out3[0] = Tr T, out3[1] = L + 2^-step ln Tr T, out3[2] = X^(n) along axis.
__global__ void __launch_bounds__(256) k_trace_x(const double* __restrict__ T, long long t_stride, Geom g,
                                                 int axis, const double* L, const int* dstep, double* out3) {
  __shared__ double sh[256];
  const int step = *dstep;
  T += (long long)blockIdx.x * t_stride;
  L += blockIdx.x;
  out3 += 3 * blockIdx.x;
  __shared__ double A[kMaxBond * kMaxBond];
  const long long P = g.P;
  double s = 0.0;
  for (long long u = threadIdx.x; u < P; u += 256) s += T[u * P + u];
  const double tr = block_sum<256>(s, sh);
  // A_{ij} = sum over the other slots (equal on both halves) with slot `axis` = i / j.
  const int Da = g.D[axis];
  const long long Sa = g.Sn[axis];
  const long long nrest = P / Da;
  for (int e = threadIdx.x; e < Da * Da; e += 256) {
    const int i = e / Da, j = e % Da;
    double acc = 0.0;
    for (long long r = 0; r < nrest; ++r) {
      // r enumerates the other slots: split r around slot `axis`
      const long long hi = r / Sa, lo = r % Sa;
      const long long base = hi * Sa * Da + lo;
      acc += T[(base + i * Sa) * P + base + j * Sa];
    }
    A[e] = acc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double trA = 0.0, trA2 = 0.0;
    for (int i = 0; i < Da; ++i) trA += A[i * Da + i];
    for (int i = 0; i < Da; ++i)
      for (int j = 0; j < Da; ++j) trA2 += A[i * Da + j] * A[j * Da + i];
    // a non-positive trace is reported by the free-energy query, not here
    out3[0] = tr;
    out3[1] = tr > 0.0 ? *L + ldexp(log(tr), -step) : nan("");
    out3[2] = trA * trA / trA2;
  }
}

// ---------------------------------------------------------------------------- mode product
// One thread per "base" (an input index with digit b = 0): it reads the Db inputs along leg b
// once and writes all Db outputs, so every input element is read from memory once.
// TWO: out also accumulates the same product of a second input with a second matrix (the
// tangent of a mode product: dX = M_U(dT) + M_dU(T)).
template <class Tin, class Tout, bool TWO>
__global__ void __launch_bounds__(256) k_mode_unprimed(const Tin* __restrict__ in, Tout* __restrict__ out,
                                                       long long total, long long stride_b, int Db,
                                                       const double* __restrict__ U, int kk,
                                                       const Tin* __restrict__ in2, const double* __restrict__ U2,
                                                       unsigned* amax) {
  using Acc = AccT<Tout>;
  __shared__ Acc W[kMaxGram];
  __shared__ Acc W2[TWO ? kMaxGram : 1];
  for (int t = threadIdx.x; t < Db * Db; t += blockDim.x) {
    W[t] = (Acc)U[(long long)kk * Db * Db + t];
    if (TWO) W2[t] = (Acc)U2[(long long)kk * Db * Db + t];
  }
  __syncthreads();
  const long long nbase = total / Db;
  float m = 0.f;  // max |out| of this thread (with amax: the bound of an fp16 operand's source)
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nbase;
       t += (long long)gridDim.x * blockDim.x) {
    const long long base = (t / stride_b) * stride_b * Db + t % stride_b;
    Acc x[kMaxBond], x2[TWO ? kMaxBond : 1];
#pragma unroll
    for (int i = 0; i < kMaxBond; ++i)
      if (i < Db) {
        x[i] = (Acc)in[base + i * stride_b];
        if (TWO) x2[i] = (Acc)in2[base + i * stride_b];
      }
    for (int j = 0; j < Db; ++j) {
      Acc acc = 0;
#pragma unroll
      for (int i = 0; i < kMaxBond; ++i)
        if (i < Db) {
          acc += W[i * Db + j] * x[i];
          if (TWO) acc += W2[i * Db + j] * x2[i];
        }
      out[base + j * stride_b] = (Tout)acc;
      if (amax) m = fmaxf(m, abs_up((Tout)acc));
    }
  }
  if (amax) {
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(amax, __float_as_uint(m));
  }
}

// ---------------------------------------------------------------------------- transpose
template <class Tout>
__global__ void __launch_bounds__(256) k_transpose(const double* __restrict__ T, Tout* __restrict__ Tt,
                                                   long long P) {
  __shared__ double tile[32][33];
  const long long r0 = (long long)blockIdx.y * 32, c0 = (long long)blockIdx.x * 32;
  for (int k = threadIdx.y; k < 32; k += 8) {
    const long long r = r0 + k, c = c0 + threadIdx.x;
    if (r < P && c < P) tile[k][threadIdx.x] = T[r * P + c];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += 8) {
    const long long r = c0 + k, c = r0 + threadIdx.x;  // Tt[r][c] = T[c][r]
    if (r < P && c < P) Tt[r * P + c] = (Tout)tile[threadIdx.x][k];
  }
}

// ---------------------------------------------------------------------------- B operand
// Bt[(j*P + n)][k] = sum_x U3[j][k_c3][x] Tt[n][k | c3 := x]
// TWO: the row also accumulates sum_x U3b[j][k_c3][x] Tt2[n][k | c3 := x] (the tangent of the
// B operand: dBt = B_U3(dTt) + B_dU3(Tt)).
template <class Tin, class Tout, bool TWO>
__global__ void __launch_bounds__(256) k_build_bt(const Tin* __restrict__ Tt, Planes<Tout> out,
                                                  long long ld, long long P,
                                                  long long Sc, int Dc, const double* __restrict__ U3,
                                                  int chi3, const Tin* __restrict__ Tt2,
                                                  const double* __restrict__ U3b) {
  using Acc = AccT<Tout>;
  extern __shared__ unsigned char smraw[];
  Acc* W = reinterpret_cast<Acc*>(smraw);  // [chi3][Dc][Dc], then the same for U3b
  const int nW = chi3 * Dc * Dc;
  Acc* W2 = W + nW;
  for (int t = threadIdx.x; t < nW; t += blockDim.x) {
    W[t] = U3 ? (Acc)U3[t] : (Acc)1;
    if (TWO) W2[t] = (Acc)U3b[t];
  }
  __syncthreads();
  const long long total = (long long)chi3 * P * P;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long k = idx % P;
    const long long row = idx / P;  // j*P + n
    const long long n = row % P;
    const int j = (int)(row / P);
    Acc acc;
    if (Sc > 0) {
      const int kc = (int)((k / Sc) % Dc);
      const long long base = n * P + k - (long long)kc * Sc;
      const Acc* w = W + ((long long)j * Dc + kc) * Dc;
      acc = 0;
      for (int x = 0; x < Dc; ++x) acc += w[x] * (Acc)Tt[base + x * Sc];
      if (TWO) {
        const Acc* w2 = W2 + ((long long)j * Dc + kc) * Dc;
        for (int x = 0; x < Dc; ++x) acc += w2[x] * (Acc)Tt2[base + x * Sc];
      }
    } else {
      acc = (Acc)Tt[n * P + k];
    }
    store_planes(out, row * ld + k, acc);
  }
}

// ---------------------------------------------------------------------------- A operand
// Y[m][k] = X[R(k) + C(m)], R(k) = sum_{b!=a} k_b Sn_b P + k_a Sn_a, C(m) = sum_{b!=a} m_b Sn_b + m_a Sn_a P.
// Tiles of 32 columns x (32 kYMT) rows; when a is the fastest slot the source is contiguous along k
// (no transpose), otherwise along m (transpose through shared memory, one 32 x 32 tile at a time).
// Warp 0 decomposes the tile's 32 k, warps 1..kYMT its rows, at the same time, in 32-bit index
// arithmetic (P < 2^31); the fp16 scale of the planes is read once per thread.
constexpr int kYMT = 4;
template <class Tin, class Tout>
__global__ void __launch_bounds__(256) k_build_y(const Tin* __restrict__ X, Planes<Tout> out, long long ld,
                                                 Geom g, int a) {
  using Acc = AccT<Tout>;
  __shared__ Acc tile[32][33];
  __shared__ long long Rk[32], Cm[32 * kYMT];
  const int P = (int)g.P;
  const long long PP = g.P;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int m0 = blockIdx.y * 32 * kYMT, k0 = blockIdx.x * 32;
  if (ty == 0) {
    const int k = k0 + tx;
    long long rk = 0;
    for (int b = 0; b < g.d; ++b) {
      const int sb = (int)g.Sn[b];
      const long long kb = (k / sb) % g.D[b];
      rk += b == a ? kb * sb : kb * sb * PP;
    }
    Rk[tx] = rk;
  } else if (ty <= kYMT) {
    const int r = (ty - 1) * 32 + tx;
    const int m = m0 + r;
    long long cm = 0;
    for (int b = 0; b < g.d; ++b) {
      const int sb = (int)g.Sn[b];
      const long long mb = (m / sb) % g.D[b];
      cm += b == a ? mb * sb * PP : mb * sb;
    }
    Cm[r] = cm;
  }
  __syncthreads();
  const float sc = plane_scale(out);
  const int k = k0 + tx;
  if (a == g.d - 1) {
    // contiguous along k: the thread's 4 kYMT loads first, then the stores
    Acc v[4 * kYMT];
#pragma unroll
    for (int q = 0; q < 4 * kYMT; ++q) {
      const int m = m0 + ty + 8 * q;
      v[q] = (m < P && k < P) ? (Acc)X[Rk[tx] + Cm[ty + 8 * q]] : (Acc)0;
    }
#pragma unroll
    for (int q = 0; q < 4 * kYMT; ++q) {
      const int m = m0 + ty + 8 * q;
      if (m < P && k < P) store_planes_sc(out, (long long)m * ld + k, v[q], sc);
    }
  } else {
    for (int t = 0; t < kYMT; ++t) {
      for (int r = ty; r < 32; r += 8) {  // r indexes k, tx indexes m
        const int kr = k0 + r, m = m0 + t * 32 + tx;
        if (m < P && kr < P) tile[r][tx] = (Acc)X[Rk[r] + Cm[t * 32 + tx]];
      }
      __syncthreads();
      for (int r = ty; r < 32; r += 8) {  // r indexes m, tx indexes k
        const int m = m0 + t * 32 + r;
        if (m < P && k < P) store_planes_sc(out, (long long)m * ld + k, tile[tx][r], sc);
      }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------- pair contraction
template <class Tin, class Tout>
__global__ void __launch_bounds__(256) k_pair_contract(const Tin* __restrict__ in, Tout* __restrict__ out,
                                                       View v, long long total, int kaxis, int Di, int Dj,
                                                       long long si, long long sj,
                                                       const double* __restrict__ U, int chi,
                                                       long long in_base, long long out_base) {
  using Acc = AccT<Tout>;
  extern __shared__ unsigned char smraw[];
  Acc* W = reinterpret_cast<Acc*>(smraw);  // [chi][Di][Dj]
  const int nW = chi * Di * Dj;
  for (int t = threadIdx.x; t < nW; t += blockDim.x) W[t] = U ? (Acc)U[t] : (Acc)1;
  __syncthreads();
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    long long rem = idx, ioff = in_base, ooff = out_base;
    int kp = 0;
    for (int ax = v.ndim - 1; ax >= 0; --ax) {
      const long long c = rem % v.shape[ax];
      rem /= v.shape[ax];
      ioff += c * v.in_stride[ax];
      ooff += c * v.out_stride[ax];
      if (ax == kaxis) kp = (int)c;
    }
    const Acc* w = W + (long long)kp * Di * Dj;
    Acc acc = 0;
    for (int i = 0; i < Di; ++i) {
      const Tin* src = in + ioff + i * si;
      for (int j = 0; j < Dj; ++j) acc += w[i * Dj + j] * (Acc)src[j * sj];
    }
    out[ooff] = (Tout)acc;
  }
}

// All chi outputs of one "rest" index per thread: out[o + k' sk] = sum_{i,j} U[k'][i][j] in[r + i si + j sj]
// (r, o: offsets of the rest index in the input and output views). Every input element is read
// once; W is held in shared memory as [i][j][k'] so a warp reads it by broadcast.
// TWO: out also accumulates the same contraction of in2 with U2 (the tangent of an epilogue
// contraction: dR' = C_U(dR) + C_dU(R)).
// N > 0: chi = Dj = N at compile time (the steady-state shape: no predicated-off loads or FMAs,
// W rows padded to 16-byte shared-memory loads); N = 0: any chi <= 16 and Dj <= 16.
template <class Tin, class Tout, bool TWO, int N>
__global__ void __launch_bounds__(256) k_pair_contract_all(const Tin* __restrict__ in, Tout* __restrict__ out,
                                                           View v, long long total, int Di, int Dj,
                                                           long long si, long long sj, long long sk,
                                                           const double* __restrict__ U, int chi,
                                                           long long in_base, long long out_base,
                                                           const Tin* __restrict__ in2,
                                                           const double* __restrict__ U2) {
  using Acc = AccT<Tout>;
  constexpr int kMaxChi = N > 0 ? N : kMaxBond;
  constexpr int kMaxJ = N > 0 ? N : kMaxBond;
  extern __shared__ __align__(16) unsigned char smraw[];
  // W row stride: chi, or N padded to a multiple of 4
  const int ws = N > 0 ? (N + 3) / 4 * 4 : chi;
  Acc* W = reinterpret_cast<Acc*>(smraw);  // [Di*Dj][ws], then the same for U2
  const int nij = Di * Dj;
  Acc* W2 = W + (long long)ws * nij;
  for (int t = threadIdx.x; t < ws * nij; t += blockDim.x) {
    const int k = t / nij, ij = t % nij;
    W[ij * ws + k] = k < chi ? (U ? (Acc)U[t] : (Acc)1) : (Acc)0;
    if (TWO) W2[ij * ws + k] = k < chi ? (Acc)U2[t] : (Acc)0;
  }
  __syncthreads();
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    long long rem = idx, ioff = in_base, ooff = out_base;
    for (int ax = v.ndim - 1; ax >= 0; --ax) {
      const long long c = rem % v.shape[ax];
      rem /= v.shape[ax];
      ioff += c * v.in_stride[ax];
      ooff += c * v.out_stride[ax];
    }
    Acc acc[kMaxChi];
#pragma unroll
    for (int k = 0; k < kMaxChi; ++k) acc[k] = 0;
    // one row of Dj loads issued before its FMAs (bytes in flight to stream HBM)
    for (int pass = 0; pass < (TWO ? 2 : 1); ++pass) {
      const Tin* base_in = pass ? in2 : in;
      const Acc* Wp = pass ? W2 : W;
      for (int i = 0; i < Di; ++i) {
        const Tin* src = base_in + ioff + i * si;
        Acc x[kMaxJ];
#pragma unroll
        for (int j = 0; j < kMaxJ; ++j) x[j] = (N > 0 || j < Dj) ? (Acc)src[j * sj] : (Acc)0;
#pragma unroll
        for (int j = 0; j < kMaxJ; ++j) {
          if (N == 0 && j >= Dj) break;
          const Acc* w = Wp + (i * Dj + j) * ws;
#pragma unroll
          for (int k = 0; k < kMaxChi; ++k)
            if (N > 0 || k < chi) acc[k] += w[k] * x[j];
        }
      }
    }
#pragma unroll
    for (int k = 0; k < kMaxChi; ++k)
      if (N > 0 || k < chi) out[ooff + k * sk] = (Tout)acc[k];
  }
}

}  // namespace

// ============================================================================ launchers
void launch_init_tensor(double* T, long long inst_stride, int batch, int d, const double* beta,
                        const double* h, cudaStream_t s, int spin_insertion) {
  const int total = 1 << (2 * d);
  dim3 grid((total + 255) / 256, batch);
  k_init_tensor<<<grid, 256, 0, s>>>(T, inst_stride, d, beta, h, spin_insertion);
  count_launches(1);
}

void launch_step_advance(int* dstep, cudaStream_t s) {
  k_step_advance<<<1, 1, 0, s>>>(dstep);
  count_launches(1);
}

void launch_norm_log(const double* x, long long n, double* partial, double* c_out, double* lnc_log,
                     double* L, const int* dstep, int* status, cudaStream_t s) {
  k_sumsq_partial<<<kNormBlocks, 256, 0, s>>>(x, n, partial);
  count_launches(1);
  k_norm_finish<<<1, 256, 0, s>>>(partial, c_out, lnc_log, L, dstep, status);
  count_launches(1);
}

void launch_init_tangent(double* dT, long long inst_stride, int batch, int d, const double* beta, const double* h,
                         int which, cudaStream_t s) {
  const int total = 1 << (2 * d);
  k_init_tangent<<<dim3((total + 255) / 256, batch), 256, 0, s>>>(dT, inst_stride, d, beta, h, which);
  count_launches(1);
}

void launch_tangent_norm(const double* T, const double* D1, const double* D2, double* dTn, long long n,
                         const double* c, double* partial, double* dlnc, double* dL, const int* dstep,
                         cudaStream_t s) {
  k_dot_partial<<<kNormBlocks, 256, 0, s>>>(T, D1, D2, n, partial);
  count_launches(1);
  k_tangent_finish<<<1, 256, 0, s>>>(partial, c, dlnc, dL, dstep);
  count_launches(1);
  k_tangent_update<<<grid_for(n, 256), 256, 0, s>>>(T, D1, D2, dTn, n, c, dlnc);
  count_launches(1);
}

void launch_trace_tangent(const double* T, const double* dT, long long t_stride, int batch, long long P,
                          const double* dL, const int* dstep, double* out, cudaStream_t s) {
  k_trace_tangent<<<batch, 256, 0, s>>>(T, dT, t_stride, P, dL, dstep, out);
  count_launches(1);
}

void launch_trace_ratio(const double* S, const double* T, long long t_stride, int batch, long long P, double* out,
                        cudaStream_t s) {
  k_trace_ratio<<<batch, 256, 0, s>>>(S, T, t_stride, P, out);
  count_launches(1);
}

void launch_scale(const double* src, double* dst, long long n, const double* c, cudaStream_t s) {
  k_scale<<<grid_for(n, 256), 256, 0, s>>>(src, dst, n, c);
  count_launches(1);
}

void launch_trace_x(const double* T, long long t_stride, int batch, Geom g, int axis, const double* L,
                    const int* dstep, double* out3, cudaStream_t s) {
  k_trace_x<<<batch, 256, 0, s>>>(T, t_stride, g, axis, L, dstep, out3);
  count_launches(1);
}

template <class Tin, class Tout>
void launch_mode_unprimed(const Tin* in, Tout* out, Geom g, int b, const double* U, int kk,
                          cudaStream_t s, const Tin* in2, const double* U2, unsigned* amax) {
  const long long total = g.P * g.P;
  const long long nbase = total / g.D[b];
  if (amax) cudaMemsetAsync(amax, 0, sizeof(unsigned), s);
  if (in2)
    k_mode_unprimed<Tin, Tout, true><<<grid_for(nbase, 256), 256, 0, s>>>(in, out, total, g.Sn[b] * g.P,
                                                                           g.D[b], U, kk, in2, U2, amax);
  else
    k_mode_unprimed<Tin, Tout, false><<<grid_for(nbase, 256), 256, 0, s>>>(in, out, total, g.Sn[b] * g.P,
                                                                            g.D[b], U, kk, nullptr, nullptr, amax);
  count_launches(1);
}

template <class T>
void launch_absmax(const T* x, long long rows, long long cols, long long ld, unsigned* out, cudaStream_t s) {
  cudaMemsetAsync(out, 0, sizeof(unsigned), s);
  k_absmax<T><<<grid_for(rows * cols, 256), 256, 0, s>>>(x, rows, cols, ld, out);
  count_launches(1);
}
template void launch_absmax<float>(const float*, long long, long long, long long, unsigned*, cudaStream_t);
template void launch_absmax<double>(const double*, long long, long long, long long, unsigned*, cudaStream_t);

template <class Tout>
void launch_transpose(const double* T, Tout* Tt, long long P, cudaStream_t s) {
  dim3 grid((unsigned)((P + 31) / 32), (unsigned)((P + 31) / 32));
  k_transpose<Tout><<<grid, dim3(32, 8), 0, s>>>(T, Tt, P);
  count_launches(1);
}

template <class Tin, class Tout>
void launch_build_bt(const Tin* Tt, const Planes<Tout>& out, long long ld, Geom g, int c3,
                     const double* U3, int chi3, cudaStream_t s, const Tin* Tt2, const double* U3b) {
  using Acc = AccT<Tout>;
  const long long Sc = c3 >= 0 ? g.Sn[c3] : 0;
  const int Dc = c3 >= 0 ? g.D[c3] : 1;
  const int nchi = c3 >= 0 ? chi3 : 1;
  const bool two = Tt2 && c3 >= 0;
  const size_t smem = sizeof(Acc) * (size_t)nchi * Dc * Dc * (two ? 2 : 1);
  const long long total = (long long)nchi * g.P * g.P;
  if (two)
    k_build_bt<Tin, Tout, true><<<grid_for(total, 256), 256, smem, s>>>(Tt, out, ld, g.P, Sc, Dc, U3, nchi,
                                                                         Tt2, U3b);
  else
    k_build_bt<Tin, Tout, false><<<grid_for(total, 256), 256, smem, s>>>(Tt, out, ld, g.P, Sc, Dc,
                                                                          c3 >= 0 ? U3 : nullptr, nchi,
                                                                          nullptr, nullptr);
  count_launches(1);
}

template <class Tin, class Tout>
void launch_build_y(const Tin* X, const Planes<Tout>& out, long long ld, Geom g, int a,
                    cudaStream_t s) {
  dim3 grid((unsigned)((g.P + 31) / 32), (unsigned)((g.P + 32 * kYMT - 1) / (32 * kYMT)));
  k_build_y<Tin, Tout><<<grid, dim3(32, 8), 0, s>>>(X, out, ld, g, a);
  count_launches(1);
}

template <class Tin, class Tout>
void launch_pair_contract(const Tin* in, Tout* out, const View& v, int kaxis, int Di, int Dj,
                          long long si, long long sj, const double* U, int chi, long long in_base,
                          long long out_base, cudaStream_t s) {
  using Acc = AccT<Tout>;
  long long total = 1;
  for (int i = 0; i < v.ndim; ++i) total *= v.shape[i];
  const int nchi = U ? chi : 1;
  const size_t smem = sizeof(Acc) * (size_t)nchi * Di * Dj;
  k_pair_contract<Tin, Tout><<<grid_for(total, 256), 256, smem, s>>>(in, out, v, total, kaxis, Di, Dj,
                                                                      si, sj, U, nchi, in_base, out_base);
  count_launches(1);
}

template <class Tin, class Tout>
void launch_pair_contract_all(const Tin* in, Tout* out, const View& rest, int Di, int Dj, long long si,
                              long long sj, long long sk, const double* U, int chi, long long in_base,
                              long long out_base, cudaStream_t s, const Tin* in2, const double* U2) {
  using Acc = AccT<Tout>;
  long long total = 1;
  for (int i = 0; i < rest.ndim; ++i) total *= rest.shape[i];
  const size_t smem = sizeof(Acc) * (size_t)chi * Di * Dj * (in2 ? 2 : 1);
  const size_t smem_pad = sizeof(Acc) * (size_t)((chi + 3) / 4 * 4) * Di * Dj;
  const int grid = grid_for(total, 256);
  if (in2) {
    k_pair_contract_all<Tin, Tout, true, 0><<<grid, 256, smem, s>>>(in, out, rest, total, Di, Dj, si, sj, sk, U,
                                                                     chi, in_base, out_base, in2, U2);
    count_launches(1);
    return;
  }
  // the steady-state FP32 shape (chi = Dj) with compile-time extents
  if constexpr (std::is_same<Tin, float>::value) {
    if (U && chi == Dj && chi >= 6) switch (chi) {
#define HOTRG_PCA(NN)                                                                                      \
  case NN:                                                                                                 \
    k_pair_contract_all<Tin, Tout, false, NN><<<grid, 256, smem_pad, s>>>(in, out, rest, total, Di, Dj, si, sj, \
                                                                          sk, U, chi, in_base, out_base,      \
                                                                          nullptr, nullptr);                  \
    count_launches(1);                                                                                     \
    return;
      HOTRG_PCA(6) HOTRG_PCA(7) HOTRG_PCA(8) HOTRG_PCA(9) HOTRG_PCA(10) HOTRG_PCA(11)
      HOTRG_PCA(12) HOTRG_PCA(13) HOTRG_PCA(14) HOTRG_PCA(15) HOTRG_PCA(16)
#undef HOTRG_PCA
        default:
          break;
      }
  }
  k_pair_contract_all<Tin, Tout, false, 0><<<grid, 256, smem, s>>>(in, out, rest, total, Di, Dj, si, sj, sk, U,
                                                                    chi, in_base, out_base, nullptr, nullptr);
  count_launches(1);
}

// The two-input contractions and B-operand builds in FP64 can need more than the default 48 KB
// of dynamic shared memory (2 x 16 x 256 doubles): raise the limit once, outside any capture.
void prepare_kernel_attributes() {
  const int big = (int)(2 * sizeof(double) * kMaxBond * kMaxGram);
  cudaFuncSetAttribute(k_pair_contract_all<double, double, true, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       big);
  cudaFuncSetAttribute(k_pair_contract_all<float, float, true, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_pair_contract_all<float, double, true, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       big);
  cudaFuncSetAttribute(k_build_bt<double, double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_build_bt<float, __nv_bfloat16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
}

// explicit instantiations: FP64 path (double everywhere) and BF16X3 path (float intermediates)
template void launch_mode_unprimed<double, double>(const double*, double*, Geom, int, const double*, int, cudaStream_t,
                                                   const double*, const double*, unsigned*);
template void launch_mode_unprimed<double, float>(const double*, float*, Geom, int, const double*, int, cudaStream_t,
                                                  const double*, const double*, unsigned*);
template void launch_mode_unprimed<float, float>(const float*, float*, Geom, int, const double*, int, cudaStream_t,
                                                 const float*, const double*, unsigned*);
template void launch_transpose<double>(const double*, double*, long long, cudaStream_t);
template void launch_transpose<float>(const double*, float*, long long, cudaStream_t);
template void launch_build_bt<double, double>(const double*, const Planes<double>&, long long, Geom, int, const double*, int,
                                              cudaStream_t, const double*, const double*);
template void launch_build_bt<float, __nv_bfloat16>(const float*, const Planes<__nv_bfloat16>&, long long, Geom, int,
                                                    const double*, int, cudaStream_t, const float*, const double*);
template void launch_build_y<double, double>(const double*, const Planes<double>&, long long, Geom, int, cudaStream_t);
template void launch_build_y<float, __nv_bfloat16>(const float*, const Planes<__nv_bfloat16>&, long long, Geom, int, cudaStream_t);
template void launch_build_y<double, __nv_bfloat16>(const double*, const Planes<__nv_bfloat16>&, long long, Geom, int, cudaStream_t);
template void launch_pair_contract<double, double>(const double*, double*, const View&, int, int, int, long long, long long, const double*, int, long long, long long, cudaStream_t);
template void launch_pair_contract<float, float>(const float*, float*, const View&, int, int, int, long long, long long, const double*, int, long long, long long, cudaStream_t);
template void launch_pair_contract<float, double>(const float*, double*, const View&, int, int, int, long long, long long, const double*, int, long long, long long, cudaStream_t);
template void launch_pair_contract_all<double, double>(const double*, double*, const View&, int, int, long long, long long,
                                                       long long, const double*, int, long long, long long, cudaStream_t,
                                                       const double*, const double*);
template void launch_pair_contract_all<float, float>(const float*, float*, const View&, int, int, long long, long long,
                                                     long long, const double*, int, long long, long long, cudaStream_t,
                                                     const float*, const double*);
template void launch_pair_contract_all<float, double>(const float*, double*, const View&, int, int, long long, long long,
                                                      long long, const double*, int, long long, long long, cudaStream_t,
                                                      const float*, const double*);

}  // namespace hotrg
