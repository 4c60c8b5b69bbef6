// Shared device/host definitions of libhotrg (GB300, sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/hotrg.h"

namespace hotrg {

constexpr int kMaxD = 4;         // lattice dimension
constexpr int kMaxLegs = 2 * kMaxD;
constexpr int kMaxBond = 16;     // Dcut upper bound (Gram matrices are at most 256 x 256)
constexpr int kMaxGram = kMaxBond * kMaxBond;

// Device status bits (OR-ed into an int in the workspace); mapped to hotrg_status on the host.
enum : int {
  ST_NUMERIC = 1,   // NaN/Inf/zero norm, non-positive trace
  ST_NOCONV = 2,    // eigensolver sweep limit reached
  ST_TIMEOUT = 4,   // bounded wait gave up
  ST_BOUNDS = 8,    // internal index check failed
  ST_Z2 = 16,       // zero-field block structure broken (an eigenvector is not parity-pure)
};

// Geometry of a site tensor in natural layout T[u_0..u_{d-1}, p_0..p_{d-1}].
struct Geom {
  int d;
  int D[kMaxD];
  long long P;              // prod D
  long long Sn[kMaxD];      // stride of slot b inside one half: prod_{c>b} D_c
};

inline __host__ __device__ Geom make_geom(int d, const int* D) {
  Geom g;
  g.d = d;
  g.P = 1;
  for (int b = 0; b < kMaxD; ++b) g.D[b] = 1;
  for (int b = 0; b < d; ++b) g.D[b] = D[b];
  for (int b = d - 1; b >= 0; --b) { g.Sn[b] = g.P; g.P *= D[b]; }
  for (int b = d; b < kMaxD; ++b) g.Sn[b] = 0;
  return g;
}

// Strided view of a tensor with up to 12 axes: used by the generic gather kernels.
constexpr int kMaxAxes = 12;
struct View {
  int ndim;
  int shape[kMaxAxes];
  long long in_stride[kMaxAxes];
  long long out_stride[kMaxAxes];
};

__device__ __forceinline__ void atomic_status(int* st, int bits) {
  if (st) atomicOr(st, bits);
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Split x into bf16 hi + lo with hi = rn(x), lo = rn(x - hi).
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// Operand planes of a split-precision GEMM operand: nparts = 2 (hi, lo) or 3 (hi, mid, lo),
// part i = rn_bf16(x - sum of the previous parts); or a single FP64 plane (nparts = 1).
template <class T>
struct Planes {
  T* p[3];
  int nparts;
};

__device__ __forceinline__ void store_planes(const Planes<__nv_bfloat16>& o, long long i, float x) {
  float r = x;
  for (int k = 0; k < o.nparts; ++k) {
    const __nv_bfloat16 v = __float2bfloat16_rn(r);
    o.p[k][i] = v;
    r -= __bfloat162float(v);
  }
}
__device__ __forceinline__ void store_planes(const Planes<double>& o, long long i, double x) { o.p[0][i] = x; }

}  // namespace hotrg
