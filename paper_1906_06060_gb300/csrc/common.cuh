// Shared device/host definitions of libhotrg (GB300, sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
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

// Exponent e of the power-of-two scale 2^e applied to an operand before its fp16 split, for an
// operand whose entries are bounded by `bound`: the largest e with bound * 2^e < 2^15, so every
// scaled entry is below 2^15 (fp16 holds up to 65504) and the largest one is at least 2^14.
// Clamped to [-60, 60] (0 for a zero or non-finite bound). Both the operand builders and the GEMM's
// epilogue (which multiplies by 2^-(eA + eB)) compute it with this function from the same inputs.
__host__ __device__ __forceinline__ int f16_scale_exponent(float bound) {
  if (!(bound > 0.f) || !(bound < 3.0e38f)) return 0;
  int ex = 0;
  frexpf(bound, &ex);  // bound = f 2^ex, 0.5 <= f < 1
  int e = 15 - ex;
  return e < -60 ? -60 : (e > 60 ? 60 : e);
}
// 2^e as a float, exactly, for |e| <= 126
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

// Operand planes of a split-precision GEMM operand: nparts = 2 (hi, lo) or 3 (hi, mid, lo),
// part i = rn(x - sum of the previous parts); or a single FP64 plane (nparts = 1).
// fmt 0: bf16 parts of x. fmt 1 (two-part only): fp16 parts of x 2^e, e = f16_scale_exponent of
// amax_mult * (*amax), where *amax holds the bits of max |x| of the operand's source (a
// non-negative float, so its bits order like its value): fp16 keeps 11 significant bits per part,
// and the exact power-of-two scale keeps the operand inside fp16's exponent range.
template <class T>
struct Planes {
  T* p[3];
  int nparts;
  int fmt = 0;
  const unsigned* amax = nullptr;
  float amax_mult = 1.f;
};

__device__ __forceinline__ float plane_bound(const unsigned* amax, float mult) {
  return mult * __uint_as_float(*amax);
}

__device__ __forceinline__ void store_planes(const Planes<__nv_bfloat16>& o, long long i, float x) {
  if (o.fmt) {
    // fp16 hi + lo of the scaled value, stored as raw 16-bit patterns in the plane arrays
    const float xs = x * pow2f(f16_scale_exponent(plane_bound(o.amax, o.amax_mult)));
    const __half hi = __float2half_rn(xs);
    const __half lo = __float2half_rn(xs - __half2float(hi));
    o.p[0][i] = __ushort_as_bfloat16(__half_as_ushort(hi));
    if (o.nparts > 1) o.p[1][i] = __ushort_as_bfloat16(__half_as_ushort(lo));
    return;
  }
  float r = x;
  for (int k = 0; k < o.nparts; ++k) {
    const __nv_bfloat16 v = __float2bfloat16_rn(r);
    o.p[k][i] = v;
    r -= __bfloat162float(v);
  }
}
__device__ __forceinline__ void store_planes(const Planes<double>& o, long long i, double x) { o.p[0][i] = x; }

// The same with the fp16 scale 2^e read once by the caller (plane_scale), for kernels that store
// many entries per thread; the plane pointers are indexed with compile-time indices only.
__device__ __forceinline__ float plane_scale(const Planes<__nv_bfloat16>& o) {
  return o.fmt ? pow2f(f16_scale_exponent(plane_bound(o.amax, o.amax_mult))) : 1.f;
}
__device__ __forceinline__ float plane_scale(const Planes<double>&) { return 1.f; }
__device__ __forceinline__ void store_planes_sc(const Planes<__nv_bfloat16>& o, long long i, float x, float sc) {
  if (o.fmt) {
    const float xs = x * sc;
    const __half hi = __float2half_rn(xs);
    const __half lo = __float2half_rn(xs - __half2float(hi));
    o.p[0][i] = __ushort_as_bfloat16(__half_as_ushort(hi));
    if (o.nparts > 1) o.p[1][i] = __ushort_as_bfloat16(__half_as_ushort(lo));
    return;
  }
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  o.p[0][i] = h;
  if (o.nparts > 1) {
    const float r1 = x - __bfloat162float(h);
    const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
    o.p[1][i] = mid;
    if (o.nparts > 2) o.p[2][i] = __float2bfloat16_rn(r1 - __bfloat162float(mid));
  }
}
__device__ __forceinline__ void store_planes_sc(const Planes<double>& o, long long i, double x, float) {
  o.p[0][i] = x;
}

}  // namespace hotrg
