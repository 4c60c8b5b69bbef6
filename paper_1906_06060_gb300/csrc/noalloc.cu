// hotrg_gemm_split_noalloc: the split-precision squeeze GEMM for callers that cannot allocate
// device memory.
//
// hotrg_gemm_split needs a caller-provided scratch buffer for the bf16 operand planes and its
// status word. Some callers have no way to provide one: a process whose device memory is
// already reserved in full by another framework's pool, or a latency-critical loop that must
// not call cudaMalloc (which can synchronise the whole device). This variant keeps that
// scratch in a fixed file-scope device array instead, so the caller passes only A, Bt and C.
//
// The array (kNoallocBytes, about 12 MiB) belongs to this library's device code: every GPU on
// which it is used holds it until the process exits. Its device address is looked up once per
// device with cudaGetSymbolAddress, on the first call made while that device is current. Every
// call synchronises its stream and copies the status word to the host, so the entry point
// cannot be used inside a stream capture at all. All calls share the array, so calls whose GPU
// work overlaps (different streams, or different host threads) race on it; calls on one stream
// are safe in sequence.
#include <mutex>

#include "kernels.h"

namespace hotrg {
namespace {

constexpr long long kNoallocMaxElems = HOTRG_GEMM_NOALLOC_MAX_ELEMS;  // (M + N) * round_up(K, 64)
constexpr size_t kNoallocStatusBytes = 256;
// six bf16 planes of (M + N) * round_up(K, 64) elements in all, each plane start rounded up to
// 256 bytes (at most 255 bytes of padding per plane): every request within the limit fits
constexpr size_t kNoallocBytes = kNoallocStatusBytes + 3 * 2 * (size_t)kNoallocMaxElems + 6 * 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set-up on first use).
void* noalloc_scratch(int* err) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    *err = HOTRG_EDEVICE;
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      *err = HOTRG_EDEVICE;
      return nullptr;
    }
    g_noalloc_addr[dev] = p;
  }
  return g_noalloc_addr[dev];
}

long long round64(long long x) { return (x + 63) / 64 * 64; }

}  // namespace
}  // namespace hotrg

using namespace hotrg;

extern "C" int hotrg_gemm_split_noalloc(const float* A, long long lda, const float* Bt, long long ldb,
                                        float* C, long long ldc, long long M, long long N, long long K,
                                        int npass, void* stream) {
  if (!A || !Bt || !C || M <= 0 || N <= 0 || K <= 0 || lda < K || ldb < K || ldc < N) return HOTRG_EINVAL;
  if (npass != 1 && npass != 3 && npass != 4 && npass != 6) return HOTRG_EINVAL;
  // the smallest problem the tensor-core kernel takes: one 128 x 256 output tile, one 64-wide k-block
  if (M < 128 || N < 256 || K < 64) return HOTRG_EINVAL;
  const long long ld = round64(K);
  if (M > kNoallocMaxElems || N > kNoallocMaxElems || (M + N) > kNoallocMaxElems / ld) return HOTRG_EINVAL;
  int err = HOTRG_OK;
  char* base = static_cast<char*>(noalloc_scratch(&err));
  if (!base) return err;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* status = reinterpret_cast<int*>(base);
  // planes packed for this call's sizes: A planes (M x ld), then B planes (N x ld), 256-B aligned
  const size_t a_plane = (size_t)((M * ld * 2 + 255) / 256 * 256);
  const size_t b_plane = (size_t)((N * ld * 2 + 255) / 256 * 256);
  char* p = base + kNoallocStatusBytes;
  if (kNoallocStatusBytes + 3 * (a_plane + b_plane) > kNoallocBytes) return HOTRG_EINVAL;
  const int nparts = npass == 1 ? 1 : (npass == 6 ? 3 : 2);
  Planes<__nv_bfloat16> Ap, Bp;
  Ap.nparts = Bp.nparts = nparts;
  for (int k = 0; k < 3; ++k) {
    Ap.p[k] = reinterpret_cast<__nv_bfloat16*>(p);
    p += a_plane;
  }
  for (int k = 0; k < 3; ++k) {
    Bp.p[k] = reinterpret_cast<__nv_bfloat16*>(p);
    p += b_plane;
  }
  // the array keeps the previous call's contents: the status word must start at zero
  if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) return HOTRG_EDEVICE;
  launch_split_rows(A, lda, M, K, Ap, ld, s);
  launch_split_rows(Bt, ldb, N, K, Bp, ld, s);
  const int rc = launch_gemm_split(Ap, ld, Bp, ld, C, ldc, M, N, K, npass, status, 4.0, s);
  if (rc) return rc;
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return HOTRG_EDEVICE;
  }
  int bits = 0;
  if (cudaMemcpy(&bits, status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return HOTRG_EDEVICE;
  if (bits & ST_TIMEOUT) return HOTRG_ETIMEOUT;
  return bits ? HOTRG_EDEVICE : HOTRG_OK;
}
