// Squeeze GEMM on the 5th-generation tensor cores (sm_103a): the O(Dcut^15) contraction of
// arXiv:1906.06060 Sec. 2 (cost statement), written as C[m][n] = sum_k A[m][k] Bt[n][k].
//
// Precision: each FP32 operand is split into bf16 planes, x = hi + lo (2 planes) or
// x = hi + mid + lo (3 planes), each plane the bf16 rounding of what the previous ones left.
// The GEMM sums plane products ("passes"): with two planes hi*hi + hi*lo + lo*hi (3 passes) or
// all four products (4 passes, adds lo*lo), with three planes hh, hm, mh, hl, mm, lh (6
// passes), accumulating in FP32 in tensor memory. Per product the dropped terms and split
// residuals are O(2^-16) relative for 3 passes, O(2^-17) unbiased for 4 and O(2^-24) for 6. The
// dropped lo*lo of 3 passes is systematic when A and B are built from the same tensor.
// fp16 planes (two of them, 3 or 4 passes): each operand is scaled by an exact power of two 2^e
// that brings its largest entry just below 2^15, then split into fp16 hi + lo (11 significant
// bits each, O(2^-22) per product); the epilogue multiplies by 2^-(eA + eB). Same MMA cost as
// bf16 (kind::f16 takes either type; A and B always share one).
//
// Batched launches: a persistent launch can cover several independent products of one shape (a
// group of instances of a temperature scan): the tile list runs over the instances one after the
// other, the operand planes are 3D tensor maps whose third coordinate is the instance, and each
// instance has its own output, block descriptor and fp16 scale bounds.
//
// Accumulation: the tensor core's FP32 accumulate rounds toward zero, so a long chain of MMAs
// into one TMEM accumulator drifts systematically towards zero by about (chain length) x 2^-25
// relative - for K = 10^4 and 3 passes about 1e-4, far above what the free energy tolerates.
// The accumulator is therefore restarted for every 64-wide k-block (chain: npass x 4 MMAs, the
// small cross terms first so the large hi*hi products meet a small accumulator) and each
// k-block's partial sum is folded into an FP32 register accumulator with round-to-nearest adds.
//
// Kernel structure (one CTA per SM, persistent over output tiles, 320 threads):
//   warp 0      TMA producer: per k-block loads every 16-bit plane of the 128 x BK A tile and
//               of the 256 x BK B tile (BK*2-byte swizzle) into one stage of a shared-memory
//               ring, so the passes of a k-block reuse the same stage (BK = 64 or 32).
//   warp 1      MMA issuer: one thread issues tcgen05.mma.cta_group::1.kind::f16 (M=128,
//               N=256, K=16) for all passes of one k-block into one of two TMEM buffers (2 x 256
//               FP32 columns), releases the stage and hands the buffer over with tcgen05.commit.
//   warps 2-9   fold/epilogue: warp w reads TMEM lanes 32*(w%4).. (its hardware quadrant),
//               columns 128*((w-2)/4).. of the buffer, adds them into 128 FP32 registers per
//               thread and frees the buffer; after the last k-block it stores its 128 columns.
//
// CTA pairs (CG = 2, a thread-block cluster of two CTAs on two SMs, one 256 x 256 output tile):
// each CTA stages its own 128 A rows and half (128) of the tile's B rows per k-block, so a stage
// is 64 KB instead of 96 KB at BK = 64 (three stages fit instead of two) and each SM moves 2/3 of
// the shared-memory operand bytes per MMA flop. The first CTA's thread issues
// tcgen05.mma.cta_group::2 (M = 256): the tensor cores of both SMs read A from their own CTA and B
// from both, and each CTA's TMEM receives its 128 rows. The first CTA's producer issues the TMA
// copies of both CTAs (the second CTA's land in its shared memory through mapa addresses) and all
// bytes count on the first CTA's stage barriers, so stage hand-over never crosses SMs; the MMA
// commits free the stage there and reach the TMEM-full barriers of both CTAs (multicast); the
// fold warps of both report freed TMEM buffers to the first CTA. Measured reasons: a single CTA's
// 128 x 256 MMA chain, with operands resident and nothing else running, kept the tensor pipe busy
// about 2/3 of the time (pairs: about 3/4); and a pair whose second CTA issued its own copies,
// counted remotely on the first CTA's barrier, lost a quarter of its rate to the cross-SM hand-over.
// Every mbarrier wait is bounded by a timeout; on expiry the CTA records ST_TIMEOUT, drains
// the copies and MMAs it issued (waits bounded by max(timeout, 1 s): issued work always
// completes, so a short caller limit never lets the CTA exit before it), frees TMEM and returns.
#include <cuda.h>

#include <algorithm>
#include <atomic>
#include <cstring>

#include "kernels.h"

namespace hotrg {

namespace {

constexpr int TC_BM = 128, TC_BN = 256;
constexpr int kMaxDevices = 64;
constexpr int TC_THREADS = 320;
constexpr int TC_FOLD_THREADS = 256;  // warps 2-9
constexpr uint32_t TMEM_COLS = 2 * TC_BN;

// k-block width BK (16-bit elements per tile row): 64 -> 128-byte swizzle, 32 -> 64-byte
// swizzle. A stage holds every plane of one k-block of the CTA's A rows (128) and B rows (256, or
// 128 for a CTA pair); as many stages as fit 216 KB, at most 6. The accumulator is folded once per
// k-block (or fold group).
template <int BK, int NPL, int CG>
struct Cfg {
  static constexpr uint32_t A_TILE = TC_BM * BK * 2;
  static constexpr uint32_t B_TILE = (TC_BN / CG) * BK * 2;
  static constexpr uint32_t STAGE_BYTES = NPL * (A_TILE + B_TILE);
  static constexpr int STAGES = (int)((216u * 1024u) / STAGE_BYTES) > 6 ? 6 : (int)((216u * 1024u) / STAGE_BYTES);
  static constexpr size_t SMEM = 1024 + STAGES * STAGE_BYTES + 256;
};

// kind::f16 instruction descriptor: D = F32 (bits 4-5 = 1), A and B format (bits 7-9, 10-12:
// 1 = BF16, 0 = F16; A and B always of the same type), both K-major, N >> 3 at bits 17-22,
// M >> 4 at bits 24-28 (M = 128 for one CTA, 256 for a CTA pair: 128 rows in each).
constexpr uint32_t idesc_for(bool f16, int cg) {
  return (1u << 4) | (f16 ? 0u : (1u << 7) | (1u << 10)) | ((uint32_t)(TC_BN >> 3) << 17) |
         ((uint32_t)((TC_BM * cg) >> 4) << 24);
}

struct TmapSet {
  CUtensorMap a[3];
  CUtensorMap b[3];
};

// plane index of A and B for each pass, smallest products first, hi*hi last
//   npass 1: hh    npass 3: hl, lh, hh    npass 4: ll, hl, lh, hh (two planes, all products)
//   npass 6: lh, mm, hl, mh, hm, hh (three planes h=0, m=1, l=2)
__host__ __device__ constexpr int pass_plane_a(int npass, int ps) {
  return npass == 1 ? 0
       : npass == 3 ? (ps == 1 ? 1 : 0)
       : npass == 4 ? ((ps == 0 || ps == 2) ? 1 : 0)
       : (ps == 0 ? 2 : (ps == 1 || ps == 3) ? 1 : 0);
}
__host__ __device__ constexpr int pass_plane_b(int npass, int ps) {
  return npass == 1 ? 0
       : npass == 3 ? (ps == 0 ? 1 : 0)
       : npass == 4 ? ((ps == 0 || ps == 1) ? 1 : 0)
       : (ps == 2 ? 2 : (ps == 1 || ps == 4) ? 1 : 0);
}
static_assert(pass_plane_a(6, 0) == 2 && pass_plane_b(6, 0) == 0, "lh first");
static_assert(pass_plane_a(6, 5) == 0 && pass_plane_b(6, 5) == 0, "hh last");
static_assert(pass_plane_a(3, 2) == 0 && pass_plane_b(3, 2) == 0, "hh last");
static_assert(pass_plane_a(4, 0) == 1 && pass_plane_b(4, 0) == 1, "ll first");

struct TcParams {
  long long M, N, K;
  int num_m, num_n, num_kb, npass;
  int group_m;     // output tiles are rastered in groups of group_m M-tiles (L2 reuse of A and B)
  float* C;
  long long ldc;
  int* status;
  unsigned long long timeout_ns;
  int vec4;
  const GemmBlocks* blk;  // null: one dense product over M x N x K
  uint32_t idesc;         // idesc_for(fp16 operands, CTA group)
  // fp16 operands carry power-of-two scales 2^eA, 2^eB (see Planes): the epilogue multiplies by
  // 2^-(eA + eB). Null amax: no scaling.
  const unsigned* amaxA;
  const unsigned* amaxB;
  float multA, multB;
  // batched launch: `batch` independent products of the same shape; instance i reads the operand
  // planes at z = i of the 3D tensor maps, writes C + i c_inst, takes the descriptor blk[i] and the
  // scale bounds amax + i amax_inst
  int batch;
  long long c_inst;
  int amax_inst;
  // wait probe: the producer issues no copies, so the first wait for a stage can never be satisfied
  // and must run out (nothing is in flight to drain)
  int stall;
};

// One output block of the product as the kernel sees it (clamped to the operand extents).
struct Blk {
  int m0, mc, n0, nc, k0, num_m, num_n, num_kb, tiles;
};

// The (at most two) blocks of instance `inst`: from its device descriptor of a block-sparse
// product (clamped to the operand extents), or the single dense block. Output tiles are
// (128 CG) x 256: a CTA pair (CG = 2) computes 256 rows.
template <int BK, int CG>
__device__ __forceinline__ int load_blocks(const TcParams& p, int inst, Blk* b) {
  int nb = 1;
  if (p.blk) {
    const GemmBlocks* g = p.blk + inst;
    nb = min(max(g->nb, 0), 2);
    for (int i = 0; i < nb; ++i) {
      const long long m0 = max(g->m0[i], 0), n0 = max(g->n0[i], 0), k0 = max(g->k0[i], 0);
      b[i].m0 = (int)min(m0, p.M);
      b[i].n0 = (int)min(n0, p.N);
      b[i].k0 = (int)min(k0, p.K);
      b[i].mc = (int)min((long long)max(g->mc[i], 0), p.M - b[i].m0);
      b[i].nc = (int)min((long long)max(g->nc[i], 0), p.N - b[i].n0);
      const int kc = (int)min((long long)max(g->kc[i], 0), p.K - b[i].k0);
      b[i].num_kb = (kc + BK - 1) / BK;
    }
  } else {
    b[0].m0 = b[0].n0 = b[0].k0 = 0;
    b[0].mc = (int)p.M;
    b[0].nc = (int)p.N;
    b[0].num_kb = p.num_kb;
  }
  for (int i = 0; i < nb; ++i) {
    b[i].num_m = (b[i].mc + TC_BM * CG - 1) / (TC_BM * CG);
    b[i].num_n = (b[i].nc + TC_BN - 1) / TC_BN;
    b[i].tiles = b[i].num_m * b[i].num_n;
  }
  return nb;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait. Returns false if another role aborted or this wait exceeded timeout_ns.
__device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                       unsigned long long timeout_ns, bool honour_abort = true) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer_ns();
  for (;;) {
#pragma unroll 1
    for (int i = 0; i < 32; ++i)
      if (mbar_try_wait(bar, parity)) return true;
    if (honour_abort && *abort_flag) return false;
    if (globaltimer_ns() - t0 > timeout_ns) {
      *abort_flag = 1;
      return false;
    }
  }
}
// Limit of the waits for work this CTA already issued (TMA copies, MMAs), which always
// completes: at least one second, so that a short caller limit cannot let the CTA exit (and
// release TMEM or shared memory) while that work is still in flight.
__device__ __forceinline__ unsigned long long drain_ns(unsigned long long timeout_ns) {
  return timeout_ns > 1000000000ull ? timeout_ns : 1000000000ull;
}
// 3D tiled load: x along K (a multiple of BK: 16-byte aligned starts), y the tile's first row, z the
// instance of a batched launch (0 otherwise)
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y,
                                            int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
      "[%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y), "r"(z)
      : "memory");
}
// The same load for a CTA pair, issued by the pair's first CTA: `dst` is a shared::cluster address in
// either CTA (mapa for the second), the bytes count on the first CTA's barrier `bar`.
__device__ __forceinline__ void tma_load_3d_pair(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y,
                                                 int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, "
      "{%3, %4, %5}], [%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y), "r"(z)
      : "memory");
}
// shared::cluster address of this CTA's shared-memory location `a` in cluster CTA `rank`
__device__ __forceinline__ uint32_t mapa_rank(uint32_t a, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// every thread of both CTAs of the cluster (release / acquire at cluster scope)
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}
// arrive on a barrier of another CTA of the cluster (shared::cluster address)
__device__ __forceinline__ void mbar_arrive_remote(uint32_t bar) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// No "memory" clobber: the MMA reads shared memory the async proxy filled and writes TMEM; its
// order against the mbarrier waits and tcgen05.commit around it is kept because all of these are
// volatile asm statements, which the compiler does not reorder among themselves.
// CG = 2: issued by the pair's first CTA; A rows and B rows come from both CTAs' shared memory
// (the same offsets), each CTA's tensor memory receives its 128 rows of D.
template <int CG>
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
  if constexpr (CG == 1)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
// Arrive on `bar` once the MMAs this thread issued so far have completed. CG = 2: on the barrier
// at the same offset in both CTAs of the pair.
template <int CG>
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  if constexpr (CG == 1)
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
  else
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            bar),
        "h"((uint16_t)3)
        : "memory");
}
// the same, on this CTA's barrier only
template <int CG>
__device__ __forceinline__ void mma_commit_local(uint32_t bar) {
  if constexpr (CG == 1)
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
  else
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
// Shared-memory matrix descriptor, K-major operand staged by TMA with a BK*2-byte swizzle:
// start address >> 4 (bits 0-13), leading byte offset 16 B (unused for these layouts, bits
// 16-29), stride byte offset = 8 rows x BK*2 bytes between 8-row groups (bits 32-45), version 1
// (bits 46-47), base offset 0 (tiles are 1024-B aligned), layout SWIZZLE_128B = 2 or
// SWIZZLE_64B = 4 (bits 61-63). Consecutive K=16 slices are 32 bytes apart inside a row.
template <int BK>
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= ((uint64_t)(BK == 64 ? 1024 : 512) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)(BK == 64 ? 2 : 4) << 61;
  return d;
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void raster(int tile, int num_m, int num_n, int group_m, int& mt, int& nt) {
  const int per_group = group_m * num_n;
  const int g = tile / per_group;
  const int first_m = g * group_m;
  const int gsz = min(num_m - first_m, group_m);
  const int local = tile - g * per_group;
  mt = first_m + local % gsz;
  nt = local / gsz;
}

// Tile -> (instance, block, M-tile, N-tile). Instances' tiles are numbered one after the other
// (prefix[i] = first tile of instance i, for block-sparse launches), and inside an instance the
// blocks' tiles one after the other.
template <int BK, int CG>
__device__ __forceinline__ void locate(const TcParams& p, const int* prefix, int tile, int& inst, Blk& bk, int& mt,
                                       int& nt) {
  Blk b[2];
  int local;
  if (!p.blk) {
    load_blocks<BK, CG>(p, 0, b);
    inst = tile / b[0].tiles;
    local = tile - inst * b[0].tiles;
    bk = b[0];
  } else {
    int lo = 0, hi = p.batch;  // prefix[lo] <= tile < prefix[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (prefix[mid] <= tile) lo = mid;
      else hi = mid;
    }
    inst = lo;
    local = tile - prefix[lo];
    const int nb = load_blocks<BK, CG>(p, inst, b);
    const int bi = (nb > 1 && local >= b[0].tiles) ? 1 : 0;
    if (bi) local -= b[0].tiles;
    bk = b[bi];
  }
  raster(local, bk.num_m, bk.num_n, p.group_m, mt, nt);
}

template <int BK, int NPL, int NPASS, int FG, int CG>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_gemm_split(const __grid_constant__ TmapSet maps, TcParams p) {
  using C = Cfg<BK, NPL, CG>;
  static_assert(FG == 1 || FG <= C::STAGES - 1, "a fold group leaves one stage to the producer");
  static_assert(CG == 1 || CG == 2, "one CTA or a CTA pair");
  constexpr int TC_STAGES = C::STAGES;
  constexpr uint32_t A_TILE = C::A_TILE, B_TILE = C::B_TILE, STAGE_BYTES = C::STAGE_BYTES;
  constexpr int TC_BK = BK;
  constexpr int B_ROWS = TC_BN / CG;  // B rows this CTA stages per k-block
  static_assert(TC_STAGES >= 2, "ring needs two stages");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  // stage s: A planes 0..NPL-1 then B planes 0..NPL-1
  auto a_tile = [&](int stage, int pl) { return smem + stage * STAGE_BYTES + pl * A_TILE; };
  auto b_tile = [&](int stage, int pl) { return smem + stage * STAGE_BYTES + NPL * A_TILE + pl * B_TILE; };
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + TC_STAGES * STAGE_BYTES);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * TC_STAGES + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const uint32_t full0 = smem_u32(bars);
  const uint32_t empty0 = full0 + 8 * TC_STAGES;
  const uint32_t tfull0 = empty0 + 8 * TC_STAGES;
  const uint32_t tempty0 = tfull0 + 16;
  const uint32_t final_bar = tempty0 + 16;
  // CTA pair: rank 0 issues the MMAs and owns the stage-full and TMEM-empty barriers both CTAs
  // signal; every CTA walks the same tiles (one per cluster)
  const uint32_t rank = CG == 2 ? cluster_rank() : 0u;
  const bool leader = rank == 0;
  const int cta0 = (int)blockIdx.x / CG, ncta = (int)gridDim.x / CG;

  __shared__ int s_prefix[kMaxGemmBatch + 1];
  __shared__ int s_total;
  if (threadIdx.x == 0) {
    Blk b[2];
    if (p.blk) {
      // first tile of every instance (block-sparse: the descriptors differ per instance)
      int t = 0;
      for (int i = 0; i < p.batch; ++i) {
        s_prefix[i] = t;
        const int nb = load_blocks<BK, CG>(p, i, b);
        t += b[0].tiles + (nb > 1 ? b[1].tiles : 0);
      }
      s_prefix[p.batch] = t;
      s_total = t;
    } else {
      load_blocks<BK, CG>(p, 0, b);
      s_total = b[0].tiles * p.batch;
    }
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull0 + 8 * b, 1);
      mbar_init(tempty0 + 8 * b, CG * TC_FOLD_THREADS / 32);
    }
    mbar_init(final_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0 && lane < 2 * NPL) {
    const CUtensorMap* m = lane < NPL ? &maps.a[lane] : &maps.b[lane - NPL];
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(m)) : "memory");
  }
  if (warp == 1) {
    if constexpr (CG == 1) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                   "r"(TMEM_COLS)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    } else {
      // one warp of each CTA of the pair allocates collectively: the same columns in both
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                   "r"(TMEM_COLS)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
  }
  tc_fence_before();
  if constexpr (CG == 1) __syncthreads();
  else cluster_sync();  // the peer's copies and arrivals target barriers initialised above
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  const int total = s_total;

  if (warp == 0) {
    if (lane == 0 && leader) {
      int stage = 0;
      uint32_t phase = 0;
      long long issued = 0;  // stages this thread filled
      bool ok = !p.stall;
      for (int tile = cta0; tile < total && ok; tile += ncta) {
        int inst, mt, nt;
        Blk bk;
        locate<BK, CG>(p, s_prefix, tile, inst, bk, mt, nt);
        const int arow = bk.m0 + mt * TC_BM * CG + (int)rank * TC_BM;
        const int brow = bk.n0 + nt * TC_BN + (int)rank * B_ROWS;
        for (int kb = 0; kb < bk.num_kb; ++kb) {
          if (!mbar_wait(empty0 + 8 * stage, phase ^ 1, abort_flag, p.timeout_ns)) { ok = false; break; }
          const uint32_t fb = full0 + 8 * stage;
          const int kx = bk.k0 + kb * TC_BK;
          if constexpr (CG == 1) {
            mbar_expect_tx(fb, STAGE_BYTES);
#pragma unroll
            for (int pl = 0; pl < NPL; ++pl) {
              tma_load_3d(smem_u32(a_tile(stage, pl)), &maps.a[pl], fb, kx, arow, inst);
              tma_load_3d(smem_u32(b_tile(stage, pl)), &maps.b[pl], fb, kx, brow, inst);
            }
          } else {
            // this CTA fills the stage in both CTAs of the pair (the second CTA's copies land at the
            // same offsets of its shared memory); all bytes count on this CTA's barrier
            mbar_expect_tx(fb, 2 * STAGE_BYTES);
#pragma unroll
            for (int pl = 0; pl < NPL; ++pl) {
              const uint32_t sa = smem_u32(a_tile(stage, pl)), sb = smem_u32(b_tile(stage, pl));
              tma_load_3d_pair(sa, &maps.a[pl], fb, kx, arow, inst);
              tma_load_3d_pair(sb, &maps.b[pl], fb, kx, brow, inst);
              tma_load_3d_pair(mapa_rank(sa, 1), &maps.a[pl], fb, kx, arow + TC_BM, inst);
              tma_load_3d_pair(mapa_rank(sb, 1), &maps.b[pl], fb, kx, brow + B_ROWS, inst);
            }
          }
          ++issued;
          if (++stage == TC_STAGES) { stage = 0; phase ^= 1; }
        }
      }
      // Drain, on every exit path: the last min(STAGES, issued) loads must land before the CTA (or
      // either CTA of a pair: the second waits at the final cluster barrier) exits - a consumer that
      // gave up may never have waited for them. Each stage holds at most one load in flight, and
      // issued copies always complete, so these waits use a floor of one second whatever the
      // caller's limit (after a normal run they return at once).
      for (long long i = (issued > TC_STAGES ? issued - TC_STAGES : 0); i < issued; ++i)
        mbar_wait(full0 + 8 * (int)(i % TC_STAGES), (uint32_t)((i / TC_STAGES) & 1), abort_flag,
                  drain_ns(p.timeout_ns), false);
    }
  } else if (warp == 1) {
    if (lane == 0 && leader) {
      int stage = 0;
      uint32_t phase = 0;
      int buf = 0;
      uint32_t bphase = 0;
      bool ok = true;
      for (int tile = cta0; tile < total && ok; tile += ncta) {
        int inst_, mt_, nt_;
        Blk bk_;
        locate<BK, CG>(p, s_prefix, tile, inst_, bk_, mt_, nt_);
        const int num_kb = bk_.num_kb;
        // Descriptors differ only in their start-address field (bits 0-13, address >> 4), so each
        // one is a base descriptor plus the tile's byte offset >> 4 (all offsets are multiples of
        // 16 bytes and the shared window is < 256 KB, so the field never carries over). Passes,
        // planes and the fold group are compile-time: a group's MMAs unroll into straight-line
        // issue code with constant offsets. A pair's MMA reads the same offsets in both CTAs.
        const uint64_t desc_base = smem_desc<BK>(smem_u32(smem));
        const uint32_t idesc = p.idesc;
        constexpr uint32_t B_OFF = NPL * A_TILE;
        for (int kb0 = 0; kb0 < num_kb && ok; kb0 += FG) {
          const int g = min(FG, num_kb - kb0);  // k-blocks in this fold group
          if (!mbar_wait(tempty0 + 8 * buf, bphase ^ 1, abort_flag, p.timeout_ns)) { ok = false; break; }
          uint32_t so[FG];  // byte offsets of the group's stages
          {
            int st = stage;
            uint32_t ph = phase;
#pragma unroll
            for (int i = 0; i < FG; ++i) {
              so[i] = (uint32_t)st * STAGE_BYTES;
              if (i < g && ok && !mbar_wait(full0 + 8 * st, ph, abort_flag, p.timeout_ns)) ok = false;
              if (++st == TC_STAGES) { st = 0; ph ^= 1; }
            }
          }
          if (!ok) break;
          tc_fence_after();
          const uint32_t d_tmem = tmem_base + (uint32_t)(buf * TC_BN);
#pragma unroll
          for (int ps = 0; ps < NPASS; ++ps) {
#pragma unroll
            for (int i = 0; i < FG; ++i) {
              if (i < g) {
                const uint64_t da = desc_base + ((so[i] + (uint32_t)pass_plane_a(NPASS, ps) * A_TILE) >> 4);
                const uint64_t db = desc_base + ((so[i] + B_OFF + (uint32_t)pass_plane_b(NPASS, ps) * B_TILE) >> 4);
#pragma unroll
                for (int k = 0; k < TC_BK / 16; ++k)
                  mma_f16<CG>(d_tmem, da + (uint64_t)(k * 2), db + (uint64_t)(k * 2), idesc,
                              (ps == 0 && i == 0 && k == 0) ? 0u : 1u);
              }
            }
          }
          for (int i = 0; i < g; ++i) {
            mma_commit_local<CG>(empty0 + 8 * stage);  // frees the stage (its copies are issued here)
            if (++stage == TC_STAGES) { stage = 0; phase ^= 1; }
          }
          mma_commit<CG>(tfull0 + 8 * buf);
          if (++buf == 2) { buf = 0; bphase ^= 1; }
        }
      }
      // all MMAs issued by this thread complete before TMEM is released (issued MMAs always
      // complete: the wait has the drain's floor, not the caller's limit)
      mma_commit_local<CG>(final_bar);
      mbar_wait(final_bar, 0, abort_flag, drain_ns(p.timeout_ns), false);
    }
  } else {
    const int q = warp & 3;          // TMEM lane quadrant this warp may access
    const int half = (warp - 2) >> 2;  // which 128 of the 256 columns
    // where this warp reports a freed TMEM buffer: the MMA-issuing CTA's barriers (contiguous in
    // its shared memory, so buffer b's barrier is 8 b bytes further in either address window)
    const uint32_t tempty_dst = CG == 2 && !leader ? mapa_rank(tempty0, 0) : tempty0;
    int buf = 0;
    uint32_t bphase = 0;
    bool ok = true;
    for (int tile = cta0; tile < total && ok; tile += ncta) {
      int num_kb;
      {
        // only the k-block count stays live through the k loop (the accumulator holds 128
        // registers); the tile is located again for the store
        int inst, mt, nt;
        Blk bk;
        locate<BK, CG>(p, s_prefix, tile, inst, bk, mt, nt);
        num_kb = bk.num_kb;
      }
      float acc[128];
#pragma unroll
      for (int j = 0; j < 128; ++j) acc[j] = 0.f;
      for (int kb = 0; kb < num_kb; kb += FG) {
        // one lane waits for the fold group's MMAs, the warp follows it
        int w = 1;
        if (lane == 0) w = mbar_wait(tfull0 + 8 * buf, bphase, abort_flag, p.timeout_ns) ? 1 : 0;
        w = __shfl_sync(0xffffffffu, w, 0);
        if (!w) { ok = false; break; }
        tc_fence_after();
        const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * TC_BN + half * 128);
#pragma unroll
        for (int c = 0; c < 4; c += 2) {
          uint32_t r0[32], r1[32];
          tmem_ld32(taddr + c * 32, r0);
          tmem_ld32(taddr + (c + 1) * 32, r1);
          tmem_ld_wait();
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            acc[c * 32 + j] += __uint_as_float(r0[j]);
            acc[(c + 1) * 32 + j] += __uint_as_float(r1[j]);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {  // one arrive per warp
          const uint32_t bar = tempty_dst + 8 * buf;
          if constexpr (CG == 1) mbar_arrive(bar);
          else if (leader) mbar_arrive(bar);
          else mbar_arrive_remote(bar);
        }
        if (++buf == 2) { buf = 0; bphase ^= 1; }
      }
      if (!ok) break;
      int inst, mt, nt;
      Blk bk;
      locate<BK, CG>(p, s_prefix, tile, inst, bk, mt, nt);
      if (p.amaxA) {
        // undo the operands' power-of-two scales (exact): the exponents the operand builders used
        const float unscale =
            pow2f(-(f16_scale_exponent(plane_bound(p.amaxA + (long long)inst * p.amax_inst, p.multA)) +
                    f16_scale_exponent(plane_bound(p.amaxB + (long long)inst * p.amax_inst, p.multB))));
#pragma unroll
        for (int j = 0; j < 128; ++j) acc[j] *= unscale;
      }
      const long long row = (long long)bk.m0 + (long long)mt * TC_BM * CG + (long long)rank * TC_BM + q * 32 + lane;
      const long long col0 = (long long)bk.n0 + (long long)nt * TC_BN + half * 128;
      const long long row_end = (long long)bk.m0 + bk.mc, col_end = (long long)bk.n0 + bk.nc;
      if (row < row_end && col0 < col_end) {
        float* dst = p.C + (long long)inst * p.c_inst + row * p.ldc + col0;
        if (p.vec4 && (bk.n0 & 3) == 0 && col0 + 128 <= col_end) {
#pragma unroll
          for (int j = 0; j < 128; j += 4)
            *reinterpret_cast<float4*>(dst + j) = make_float4(acc[j], acc[j + 1], acc[j + 2], acc[j + 3]);
        } else {
#pragma unroll
          for (int j = 0; j < 128; ++j)
            if (col0 + j < col_end) dst[j] = acc[j];
        }
      }
    }
  }
  if constexpr (CG == 1) {
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag) atomic_status(p.status, ST_TIMEOUT);
    if (warp == 1) {
      tc_fence_after();
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                   : "memory");
    }
  } else {
    __syncwarp();
    // every role of both CTAs is done: the pair's copies have landed (the first CTA's drain) and its
    // MMAs have completed, so neither CTA's shared or tensor memory is still in use
    cluster_sync();
    if (threadIdx.x == 0 && *abort_flag) atomic_status(p.status, ST_TIMEOUT);
    if (warp == 1) {
      tc_fence_after();
      asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                   : "memory");
    }
  }
}

__global__ void k_split_rows(const float* __restrict__ X, long long ldx, long long rows, long long cols,
                             Planes<__nv_bfloat16> out, long long ld) {
  const long long total = rows * cols;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / cols, c = i % cols;
    store_planes(out, r * ld + c, X[r * ldx + c]);
  }
}

// ------------------------------------------------------------------ host: tensor maps
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(ptr);
  }
  return fn;
}

// 3D map of `batch` planes of rows x cols (row stride ld, instance stride inst elements), boxes of
// box_rows x bk x 1.
bool make_map(CUtensorMap* m, const __nv_bfloat16* ptr, long long rows, long long cols, long long ld, int batch,
              long long inst, int box_rows, int bk, bool f16) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)batch};
  cuuint64_t strides[2] = {(cuuint64_t)ld * 2, (cuuint64_t)inst * 2};
  cuuint32_t box[3] = {(cuuint32_t)bk, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  return enc(m, f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
             const_cast<__nv_bfloat16*>(ptr), dims, strides, box,
             estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             bk == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// SM count of the current device (cached per device)
int num_sms();

// Encodes the tensor maps and launches one kernel variant. The maps' box sizes, the stage slot
// sizes and the expected transaction bytes all derive from the same compile-time BK, NPL and CG,
// so a TMA copy can never be larger than the stage slot it lands in. Persistent launch: as many
// CTAs (CG = 2: clusters of two) as can be resident at once, one per SM, and no more than the
// tiles (tiles < 0: counted on the device).
template <int BK, int NPL, int NPASS, int FG, int CG>
int launch_variant(long long tiles, const Planes<__nv_bfloat16>& A, long long lda, const Planes<__nv_bfloat16>& B,
                   long long ldb, long long a_inst, long long b_inst, const TcParams& p, cudaStream_t s) {
  using Cf = Cfg<BK, NPL, CG>;
  static_assert(Cf::STAGE_BYTES == NPL * (TC_BM + TC_BN / CG) * BK * 2, "stage holds exactly the boxes");
  TmapSet maps;
  std::memset(&maps, 0, sizeof(maps));
  for (int i = 0; i < NPL; ++i)
    if (!make_map(&maps.a[i], A.p[i], p.M, p.K, lda, p.batch, a_inst, TC_BM, BK, A.fmt == 1) ||
        !make_map(&maps.b[i], B.p[i], p.N, p.K, ldb, p.batch, b_inst, TC_BN / CG, BK, B.fmt == 1))
      return HOTRG_EDEVICE;
  auto kern = k_gemm_split<BK, NPL, NPASS, FG, CG>;
  // the dynamic shared-memory limit is a per-device attribute of the kernel: set it once on each
  // device this variant launches on; so is the number of resident CTAs or clusters
  static std::atomic<int> resident[kMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HOTRG_EDEVICE;
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CG;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(TC_THREADS);
  cfg.dynamicSmemBytes = Cf::SMEM;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = CG > 1 ? 1 : 0;
  int n = resident[dev].load();
  if (n <= 0) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cf::SMEM) != cudaSuccess)
      return HOTRG_EDEVICE;
    if (CG == 1) {
      n = num_sms();
    } else {
      cfg.gridDim = dim3((unsigned)(CG * std::max(1, num_sms() / CG)));
      if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess || n <= 0) {
        cudaGetLastError();
        return HOTRG_EDEVICE;
      }
    }
    resident[dev].store(n);
  }
  const long long units = tiles >= 0 && tiles < n ? (tiles > 0 ? tiles : 1) : n;
  cfg.gridDim = dim3((unsigned)(units * CG));
  if (cudaLaunchKernelEx(&cfg, kern, maps, p) != cudaSuccess) {
    cudaGetLastError();
    return HOTRG_EDEVICE;
  }
  return HOTRG_OK;
}

// SM count of the current device (cached per device)
int num_sms() {
  static std::atomic<int> cache[kMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return 1;
  }
  int n = cache[dev].load();
  if (n <= 0) {
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
      cudaGetLastError();
      n = 1;
    }
    cache[dev].store(n);
  }
  return n;
}

}  // namespace

int launch_gemm_split(const Planes<__nv_bfloat16>& A, long long lda, const Planes<__nv_bfloat16>& B,
                      long long ldb, float* C, long long ldc, long long M, long long N, long long K,
                      int npass, int* status, double timeout_s, cudaStream_t s, int bk, int group_m,
                      int fold_group, const GemmBlocks* blk, const GemmBatch* bat, bool stall, int cta_group) {
  if (bk != 32 && bk != 64) return HOTRG_EINVAL;
  if (cta_group == 0) cta_group = kDefaultCtaGroup;
  if (cta_group != 1 && cta_group != 2) return HOTRG_EINVAL;
  if (group_m < 1 || group_m > 64 || fold_group < 1) return HOTRG_EINVAL;
  if (M < TC_BM || N < TC_BN || K < 64 || (npass != 1 && npass != 3 && npass != 4 && npass != 6))
    return HOTRG_EINVAL;
  const int nplanes = npass == 1 ? 1 : (npass == 6 ? 3 : 2);
  if (nplanes == 3) bk = 32;  // three 64-wide planes do not fit two ring stages: resolved first
  if (nplanes == 1) bk = 64;  // single-plane GEMMs use 64-wide stages
  if (A.nparts < nplanes || B.nparts < nplanes) return HOTRG_EINVAL;
  // fp16 planes: both operands (one MMA type), two planes at most, each with its scale bound
  if (A.fmt != B.fmt || A.fmt < 0 || A.fmt > 1) return HOTRG_EINVAL;
  if (A.fmt == 1 && (nplanes > 2 || !A.amax || !B.amax)) return HOTRG_EINVAL;
  if ((lda % 8) || (ldb % 8) || lda < K || ldb < K || ldc < N) return HOTRG_EINVAL;
  if (M > 0x7fffffffLL || N > 0x7fffffffLL || K > 0x7fffffffLL) return HOTRG_EINVAL;
  auto al16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
  for (int i = 0; i < nplanes; ++i)
    if (!al16(A.p[i]) || !al16(B.p[i])) return HOTRG_EINVAL;
  // batched launch: instances' planes apart by at least a whole plane, 16-byte aligned
  const int batch = bat ? bat->batch : 1;
  const long long a_inst = bat ? bat->a_inst : M * lda, b_inst = bat ? bat->b_inst : N * ldb;
  if (batch < 1 || batch > kMaxGemmBatch) return HOTRG_EINVAL;
  if (batch > 1 && (a_inst < M * lda || b_inst < N * ldb || (a_inst % 8) || (b_inst % 8) ||
                    bat->c_inst < M * ldc || bat->amax_inst < 0))
    return HOTRG_EINVAL;
  TcParams p;
  p.M = M;
  p.N = N;
  p.K = K;
  p.num_m = (int)((M + TC_BM - 1) / TC_BM);
  p.num_n = (int)((N + TC_BN - 1) / TC_BN);
  p.num_kb = (int)((K + bk - 1) / bk);
  p.npass = npass;
  p.group_m = group_m;
  p.C = C;
  p.ldc = ldc;
  p.status = status;
  p.timeout_ns = (unsigned long long)(timeout_s * 1e9);
  p.vec4 = ((ldc % 4) == 0) && ((reinterpret_cast<uintptr_t>(C) & 15) == 0);
  p.blk = blk;
  p.idesc = idesc_for(A.fmt == 1, cta_group);
  p.amaxA = A.fmt == 1 ? A.amax : nullptr;
  p.amaxB = A.fmt == 1 ? B.amax : nullptr;
  p.multA = A.amax_mult;
  p.multB = B.amax_mult;
  p.batch = batch;
  p.c_inst = bat ? bat->c_inst : 0;
  p.amax_inst = bat ? bat->amax_inst : 0;
  p.stall = stall ? 1 : 0;
  // output tiles: 128 x 256 per CTA, 256 x 256 per CTA pair
  const long long tiles = (long long)((M + (long long)TC_BM * cta_group - 1) / ((long long)TC_BM * cta_group)) *
                          p.num_n * batch;
  if (tiles > 0x7fffffffLL) return HOTRG_EINVAL;
  // supported variants (fold groups beyond a variant's maximum are clamped to it)
  const int fg = std::max(1, std::min(fold_group, max_fold_group(npass, bk)));
  // with device-side blocks the tile count is known only on the device
  const long long t = blk ? -1 : tiles;
  int rc = HOTRG_EINVAL;
#define HOTRG_GEMM_VARIANT(BK_, NPL_, NP_, FG_)                                                        \
  if (bk == BK_ && nplanes == NPL_ && npass == NP_ && fg == FG_)                                      \
    rc = cta_group == 2 ? launch_variant<BK_, NPL_, NP_, FG_, 2>(t, A, lda, B, ldb, a_inst, b_inst, p, s) \
                        : launch_variant<BK_, NPL_, NP_, FG_, 1>(t, A, lda, B, ldb, a_inst, b_inst, p, s);
  HOTRG_GEMM_VARIANT(64, 1, 1, 1)
  HOTRG_GEMM_VARIANT(64, 1, 1, 2)
  HOTRG_GEMM_VARIANT(64, 2, 3, 1)
  HOTRG_GEMM_VARIANT(64, 2, 4, 1)
  HOTRG_GEMM_VARIANT(32, 2, 3, 1)
  HOTRG_GEMM_VARIANT(32, 2, 3, 2)
  HOTRG_GEMM_VARIANT(32, 2, 4, 1)
  HOTRG_GEMM_VARIANT(32, 2, 4, 2)
  HOTRG_GEMM_VARIANT(32, 3, 6, 1)
  HOTRG_GEMM_VARIANT(32, 3, 6, 2)
#undef HOTRG_GEMM_VARIANT
  if (rc) return rc;
  count_launches(1);
  return HOTRG_OK;
}

int max_fold_group(int npass, int bk) {
  if (npass == 6) return 2;        // 32-wide stages, three planes, 3-stage ring
  if (npass == 1) return 2;        // 64-wide stages, one plane, 4-stage ring
  return bk == 64 ? 1 : 2;         // two planes: 2-stage ring at 64, 4-stage ring at 32
}

void launch_split_rows(const float* X, long long ldx, long long rows, long long cols,
                       const Planes<__nv_bfloat16>& out, long long ld, cudaStream_t s) {
  const long long total = rows * cols;
  long long g = (total + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  if (g < 1) g = 1;
  k_split_rows<<<(int)g, 256, 0, s>>>(X, ldx, rows, cols, out, ld);
  count_launches(1);
}

}  // namespace hotrg
