// gemm_ozaki.cu -- FP64 products computed exactly from BF16 slices on the
// tcgen05 tensor cores (an error-free splitting in the manner of Ozaki et al.;
// the slices and their scales come from slices.cu).
//
// Why: the scaling-and-squaring cost is the number of dense products (Section 1,
// Section 4 of Bader-Blanes-Casas). GB300 runs FP64 at ~1.25 TFLOP/s but dense
// BF16 at ~2 PFLOP/s, so a product rebuilt from k^2/2 BF16 products is far
// faster than one FP64 product, and it is exact up to the slicing.
//
// Exact products. Pairs (p, q) with g = p + q <= k - 1 are kept (the triangle),
// C_ij = 2^(e_i + f_j - 16) sum_g 2^(-8g) S_g with S_g = sum_{p+q=g} sum_k d^P d^Q,
// an error of order 2^(-8k) relative to the row and column scales.
//  * High groups g <= 4 carry weights down to 2^-32 and are summed exactly.
//    A product of digits is at most 2^14, so a sum of up to 1024 of them is an
//    integer below 2^24 and FP32 holds it exactly: the K loop of these pairs is
//    cut into 1024-wide chunks, and after each chunk the FP32 tile is drained from
//    TMEM, converted to int32 and added, shifted by 2^(8(4-g)), into an integer
//    accumulator R (64 bits per element, held in registers; |R| < 2^61 for N <= 16384).
//  * Low groups g >= 5 weigh at most 2^-40. They accumulate in an FP32 TMEM
//    tile over the whole K, Horner-style from the smallest weight up, the MMA
//    scaling the running sum by 2^-8 (scale-input-d) at each change of group.
//    That FP32 sum of up to ~10^5 terms loses roughly 2^-16 of itself, i.e. about
//    2^-56 of the result. (With the exact/FP32 boundary one group lower, at g = 4,
//    the same loss showed up as ~1e-14 relative error per product at N = 4096.)
//  C_ij = 2^(e_i + f_j - 48) (R + 2^-8 LOW), to which the epilogue adds back the
//  diagonals the slices left out: + P_ii Q_ij + P_ij Q_jj - [i = j] P_ii Q_jj.
//
// The product kernel, k_ozaki_pair, is described at its definition: CTA pairs
// (tcgen05.mma.cta_group::2) on persistent 256 x 128 output tiles, TMA-fed.
// Every mbarrier wait is bounded in time; on expiry the kernel records a
// timeout in the status word, lets its copies and MMAs finish (bounded again),
// frees TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>
#include <map>
#include <tuple>
#include <vector>
#include <cstring>
#include <mutex>

#include "internal.h"
#include "slices.h"

namespace bbc {
namespace {

using slices::OzLayout;
using slices::layout;
constexpr int TILE = slices::PAD;  // rows per CTA and columns of an output tile
constexpr int ROW_BYTES = 128;     // bytes of one swizzle row of a K step, either element type
constexpr int CHUNK_STEPS = 16;    // 16 x 64 = 1024 K per exact FP32 chunk
constexpr int G_EXACT = 5;         // groups 0..4 are summed exactly
constexpr unsigned long long TIMEOUT_NS = 2000000000ull;  // 2 s per wait
constexpr unsigned int STATUS_TIMEOUT = 2u;    // bit of the handle's status word

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major tile, rows of 128 bytes, 128-byte
// swizzle, 8-row core groups 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);         // start address
  d |= (uint64_t)1 << 16;                          // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset
  d |= (uint64_t)1 << 46;                          // descriptor version
  d |= (uint64_t)2 << 61;                          // 128-byte swizzle
  return d;
}
// 32 lanes x 16 (8) consecutive 32-bit TMEM columns: thread t gets lane (base + t).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ------------------------------------------------------------ the product kernel
// k_ozaki_pair: a cluster of two CTAs computes 256 x 128 output tiles with
// tcgen05.mma.cta_group::2 (M = 256, N = 128, K = 16): CTA r of the pair stages rows
// [128 r, 128 r + 128) of the P slice tile and rows [64 r, 64 r + 64) of the Q^T slice
// tile, and its TMEM receives its 128 x 128 half of the output tile. Per SM that is
// 24 KB of operands per 64-wide K step (a lone 128 x 128 tile needs 32 KB), so nine
// steps fit in flight and the L2 serves a quarter fewer bytes per flop.
//
// The exact integer accumulator R of the high groups lives in the registers of eight
// drain warps (64 columns x 64 bits each), which leaves TMEM for two high-group FP32
// buffers (the MMAs never wait for a drain) and two low-group buffers. The kernel is
// persistent: every tile runs its low items first, so the MMAs of tile t + 1 proceed
// while the drain warps compute the epilogue of tile t from R and the other low buffer.
//
// Roles (320 threads per CTA): warp 0 TMA producer (both CTAs; their copies signal the
// even CTA's "full" barriers), warp 1 MMA issuer (even CTA only; commits are multicast
// to both CTAs), warps 2..9 drains and epilogue (both CTAs; they release buffers by
// arriving on the even CTA's barriers). 320 threads cap registers at 168 per thread
// (the register file is split over four sub-partitions and one of them holds three
// warps), which is why TMEM loads go 16 (drain) and 8 (epilogue) columns at a time.
// TMEM columns per CTA: [0,128) and [128,256) high buffers, [256,384) and [384,512)
// low buffers.
constexpr int P_STAGES = 8;
constexpr int P_A_BYTES = TILE * ROW_BYTES;          // 128 rows of a P slice plane
constexpr int P_B_BYTES = (TILE / 2) * ROW_BYTES;    // 64 rows of a Q^T slice plane
constexpr int P_STAGE_BYTES = P_A_BYTES + P_B_BYTES;
constexpr int P_THREADS = 320;
constexpr int P_DRAIN_WARPS = 8;
constexpr int P_GROUP_M = 8;                         // raster: 8 tile rows per column sweep
// Instruction descriptor, kind::f16: D = F32 (bit 4), A = B = BF16 (bits 7-9, 10-12 = 1), both
// K-major, N = 128 (bits 17-22: N / 8), M = 256 (bits 24-28: M / 16). kind::tf32 takes the same
// layout with A = B = TF32 (format 2); its MMA covers K = 8 (32 bytes), as K = 16 does in BF16.
constexpr uint32_t IDESC_PAIR = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TILE >> 3) << 17) |
                                ((uint32_t)(2 * TILE >> 4) << 24);
constexpr uint32_t IDESC_PAIR_TF32 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TILE >> 3) << 17) |
                                     ((uint32_t)(2 * TILE >> 4) << 24);
// Operand element type of a launch: BF16 slices (exact form and literal BF16 terms) or
// TF32 terms (literal TF32 split). KS = elements per K step (one 128-byte swizzle row).
template <bool TF32>
struct OperandKind {
  static constexpr int KS = TF32 ? 32 : 64;
  static constexpr uint32_t IDESC = TF32 ? IDESC_PAIR_TF32 : IDESC_PAIR;
};

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ int cluster_index() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return (int)r;
}
__device__ __forceinline__ int cluster_count() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
  return (int)r;
}
// Address of the same shared variable in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t peer_addr(const void* p, uint32_t rank) {
  uint32_t out;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"(smem_u32(p)), "r"(rank));
  return out;
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait_cl(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait by a whole warp: all 32 lanes call it together and get the same
// answer. The roles that issue TMA copies and MMAs run as whole warps with one
// elected lane issuing: measured on GB300, a loop run by a single lane (its 31
// siblings parked) pays ~250 cycles per mbarrier wait, enough to idle the tensor
// pipe between 4-MMA stages; the converged warp pays almost nothing.
__device__ __noinline__ bool mbar_wait_warp_slow(uint64_t* bar, uint32_t parity, volatile int* cta_err,
                                                 bool cluster_scope) {
  const unsigned long long t0 = globaltimer();
  for (uint32_t it = 1;; ++it) {
    const bool done = cluster_scope ? mbar_try_wait_cl(bar, parity) : mbar_try_wait(bar, parity);
    if (__any_sync(0xffffffffu, done)) return true;  // a completed phase stays completed
    if ((it & 63) == 0) {
      int stop = 0;
      if (*cta_err) stop = 1;
      else if (globaltimer() - t0 > TIMEOUT_NS) stop = 2;
      stop = __shfl_sync(0xffffffffu, stop, 0);
      if (stop) {
        if (stop == 2 && (threadIdx.x & 31) == 0) *cta_err = 1;
        return false;
      }
    }
  }
}
__device__ __forceinline__ bool mbar_wait_warp(uint64_t* bar, uint32_t parity, volatile int* cta_err) {
  if (__all_sync(0xffffffffu, mbar_try_wait(bar, parity))) return true;
  return mbar_wait_warp_slow(bar, parity, cta_err, false);
}
__device__ __forceinline__ bool mbar_wait_warp_cl(uint64_t* bar, uint32_t parity, volatile int* cta_err) {
  if (__all_sync(0xffffffffu, mbar_try_wait_cl(bar, parity))) return true;
  return mbar_wait_warp_slow(bar, parity, cta_err, true);
}
// Self-test of failure detection: one warp waits, through the same bounded
// wait as the product kernel, on an mbarrier that nothing ever arrives at. The
// wait gives up after TIMEOUT_NS and the kernel records STATUS_TIMEOUT in the
// status word and returns, as a product whose partner CTA never arrived would.
__global__ void k_wait_selftest(unsigned int* status) {
  __shared__ uint64_t bar;
  __shared__ int err;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const bool ok = mbar_wait_warp(&bar, 0u, &err);
  if (threadIdx.x == 0 && (!ok || err)) atomicOr(status, STATUS_TIMEOUT);
}
// One lane of the (converged) warp, chosen by the hardware.
__device__ __forceinline__ bool elect_one() {
  uint32_t pred;
  asm volatile("{\n .reg .pred P;\n .reg .b32 R;\n elect.sync R|P, 0xffffffff;\n selp.u32 %0, 1, 0, P;\n}\n"
               : "=r"(pred));
  return pred != 0;
}
// TMA tile load into this CTA's shared memory, completing bytes on a barrier that may
// belong to the peer CTA (cluster address).
__device__ __forceinline__ void tma_load_3d_pair(void* dst, const CUtensorMap* map, uint32_t bar_cluster, int x,
                                                 int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, "
      "%5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(bar_cluster), "r"(x), "r"(y), "r"(z)
      : "memory");
}
template <bool TF32>
__device__ __forceinline__ void mma_pair(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  if (TF32)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::
            "r"(d_tmem),
        "l"(a), "l"(b), "r"(IDESC_PAIR_TF32), "r"(accumulate)
        : "memory");
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::
            "r"(d_tmem),
        "l"(a), "l"(b), "r"(IDESC_PAIR), "r"(accumulate)
        : "memory");
}
// The exact form only (BF16): accumulate onto 2^-8 times the running sum.
__device__ __forceinline__ void mma_pair_scaled(uint32_t d_tmem, uint64_t a, uint64_t b) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, 1, 0;\n tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p, 8;\n}\n" ::"r"(
          d_tmem),
      "l"(a), "l"(b), "r"(IDESC_PAIR)
      : "memory");
}
// Arrive on the barrier at this offset in both CTAs once all prior MMAs completed.
__device__ __forceinline__ void commit_pair(uint64_t* bar) {
  const uint16_t both = 3;
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_u32(bar)),
      "h"(both)
      : "memory");
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

struct PairShared {
  uint64_t full[P_STAGES];   // even CTA: both CTAs' copies of a stage landed
  uint64_t empty[P_STAGES];  // each CTA: the MMAs reading its stage completed
  uint64_t acc_full[2];      // each CTA: a high buffer holds a finished chunk
  uint64_t acc_empty[2];     // even CTA: all 16 drain warps read that buffer
  uint64_t low_full[2];      // each CTA: a low buffer holds a tile's low groups
  uint64_t low_empty[2];     // even CTA: all 16 drain warps read that low buffer
  uint64_t mma_done;
  uint32_t tmem_base;
  int err;
  double epi[P_DRAIN_WARPS][32 * 9];  // per drain warp: 32 rows x 8 columns of results (rows padded to 9)
};
constexpr size_t PAIR_SMEM_BYTES = (size_t)P_STAGES * P_STAGE_BYTES + sizeof(PairShared) + 1024;

// Tile t -> (pair row block mp, column block nt); P_GROUP_M row blocks sweep the
// columns together so that concurrently running tiles share operand rows in L2.
__device__ __forceinline__ void pair_tile(int t, int tiles_m, int tiles_n, int* mp, int* nt) {
  const int per_group = P_GROUP_M * tiles_n;
  const int grp = t / per_group;
  const int first = grp * P_GROUP_M;
  const int rows = min(P_GROUP_M, tiles_m - first);
  const int w = t - grp * per_group;
  *mp = first + w % rows;
  *nt = w / rows;
}

// The K steps one output tile needs: all of them, or for upper triangular P and
// Q the steps meeting [first row, last column] (P_ik = 0 for k < i, Q_kj = 0 for
// k > j); tiles strictly below the diagonal need none (their epilogue writes the
// zeros). Chunks are consecutive blocks of at most 1024 K (CHUNK_STEPS steps),
// counted from the range's own first step, so a short range takes as few chunks
// (and drains) as its length allows.
struct TileWork {
  int mp, nt;          // pair row block, column block
  int ks_lo, ks_hi;    // K steps [ks_lo, ks_hi)
  int nch;             // number of chunks
};
__device__ __forceinline__ TileWork tile_work(int t, const uint32_t* __restrict__ list, int tiles_m, int tiles_n,
                                              int nksteps, int upper, int ks) {
  TileWork w;
  if (list) {
    const uint32_t code = __ldg(list + t);
    w.mp = (int)(code >> 16);
    w.nt = (int)(code & 0xFFFFu);
  } else {
    pair_tile(t, tiles_m, tiles_n, &w.mp, &w.nt);
  }
  w.ks_lo = upper ? min(nksteps, w.mp * (2 * TILE / ks)) : 0;
  w.ks_hi = upper ? min(nksteps, (w.nt + 1) * (TILE / ks)) : nksteps;
  w.nch = (w.ks_hi <= w.ks_lo) ? 0 : (w.ks_hi - w.ks_lo + CHUNK_STEPS - 1) / CHUNK_STEPS;
  return w;
}

// Work items of one output tile, in the order all three roles walk them: the low
// groups first (g = k-1 down to G_EXACT: the Horner order; inside a group the slice
// pairs p = 0..g (q = g - p), inside a pair the K chunks c), then the high groups
// chunk-major: for each K chunk c every group g = 0..gh-1 and its pairs p = 0..g,
// so that the slice tiles of a chunk, each used by several pairs, are read again
// soon after the first read (while L2 still holds them); every high item is drained
// on its own, so their order does not change any sum. Advancing needs no division
// (the MMA issuer's time per item matters: it must keep a new MMA ready every ~65
// cycles).
struct ItemCursor {
  int g, p, c;
  bool low;
  int nch, glo, gh;  // glo: lowest low group (G_EXACT; 0 for the literal split, which has no exact
                     // groups); gh: number of high groups
  __device__ ItemCursor(int k, int nch_, int glo_) : p(0), c(0), nch(nch_), glo(glo_) {
    gh = min(k, glo_);
    low = k > glo;
    g = low ? k - 1 : 0;
  }
  __device__ void advance() {
    if (low) {
      if (++c < nch) return;
      c = 0;
      if (++p <= g) return;
      p = 0;
      if (--g < glo) {
        low = false;
        g = 0;
      }
      return;
    }
    if (++p <= g) return;
    p = 0;
    if (++g < gh) return;
    g = 0;
    ++c;
  }
};

template <bool TF32, bool TERMS>
__global__ void __launch_bounds__(P_THREADS, 1)
k_ozaki_pair(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
             const int* __restrict__ erow, const int* __restrict__ fcol, const double* __restrict__ P,
             const double* __restrict__ Q, const double* __restrict__ pdiag, const double* __restrict__ qdiag,
             int64_t N, double alpha, int nslices, int nksteps, int tiles_m, int tiles_n, const Epilogue e,
             unsigned int* __restrict__ status, const uint32_t* __restrict__ tile_list, int upper, int literal) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
  uint8_t* smA = smem;
  uint8_t* smB = smem + P_STAGES * P_A_BYTES;
  PairShared* sh = reinterpret_cast<PairShared*>(smem + P_STAGES * P_STAGE_BYTES);
  volatile int* cta_err = &sh->err;

  constexpr int KS = OperandKind<TF32>::KS;  // elements per K step
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const int cid = cluster_index(), ncl = cluster_count();
  const int ntiles = tiles_m * tiles_n;
  // high groups 0..gh-1; the literal split has none: every pair accumulates in FP32
  const int glo = literal ? 0 : G_EXACT;
  const int gh = min(nslices, glo);
  const int pairs_h = gh * (gh + 1) / 2;                            // high slice pairs
  const int pairs_l = nslices * (nslices + 1) / 2 - pairs_h;        // low slice pairs

  if (threadIdx.x == 0) {
    for (int s = 0; s < P_STAGES; ++s) { mbar_init(&sh->full[s], 1); mbar_init(&sh->empty[s], 1); }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sh->acc_full[b], 1);
      mbar_init(&sh->acc_empty[b], 2 * P_DRAIN_WARPS);
      mbar_init(&sh->low_full[b], 1);
      mbar_init(&sh->low_empty[b], 2 * P_DRAIN_WARPS);
    }
    mbar_init(&sh->mma_done, 1);
    sh->err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {  // one warp of each CTA of the pair allocates, together
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&sh->tmem_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();  // the peer's barriers are initialised before any remote arrival
  tc_fence_after();
  const uint32_t tmem = sh->tmem_base;

  if (warp == 0) {
    // ---------------- TMA producer (both CTAs; the whole warp walks the schedule)
    const bool leader_lane = elect_one();
    if (leader_lane) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(&tmA) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(&tmB) : "memory");
    }
    int s = 0;
    uint32_t ph = 0;
    bool ok = true;
    for (int t = cid; t < ntiles && ok; t += ncl) {
      const TileWork w = tile_work(t, tile_list, tiles_m, tiles_n, nksteps, upper, KS);
      const int arow = w.mp * 2 * TILE + (int)rank * TILE;
      const int brow = w.nt * TILE + (int)rank * (TILE / 2);
      const int nunits = (pairs_h + pairs_l) * w.nch;
      ItemCursor cur(nslices, w.nch, glo);
      for (int idx = 0; idx < nunits && ok; ++idx, cur.advance()) {
        const int kc = w.ks_lo + cur.c * CHUNK_STEPS;
        const int ks1 = min(w.ks_hi, kc + CHUNK_STEPS);
        for (int ks = kc; ks < ks1; ++ks) {
          if (!mbar_wait_warp(&sh->empty[s], ph ^ 1u, cta_err)) { ok = false; break; }
          if (leader_lane) {
            if (rank == 0) mbar_arrive_expect_tx(&sh->full[s], 2 * P_STAGE_BYTES);
            const uint32_t fb = peer_addr(&sh->full[s], 0);
            tma_load_3d_pair(smA + s * P_A_BYTES, &tmA, fb, ks * KS, arow, cur.p);
            tma_load_3d_pair(smB + s * P_B_BYTES, &tmB, fb, ks * KS, brow, cur.g - cur.p);
          }
          __syncwarp();
          if (++s == P_STAGES) { s = 0; ph ^= 1u; }
        }
      }
    }
    if (!ok) {  // give copies already issued time to land (error path only)
      const unsigned long long t0 = globaltimer();
      while (globaltimer() - t0 < 1000000ull) {
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer (the whole warp of the even CTA walks the schedule,
    // one elected lane issues). The first K step of each item is peeled off: it
    // alone carries the accumulate / scale choice, so the steady loop is four
    // unconditional MMAs and a commit.
    if (rank == 0) {
      const bool issuer = elect_one();
      const uint64_t dA0 = smem_desc(smem_u32(smA)), dB0 = smem_desc(smem_u32(smB));
      int s = 0;
      uint32_t ph = 0;
      int hc = 0, ln = 0;  // high items and low-buffer uses so far (the drains count alike)
      bool ok = true;
      for (int t = cid; t < ntiles && ok; t += ncl) {
        const TileWork w = tile_work(t, tile_list, tiles_m, tiles_n, nksteps, upper, KS);
        const int nL = pairs_l * w.nch, nunits = (pairs_h + pairs_l) * w.nch;
        const int lb = ln & 1;
        if (nL > 0) {
          if (!mbar_wait_warp_cl(&sh->low_empty[lb], ((uint32_t)(ln >> 1) & 1u) ^ 1u, cta_err)) { ok = false; break; }
          tc_fence_after();
        }
        ItemCursor cur(nslices, w.nch, glo);
        for (int idx = 0; idx < nunits && ok; ++idx, cur.advance()) {
          uint32_t d_tmem;
          int b = 0, kind0;  // first MMA: 0 fresh, 1 accumulate, 2 accumulate onto 2^-8 x the sum so far
          if (cur.low) {
            d_tmem = tmem + 256u + (uint32_t)(lb * TILE);
            kind0 = (idx == 0) ? 0 : ((!literal && cur.p == 0 && cur.c == 0) ? 2 : 1);
          } else {
            b = hc & 1;
            if (!mbar_wait_warp_cl(&sh->acc_empty[b], ((uint32_t)(hc >> 1) & 1u) ^ 1u, cta_err)) { ok = false; break; }
            tc_fence_after();  // the drains' TMEM reads of this buffer come before these MMAs
            d_tmem = tmem + (uint32_t)(b * TILE);
            kind0 = 0;
          }
          const int ks0 = w.ks_lo + cur.c * CHUNK_STEPS, ks1 = min(w.ks_hi, ks0 + CHUNK_STEPS);
          if (!mbar_wait_warp_cl(&sh->full[s], ph, cta_err)) { ok = false; break; }
          if (issuer) {
            const uint64_t da = dA0 + (uint64_t)(s * (P_A_BYTES >> 4)), db = dB0 + (uint64_t)(s * (P_B_BYTES >> 4));
            if (!TF32 && kind0 == 2) mma_pair_scaled(d_tmem, da, db);
            else mma_pair<TF32>(d_tmem, da, db, (uint32_t)(kind0 != 0));
            mma_pair<TF32>(d_tmem, da + 2, db + 2, 1u);  // +32 bytes per MMA (K = 16 BF16, 8 TF32)
            mma_pair<TF32>(d_tmem, da + 4, db + 4, 1u);
            mma_pair<TF32>(d_tmem, da + 6, db + 6, 1u);
            commit_pair(&sh->empty[s]);
          }
          __syncwarp();
          if (++s == P_STAGES) { s = 0; ph ^= 1u; }
          for (int ks = ks0 + 1; ks < ks1; ++ks) {
            if (!mbar_wait_warp_cl(&sh->full[s], ph, cta_err)) { ok = false; break; }
            if (issuer) {
              const uint64_t da = dA0 + (uint64_t)(s * (P_A_BYTES >> 4)), db = dB0 + (uint64_t)(s * (P_B_BYTES >> 4));
              mma_pair<TF32>(d_tmem, da, db, 1u);
              mma_pair<TF32>(d_tmem, da + 2, db + 2, 1u);
              mma_pair<TF32>(d_tmem, da + 4, db + 4, 1u);
              mma_pair<TF32>(d_tmem, da + 6, db + 6, 1u);
              commit_pair(&sh->empty[s]);
            }
            __syncwarp();
            if (++s == P_STAGES) { s = 0; ph ^= 1u; }
          }
          if (!ok) break;
          if (!cur.low) {
            if (issuer) commit_pair(&sh->acc_full[b]);
            ++hc;
          } else if (idx == nL - 1) {
            if (issuer) commit_pair(&sh->low_full[lb]);
          }
          __syncwarp();
        }
        if (nL > 0) ++ln;
      }
      if (issuer) commit_pair(&sh->mma_done);
      __syncwarp();
    }
    if (lane == 0) {  // no MMA may still write either CTA's TMEM when it is freed
      const unsigned long long t0 = globaltimer();
      while (!mbar_try_wait(&sh->mma_done, 0u) && globaltimer() - t0 < TIMEOUT_NS) {
      }
    }
  } else {
    // ---------------- drains + epilogue (warps 2..9 of both CTAs)
    const int q = warp & 3;                // TMEM lane quarter this warp may access
    const int half = (warp - 2) >> 2;      // which 64 of the tile's 128 columns
    const int row_in_tile = q * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(half * 64);
    int hc = 0, ln = 0;
    bool ok = true;
    for (int t = cid; t < ntiles && ok; t += ncl) {
      const TileWork w = tile_work(t, tile_list, tiles_m, tiles_n, nksteps, upper, KS);
      const int nL = pairs_l * w.nch;
      long long R[64];
#pragma unroll
      for (int i = 0; i < 64; ++i) R[i] = 0;
      // the high items chunk-major, as ItemCursor walks them: per chunk, group g = 0..gh-1
      // and its (g + 1) pairs; dg / dn track the group and the pair within it
      int dg = 0, dn = 0;
      for (int it = pairs_h * w.nch; it > 0 && ok; --it) {
        {
          const int shift = 8 * (G_EXACT - 1 - dg);
          const int b = hc & 1;
          ok = mbar_wait_warp(&sh->acc_full[b], (uint32_t)(hc >> 1) & 1u, cta_err);
          if (!ok) break;
          tc_fence_after();
#pragma unroll
          for (int pc = 0; pc < 4; ++pc) {
            uint32_t a[16];
            tmem_ld16(lane_base + (uint32_t)(b * TILE + 16 * pc), a);
            tmem_wait_ld();
            if (pc == 3) {  // the whole buffer is in registers: hand it back to the MMAs
              tc_fence_before();
              __syncwarp();
              if (lane == 0) mbar_arrive_cluster(peer_addr(&sh->acc_empty[b], 0));
            }
#pragma unroll
            for (int i = 0; i < 16; ++i)
              R[16 * pc + i] += (long long)__float2int_rn(__uint_as_float(a[i])) << shift;
          }
          ++hc;
        }
        if (++dn > dg) {
          dn = 0;
          if (++dg == gh) dg = 0;
        }
      }
      if (!ok) break;
      const int lb = ln & 1;
      if (nL > 0) {
        ok = mbar_wait_warp(&sh->low_full[lb], (uint32_t)(ln >> 1) & 1u, cta_err);
        if (!ok) break;
        tc_fence_after();
      }
      const int64_t row = (int64_t)w.mp * 2 * TILE + (int64_t)rank * TILE + row_in_tile;
      const int64_t col0 = (int64_t)w.nt * TILE + half * 64;
      if (upper && w.nt * TILE + TILE <= w.mp * 2 * TILE) {  // strictly below the diagonal: zeros
        // the warp's 32 rows one after another, its lanes across the 64 columns: each
        // store instruction writes whole row segments
        for (int rl = 0; rl < 32; ++rl) {
          const int64_t r = row - lane + rl;
          if (r >= N) break;
          for (int cc = lane; cc < 64; cc += 32)
            if (col0 + cc < N) zero_epilogue(e, N, r, col0 + cc);
        }
        continue;
      }
      // Each pass takes 8 columns: the warp's 32 threads (one row each) rebuild the
      // scaled slice sums and stage them in shared memory; then 8 threads per row
      // (4 rows per access, 64 contiguous bytes each) add the deflation terms and
      // run the fused epilogue, so its FP64 loads and stores move whole sectors.
      const int er = (row < N) ? erow[row] : 0;
      double* stage = sh->epi[warp - 2];
      const int tr = lane >> 3, tc = lane & 7;
      const int64_t rbase = row - lane;
#pragma unroll
      for (int pc = 0; pc < 8; ++pc) {
        uint32_t lw[8];
        if (nL > 0) {
          tmem_ld8(lane_base + 256u + (uint32_t)(lb * TILE + 8 * pc), lw);
          tmem_wait_ld();
          if (pc == 7) {
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive_cluster(peer_addr(&sh->low_empty[lb], 0));
          }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int64_t col = col0 + 8 * pc + i;
          const int fc = (col < N) ? fcol[col] : 0;
          double v;
          int ex;
          if (literal) {  // the FP32 sum of all term products, scaled back
            v = (nL > 0) ? (double)__uint_as_float(lw[i]) : 0.0;
            ex = er + fc;
          } else {
            v = (double)R[8 * pc + i];  // rounds to 53 bits when |R| >= 2^53
            if (nL > 0) v = fma((double)__uint_as_float(lw[i]), 0.00390625, v);
            ex = er + fc - 16 - 8 * (G_EXACT - 1);
          }
          const double scl = (ex >= -1022 && ex <= 1023) ? __longlong_as_double((long long)(ex + 1023) << 52)
                                                        : ldexp(1.0, ex);
          stage[lane * 9 + i] = v * scl;
        }
        __syncwarp();
        const int64_t col = col0 + 8 * pc + tc;
        const double qjj = (col < N) ? qdiag[col] : 0.0;
#pragma unroll 2
        for (int j = 0; j < 8; ++j) {
          const int rl = tr + 4 * j;
          const int64_t r = rbase + rl;
          if (r < N && col < N) {
            // the deflated diagonals: + P_ii Q_ij + P_ij Q_jj - [i = j] P_ii Q_jj
            const double pii = pdiag[r];
            double d = fma(pii, __ldg(Q + r * N + col), stage[rl * 9 + tc]);
            d = fma(__ldg(P + r * N + col), qjj, d);
            if (r == col) d = fma(-pii, qjj, d);
            apply_epilogue_t<TERMS>(e, N, r, col, alpha * d);
          }
        }
        __syncwarp();
      }
      if (nL > 0) ++ln;
    }
  }

  tc_fence_before();
  __syncthreads();
  cluster_sync_all();  // neither CTA leaves while the other may still reach its memory
  if (threadIdx.x == 0 && sh->err) atomicOr(status, STATUS_TIMEOUT);
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

// ------------------------------------------------------------ host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// k planes [k][Rp][Kp] of BF16 (or, tf32, of 32-bit TF32 words); boxes of one
// 128-byte swizzle row (64 or 32 elements) by box_rows rows.
bool make_map(CUtensorMap* m, void* base, int64_t Rp, int64_t Kp, int k, int box_rows, bool tf32) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t esz = tf32 ? 4 : 2;
  const cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)Rp, (cuuint64_t)k};
  const cuuint64_t strides[2] = {(cuuint64_t)Kp * esz, (cuuint64_t)(Rp * Kp * esz)};
  const cuuint32_t box[3] = {(cuuint32_t)(ROW_BYTES / esz), (cuuint32_t)box_rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(m, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

namespace {
// Clusters of two k_ozaki_pair CTAs that fit on the device at once (cached per device;
// every operand kind and epilogue form uses the same resources).
int pair_clusters() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  if (cached[dev] > 0) return cached[dev];
  if (cudaFuncSetAttribute(k_ozaki_pair<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)PAIR_SMEM_BYTES) != cudaSuccess ||
      cudaFuncSetAttribute(k_ozaki_pair<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)PAIR_SMEM_BYTES) != cudaSuccess ||
      cudaFuncSetAttribute(k_ozaki_pair<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)PAIR_SMEM_BYTES) != cudaSuccess ||
      cudaFuncSetAttribute(k_ozaki_pair<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)PAIR_SMEM_BYTES) != cudaSuccess)
    return 0;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(2 * 1024, 1, 1);
  cfg.blockDim = dim3(P_THREADS, 1, 1);
  cfg.dynamicSmemBytes = PAIR_SMEM_BYTES;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_ozaki_pair<false, false>, &cfg) != cudaSuccess || n <= 0) {
    // clusters are independent: any count is correct, the SM count / 2 is the natural one
    cudaGetLastError();
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess) n = sms / 2;
  }
  cached[dev] = n;
  return n;
}

// Tile order for triangular products, where tiles cost from nothing (below the
// diagonal) to a full K sweep (top right): sorted by cost and dealt to the
// clusters in a snake (cluster c takes list entries c, c + ncl, ...), so every
// cluster gets about the same number of K steps. Kept per (tiles, clusters) in
// mapped pinned host memory that the kernel reads directly (each CTA reads a few
// entries), so no copy is queued before a launch. Null when that memory is
// unavailable.
const uint32_t* upper_tile_order(int tiles_m, int tiles_n, int nksteps, int ncl, int ks) {
  static std::mutex mu;
  static std::map<std::tuple<int, int, int, int>, const uint32_t*> cache;
  std::lock_guard<std::mutex> lk(mu);
  auto key = std::make_tuple(tiles_m, tiles_n, nksteps, ncl);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  struct T { int cost; uint32_t code; };
  std::vector<T> v;
  for (int mp = 0; mp < tiles_m; ++mp)
    for (int nt = 0; nt < tiles_n; ++nt) {
      const int lo = std::min(nksteps, mp * (2 * TILE / ks)), hi = std::min(nksteps, (nt + 1) * (TILE / ks));
      v.push_back({std::max(0, hi - lo), ((uint32_t)mp << 16) | (uint32_t)nt});
    }
  std::stable_sort(v.begin(), v.end(), [](const T& a, const T& b) { return a.cost > b.cost; });
  uint32_t* host = nullptr;
  if (cudaHostAlloc((void**)&host, v.size() * sizeof(uint32_t), cudaHostAllocMapped | cudaHostAllocPortable) !=
      cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  const size_t n = v.size();
  for (size_t r0 = 0, round = 0; r0 < n; r0 += (size_t)ncl, ++round) {
    const size_t m = std::min((size_t)ncl, n - r0);
    for (size_t c = 0; c < m; ++c) host[r0 + c] = v[r0 + ((round & 1) ? m - 1 - c : c)].code;
  }
  uint32_t* dev = nullptr;
  if (cudaHostGetDevicePointer((void**)&dev, host, 0) != cudaSuccess) {
    cudaGetLastError();
    cudaFreeHost(host);
    return nullptr;
  }
  cache.emplace(key, dev);
  return dev;
}

template <bool TF32>
cudaError_t launch_pair(const OzLayout& L, const double* P, const double* Q, int64_t N, double alpha,
                        const Epilogue& e, int slices, unsigned int* flag, cudaStream_t st, bool upper,
                        bool literal) {
  constexpr int KS = OperandKind<TF32>::KS;
  CUtensorMap ta, tb;
  if (!make_map(&ta, L.Ps, L.Rp, L.Rp, slices, TILE, TF32) || !make_map(&tb, L.Qs, L.Rp, L.Rp, slices, TILE / 2, TF32))
    return cudaErrorNotSupported;
  const int ncl_max = pair_clusters();
  if (ncl_max <= 0) return cudaErrorNotSupported;
  const int tiles_m = (int)((L.Rp + 2 * TILE - 1) / (2 * TILE));
  const int tiles_n = (int)(L.Rp / TILE);
  const int ncl = std::min(ncl_max, tiles_m * tiles_n);
  // triangular products: the balanced tile order (without it, the plain raster order, equally correct)
  const uint32_t* list = upper ? upper_tile_order(tiles_m, tiles_n, (int)(L.Rp / KS), ncl, KS) : nullptr;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)(2 * ncl), 1, 1);
  cfg.blockDim = dim3(P_THREADS, 1, 1);
  cfg.dynamicSmemBytes = PAIR_SMEM_BYTES;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  auto kern = (e.ny > 0) ? k_ozaki_pair<TF32, true> : k_ozaki_pair<TF32, false>;
  return cudaLaunchKernelEx(&cfg, kern, ta, tb, (const int*)L.erow, (const int*)L.fcol, P, Q,
                            (const double*)L.pdiag, (const double*)L.qdiag, N, alpha, slices, (int)(L.Rp / KS),
                            tiles_m, tiles_n, e, flag, list, upper ? 1 : 0, literal ? 1 : 0);
}
}  // namespace

cudaError_t ozaki_product(const double* P, const double* Q, int64_t N, double alpha, const Epilogue& e, int slices,
                          void* work, unsigned int* flag, cudaStream_t st, bool upper, int mode) {
  const int kmax = (mode == SPLIT_LITERAL_TF32) ? 4 : 8;
  if (!ozaki_supported(N) || slices < 2 || slices > kmax || !work || !flag || mode < 0 || mode > 2)
    return cudaErrorInvalidValue;
  if (mode == SPLIT_LITERAL_TF32)  // TF32 planes take the room of two BF16 planes each
    return launch_pair<true>(layout(work, N, 2 * slices), P, Q, N, alpha, e, slices, flag, st, upper, true);
  return launch_pair<false>(layout(work, N, slices), P, Q, N, alpha, e, slices, flag, st, upper,
                            mode == SPLIT_LITERAL_BF16);
}

cudaError_t wait_selftest(unsigned int* status, cudaStream_t st) {
  if (!status) return cudaErrorInvalidValue;
  k_wait_selftest<<<1, 32, 0, st>>>(status);
  return cudaGetLastError();
}

}  // namespace bbc
