// lu_blocked.cu -- the Pade comparator's solve (v - u) R = u + v (eq. pade10 /
// eq. pade26) for N > 112: a blocked LU factorisation with partial pivoting of
// M = v - u, carried out on the augmented system [M | B] (B = u + v), followed by
// the blocked back substitution U R = Y. The paper counts the whole solve as 4/3
// of a product (Section 1): 2N^3/3 flops for the factorisation, N^3 for the
// forward substitution of the N right-hand sides and N^3 for the back
// substitution; here all of it but the panels runs as rank-NB FP64 updates.
//
// Per panel of NB = 32 columns starting at j0 (rows j0..N-1):
//  1. k_panel_lu: one thread-block cluster factors the panel with partial
//     pivoting, its rows spread over the cluster's shared memory. Per column: each
//     CTA's largest |entry| goes to CTA 0, a cluster barrier, every CTA picks the
//     same pivot (ties to the smaller row) and reads the pivot row from its owner,
//     a second barrier, the two rows are exchanged and every CTA eliminates below
//     the pivot in its own rows. No spin-wait: the cluster barriers are hardware.
//  2. k_row_swaps: the panel's row interchanges, in order, applied to the columns
//     right of the panel and to all of B (columns left of the panel hold L entries
//     that nothing reads again).
//  3. k_trsm_lower_unit: rows j0..j0+NB-1 of those columns become L11^-1 times
//     themselves (U12, and the forward-substituted rows of B).
//  4. k_update: the trailing rows of those columns lose L21 times those rows.
// Then, from the last block row up: k_trsm_upper turns block row i of Y into
// U_ii^-1 Y_i (= R_i), and k_update removes U[0:i0, block i] R_i from the rows above.
// Scratch: the N pivot indices only, in the caller's scratch buffer: nothing is
// allocated, so the solve can be captured in a CUDA graph.
#include <math.h>

#include <algorithm>
#include <mutex>

#include "internal.h"

namespace bbc {
namespace {

constexpr int NB = 32;              // panel width
constexpr int PANEL_THREADS = 256;  // 8 warps
constexpr int UPD_THREADS = 256;
constexpr int UPD_TILE = 64;        // 64 x 64 output tiles, K = NB

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint32_t cl_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cl_size() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t remote(const void* p, uint32_t rank) {
  uint32_t out;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"(smem_u32(p)), "r"(rank));
  return out;
}
__device__ __forceinline__ void st_remote_f64(uint32_t addr, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}
__device__ __forceinline__ void st_remote_s32(uint32_t addr, int v) {
  asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ double ld_remote_f64(uint32_t addr) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ int ld_remote_s32(uint32_t addr) {
  int v;
  asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// (value, row) of the larger |entry|; ties to the smaller row; NaN never wins.
__device__ __forceinline__ bool better(double v, int i, double bv, int bi) {
  return v > bv || (v == bv && i < bi);
}

// Panel factorisation. Panel rows are j0..N-1 (panel index i = row - j0), columns
// j0..j0+nb-1. CTA r of the cluster owns panel rows [r * per, min(R, (r + 1) * per))
// in shared memory, row-major with nb columns. piv[j0 + c] receives the pivot row.
__global__ void __launch_bounds__(PANEL_THREADS, 1)
k_panel_lu(double* __restrict__ M, int64_t N, int64_t j0, int nb, int per, int* __restrict__ piv,
           unsigned int* __restrict__ flag) {
  extern __shared__ double rows[];  // per x NB
  __shared__ double cand_v[16];
  __shared__ int cand_i[16];
  __shared__ double prow[NB], crow[NB];
  __shared__ double red_v[PANEL_THREADS / 32];
  __shared__ int red_i[PANEL_THREADS / 32];
  __shared__ int s_p;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t rank = cl_rank(), csize = cl_size();
  const int R = (int)(N - j0);
  const int r0 = (int)rank * per, r1 = min(R, r0 + per);
  const int nloc = max(0, r1 - r0);

  for (int e = tid; e < nloc * NB; e += PANEL_THREADS) {
    const int li = e / NB, c = e % NB;
    rows[li * NB + c] = (c < nb) ? M[(j0 + r0 + li) * N + j0 + c] : 0.0;
  }
  __syncthreads();
  cluster_barrier();

  bool singular = false;
  for (int c = 0; c < nb; ++c) {
    // 1. this CTA's candidate among its rows with panel index >= c
    double bv = -1.0;
    int bi = R;
    for (int li = tid; li < nloc; li += PANEL_THREADS) {
      const int i = r0 + li;
      if (i < c) continue;
      const double v = fabs(rows[li * NB + c]);
      if (better(v, i, bv, bi)) { bv = v; bi = i; }
    }
    for (int off = 16; off > 0; off >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, bv, off);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
      if (better(ov, oi, bv, bi)) { bv = ov; bi = oi; }
    }
    if (lane == 0) { red_v[warp] = bv; red_i[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      for (int w = 1; w < PANEL_THREADS / 32; ++w)
        if (better(red_v[w], red_i[w], red_v[0], red_i[0])) { red_v[0] = red_v[w]; red_i[0] = red_i[w]; }
      st_remote_f64(remote(&cand_v[rank], 0), red_v[0]);
      st_remote_s32(remote(&cand_i[rank], 0), red_i[0]);
    }
    cluster_barrier();
    // 2. the cluster's pivot, the same in every CTA (one lane per candidate reads it
    //    from CTA 0, all reads in flight together, then a shuffle reduction); the
    //    pivot row from its owner
    if (warp == 0) {
      double gv = -1.0;
      int gi = R;
      if ((uint32_t)lane < csize) {
        gv = ld_remote_f64(remote(&cand_v[lane], 0));
        gi = ld_remote_s32(remote(&cand_i[lane], 0));
      }
      for (int off = 16; off > 0; off >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, gv, off);
        const int oi = __shfl_xor_sync(0xffffffffu, gi, off);
        if (better(ov, oi, gv, gi)) { gv = ov; gi = oi; }
      }
      if (lane == 0) {
        if (!(gv > 0.0) || gi >= R) {  // no usable pivot: keep the row, report, carry on
          singular = true;
          gi = c;
        }
        s_p = gi;
        if (rank == 0) piv[j0 + c] = (int)(j0 + gi);
      }
    }
    __syncthreads();
    const int p = s_p;
    const uint32_t owner_p = (uint32_t)(p / per), owner_c = (uint32_t)(c / per);
    if (tid < NB) {
      prow[tid] = ld_remote_f64(remote(&rows[(p - (int)owner_p * per) * NB + tid], owner_p));
      if (rank == owner_p && p != c)
        crow[tid] = ld_remote_f64(remote(&rows[(c - (int)owner_c * per) * NB + tid], owner_c));
    }
    cluster_barrier();
    // 3. exchange rows c and p, then eliminate below the pivot in this CTA's rows
    if (tid < NB) {
      if (rank == owner_c) rows[(c - r0) * NB + tid] = prow[tid];
      if (rank == owner_p && p != c) rows[(p - r0) * NB + tid] = crow[tid];
    }
    __syncthreads();
    const double d = prow[c];
    for (int li = warp; li < nloc; li += PANEL_THREADS / 32) {
      const int i = r0 + li;
      if (i <= c) continue;
      // one lane divides (FP64 division is costly on this GPU), the warp shares the quotient
      double l = 0.0;
      if (lane == 0) l = rows[li * NB + c] / d;
      l = __shfl_sync(0xffffffffu, l, 0);
      if (lane > c && lane < nb) rows[li * NB + lane] = fma(-l, prow[lane], rows[li * NB + lane]);
      if (lane == c) rows[li * NB + c] = l;
    }
    __syncthreads();
  }
  for (int e = tid; e < nloc * NB; e += PANEL_THREADS) {
    const int li = e / NB, c = e % NB;
    if (c < nb) M[(j0 + r0 + li) * N + j0 + c] = rows[li * NB + c];
  }
  if (singular && tid == 0 && rank == 0 && flag) atomicOr(flag, 1u);
  cluster_barrier();  // no CTA leaves while another may still read its shared memory
}

// The panel's interchanges, in order, on the augmented columns right of the panel:
// column g < W of M (its column j0 + nb + g) or column g - W of B (W = N - j0 - nb).
__global__ void __launch_bounds__(256)
k_row_swaps(double* M, double* B, int64_t N, int64_t j0, int nb,
            const int* __restrict__ piv) {
  __shared__ int s_piv[NB];
  if (threadIdx.x < nb) s_piv[threadIdx.x] = piv[j0 + threadIdx.x];
  __syncthreads();
  const int64_t W = N - j0 - nb;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= W + N) return;
  double* base = (g < W) ? M + j0 + nb + g : B + (g - W);
  for (int c = 0; c < nb; ++c) {
    const int64_t r1 = j0 + c, r2 = s_piv[c];
    if (r2 != r1) {
      const double t = base[r1 * N];
      base[r1 * N] = base[r2 * N];
      base[r2 * N] = t;
    }
  }
}

// Rows j0..j0+nb-1 of the augmented columns right of the panel <- L11^-1 times
// themselves (L11: the panel's unit lower triangle). One column per thread.
__global__ void __launch_bounds__(256)
k_trsm_lower_unit(double* M, double* __restrict__ B, int64_t N, int64_t j0, int nb) {
  __shared__ double L[NB][NB + 1];
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, q = e % NB;
    L[r][q] = (r < nb && q < nb) ? M[(j0 + r) * N + j0 + q] : 0.0;
  }
  __syncthreads();
  const int64_t W = N - j0 - nb;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= W + N) return;
  double* base = (g < W) ? M + j0 + nb + g : B + (g - W);
  double x[NB];
#pragma unroll
  for (int r = 0; r < NB; ++r) x[r] = (r < nb) ? base[(j0 + r) * N] : 0.0;
#pragma unroll
  for (int r = 1; r < NB; ++r) {
    double acc = x[r];
#pragma unroll
    for (int q = 0; q < r; ++q) acc = fma(-L[r][q], x[q], acc);
    x[r] = acc;
  }
#pragma unroll
  for (int r = 0; r < NB; ++r)
    if (r < nb) base[(j0 + r) * N] = x[r];
}

// Block row i0..i0+nb-1 of B <- U_ii^-1 times itself (U_ii: the diagonal block's upper
// triangle, diagonal included). One column per thread; a non-finite result sets flag.
__global__ void __launch_bounds__(256)
k_trsm_upper(const double* M, double* B, int64_t N, int64_t i0, int nb,
             unsigned int* __restrict__ flag) {
  __shared__ double U[NB][NB + 1];
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, q = e % NB;
    U[r][q] = (r < nb && q < nb) ? M[(i0 + r) * N + i0 + q] : 0.0;
  }
  __syncthreads();
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  double x[NB];
#pragma unroll
  for (int r = 0; r < NB; ++r) x[r] = (r < nb) ? B[(i0 + r) * N + j] : 0.0;
  bool bad = false;
#pragma unroll
  for (int r = NB - 1; r >= 0; --r) {
    if (r >= nb) continue;
    double acc = x[r];
#pragma unroll
    for (int q = r + 1; q < NB; ++q)
      if (q < nb) acc = fma(-U[r][q], x[q], acc);
    x[r] = acc / U[r][r];
    bad |= !isfinite(x[r]);
  }
#pragma unroll
  for (int r = 0; r < NB; ++r)
    if (r < nb) B[(i0 + r) * N + j] = x[r];
  if (bad && flag) atomicOr(flag, 1u);
}

// C[rows x cols] -= L[rows x nb] U[nb x cols] on up to two column ranges at once:
// column tiles [0, tiles0) address (C0, U0) with cols0 columns, the rest (C1, U1)
// with cols1 columns. All matrices have leading dimension N. 64 x 64 tiles, the
// whole K = nb slab in shared memory, a 4 x 4 register block per thread with rows
// and columns strided by 16.
__global__ void __launch_bounds__(UPD_THREADS, 3)
k_update(const double* L, int64_t rows, int nb, const double* U0, double* C0, int64_t cols0, int tiles0,
         const double* U1, double* C1, int64_t cols1, int64_t N) {
  __shared__ double Ls[NB][UPD_TILE];
  __shared__ double Us[NB][UPD_TILE];
  const bool first = (int)blockIdx.x < tiles0;
  const double* Up = first ? U0 : U1;
  double* Cp = first ? C0 : C1;
  const int64_t cols = first ? cols0 : cols1;
  const int64_t n0 = (int64_t)(first ? blockIdx.x : blockIdx.x - tiles0) * UPD_TILE;
  const int64_t m0 = (int64_t)blockIdx.y * UPD_TILE;
  const int t = threadIdx.x, tx = t % 16, ty = t / 16;
  for (int e = t; e < NB * UPD_TILE; e += UPD_THREADS) {
    const int k = e % NB, r = e / NB;            // L: consecutive threads walk k (contiguous in a row)
    const int64_t gr = m0 + r;
    Ls[k][r] = (gr < rows && k < nb) ? L[gr * N + k] : 0.0;
    const int kc = e / UPD_TILE, c = e % UPD_TILE;  // U: consecutive threads walk columns
    const int64_t gc = n0 + c;
    Us[kc][c] = (gc < cols && kc < nb) ? Up[(int64_t)kc * N + gc] : 0.0;
  }
  __syncthreads();
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
#pragma unroll 8
  for (int k = 0; k < NB; ++k) {
    double a[4], b[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = Ls[k][ty + 16 * i];
#pragma unroll
    for (int j = 0; j < 4; ++j) b[j] = Us[k][tx + 16 * j];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t r = m0 + ty + 16 * i;
    if (r >= rows) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t c = n0 + tx + 16 * j;
      if (c < cols) Cp[r * N + c] -= acc[i][j];
    }
  }
}

// Cluster shape of the panel kernel on this device, set up once per device (the
// attributes and the occupancy query are host calls made outside any capture when
// the first solve of the device runs): the most CTAs (16, else 8) of which one fits
// an SM with the largest dynamic shared memory the device allows.
struct PanelShape { int csize = 0; size_t max_smem = 0; };
std::mutex g_panel_mu;
bool g_panel_done[64] = {};
PanelShape panel_shape() {
  static PanelShape cache[64];
  std::mutex& mu = g_panel_mu;
  bool* done = g_panel_done;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return PanelShape{};
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev]) return cache[dev];
  done[dev] = true;
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return cache[dev];
  const size_t static_bytes = 4096;  // the kernel's own arrays (candidates, two rows, reductions), rounded up
  const size_t smem = ((size_t)optin - static_bytes) / (NB * sizeof(double)) * (NB * sizeof(double));
  if (cudaFuncSetAttribute(k_panel_lu, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaFuncSetAttribute(k_panel_lu, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return cache[dev];
  }
  for (int cs : {16, 8}) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)cs, 1, 1);
    cfg.blockDim = dim3(PANEL_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_panel_lu, &cfg) != cudaSuccess || n < 1) {
      cudaGetLastError();
      continue;
    }
    cache[dev].csize = cs;
    cache[dev].max_smem = smem;
    break;
  }
  return cache[dev];
}

cudaError_t launch_update(const double* L, int64_t rows, int nb, const double* U0, double* C0, int64_t cols0,
                          const double* U1, double* C1, int64_t cols1, int64_t N, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  const int tiles0 = (int)((cols0 + UPD_TILE - 1) / UPD_TILE);
  const int tiles1 = (int)((cols1 + UPD_TILE - 1) / UPD_TILE);
  if (tiles0 + tiles1 == 0) return cudaSuccess;
  const dim3 grid((unsigned)(tiles0 + tiles1), (unsigned)((rows + UPD_TILE - 1) / UPD_TILE));
  k_update<<<grid, UPD_THREADS, 0, st>>>(L, rows, nb, U0, C0, cols0, tiles0, U1, C1, cols1, N);
  return cudaGetLastError();
}

}  // namespace

bool lu_blocked_ready() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
  std::lock_guard<std::mutex> lk(g_panel_mu);
  return g_panel_done[dev];
}

int64_t lu_blocked_max_n() {
  const PanelShape ps = panel_shape();
  return (int64_t)ps.csize * (int64_t)(ps.max_smem / (NB * sizeof(double)));
}

cudaError_t lu_blocked_solve(double* M, double* B, int64_t N, unsigned int* flag, cudaStream_t st, void* scratch) {
  const PanelShape ps = panel_shape();
  if (ps.csize == 0) return cudaErrorNotSupported;
  if (N < 1 || !scratch || (size_t)((N + ps.csize - 1) / ps.csize) * NB * sizeof(double) > ps.max_smem)
    return cudaErrorInvalidValue;
  int* piv = static_cast<int*>(scratch);
  cudaError_t err;
  // factorisation of [M | B]: M = P^T L U, B <- L^-1 P B
  for (int64_t j0 = 0; j0 < N; j0 += NB) {
    const int nb = (int)std::min<int64_t>(NB, N - j0);
    const int64_t R = N - j0;
    const int per = (int)((R + ps.csize - 1) / ps.csize);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)ps.csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)ps.csize, 1, 1);
    cfg.blockDim = dim3(PANEL_THREADS, 1, 1);
    cfg.dynamicSmemBytes = (size_t)per * NB * sizeof(double);
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if ((err = cudaLaunchKernelEx(&cfg, k_panel_lu, M, N, j0, nb, per, piv, flag)) != cudaSuccess) return err;
    const int64_t W = N - j0 - nb;
    const unsigned g = (unsigned)((W + N + 255) / 256);
    k_row_swaps<<<g, 256, 0, st>>>(M, B, N, j0, nb, piv);
    k_trsm_lower_unit<<<g, 256, 0, st>>>(M, B, N, j0, nb);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    // trailing rows: [M(j0+nb:, j0+nb:) | B(j0+nb:, :)] -= L21 [U12 | Y1]
    if ((err = launch_update(M + (j0 + nb) * N + j0, R - nb, nb, M + j0 * N + j0 + nb, M + (j0 + nb) * N + j0 + nb,
                             W, B + j0 * N, B + (j0 + nb) * N, N, N, st)) != cudaSuccess)
      return err;
  }
  // back substitution U R = Y, block rows from the bottom
  const int64_t nblk = (N + NB - 1) / NB;
  for (int64_t bi = nblk - 1; bi >= 0; --bi) {
    const int64_t i0 = bi * NB;
    const int nb = (int)std::min<int64_t>(NB, N - i0);
    k_trsm_upper<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(M, B, N, i0, nb, flag);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    // rows above: B(0:i0, :) -= U(0:i0, i0:i0+nb) R_i
    if ((err = launch_update(M + i0, i0, nb, B + i0 * N, B, N, nullptr, nullptr, 0, N, st)) != cudaSuccess)
      return err;
  }
  return cudaSuccess;
}

}  // namespace bbc
