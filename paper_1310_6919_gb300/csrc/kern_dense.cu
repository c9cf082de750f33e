// K4: S-CHOLESKY, type (i) of Sec. 3.1: dense Cholesky of the SCM B and the solve of the
// Schur complement equation B dz = g (eq. SCE).
//
// B (internal constraint order) is stored column-major with one extra row: row m holds g^T.
// A right-looking blocked factorisation of the leading m columns carries that row through the
// panel solves and trailing updates, so on exit row m holds (L^{-1} g)^T and only the backward
// substitution L^T dz = L^{-1} g remains.  FP64 throughout.
#include <cuda_runtime.h>

#include <cmath>

#include "internal.h"

namespace mcsdp {

constexpr int NB = 64;  // panel width

// Cholesky of the nb x nb diagonal block at (k0, k0), one CTA.
__global__ void k_potrf_diag(double *B, int64_t ldb, int k0, int nb, int *status) {
  __shared__ double A[NB * NB];
  __shared__ double s_inv;
  const int tid = threadIdx.x, bd = blockDim.x;
  for (int idx = tid; idx < nb * nb; idx += bd) {
    int i = idx % nb, j = idx / nb;
    A[idx] = (i >= j) ? B[(k0 + i) + (int64_t)(k0 + j) * ldb] : 0.0;
  }
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (tid == 0) {
      double d = A[j + j * nb];
      if (!(d > 0.0)) {
        atomicOr(status, ST_NOT_PD);
        d = 1.0;
      }
      d = sqrt(d);
      A[j + j * nb] = d;
      s_inv = 1.0 / d;
    }
    __syncthreads();
    for (int i = j + 1 + tid; i < nb; i += bd) A[i + j * nb] *= s_inv;
    __syncthreads();
    const int w = nb - j - 1;
    for (int idx = tid; idx < w * w; idx += bd) {
      int kk = j + 1 + idx / w, ii = j + 1 + idx % w;
      if (ii >= kk) A[ii + kk * nb] -= A[ii + j * nb] * A[kk + j * nb];
    }
    __syncthreads();
  }
  for (int idx = tid; idx < nb * nb; idx += bd) {
    int i = idx % nb, j = idx / nb;
    if (i >= j) B[(k0 + i) + (int64_t)(k0 + j) * ldb] = A[idx];
  }
}

// Rows [r0, rend) of the panel columns [k0, k0+nb): X <- X L_kk^{-T}.  One warp per 8 rows,
// lanes over columns; the dependency along the columns is resolved by shuffles.
constexpr int TRSM_ROWS_PER_WARP = 8;
constexpr int TRSM_WARPS = 4;

__global__ void k_trsm_panel(double *B, int64_t ldb, int k0, int nb, int r0, int rend) {
  __shared__ double L[NB * NB];
  __shared__ double rdiag[NB];
  const int tid = threadIdx.x, bd = blockDim.x;
  for (int idx = tid; idx < nb * nb; idx += bd) {
    int i = idx % nb, j = idx / nb;
    L[idx] = (i >= j) ? B[(k0 + i) + (int64_t)(k0 + j) * ldb] : 0.0;
  }
  __syncthreads();
  for (int j = tid; j < nb; j += bd) rdiag[j] = 1.0 / L[j + j * nb];
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31;
  const int rbase = r0 + (blockIdx.x * TRSM_WARPS + warp) * TRSM_ROWS_PER_WARP;
  double acc0[TRSM_ROWS_PER_WARP], acc1[TRSM_ROWS_PER_WARP];
#pragma unroll
  for (int q = 0; q < TRSM_ROWS_PER_WARP; ++q) {
    const int row = rbase + q;
    acc0[q] = (row < rend && lane < nb) ? B[row + (int64_t)(k0 + lane) * ldb] : 0.0;
    acc1[q] = (row < rend && lane + 32 < nb) ? B[row + (int64_t)(k0 + lane + 32) * ldb] : 0.0;
  }
  for (int c = 0; c < nb; ++c) {
    const int owner = c & 31;
    const bool hi = c >= 32;
#pragma unroll
    for (int q = 0; q < TRSM_ROWS_PER_WARP; ++q) {
      double mine = hi ? acc1[q] : acc0[q];
      double xc = __shfl_sync(0xffffffffu, mine, owner) * rdiag[c];
      if (lane == owner) {
        if (hi) acc1[q] = xc;
        else acc0[q] = xc;
      }
      // columns c' > c owned by this lane
      if (lane > c && lane < nb) acc0[q] = fma(-xc, L[lane + c * nb], acc0[q]);
      if (lane + 32 > c && lane + 32 < nb) acc1[q] = fma(-xc, L[(lane + 32) + c * nb], acc1[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < TRSM_ROWS_PER_WARP; ++q) {
    const int row = rbase + q;
    if (row < rend) {
      if (lane < nb) B[row + (int64_t)(k0 + lane) * ldb] = acc0[q];
      if (lane + 32 < nb) B[row + (int64_t)(k0 + lane + 32) * ldb] = acc1[q];
    }
  }
}

// Trailing update C -= P P^T on the lower 64 x 64 tiles of rows [r0, rend), columns [r0, cend).
// P = columns [k0, k0+nb) of the rows.  256 threads, 4 x 4 register blocking.
__global__ void k_syrk_tiles(double *B, int64_t ldb, int k0, int nb, int r0, int rend, int cend) {
  extern __shared__ double smd[];
  double *Ai = smd;              // [nb][64] (k-major)
  double *Aj = smd + NB * 64;    // [nb][64]
  // tile index -> (ti, tj), ti >= tj
  const int t = blockIdx.x;
  int ti = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
  while (ti * (ti + 1) / 2 > t) --ti;
  const int tj = t - ti * (ti + 1) / 2;
  const int rb = r0 + ti * 64, cb = r0 + tj * 64;
  if (cb >= cend) return;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < nb * 64; idx += 256) {
    const int r = idx % 64, l = idx / 64;
    const int gi = rb + r, gj = cb + r;
    Ai[l * 64 + r] = (gi < rend) ? B[gi + (int64_t)(k0 + l) * ldb] : 0.0;
    Aj[l * 64 + r] = (gj < rend) ? B[gj + (int64_t)(k0 + l) * ldb] : 0.0;
  }
  __syncthreads();
  const int tx = tid & 15, ty = tid >> 4;
  double acc[4][4] = {};
  for (int l = 0; l < nb; ++l) {
    double a[4], b[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      a[q] = Ai[l * 64 + ty * 4 + q];
      b[q] = Aj[l * 64 + tx * 4 + q];
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], b[q], acc[p][q]);
  }
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int gi = rb + ty * 4 + p;
    if (gi >= rend) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int gj = cb + tx * 4 + q;
      if (gj < cend && gi >= gj) B[gi + (int64_t)gj * ldb] -= acc[p][q];
    }
  }
}

int dense_chol_bordered(double *B, int64_t ldb, int m, int *status, cudaStream_t st) {
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(k_syrk_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(2 * NB * 64 * sizeof(double)));
    configured = true;
  }
  const int rows = m + 1;  // including the border row
  int launches = 0;
  for (int k0 = 0; k0 < m; k0 += NB) {
    const int nb = (m - k0) < NB ? (m - k0) : NB;
    k_potrf_diag<<<1, 256, 0, st>>>(B, ldb, k0, nb, status);
    ++launches;
    const int r0 = k0 + nb;
    const int nr = rows - r0;
    if (nr > 0) {
      const int per_cta = TRSM_WARPS * TRSM_ROWS_PER_WARP;
      k_trsm_panel<<<(nr + per_cta - 1) / per_cta, 32 * TRSM_WARPS, 0, st>>>(B, ldb, k0, nb, r0, rows);
      const int nt = (nr + 63) / 64;
      const int ntiles = nt * (nt + 1) / 2;
      k_syrk_tiles<<<ntiles, 256, 2 * NB * 64 * sizeof(double), st>>>(B, ldb, k0, nb, r0, rows, m);
      launches += 2;
    }
  }
  return launches;
}

// Backward substitution L^T x = y, y = row m of B, blocks of 64 from the bottom.
__global__ void k_bs_diag(const double *B, int64_t ldb, int b0, int nb, double *x) {
  // one warp: x[b0..b0+nb) <- L_bb^{-T} x[b0..b0+nb)
  const int lane = threadIdx.x;
  double x0 = (lane < nb) ? x[b0 + lane] : 0.0;
  double x1 = (lane + 32 < nb) ? x[b0 + lane + 32] : 0.0;
  for (int c = nb - 1; c >= 0; --c) {
    const int owner = c & 31;
    const bool hi = c >= 32;
    double mine = hi ? x1 : x0;
    double xc = __shfl_sync(0xffffffffu, mine, owner) / B[(b0 + c) + (int64_t)(b0 + c) * ldb];
    if (lane == owner) {
      if (hi) x1 = xc;
      else x0 = xc;
    }
    if (lane < c) x0 = fma(-xc, B[(b0 + c) + (int64_t)(b0 + lane) * ldb], x0);
    if (lane + 32 < c) x1 = fma(-xc, B[(b0 + c) + (int64_t)(b0 + lane + 32) * ldb], x1);
  }
  if (lane < nb) x[b0 + lane] = x0;
  if (lane + 32 < nb) x[b0 + lane + 32] = x1;
}

// x[j] -= sum_{i in block} L[i][j] x[i] for j < b0
__global__ void k_bs_update(const double *B, int64_t ldb, int b0, int nb, double *x) {
  __shared__ double xb[NB];
  if (threadIdx.x < nb) xb[threadIdx.x] = x[b0 + threadIdx.x];
  __syncthreads();
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < b0; j += gridDim.x * blockDim.x) {
    const double *col = B + (int64_t)j * ldb + b0;
    double acc = 0.0;
    for (int i = 0; i < nb; ++i) acc = fma(col[i], xb[i], acc);
    x[j] -= acc;
  }
}

__global__ void k_copy_border(const double *B, int64_t ldb, int m, double *x) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x)
    x[j] = B[m + (int64_t)j * ldb];
}

int dense_backsolve(const double *B, int64_t ldb, int m, double *x, cudaStream_t st) {
  k_copy_border<<<(m + 255) / 256, 256, 0, st>>>(B, ldb, m, x);
  int launches = 1;
  const int nblk = (m + NB - 1) / NB;
  for (int bk = nblk - 1; bk >= 0; --bk) {
    const int b0 = bk * NB;
    const int nb = (m - b0) < NB ? (m - b0) : NB;
    k_bs_diag<<<1, 32, 0, st>>>(B, ldb, b0, nb, x);
    ++launches;
    if (b0 > 0) {
      k_bs_update<<<(b0 + 127) / 128, 128, 0, st>>>(B, ldb, b0, nb, x);
      ++launches;
    }
  }
  return launches;
}

// row m of B <- g_i = b_{user(i)} - beta mu h_i   (internal order)
__global__ void k_rhs_border(DevSym S, double *B, int64_t ldb, const double *hvec, double betamu) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S.m; i += gridDim.x * blockDim.x)
    B[S.m + (int64_t)i * ldb] = S.b[S.con_order[i]] - betamu * hvec[i];
}

void launch_rhs_border(const DevSym &S, double *B, int64_t ldb, const double *hvec, double betamu,
                       cudaStream_t st) {
  k_rhs_border<<<(S.m + 255) / 256, 256, 0, st>>>(S, B, ldb, hvec, betamu);
}

__global__ void k_dz_to_user(DevSym S, const double *x, double *dz) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S.m; i += gridDim.x * blockDim.x)
    dz[S.con_order[i]] = x[i];
}

void launch_dz_to_user(const DevSym &S, const double *x, double *dz, cudaStream_t st) {
  k_dz_to_user<<<(S.m + 255) / 256, 256, 0, st>>>(S, x, dz);
}

__global__ void k_B_to_user(DevSym S, const double *Bi, int64_t ldi, double *Bo, int64_t ldo,
                            const double *hi, double *ho) {
  const int64_t m = S.m;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < m * m;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % m), j = (int)(idx / m);
    if (i < j) continue;
    const int ui = S.con_order[i], uj = S.con_order[j];
    const int r = ui > uj ? ui : uj, c = ui > uj ? uj : ui;
    Bo[r + (int64_t)c * ldo] = Bi[i + (int64_t)j * ldi];
  }
  if (ho)
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
      ho[S.con_order[i]] = hi[i];
}

void launch_B_to_user(const DevSym &S, const double *Bi, int64_t ldi, double *Bo, int64_t ldo,
                      const double *hi, double *ho, cudaStream_t st) {
  int64_t tot = (int64_t)S.m * S.m;
  int blocks = (int)((tot + 255) / 256);
  if (blocks > 8192) blocks = 8192;
  k_B_to_user<<<blocks, 256, 0, st>>>(S, Bi, ldi, Bo, ldo, hi, ho);
}

}  // namespace mcsdp
