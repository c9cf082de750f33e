// K4: S-CHOLESKY, type (i) of Sec. 3.1: dense Cholesky of the SCM B and the solve of the
// Schur complement equation B dz = g (eq. SCE).
//
// B (internal constraint order) is stored column-major with one extra row: row m holds g^T.
// A right-looking blocked factorisation of the leading m columns carries that row through the
// panel solves and trailing updates, so on exit row m holds (L^{-1} g)^T and only the backward
// substitution L^T dz = L^{-1} g remains.  FP64 throughout.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/mcsdp.h"
#include "internal.h"

namespace mcsdp {

constexpr int NB = 64;  // panel width

// Cholesky of the nb x nb diagonal block at (k0, k0), one CTA of 256 threads, and the inverse
// of the factor (stored in Linv, nb x nb column-major, ld NB).  Thread (r, q) = (tid / 4, tid % 4)
// owns row r of the block and every 4th column of the trailing update.
__global__ void k_potrf_diag(double *B, int64_t ldb, int k0, int nb, int *status, double *Linv) {
  extern __shared__ double smp[];
  double *A = smp;                  // row-major, padded: A[r * (NB+1) + c]
  double *T = smp + NB * (NB + 1);  // inverse, column-major
  __shared__ double rdg[NB];
  __shared__ double piv[2];
  const int tid = threadIdx.x;
  const int r = tid & 63, q = tid >> 6;
  constexpr int LD = NB + 1;
  for (int idx = tid; idx < nb * nb; idx += 256) {
    const int i = idx % nb, j = idx / nb;
    A[i * LD + j] = (i >= j) ? B[(k0 + i) + (int64_t)(k0 + j) * ldb] : 0.0;
  }
  __syncthreads();
  bool bad = false;
  for (int j = 0; j < nb; ++j) {
    if (tid == 0) {  // one thread: FP64 sqrt / division are long multi-instruction sequences
      double d = A[j * LD + j];
      if (!(d > 0.0)) {
        bad = true;
        d = 1.0;
      }
      const double sd = sqrt(d);
      piv[0] = sd;
      piv[1] = 1.0 / sd;
    }
    __syncthreads();
    if (q == 0 && r < nb) {
      if (r == j) A[j * LD + j] = piv[0];
      else if (r > j) A[r * LD + j] *= piv[1];
    }
    __syncthreads();
    if (r > j && r < nb) {
      const double arj = A[r * LD + j];
      for (int kk = j + 1 + q; kk <= r; kk += 4) A[r * LD + kk] -= arj * A[kk * LD + j];
    }
    __syncthreads();  // the next pivot is final
  }
  if (bad && tid == 0) atomicOr(status, ST_NOT_PD);
  __syncthreads();
  if (tid < nb) rdg[tid] = 1.0 / A[tid * LD + tid];
  __syncthreads();
  // inverse of the lower-triangular factor: column j of T by forward substitution
  if (tid < nb) {
    const int j = tid;
    T[j + j * NB] = rdg[j];
    for (int i = j + 1; i < nb; ++i) {
      double s0 = 0.0, s1 = 0.0;
      int l = j;
      for (; l + 1 < i; l += 2) {
        s0 = fma(A[i * LD + l], T[l + j * NB], s0);
        s1 = fma(A[i * LD + l + 1], T[l + 1 + j * NB], s1);
      }
      if (l < i) s0 = fma(A[i * LD + l], T[l + j * NB], s0);
      T[i + j * NB] = -(s0 + s1) * rdg[i];
    }
    for (int i = 0; i < j; ++i) T[i + j * NB] = 0.0;
  }
  __syncthreads();
  for (int idx = tid; idx < nb * nb; idx += 256) {
    const int i = idx % nb, j = idx / nb;
    if (i >= j) B[(k0 + i) + (int64_t)(k0 + j) * ldb] = A[i * LD + j];
    Linv[i + j * NB] = T[i + j * NB];
  }
}

// Rows [r0, rend) of the panel columns [k0, k0+nb): X <- X L_kk^{-T} = X Linv^T.  CTA = 16 rows
// x nb columns (256 threads, 4 outputs each), so the panel solve spreads over many SMs.
constexpr int TRSM_ROWS = 16;
__global__ void k_trsm_panel(double *B, int64_t ldb, int k0, int nb, int r0, int rend,
                             const double *__restrict__ Linv) {
  extern __shared__ double smt[];
  double *Xs = smt;                   // [l][row], TRSM_ROWS rows
  double *Ts = smt + NB * TRSM_ROWS;  // [l][col] = Linv[col][l]
  const int tid = threadIdx.x;
  const int rb = r0 + blockIdx.x * TRSM_ROWS;
  for (int idx = tid; idx < nb * TRSM_ROWS; idx += 256) {
    const int rr = idx % TRSM_ROWS, l = idx / TRSM_ROWS;
    const int gi = rb + rr;
    Xs[l * TRSM_ROWS + rr] = (gi < rend) ? B[gi + (int64_t)(k0 + l) * ldb] : 0.0;
  }
  for (int idx = tid; idx < nb * 64; idx += 256) {
    const int cc = idx % 64, l = idx / 64;
    Ts[l * 64 + cc] = (cc < nb) ? Linv[cc + l * NB] : 0.0;
  }
  __syncthreads();
  const int tx = tid & 15, ty = tid >> 4;  // row ty, columns tx*4 .. tx*4+3
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int l = 0; l < nb; ++l) {
    const double a = Xs[l * TRSM_ROWS + ty];
#pragma unroll
    for (int t = 0; t < 4; ++t) acc[t] = fma(a, Ts[l * 64 + tx * 4 + t], acc[t]);
  }
  const int gi = rb + ty;
  if (gi < rend) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int c = tx * 4 + t;
      if (c < nb) B[gi + (int64_t)(k0 + c) * ldb] = acc[t];
    }
  }
}

// Trailing update C -= P P^T on the lower TS x TS tiles of rows [r0, rend), columns [r0, cend).
// P = columns [k0, k0+nb) of the rows.  256 threads, 2 x 2 register blocking; small tiles keep
// all SMs busy on the later panels (one FP64 tile of 64 x 64 x 64 would take ~60 us on one SM).
constexpr int TS = 32;
__global__ void k_syrk_tiles(double *B, int64_t ldb, int k0, int nb, int r0, int rend, int cend) {
  extern __shared__ double smd[];
  double *Ai = smd;             // [nb][TS] (k-major)
  double *Aj = smd + NB * TS;   // [nb][TS]
  const int t = blockIdx.x;
  int ti = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
  while (ti * (ti + 1) / 2 > t) --ti;
  const int tj = t - ti * (ti + 1) / 2;
  const int rb = r0 + ti * TS, cb = r0 + tj * TS;
  if (cb >= cend) return;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < nb * TS; idx += 256) {
    const int rr = idx % TS, l = idx / TS;
    const int gi = rb + rr, gj = cb + rr;
    Ai[l * TS + rr] = (gi < rend) ? B[gi + (int64_t)(k0 + l) * ldb] : 0.0;
    Aj[l * TS + rr] = (gj < rend) ? B[gj + (int64_t)(k0 + l) * ldb] : 0.0;
  }
  __syncthreads();
  const int tx = tid & 15, ty = tid >> 4;
  double acc[2][2] = {};
  for (int l = 0; l < nb; ++l) {
    const double a0 = Ai[l * TS + ty * 2], a1 = Ai[l * TS + ty * 2 + 1];
    const double b0 = Aj[l * TS + tx * 2], b1 = Aj[l * TS + tx * 2 + 1];
    acc[0][0] = fma(a0, b0, acc[0][0]);
    acc[0][1] = fma(a0, b1, acc[0][1]);
    acc[1][0] = fma(a1, b0, acc[1][0]);
    acc[1][1] = fma(a1, b1, acc[1][1]);
  }
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const int gi = rb + ty * 2 + p;
    if (gi >= rend) continue;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int gj = cb + tx * 2 + q;
      if (gj < cend && gi >= gj) B[gi + (int64_t)gj * ldb] -= acc[p][q];
    }
  }
}

int dense_chol_bordered(double *B, int64_t ldb, int m, int *status, double *Linv_all,
                        cudaStream_t st) {
  const int smem_potrf = (NB * (NB + 1) + NB * NB) * (int)sizeof(double);
  const int smem_trsm = (NB * TRSM_ROWS + NB * 64) * (int)sizeof(double);
  const int smem_tile = 2 * NB * TS * (int)sizeof(double);
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(k_syrk_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_tile);
    cudaFuncSetAttribute(k_trsm_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_trsm);
    cudaFuncSetAttribute(k_potrf_diag, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_potrf);
    configured = true;
  }
  const int rows = m + 1;  // including the border row
  int launches = 0;
  for (int k0 = 0; k0 < m; k0 += NB) {
    const int nb = (m - k0) < NB ? (m - k0) : NB;
    double *Linv = Linv_all + (int64_t)(k0 / NB) * NB * NB;
    k_potrf_diag<<<1, 256, smem_potrf, st>>>(B, ldb, k0, nb, status, Linv);
    ++launches;
    const int r0 = k0 + nb;
    const int nr = rows - r0;
    if (nr > 0) {
      k_trsm_panel<<<(nr + TRSM_ROWS - 1) / TRSM_ROWS, 256, smem_trsm, st>>>(B, ldb, k0, nb, r0, rows, Linv);
      const int nt = (nr + TS - 1) / TS;
      const int ntiles = nt * (nt + 1) / 2;
      k_syrk_tiles<<<ntiles, 256, smem_tile, st>>>(B, ldb, k0, nb, r0, rows, m);
      launches += 2;
    }
  }
  return launches;
}

// Backward substitution L^T x = y, y = row m of B, blocks of 64 from the bottom; the diagonal
// block step is x_b <- Linv_b^T x_b with the inverses stored by the factorisation.
__global__ void k_bs_diag(const double *__restrict__ Linv, int b0, int nb, double *x) {
  __shared__ double xs[NB];
  const int t = threadIdx.x;
  if (t < nb) xs[t] = x[b0 + t];
  __syncthreads();
  if (t < nb) {
    double acc = 0.0;
    for (int i = t; i < nb; ++i) acc = fma(Linv[i + t * NB], xs[i], acc);  // Linv[i][t]
    x[b0 + t] = acc;
  }
}

// x[j] -= sum_{i in block} L[i][j] x[i] for j < b0
__global__ void k_bs_update(const double *B, int64_t ldb, int b0, int nb, double *x) {
  __shared__ double xb[NB];
  if (threadIdx.x < nb) xb[threadIdx.x] = x[b0 + threadIdx.x];
  __syncthreads();
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < b0; j += gridDim.x * blockDim.x) {
    const double *col = B + (int64_t)j * ldb + b0;
    double a0 = 0.0, a1 = 0.0;
    int i = 0;
    for (; i + 1 < nb; i += 2) {
      a0 = fma(col[i], xb[i], a0);
      a1 = fma(col[i + 1], xb[i + 1], a1);
    }
    if (i < nb) a0 = fma(col[i], xb[i], a0);
    x[j] -= a0 + a1;
  }
}

__global__ void k_copy_border(const double *B, int64_t ldb, int m, double *x) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x)
    x[j] = B[m + (int64_t)j * ldb];
}

int dense_backsolve(const double *B, int64_t ldb, int m, const double *Linv_all, double *x,
                    cudaStream_t st) {
  k_copy_border<<<(m + 255) / 256, 256, 0, st>>>(B, ldb, m, x);
  int launches = 1;
  const int nblk = (m + NB - 1) / NB;
  for (int bk = nblk - 1; bk >= 0; --bk) {
    const int b0 = bk * NB;
    const int nb = (m - b0) < NB ? (m - b0) : NB;
    k_bs_diag<<<1, NB, 0, st>>>(Linv_all + (int64_t)bk * NB * NB, b0, nb, x);
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


// ---------------------------------------------------------------------------------------------
// Allocation-free Schur complement solve.  Working storage: the bordered copy of B
// ((m+1) x m, leading dimension m+1), the inverses of the 64 x 64 diagonal blocks, and one
// status word, all in one file-scope device array.
constexpr int NA_MAX_M = MCSDP_SCE_NOALLOC_MAX_M;
constexpr size_t NA_B = (size_t)(NA_MAX_M + 1) * NA_MAX_M;
constexpr size_t NA_INV = (size_t)((NA_MAX_M + NB - 1) / NB) * NB * NB;
constexpr size_t NA_TOTAL = NA_B + NA_INV + 32;

static __device__ __align__(256) double g_sce_noalloc_scratch[NA_TOTAL];

// copy lower(B) and g into the bordered working matrix; clear the status word
__global__ void k_noalloc_setup(double *Bw, int64_t ldw, const double *__restrict__ B, int64_t ldb,
                                const double *__restrict__ g, int m, int *status) {
  const int64_t total = (int64_t)m * m;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % m), j = (int)(idx / m);
    if (i >= j) Bw[i + j * ldw] = B[i + j * ldb];
  }
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x)
    Bw[m + j * ldw] = g[j];
  if (blockIdx.x == 0 && threadIdx.x == 0) *status = 0;
}

}  // namespace mcsdp

namespace {
std::mutex g_na_mu;
double *g_na_ptr[64] = {};  // device address of the scratch array, per device ordinal
}  // namespace

extern "C" mcsdp_status mcsdp_sce_solve_noalloc(const double *B, int64_t ldb, const double *g,
                                                double *x, int32_t m, void *stream) {
  using namespace mcsdp;
  if (m <= 0 || m > NA_MAX_M || ldb < m || !B || !g || !x) return MCSDP_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return MCSDP_ERR_CUDA;
  double *base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_sce_noalloc_scratch) != cudaSuccess || !p) return MCSDP_ERR_CUDA;
      g_na_ptr[dev] = static_cast<double *>(p);
    }
    base = g_na_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t ldw = (int64_t)m + 1;
  double *Bw = base;
  double *Binv = base + NA_B;
  int *status = reinterpret_cast<int *>(base + NA_B + NA_INV);
  int blocks = (int)(((int64_t)m * m + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  k_noalloc_setup<<<blocks, 256, 0, st>>>(Bw, ldw, B, ldb, g, m, status);
  dense_chol_bordered(Bw, ldw, m, status, Binv, st);
  dense_backsolve(Bw, ldw, m, Binv, x, st);
  if (cudaGetLastError() != cudaSuccess) return MCSDP_ERR_CUDA;
  int hst = 0;
  if (cudaMemcpyAsync(&hst, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return MCSDP_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return MCSDP_ERR_CUDA;
  return (hst & ST_NOT_PD) ? MCSDP_ERR_NOT_PD : MCSDP_OK;
}
