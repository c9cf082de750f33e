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

constexpr int NB = 32;  // panel width (FP64 on one SM is slow: a narrow panel keeps the
                        // serial factor-and-invert step short)

// Cholesky of the nb x nb diagonal block at (k0, k0), one CTA of 256 threads, and the inverse
// of the factor (stored in Linv, nb x nb column-major, ld NB).  Thread (r, q) = (tid % NB,
// tid / NB) owns row r and every 8th column of the trailing update; the inverse is formed
// row-step by row-step with all threads (T <- rows of L^{-1}), not one column per thread.
template <class T>
__global__ void k_potrf_diag(T *B, int64_t ldb, int k0, int nb, int *status, T *Linv) {
  constexpr int LD = NB + 1;
  constexpr int NQ = 256 / NB;
  __shared__ T A[NB * LD];  // row-major, padded
  __shared__ T Ti[NB * LD];  // inverse, row-major
  __shared__ T piv[2];
  const int tid = threadIdx.x;
  const int r = tid % NB, q = tid / NB;
  for (int idx = tid; idx < NB * NB; idx += 256) {
    const int i = idx % NB, j = idx / NB;
    A[i * LD + j] = (i >= j && i < nb && j < nb) ? B[(k0 + i) + (int64_t)(k0 + j) * ldb] : T(0);
    Ti[i * LD + j] = (i == j) ? T(1) : T(0);
  }
  __syncthreads();
  bool bad = false;
  for (int j = 0; j < nb; ++j) {
    if (tid == 0) {
      T d = A[j * LD + j];
      if (!(d > T(0))) {
        bad = true;
        d = T(1);
      }
      const T sd = sqrt(d);
      piv[0] = sd;
      piv[1] = T(1) / sd;
    }
    __syncthreads();
    if (q == 0 && r < nb) {
      if (r == j) A[j * LD + j] = piv[0];
      else if (r > j) A[r * LD + j] *= piv[1];
    }
    __syncthreads();
    if (r > j && r < nb) {
      const T arj = A[r * LD + j];
      for (int kk = j + 1 + q; kk <= r; kk += NQ) A[r * LD + kk] -= arj * A[kk * LD + j];
    }
    __syncthreads();
  }
  if (bad && tid == 0) atomicOr(status, ST_NOT_PD);
  // T = L^{-1}: forward elimination on the identity, one pivot row at a time; step k scales row
  // k of T by 1/L[k][k] and removes L[i][k] times it from the rows i > k (all threads)
  for (int k = 0; k < nb; ++k) {
    const T rk = T(1) / A[k * LD + k];
    __syncthreads();
    if (q == 0 && r <= k) Ti[k * LD + r] *= rk;
    __syncthreads();
    // rows i > k, columns c <= k
    for (int e = tid; e < (nb - k - 1) * (k + 1); e += 256) {
      const int i = k + 1 + e / (k + 1), c = e % (k + 1);
      Ti[i * LD + c] -= A[i * LD + k] * Ti[k * LD + c];
    }
  }
  __syncthreads();
  for (int idx = tid; idx < NB * NB; idx += 256) {
    const int i = idx % NB, j = idx / NB;
    if (i < nb && j < nb && i >= j) B[(k0 + i) + (int64_t)(k0 + j) * ldb] = A[i * LD + j];
    Linv[i + j * NB] = (i < nb && j < nb && i >= j) ? Ti[i * LD + j] : T(0);
  }
}

// Rows [r0, rend) of the panel columns [k0, k0+nb): X <- X L_kk^{-T} = X Linv^T.  CTA = 16 rows
// x nb columns (256 threads, 4 outputs each), so the panel solve spreads over many SMs.
constexpr int TRSM_ROWS = 16;
template <class T>
__global__ void k_trsm_panel(T *B, int64_t ldb, int k0, int nb, int r0, int rend,
                             const T *__restrict__ Linv) {
  extern __shared__ __align__(16) unsigned char smt_raw[];
  T *smt = reinterpret_cast<T *>(smt_raw);
  T *Xs = smt;                   // [l][row], TRSM_ROWS rows
  T *Ts = smt + NB * TRSM_ROWS;  // [l][col] = Linv[col][l], NB columns
  const int tid = threadIdx.x;
  const int rb = r0 + blockIdx.x * TRSM_ROWS;
  for (int idx = tid; idx < nb * TRSM_ROWS; idx += 256) {
    const int rr = idx % TRSM_ROWS, l = idx / TRSM_ROWS;
    const int gi = rb + rr;
    Xs[l * TRSM_ROWS + rr] = (gi < rend) ? B[gi + (int64_t)(k0 + l) * ldb] : T(0);
  }
  for (int idx = tid; idx < nb * NB; idx += 256) {
    const int cc = idx % NB, l = idx / NB;
    Ts[l * NB + cc] = Linv[cc + l * NB];
  }
  __syncthreads();
  constexpr int CPT = NB * TRSM_ROWS / 256;  // columns per thread
  const int tx = tid % (NB / CPT), ty = tid / (NB / CPT);
  T acc[CPT];
#pragma unroll
  for (int t = 0; t < CPT; ++t) acc[t] = T(0);
  for (int l = 0; l < nb; ++l) {
    const T a = Xs[l * TRSM_ROWS + ty];
#pragma unroll
    for (int t = 0; t < CPT; ++t) acc[t] = fma(a, Ts[l * NB + tx * CPT + t], acc[t]);
  }
  const int gi = rb + ty;
  if (gi < rend) {
#pragma unroll
    for (int t = 0; t < CPT; ++t) {
      const int c = tx * CPT + t;
      if (c < nb) B[gi + (int64_t)(k0 + c) * ldb] = acc[t];
    }
  }
}

// Trailing update C -= P P^T for the columns [c_lo, c_hi) of the rows [c_lo, rend), lower part
// (gi >= gj), with P = columns [k0, k0+nb) of the same rows; CTA = one TS x TS tile
// (blockIdx.x: row tile from c_lo, blockIdx.y: column tile from c_lo).  256 threads, 2 x 2
// register blocking; small tiles keep all SMs busy (a 64 x 64 x 64 FP64 tile takes ~60 us on
// one SM of this part).
constexpr int TS = 32;
template <class T>
__global__ void k_syrk_tiles(T *B, int64_t ldb, int k0, int nb, int c_lo, int c_hi,
                             int rend) {
  extern __shared__ __align__(16) unsigned char smd_raw[];
  T *smd = reinterpret_cast<T *>(smd_raw);
  T *Ai = smd;             // [nb][TS] (k-major)
  T *Aj = smd + NB * TS;   // [nb][TS]
  const int ti = blockIdx.x, tj = blockIdx.y;
  if (ti < tj) return;
  const int rb = c_lo + ti * TS, cb = c_lo + tj * TS;
  if (cb >= c_hi || rb >= rend) return;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < nb * TS; idx += 256) {
    const int rr = idx % TS, l = idx / TS;
    const int gi = rb + rr, gj = cb + rr;
    Ai[l * TS + rr] = (gi < rend) ? B[gi + (int64_t)(k0 + l) * ldb] : T(0);
    Aj[l * TS + rr] = (gj < c_hi) ? B[gj + (int64_t)(k0 + l) * ldb] : T(0);
  }
  __syncthreads();
  const int tx = tid & 15, ty = tid >> 4;
  T acc[2][2] = {};
  for (int l = 0; l < nb; ++l) {
    const T a0 = Ai[l * TS + ty * 2], a1 = Ai[l * TS + ty * 2 + 1];
    const T b0 = Aj[l * TS + tx * 2], b1 = Aj[l * TS + tx * 2 + 1];
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
      if (gj < c_hi && gi >= gj) B[gi + (int64_t)gj * ldb] -= acc[p][q];
    }
  }
}

template <class T>
static void launch_syrk(T *B, int64_t ldb, int k0, int nb, int c_lo, int c_hi, int rend,
                        int smem, cudaStream_t st) {
  if (c_lo >= c_hi) return;
  const int nti = (rend - c_lo + TS - 1) / TS, ntj = (c_hi - c_lo + TS - 1) / TS;
  k_syrk_tiles<T><<<dim3(nti, ntj), 256, smem, st>>>(B, ldb, k0, nb, c_lo, c_hi, rend);
}

// Right-looking blocked Cholesky of the leading m columns of a rows x m matrix (rows = m + 1 for
// the bordered right-hand side, m otherwise) with lookahead: on st (the critical path) panel k is factored (potrf), its rows below are solved
// (trsm) and its update is applied to block column k+1; the rest of its update (block columns
// >= k+2) runs on st2, overlapping the next panel's factor-and-solve.  ev_next[k%2] /
// ev_rest[k%2] order the two streams so no block is updated by both at once; st waits for st2
// at the end.  With st2 == nullptr everything runs on st.
template <class T>
static int dense_chol(T *B, int64_t ldb, int m, int rows, int *status, T *Linv_all, cudaStream_t st,
                      cudaStream_t st2, cudaEvent_t *ev_next, cudaEvent_t *ev_rest) {
  const int smem_trsm = (NB * TRSM_ROWS + NB * NB) * (int)sizeof(T);
  const int smem_tile = 2 * NB * TS * (int)sizeof(T);
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(k_syrk_tiles<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_tile);
    cudaFuncSetAttribute(k_trsm_panel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_trsm);
    configured = true;
  }
  int launches = 0;
  const bool la = st2 != nullptr;
  for (int k0 = 0, k = 0; k0 < m; k0 += NB, ++k) {
    const int nb = (m - k0) < NB ? (m - k0) : NB;
    T *Linv = Linv_all + (int64_t)k * NB * NB;
    k_potrf_diag<T><<<1, 256, 0, st>>>(B, ldb, k0, nb, status, Linv);
    ++launches;
    const int r0 = k0 + nb;
    const int nr = rows - r0;
    if (nr <= 0) continue;
    k_trsm_panel<T><<<(nr + TRSM_ROWS - 1) / TRSM_ROWS, 256, smem_trsm, st>>>(B, ldb, k0, nb, r0, rows, Linv);
    ++launches;
    const int c_next = r0 + NB < m ? r0 + NB : m;  // block column k+1 = [r0, c_next)
    if (!la) {
      launch_syrk<T>(B, ldb, k0, nb, r0, m, rows, smem_tile, st);
      ++launches;
      continue;
    }
    if (k >= 1) cudaStreamWaitEvent(st, ev_rest[(k - 1) & 1], 0);  // st2 finished panel k-1
    launch_syrk<T>(B, ldb, k0, nb, r0, c_next, rows, smem_tile, st);
    cudaEventRecord(ev_next[k & 1], st);
    ++launches;
    if (c_next < m) {
      cudaStreamWaitEvent(st2, ev_next[k & 1], 0);
      launch_syrk<T>(B, ldb, k0, nb, c_next, m, rows, smem_tile, st2);
      ++launches;
    }
    cudaEventRecord(ev_rest[k & 1], st2);
  }
  if (la) {
    cudaEventRecord(ev_rest[0], st2);
    cudaStreamWaitEvent(st, ev_rest[0], 0);
  }
  return launches;
}

int dense_chol_bordered(double *B, int64_t ldb, int m, int *status, double *Linv_all,
                        cudaStream_t st, cudaStream_t st2, cudaEvent_t *ev_next,
                        cudaEvent_t *ev_rest) {
  return dense_chol<double>(B, ldb, m, m + 1, status, Linv_all, st, st2, ev_next, ev_rest);
}

int dense_chol_f32(float *B, int64_t ldb, int m, int *status, float *Linv_all, cudaStream_t st,
                   cudaStream_t st2, cudaEvent_t *ev_next, cudaEvent_t *ev_rest) {
  return dense_chol<float>(B, ldb, m, m, status, Linv_all, st, st2, ev_next, ev_rest);
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
// Mixed precision: FP32 factor of B, FP64 iterative refinement against the FP64 B.
//
// B32 <- lower(B) in FP32 (ld m)
__global__ void k_lower_to_f32(const double *__restrict__ B, int64_t ldb, float *B32, int m) {
  const int64_t tot = (int64_t)m * m;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % m), j = (int)(idx / m);
    if (i >= j) B32[idx] = (float)B[i + (int64_t)j * ldb];
  }
}

// after the FP32 factorisation: copy L into the unused upper triangle as L^T (coalesced backward
// substitution)
__global__ void k_lower_to_upper_f32(float *L, int m) {
  const int64_t tot = (int64_t)m * m;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % m), j = (int)(idx / m);
    if (i > j) L[j + (int64_t)i * m] = L[idx];
  }
}

// x += L^{-T} L^{-1} r with the FP32 factor (ld m; L^T in the upper triangle) and the inverses of
// its NB x NB diagonal blocks; one CTA of 1024 threads, the vector in shared memory (m floats).
__global__ void k_refine_solve_f32(const float *__restrict__ L, int m, const float *__restrict__ Linv,
                                   const double *__restrict__ r, double *x) {
  extern __shared__ float ys[];
  __shared__ float tb[NB];
  const int tid = threadIdx.x, bd = blockDim.x;
  for (int i = tid; i < m; i += bd) ys[i] = (float)r[i];
  __syncthreads();
  const int nblk = (m + NB - 1) / NB;
  // forward: y = L^{-1} r, right-looking by blocks
  for (int kb = 0; kb < nblk; ++kb) {
    const int b0 = kb * NB, nb = m - b0 < NB ? m - b0 : NB;
    const float *Li = Linv + (int64_t)kb * NB * NB;
    if (tid < nb) {
      float a = 0.f;
      for (int l = 0; l <= tid; ++l) a = fmaf(Li[tid + l * NB], ys[b0 + l], a);
      tb[tid] = a;
    }
    __syncthreads();
    if (tid < nb) ys[b0 + tid] = tb[tid];
    __syncthreads();
    for (int i = b0 + nb + tid; i < m; i += bd) {
      float a = 0.f;
      for (int l = 0; l < nb; ++l) a = fmaf(L[i + (int64_t)(b0 + l) * m], tb[l], a);
      ys[i] -= a;
    }
    __syncthreads();
  }
  // backward: x = L^{-T} y, by blocks from the last; L^T read from the upper triangle
  for (int kb = nblk - 1; kb >= 0; --kb) {
    const int b0 = kb * NB, nb = m - b0 < NB ? m - b0 : NB;
    const float *Li = Linv + (int64_t)kb * NB * NB;
    if (tid < nb) {
      float a = 0.f;
      for (int l = tid; l < nb; ++l) a = fmaf(Li[l + tid * NB], ys[b0 + l], a);  // Linv[l][tid]
      tb[tid] = a;
    }
    __syncthreads();
    if (tid < nb) ys[b0 + tid] = tb[tid];
    __syncthreads();
    for (int i = tid; i < b0; i += bd) {
      float a = 0.f;
      for (int l = 0; l < nb; ++l) a = fmaf(L[i + (int64_t)(b0 + l) * m], tb[l], a);  // L^T[i][b0+l]
      ys[i] -= a;
    }
    __syncthreads();
  }
  for (int i = tid; i < m; i += bd) x[i] += (double)ys[i];
}

// y = B x and ay_i = sum_j |B_ij x_j| for the symmetric B stored in its lower triangle (FP64).
// CTA = 32 rows (256 threads): the part j <= i is read along rows (lane = row, 8 column phases),
// the part j > i along the columns of the block (warp = column, lanes over j), both coalesced.
__global__ void k_symv_f64(const double *__restrict__ B, int64_t ldb, int m,
                           const double *__restrict__ x, double *y, double *ay) {
  __shared__ double p1[8][33], a1[8][33];
  __shared__ double p2[32], a2[32];
  const int il = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int ib = blockIdx.x * 32, i = ib + il;
  double s = 0.0, sa = 0.0;
  if (i < m)
    for (int j = w; j <= i; j += 8) {
      const double v = B[i + (int64_t)j * ldb] * x[j];
      s += v;
      sa += fabs(v);
    }
  p1[w][il] = s;
  a1[w][il] = sa;
  for (int cc = w; cc < 32; cc += 8) {
    const int ii = ib + cc;
    double t = 0.0, ta = 0.0;
    if (ii < m)
      for (int j = ii + 1 + il; j < m; j += 32) {
        const double v = B[j + (int64_t)ii * ldb] * x[j];
        t += v;
        ta += fabs(v);
      }
    for (int o = 16; o > 0; o >>= 1) {
      t += __shfl_xor_sync(0xffffffffu, t, o);
      ta += __shfl_xor_sync(0xffffffffu, ta, o);
    }
    if (il == 0) {
      p2[cc] = t;
      a2[cc] = ta;
    }
  }
  __syncthreads();
  if (w == 0 && i < m) {
    double r = p2[il], ra = a2[il];
    for (int q = 0; q < 8; ++q) {
      r += p1[q][il];
      ra += a1[q][il];
    }
    y[i] = r;
    ay[i] = ra;
  }
}

// r = g - y; out[0] = max_i |r_i|, out[1] = max_i (ay_i + |g_i|)  (one CTA)
__global__ void k_resid(const double *__restrict__ g, const double *__restrict__ y,
                        const double *__restrict__ ay, double *r, int m, double *out) {
  __shared__ double mr[32], mg[32];
  double ar = 0.0, ag = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double v = g[i] - y[i];
    r[i] = v;
    ar = fmax(ar, fabs(v));
    ag = fmax(ag, ay[i] + fabs(g[i]));
  }
  for (int o = 16; o > 0; o >>= 1) {
    ar = fmax(ar, __shfl_down_sync(0xffffffffu, ar, o));
    ag = fmax(ag, __shfl_down_sync(0xffffffffu, ag, o));
  }
  if ((threadIdx.x & 31) == 0) {
    mr[threadIdx.x >> 5] = ar;
    mg[threadIdx.x >> 5] = ag;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double u = 0.0, v = 0.0;
    for (int q = 0; q < (int)(blockDim.x + 31) / 32; ++q) {
      u = fmax(u, mr[q]);
      v = fmax(v, mg[q]);
    }
    out[0] = u;
    out[1] = v;
  }
}

// g <- row m of B (the right-hand side border), r <- g, x <- 0
__global__ void k_mixed_init(const double *__restrict__ B, int64_t ldb, int m, double *g, double *r,
                             double *x) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
    const double v = B[m + (int64_t)j * ldb];
    g[j] = v;
    r[j] = v;
    x[j] = 0.0;
  }
}

int mixed_factor(const double *B, int64_t ldb, int m, float *B32, float *Linv32, int *status,
                 double *g, double *r, double *x, cudaStream_t st, cudaStream_t st2,
                 cudaEvent_t *ev_next, cudaEvent_t *ev_rest) {
  k_mixed_init<<<(m + 255) / 256, 256, 0, st>>>(B, ldb, m, g, r, x);
  int blocks = (int)(((int64_t)m * m + 255) / 256);
  if (blocks > 8192) blocks = 8192;
  k_lower_to_f32<<<blocks, 256, 0, st>>>(B, ldb, B32, m);
  int nl = 1 + dense_chol_f32(B32, m, m, status, Linv32, st, st2, ev_next, ev_rest);
  k_lower_to_upper_f32<<<blocks, 256, 0, st>>>(B32, m);
  return nl + 2;
}

int mixed_refine_step(const double *B, int64_t ldb, int m, const float *L32, const float *Linv32,
                      const double *g, double *x, double *r, double *y, double *ay, double *norms,
                      cudaStream_t st) {
  const size_t smem = (size_t)m * sizeof(float);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_refine_solve_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_refine_solve_f32<<<1, 1024, smem, st>>>(L32, m, Linv32, r, x);
  k_symv_f64<<<(m + 31) / 32, 256, 0, st>>>(B, ldb, m, x, y, ay);
  k_resid<<<1, 1024, 0, st>>>(g, y, ay, r, m, norms);
  return 3;
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
  dense_chol_bordered(Bw, ldw, m, status, Binv, st, nullptr, nullptr, nullptr);
  dense_backsolve(Bw, ldw, m, Binv, x, st);
  if (cudaGetLastError() != cudaSuccess) return MCSDP_ERR_CUDA;
  int hst = 0;
  if (cudaMemcpyAsync(&hst, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return MCSDP_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return MCSDP_ERR_CUDA;
  return (hst & ST_NOT_PD) ? MCSDP_ERR_NOT_PD : MCSDP_OK;
}
