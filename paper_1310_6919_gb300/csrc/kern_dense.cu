// K4: S-CHOLESKY, type (i) of Sec. 3.1: dense Cholesky of the SCM B and the solve of the
// Schur complement equation B dz = g (eq. SCE).
//
// B (internal constraint order) is stored column-major with one extra row: row m holds g^T.
// A right-looking blocked factorisation of the leading m columns carries that row through the
// panel solves and trailing updates, so on exit row m holds (L^{-1} g)^T and only the backward
// substitution L^T dz = L^{-1} g remains.  In FP64 the factorisation is one persistent
// task-queue launch (k_chol_dag); the launch-per-panel form serves the mixed form's FP32 factor
// (graph-captured, lookahead streams) and the allocation-free solve (one stream).  The mixed
// form's FP32 factor and FP64 refinement are at the end of the file.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <type_traits>

#include "../../include/mcsdp.h"
#include "internal.h"
#include "tc.h"

namespace mcsdp {

constexpr int NB = 32;  // panel width (FP64 on one SM is slow: a narrow panel keeps the
                        // serial factor-and-invert step short)

// Cholesky of the nb x nb diagonal block at (k0, k0), one CTA of 256 threads, and the inverse
// of the factor (stored in Linv, nb x nb column-major, ld NB).  The serial column loop is the
// critical path of the whole factorisation, so it is warp-specialised with one barrier per
// column: at step j, warp 0 brings column j+1 up to date, takes its pivot d_{j+1}, the
// reciprocal and the scaled column U[:, j+1] (five dependent FP64 operations: the update, three
// for the reciprocal, the scaling; the pivot test is integer); warps 1-7 meanwhile apply step j
// to the columns >= j+2 and step j of the inverse U^{-1} (forward elimination, row j final).
// FP64 on this part issues one warp instruction per 64 cycles per warp and about one per 16
// cycles per SM, so the bulk work of a step is packed densely (at most three elements per
// thread) and each thread loads all its operands before its independent FMAs.  This is
// A = U D U^T with U unit lower; L = U D^{1/2} and L^{-1} = D^{-1/2} U^{-1} follow with the nb
// square roots taken in parallel.
template <class T>
struct PotrfSmem {
  T A[NB * (NB + 1)];  // working copy, row-major; the trailing part is updated in place
  T U[NB * (NB + 1)];  // unit lower factor, row-major
  T V[NB * (NB + 1)];  // U^{-1}, row-major
  T rd[NB], dd[NB];
  unsigned char pr[NB * (NB - 1) / 2], pc[NB * (NB - 1) / 2];  // packed e -> (row, column)
};

// CG: read B through L2 only (the task-queue factorisation, whose tiles other SMs write)
template <class T, bool CG>
__device__ __forceinline__ void potrf_block(T *B, int64_t ldb, int k0, int nb, int *status,
                                            T *Linv, PotrfSmem<T> &sm) {
  constexpr int LD = NB + 1;
  constexpr int NBULK = 224;  // warps 1-7
  constexpr int SLOTS = 3;    // elements per bulk thread and step: at most 496 <= 3 x 224
  T *A = sm.A, *U = sm.U, *V = sm.V, *rd = sm.rd, *dd = sm.dd;
  unsigned char *pr = sm.pr, *pc = sm.pc;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int idx = tid; idx < NB * NB; idx += 256) {
    const int i = idx % NB, j = idx / NB;
    const T *src = B + (k0 + i) + (int64_t)(k0 + j) * ldb;
    A[i * LD + j] = (i >= j && i < nb && j < nb) ? (CG ? __ldcg(src) : *src) : T(0);
    V[i * LD + j] = (i == j) ? T(1) : T(0);
    U[i * LD + j] = (i == j) ? T(1) : T(0);
  }
  if (tid < NB - 1)
    for (int c = 0; c <= tid; ++c) {
      pr[tid * (tid + 1) / 2 + c] = (unsigned char)tid;
      pc[tid * (tid + 1) / 2 + c] = (unsigned char)c;
    }
  __syncthreads();
  bool bad = false;
  if (warp == 0) {  // column 0: pivot, reciprocal, scaled column
    T d = A[0];
    if (!pivot_positive(d)) {
      bad = true;
      d = T(1);
    }
    const T r0 = pivot_rcp<T>(d);
    if (lane == 0) dd[0] = d;
    if (lane >= 1 && lane < nb) U[lane * LD] = A[lane * LD] * r0;
  }
  __syncthreads();
  const int bt = tid - 32;  // bulk thread index (warps 1-7)
  for (int j = 0; j < nb; ++j) {
    if (warp == 0) {
      if (j + 1 < nb) {
        // column j+1 (rows >= j+1) receives step j, then its pivot and scaled column; every
        // lane takes the pivot and its reciprocal (no second shuffle)
        const int r = j + 1 + lane;
        T a = T(0);
        if (r < nb) {
          a = fma(-U[r * LD + j], A[(j + 1) * LD + j], A[r * LD + j + 1]);
          A[r * LD + j + 1] = a;
        }
        T d = __shfl_sync(0xffffffffu, a, 0);
        if (!pivot_positive(d)) {
          bad = true;
          d = T(1);
        }
        const T rj = pivot_rcp<T>(d);
        if (lane == 0) dd[j + 1] = d;
        if (r < nb && lane >= 1) U[r * LD + j + 1] = a * rj;
      }
    } else {
      // step j on columns >= j+2 (rows >= column): A[ii][kk] -= U[ii][j] A[kk][j]; and step j
      // of the inverse: V[i][c] -= U[i][j] V[j][c] for i > j, c <= j (element f of the
      // (nb-1-j) x (j+1) block: i = j+1 + f div (j+1), by an FP32 product exact for f < 1024)
      const int s = nb - 2 - j;
      const int ntr = s > 0 ? s * (s + 1) / 2 : 0;
      const int w = j + 1, ntot = ntr + (nb - 1 - j) * w;
      const float rw = 1.0f / (float)w;
      T x[SLOTS], u[SLOTS], v[SLOTS];
      T *dst[SLOTS];
#pragma unroll
      for (int q = 0; q < SLOTS; ++q) {
        const int e = bt + q * NBULK;
        dst[q] = nullptr;
        if (e < ntr) {
          const int ii = j + 2 + pr[e], kk = j + 2 + pc[e];
          dst[q] = &A[ii * LD + kk];
          u[q] = U[ii * LD + j];
          v[q] = A[kk * LD + j];
        } else if (e < ntot) {
          const int f = e - ntr, qq = (int)(((float)f + 0.5f) * rw);
          const int i = j + 1 + qq, c = f - qq * w;
          dst[q] = &V[i * LD + c];
          u[q] = U[i * LD + j];
          v[q] = V[j * LD + c];
        }
        if (dst[q]) x[q] = *dst[q];
      }
#pragma unroll
      for (int q = 0; q < SLOTS; ++q)
        if (dst[q]) *dst[q] = fma(-u[q], v[q], x[q]);
    }
    __syncthreads();
  }
  if (bad && lane == 0) atomicOr(status, ST_NOT_PD);  // warp 0's lanes saw the same pivots
  if (tid < nb) {
    const T sq = sqrt(dd[tid]);
    dd[tid] = sq;
    rd[tid] = pivot_rcp<T>(sq);
  }
  __syncthreads();
  for (int idx = tid; idx < NB * NB; idx += 256) {
    const int i = idx % NB, j = idx / NB;
    const bool in = i < nb && j < nb && i >= j;
    if (in) {
      const T v = (i == j) ? dd[j] : U[i * LD + j] * dd[j];
      B[(k0 + i) + (int64_t)(k0 + j) * ldb] = v;
      if (i > j) B[(k0 + j) + (int64_t)(k0 + i) * ldb] = v;  // L^T in the strict upper triangle
    }
    Linv[i + j * NB] = in ? V[i * LD + j] * rd[i] : T(0);
  }
}

template <class T>
__global__ void __launch_bounds__(256)
    k_potrf_diag(T *B, int64_t ldb, int k0, int nb, int *status, T *Linv) {
  __shared__ PotrfSmem<T> sm;
  potrf_block<T, false>(B, ldb, k0, nb, status, Linv, sm);
}

// FP32 diagonal block (the mixed form's factor): one warp, lane r holds row r of the block in
// registers.  Column j: every lane takes the pivot by a shuffle, the column is scaled, and row r
// receives - L[r][j] L[kk][j] for every kk <= r, L[kk][j] shuffled from lane kk; the inverse is
// formed the same way (row k of L^{-1} final after step k, then broadcast).  No barriers and no
// shared memory: FP32 arithmetic is cheap here, the serial chain is shuffles.
__global__ void __launch_bounds__(32)
    k_potrf_warp_f32(float *B, int64_t ldb, int k0, int nb, int *status, float *Linv) {
  const int lane = threadIdx.x;
  float a[NB], t[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    a[j] = (lane < nb && j < nb && lane >= j) ? B[(k0 + lane) + (int64_t)(k0 + j) * ldb] : 0.f;
    t[j] = (j == lane) ? 1.f : 0.f;
  }
  bool bad = false;
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    if (j < nb) {
      float d = __shfl_sync(0xffffffffu, a[j], j);
      if (!(d > 0.f)) {
        bad = true;
        d = 1.f;
      }
      const float sq = __fsqrt_rn(d), rs = __frcp_rn(sq);
      if (lane == j) a[j] = sq;
      else if (lane > j) a[j] *= rs;
#pragma unroll
      for (int kk = j + 1; kk < NB; ++kk) {
        const float lkj = __shfl_sync(0xffffffffu, a[j], kk);
        if (lane >= kk) a[kk] = fmaf(-a[j], lkj, a[kk]);
      }
    }
  }
  // L^{-1}: step k scales row k (lane k) by 1 / L[k][k] and removes L[r][k] times it from rows r > k
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    if (k < nb) {
      const float rk = __frcp_rn(__shfl_sync(0xffffffffu, a[k], k));
      if (lane == k) {
#pragma unroll
        for (int c = 0; c <= k; ++c) t[c] *= rk;
      }
#pragma unroll
      for (int c = 0; c <= k; ++c) {
        const float tkc = __shfl_sync(0xffffffffu, t[c], k);
        if (lane > k) t[c] = fmaf(-a[k], tkc, t[c]);
      }
    }
  }
  if (lane < nb) {
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      if (j <= lane && j < nb) {
        B[(k0 + lane) + (int64_t)(k0 + j) * ldb] = a[j];
        if (j < lane) B[(k0 + j) + (int64_t)(k0 + lane) * ldb] = a[j];  // L^T, upper triangle
      }
    }
  }
#pragma unroll
  for (int c = 0; c < NB; ++c)
    Linv[lane + c * NB] = (lane < nb && c <= lane && c < nb) ? t[c] : 0.f;
  if (bad && lane == 0) atomicOr(status, ST_NOT_PD);  // every lane saw the same pivots
}

// Rows [r0, rend) of the panel columns [k0, k0+nb): X <- X L_kk^{-T} = X Linv^T.  CTA = 4 rows
// x 32 columns (128 threads, one output each: thread = (row, column = lane)); a CTA owns whole
// rows, so it solves them in place.  Small CTAs spread the panel solve over all SMs (FP64 runs
// at two lanes per cycle per SM here).  Rows below ncl (the matrix proper, not the border row)
// are also stored transposed into the strict upper triangle, so the factor's rows can later be
// read as contiguous columns.
constexpr int TRSM_ROWS = 4;
template <class T>
__global__ void k_trsm_panel(T *B, int64_t ldb, int k0, int nb, int r0, int rend, int ncl,
                             const T *__restrict__ Linv) {
  __shared__ T Xs[TRSM_ROWS][NB + 1];
  __shared__ T Ts[NB][NB + 1];  // Ts[l][c] = Linv[c][l]
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int gi = r0 + blockIdx.x * TRSM_ROWS + w;
  Xs[w][lane] = (gi < rend && lane < nb) ? B[gi + (int64_t)(k0 + lane) * ldb] : T(0);
  for (int idx = tid; idx < NB * NB; idx += TRSM_ROWS * 32) {
    const int c = idx % NB, l = idx / NB;
    Ts[l][c] = Linv[c + l * NB];
  }
  __syncthreads();
  T acc = T(0);
#pragma unroll 8
  for (int l = 0; l < NB; ++l) acc = fma(Xs[w][l], Ts[l][lane], acc);
  if (gi < rend && lane < nb) {
    B[gi + (int64_t)(k0 + lane) * ldb] = acc;
    if (gi < ncl) B[(k0 + lane) + (int64_t)gi * ldb] = acc;
  }
}

// Update of block column k+1 (columns [c0, c1), c1 - c0 <= 32) by panel k (columns [k0, k0+nb))
// for the rows [c0, rend), lower part: C[i][c] -= sum_l P[i][l] P[c][l].  CTA = 4 rows x 32
// columns (128 threads, thread = (row, column = lane)); on the critical path, so the work is
// spread over many small CTAs.
template <class T>
__global__ void k_syrk_next(T *B, int64_t ldb, int k0, int nb, int c0, int c1, int rend) {
  __shared__ T Pi[TRSM_ROWS][NB + 1];
  __shared__ T Pc[NB][NB + 1];  // Pc[l][c] = P[c0 + c][l]
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int gi = c0 + blockIdx.x * TRSM_ROWS + w;
  Pi[w][lane] = (gi < rend && lane < nb) ? B[gi + (int64_t)(k0 + lane) * ldb] : T(0);
  for (int idx = tid; idx < NB * NB; idx += TRSM_ROWS * 32) {
    const int c = idx % NB, l = idx / NB;
    Pc[l][c] = (c0 + c < c1 && l < nb) ? B[(c0 + c) + (int64_t)(k0 + l) * ldb] : T(0);
  }
  __syncthreads();
  T acc = T(0);
#pragma unroll 8
  for (int l = 0; l < NB; ++l) acc = fma(Pi[w][l], Pc[l][lane], acc);
  const int gc = c0 + lane;
  if (gi < rend && gc < c1 && gi >= gc) B[gi + (int64_t)gc * ldb] -= acc;
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

// ---- Task-queue factorisation (FP64): one persistent launch ----
// The right-looking blocked Cholesky as tasks on 32 x 32 tiles (R row tiles of the rows x m
// matrix, C column tiles):
//   POTRF(k)      diagonal tile k: factor and inverse (potrf_block)
//   TRSM(i, k)    tile (i, k), i > k: L(i, k) = A(i, k) L(k, k)^{-T}
//   UPD(i, j, k)  tile (i, j), i >= j > k: A(i, j) -= L(i, k) L(j, k)^T (lower part if i == j)
// The chain from one diagonal tile to the next is what bounds the last panels, so its tiles are
// split over several CTAs: TRSM(p, p-1) over eight tasks TS(p, s) of four rows, UPD(p, p, p-1)
// over eight tasks UD(p, s) of four rows, then NEXT(p) = POTRF(p).
// CTAs take tickets from one counter; ticket order puts every dependency before its dependants:
//   POTRF(0), TRSM(2..R-1, 0), TS(1, 0..7), UD(1, 0..7), NEXT(1), then for k = 0 .. C-2:
//     UPD(i, j, k) for j >= k+2      the rest of panel k's update (column k+2 first), with
//     UPD(k+2.., k+1, k)             the rest of the next column placed DAG_DEFER_COL tickets
//                                    into it, right after it the chain step to tile k+2,
//     TS(k+2, .), UD(k+2, .), NEXT(k+2)  which needs only UPD(k+2, k+2, k) and UPD(k+2, k+1, k)
//                                    of this panel (so it runs one panel ahead), and
//     TRSM(k+3.., k+1)               DAG_DEFER_TRSM tickets in, when NEXT(k+1) has normally
//                                    finished.
// A CTA holding the smallest unfinished ticket finds all its dependencies done, so the queue
// always progresses whatever the residency (no co-scheduling needed).  Per tile (i, j) the host
// zeroes upd[i][j] (updates applied; UPD(i, j, k) waits for k of them, which also serialises
// the updates of one tile) and fin[i][j] (1 once L(i, j) is final).  The tiles are written and
// read through L2 (ld.global.cg; release = fence + atomic add, acquire = ld.acquire.gpu).  Every
// wait is bounded: on timeout the CTA sets the abort word and ST_TIMEOUT and every CTA leaves.
// Against the launch-per-panel form this keeps the trailing tiles flowing across panels (no
// launch gaps, no half-empty last waves per panel) while the next column's chain runs ahead.
constexpr int DAG_THREADS = 256;
// CTAs per SM: while one loads its tiles, waits or synchronises, the others keep the FP64 pipe
// busy (m = 8000: 164 ms per factorisation with two, 154 with three, 150 with four; four hold
// the kernel to 64 registers a thread, without spills)
constexpr int DAG_CTAS_PER_SM = 4;
constexpr int64_t DAG_SPIN_LIMIT = 1 << 23;  // polls per wait (a few seconds with backoff)
constexpr int64_t DAG_DEFER_COL = 64;    // tickets of panel k's rest before UPD(., k+1, k)
constexpr int64_t DAG_DEFER_TRSM = 256;  // and before TRSM(., k+1)

struct DagSync {
  int *ticket, *abort, *upd, *fin;
  int *smbusy;  // per SM: 1 while a task of the diagonal chain runs there
  int C;
  long long budget;  // SM clock cycles one wait may take before it gives up
};
constexpr long long DAG_DEFAULT_BUDGET = 1ll << 32;  // about two seconds at 2 GHz
constexpr int DAG_MAX_SM = 1024;                     // words of the per-SM flags
// The chain's tasks (TS, UD, the diagonal factor) bound the last panels and FP64 issue is shared
// by the SM: while one runs, the other CTA on its SM holds back its next panel solve or update
// (at most this many cycles, a scheduling hint only: it then goes ahead, so it never deadlocks)
constexpr long long DAG_YIELD_CYCLES = 100000;

__device__ __forceinline__ unsigned sm_id() {
  unsigned v;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(v));
  return v;
}

__device__ __forceinline__ int ld_acquire(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// thread 0: wait until every *f[x] >= tg[x] (x < n), the flags polled together; false on abort
// or once the wait has taken q.budget cycles (or DAG_SPIN_LIMIT polls), which raises the abort
// word and ST_TIMEOUT
__device__ bool dag_wait_all(const int *const *f, const int *tg, int n, const DagSync &q,
                             int *status) {
  unsigned ns = 32;
  const long long t0 = clock64();
  for (int64_t it = 0;; ++it) {
    int v[3];
    for (int x = 0; x < n; ++x) v[x] = ld_acquire(f[x]);
    bool ready = true;
    for (int x = 0; x < n; ++x) ready = ready && v[x] >= tg[x];
    if (ready) return true;
    if (ld_acquire(q.abort)) return false;
    if (it >= DAG_SPIN_LIMIT || clock64() - t0 > q.budget) break;
    __nanosleep(ns);
    if (ns < 256) ns <<= 1;
  }
  atomicExch(q.abort, 1);
  atomicOr(status, ST_TIMEOUT);
  return false;
}

// sum_{j = a}^{C-1} (R - j)
__device__ __host__ __forceinline__ int64_t dag_tail(int64_t a, int64_t R, int64_t C) {
  if (a >= C) return 0;
  const int64_t u = C - a;
  return u * R - (u * (a + C - 1)) / 2;
}
// first row tile of the TRSM block of iteration k (tile (k+2, k+1) belongs to NEXT(k+2))
__device__ __host__ __forceinline__ int64_t dag_trsm_lo(int64_t k, int64_t C) {
  return k + 2 < C ? k + 3 : k + 2;
}
constexpr int DAG_TS = NB / 4;  // TS tasks per chain step
// tickets of the chain step to diagonal tile p (TS, UD, NEXT); none past the last tile
__device__ __host__ __forceinline__ int64_t dag_head(int64_t p, int64_t C) {
  return p <= C - 1 ? 2 * DAG_TS + 1 : 0;
}
// tickets of iteration k (k = 0 .. C-2): panel k's rest, the next column's rest, the chain step
// to tile k+2, the panel solves of column k+1
__device__ __host__ __forceinline__ int64_t dag_iter_size(int64_t k, int64_t R, int64_t C) {
  const int64_t lo = dag_trsm_lo(k, C);
  return dag_tail(k + 2, R, C) + (R - k - 2) + dag_head(k + 2, C) + (R > lo ? R - lo : 0);
}
// completions that make tile (i, k) final: eight TS tasks for a tile left of a diagonal tile
__device__ __forceinline__ int dag_fin_target(int i, int k, int C) {
  return (i == k + 1 && i < C) ? DAG_TS : 1;
}

// tickets before iteration 0: POTRF(0), TRSM(lo0.., 0) (npre of them), the chain step to tile 1
struct DagPrefix {
  int lo0;
  int64_t npre, pre;
};
__device__ __host__ __forceinline__ DagPrefix dag_prefix(int R, int C) {
  DagPrefix d;
  d.lo0 = C > 1 ? 2 : 1;  // first TRSM(., 0) row tile (tile (1, 0) belongs to the chain step)
  d.npre = 1 + (R > d.lo0 ? R - d.lo0 : 0);
  d.pre = d.npre + dag_head(1, C);
  return d;
}
// all tickets of an R x C tile factorisation
__device__ __host__ __forceinline__ int64_t dag_total(int R, int C) {
  int64_t total = dag_prefix(R, C).pre;
  for (int64_t k = 0; k + 1 < C; ++k) total += dag_iter_size(k, R, C);
  return total;
}

// Ticket t -> task (type, i, j, k): 0 POTRF(0), 1 TRSM(i, k), 2 UPD(i, j, k), 3 NEXT(k) (the
// factor of diagonal tile k), 4 TS(k, s = j), 5 UD(k, s = j).  (kcur, kstart) carry the
// iteration found for the previous, smaller ticket of the caller (start: 0, dag_prefix().pre).
struct DagTask {
  int type, i, j, k;
};
__device__ __host__ __forceinline__ DagTask dag_decode(int64_t t, int R, int C, const DagPrefix &pf,
                                                       int &kcur, int64_t &kstart) {
  DagTask d{0, 0, 0, 0};
  int hp = -1;  // chain step to tile hp, element he of its header
  int64_t he = 0;
  if (t == 0) {
    return d;
  } else if (t < pf.npre) {
    d.type = 1; d.i = pf.lo0 + (int)t - 1;
    return d;
  } else if (t < pf.pre) {
    hp = 1; he = t - pf.npre;
  } else {
    while (kcur + 1 < C && t >= kstart + dag_iter_size(kcur, R, C)) {
      kstart += dag_iter_size(kcur, R, C);
      ++kcur;
    }
    int64_t e = t - kstart;
    const int k = kcur, n1 = R - k - 2;
    // rest[0, dc) | next column (n1) | chain step to k+2 (nh) | rest[dc, dt) | TRSM block |
    // rest[dt, ..): the chain step needs rest[0] = UPD(k+2, k+2, k) and the next column's
    // UPD(k+2, k+1, k) before it, so it runs one panel ahead of the trailing work
    const int64_t rest = dag_tail(k + 2, R, C), lo = dag_trsm_lo(k, C);
    const int64_t ntr = R > lo ? R - lo : 0, nh = dag_head(k + 2, C);
    int64_t dc = rest < DAG_DEFER_COL ? rest : DAG_DEFER_COL;
    if (dc < 1 && rest > 0) dc = 1;
    int64_t dt = rest < DAG_DEFER_TRSM ? rest : DAG_DEFER_TRSM;
    if (dt < dc) dt = dc;
    int64_t ri = -1;
    if (e < dc) {
      ri = e;
    } else if (e < dc + n1) {
      d.type = 2; d.i = k + 2 + (int)(e - dc); d.j = k + 1; d.k = k;
    } else if (e < dc + n1 + nh) {
      hp = k + 2; he = e - dc - n1;
    } else if (e < dt + n1 + nh) {
      ri = e - n1 - nh;
    } else if (e < dt + n1 + nh + ntr) {
      d.type = 1; d.i = (int)(lo + e - dt - n1 - nh); d.j = d.k = k + 1;
    } else {
      ri = e - n1 - nh - ntr;
    }
    if (ri >= 0) {
      int j = k + 2;
      while (j < C && ri >= R - j) {
        ri -= R - j;
        ++j;
      }
      d.type = 2; d.i = j + (int)ri; d.j = j; d.k = k;  // j < C for every ticket below total
    }
  }
  if (hp >= 0) {  // TS(hp, s), UD(hp, s), NEXT(hp)
    d.i = d.k = hp;
    if (he < DAG_TS) {
      d.type = 4; d.j = (int)he;
    } else if (he < 2 * DAG_TS) {
      d.type = 5; d.j = (int)(he - DAG_TS);
    } else {
      d.type = 3; d.j = hp;
    }
  }
  return d;
}

// TRSM(i, k): rows [i0, i0 + h) of columns [k0, k0 + nb).  Thread = (row r = tid / 8, columns
// c = tid % 8 + 8 q, q < 4): four independent 32-term dot products with the inverse's rows.
template <class T>
__device__ void dag_trsm(T *B, int64_t ldb, int i0, int h, int k0, int nb, int ncl,
                         const T *Linv, T *sm) {
  constexpr int LD = NB + 1;
  T *Xs = sm, *Ls = sm + NB * LD;  // Xs[r][l]; Ls[l][c] = Linv[c][l]
  const int tid = threadIdx.x;
  for (int idx = tid; idx < NB * NB; idx += DAG_THREADS) {
    const int r = idx & (NB - 1), l = idx / NB;
    Xs[r * LD + l] = (r < h && l < nb) ? __ldcg(B + (i0 + r) + (int64_t)(k0 + l) * ldb) : T(0);
    Ls[l * LD + r] = __ldcg(Linv + r + l * NB);  // here r plays the column c
  }
  __syncthreads();
  const int r = tid >> 3, c0 = tid & 7;
  T acc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll 8
  for (int l = 0; l < NB; ++l) {
    const T x = Xs[r * LD + l];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = fma(x, Ls[l * LD + c0 + 8 * q], acc[q]);
  }
  if (r < h) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = c0 + 8 * q;
      if (c < nb) {
        B[(i0 + r) + (int64_t)(k0 + c) * ldb] = acc[q];
        if (i0 + r < ncl) B[(k0 + c) + (int64_t)(i0 + r) * ldb] = acc[q];  // L^T, upper part
      }
    }
  }
}

// TS(p, s): rows i0 .. i0 + h (h <= 4) of the tile left of diagonal tile p, L = X Linv^T with
// the full-width previous panel (nb = NB); two threads per output split the 32 terms.
template <class T>
__device__ void dag_trsm4(T *B, int64_t ldb, int i0, int h, int k0, int ncl, const T *Linv,
                          T *sm) {
  constexpr int LD = NB + 1;
  T *Xs = sm, *Ls = sm + 4 * LD;  // Xs[r][l]; Ls[l][c] = Linv[c][l]
  const int tid = threadIdx.x;
  if (tid < 4 * NB) {
    const int r = tid & 3, l = tid >> 2;
    Xs[r * LD + l] = r < h ? __ldcg(B + (i0 + r) + (int64_t)(k0 + l) * ldb) : T(0);
  }
  for (int idx = tid; idx < NB * NB; idx += DAG_THREADS) {
    const int c = idx & (NB - 1), l = idx / NB;
    Ls[l * LD + c] = __ldcg(Linv + c + l * NB);
  }
  __syncthreads();
  const int o = tid >> 1, half = tid & 1, r = o >> 5, c = o & (NB - 1);
  T a0 = T(0), a1 = T(0);
#pragma unroll
  for (int l = half * 16; l < half * 16 + 16; l += 2) {
    a0 = fma(Xs[r * LD + l], Ls[l * LD + c], a0);
    a1 = fma(Xs[r * LD + l + 1], Ls[(l + 1) * LD + c], a1);
  }
  T acc = a0 + a1;
  acc += __shfl_xor_sync(0xffffffffu, acc, 1);
  if (half == 0 && r < h) {
    B[(i0 + r) + (int64_t)(k0 + c) * ldb] = acc;
    if (i0 + r < ncl) B[(k0 + c) + (int64_t)(i0 + r) * ldb] = acc;  // L^T, upper part
  }
}

// UD(p, s): rows r0 .. r0 + h (h <= 4) of the diagonal tile at (k0, k0) (with the
// right-hand-side row when it lies in that tile row), columns c <= r, c < nb, minus
// L(p, p-1)[r] . L(p, p-1)[c] (the previous panel, full width); two threads per output.
template <class T>
__device__ void dag_upd4(T *B, int64_t ldb, int k0, int r0, int h, int nb, T *sm) {
  constexpr int LD = NB + 1;
  T *Lr = sm, *Lc = sm + 4 * LD;  // Lr[r][l] rows r0.., Lc[c][l] rows k0..
  const int tid = threadIdx.x;
  const int q0 = k0 - NB;
  if (tid < 4 * NB) {
    const int r = tid & 3, l = tid >> 2;
    Lr[r * LD + l] = r < h ? __ldcg(B + (k0 + r0 + r) + (int64_t)(q0 + l) * ldb) : T(0);
  }
  for (int idx = tid; idx < NB * NB; idx += DAG_THREADS) {
    const int c = idx & (NB - 1), l = idx / NB;
    Lc[c * LD + l] = c < nb ? __ldcg(B + (k0 + c) + (int64_t)(q0 + l) * ldb) : T(0);
  }
  __syncthreads();
  const int o = tid >> 1, half = tid & 1, r = o >> 5, c = o & (NB - 1);
  T a0 = T(0), a1 = T(0);
#pragma unroll
  for (int l = half * 16; l < half * 16 + 16; l += 2) {
    a0 = fma(Lr[r * LD + l], Lc[c * LD + l], a0);
    a1 = fma(Lr[r * LD + l + 1], Lc[c * LD + l + 1], a1);
  }
  T acc = a0 + a1;
  acc += __shfl_xor_sync(0xffffffffu, acc, 1);
  if (half == 0 && r < h && c < nb && c <= r0 + r) {
    T *dst = B + (k0 + r0 + r) + (int64_t)(k0 + c) * ldb;
    *dst = __ldcg(dst) - acc;
  }
}

// UPD(i, j, k): C rows [i0, i0 + h) x columns [j0, j0 + w) -= L(i, k) L(j, k)^T, the lower part
// only on a diagonal tile (diag).  2 x 2 outputs per thread, K = nb.
template <class T>
__device__ void dag_upd(T *B, int64_t ldb, int i0, int h, int j0, int w, int k0, int nb, bool diag,
                        T *sm) {
  T *Ai = sm, *Aj = sm + NB * NB;  // [l][row]
  const int tid = threadIdx.x;
  for (int idx = tid; idx < NB * NB; idx += DAG_THREADS) {
    const int rr = idx & (NB - 1), l = idx / NB;
    const bool lk = l < nb;
    Ai[l * NB + rr] = (lk && rr < h) ? __ldcg(B + (i0 + rr) + (int64_t)(k0 + l) * ldb) : T(0);
    Aj[l * NB + rr] = (lk && rr < w) ? __ldcg(B + (j0 + rr) + (int64_t)(k0 + l) * ldb) : T(0);
  }
  __syncthreads();
  const int tx = tid & 15, ty = tid >> 4;
  T acc[2][2] = {};
#pragma unroll 8
  for (int l = 0; l < NB; ++l) {
    const T a0 = Ai[l * NB + ty * 2], a1 = Ai[l * NB + ty * 2 + 1];
    const T b0 = Aj[l * NB + tx * 2], b1 = Aj[l * NB + tx * 2 + 1];
    acc[0][0] = fma(a0, b0, acc[0][0]);
    acc[0][1] = fma(a0, b1, acc[0][1]);
    acc[1][0] = fma(a1, b0, acc[1][0]);
    acc[1][1] = fma(a1, b1, acc[1][1]);
  }
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const int r = ty * 2 + p;
    if (r >= h) continue;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int c = tx * 2 + q;
      if (c < w && (!diag || r >= c)) {
        T *dst = B + (i0 + r) + (int64_t)(j0 + c) * ldb;
        *dst = __ldcg(dst) - acc[p][q];
      }
    }
  }
}

// Several independent factorisations in one queue (the diagonal blocks of a block-diagonal B):
// block b is the bordered matrix at rows and columns off[b] (mb[b] columns, its right-hand side
// in row off[b] + mb[b]); its tile counters (upd, then fin) start at word soff[b] after the
// queue's eight header words, its diagonal-tile inverses at Linv_all + loff[b].  Each block's
// tickets fall into phases (the prefix, then iteration k = 0 .. C-2 of its single-matrix order);
// the queue interleaves the blocks phase by phase: segment s (ordered by seg_start) holds the
// tickets of block seg_blk[s] from its local ticket seg_l0[s] on, its iteration seg_k[s] (-1 for
// the prefix).  A block's own tickets keep their order and blocks share no dependency, so every
// dependency still precedes its dependants, and the blocks' chains run side by side instead of
// one block at a time.  nblk = 0: one matrix.
struct DagBlocks {
  int nblk = 0, nseg = 0;
  const int *off = nullptr, *mb = nullptr;
  const int64_t *soff = nullptr, *loff = nullptr;
  const int64_t *seg_start = nullptr, *seg_l0 = nullptr;  // nseg + 1 / nseg
  const int *seg_blk = nullptr, *seg_k = nullptr;          // nseg
};

// the segment of block-queue ticket t: the last one starting at or before it
__device__ __host__ __forceinline__ int dag_block_segment(int64_t t, const int64_t *seg_start,
                                                          int nseg) {
  int lo = 0, hi = nseg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (seg_start[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <class T>
__global__ void __launch_bounds__(DAG_THREADS, DAG_CTAS_PER_SM)
    k_chol_dag(T *B0, int64_t ldb, int m, int rows, int *status, T *Linv0, DagSync q,
               int64_t total, DagBlocks bl) {
  extern __shared__ __align__(16) unsigned char smd_raw[];
  T *sm = reinterpret_cast<T *>(smd_raw);
  __shared__ int s_task[3];  // [0] first ticket, [1] next ticket, [2] dependencies met
  const int tid = threadIdx.x;
  T *B = B0, *Linv_all = Linv0;
  int R = (rows + NB - 1) / NB, C = q.C;
  DagPrefix pf = dag_prefix(R, C);
  int kcur = 0;
  int64_t kstart = pf.pre;  // first ticket of iteration kcur
  int blk = -1;
  int *const upd0 = q.upd;
  if (tid == 0) s_task[0] = atomicAdd(q.ticket, 1);
  __syncthreads();
  int t = s_task[0];
  while (t < total) {
    if (tid == 0) s_task[1] = atomicAdd(q.ticket, 1);  // the next ticket, fetched early
    int64_t tl = t;
    if (bl.nblk > 0) {  // block mode: the segment holding t, its block and local ticket
      const int lo = dag_block_segment(t, bl.seg_start, bl.nseg);
      if (bl.seg_blk[lo] != blk) {
        blk = bl.seg_blk[lo];
        const int o = bl.off[blk];
        m = bl.mb[blk];
        rows = m + 1;
        B = B0 + o + (int64_t)o * ldb;
        Linv_all = Linv0 + bl.loff[blk];
        R = (rows + NB - 1) / NB;
        C = (m + NB - 1) / NB;
        q.C = C;
        q.upd = upd0 + bl.soff[blk];
        q.fin = q.upd + (int64_t)R * C;
        pf = dag_prefix(R, C);
      }
      tl = bl.seg_l0[lo] + (t - bl.seg_start[lo]);
      if (bl.seg_k[lo] >= 0) {  // dag_decode's search starts at the segment's iteration
        kcur = bl.seg_k[lo];
        kstart = bl.seg_l0[lo];
      }
    }
    const DagTask task = dag_decode(tl, R, C, pf, kcur, kstart);
    const int type = task.type, ti = task.i, tj = task.j, tk = task.k;
    // dependencies (thread 0 waits, the CTA follows)
    bool ok = true;
    if (tid == 0) {
      const int C_ = q.C;
      const int *f[3];
      int tg[3], n = 0;
      if (type == 4) {  // TS(p, s): rows of L(p, p-1)
        f[0] = q.fin + (tk - 1) * C_ + (tk - 1); tg[0] = 1;
        f[1] = q.upd + tk * C_ + (tk - 1); tg[1] = tk - 1;
        n = 2;
      } else if (type == 5) {  // UD(p, s): rows of the diagonal tile's update by panel p-1
        f[0] = q.fin + tk * C_ + (tk - 1); tg[0] = DAG_TS;
        f[1] = q.upd + tk * C_ + tk; tg[1] = tk - 1;
        n = 2;
      } else if (type == 3) {  // NEXT(p) = POTRF(p): every UD(p, .) done
        f[0] = q.upd + tk * C_ + tk; tg[0] = tk - 1 + DAG_TS;
        n = 1;
      } else if (type == 1) {
        f[0] = q.fin + tk * C_ + tk; tg[0] = 1;
        f[1] = q.upd + ti * C_ + tk; tg[1] = tk;
        n = 2;
      } else if (type == 2) {
        f[0] = q.fin + ti * C_ + tk; tg[0] = dag_fin_target(ti, tk, C_);
        f[1] = q.fin + tj * C_ + tk; tg[1] = dag_fin_target(tj, tk, C_);
        f[2] = q.upd + ti * C_ + tj; tg[2] = tk;
        n = 3;
      }  // type 0, POTRF(0): nothing before it
      ok = n == 0 || dag_wait_all(f, tg, n, q, status);
      const unsigned sid = sm_id() % DAG_MAX_SM;
      if (ok && (type == 0 || type == 3 || type == 4 || type == 5)) {  // the chain's tasks
        atomicExch(q.smbusy + sid, 1);
      } else if (ok && (type == 1 || type == 2)) {
        const long long y0 = clock64();
        while (ld_acquire(q.smbusy + sid) != 0 && clock64() - y0 < DAG_YIELD_CYCLES)
          __nanosleep(128);
      }
      s_task[2] = ok ? 1 : 0;
    }
    __syncthreads();
    if (!s_task[2]) break;
    const int k0 = tk * NB, nb = min(NB, m - k0);
    if (type == 4) {
      const int i0 = k0 + 4 * tj, h = max(0, min(4, min(rows, k0 + NB) - i0));
      dag_trsm4<T>(B, ldb, i0, h, k0 - NB, m, Linv_all + (int64_t)(tk - 1) * NB * NB, sm);
    } else if (type == 5) {
      const int r0 = 4 * tj, h = max(0, min(4, min(rows, k0 + NB) - k0 - r0));
      dag_upd4<T>(B, ldb, k0, r0, h, nb, sm);
    } else if (type == 0 || type == 3) {
      T *Lk = Linv_all + (int64_t)tk * NB * NB;
      potrf_block<T, true>(B, ldb, k0, nb, status, Lk, *reinterpret_cast<PotrfSmem<T> *>(sm));
      // when m is not a multiple of NB the last diagonal tile's row block also holds the
      // right-hand-side row m: solve it here (no TRSM task covers rows of a diagonal tile)
      const int r0 = k0 + nb, r1 = min(rows, k0 + NB);
      if (r0 < r1) {
        __syncthreads();  // Lk stored by this CTA
        dag_trsm<T>(B, ldb, r0, r1 - r0, k0, nb, m, Lk, sm);
      }
    } else if (type == 1) {
      const int i0 = ti * NB;
      dag_trsm<T>(B, ldb, i0, min(NB, rows - i0), k0, nb, m, Linv_all + (int64_t)tk * NB * NB,
                  sm);
    } else {
      const int i0 = ti * NB, j0 = tj * NB;
      dag_upd<T>(B, ldb, i0, min(NB, rows - i0), j0, min(NB, m - j0), k0, nb, ti == tj, sm);
    }
    __syncthreads();  // every store of the task issued; the next ticket visible
    if (tid == 0) {
      if (type == 0 || type >= 3) atomicExch(q.smbusy + sm_id() % DAG_MAX_SM, 0);
      __threadfence();
      if (type == 2) atomicAdd(q.upd + ti * q.C + tj, 1);
      else if (type == 5) atomicAdd(q.upd + tk * q.C + tk, 1);        // one of DAG_TS on (p, p)
      else if (type == 4) atomicAdd(q.fin + tk * q.C + (tk - 1), 1);  // one of DAG_TS
      else atomicAdd(q.fin + ti * q.C + tk, 1);  // POTRF / NEXT: fin[p][p]; TRSM: fin[i][k]
    }
    t = s_task[1];
    __syncthreads();  // s_task reused by the next iteration
  }
}

// words of the task queue's synchronisation buffer for an m-column factorisation of rows rows
size_t chol_dag_words(int m, int rows) {
  const size_t R = (size_t)(rows + NB - 1) / NB, C = (size_t)(m + NB - 1) / NB;
  return 8 + 2 * R * C + DAG_MAX_SM;
}

template <class T>
static int dense_chol_dag(T *B, int64_t ldb, int m, int rows, int *status, T *Linv_all,
                          cudaStream_t st, int *sync, long long budget) {
  const int R = (rows + NB - 1) / NB, C = (m + NB - 1) / NB;
  const int64_t total = dag_total(R, C);
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 1;
  }
  const size_t smem = std::max(sizeof(PotrfSmem<T>), (size_t)2 * NB * (NB + 1) * sizeof(T));
  cudaMemsetAsync(sync, 0, chol_dag_words(m, rows) * sizeof(int), st);
  DagSync q{sync, sync + 1, sync + 8, sync + 8 + (size_t)R * C, sync + 8 + 2 * (size_t)R * C, C,
            budget > 0 ? budget : DAG_DEFAULT_BUDGET};
  // DAG_CTAS_PER_SM CTAs per SM.  A small matrix (C tile columns) never has more than about
  // C^2 / 4 tasks ready at once, so its grid stops there: the CTAs it would not use would hold
  // registers that concurrent solves (mcsdp_solve_batch) need
  const int64_t useful = std::max<int64_t>(8, (int64_t)C * C / 4);
  const int grid = (int)std::min<int64_t>(std::min<int64_t>(DAG_CTAS_PER_SM * (int64_t)nsm, useful), total);
  k_chol_dag<T><<<grid, DAG_THREADS, smem, st>>>(B, ldb, m, rows, status, Linv_all, q, total,
                                                  DagBlocks{});
  return 1;  // kernel launches (the memset is not one of ours)
}

void chol_dag_block_plan(const std::vector<int> &mb, DagBlockPlan &pl) {
  const int nblk = (int)mb.size();
  pl = DagBlockPlan{};
  std::vector<std::vector<int64_t>> ph(nblk);  // per block: prefix, iteration 0, 1, ...
  size_t nph = 0;
  for (int b = 0; b < nblk; ++b) {
    const int R = (mb[b] + 1 + NB - 1) / NB, C = (mb[b] + NB - 1) / NB;
    pl.soff.push_back((int64_t)pl.tile_words);
    pl.tile_words += 2 * (size_t)R * C;
    pl.useful_ctas += (int64_t)C * C / 4;
    ph[b].assign(1, dag_prefix(R, C).pre);
    for (int64_t k = 0; k + 1 < C; ++k) ph[b].push_back(dag_iter_size(k, R, C));
    nph = std::max(nph, ph[b].size());
  }
  std::vector<int64_t> local(nblk, 0);
  for (size_t p = 0; p < nph; ++p)
    for (int b = 0; b < nblk; ++b) {
      if (p >= ph[b].size() || ph[b][p] == 0) continue;
      pl.seg_start.push_back(pl.total);
      pl.seg_l0.push_back(local[b]);
      pl.seg_blk.push_back(b);
      pl.seg_k.push_back((int)p - 1);
      pl.total += ph[b][p];
      local[b] += ph[b][p];
    }
  pl.seg_start.push_back(pl.total);
  pl.words = chol_dag_blocks_words(pl.tile_words);
}

size_t chol_dag_blocks_words(size_t tile_words) { return 8 + tile_words + DAG_MAX_SM; }

int dense_chol_dag_blocks(double *B, int64_t ldb, const DagBlockTables &bt, int *status,
                          double *Linv_all, cudaStream_t st, int *sync, long long budget) {
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 1;
  }
  const size_t smem = std::max(sizeof(PotrfSmem<double>), (size_t)2 * NB * (NB + 1) * sizeof(double));
  cudaMemsetAsync(sync, 0, bt.words * sizeof(int), st);
  DagSync q{sync, sync + 1, sync + 8, nullptr, sync + 8 + bt.tile_words, 0,
            budget > 0 ? budget : DAG_DEFAULT_BUDGET};
  DagBlocks bl;
  bl.nblk = bt.nblk;
  bl.nseg = bt.nseg;
  bl.off = bt.off;
  bl.mb = bt.mb;
  bl.soff = bt.soff;
  bl.loff = bt.loff;
  bl.seg_start = bt.seg_start;
  bl.seg_l0 = bt.seg_l0;
  bl.seg_blk = bt.seg_blk;
  bl.seg_k = bt.seg_k;
  const int64_t useful = std::max<int64_t>(8, bt.useful_ctas);
  const int grid = (int)std::min<int64_t>(std::min<int64_t>(DAG_CTAS_PER_SM * (int64_t)nsm, useful), bt.total);
  k_chol_dag<double><<<grid, DAG_THREADS, smem, st>>>(B, ldb, 0, 0, status, Linv_all, q, bt.total,
                                                      bl);
  return 1;
}

template <class T>
static int dense_chol(T *B, int64_t ldb, int m, int rows, int *status, T *Linv_all,
                      cudaStream_t st_caller, const CholStreams *cs);

__global__ void k_or_status(int *status, int bits) { atomicOr(status, bits); }
// a host-side failure inside a launch sequence (a tensor map that could not be made): reported
// through the status word like a device failure
static void atomic_status_host_fail(int *status, cudaStream_t st) {
  k_or_status<<<1, 1, 0, st>>>(status, ST_NUMERIC);
}

// FP32 Cholesky of an m x m matrix with the trailing updates on the tensor cores: panels of
// TC_PANEL columns, each factored by the 32-column kernels below (over all its rows), its rows
// below the panel split into TF32 hi / lo K-major copies (and written transposed above the
// diagonal, where the refinement's substitutions read L^T), then the trailing lower triangle
// updated by the tcgen05 product C -= P P^T with K = the panel width.
// One panel of the tensor-core Cholesky: the leading pw columns of the rows x pw block Bp, in
// sub-panels of TC_SUB columns: each factored by the 32-column kernels (its rows below solved),
// the panel's columns right of it then updated on the tensor cores (C -= L_s L_s^T over the rows
// from the next sub-panel down, K = TC_SUB), so the 32-column kernels' FFMA updates stay inside a
// sub-panel.  The sub-panel's split also writes its rows transposed above the diagonal.
static int panel_chol_tc(float *Bp, int64_t ldb, int pw, int rows, int *status, float *Linv,
                         cudaStream_t st, const CholStreams *cs, float *sub_hi, float *sub_lo) {
  constexpr int TC_SUB = 128;
  int nl = 0;
  for (int s0 = 0; s0 < pw; s0 += TC_SUB) {
    const int sw = std::min(TC_SUB, pw - s0);
    nl += dense_chol<float>(Bp + s0 + (int64_t)s0 * ldb, ldb, sw, rows - s0, status,
                            Linv + (int64_t)(s0 / NB) * NB * NB, st, nullptr);
    const int r0 = s0 + sw;
    if (r0 >= pw) break;
    split_tf32(Bp + r0 + (int64_t)s0 * ldb, 1, ldb, rows - r0, sw, sub_hi, sub_lo, TC_SUB,
               Bp + s0 + (int64_t)r0 * ldb, ldb, st);
    TcOperand Oa, Ob;
    Oa.x = Oa.y = Ob.x = Ob.y = 0;
    if (!make_tmap_kmajor(&Oa.hi, sub_hi, TC_SUB, sw, rows - r0) ||
        !make_tmap_kmajor(&Oa.lo, sub_lo, TC_SUB, sw, rows - r0) ||
        !make_tmap_kmajor(&Ob.hi, sub_hi, TC_SUB, sw, pw - r0) ||
        !make_tmap_kmajor(&Ob.lo, sub_lo, TC_SUB, sw, pw - r0)) {
      atomic_status_host_fail(status, st);
      return nl;
    }
    gemm_3xtf32(Oa, Ob, rows - r0, pw - r0, sw, Bp + r0 + (int64_t)r0 * ldb, 1, ldb, -1.f, 1.f,
                true, false, cs->tc_err ? cs->tc_err : status, st);
    nl += 2;
  }
  return nl;
}

// The tensor-core FP32 Cholesky, right-looking by panels of P columns with lookahead of one
// panel.  On st (the chain): F(k) factors panel k (panel_chol_tc), S(k) splits its rows below
// into buffer k % 2 (and writes them transposed above the diagonal), N(k) updates panel k + 1's
// columns.  On cs->rest: R(k) updates every column beyond panel k + 1, so the chain's
// F(k + 1), S(k + 1) overlap R(k).  Order: F(k) and S(k) after R(k - 2) (it updates panel k and
// read buffer k % 2), N(k) after R(k - 1) (both update panel k + 1), R(k) after S(k).
static int dense_chol_f32_tc(float *B, int64_t ldb, int m, int *status, float *Linv_all,
                             cudaStream_t st, const CholStreams *cs) {
  int nl = 0;
  const int P = tc_panel(m);
  const int np = (m + P - 1) / P;
  const int64_t bufsz = (int64_t)P * m;
  cudaStream_t rs = cs->rest;
  int *err = cs->tc_err ? cs->tc_err : status;
  cudaEventRecord(cs->fork, st);
  cudaStreamWaitEvent(rs, cs->fork, 0);
  for (int k = 0; k < np; ++k) {
    const int k0 = k * P, pw = std::min(P, m - k0), r0 = k0 + pw;
    float *hi = cs->tc_hi + (k & 1) * bufsz, *lo = cs->tc_lo + (k & 1) * bufsz;
    if (k >= 2) cudaStreamWaitEvent(st, cs->rest_ev[k & 1], 0);  // R(k - 2) done
    nl += panel_chol_tc(B + k0 + (int64_t)k0 * ldb, ldb, pw, m - k0, status,
                        Linv_all + (int64_t)(k0 / NB) * NB * NB, st, cs, hi, lo);
    if (r0 >= m) break;
    split_tf32(B + r0 + (int64_t)k0 * ldb, 1, ldb, m - r0, pw, hi, lo, P, B + k0 + (int64_t)r0 * ldb,
               ldb, st);
    cudaEventRecord(cs->next[k & 1], st);  // S(k) done
    const int pn = std::min(P, m - r0);    // width of panel k + 1
    TcOperand Oa, Ob;
    Oa.x = Oa.y = Ob.x = Ob.y = 0;
    if (!make_tmap_kmajor(&Oa.hi, hi, P, pw, m - r0) || !make_tmap_kmajor(&Oa.lo, lo, P, pw, m - r0) ||
        !make_tmap_kmajor(&Ob.hi, hi, P, pw, pn) || !make_tmap_kmajor(&Ob.lo, lo, P, pw, pn)) {
      atomic_status_host_fail(status, st);
      break;
    }
    // N(k): panel k + 1's columns, every row from r0 down
    if (k >= 1) cudaStreamWaitEvent(st, cs->rest_ev[(k - 1) & 1], 0);  // R(k - 1) done
    gemm_3xtf32(Oa, Ob, m - r0, pn, pw, B + r0 + (int64_t)r0 * ldb, 1, ldb, -1.f, 1.f, true, false,
                err, st);
    nl += 2;
    // R(k): the columns beyond panel k + 1, rows from r2 down (buffer rows from r2 - r0)
    const int r2 = r0 + pn;
    if (r2 < m) {
      TcOperand Oc;
      Oc.x = Oc.y = 0;
      const int64_t off = (int64_t)(r2 - r0) * P;
      if (!make_tmap_kmajor(&Oc.hi, hi + off, P, pw, m - r2) ||
          !make_tmap_kmajor(&Oc.lo, lo + off, P, pw, m - r2)) {
        atomic_status_host_fail(status, st);
        break;
      }
      cudaStreamWaitEvent(rs, cs->next[k & 1], 0);
      gemm_3xtf32(Oc, Oc, m - r2, m - r2, pw, B + r2 + (int64_t)r2 * ldb, 1, ldb, -1.f, 1.f, true,
                  false, err, rs);
      ++nl;
    }
    cudaEventRecord(cs->rest_ev[k & 1], rs);
  }
  cudaEventRecord(cs->chain_done, rs);
  cudaStreamWaitEvent(st, cs->chain_done, 0);
  return nl;
}

// Right-looking blocked Cholesky of the leading m columns of a rows x m matrix (rows = m + 1 for
// the bordered right-hand side, m otherwise) with lookahead: on st (the critical path) panel k is factored (potrf), its rows below are solved
// (trsm) and its update is applied to block column k+1; the rest of its update (block columns
// >= k+2) runs on st2, overlapping the next panel's factor-and-solve.  ev_next[k%2] /
// ev_rest[k%2] order the two streams so no block is updated by both at once; st waits for st2
// at the end.  With st2 == nullptr everything runs on st.
template <class T>
static int dense_chol(T *B, int64_t ldb, int m, int rows, int *status, T *Linv_all,
                      cudaStream_t st_caller, const CholStreams *cs) {
  if constexpr (std::is_same<T, float>::value) {
    if (cs && cs->tc_hi && rows == m && m >= 2 * TC_PANEL && m <= cs->tc_rows)
      return dense_chol_f32_tc(B, ldb, m, status, Linv_all, st_caller, cs);
  }
  // critical path on st (high priority), trailing updates on st2 (low priority)
  const bool la = cs != nullptr;
  cudaStream_t st = la ? cs->chain : st_caller, st2 = la ? cs->rest : nullptr;
  const cudaEvent_t *ev_next = la ? cs->next : nullptr, *ev_rest = la ? cs->rest_ev : nullptr;
  if (la) {
    cudaEventRecord(cs->fork, st_caller);
    cudaStreamWaitEvent(st, cs->fork, 0);
    cudaStreamWaitEvent(st2, cs->fork, 0);
  }
  const int smem_tile = 2 * NB * TS * (int)sizeof(T);
  smem_optin((const void *)k_syrk_tiles<T>);
  int launches = 0;
  for (int k0 = 0, k = 0; k0 < m; k0 += NB, ++k) {
    const int nb = (m - k0) < NB ? (m - k0) : NB;
    T *Linv = Linv_all + (int64_t)k * NB * NB;
    if constexpr (std::is_same<T, float>::value)
      k_potrf_warp_f32<<<1, 32, 0, st>>>(B, ldb, k0, nb, status, Linv);
    else
      k_potrf_diag<T><<<1, 256, 0, st>>>(B, ldb, k0, nb, status, Linv);
    ++launches;
    const int r0 = k0 + nb;
    const int nr = rows - r0;
    if (nr <= 0) continue;
    k_trsm_panel<T><<<(nr + TRSM_ROWS - 1) / TRSM_ROWS, TRSM_ROWS * 32, 0, st>>>(B, ldb, k0, nb, r0, rows, m, Linv);
    ++launches;
    const int c_next = r0 + NB < m ? r0 + NB : m;  // block column k+1 = [r0, c_next)
    if (!la) {
      launch_syrk<T>(B, ldb, k0, nb, r0, m, rows, smem_tile, st);
      ++launches;
      continue;
    }
    if (k >= 1) cudaStreamWaitEvent(st, ev_rest[(k - 1) & 1], 0);  // st2 finished panel k-1
    k_syrk_next<T><<<(nr + TRSM_ROWS - 1) / TRSM_ROWS, TRSM_ROWS * 32, 0, st>>>(B, ldb, k0, nb, r0, c_next, rows);
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
    cudaEventRecord(cs->rest_ev[0], st2);
    cudaEventRecord(cs->chain_done, st);
    cudaStreamWaitEvent(st_caller, cs->rest_ev[0], 0);
    cudaStreamWaitEvent(st_caller, cs->chain_done, 0);
  }
  return launches;
}

// the factorisation through the graph cache of cs: the first call for a (type, matrix, size)
// runs eagerly (it also sets the kernels' shared-memory attributes), the second captures the
// sequence into a graph, every later one replays it
template <class T>
static int dense_chol_graph(T *B, int64_t ldb, int m, int rows, int *status, T *Linv,
                            cudaStream_t st, CholStreams *cs);

// runs on the chain stream (created by the library, so capturable whatever the caller's stream
// is), ordered after and joined back into the caller's stream
template <class T>
static int dense_chol_cached(T *B, int64_t ldb, int m, int rows, int *status, T *Linv,
                             cudaStream_t st_caller, CholStreams *cs) {
  if (!cs) return dense_chol<T>(B, ldb, m, rows, status, Linv, st_caller, nullptr);
  // FP64: the task queue.  FP32 keeps the launch per panel (graph-captured): its tiles take a
  // fraction of a microsecond, so the queue's per-task overheads dominate (measured slower).
  if constexpr (std::is_same<T, double>::value) {
    if (cs->dag_sync && cs->dag_words >= chol_dag_words(m, rows))
      return dense_chol_dag<T>(B, ldb, m, rows, status, Linv, st_caller, cs->dag_sync,
                               cs->dag_budget);
  }
  cudaEventRecord(cs->entry, st_caller);
  cudaStreamWaitEvent(cs->chain, cs->entry, 0);
  const int nl = dense_chol_graph<T>(B, ldb, m, rows, status, Linv, cs->chain, cs);
  cudaEventRecord(cs->exit, cs->chain);
  cudaStreamWaitEvent(st_caller, cs->exit, 0);
  return nl;
}

template <class T>
static int dense_chol_graph(T *B, int64_t ldb, int m, int rows, int *status, T *Linv,
                            cudaStream_t st, CholStreams *cs) {
  CholGraph *g = nullptr, *freeg = nullptr;
  for (CholGraph &x : cs->graphs) {
    if (x.B == B && x.Linv == Linv && x.status == status && x.ldb == ldb && x.m == m &&
        x.rows == rows && x.esize == (int)sizeof(T))
      g = &x;
    else if (!x.B && !freeg)
      freeg = &x;
  }
  if (!g && freeg) {
    g = freeg;
    g->B = B;
    g->Linv = Linv;
    g->status = status;
    g->ldb = ldb;
    g->m = m;
    g->rows = rows;
    g->esize = (int)sizeof(T);
  }
  if (!g || g->runs <= 0) {  // no slot left, first use, or capture unavailable: eager
    if (g && g->runs == 0) g->runs = 1;
    return dense_chol<T>(B, ldb, m, rows, status, Linv, st, cs);
  }
  if (!g->exec) {
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      (void)cudaGetLastError();
      g->runs = -1;
      return dense_chol<T>(B, ldb, m, rows, status, Linv, st, cs);
    }
    const int nl = dense_chol<T>(B, ldb, m, rows, status, Linv, st, cs);
    if (cudaStreamEndCapture(st, &graph) != cudaSuccess || !graph) {
      (void)cudaGetLastError();
      g->runs = -1;
      return dense_chol<T>(B, ldb, m, rows, status, Linv, st, cs);
    }
    // node priorities from the capturing streams: the chain's kernels go ahead of the trailing
    // updates when both wait for an SM
    if (cudaGraphInstantiate(&g->exec, graph, cudaGraphInstantiateFlagUseNodePriority) != cudaSuccess) {
      (void)cudaGetLastError();
      g->exec = nullptr;
    }
    cudaGraphDestroy(graph);
    if (!g->exec) {
      g->runs = -1;
      return dense_chol<T>(B, ldb, m, rows, status, Linv, st, cs);
    }
    g->kernels = nl;
  }
  cudaGraphLaunch(g->exec, st);
  return g->kernels;  // kernels launched (as graph nodes)
}

void chol_graphs_destroy(CholStreams *cs) {
  for (CholGraph &x : cs->graphs) {
    if (x.exec) cudaGraphExecDestroy(x.exec);
    x = CholGraph{};
  }
}

int dense_potrf(double *A, int64_t ld, int n, int *status, double *Linv, cudaStream_t st, int *sync,
                long long budget) {
  return dense_chol_dag<double>(A, ld, n, n, status, Linv, st, sync, budget);
}

int dense_chol_bordered(double *B, int64_t ldb, int m, int *status, double *Linv_all,
                        cudaStream_t st, CholStreams *cs) {
  return dense_chol_cached<double>(B, ldb, m, m + 1, status, Linv_all, st, cs);
}

int dense_chol_f32(float *B, int64_t ldb, int m, int *status, float *Linv_all, cudaStream_t st,
                   CholStreams *cs) {
  return dense_chol_cached<float>(B, ldb, m, m, status, Linv_all, st, cs);
}

// Backward substitution L^T x = y, y = row m of B, blocks of NB (32) from the bottom; the diagonal
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

// Backward substitution L^T x = y (y = row m of B) by one cluster of BCL CTAs: row block kb
// belongs to CTA kb % BCL, which keeps those entries of the vector in shared memory.  Step kb
// (from the last block): the owner forms x_kb = Linv_kb^T y_kb and writes it into every CTA's
// shared memory, one cluster barrier, then each CTA removes L_{kb,i} x_kb from its own rows i
// above the block, reading L^T from the strict upper triangle, where the factorisation stored
// it (coalesced).  The factor entries of a step are loaded before its barrier.  Per step: one
// hardware cluster barrier.
constexpr int BCL = 8;
constexpr int BTH = 256;
// Block mode (boff != nullptr): cluster b solves the diagonal block b of a block-diagonal B (rows
// and columns from boff[b], bm[b] of them, right-hand side in the row after the block, inverses
// at Linv + bloff[b]) into x + boff[b].
__global__ void __cluster_dims__(BCL, 1, 1) __launch_bounds__(BTH)
    k_backsolve_cluster(const double *__restrict__ B, int64_t ldb, int m,
                        const double *__restrict__ Linv, double *x, const int *__restrict__ boff,
                        const int *__restrict__ bm, const int64_t *__restrict__ bloff) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  if (boff) {
    const int b = blockIdx.x / BCL, o = boff[b];
    m = bm[b];
    B += o + (int64_t)o * ldb;
    Linv += bloff[b];
    x += o;
  }
  extern __shared__ double yv[];  // m doubles; the CTA's own rows are used
  __shared__ double xb[2][NB];
  __shared__ double tb[NB];
  const int rank = (int)cl.block_rank();
  const int tid = threadIdx.x;
  const int nblk = (m + NB - 1) / NB;
  for (int i = tid; i < m; i += BTH)
    if ((i / NB) % BCL == rank) yv[i] = B[m + (int64_t)i * ldb];
  __syncthreads();
  int step = 0;
  for (int kb = nblk - 1; kb >= 0; --kb, ++step) {
    const int b0 = kb * NB, nb = min(NB, m - b0), buf = step & 1;
    const int nown = rank < kb ? (kb - 1 - rank) / BCL + 1 : 0;
    double lv[NB];
    int i0 = -1;
    if (tid < nown * NB) {
      i0 = (rank + (tid / NB) * BCL) * NB + tid % NB;
#pragma unroll
      for (int l = 0; l < NB; ++l) lv[l] = (l < nb) ? B[i0 + (int64_t)(b0 + l) * ldb] : 0.0;
    }
    if (kb % BCL == rank) {
      // x_kb = Linv_kb^T y_kb: eight threads per output, four terms each, summed by shuffles
      // (Linv is zero above the diagonal and past nb)
      const double *Li = Linv + (int64_t)kb * NB * NB;
      const int o = tid >> 3, l0 = (tid & 7) * 4;
      double a = 0.0;
#pragma unroll
      for (int q = 0; q < 4; ++q)
        a = fma(Li[l0 + q + o * NB], l0 + q < nb ? yv[b0 + l0 + q] : 0.0, a);
      a += __shfl_xor_sync(0xffffffffu, a, 1);
      a += __shfl_xor_sync(0xffffffffu, a, 2);
      a += __shfl_xor_sync(0xffffffffu, a, 4);
      if ((tid & 7) == 0) tb[o] = a;
      __syncthreads();
      if (tid < NB) {
        const double v = tid < nb ? tb[tid] : 0.0;
        if (tid < nb) yv[b0 + tid] = v;
        for (int q = 0; q < BCL; ++q) cl.map_shared_rank(&xb[buf][0], q)[tid] = v;
      }
    }
    cl.sync();
    if (i0 >= 0) {
      double a0 = 0.0, a1 = 0.0;
#pragma unroll
      for (int l = 0; l < NB; l += 2) {
        a0 = fma(lv[l], xb[buf][l], a0);
        a1 = fma(lv[l + 1], xb[buf][l + 1], a1);
      }
      yv[i0] -= a0 + a1;
    }
    for (int slot = tid + BTH; slot < nown * NB; slot += BTH) {
      const int i = (rank + (slot / NB) * BCL) * NB + slot % NB;
      double a = 0.0;
      for (int l = 0; l < nb; ++l) a = fma(B[i + (int64_t)(b0 + l) * ldb], xb[buf][l], a);
      yv[i] -= a;
    }
    __syncthreads();
  }
  for (int i = tid; i < m; i += BTH)
    if ((i / NB) % BCL == rank) x[i] = yv[i];
  cl.sync();  // no CTA leaves while another may still write into its shared memory
}

constexpr int BS_CLUSTER_MAX_M = 24 * 1024;  // the vector must fit the shared memory of a CTA

int dense_backsolve(const double *B, int64_t ldb, int m, const double *Linv_all, double *x,
                    cudaStream_t st) {
  if (m <= BS_CLUSTER_MAX_M) {
    const size_t smem = (size_t)m * sizeof(double);
    if (smem > 48 * 1024) smem_optin((const void *)k_backsolve_cluster);
    k_backsolve_cluster<<<BCL, BTH, smem, st>>>(B, ldb, m, Linv_all, x, nullptr, nullptr, nullptr);
    return 1;
  }
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

int dense_backsolve_blocks(const double *B, int64_t ldb, const DagBlockTables &bt,
                           const double *Linv_all, double *x, cudaStream_t st) {
  if (bt.max_m > BS_CLUSTER_MAX_M) return -1;
  const size_t smem = (size_t)bt.max_m * sizeof(double);
  if (smem > 48 * 1024) smem_optin((const void *)k_backsolve_cluster);
  k_backsolve_cluster<<<BCL * bt.nblk, BTH, smem, st>>>(B, ldb, 0, Linv_all, x, bt.off, bt.mb,
                                                        bt.loff);
  return 1;
}

// row m of B <- g_i = b_{user(i)} - beta mu h_i   (internal order; with a block-diagonal B, row
// S.bord[i], the row after i's diagonal block)
__global__ void k_rhs_border(DevSym S, double *B, int64_t ldb, const double *hvec, double betamu,
                             const double *__restrict__ betamu_dev) {
  if (betamu_dev) betamu = *betamu_dev;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S.m; i += gridDim.x * blockDim.x)
    B[(S.bord ? S.bord[i] : S.m) + (int64_t)i * ldb] = S.b[S.con_order[i]] - betamu * hvec[i];
}

void launch_rhs_border(const DevSym &S, double *B, int64_t ldb, const double *hvec, double betamu,
                       cudaStream_t st, const double *betamu_dev) {
  k_rhs_border<<<(S.m + 255) / 256, 256, 0, st>>>(S, B, ldb, hvec, betamu, betamu_dev);
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
    // a block-diagonal B stores nothing between components (those entries are zero; the
    // right-hand side of a block may sit there)
    const bool cross = S.bord && S.bord[i] != S.bord[j];
    Bo[r + (int64_t)c * ldo] = cross ? 0.0 : Bi[i + (int64_t)j * ldi];
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
// Preparation, 32 x 32 tiles of the lower triangle (tile row ti >= tile column tj): B32 <- the
// tile rounded to FP32 (ld m), and the FP64 B made fully symmetric (the tile's transpose written
// into the strict upper triangle, staged through shared memory so both sides are coalesced), so
// the refinement's matrix-vector product is a plain column-major product.
__global__ void k_mixed_prep(double *B, int64_t ldb, float *B32, int m,
                             const double *__restrict__ dsc, double shift) {
  __shared__ double t[32][33];
  const int ti = blockIdx.x, tj = blockIdx.y;
  if (ti < tj) return;
  const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;  // 256 threads: 32 x 8
  const int i0 = ti * 32, j0 = tj * 32;
  for (int c = ly; c < 32; c += 8) {
    const int i = i0 + lx, j = j0 + c;
    double v = 0.0;
    if (i < m && j < m && i >= j) {
      v = B[i + (int64_t)j * ldb];
      B32[i + (int64_t)j * m] = (float)((dsc ? v * dsc[i] * dsc[j] : v) + (i == j ? shift : 0.0));
    }
    t[lx][c] = v;
  }
  __syncthreads();
  // transposed write: B[j][i] for i > j, i.e. row j0+lx... column i0+c
  for (int c = ly; c < 32; c += 8) {
    const int j = j0 + lx, i = i0 + c;
    if (i < m && j < m && i > j) B[j + (int64_t)i * ldb] = t[c][lx];
  }
}

// x += L^{-T} L^{-1} r with the FP32 factor (ld m; L^T in the strict upper triangle) and the
// inverses of its NB x NB diagonal blocks.  One cluster of RCL CTAs: row block kb belongs to CTA
// kb % RCL, which keeps those rows of the vector in its shared memory.  Step kb of the forward
// substitution: the owner forms y_kb = Linv_kb (rows kb) and writes it into every CTA's shared
// memory (distributed shared memory), one cluster barrier, then every CTA removes L_{i,kb} y_kb
// from its own rows i below the block.  The backward substitution runs the same way from the
// last block with L^T.  Each thread loads the factor entries of its next update before the
// barrier, so their latency overlaps the owner's step.  Per step: one hardware cluster barrier
// (no spin loop).
constexpr int RCL = 8;
constexpr int RTH = 256;
__global__ void __cluster_dims__(RCL, 1, 1) __launch_bounds__(RTH)
    k_refine_solve_f32(const float *__restrict__ L, int m, const float *__restrict__ Linv,
                       const double *__restrict__ r, double *x) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ float ys[];  // m floats; the CTA's own rows are used
  __shared__ float yb[2][NB];
  __shared__ float tb[NB];
  const int rank = (int)cl.block_rank();
  const int tid = threadIdx.x;
  const int nblk = (m + NB - 1) / NB;
  for (int i = tid; i < m; i += RTH)
    if ((i / NB) % RCL == rank) ys[i] = (float)r[i];
  __syncthreads();
  int step = 0;
  // ---- forward: y = L^{-1} r
  for (int kb = 0; kb < nblk; ++kb, ++step) {
    const int b0 = kb * NB, nb = min(NB, m - b0), buf = step & 1;
    // own row blocks after kb: kb' = first + q * RCL
    const int first = kb + 1 + ((rank - (kb + 1)) % RCL + RCL) % RCL;
    const int nown = first < nblk ? (nblk - 1 - first) / RCL + 1 : 0;
    // prefetch the first slot's factor entries
    const int slot0 = tid;
    float lv[NB];
    int i0 = -1;
    if (slot0 < nown * NB) {
      i0 = (first + (slot0 / NB) * RCL) * NB + slot0 % NB;
      if (i0 < m) {
#pragma unroll
        for (int l = 0; l < NB; ++l) lv[l] = (l < nb) ? L[i0 + (int64_t)(b0 + l) * m] : 0.f;
      } else {
        i0 = -1;
      }
    }
    if (kb % RCL == rank) {
      if (tid < nb) {
        const float *Li = Linv + (int64_t)kb * NB * NB;  // zero above the diagonal
        float a = 0.f;
#pragma unroll
        for (int l = 0; l < NB; ++l) a = fmaf(Li[tid + l * NB], l < nb ? ys[b0 + l] : 0.f, a);
        tb[tid] = a;
      }
      __syncthreads();
      if (tid < NB) {  // the whole block, zero past nb, so the unrolled updates read no stale values
        const float v = tid < nb ? tb[tid] : 0.f;
        if (tid < nb) ys[b0 + tid] = v;
        for (int q = 0; q < RCL; ++q) cl.map_shared_rank(&yb[buf][0], q)[tid] = v;
      }
    }
    cl.sync();
    if (i0 >= 0) {
      float a = 0.f;
#pragma unroll
      for (int l = 0; l < NB; ++l) a = fmaf(lv[l], yb[buf][l], a);
      ys[i0] -= a;
    }
    for (int slot = tid + RTH; slot < nown * NB; slot += RTH) {
      const int i = (first + (slot / NB) * RCL) * NB + slot % NB;
      if (i >= m) continue;
      float a = 0.f;
      for (int l = 0; l < nb; ++l) a = fmaf(L[i + (int64_t)(b0 + l) * m], yb[buf][l], a);
      ys[i] -= a;
    }
    __syncthreads();
  }
  // ---- backward: x = L^{-T} y
  for (int kb = nblk - 1; kb >= 0; --kb, ++step) {
    const int b0 = kb * NB, nb = min(NB, m - b0), buf = step & 1;
    // own row blocks before kb: kb' = q * RCL + rank < kb
    const int nown = rank < kb ? (kb - 1 - rank) / RCL + 1 : 0;
    float lv[NB];
    int i0 = -1;
    if (tid < nown * NB) {
      i0 = (rank + (tid / NB) * RCL) * NB + tid % NB;
#pragma unroll
      for (int l = 0; l < NB; ++l) lv[l] = (l < nb) ? L[i0 + (int64_t)(b0 + l) * m] : 0.f;
    }
    if (kb % RCL == rank) {
      if (tid < nb) {
        const float *Li = Linv + (int64_t)kb * NB * NB;  // zero above the diagonal
        float a = 0.f;
#pragma unroll
        for (int l = 0; l < NB; ++l) a = fmaf(Li[l + tid * NB], l < nb ? ys[b0 + l] : 0.f, a);
        tb[tid] = a;
      }
      __syncthreads();
      if (tid < NB) {  // the whole block, zero past nb, so the unrolled updates read no stale values
        const float v = tid < nb ? tb[tid] : 0.f;
        if (tid < nb) ys[b0 + tid] = v;
        for (int q = 0; q < RCL; ++q) cl.map_shared_rank(&yb[buf][0], q)[tid] = v;
      }
    }
    cl.sync();
    if (i0 >= 0) {
      float a = 0.f;
#pragma unroll
      for (int l = 0; l < NB; ++l) a = fmaf(lv[l], yb[buf][l], a);
      ys[i0] -= a;
    }
    for (int slot = tid + RTH; slot < nown * NB; slot += RTH) {
      const int i = (rank + (slot / NB) * RCL) * NB + slot % NB;
      float a = 0.f;
      for (int l = 0; l < nb; ++l) a = fmaf(L[i + (int64_t)(b0 + l) * m], yb[buf][l], a);
      ys[i] -= a;
    }
    __syncthreads();
  }
  for (int i = tid; i < m; i += RTH)
    if ((i / NB) % RCL == rank) x[i] += (double)ys[i];
  cl.sync();  // no CTA leaves while another may still write into its shared memory
}

// The refinement's substitutions for large m: x += L^{-T} L^{-1} r (FP32 factor, ld m, L^T in the
// strict upper triangle; FP64 r and x), blocked by panels of TP rows so that no kernel waits on
// another CTA.  Forward, per panel [k0, k0 + TP): one CTA of 1024 threads solves the panel's
// triangle (blocks of NB: the block's inverse applied by warp 0, then thread t removes the
// block's part from row k0 + t; the panel's y in shared memory), then every row below the
// panel takes off L[r, panel] y_panel (k_trsv_update: CTA = 32 rows x 8 column phases, every
// load a 128-byte row segment, bandwidth-bound over all SMs).  Backward: panels from the last,
// with L^T read from the upper triangle (the same coalesced row segments), the update going to
// the rows above.  The vector lives in FP32 (y), x is updated in FP64 at the end.
constexpr int TRSV_WIDE_M = 4096;  // from here on the blocked substitutions
constexpr int TP = 1024;

template <bool FWD>
__global__ void __launch_bounds__(TP) k_trsv_panel(const float *__restrict__ L, int m,
                                                   const float *__restrict__ Linv, int k0,
                                                   float *y) {
  static_assert(NB * NB == TP, "one inverse entry per thread");
  __shared__ float ys[TP];
  __shared__ float yb[NB];
  __shared__ float ls[2][NB * (NB + 1)];  // row r of the inverse at r (NB + 1): conflict-free
  const int pw = min(TP, m - k0), t = threadIdx.x, lane = t & 31;
  if (t < pw) ys[t] = y[k0 + t];
  const int nb_tot = (pw + NB - 1) / NB;
  const int row = k0 + t;
  // the NB factor entries of this thread's row in block b (row segments of L below the
  // diagonal, of L^T above it) are loaded one block ahead, so their latency overlaps the barrier
  // and the diagonal step; the block's inverse likewise, one entry per thread into shared memory
  auto first_of = [&](int s) { return FWD ? s : nb_tot - 1 - s; };
  auto needs = [&](int b) {
    const int b0 = b * NB;
    return FWD ? (t >= b0 + min(NB, pw - b0) && t < pw) : (t < b0);
  };
  float lv[NB];
  auto load_row = [&](int b) {
    const int b0 = b * NB, nb = min(NB, pw - b0);
    const bool need = needs(b);
#pragma unroll
    for (int c = 0; c < NB; ++c)
      lv[c] = (need && c < nb) ? L[row + (int64_t)(k0 + b0 + c) * m] : 0.f;
  };
  auto load_inv = [&](int b, int buf) {
    // Linv column-major (entry (r, c) at r + c NB), stored at r + c (NB + 1)
    ls[buf][(t % NB) + (t / NB) * (NB + 1)] = Linv[(int64_t)((k0 + b * NB) / NB) * NB * NB + t];
  };
  load_row(first_of(0));
  load_inv(first_of(0), 0);
  __syncthreads();
  for (int s = 0; s < nb_tot; ++s) {
    const int b = first_of(s);
    const int b0 = b * NB, nb = min(NB, pw - b0);
    if (t < 32) {
      const float *Li = ls[s & 1];
      const float rl = lane < nb ? ys[b0 + lane] : 0.f;
      float v = 0.f;
#pragma unroll
      for (int l = 0; l < NB; ++l)
        v = fmaf(FWD ? Li[lane + l * (NB + 1)] : Li[l + lane * (NB + 1)],
                 __shfl_sync(0xffffffffu, rl, l), v);
      if (lane < nb) ys[b0 + lane] = v;
      yb[lane] = lane < nb ? v : 0.f;
    }
    __syncthreads();
    if (needs(b)) {
      float a = 0.f;
#pragma unroll
      for (int c = 0; c < NB; ++c) a = fmaf(lv[c], yb[c], a);
      ys[t] -= a;
    }
    if (s + 1 < nb_tot) {
      load_row(first_of(s + 1));
      load_inv(first_of(s + 1), (s + 1) & 1);
    }
    __syncthreads();
  }
  if (t < pw) y[k0 + t] = ys[t];
}

// forward: y[r] -= sum_c L[r, k0 + c] y[k0 + c] for the rows r >= k0 + pw; backward: for the rows
// r < k0, with L^T (the upper triangle holds L^T[r][k0 + c] at [r + (k0 + c) m])
template <bool FWD>
__global__ void __launch_bounds__(256) k_trsv_update(const float *__restrict__ L, int m, int k0,
                                                    int pw, const float *ysrc, float *y) {
  __shared__ float part[8][33];
  __shared__ float yp[TP];
  const int il = threadIdx.x & 31, ph = threadIdx.x >> 5;
  for (int c = threadIdx.x; c < pw; c += 256) yp[c] = ysrc[k0 + c];
  __syncthreads();
  const int r = (FWD ? k0 + pw : 0) + blockIdx.x * 32 + il;
  const int rend = FWD ? m : k0;
  float a0 = 0.f, a1 = 0.f;
  if (r < rend) {
    int c = ph;
    for (; c + 8 < pw; c += 16) {
      a0 = fmaf(L[r + (int64_t)(k0 + c) * m], yp[c], a0);
      a1 = fmaf(L[r + (int64_t)(k0 + c + 8) * m], yp[c + 8], a1);
    }
    for (; c < pw; c += 8) a0 = fmaf(L[r + (int64_t)(k0 + c) * m], yp[c], a0);
  }
  part[ph][il] = a0 + a1;
  __syncthreads();
  if (ph == 0 && r < rend) {
    float a = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) a += part[q][il];
    y[r] -= a;
  }
}

// y = S r in FP32, and x += S y in FP64, S = diag(dsc) (the factor's equilibration; none if null)
__global__ void k_trsv_load(const double *__restrict__ r, float *y, int m,
                            const double *__restrict__ dsc) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
    y[i] = (float)(dsc ? r[i] * dsc[i] : r[i]);
}
__global__ void k_trsv_store(const float *__restrict__ y, double *x, int m,
                             const double *__restrict__ dsc) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
    x[i] += dsc ? (double)y[i] * dsc[i] : (double)y[i];
}

static int trsv_blocked(const float *L, int m, const float *Linv, const double *r, double *x,
                        float *y, const double *dsc, cudaStream_t st) {
  const int blocks = std::min(152 * 8, (m + 255) / 256);
  k_trsv_load<<<blocks, 256, 0, st>>>(r, y, m, dsc);
  int nl = 2;
  for (int k0 = 0; k0 < m; k0 += TP) {
    const int pw = std::min(TP, m - k0);
    k_trsv_panel<true><<<1, TP, 0, st>>>(L, m, Linv, k0, y);
    ++nl;
    const int rows = m - k0 - pw;
    if (rows > 0) {
      k_trsv_update<true><<<(rows + 31) / 32, 256, 0, st>>>(L, m, k0, pw, y, y);
      ++nl;
    }
  }
  const int last = ((m - 1) / TP) * TP;
  for (int k0 = last; k0 >= 0; k0 -= TP) {
    k_trsv_panel<false><<<1, TP, 0, st>>>(L, m, Linv, k0, y);
    ++nl;
    if (k0 > 0) {
      k_trsv_update<false><<<(k0 + 31) / 32, 256, 0, st>>>(L, m, k0, std::min(TP, m - k0), y, y);
      ++nl;
    }
  }
  k_trsv_store<<<blocks, 256, 0, st>>>(y, x, m, dsc);
  return nl;
}

// The same substitutions with the inverses T_p of the factor's diagonal blocks of TP rows
// precomputed (trsv_prepare_blocks): each panel is one product with T_p (FWD: T_p y, lower; BWD:
// T_p^T y) instead of a serial chain of 32-row blocks, so a solve is 2 x 2 x (m / TP) launches
// of bandwidth-bound work.  The panel's values are read from src and written to dst (no CTA
// overwrites what another still reads).
template <bool FWD>
__global__ void __launch_bounds__(256) k_trsv_diag(const float *__restrict__ T, int pw,
                                                  const float *__restrict__ src, float *dst) {
  __shared__ float ys[TP];
  __shared__ float part[8][33];
  for (int c = threadIdx.x; c < pw; c += 256) ys[c] = src[c];
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (FWD) {  // CTA = 32 rows x 8 column phases; lanes take consecutive rows of a column of T
    const int r = blockIdx.x * 32 + lane;
    float a = 0.f;
    if (r < pw)
      for (int c = w; c <= r; c += 8) a = fmaf(T[r + (int64_t)c * TP], ys[c], a);
    part[w][lane] = a;
    __syncthreads();
    if (w == 0 && r < pw) {
      float t = 0.f;
#pragma unroll
      for (int q = 0; q < 8; ++q) t += part[q][lane];
      dst[r] = t;
    }
  } else {  // a warp per output r: column r of T (rows c >= r, contiguous), lanes along it
    const int r = blockIdx.x * 8 + w;
    if (r >= pw) return;
    float a = 0.f;
    for (int c = r + lane; c < pw; c += 32) a = fmaf(T[c + (int64_t)r * TP], ys[c], a);
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) dst[r] = a;
  }
}

// T_p = inverse of the factor's diagonal block p (TP x TP, lower; column-major, ld TP, at
// tinv + p TP^2), from the 32 x 32 block inverses; work: 256 (TP + 256) floats
int trsv_prepare_blocks(const float *L, int m, const float *Linv, float *tinv, float *work,
                        cudaStream_t st) {
  int nl = 0;
  for (int k0 = 0, p = 0; k0 < m; k0 += TP, ++p)
    nl += dense_trtri<float>(L + k0 + (int64_t)k0 * m, m, Linv + (int64_t)(k0 / NB) * NB * NB,
                             tinv + (int64_t)p * TP * TP, TP, std::min(TP, m - k0), work, st);
  return nl;
}

static int trsv_blocked_inv(const float *L, int m, const float *tinv, const double *r, double *x,
                            float *ya, float *yb, const double *dsc, cudaStream_t st) {
  const int blocks = std::min(152 * 8, (m + 255) / 256);
  k_trsv_load<<<blocks, 256, 0, st>>>(r, ya, m, dsc);
  int nl = 2;
  const int np = (m + TP - 1) / TP;
  for (int p = 0; p < np; ++p) {  // forward: yb_p = T_p ya_p, then the rows below in ya
    const int k0 = p * TP, pw = std::min(TP, m - k0);
    k_trsv_diag<true><<<(pw + 31) / 32, 256, 0, st>>>(tinv + (int64_t)p * TP * TP, pw, ya + k0,
                                                      yb + k0);
    ++nl;
    const int rows = m - k0 - pw;
    if (rows > 0) {
      k_trsv_update<true><<<(rows + 31) / 32, 256, 0, st>>>(L, m, k0, pw, yb, ya);
      ++nl;
    }
  }
  for (int p = np - 1; p >= 0; --p) {  // backward: ya_p = T_p^T yb_p, then the rows above in yb
    const int k0 = p * TP, pw = std::min(TP, m - k0);
    k_trsv_diag<false><<<(pw + 7) / 8, 256, 0, st>>>(tinv + (int64_t)p * TP * TP, pw, yb + k0,
                                                     ya + k0);
    ++nl;
    if (k0 > 0) {
      k_trsv_update<false><<<(k0 + 31) / 32, 256, 0, st>>>(L, m, k0, pw, ya, yb);
      ++nl;
    }
  }
  k_trsv_store<<<blocks, 256, 0, st>>>(ya, x, m, dsc);
  return nl;
}

// Partial products of y = B x with the full symmetric FP64 B (column-major): CTA (row block of
// 32, column chunk J of MV_CHUNK columns), 256 threads = 32 rows x 8 column phases; writes
// P[J][i] = sum_{j in J} B_ij x_j and A[J][i] = sum_{j in J} |B_ij x_j|.
constexpr int MV_CHUNK = 256;
__global__ void k_gemv_part(const double *__restrict__ B, int64_t ldb, int m,
                            const double *__restrict__ x, double *P, double *A) {
  __shared__ double ps[8][33], as[8][33];
  const int il = threadIdx.x & 31, ph = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + il;
  const int j0 = blockIdx.y * MV_CHUNK, j1 = min(m, j0 + MV_CHUNK);
  double s0 = 0.0, s1 = 0.0, a0 = 0.0, a1 = 0.0;
  if (i < m) {
    int j = j0 + ph;
    for (; j + 8 < j1; j += 16) {
      const double v0 = B[i + (int64_t)j * ldb] * x[j];
      const double v1 = B[i + (int64_t)(j + 8) * ldb] * x[j + 8];
      s0 += v0;
      s1 += v1;
      a0 += fabs(v0);
      a1 += fabs(v1);
    }
    for (; j < j1; j += 8) {
      const double v0 = B[i + (int64_t)j * ldb] * x[j];
      s0 += v0;
      a0 += fabs(v0);
    }
  }
  ps[ph][il] = s0 + s1;
  as[ph][il] = a0 + a1;
  __syncthreads();
  if (ph == 0 && i < m) {
    double u = 0.0, v = 0.0;
    for (int q = 0; q < 8; ++q) {
      u += ps[q][il];
      v += as[q][il];
    }
    P[(int64_t)blockIdx.y * m + i] = u;
    A[(int64_t)blockIdx.y * m + i] = v;
  }
}

// r = g - sum_J P[J]; out[0] = max_i |r_i|, out[1] = max_i (sum_J A[J][i] + |g_i|)  (one CTA)
__global__ void k_resid(const double *__restrict__ g, const double *__restrict__ P,
                        const double *__restrict__ A, int nchunk, double *r, int m, double *out) {
  __shared__ double mr[32], mg[32];
  double ar = 0.0, ag = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    double y = 0.0, ay = 0.0;
    for (int q = 0; q < nchunk; ++q) {
      y += P[(int64_t)q * m + i];
      ay += A[(int64_t)q * m + i];
    }
    const double v = g[i] - y;
    r[i] = v;
    ar = fmax(ar, fabs(v));
    ag = fmax(ag, ay + fabs(g[i]));
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

int mixed_chunks(int m) { return (m + MV_CHUNK - 1) / MV_CHUNK; }

// dsc[i] = 1 / sqrt(B_ii) (1 where B_ii <= 0: the factorisation then reports the breakdown)
__global__ void k_mixed_scale(const double *__restrict__ B, int64_t ldb, int m, double *dsc) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const double d = B[i + (int64_t)i * ldb];
    dsc[i] = d > 0.0 ? 1.0 / sqrt(d) : 1.0;
  }
}

int mixed_factor(double *B, int64_t ldb, int m, float *B32, float *Linv32, int *status,
                 double *g, double *r, double *x, double *dsc, double shift, float *tinv,
                 cudaStream_t st, CholStreams *cs) {
  k_mixed_init<<<(m + 255) / 256, 256, 0, st>>>(B, ldb, m, g, r, x);
  const int nt = (m + 31) / 32;
  const bool eq = dsc && m >= TRSV_WIDE_M;
  if (eq) k_mixed_scale<<<(m + 255) / 256, 256, 0, st>>>(B, ldb, m, dsc);
  k_mixed_prep<<<dim3(nt, nt), 256, 0, st>>>(B, ldb, B32, m, eq ? dsc : nullptr, shift);
  // the factorisation leaves L^T in the strict upper triangle of B32 as well
  int nl = 2 + (eq ? 1 : 0) + dense_chol_f32(B32, m, m, status, Linv32, st, cs);
  if (tinv && m >= TRSV_WIDE_M)
    nl += trsv_prepare_blocks(B32, m, Linv32, tinv, tinv + trsv_tinv_floats(m), st);
  return nl;
}

int64_t trsv_tinv_floats(int m) { return (int64_t)((m + TP - 1) / TP) * TP * TP; }
int64_t trsv_tinv_buffer_floats(int m) { return trsv_tinv_floats(m) + (int64_t)256 * (TP + 256); }

int mixed_refine_step(const double *B, int64_t ldb, int m, const float *L32, const float *Linv32,
                      const double *g, double *x, double *r, double *P, double *A, double *norms,
                      const double *dsc, const float *tinv, cudaStream_t st) {
  int nl = 2;
  if (m >= TRSV_WIDE_M) {
    // P (chunks x m doubles) is free until the product below: the FP32 vectors
    float *ya = reinterpret_cast<float *>(P);
    nl += tinv ? trsv_blocked_inv(L32, m, tinv, r, x, ya, ya + m, dsc, st)
               : trsv_blocked(L32, m, Linv32, r, x, ya, dsc, st);
  } else {
    ++nl;
    const size_t smem = (size_t)m * sizeof(float);
    if (smem > 48 * 1024) smem_optin((const void *)k_refine_solve_f32);
    k_refine_solve_f32<<<RCL, RTH, smem, st>>>(L32, m, Linv32, r, x);
  }
  const int nch = mixed_chunks(m);
  k_gemv_part<<<dim3((m + 31) / 32, nch), 256, 0, st>>>(B, ldb, m, x, P, A);
  k_resid<<<1, 1024, 0, st>>>(g, P, A, nch, r, m, norms);
  return nl;
}

// The pieces of the GMRES form of the mixed SCE solve (large m): out = B v (the full symmetric
// FP64 B, the refinement's partial products summed per row in a fixed order), w = S M^{-1} S u
// with M = L32 L32^T the FP32 factor of the equilibrated S B S (the blocked substitutions), and
// the true residual r = g - B x with its norms.
__global__ void k_sum_parts(const double *__restrict__ P, int nchunk, int m, double *out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    double y = 0.0;
    for (int q = 0; q < nchunk; ++q) y += P[(int64_t)q * m + i];
    out[i] = y;
  }
}

int mixed_matvec(const double *B, int64_t ldb, int m, const double *v, double *out, double *P,
                 double *A, cudaStream_t st) {
  const int nch = mixed_chunks(m);
  k_gemv_part<<<dim3((m + 31) / 32, nch), 256, 0, st>>>(B, ldb, m, v, P, A);
  k_sum_parts<<<std::min(152 * 8, (m + 255) / 256), 256, 0, st>>>(P, nch, m, out);
  return 2;
}

int mixed_precond(const float *L32, int m, const float *Linv32, const double *u, double *w,
                  double *P, const double *dsc, const float *tinv, cudaStream_t st) {
  cudaMemsetAsync(w, 0, (size_t)m * sizeof(double), st);
  float *ya = reinterpret_cast<float *>(P);
  return tinv ? trsv_blocked_inv(L32, m, tinv, u, w, ya, ya + m, dsc, st)
              : trsv_blocked(L32, m, Linv32, u, w, ya, dsc, st);
}

int mixed_residual(const double *B, int64_t ldb, int m, const double *g, const double *x,
                   double *r, double *P, double *A, double *norms, cudaStream_t st) {
  const int nch = mixed_chunks(m);
  k_gemv_part<<<dim3((m + 31) / 32, nch), 256, 0, st>>>(B, ldb, m, x, P, A);
  k_resid<<<1, 1024, 0, st>>>(g, P, A, nch, r, m, norms);
  return 2;
}

// ---------------------------------------------------------------------------------------------
// Allocation-free Schur complement solve.  Working storage: the bordered copy of B
// ((m+1) x m, leading dimension m+1), the inverses of the NB x NB (32 x 32) diagonal blocks, and one
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

extern "C" mcsdp_status mcsdp_sce_solve_noalloc(const double *B, int64_t ldb, const double *g,
                                                double *x, int32_t m, void *stream) {
  using namespace mcsdp;
  if (m <= 0 || m > NA_MAX_M || ldb < m || !B || !g || !x) return MCSDP_ERR_ARG;
  // errors left by earlier, unrelated work would otherwise be reported as this call's
  (void)cudaGetLastError();
  // The array's device address is looked up on every call (no allocation, no synchronisation):
  // a cached address would go stale if the caller reset the device, since the module is then
  // loaded again elsewhere.  On the first call on a device this also loads the module.
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, g_sce_noalloc_scratch) != cudaSuccess || !p) return MCSDP_ERR_CUDA;
  double *base = static_cast<double *>(p);
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t ldw = (int64_t)m + 1;
  double *Bw = base;
  double *Binv = base + NA_B;
  int *status = reinterpret_cast<int *>(base + NA_B + NA_INV);
  int blocks = (int)(((int64_t)m * m + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  k_noalloc_setup<<<blocks, 256, 0, st>>>(Bw, ldw, B, ldb, g, m, status);
  dense_chol_bordered(Bw, ldw, m, status, Binv, st, nullptr);
  dense_backsolve(Bw, ldw, m, Binv, x, st);
  if (cudaGetLastError() != cudaSuccess) return MCSDP_ERR_CUDA;
  int hst = 0;
  if (cudaMemcpyAsync(&hst, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return MCSDP_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return MCSDP_ERR_CUDA;
  return (hst & ST_NOT_PD) ? MCSDP_ERR_NOT_PD : MCSDP_OK;
}

namespace mcsdp {
__global__ void k_pivot_rcp(const double *__restrict__ d, double *__restrict__ r, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    r[i] = pivot_rcp<double>(d[i]);
}
}  // namespace mcsdp

extern "C" mcsdp_status mcsdp_pivot_reciprocal(const double *d, double *r, int64_t n,
                                               void *stream) {
  if (n < 0 || (n > 0 && (!d || !r))) return MCSDP_ERR_ARG;
  if (n == 0) return MCSDP_OK;
  const int64_t want = (n + 255) / 256;
  const int blocks = want > 4096 ? 4096 : (int)want;
  mcsdp::k_pivot_rcp<<<blocks, 256, 0, (cudaStream_t)stream>>>(d, r, n);
  return cudaGetLastError() == cudaSuccess ? MCSDP_OK : MCSDP_ERR_CUDA;
}

extern "C" mcsdp_status mcsdp_chol_block_task_order(int32_t nblk, const int32_t *mb,
                                                    int64_t *ntask, int32_t *tasks) {
  if (nblk <= 0 || !mb || !ntask) return MCSDP_ERR_ARG;
  for (int b = 0; b < nblk; ++b)
    if (mb[b] <= 0) return MCSDP_ERR_ARG;
  mcsdp::DagBlockPlan pl;
  mcsdp::chol_dag_block_plan(std::vector<int>(mb, mb + nblk), pl);
  *ntask = pl.total;
  if (!tasks) return MCSDP_OK;
  // the kernel's decode: segment lookup, then the block's own decode started at the segment
  int blk = -1, R = 0, C = 0, kcur = 0;
  int64_t kstart = 0;
  mcsdp::DagPrefix pf{};
  const int nseg = (int)pl.seg_blk.size();
  for (int64_t t = 0; t < pl.total; ++t) {
    const int sg = mcsdp::dag_block_segment(t, pl.seg_start.data(), nseg);
    if (pl.seg_blk[sg] != blk) {
      blk = pl.seg_blk[sg];
      R = (mb[blk] + 1 + mcsdp::NB - 1) / mcsdp::NB;
      C = (mb[blk] + mcsdp::NB - 1) / mcsdp::NB;
      pf = mcsdp::dag_prefix(R, C);
    }
    const int64_t tl = pl.seg_l0[sg] + (t - pl.seg_start[sg]);
    if (pl.seg_k[sg] >= 0) {
      kcur = pl.seg_k[sg];
      kstart = pl.seg_l0[sg];
    }
    const mcsdp::DagTask d = mcsdp::dag_decode(tl, R, C, pf, kcur, kstart);
    tasks[5 * t] = blk;
    tasks[5 * t + 1] = d.type;
    tasks[5 * t + 2] = d.i;
    tasks[5 * t + 3] = d.j;
    tasks[5 * t + 4] = d.k;
  }
  return MCSDP_OK;
}

extern "C" mcsdp_status mcsdp_chol_task_order(int32_t m, int32_t rows, int64_t *ntask,
                                              int32_t *tasks) {
  if (m <= 0 || rows < m || !ntask) return MCSDP_ERR_ARG;
  const int R = (rows + mcsdp::NB - 1) / mcsdp::NB, C = (m + mcsdp::NB - 1) / mcsdp::NB;
  const int64_t total = mcsdp::dag_total(R, C);
  *ntask = total;
  if (!tasks) return MCSDP_OK;
  const mcsdp::DagPrefix pf = mcsdp::dag_prefix(R, C);
  int kcur = 0;
  int64_t kstart = pf.pre;
  for (int64_t t = 0; t < total; ++t) {
    const mcsdp::DagTask d = mcsdp::dag_decode(t, R, C, pf, kcur, kstart);
    tasks[4 * t] = d.type;
    tasks[4 * t + 1] = d.i;
    tasks[4 * t + 2] = d.j;
    tasks[4 * t + 3] = d.k;
  }
  return MCSDP_OK;
}
