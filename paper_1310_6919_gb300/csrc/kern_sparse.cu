// Sparse-structure kernels of the MC-PDIPM iteration:
//   K2  Y = N N^T (supernodal, left-looking, one level of the supernode tree per launch)
//   K1  Algorithm 1 (Sec. 3.1): L̂ with X̂^{-1} = L̂ L̂^T, one CTA per clique
//   K5  Y / dY on the aggregate pattern
//   K6  P-MATRIX (eq. newdX2), one warp per column
//   K7  clique-wise primal step length (eq. primal_length2)
//   K8  scalars and update
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"
#include "warp_solve.cuh"

namespace mcsdp {

// A CTA-wide early exit on a flag that other CTAs may set while this one runs: thread 0 reads
// it once and the whole CTA follows that reading (every thread then reaches the same barriers).
__device__ __forceinline__ bool cta_flag_set(const int *flag, int mask) {
  __shared__ int v;
  if (threadIdx.x == 0) v = (*(volatile const int *)flag) & mask;
  __syncthreads();
  const bool r = v != 0;
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------------------------------------
// K5: out[slot] = c0 * A_0[slot] + c1 * sum_k vec[k] A_k[slot]
__global__ void k_slot_combine(DevSym S, double *out, const double *__restrict__ vec, double c0,
                               double c1) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S.nslot;
       s += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int q = S.slot_ptr[s]; q < S.slot_ptr[s + 1]; ++q) {
      int k = S.slot_k[q];
      if (k > 0) acc = fma(S.slot_val[q], vec[k - 1], acc);
    }
    out[S.slot_off[s]] = c0 * S.slot_a0[s] + c1 * acc;
  }
}

void launch_slot_combine(const DevSym &S, double *out, const double *vec, double c0, double c1,
                         cudaStream_t st) {
  int blocks = (int)((S.nslot + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  k_slot_combine<<<blocks, 256, 0, st>>>(S, out, vec, c0, c1);
}

// ---------------------------------------------------------------------------------------------
// dense Cholesky of an nrow x ncol column-major panel in shared memory (lower, in place):
// the leading ncol x ncol block is factored, the rows below are solved against it.  The serial
// column loop is warp-specialised with one barrier per column: at step j, warp 0 writes the
// finished column j-1 back, brings column j+1 up to date, takes its pivot d_{j+1}, the
// reciprocal (FP32 seed and two Newton steps) and the scaled column u_{j+1} = F[:, j+1] / d_{j+1}
// (kept aside, so the column stays unscaled while the others read it); the other warps apply
// step j to the columns >= j+2.  This is F = U D U^T with U unit lower; the square roots of D
// are taken in parallel at the end (L = U D^{1/2}).  Needs >= 2 warps.
// scr: 2 * nrow + ncol doubles.
__device__ void chol_panel_smem(double *F, int nrow, int ncol, int *status_word, int flag,
                                double *scr) {
  double *uc = scr, *dv = scr + 2 * nrow;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nth = blockDim.x - 32;
  bool bad = false;
  if (warp == 0 && ncol > 0) {  // column 0: pivot, reciprocal, scaled column
    double r0 = 0.0;
    if (lane == 0) {
      double d = F[0];
      if (!(d > 0.0)) {
        bad = true;
        d = 1.0;
      }
      dv[0] = d;
      r0 = pivot_rcp<double>(d);
    }
    r0 = __shfl_sync(0xffffffffu, r0, 0);
    for (int i = 1 + lane; i < nrow; i += 32) uc[i] = F[i] * r0;
  }
  __syncthreads();
  for (int j = 0; j < ncol; ++j) {
    const double *u = uc + (j & 1) * nrow;  // u_j
    if (warp == 0) {
      if (j >= 1) {  // column j-1 is no longer read: store u_{j-1} (rows > j-1)
        const double *up = uc + ((j - 1) & 1) * nrow;
        for (int i = j + lane; i < nrow; i += 32) F[i + (int64_t)(j - 1) * nrow] = up[i];
      }
      __syncwarp();
      if (j + 1 < ncol) {
        double *un = uc + ((j + 1) & 1) * nrow;
        const double fj = F[(j + 1) + (int64_t)j * nrow];
        double a0 = 0.0;
        for (int i = j + 1 + lane; i < nrow; i += 32) {
          const double a = F[i + (int64_t)(j + 1) * nrow] - u[i] * fj;
          F[i + (int64_t)(j + 1) * nrow] = a;
          if (i == j + 1) a0 = a;
        }
        double rj = 0.0;
        if (lane == 0) {
          double d = a0;
          if (!(d > 0.0)) {
            bad = true;
            d = 1.0;
          }
          dv[j + 1] = d;
          rj = pivot_rcp<double>(d);
        }
        rj = __shfl_sync(0xffffffffu, rj, 0);
        __syncwarp();
        for (int i = j + 2 + lane; i < nrow; i += 32) un[i] = F[i + (int64_t)(j + 1) * nrow] * rj;
      }
    } else {
      // step j on the columns >= j+2 (rows >= column); column j is only read
      const int w = ncol - j - 2, hgt = nrow - j - 2;
      const int nwork = (w > 0 && hgt > 0) ? w * hgt : 0;
      for (int idx = tid - 32; idx < nwork; idx += nth) {
        const int kk = j + 2 + idx / hgt, ii = j + 2 + idx % hgt;
        if (ii >= kk) F[ii + (int64_t)kk * nrow] -= u[ii] * F[kk + (int64_t)j * nrow];
      }
    }
    __syncthreads();
  }
  if (bad) atomicOr(status_word, flag);
  if (ncol > 0 && warp == 0) {
    const double *up = uc + ((ncol - 1) & 1) * nrow;
    for (int i = ncol + lane; i < nrow; i += 32) F[i + (int64_t)(ncol - 1) * nrow] = up[i];
  }
  for (int j = tid; j < ncol; j += blockDim.x) dv[j] = sqrt(dv[j]);
  __syncthreads();
  for (int idx = tid; idx < nrow * ncol; idx += blockDim.x) {
    const int i = idx % nrow, j = idx / nrow;
    if (i > j) F[i + (int64_t)j * nrow] *= dv[j];
    else if (i == j) F[i + (int64_t)j * nrow] = dv[j];
  }
  __syncthreads();
}

// D = L^{-1} for the leading ncol x ncol lower block L of F (ld = ld), D column-major (ld ncol).
// With U = L diag(L)^{-1} (unit lower), L^{-1} = diag(L)^{-1} U^{-1}; U^{-1} is found by forward
// elimination on the identity, one barrier per step, the (ncol-1-k)(k+1) entries of step k
// spread over all threads.  rdv: ncol doubles of scratch.
__device__ void tri_inverse_smem(const double *F, int ld, int ncol, double *D, double *rdv) {
  const int tid = threadIdx.x, bd = blockDim.x;
  for (int j = tid; j < ncol; j += bd) rdv[j] = 1.0 / F[j + (int64_t)j * ld];
  for (int idx = tid; idx < ncol * ncol; idx += bd) D[idx] = (idx % ncol == idx / ncol) ? 1.0 : 0.0;
  __syncthreads();
  for (int k = 0; k + 1 < ncol; ++k) {
    const int w = k + 1, cnt = (ncol - 1 - k) * w;
    const double rk = rdv[k];
    for (int e = tid; e < cnt; e += bd) {
      const int q = e / w;
      const int i = k + 1 + q, c = e - q * w;
      D[i + (int64_t)c * ncol] -= F[i + (int64_t)k * ld] * rk * D[k + (int64_t)c * ncol];
    }
    __syncthreads();
  }
  for (int idx = tid; idx < ncol * ncol; idx += bd) D[idx] *= rdv[idx % ncol];
  __syncthreads();
}

// F[rel rows, rel cols] += sgn * L_s[p1:, :] L_s[p1:p2, :]^T for the updates [ub, ue) of t
__device__ void ychol_pull(const DevSym &S, int ub, int ue, const double *N, double *F, int nrow,
                           double sgn) {
  const int tid = threadIdx.x, bd = blockDim.x;
  for (int u = ub; u < ue; ++u) {
    const int s = S.upd_src[u], p1 = S.upd_p1[u], p2 = S.upd_p2[u];
    const int *rel = S.upd_rel + S.upd_relptr[u];
    const int snrow = (int)(S.sn_rowptr[s + 1] - S.sn_rowptr[s]);
    const int sncol = S.sn_col[s + 1] - S.sn_col[s];
    const double *Ls = N + S.sn_valptr[s];
    const int na = snrow - p1, nb = p2 - p1;
    for (int idx = tid; idx < na * nb; idx += bd) {
      const int ia = idx % na, ib = idx / na;
      if (ia < ib) continue;
      double acc = 0.0;
      for (int k = 0; k < sncol; ++k)
        acc = fma(Ls[p1 + ia + (int64_t)k * snrow], Ls[p1 + ib + (int64_t)k * snrow], acc);
      F[rel[ia] + (int64_t)rel[ib] * nrow] += sgn * acc;
    }
    __syncthreads();
  }
}

// extra update chunks of a level: Pf[cand][slot] = sum of the chunk's updates (nrow_t x ncol_t)
__global__ void k_ychol_partial(DevSym S, int x0, const double *__restrict__ Nbuf, double *Pf,
                                const int *status) {
  extern __shared__ double F[];
  const int x = x0 + blockIdx.x;
  const int c = blockIdx.y;
  if (cta_flag_set(&status[c], ST_NOT_PD)) return;
  const int t = S.xch_t[x];
  const int nrow = (int)(S.sn_rowptr[t + 1] - S.sn_rowptr[t]);
  const int ncol = S.sn_col[t + 1] - S.sn_col[t];
  const int sz = nrow * ncol;
  for (int i = threadIdx.x; i < sz; i += blockDim.x) F[i] = 0.0;
  __syncthreads();
  ychol_pull(S, S.xch_ub[x], S.xch_ue[x], Nbuf + (int64_t)c * S.nnzL, F, nrow, 1.0);
  double *P = Pf + (int64_t)c * S.nslotf + S.xch_slotf[x];
  for (int i = threadIdx.x; i < sz; i += blockDim.x) P[i] = F[i];
}

// the extra chunks of a target summed into the slot of its first chunk.  CTA = 32 entries x 8
// chunk phases (phase p sums the chunks x + p, x + p + 8, ...), then the 8 phase sums are added
// in order (deterministic); grid (entry blocks, target, candidate)
__global__ void k_ychol_reduce(DevSym S, int f0, double *Pf, const int *status) {
  __shared__ double part[8][33];
  const int x = S.xfst[f0 + blockIdx.y];
  const int c = blockIdx.z;
  if (cta_flag_set(&status[c], ST_NOT_PD)) return;
  const int t = S.xch_t[x];
  const int xe = S.xch_end[t];
  const int sz = (int)(S.sn_rowptr[t + 1] - S.sn_rowptr[t]) * (S.sn_col[t + 1] - S.sn_col[t]);
  if ((int)blockIdx.x * 32 >= sz) return;
  const int lane = threadIdx.x & 31, ph = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + lane;
  double *P = Pf + (int64_t)c * S.nslotf;
  double a = 0.0;
  if (i < sz)
    for (int xx = x + ph; xx < xe; xx += 8) a += P[S.xch_slotf[xx] + i];
  part[ph][lane] = a;
  __syncthreads();
  if (ph == 0 && i < sz) {
    double s = part[0][lane];
    for (int q = 1; q < 8; ++q) s += part[q][lane];
    P[S.xch_slotf[x] + i] = s;
  }
}

void launch_ychol_partials(const DevSym &S, int x0, int nx, int f0, int nf, int ncand,
                           const double *Nbuf, double *Pf, const int *status, cudaStream_t st) {
  if (nx <= 0) return;
  const size_t smem = (size_t)S.max_nrow * S.max_ncol * 8;
  smem_optin((const void *)k_ychol_partial);
  dim3 grid(nx, ncand);
  k_ychol_partial<<<grid, 256, smem, st>>>(S, x0, Nbuf, Pf, status);
  if (nf > 0) {
    const int gx = (S.max_nrow * S.max_ncol + 31) / 32;
    k_ychol_reduce<<<dim3(gx, nf, ncand), 256, 0, st>>>(S, f0, Pf, status);
  }
}

__global__ void k_ychol(DevSym S, int lvl_begin, const double *__restrict__ alpha,
                        const double *__restrict__ Yb, const double *__restrict__ dY, double *Nbuf,
                        double *Dbuf, int *status, const double *__restrict__ Pf) {
  extern __shared__ double F[];
  const int t = S.lvl_sn[lvl_begin + blockIdx.x];
  const int c = blockIdx.y;
  if (cta_flag_set(&status[c], ST_NOT_PD)) return;
  double *N = Nbuf + (int64_t)c * S.nnzL;
  double *Dc = Dbuf ? Dbuf + (int64_t)c * S.nnzD : nullptr;
  const double a = alpha ? alpha[c] : 0.0;
  const int64_t r0 = S.sn_rowptr[t];
  const int nrow = (int)(S.sn_rowptr[t + 1] - r0);
  const int c0 = S.sn_col[t], ncol = S.sn_col[t + 1] - c0;
  const int64_t v0 = S.sn_valptr[t];
  const int sz = nrow * ncol;
  const int tid = threadIdx.x, bd = blockDim.x;
  for (int i = tid; i < sz; i += bd) F[i] = dY ? fma(a, dY[v0 + i], Yb[v0 + i]) : Yb[v0 + i];
  __syncthreads();
  ychol_pull(S, S.upd_ptr[t], S.upd_c0end[t], N, F, nrow, -1.0);
  if (S.xch_end[t] > S.xch_beg[t]) {  // the extra chunks, already summed into the first slot
    const double *P = Pf + (int64_t)c * S.nslotf + S.xch_slotf[S.xch_beg[t]];
    for (int i = tid; i < sz; i += bd) F[i] -= P[i];
    __syncthreads();
  }
  double *Dsm = F + sz;
  double *scr = Dsm + ncol * ncol;
  chol_panel_smem(F, nrow, ncol, &status[c], ST_NOT_PD, scr);
  for (int i = tid; i < sz; i += bd) N[v0 + i] = F[i];
  if (!Dbuf) return;  // step-length candidates: only the success of the factorisation matters
  tri_inverse_smem(F, nrow, ncol, Dsm, scr);
  const int64_t d0 = S.sn_dptr[t];
  for (int i = tid; i < ncol * ncol; i += bd) Dc[d0 + i] = Dsm[i];
  (void)c0;
}

size_t ychol_smem_bytes(const DevSym &S) {
  return ((size_t)S.max_nrow * S.max_ncol + (size_t)S.max_ncol * S.max_ncol + 2 * (size_t)S.max_nrow +
          S.max_ncol) * 8;
}

void launch_ychol_level(const DevSym &S, int lvl_begin, int lvl_count, int ncand,
                        const double *alpha, const double *Yb, const double *dY, double *Nbuf,
                        double *Dbuf, int *status, const double *Pf, cudaStream_t st) {
  dim3 grid(lvl_count, ncand);
  const size_t smem = ychol_smem_bytes(S);
  smem_optin((const void *)k_ychol);
  k_ychol<<<grid, 256, smem, st>>>(S, lvl_begin, alpha, Yb, dY, Nbuf, Dbuf, status, Pf);
}

// ---------------------------------------------------------------------------------------------
// K1: Algorithm 1.  For clique r with k = |C_r|: the reversed block P X̄_CC P (Step 2-1) is
// Cholesky-factored, M = chol(P X̄_CC P) (Step 2-2); L_r = P M^{-T} P (Step 2-3) and its first
// |S_r| columns are stored as L̂_{C_r S_r} (Step 3).
__global__ void k_alg1(DevSym S, const double *__restrict__ X, double *Lh, double *DL,
                       int *status) {
  extern __shared__ double sm[];
  const int r = blockIdx.x;
  const int64_t r0 = S.sn_rowptr[r];
  const int k = (int)(S.sn_rowptr[r + 1] - r0);
  const int c0 = S.sn_col[r], ns = S.sn_col[r + 1] - c0;
  const int64_t v0 = S.sn_valptr[r];
  double *A = sm;                      // k x k
  double *T = sm + (int64_t)k * k;     // k x k, inverse of M
  double *rd = T + (int64_t)k * k;     // 3k doubles of scratch
  const int tid = threadIdx.x, bd = blockDim.x;
  for (int idx = tid; idx < k * k; idx += bd) {
    const int a = idx % k, b = idx / k;
    if (a < b) continue;
    const double v = clique_entry(S, X, r, a, b);
    A[(k - 1 - a) + (int64_t)(k - 1 - b) * k] = v;
    A[(k - 1 - b) + (int64_t)(k - 1 - a) * k] = v;
  }
  __syncthreads();
  chol_panel_smem(A, k, k, status, ST_NOT_PD, rd);
  tri_inverse_smem(A, k, k, T, rd);  // T = M^{-1}
  // L_r[a][b] = (P M^{-T} P)[a][b] = T[k-1-b][k-1-a]
  for (int idx = tid; idx < k * ns; idx += bd) {
    const int a = idx % k, b = idx / k;
    Lh[v0 + idx] = (a >= b) ? T[(k - 1 - b) + (int64_t)(k - 1 - a) * k] : 0.0;
  }
  // (L_r)_SS^{-1} is the leading block of L_r^{-1} = P M^T P: entry [a][b] = M[k-1-b][k-1-a]
  const int64_t d0 = S.sn_dptr[r];
  for (int idx = tid; idx < ns * ns; idx += bd) {
    const int a = idx % ns, b = idx / ns;
    DL[d0 + idx] = (a >= b) ? A[(k - 1 - b) + (int64_t)(k - 1 - a) * k] : 0.0;
  }
  (void)c0;
}

size_t alg1_smem_bytes(const DevSym &S) {
  return ((size_t)2 * S.max_nrow * S.max_nrow + 3 * (size_t)S.max_nrow) * 8;
}

void launch_alg1(const DevSym &S, const double *X, double *Lh, double *DL, int *status,
                 cudaStream_t st) {
  if (S.nforest <= 0) return;
  const size_t smem = alg1_smem_bytes(S);
  smem_optin((const void *)k_alg1);
  k_alg1<<<S.nforest, 256, smem, st>>>(S, X, Lh, DL, status);
}

// ---------------------------------------------------------------------------------------------
// K6: P-MATRIX, eq. (newdX2), column k per warp:
//   y = N^{-T} N^{-1} e_k         (Y^{-1} e_k)
//   w = L̂^{-T} L̂^{-1} (dY y)      (X̂ dY Y^{-1} e_k)
// and the entries on E are stored: Y^{-1} on lower(E), M = X̂ dY Y^{-1} at (i, k) for rows i of
// column k (Mlow) and at the transposed position for rows i < k (Mup).

// K6 pieces.  For the columns k in [k0, k0 + nc) solved into W (row-major, ld = ldw):
// lower(E) entries of column k: outE[(i, k)] = W[i][k - k0] for the rows i >= k of k's clique
template <class T>
__global__ void k_extract_lowerE(DevSym S, const T *__restrict__ W, int64_t ldw, int k0, int nc,
                                 double *outE) {
  const int j = blockIdx.x * blockDim.y + threadIdx.y;
  if (j >= nc) return;
  const int k = k0 + j;
  const int t = S.col2sn[k];
  const int64_t r0 = S.sn_rowptr[t];
  const int nrow = (int)(S.sn_rowptr[t + 1] - r0);
  const int lc = k - S.sn_col[t];
  const int64_t cbase = S.sn_valptr[t] + (int64_t)lc * nrow;
  for (int p = lc + threadIdx.x; p < nrow; p += blockDim.x)
    outE[cbase + p] = (double)W[(int64_t)S.rows[r0 + p] * ldw + j];
}

// transposed entries: for rows i < k with (k, i) in E, outE[(k, i)] = W[i][k - k0]
template <class T>
__global__ void k_extract_upperE(DevSym S, const T *__restrict__ W, int64_t ldw, int k0, int nc,
                                 double *outE) {
  const int j = blockIdx.x * blockDim.y + threadIdx.y;
  if (j >= nc) return;
  const int k = k0 + j;
  for (int q = S.rs_ptr[k] + threadIdx.x; q < S.rs_ptr[k + 1]; q += blockDim.x)
    outE[S.rs_off[q]] = (double)W[(int64_t)S.rs_col[q] * ldw + j];
}

template <class T>
void launch_extract_lowerE(const DevSym &S, const T *W, int64_t ldw, int k0, int nc,
                           double *outE, cudaStream_t st) {
  if (nc <= 0) return;
  dim3 blk(32, 8);
  k_extract_lowerE<T><<<(nc + 7) / 8, blk, 0, st>>>(S, W, ldw, k0, nc, outE);
}

template <class T>
void launch_extract_upperE(const DevSym &S, const T *W, int64_t ldw, int k0, int nc,
                           double *outE, cudaStream_t st) {
  if (nc <= 0) return;
  dim3 blk(32, 8);
  k_extract_upperE<T><<<(nc + 7) / 8, blk, 0, st>>>(S, W, ldw, k0, nc, outE);
}

// Ww = dY Wy on the aggregate pattern (full symmetric row lists), row i per CTA row
template <class T>
__global__ void k_dY_times(DevSym S, const double *__restrict__ dY, const T *__restrict__ Wy,
                          T *Ww, int64_t ldw, int nc) {
  const int i = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nc) return;
  T acc = T(0);
  for (int q = S.arow_ptr[i]; q < S.arow_ptr[i + 1]; ++q)
    acc = fma((T)dY[S.arow_off[q]], Wy[(int64_t)S.arow_col[q] * ldw + j], acc);
  Ww[(int64_t)i * ldw + j] = acc;
}

template <class T>
void launch_dY_times(const DevSym &S, const double *dY, const T *Wy, T *Ww, int64_t ldw,
                     int nc, cudaStream_t st) {
  if (nc <= 0) return;
  dim3 grid((nc + 127) / 128, S.n);
  k_dY_times<T><<<grid, 128, 0, st>>>(S, dY, Wy, Ww, ldw, nc);
}

#define MCSDP_PM_INST(T)                                                                        \
  template void launch_extract_lowerE<T>(const DevSym &, const T *, int64_t, int, int, double *, \
                                         cudaStream_t);                                         \
  template void launch_extract_upperE<T>(const DevSym &, const T *, int64_t, int, int, double *, \
                                         cudaStream_t);                                         \
  template void launch_dY_times<T>(const DevSym &, const double *, const T *, T *, int64_t, int, \
                                   cudaStream_t);
MCSDP_PM_INST(double)
MCSDP_PM_INST(float)
#undef MCSDP_PM_INST

// out[i] = (float) in[i]
__global__ void k_cast_f32(const double *__restrict__ in, float *out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

void launch_cast_f32(const double *in, float *out, int64_t n, cudaStream_t st) {
  if (n <= 0) return;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  k_cast_f32<<<blocks, 256, 0, st>>>(in, out, n);
}

// dX on lower(E): beta mu Y^{-1} - X̄ - (M + M^T)/2   (eq. dX with the symmetrisation)
__global__ void k_dx_combine(DevSym S, double betamu, const double *__restrict__ X,
                             const double *__restrict__ YinvE, const double *__restrict__ Mlow,
                             const double *__restrict__ Mup, double *dX,
                             const double *__restrict__ betamu_dev) {
  if (betamu_dev) betamu = *betamu_dev;
  const int s = blockIdx.x;
  const int nrow = (int)(S.sn_rowptr[s + 1] - S.sn_rowptr[s]);
  const int ncol = S.sn_col[s + 1] - S.sn_col[s];
  const int64_t v0 = S.sn_valptr[s];
  for (int idx = threadIdx.x; idx < nrow * ncol; idx += blockDim.x) {
    const int p = idx % nrow, lc = idx / nrow;
    const int64_t o = v0 + idx;
    double v;
    if (p < lc) v = 0.0;
    else if (p == lc) v = betamu * YinvE[o] - X[o] - Mlow[o];
    else v = betamu * YinvE[o] - X[o] - 0.5 * (Mlow[o] + Mup[o]);
    dX[o] = v;
  }
}

void launch_dx_combine(const DevSym &S, double betamu, const double *X, const double *YinvE,
                       const double *Mlow, const double *Mup, double *dX, cudaStream_t st,
                       const double *betamu_dev) {
  if (S.nforest <= 0) return;
  k_dx_combine<<<S.nforest, 128, 0, st>>>(S, betamu, X, YinvE, Mlow, Mup, dX, betamu_dev);
}

// ---------------------------------------------------------------------------------------------
// K7: alpha_r = max{alpha in (0,1] : X̄_CC + alpha dX_CC psd} (eq. primal_length2):
// X̄_CC = L L^T, W = L^{-1} dX_CC L^{-T}, Householder tridiagonalisation of W, smallest
// eigenvalue by Sturm-count multisection; alpha_r = min(1, -1/lambda_min).
// Number of eigenvalues below sig of the symmetric tridiagonal matrix T (diagonal d, squared
// off-diagonal e2, entries scaled to magnitude <= 1): the sign changes of the leading principal
// minors p_i = det(T_i - sig I), p_0 = 1, from the three-term recurrence
// p_i = (d_{i-1} - sig) p_{i-1} - e2_{i-2} p_{i-2} (Sturm sequence; a zero minor takes the sign
// opposite to its predecessor).  No division, one dependent multiply-add per step; the pair
// (p_i, p_{i-1}) is rescaled by a power of two (exact) every eighth step.
__device__ int sturm_count_p(const double *d, const double *e2, int k, double sig) {
  double pm = 1.0, p = d[0] - sig;
  bool sp = (p < 0.0) || (p == 0.0);
  int cnt = sp ? 1 : 0;
  for (int i = 1; i < k; ++i) {
    const double pn = fma(d[i] - sig, p, -e2[i - 1] * pm);
    pm = p;
    p = pn;
    const bool s = (p < 0.0) || (p == 0.0 && !sp);
    cnt += (s != sp) ? 1 : 0;
    sp = s;
    if ((i & 7) == 0) {
      const double a = fmax(fabs(p), fabs(pm));
      if (a > 0x1p+400) {
        p *= 0x1p-400;
        pm *= 0x1p-400;
      } else if (a < 0x1p-400 && a > 0.0) {
        p *= 0x1p+400;
        pm *= 0x1p+400;
      }
    }
  }
  return cnt;
}

__global__ void k_primal_step(DevSym S, const double *__restrict__ X, const double *__restrict__ D,
                              double *alpha_r, int *status) {
  extern __shared__ double sm[];
  __shared__ double red[32];
  __shared__ double sh[4];
  const int r = blockIdx.x;
  const int64_t r0 = S.sn_rowptr[r];
  const int k = (int)(S.sn_rowptr[r + 1] - r0);
  double *Xs = sm;
  double *W = Xs + (int64_t)k * k;
  double *rd = W + (int64_t)k * k;
  double *dd = rd + k;
  double *ee = dd + k;
  double *v = ee + k;
  double *q = v + k;
  const int tid = threadIdx.x, bd = blockDim.x;
  for (int idx = tid; idx < k * k; idx += bd) {
    const int a = idx % k, b = idx / k;
    if (a < b) continue;
    const double xv = clique_entry(S, X, r, a, b);
    const double dv = clique_entry(S, D, r, a, b);
    Xs[a + (int64_t)b * k] = xv;
    Xs[b + (int64_t)a * k] = xv;
    W[a + (int64_t)b * k] = dv;
    W[b + (int64_t)a * k] = dv;
  }
  __syncthreads();
  chol_panel_smem(Xs, k, k, status, ST_NOT_PD, q + k);
  for (int j = tid; j < k; j += bd) rd[j] = 1.0 / Xs[j + (int64_t)j * k];
  __syncthreads();
  for (int pass = 0; pass < 2; ++pass) {
    // W <- L^{-1} W (columns independent), then transpose
    for (int col = tid; col < k; col += bd) {
      double *wc = W + (int64_t)col * k;
      for (int i = 0; i < k; ++i) {
        double s = wc[i];
        for (int l = 0; l < i; ++l) s = fma(-Xs[i + (int64_t)l * k], wc[l], s);
        wc[i] = s * rd[i];
      }
    }
    __syncthreads();
    for (int idx = tid; idx < k * k; idx += bd) {
      const int a = idx % k, b = idx / k;
      if (a < b) {
        double t1 = W[a + (int64_t)b * k];
        W[a + (int64_t)b * k] = W[b + (int64_t)a * k];
        W[b + (int64_t)a * k] = t1;
      }
    }
    __syncthreads();
  }
  for (int idx = tid; idx < k * k; idx += bd) {
    const int a = idx % k, b = idx / k;
    if (a < b) {
      double m = 0.5 * (W[a + (int64_t)b * k] + W[b + (int64_t)a * k]);
      W[a + (int64_t)b * k] = m;
      W[b + (int64_t)a * k] = m;
    }
  }
  __syncthreads();
  // Householder tridiagonalisation of the symmetric k x k matrix W
  for (int j = 0; j + 2 < k; ++j) {
    const int mlen = k - j - 1;
    double part = 0.0;
    for (int i = tid; i < mlen; i += bd) {
      double x = W[(j + 1 + i) + (int64_t)j * k];
      part += x * x;
    }
    const double ss = block_reduce_sum(part, red);
    const double x0 = W[(j + 1) + (int64_t)j * k];
    if (ss - x0 * x0 <= 1e-300 * (ss + 1e-300) || ss == 0.0) {
      if (tid == 0) { ee[j] = x0; dd[j] = W[j + (int64_t)j * k]; }
      __syncthreads();
      continue;
    }
    const double alpha = x0 >= 0 ? -sqrt(ss) : sqrt(ss);
    const double vn2 = ss - x0 * x0 + (x0 - alpha) * (x0 - alpha);
    const double tau = 2.0 / vn2;
    for (int i = tid; i < mlen; i += bd) v[i] = (i == 0) ? (x0 - alpha) : W[(j + 1 + i) + (int64_t)j * k];
    __syncthreads();
    double pv = 0.0;
    for (int i = tid; i < mlen; i += bd) {
      double s = 0.0;
      for (int l = 0; l < mlen; ++l) s = fma(W[(j + 1 + i) + (int64_t)(j + 1 + l) * k], v[l], s);
      q[i] = tau * s;
      pv += q[i] * v[i];
    }
    const double K = 0.5 * tau * block_reduce_sum(pv, red);
    for (int i = tid; i < mlen; i += bd) q[i] -= K * v[i];
    __syncthreads();
    for (int idx = tid; idx < mlen * mlen; idx += bd) {
      const int i = idx % mlen, l = idx / mlen;
      W[(j + 1 + i) + (int64_t)(j + 1 + l) * k] -= v[i] * q[l] + q[i] * v[l];
    }
    if (tid == 0) { ee[j] = alpha; dd[j] = W[j + (int64_t)j * k]; }
    __syncthreads();
  }
  if (tid == 0) {
    if (k >= 2) {
      dd[k - 2] = W[(k - 2) + (int64_t)(k - 2) * k];
      ee[k - 2] = W[(k - 1) + (int64_t)(k - 2) * k];
    }
    dd[k - 1] = W[(k - 1) + (int64_t)(k - 1) * k];
  }
  __syncthreads();
  // scale T by a power of two (exact) so its entries are at most 1 in magnitude
  if (tid == 0) {
    double amax = 0.0;
    for (int i = 0; i < k; ++i) amax = fmax(amax, fabs(dd[i]));
    for (int i = 0; i + 1 < k; ++i) amax = fmax(amax, fabs(ee[i]));
    sh[1] = amax > 0.0 ? ldexp(1.0, ilogb(amax) + 1) : 1.0;
  }
  __syncthreads();
  const double sc = sh[1], isc = 1.0 / sc;
  for (int i = tid; i < k; i += bd) {
    dd[i] *= isc;
    if (i + 1 < k) v[i] = (ee[i] * isc) * (ee[i] * isc);
  }
  __syncthreads();
  // alpha_r = 1 unless lambda_min(W) < -1
  if (tid == 0) sh[2] = (double)sturm_count_p(dd, v, k, -isc);
  __syncthreads();
  if (sh[2] == 0.0) {
    if (tid == 0) alpha_r[r] = 1.0;
    return;
  }
  // lambda_min in [Gershgorin lower bound, -1): multisection, one shift per thread per round
  __shared__ double bnd[2];
  __shared__ int wfirst[32];
  if (tid == 0) {
    double lo = 1e300;
    for (int i = 0; i < k; ++i) {
      const double rad = (i > 0 ? fabs(ee[i - 1]) : 0.0) + (i + 1 < k ? fabs(ee[i]) : 0.0);
      lo = fmin(lo, dd[i] - rad * isc);
    }
    bnd[0] = lo - 1e-12 * (fabs(lo) + 1.0);
    bnd[1] = -isc;
  }
  __syncthreads();
  const int lane = tid & 31, warp = tid >> 5, nw = bd >> 5;
  for (int it = 0; it < 16; ++it) {
    const double lo = bnd[0], hi = bnd[1];
    if (hi - lo <= 4e-16 * fmax(fabs(lo), fabs(hi))) break;
    const double sig = lo + ((hi - lo) / (double)(bd + 1)) * (double)(tid + 1);
    const unsigned ball = __ballot_sync(0xffffffffu, sturm_count_p(dd, v, k, sig) >= 1);
    if (lane == 0) wfirst[warp] = ball ? warp * 32 + __ffs(ball) - 1 : (1 << 30);
    __syncthreads();
    if (tid == 0) {
      int f = 1 << 30;
      for (int w = 0; w < nw; ++w) f = min(f, wfirst[w]);
      const double step = (hi - lo) / (double)(bd + 1);
      if (f == (1 << 30)) {
        bnd[0] = lo + step * (double)bd;
      } else {
        bnd[1] = lo + step * (double)(f + 1);
        if (f > 0) bnd[0] = lo + step * (double)f;
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    const double lam = 0.5 * (bnd[0] + bnd[1]) * sc;
    alpha_r[r] = lam < -1.0 ? -1.0 / lam : 1.0;
  }
}

size_t primal_step_smem_bytes(const DevSym &S) {
  return ((size_t)2 * S.max_nrow * S.max_nrow + 8 * (size_t)S.max_nrow) * 8;
}

void launch_primal_step(const DevSym &S, const double *X, const double *D, double *alpha_r,
                        int *status, cudaStream_t st) {
  if (S.nforest <= 0) return;
  const size_t smem = primal_step_smem_bytes(S);
  smem_optin((const void *)k_primal_step);
  k_primal_step<<<S.nforest, 256, smem, st>>>(S, X, D, alpha_r, status);
}

// ---------------------------------------------------------------------------------------------
// K8: scalars, single CTA, fixed-order reductions (bitwise reproducible)
// The scalars of the stopping test and the step lengths, in two deterministic stages: MS_PARTS
// CTAs each reduce a fixed contiguous share of the slots, constraints and cliques into six
// partials (sums X.Y, A_0.X, b.z; maxima |A(X)-b|, |b|; minimum alpha_r), then one CTA combines
// the partials in a fixed order.
constexpr int MS_PARTS = 64;
constexpr int MS_THREADS = 256;

__global__ void __launch_bounds__(MS_THREADS)
    k_measures_part(DevSym S, const double *__restrict__ X, const double *__restrict__ Y,
                    const double *__restrict__ z, const double *__restrict__ alpha_r,
                    double *part) {
  __shared__ double red[32];
  const int tid = threadIdx.x, b = blockIdx.x;
  auto share = [&](int64_t n, int64_t &lo, int64_t &hi) {
    const int64_t per = (n + MS_PARTS - 1) / MS_PARTS;
    lo = b * per;
    hi = lo + per < n ? lo + per : n;
  };
  int64_t lo, hi;
  double xy = 0.0, pobj = 0.0;
  share(S.nslot, lo, hi);
  for (int64_t s = lo + tid; s < hi; s += MS_THREADS) {
    const int64_t o = S.slot_off[s];
    const double mult = (S.slot_i[s] == S.slot_j[s]) ? 1.0 : 2.0;
    xy += mult * X[o] * Y[o];
    pobj += mult * S.slot_a0[s] * X[o];
  }
  double pinf = 0.0, dobj = 0.0, maxb = 0.0;
  share(S.m, lo, hi);
  for (int64_t k = lo + tid; k < hi; k += MS_THREADS) {
    double ax = 0.0;
    for (int q = S.con_ptr[k]; q < S.con_ptr[k + 1]; ++q) ax = fma(S.con_w[q], X[S.con_off[q]], ax);
    pinf = fmax(pinf, fabs(ax - S.b[k]));
    dobj = fma(S.b[k], z[k], dobj);
    maxb = fmax(maxb, fabs(S.b[k]));
  }
  double amin = 1.0;
  if (alpha_r) {
    share(S.ns, lo, hi);
    for (int64_t r = lo + tid; r < hi; r += MS_THREADS) amin = fmin(amin, alpha_r[r]);
  }
  xy = block_reduce_sum(xy, red);
  pobj = block_reduce_sum(pobj, red);
  dobj = block_reduce_sum(dobj, red);
  __shared__ double mx[3][32];
  for (int o = 16; o > 0; o >>= 1) {
    pinf = fmax(pinf, __shfl_down_sync(0xffffffffu, pinf, o));
    maxb = fmax(maxb, __shfl_down_sync(0xffffffffu, maxb, o));
    amin = fmin(amin, __shfl_down_sync(0xffffffffu, amin, o));
  }
  if ((tid & 31) == 0) { mx[0][tid >> 5] = pinf; mx[1][tid >> 5] = maxb; mx[2][tid >> 5] = amin; }
  __syncthreads();
  if (tid == 0) {
    double a = 0.0, b2 = 0.0, c = 1.0;
    for (int i = 0; i < MS_THREADS / 32; ++i) { a = fmax(a, mx[0][i]); b2 = fmax(b2, mx[1][i]); c = fmin(c, mx[2][i]); }
    double *pb = part + 6 * b;
    pb[0] = xy; pb[1] = pobj; pb[2] = dobj; pb[3] = a; pb[4] = b2; pb[5] = c;
  }
}

__global__ void k_measures_fin(const double *__restrict__ part, double *scal) {
  __shared__ double ps[6 * MS_PARTS];
  for (int e = threadIdx.x; e < 6 * MS_PARTS; e += blockDim.x) ps[e] = part[e];  // loads in parallel
  __syncthreads();
  if (threadIdx.x != 0) return;
  double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 1.0};
  for (int b = 0; b < MS_PARTS; ++b) {  // fixed order
    const double *pb = ps + 6 * b;
    v[0] += pb[0]; v[1] += pb[1]; v[2] += pb[2];
    v[3] = fmax(v[3], pb[3]); v[4] = fmax(v[4], pb[4]); v[5] = fmin(v[5], pb[5]);
  }
  for (int q = 0; q < 6; ++q) scal[q] = v[q];
}

void launch_measures(const DevSym &S, const double *X, const double *Y, const double *z,
                     const double *alpha_r, double *scal, cudaStream_t st) {
  k_measures_part<<<MS_PARTS, MS_THREADS, 0, st>>>(S, X, Y, z, alpha_r, scal + 16);
  k_measures_fin<<<1, 128, 0, st>>>(scal + 16, scal);
}

__global__ void k_update(int64_t nnz, double *X, const double *__restrict__ dX, double ap, int m,
                         double *z, const double *__restrict__ dz, double ad,
                         const double *__restrict__ steps_dev) {
  if (steps_dev) {  // (gamma alpha_p, gamma alpha_d, failure): nothing moves after a failure
    if (steps_dev[2] != 0.0) return;
    ap = steps_dev[0];
    ad = steps_dev[1];
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nnz;
       i += (int64_t)gridDim.x * blockDim.x)
    X[i] = fma(ap, dX[i], X[i]);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    z[i] = fma(ad, dz[i], z[i]);
}

void launch_update(const DevSym &S, double *X, const double *dX, double ap, double *z,
                   const double *dz, double ad, cudaStream_t st, const double *steps_dev) {
  int blocks = (int)((S.nnzL + 255) / 256);
  if (blocks > 2048) blocks = 2048;
  k_update<<<blocks, 256, 0, st>>>(S.nnzL, X, dX, ap, S.m, z, dz, ad, steps_dev);
}

// ---- the graph form of an iteration (FP64, no dense root): step lengths on the device ----
// g[0] beta mu; g[3] lo, g[4] hi (< 0: none failed yet), g[5] bracket frozen; g[6] gamma alpha_p,
// g[7] gamma alpha_d, g[8] failure (1: dual step collapsed, 2: SCM not positive definite or a
// factorisation timed out); g[9] alpha_p, g[10] alpha_d; g[11] the SCM factorisation's status
__global__ void k_graph_betamu(const double *__restrict__ scal, int n, double beta, double *g) {
  if (threadIdx.x == 0) {
    g[0] = beta * (scal[0] / n);  // the host loop's order: mu first
    g[3] = 0.0;
    g[4] = -1.0;
    g[5] = 0.0;
  }
}
// round r's NCAND candidates from the bracket (the host loop's rule: fixed first round, then
// equal spacing inside (lo, hi], or geometric below hi while everything failed)
// (first: the first round's candidates; geo: 0.3^(i+1), both from the host, so that every
// candidate is the host loop's value bit for bit; the rounded operations below keep its order)
__global__ void k_dual_cands(const double *__restrict__ g, int round, double *cand, int ncand,
                             DualTables t, int *cst) {
  const int i = threadIdx.x;
  if (i >= ncand) return;
  // the candidates' statuses: cleared, or, once the bracket is frozen, marked failed so that the
  // round's factorisation kernels return at once (their CTAs test the status first)
  cst[i] = g[5] != 0.0 ? ST_NOT_PD : 0;
  const double lo = g[3], hi = g[4];
  double v;
  if (round == 0) {
    v = t.first[i];
  } else if (lo == 0.0 && hi > 0) {
    v = __dmul_rn(hi, t.geo[i]);
  } else {
    const double H = hi < 0 ? 1.0 : hi;
    v = __dadd_rn(lo, __ddiv_rn(__dmul_rn(__dsub_rn(H, lo), (double)(i + 1)), (double)(ncand + 1)));
  }
  cand[i] = v;
}
// the bracket from the candidates' factorisation statuses (0 = positive definite); frozen once
// the host loop would have stopped (lo >= 1, or the bracket within 1e-3 of lo)
__global__ void k_dual_update(const int *__restrict__ cst, const double *__restrict__ cand,
                              int ncand, double *g) {
  if (threadIdx.x != 0 || g[5] != 0.0) return;
  double lo = g[3], hi = g[4];
  for (int i = 0; i < ncand; ++i) {
    if (cst[i] == 0) lo = fmax(lo, cand[i]);
    else hi = hi < 0 ? cand[i] : fmin(hi, cand[i]);
  }
  g[3] = lo;
  g[4] = hi;
  if (lo >= 1.0 || (lo > 0 && hi > 0 && (hi - lo) <= 1e-3 * lo)) g[5] = 1.0;
}
__global__ void k_graph_steps(const double *__restrict__ scal, const int *__restrict__ status,
                              double gamma, double *g) {
  if (threadIdx.x != 0) return;
  const double ap = scal[5], lo = g[3];
  const double ad = fmin(lo, 1.0);
  double fail = 0.0;
  if (lo <= 0.0) fail = 1.0;
  if (status[2] & (ST_NOT_PD | ST_TIMEOUT)) fail = 2.0;
  g[6] = gamma * ap;
  g[7] = gamma * ad;
  g[8] = fail;
  g[9] = ap;
  g[10] = ad;
  g[11] = (double)status[2];
}
void launch_graph_betamu(const double *scal, int n, double beta, double *g, cudaStream_t st) {
  k_graph_betamu<<<1, 32, 0, st>>>(scal, n, beta, g);
}
void launch_dual_cands(const double *g, int round, double *cand, int ncand, const DualTables &t,
                       int *cst, cudaStream_t st) {
  k_dual_cands<<<1, 32, 0, st>>>(g, round, cand, ncand, t, cst);
}
void launch_dual_update(const int *cst, const double *cand, int ncand, double *g, cudaStream_t st) {
  k_dual_update<<<1, 32, 0, st>>>(cst, cand, ncand, g);
}
void launch_graph_steps(const double *scal, const int *status, double gamma, double *g,
                        cudaStream_t st) {
  k_graph_steps<<<1, 32, 0, st>>>(scal, status, gamma, g);
}

// The loop test of the solve graph (options.graph = 2), after each iteration it ran: the host
// loop's own tests at the top of its next iteration, on the new iterate's scalars (the same
// FP64 operations in the same order, so the same decisions) — a failed step (g[8]), a failed
// factorisation of Y or of a clique block of X̄ (status words 0 and 1), a non-finite scalar,
// convergence (relative gap and primal residual), or the iteration limit (cnt[1] iterations in
// this launch) — ends the loop.  cnt[0] counts the iterations run.
__global__ void k_graph_cond(cudaGraphConditionalHandle h, const double *__restrict__ scal,
                             const int *__restrict__ status, const double *__restrict__ g,
                             int *cnt, int n, double gap_tol, double feas_tol) {
  if (threadIdx.x != 0) return;
  const int k = ++cnt[0];
  const double mu = scal[0] / n, pobj = scal[1], dobj = scal[2];
  const double gap = fabs(pobj - dobj) / fmax(1.0, (fabs(pobj) + fabs(dobj)) / 2);
  const double pinf = scal[3] / fmax(1.0, scal[4]);
  const int bad = (status[0] | status[1]) & (ST_NOT_PD | ST_TIMEOUT | ST_NUMERIC);
  const bool stop = g[8] != 0.0 || bad != 0 || !isfinite(pobj) || !isfinite(dobj) ||
                    !isfinite(mu) || (gap <= gap_tol && pinf <= feas_tol) || k >= cnt[1];
  cudaGraphSetConditional(h, stop ? 0u : 1u);
}

void launch_graph_cond(cudaGraphConditionalHandle h, const double *scal, const int *status,
                       const double *g, int *cnt, int n, double gap_tol, double feas_tol,
                       cudaStream_t st) {
  k_graph_cond<<<1, 32, 0, st>>>(h, scal, status, g, cnt, n, gap_tol, feas_tol);
}

// one thread per constraint k: r = b_k - A_k . X̄ - A_k . dX, c = r / (A_k . A_k), dX += c A_k on
// A_k's positions (no other constraint touches them)
__global__ void k_project_primal(DevSym S, const double *__restrict__ X, double *dX) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= S.m) return;
  double ax = 0.0, ad = 0.0, aa = 0.0;
  for (int q = S.con_ptr[k]; q < S.con_ptr[k + 1]; ++q) {
    const double w = S.con_w[q];
    ax = fma(w, X[S.con_off[q]], ax);
    ad = fma(w, dX[S.con_off[q]], ad);
    aa = fma(w, S.con_v[q], aa);
  }
  if (aa == 0.0) return;
  const double cc = (S.b[k] - ax - ad) / aa;
  for (int q = S.con_ptr[k]; q < S.con_ptr[k + 1]; ++q) dX[S.con_off[q]] += cc * S.con_v[q];
}

void launch_project_primal(const DevSym &S, const double *Xbar, double *dX, cudaStream_t st) {
  k_project_primal<<<(S.m + 255) / 256, 256, 0, st>>>(S, Xbar, dX);
}

__global__ void k_set_identity(DevSym S, double *X) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < S.n; j += gridDim.x * blockDim.x) {
    const int t = S.col2sn[j];
    const int nrow = (int)(S.sn_rowptr[t + 1] - S.sn_rowptr[t]);
    const int lc = j - S.sn_col[t];
    X[S.sn_valptr[t] + lc + (int64_t)lc * nrow] = 1.0;
  }
}

void launch_set_identity(const DevSym &S, double *X, cudaStream_t st) {
  k_set_identity<<<(S.n + 255) / 256, 256, 0, st>>>(S, X);
}

}  // namespace mcsdp

namespace mcsdp {

// ---------------------------------------------------------------------------------------------
// Differentiation of the central-path point (mcsdp_backward)

// Wout[i][j] = sum_l D_il Win[l][j] for the symmetric D stored on lower(E) in the layout:
// row i's strict-lower entries (rs_* lists) and column i's entries on and below the diagonal
__global__ void k_E_times(DevSym S, const double *__restrict__ D, const double *__restrict__ Win,
                          double *Wout, int64_t ldw, int nc) {
  const int i = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nc) return;
  double acc = 0.0;
  for (int q = S.rs_ptr[i]; q < S.rs_ptr[i + 1]; ++q)
    acc = fma(D[S.rs_off[q]], Win[(int64_t)S.rs_col[q] * ldw + j], acc);
  const int t = S.col2sn[i];
  const int64_t r0 = S.sn_rowptr[t];
  const int nrow = (int)(S.sn_rowptr[t + 1] - r0);
  const int lc = i - S.sn_col[t];
  const int64_t base = S.sn_valptr[t] + (int64_t)lc * nrow;
  for (int p = lc; p < nrow; ++p) acc = fma(D[base + p], Win[(int64_t)S.rows[r0 + p] * ldw + j], acc);
  Wout[(int64_t)i * ldw + j] = acc;
}

void launch_E_times(const DevSym &S, const double *D, const double *Win, double *Wout, int64_t ldw,
                    int nc, cudaStream_t st) {
  if (nc <= 0) return;
  dim3 grid((nc + 127) / 128, S.n);
  k_E_times<<<grid, 128, 0, st>>>(S, D, Win, Wout, ldw, nc);
}

// out = the symmetric matrix whose entries on lower(E) dotted with a symmetric X give the layout
// dot product sum g . X: off-diagonal layout values halved (they stand for both triangles), the
// diagonal kept; positions of the layout above a supernode's diagonal set to zero
__global__ void k_layout_sym(DevSym S, const double *__restrict__ g, double *out) {
  const int t = blockIdx.x;
  const int64_t v0 = S.sn_valptr[t];
  const int nrow = (int)(S.sn_rowptr[t + 1] - S.sn_rowptr[t]);
  const int ncol = S.sn_col[t + 1] - S.sn_col[t];
  for (int e = threadIdx.x; e < nrow * ncol; e += blockDim.x) {
    const int p = e % nrow, lc = e / nrow;
    out[v0 + e] = p == lc ? g[v0 + e] : (p > lc ? 0.5 * g[v0 + e] : 0.0);
  }
}

void launch_layout_sym(const DevSym &S, const double *g, double *out, cudaStream_t st) {
  k_layout_sym<<<S.ns, 128, 0, st>>>(S, g, out);
}

// out = sym(M) on lower(E) from M's lower (Mlow) and transposed (Mup) entries on E
__global__ void k_sym_combine(DevSym S, const double *__restrict__ Mlow,
                              const double *__restrict__ Mup, double *out) {
  const int t = blockIdx.x;
  const int64_t v0 = S.sn_valptr[t];
  const int nrow = (int)(S.sn_rowptr[t + 1] - S.sn_rowptr[t]);
  const int ncol = S.sn_col[t + 1] - S.sn_col[t];
  for (int e = threadIdx.x; e < nrow * ncol; e += blockDim.x) {
    const int p = e % nrow, lc = e / nrow;
    out[v0 + e] = p == lc ? Mlow[v0 + e] : (p > lc ? 0.5 * (Mlow[v0 + e] + Mup[v0 + e]) : 0.0);
  }
}

void launch_sym_combine(const DevSym &S, const double *Mlow, const double *Mup, double *out,
                        cudaStream_t st) {
  k_sym_combine<<<S.ns, 128, 0, st>>>(S, Mlow, Mup, out);
}

// y = a x + y on n entries
__global__ void k_axpy(int64_t n, double a, const double *__restrict__ x, double *y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fma(a, x[i], y[i]);
}
void launch_axpy(int64_t n, double a, const double *x, double *y, cudaStream_t st) {
  int blocks = (int)std::min<int64_t>(4096, (n + 255) / 256);
  if (blocks > 0) k_axpy<<<blocks, 256, 0, st>>>(n, a, x, y);
}

// out[k] = A_k . M + add[k] (caller order) for M on the layout
__global__ void k_con_apply(DevSym S, const double *__restrict__ M, const double *__restrict__ add,
                            double *out) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < S.m; k += gridDim.x * blockDim.x) {
    double a = 0.0;
    for (int q = S.con_ptr[k]; q < S.con_ptr[k + 1]; ++q) a = fma(S.con_w[q], M[S.con_off[q]], a);
    out[k] = add ? a + add[k] : a;
  }
}
void launch_con_apply(const DevSym &S, const double *M, const double *add, double *out,
                      cudaStream_t st) {
  k_con_apply<<<(S.m + 255) / 256, 256, 0, st>>>(S, M, add, out);
}

// row m of B (row S.bord[i] for a block-diagonal B) <- rhs (caller order) in the internal
// constraint order
__global__ void k_border_from_user(DevSym S, double *B, int64_t ldb, const double *__restrict__ rhs) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S.m; i += gridDim.x * blockDim.x)
    B[(S.bord ? S.bord[i] : S.m) + (int64_t)i * ldb] = rhs[S.con_order[i]];
}
void launch_border_from_user(const DevSym &S, double *B, int64_t ldb, const double *rhs,
                             cudaStream_t st) {
  k_border_from_user<<<(S.m + 255) / 256, 256, 0, st>>>(S, B, ldb, rhs);
}

// per stored input entry e: gradient f_e g_{A_k}[off_e] with g_{A_0} = gA0 and
// g_{A_k} = -z_k gA0 - v_k X (k >= 1); f_e = 2 for an off-diagonal entry (it sets both
// triangles), with the sign of the input form for matrix 0
__global__ void k_entry_grads(int64_t nnz, const int64_t *__restrict__ off, const int *__restrict__ kk,
                              const int *__restrict__ pos, const double *__restrict__ f,
                              const double *__restrict__ gA0, const double *__restrict__ X,
                              const double *__restrict__ z, const double *__restrict__ v,
                              double *gC, double *gA) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int k = kk[e];
    const double g0 = gA0[off[e]];
    if (k == 0) {
      if (gC) gC[pos[e]] = f[e] * g0;
    } else if (gA) {
      gA[pos[e]] = f[e] * (-z[k - 1] * g0 - v[k - 1] * X[off[e]]);
    }
  }
}
void launch_entry_grads(int64_t nnz, const int64_t *off, const int *k, const int *pos,
                        const double *f, const double *gA0, const double *X, const double *z,
                        const double *v, double *gC, double *gA, cudaStream_t st) {
  int blocks = (int)std::min<int64_t>(4096, (nnz + 255) / 256);
  if (blocks > 0) k_entry_grads<<<blocks, 256, 0, st>>>(nnz, off, k, pos, f, gA0, X, z, v, gC, gA);
}

}  // namespace mcsdp
