// Warp-level supernodal triangular solves with one right-hand side per warp.
//
// Type (iv)/(v) of Sec. 3.1: forward/backward substitution with L̂ or N stored in the supernodal
// layout (supernode s = column-major nrow x ncol block, rows = clique C_s).  One warp owns one
// dense n-vector W (shared or global memory) and walks the supernodes; no other warp touches W,
// so the only synchronisation is __syncwarp.  Within a supernode the ncol x ncol diagonal block is
// solved column by column (lanes over rows) and the off-diagonal block is a lane-parallel GEMV.
#pragma once
#include "internal.h"

namespace mcsdp {

// W[S_s] <- L_SS^{-1} W[S_s];  W[U_s] -= L_US W[S_s]
__device__ __forceinline__ void warp_fwd_sn(const DevSym &S, const double *__restrict__ L,
                                            const double *__restrict__ dinv, double *W, int s,
                                            int lane) {
  const int c0 = S.sn_col[s];
  const int ncol = S.sn_col[s + 1] - c0;
  const int64_t r0 = S.sn_rowptr[s];
  const int nrow = (int)(S.sn_rowptr[s + 1] - r0);
  const double *Ls = L + S.sn_valptr[s];
  const int *rw = S.rows + r0;
  for (int j = 0; j < ncol; ++j) {
    const double xj = W[c0 + j] * dinv[c0 + j];
    __syncwarp();
    if (lane == 0) W[c0 + j] = xj;
    const double *col = Ls + (int64_t)j * nrow;
    for (int i = j + 1 + lane; i < ncol; i += 32) W[c0 + i] -= col[i] * xj;
    __syncwarp();
  }
  for (int p = ncol + lane; p < nrow; p += 32) {
    double acc = 0.0;
    for (int j = 0; j < ncol; ++j) acc = fma(Ls[p + (int64_t)j * nrow], W[c0 + j], acc);
    W[rw[p]] -= acc;
  }
  __syncwarp();
}

// W[S_s] -= L_US^T W[U_s];  W[S_s] <- L_SS^{-T} W[S_s]
__device__ __forceinline__ void warp_bwd_sn(const DevSym &S, const double *__restrict__ L,
                                            const double *__restrict__ dinv, double *W, int s,
                                            int lane) {
  const int c0 = S.sn_col[s];
  const int ncol = S.sn_col[s + 1] - c0;
  const int64_t r0 = S.sn_rowptr[s];
  const int nrow = (int)(S.sn_rowptr[s + 1] - r0);
  const double *Ls = L + S.sn_valptr[s];
  const int *rw = S.rows + r0;
  if (nrow > ncol) {
    for (int j = lane; j < ncol; j += 32) {
      const double *col = Ls + (int64_t)j * nrow;
      double acc = 0.0;
      for (int p = ncol; p < nrow; ++p) acc = fma(col[p], W[rw[p]], acc);
      W[c0 + j] -= acc;
    }
    __syncwarp();
  }
  for (int j = ncol - 1; j >= 0; --j) {
    const double xj = W[c0 + j] * dinv[c0 + j];
    __syncwarp();
    if (lane == 0) W[c0 + j] = xj;
    for (int i = lane; i < j; i += 32) W[c0 + i] -= Ls[j + (int64_t)i * nrow] * xj;
    __syncwarp();
  }
}

__device__ __forceinline__ int64_t layout_offset(const DevSym &S, int r, int c) {
  // position of lower entry (r >= c, new indices) in the layout
  const int t = S.col2sn[c];
  const int64_t r0 = S.sn_rowptr[t];
  const int nrow = (int)(S.sn_rowptr[t + 1] - r0);
  const int lc = c - S.sn_col[t];
  int lo = lc, hi = nrow - 1;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (S.rows[r0 + mid] < r) lo = mid + 1;
    else hi = mid;
  }
  return S.sn_valptr[t] + lo + (int64_t)lc * nrow;
}

// value of X̄ at local positions (a, b) of clique r (a, b < nrow_r)
__device__ __forceinline__ double clique_entry(const DevSym &S, const double *X, int r, int a,
                                               int b) {
  const int64_t r0 = S.sn_rowptr[r];
  const int k = (int)(S.sn_rowptr[r + 1] - r0);
  const int ns = S.sn_col[r + 1] - S.sn_col[r];
  const int hi = a > b ? a : b, lo = a > b ? b : a;
  if (lo < ns) return X[S.sn_valptr[r] + hi + (int64_t)lo * k];
  return X[layout_offset(S, S.rows[r0 + hi], S.rows[r0 + lo])];
}

__device__ __forceinline__ double block_reduce_sum(double v, double *red) {
  // deterministic: fixed shuffle tree then fixed-order sum of warp partials
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  const int nw = (blockDim.x + 31) >> 5;
  for (int i = 0; i < nw; ++i) s += red[i];
  __syncthreads();
  return s;
}

}  // namespace mcsdp
