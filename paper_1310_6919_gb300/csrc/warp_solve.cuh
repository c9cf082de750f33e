// Supernodal triangular solves, type (iv)/(v) of Sec. 3.1: forward/backward substitution with L̂
// or N stored in the supernodal layout (supernode s = column-major nrow x ncol block, rows =
// clique C_s), many right-hand sides at once.
//
// A CTA of several warps walks one supernode sequence; each warp owns one right-hand side W (a
// dense n-vector in shared memory when it fits, else global memory) and no other warp touches it,
// so within a step only __syncwarp is needed.  The factor block, the inverse of its diagonal block
// and its row indices are staged once per CTA into shared memory with cp.async, double buffered,
// so the next supernode's blocks load while the current one is processed.
#pragma once
#include "internal.h"

namespace mcsdp {

constexpr int WS_MAX_ROWS_PER_LANE = 3;  // supernodes of up to 96 columns

// dot product of a strided row of a matrix with a dense vector, four independent accumulators
// (breaks the dependent FMA chain); M[k * ms] * v[k] for k in [k0, k1)
__device__ __forceinline__ double dot4(const double *M, int ms, const double *v, int k0, int k1) {
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int k = k0;
  for (; k + 3 < k1; k += 4) {
    a0 = fma(M[k * ms], v[k], a0);
    a1 = fma(M[(k + 1) * ms], v[k + 1], a1);
    a2 = fma(M[(k + 2) * ms], v[k + 2], a2);
    a3 = fma(M[(k + 3) * ms], v[k + 3], a3);
  }
  for (; k < k1; ++k) a0 = fma(M[k * ms], v[k], a0);
  return (a0 + a1) + (a2 + a3);
}

// same with an index-gathered vector v[idx[k]]
__device__ __forceinline__ double dot4g(const double *M, int ms, const double *v, const int *idx,
                                        int k0, int k1) {
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int k = k0;
  for (; k + 3 < k1; k += 4) {
    a0 = fma(M[k * ms], v[idx[k]], a0);
    a1 = fma(M[(k + 1) * ms], v[idx[k + 1]], a1);
    a2 = fma(M[(k + 2) * ms], v[idx[k + 2]], a2);
    a3 = fma(M[(k + 3) * ms], v[idx[k + 3]], a3);
  }
  for (; k < k1; ++k) a0 = fma(M[k * ms], v[idx[k]], a0);
  return (a0 + a1) + (a2 + a3);
}

// One supernode step for one right-hand side held by a warp in W (shared or global memory).
// Lb = the nrow x ncol block of L (column-major), D = L_SS^{-1} (ncol x ncol, lower,
// column-major), rw = the clique rows; both steps are lane-parallel GEMVs.
// forward:  W[S] <- D W[S];  W[U] -= L_US W[S]
__device__ __forceinline__ void warp_fwd_blk(const double *Lb, int nrow, const double *D, int ncol,
                                             const int *rw, int c0, double *W, int lane) {
  double x[WS_MAX_ROWS_PER_LANE];
  const double *ws = W + c0;
#pragma unroll
  for (int q = 0; q < WS_MAX_ROWS_PER_LANE; ++q) {
    const int i = lane + 32 * q;
    x[q] = (i < ncol) ? dot4(D + i, ncol, ws, 0, i + 1) : 0.0;
  }
  __syncwarp();
#pragma unroll
  for (int q = 0; q < WS_MAX_ROWS_PER_LANE; ++q)
    if (lane + 32 * q < ncol) W[c0 + lane + 32 * q] = x[q];
  __syncwarp();
  for (int p = ncol + lane; p < nrow; p += 32) W[rw[p]] -= dot4(Lb + p, nrow, ws, 0, ncol);
  __syncwarp();
}

// backward: W[S] -= L_US^T W[U];  W[S] <- D^T W[S].
// transposed = true: Lb holds L^T (ncol x nrow, column-major, i.e. Lb[j + p*ncol] = L[p][j]) and
// D holds D^T, the layout staged for this pass so that lanes read consecutive words.
__device__ __forceinline__ void warp_bwd_blk(const double *Lb, int nrow, const double *D, int ncol,
                                             const int *rw, int c0, double *W, int lane,
                                             bool transposed) {
  if (nrow > ncol) {
    for (int j = lane; j < ncol; j += 32) {
      const double acc = transposed ? dot4g(Lb + j, ncol, W, rw, ncol, nrow)
                                    : dot4g(Lb + j * nrow, 1, W, rw, ncol, nrow);
      W[c0 + j] -= acc;
    }
    __syncwarp();
  }
  double x[WS_MAX_ROWS_PER_LANE];
  const double *ws = W + c0;
#pragma unroll
  for (int q = 0; q < WS_MAX_ROWS_PER_LANE; ++q) {
    const int i = lane + 32 * q;
    x[q] = (i < ncol) ? (transposed ? dot4(D + i, ncol, ws, i, ncol) : dot4(D + i * ncol, 1, ws, i, ncol))
                      : 0.0;
  }
  __syncwarp();
#pragma unroll
  for (int q = 0; q < WS_MAX_ROWS_PER_LANE; ++q)
    if (lane + 32 * q < ncol) W[c0 + lane + 32 * q] = x[q];
  __syncwarp();
}

// ---- CTA-shared staging of supernode blocks (cp.async, double buffered) ----
__device__ __forceinline__ void cp_async8(void *smem_dst, const void *gsrc) {
  unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc));
}
__device__ __forceinline__ void cp_async4(void *smem_dst, const void *gsrc) {
  unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all_but1() {
  asm volatile("cp.async.wait_group 1;\n" ::);
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

// Stage buffer: [cap doubles of L][cap_d doubles of D][cap_r ints of rows]
struct Stage {
  double *L;
  double *D;
  int *R;
  int cap, cap_d, cap_r;
};

// Supernode descriptor, loaded ahead of use so that its global-memory latency overlaps the
// previous step.
struct SnD {
  int s, c0, ncol, nrow;
  int64_t v0, d0, r0;
};

__device__ __forceinline__ SnD load_desc(const DevSym &S, int s) {
  SnD d;
  d.s = s;
  if (s < 0) {
    d.c0 = d.ncol = d.nrow = 0;
    d.v0 = d.d0 = d.r0 = 0;
    return d;
  }
  d.c0 = S.sn_col[s];
  d.ncol = S.sn_col[s + 1] - d.c0;
  d.r0 = S.sn_rowptr[s];
  d.nrow = (int)(S.sn_rowptr[s + 1] - d.r0);
  d.v0 = S.sn_valptr[s];
  d.d0 = S.sn_dptr[s];
  return d;
}

__device__ __forceinline__ bool stage_fits(const SnD &d, const Stage &st) {
  return d.nrow * d.ncol <= st.cap && d.ncol * d.ncol <= st.cap_d && d.nrow <= st.cap_r;
}

// Copies the blocks of a supernode into the stage (transposed for backward passes).
template <bool FWD>
__device__ __forceinline__ void stage_issue(const DevSym &S, const double *L, const double *Dall,
                                            const SnD &d, const Stage &st) {
  if (d.s < 0 || !stage_fits(d, st)) return;
  const double *gL = L + d.v0;
  const double *gD = Dall + d.d0;
  const int *gR = S.rows + d.r0;
  const int nr = d.nrow, nc = d.ncol;
  for (int i = threadIdx.x; i < nr * nc; i += blockDim.x) {
    const int p = i % nr, j = i / nr;
    cp_async8(st.L + (FWD ? i : j + p * nc), gL + i);
  }
  for (int i = threadIdx.x; i < nc * nc; i += blockDim.x) {
    const int a = i % nc, b = i / nc;
    cp_async8(st.D + (FWD ? i : b + a * nc), gD + i);
  }
  for (int i = threadIdx.x; i < nr; i += blockDim.x) cp_async4(st.R + i, gR + i);
}

// One pass over a supernode sequence for every warp of the CTA (each warp owns W_warp).
// it.first() / it.next(cur) enumerate the supernodes (-1 at the end); every thread of the CTA
// walks the same sequence.  Descriptors are loaded two steps ahead, blocks staged one step ahead.
template <bool FWD, class It>
__device__ void cta_pass(const DevSym &S, const double *L, const double *Dall, double *W,
                         Stage st[2], It it, int lane, bool active) {
  SnD d0 = load_desc(S, it.first());
  if (d0.s < 0) return;
  SnD d1 = load_desc(S, it.next(d0.s));
  int b = 0;
  stage_issue<FWD>(S, L, Dall, d0, st[0]);
  cp_async_commit();
  while (d0.s >= 0) {
    const SnD d2 = load_desc(S, d1.s >= 0 ? it.next(d1.s) : -1);
    stage_issue<FWD>(S, L, Dall, d1, st[b ^ 1]);
    cp_async_commit();
    cp_async_wait_all_but1();
    __syncthreads();
    if (active) {
      const bool staged = stage_fits(d0, st[b]);
      const double *Lb = staged ? st[b].L : L + d0.v0;
      const double *Db = staged ? st[b].D : Dall + d0.d0;
      const int *rw = staged ? st[b].R : S.rows + d0.r0;
      if (FWD) warp_fwd_blk(Lb, d0.nrow, Db, d0.ncol, rw, d0.c0, W, lane);
      else warp_bwd_blk(Lb, d0.nrow, Db, d0.ncol, rw, d0.c0, W, lane, staged);
    }
    __syncthreads();
    d0 = d1;
    d1 = d2;
    b ^= 1;
  }
  cp_async_wait_all();
}

__device__ __forceinline__ void stage_setup(Stage st[2], unsigned char *base, int cap, int cap_d,
                                            int cap_r) {
  for (int b = 0; b < 2; ++b) {
    st[b].L = reinterpret_cast<double *>(base);
    base += (size_t)cap * 8;
    st[b].D = reinterpret_cast<double *>(base);
    base += (size_t)cap_d * 8;
    st[b].R = reinterpret_cast<int *>(base);
    base += ((size_t)cap_r * 4 + 15) / 16 * 16;
    st[b].cap = cap;
    st[b].cap_d = cap_d;
    st[b].cap_r = cap_r;
  }
}

__host__ __device__ inline size_t stage_bytes(int cap, int cap_d, int cap_r) {
  return 2 * ((size_t)cap * 8 + (size_t)cap_d * 8 + ((size_t)cap_r * 4 + 15) / 16 * 16);
}

// sequences
struct SeqList {  // an explicit list, ascending or descending
  const int *v;
  int64_t n, i;
  bool rev;
  __device__ int at(int64_t k) const { return k < n ? v[rev ? n - 1 - k : k] : -1; }
  __device__ int first() { i = 0; return at(0); }
  __device__ int next(int) { ++i; return at(i); }
};
struct SeqAll {  // every supernode, ascending or descending
  int ns;
  bool rev;
  __device__ int first() const { return ns > 0 ? (rev ? ns - 1 : 0) : -1; }
  __device__ int next(int cur) const { return rev ? cur - 1 : (cur + 1 < ns ? cur + 1 : -1); }
};

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
  const int i = hi - ns, j = lo - ns;
  (void)r0;
  return X[S.cmap_off[S.cmap_ptr[r] + (int64_t)i * (i + 1) / 2 + j]];
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
