// Level-scheduled supernodal triangular solves for many right-hand sides at once (type (iv)/(v)
// of Sec. 3.1: forward/backward substitution with L̂ or N in the supernodal layout).
//
// The right-hand sides are the columns of a row-major n x ldw matrix W.  One launch handles one
// level of the supernodal elimination tree for every right-hand side: CTA = (supernode t of the
// level, tile of 32 right-hand sides), one lane per right-hand side, so every factor entry is
// loaded once per CTA (a broadcast) and reused by 32 columns, and every access to W is one
// coalesced 256-byte row segment.
//   forward  (levels bottom-up, left-looking): W[S_t] -= sum over descendants d that update t of
//            L_d[rows in S_t, :] W[S_d];  W[S_t] <- D_t W[S_t]
//   backward (levels top-down):  W[S_t] -= L_{U_t S_t}^T W[U_t];  W[S_t] <- D_t^T W[S_t]
// Each CTA writes only the rows S_t of its own supernode, so no two CTAs of a launch touch the
// same entry.  D_t = L_{S_t S_t}^{-1} is written by the factorisation kernels.
// Optional skip bitmaps drop (supernode, tile) pairs whose right-hand sides are zero there
// (forward reach of unit columns) or whose result is not needed (backward).
#include <cuda_runtime.h>

#include "internal.h"

namespace mcsdp {

constexpr int LS_CH = 8;

__device__ __forceinline__ bool ls_skip(const LsSkip &sk, int t, int tile) {
  if (!sk.bits) return false;
  const int2 kr = sk.tile_keys[tile];
  for (int key = kr.x; key <= kr.y; ++key)
    if (sk.bits[(int64_t)key * sk.words + (t >> 5)] & (1u << (t & 31))) return false;
  return true;
}

// acc[c][lane] -= sum over updates [ub, ue) of target t of L_d[rows in S_t, :] W[S_d]
__device__ __forceinline__ void lfwd_pull(const DevSym &S, int ub, int ue, const double *L,
                                          const double *Wc, int64_t ldw, bool act, double *acc,
                                          int lane) {
  for (int u = ub; u < ue; ++u) {
    const int d = S.upd_src[u], p1 = S.upd_p1[u], p2 = S.upd_p2[u];
    const int *rel = S.upd_rel + S.upd_relptr[u];
    const int dc0 = S.sn_col[d];
    const int dncol = S.sn_col[d + 1] - dc0;
    const int dnrow = (int)(S.sn_rowptr[d + 1] - S.sn_rowptr[d]);
    const double *Ld = L + S.sn_valptr[d];
    for (int j0 = 0; j0 < dncol; j0 += LS_CH) {
      const int cw = dncol - j0 < LS_CH ? dncol - j0 : LS_CH;
      double x[LS_CH];
#pragma unroll
      for (int q = 0; q < LS_CH; ++q) x[q] = (q < cw && act) ? Wc[(int64_t)(dc0 + j0 + q) * ldw] : 0.0;
      const double *base = Ld + (int64_t)j0 * dnrow;
      for (int p = p1; p < p2; ++p) {
        double a = 0.0;
#pragma unroll
        for (int q = 0; q < LS_CH; ++q)
          if (q < cw) a = fma(base[p + (int64_t)q * dnrow], x[q], a);
        acc[rel[p - p1] * 32 + lane] -= a;
      }
    }
  }
}

// extra chunks: Pw[slot + c][col] = -(sum over the chunk's updates) for c < ncol_t
__global__ void k_lfwd_partial(DevSym S, int x0, int ntiles, const double *__restrict__ L,
                               const double *__restrict__ W, int64_t ldw, int ncolsW,
                               LsSkip sk, double *Pw) {
  extern __shared__ double acc[];
  const int lane = threadIdx.x;
  const int x = x0 + blockIdx.x / ntiles;
  const int tile = blockIdx.x % ntiles;
  const int t = S.xch_t[x];
  if (ls_skip(sk, t, tile)) return;
  const int col = tile * 32 + lane;
  const bool act = col < ncolsW;
  const int ncol = S.sn_col[t + 1] - S.sn_col[t];
  for (int c = 0; c < ncol; ++c) acc[c * 32 + lane] = 0.0;
  lfwd_pull(S, S.xch_ub[x], S.xch_ue[x], L, W + (act ? col : 0), ldw, act, acc, lane);
  double *P = Pw + S.xch_slotw[x] * ldw + (act ? col : 0);
  if (act)
    for (int c = 0; c < ncol; ++c) P[(int64_t)c * ldw] = acc[c * 32 + lane];
}

__global__ void k_lfwd(DevSym S, int lvl_begin, int ntiles, const double *__restrict__ L,
                       const double *__restrict__ Dall, double *W, int64_t ldw, int ncolsW,
                       LsSkip sk, const double *__restrict__ Pw) {
  extern __shared__ double acc[];  // [ncol][32]
  const int lane = threadIdx.x;
  const int t = S.lvl_sn[lvl_begin + blockIdx.x / ntiles];
  const int tile = blockIdx.x % ntiles;
  if (ls_skip(sk, t, tile)) return;
  const int col = tile * 32 + lane;
  const bool act = col < ncolsW;
  const int c0 = S.sn_col[t];
  const int ncol = S.sn_col[t + 1] - c0;
  double *Wc = W + (act ? col : 0);
  for (int c = 0; c < ncol; ++c) acc[c * 32 + lane] = act ? Wc[(int64_t)(c0 + c) * ldw] : 0.0;
  lfwd_pull(S, S.upd_ptr[t], S.upd_c0end[t], L, Wc, ldw, act, acc, lane);
  for (int x = S.xch_beg[t]; x < S.xch_end[t]; ++x) {
    const double *P = Pw + S.xch_slotw[x] * ldw + (act ? col : 0);
    for (int c = 0; c < ncol; ++c) acc[c * 32 + lane] += act ? P[(int64_t)c * ldw] : 0.0;
  }
  const double *D = Dall + S.sn_dptr[t];
  for (int i = 0; i < ncol; ++i) {
    double a0 = 0.0, a1 = 0.0;
    int j = 0;
    for (; j + 1 <= i; j += 2) {
      a0 = fma(D[i + j * ncol], acc[j * 32 + lane], a0);
      a1 = fma(D[i + (j + 1) * ncol], acc[(j + 1) * 32 + lane], a1);
    }
    if (j <= i) a0 = fma(D[i + j * ncol], acc[j * 32 + lane], a0);
    if (act) Wc[(int64_t)(c0 + i) * ldw] = a0 + a1;
  }
}

__global__ void k_lbwd(DevSym S, int lvl_begin, int ntiles, const double *__restrict__ L,
                       const double *__restrict__ Dall, double *W, int64_t ldw, int ncolsW,
                       LsSkip sk) {
  extern __shared__ double acc[];  // [ncol][32]
  const int lane = threadIdx.x;
  const int t = S.lvl_sn[lvl_begin + blockIdx.x / ntiles];
  const int tile = blockIdx.x % ntiles;
  if (ls_skip(sk, t, tile)) return;
  const int col = tile * 32 + lane;
  const bool act = col < ncolsW;
  const int c0 = S.sn_col[t];
  const int ncol = S.sn_col[t + 1] - c0;
  const int64_t r0 = S.sn_rowptr[t];
  const int nrow = (int)(S.sn_rowptr[t + 1] - r0);
  const int *rw = S.rows + r0;
  const double *Lt = L + S.sn_valptr[t];
  double *Wc = W + (act ? col : 0);
  for (int j0 = 0; j0 < ncol; j0 += LS_CH) {
    const int cw = ncol - j0 < LS_CH ? ncol - j0 : LS_CH;
    double a[LS_CH];
#pragma unroll
    for (int q = 0; q < LS_CH; ++q) a[q] = (q < cw && act) ? Wc[(int64_t)(c0 + j0 + q) * ldw] : 0.0;
    const double *base = Lt + (int64_t)j0 * nrow;
    int p = ncol;
    for (; p + 1 < nrow; p += 2) {
      const double w0 = act ? Wc[(int64_t)rw[p] * ldw] : 0.0;
      const double w1 = act ? Wc[(int64_t)rw[p + 1] * ldw] : 0.0;
#pragma unroll
      for (int q = 0; q < LS_CH; ++q)
        if (q < cw) {
          a[q] = fma(-base[p + (int64_t)q * nrow], w0, a[q]);
          a[q] = fma(-base[p + 1 + (int64_t)q * nrow], w1, a[q]);
        }
    }
    for (; p < nrow; ++p) {
      const double w0 = act ? Wc[(int64_t)rw[p] * ldw] : 0.0;
#pragma unroll
      for (int q = 0; q < LS_CH; ++q)
        if (q < cw) a[q] = fma(-base[p + (int64_t)q * nrow], w0, a[q]);
    }
#pragma unroll
    for (int q = 0; q < LS_CH; ++q)
      if (q < cw) acc[(j0 + q) * 32 + lane] = a[q];
  }
  const double *D = Dall + S.sn_dptr[t];
  for (int i = 0; i < ncol; ++i) {
    const double *di = D + i * ncol;  // D[j][i] = di[j]
    double a0 = 0.0, a1 = 0.0;
    int j = i;
    for (; j + 1 < ncol; j += 2) {
      a0 = fma(di[j], acc[j * 32 + lane], a0);
      a1 = fma(di[j + 1], acc[(j + 1) * 32 + lane], a1);
    }
    if (j < ncol) a0 = fma(di[j], acc[j * 32 + lane], a0);
    if (act) Wc[(int64_t)(c0 + i) * ldw] = a0 + a1;
  }
}

int lsolve(const DevSym &S, const int *lvl_ptr_host, const int *lvl_xptr_host, int height, bool fwd,
           const double *L, const double *D, double *W, int64_t ldw, int ncolsW, const LsSkip &sk,
           double *Pw, cudaStream_t st) {
  if (ncolsW <= 0) return 0;
  const int ntiles = (ncolsW + 31) / 32;
  const size_t smem = (size_t)S.max_ncol * 32 * 8;
  static size_t configured = 0;
  if (smem > 48 * 1024 && smem > configured) {
    cudaFuncSetAttribute(k_lfwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_lbwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_lfwd_partial, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    configured = smem;
  }
  int launches = 0;
  for (int li = 0; li < height; ++li) {
    const int l = fwd ? li : height - 1 - li;
    const int b = lvl_ptr_host[l], cnt = lvl_ptr_host[l + 1] - b;
    const int64_t blocks = (int64_t)cnt * ntiles;
    if (blocks <= 0) continue;
    if (fwd) {
      const int xb = lvl_xptr_host[l], xc = lvl_xptr_host[l + 1] - xb;
      if (xc > 0) {
        k_lfwd_partial<<<(unsigned)((int64_t)xc * ntiles), 32, smem, st>>>(S, xb, ntiles, L, W, ldw,
                                                                           ncolsW, sk, Pw);
        ++launches;
      }
      k_lfwd<<<(unsigned)blocks, 32, smem, st>>>(S, b, ntiles, L, D, W, ldw, ncolsW, sk, Pw);
    }
    else k_lbwd<<<(unsigned)blocks, 32, smem, st>>>(S, b, ntiles, L, D, W, ldw, ncolsW, sk);
    ++launches;
  }
  return launches;
}

// W[rowof[j] * ldw + j] = 1 for the unit right-hand sides (W zeroed before)
__global__ void k_rhs_unit(double *W, int64_t ldw, const int *rowof, int nrhs) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < nrhs) W[(int64_t)rowof[j] * ldw + j] = 1.0;
}

void launch_rhs_unit(double *W, int64_t ldw, const int *rowof, int nrhs, cudaStream_t st) {
  if (nrhs > 0) k_rhs_unit<<<(nrhs + 255) / 256, 256, 0, st>>>(W, ldw, rowof, nrhs);
}

}  // namespace mcsdp
