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

#include <algorithm>

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

// acc[c][lane] -= sum over updates [ub, ue) of target t of L_d[rows in S_t, :] W[S_d].
// Each update block L_d[p1:p2, j0:j0+8] is loaded by the 32 lanes together into the warp's stage
// (one memory round trip), the 8 source values per lane in parallel with it.
// one chunk of CW source columns: acc[srel[p]] -= sum_q stg[q][p] x[q]  (exact width, so no
// FP64 instruction slot is spent on a predicated-off column)
template <int CW>
__device__ __forceinline__ void lfwd_chunk(const double *Wc, int64_t ldw, bool act, int dc0j,
                                           const double *base, int dnrow, int np, double *acc,
                                           double *stg, const int *srel, int lane) {
  double x[CW];
#pragma unroll
  for (int q = 0; q < CW; ++q) x[q] = act ? Wc[(int64_t)(dc0j + q) * ldw] : 0.0;
  for (int e = lane; e < np * CW; e += 32) {
    const int p = e % np, q = e / np;
    stg[q * np + p] = base[p + (int64_t)q * dnrow];
  }
  __syncwarp();
  int p = 0;
  for (; p + 1 < np; p += 2) {  // two rows at a time: independent chains
    double a0 = 0.0, a1 = 0.0;
#pragma unroll
    for (int q = 0; q < CW; ++q) {
      a0 = fma(stg[q * np + p], x[q], a0);
      a1 = fma(stg[q * np + p + 1], x[q], a1);
    }
    const int r0 = srel[p] * 32 + lane, r1 = srel[p + 1] * 32 + lane;
    const double v0 = acc[r0], v1 = acc[r1];
    acc[r0] = v0 - a0;
    acc[r1] = v1 - a1;
  }
  if (p < np) {
    double a0 = 0.0;
#pragma unroll
    for (int q = 0; q < CW; ++q) a0 = fma(stg[q * np + p], x[q], a0);
    acc[srel[p] * 32 + lane] -= a0;
  }
  __syncwarp();
}

__device__ __forceinline__ void lfwd_pull(const DevSym &S, int ub, int ue, const double *L,
                                          const double *Wc, int64_t ldw, bool act, double *acc,
                                          double *stg, int *srel, int lane) {
  for (int u0 = ub; u0 < ue; u0 += 32) {
    // metadata of up to 32 updates, one per lane, then broadcast by shuffles
    int m_p1 = 0, m_np = 0, m_dc0 = 0, m_dncol = 0, m_dnrow = 0;
    int64_t m_rel = 0, m_val = 0;
    if (u0 + lane < ue) {
      const int u = u0 + lane;
      const int d = S.upd_src[u];
      m_p1 = S.upd_p1[u];
      m_np = S.upd_p2[u] - m_p1;
      m_rel = S.upd_relptr[u];
      m_dc0 = S.sn_col[d];
      m_dncol = S.sn_col[d + 1] - m_dc0;
      m_dnrow = (int)(S.sn_rowptr[d + 1] - S.sn_rowptr[d]);
      m_val = S.sn_valptr[d];
    }
    const int cnt = ue - u0 < 32 ? ue - u0 : 32;
    for (int k = 0; k < cnt; ++k) {
      const int p1 = __shfl_sync(0xffffffffu, m_p1, k);
      const int np = __shfl_sync(0xffffffffu, m_np, k);
      const int dc0 = __shfl_sync(0xffffffffu, m_dc0, k);
      const int dncol = __shfl_sync(0xffffffffu, m_dncol, k);
      const int dnrow = __shfl_sync(0xffffffffu, m_dnrow, k);
      const int64_t relp = __shfl_sync(0xffffffffu, m_rel, k);
      const int64_t valp = __shfl_sync(0xffffffffu, m_val, k);
      const int *rel = S.upd_rel + relp;
      const double *Ld = L + valp;
      for (int p = lane; p < np; p += 32) srel[p] = rel[p];
      for (int j0 = 0; j0 < dncol; j0 += LS_CH) {
        const int cw = dncol - j0 < LS_CH ? dncol - j0 : LS_CH;
        const double *base = Ld + (int64_t)j0 * dnrow + p1;
        switch (cw) {
          case 1: lfwd_chunk<1>(Wc, ldw, act, dc0 + j0, base, dnrow, np, acc, stg, srel, lane); break;
          case 2: lfwd_chunk<2>(Wc, ldw, act, dc0 + j0, base, dnrow, np, acc, stg, srel, lane); break;
          case 3: lfwd_chunk<3>(Wc, ldw, act, dc0 + j0, base, dnrow, np, acc, stg, srel, lane); break;
          case 4: lfwd_chunk<4>(Wc, ldw, act, dc0 + j0, base, dnrow, np, acc, stg, srel, lane); break;
          case 5: lfwd_chunk<5>(Wc, ldw, act, dc0 + j0, base, dnrow, np, acc, stg, srel, lane); break;
          case 6: lfwd_chunk<6>(Wc, ldw, act, dc0 + j0, base, dnrow, np, acc, stg, srel, lane); break;
          case 7: lfwd_chunk<7>(Wc, ldw, act, dc0 + j0, base, dnrow, np, acc, stg, srel, lane); break;
          default: lfwd_chunk<8>(Wc, ldw, act, dc0 + j0, base, dnrow, np, acc, stg, srel, lane); break;
        }
      }
    }
  }
}

// extra chunks: Pw[slot + c][col] = -(sum over the chunk's updates) for c < ncol_t
__global__ void k_lfwd_partial(DevSym S, int x0, int ntiles, const double *__restrict__ L,
                               const double *__restrict__ W, int64_t ldw, int ncolsW,
                               LsSkip sk, double *Pw) {
  extern __shared__ double acc[];
  double *stg = acc + S.max_ncol * 32;
  int *srel = reinterpret_cast<int *>(stg + LS_CH * S.max_nrow);
  const int lane = threadIdx.x;
  const int x = x0 + blockIdx.x / ntiles;
  const int tile = blockIdx.x % ntiles;
  const int t = S.xch_t[x];
  if (ls_skip(sk, t, tile)) return;
  const int col = tile * 32 + lane;
  const bool act = col < ncolsW;
  const int ncol = S.sn_col[t + 1] - S.sn_col[t];
  for (int c = 0; c < ncol; ++c) acc[c * 32 + lane] = 0.0;
  lfwd_pull(S, S.xch_ub[x], S.xch_ue[x], L, W + (act ? col : 0), ldw, act, acc, stg, srel, lane);
  double *P = Pw + S.xch_slotw[x] * ldw + (act ? col : 0);
  if (act)
    for (int c = 0; c < ncol; ++c) P[(int64_t)c * ldw] = acc[c * 32 + lane];
}

// W[S_t] += sum of the partial slots of t (in chunk order), one thread per (row of S_t, column),
// for every target of the level that has extra update chunks (grid row y = chunk index; only
// the first chunk of each target does the work)
__global__ void k_lfwd_reduce(DevSym S, int x0, int nx, const double *__restrict__ Pw, double *W,
                              int64_t ldw, int ncolsW, LsSkip sk) {
  const int x = x0 + blockIdx.y;
  if (x >= x0 + nx) return;
  const int t = S.xch_t[x];
  if (S.xch_beg[t] != x) return;
  const int c0 = S.sn_col[t];
  const int ncol = S.sn_col[t + 1] - c0;
  const int xb = S.xch_beg[t], xe = S.xch_end[t];
  const int64_t tot = (int64_t)ncol * ncolsW;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e / ncolsW), col = (int)(e % ncolsW);
    if (ls_skip(sk, t, col / 32)) continue;
    double sacc = 0.0;
    for (int xx = xb; xx < xe; ++xx) sacc += Pw[(S.xch_slotw[xx] + c) * ldw + col];
    W[(int64_t)(c0 + c) * ldw + col] += sacc;
  }
}

__global__ void k_lfwd(DevSym S, int lvl_begin, int ntiles, const double *__restrict__ L,
                       const double *__restrict__ Dall, double *W, int64_t ldw, int ncolsW,
                       LsSkip sk, const double *__restrict__ Pw) {
  extern __shared__ double acc[];  // [ncol][32], then the update stage
  double *stg = acc + S.max_ncol * 32;
  int *srel = reinterpret_cast<int *>(stg + LS_CH * S.max_nrow);
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
  lfwd_pull(S, S.upd_ptr[t], S.upd_c0end[t], L, Wc, ldw, act, acc, stg, srel, lane);
  // the extra chunks of t were already added to W[S_t] by k_lfwd_reduce
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

// a[q] = W[c0j + q] - sum_{p >= ncol} L[p][j0 + q] W[rw[p]] for the CW columns of one chunk,
// stored in acc[q][lane]
template <int CW>
__device__ __forceinline__ void lbwd_chunk(const double *Wc, int64_t ldw, bool act, int c0j,
                                           const double *base, int nrow, int ncol, const int *rw,
                                           double *acc, int lane) {
  double a[CW], b[CW];  // two independent chains per column (even / odd rows)
#pragma unroll
  for (int q = 0; q < CW; ++q) {
    a[q] = act ? Wc[(int64_t)(c0j + q) * ldw] : 0.0;
    b[q] = 0.0;
  }
  int p = ncol;
  for (; p + 3 < nrow; p += 4) {
    const double w0 = act ? Wc[(int64_t)rw[p] * ldw] : 0.0;
    const double w1 = act ? Wc[(int64_t)rw[p + 1] * ldw] : 0.0;
    const double w2 = act ? Wc[(int64_t)rw[p + 2] * ldw] : 0.0;
    const double w3 = act ? Wc[(int64_t)rw[p + 3] * ldw] : 0.0;
#pragma unroll
    for (int q = 0; q < CW; ++q) {
      a[q] = fma(-base[p + (int64_t)q * nrow], w0, a[q]);
      b[q] = fma(-base[p + 1 + (int64_t)q * nrow], w1, b[q]);
      a[q] = fma(-base[p + 2 + (int64_t)q * nrow], w2, a[q]);
      b[q] = fma(-base[p + 3 + (int64_t)q * nrow], w3, b[q]);
    }
  }
  for (; p < nrow; ++p) {
    const double w0 = act ? Wc[(int64_t)rw[p] * ldw] : 0.0;
#pragma unroll
    for (int q = 0; q < CW; ++q) a[q] = fma(-base[p + (int64_t)q * nrow], w0, a[q]);
  }
#pragma unroll
  for (int q = 0; q < CW; ++q) acc[q * 32 + lane] = a[q] + b[q];
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
    const double *base = Lt + (int64_t)j0 * nrow;
    switch (cw) {
      case 1: lbwd_chunk<1>(Wc, ldw, act, c0 + j0, base, nrow, ncol, rw, acc + j0 * 32, lane); break;
      case 2: lbwd_chunk<2>(Wc, ldw, act, c0 + j0, base, nrow, ncol, rw, acc + j0 * 32, lane); break;
      case 3: lbwd_chunk<3>(Wc, ldw, act, c0 + j0, base, nrow, ncol, rw, acc + j0 * 32, lane); break;
      case 4: lbwd_chunk<4>(Wc, ldw, act, c0 + j0, base, nrow, ncol, rw, acc + j0 * 32, lane); break;
      case 5: lbwd_chunk<5>(Wc, ldw, act, c0 + j0, base, nrow, ncol, rw, acc + j0 * 32, lane); break;
      case 6: lbwd_chunk<6>(Wc, ldw, act, c0 + j0, base, nrow, ncol, rw, acc + j0 * 32, lane); break;
      case 7: lbwd_chunk<7>(Wc, ldw, act, c0 + j0, base, nrow, ncol, rw, acc + j0 * 32, lane); break;
      default: lbwd_chunk<8>(Wc, ldw, act, c0 + j0, base, nrow, ncol, rw, acc + j0 * 32, lane); break;
    }
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
  const size_t smem = (size_t)S.max_ncol * 32 * 8 + (size_t)LS_CH * S.max_nrow * 8 + (size_t)S.max_nrow * 4 + 16;
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
        const int rb = (int)std::min<int64_t>(1024, ((int64_t)S.max_ncol * ncolsW + 255) / 256);
        k_lfwd_reduce<<<dim3(rb, xc), 256, 0, st>>>(S, xb, xc, Pw, W, ldw, ncolsW, sk);
        launches += 2;
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
