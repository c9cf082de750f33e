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
#include <type_traits>

#include "../../include/mcsdp.h"
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
  if (lane == 0) S.xvalid[(int64_t)x * S.xv_stride + tile] = 1;
  double *P = Pw + S.xch_slotw[x] * ldw + (act ? col : 0);
  if (act)
    for (int c = 0; c < ncol; ++c) P[(int64_t)c * ldw] = acc[c * 32 + lane];
}

// W[S_t] += sum of the partial slots of t (those marked valid), for every target of the level
// with extra update chunks.  CTA = (32 columns, row c of S_t, target) x 8 chunk phases: phase p sums the chunks
// xb + p, xb + p + 8, ..., then the 8 phase sums are added in order (deterministic).
template <class T>
__global__ void k_lfwd_reduce(DevSym S, int f0, const T *__restrict__ Pw, T *W,
                              int64_t ldw, int ncolsW, LsSkip sk) {
  __shared__ T part[8][33];
  const int xb = S.xfst[f0 + blockIdx.z];
  const int t = S.xch_t[xb];
  const int c0 = S.sn_col[t];
  const int ncol = S.sn_col[t + 1] - c0;
  const int c = blockIdx.y;
  if (c >= ncol) return;
  const int tile = blockIdx.x;
  if (ls_skip(sk, t, tile)) return;
  const int lane = threadIdx.x & 31, ph = threadIdx.x >> 5;
  const int col = tile * 32 + lane;
  const int xe = S.xch_end[t];
  T a = T(0);
  if (col < ncolsW)
    for (int xx = xb + ph; xx < xe; xx += 8)
      if (S.xvalid[(int64_t)xx * S.xv_stride + tile]) a += Pw[(S.xch_slotw[xx] + c) * ldw + col];
  part[ph][lane] = a;
  __syncthreads();
  if (ph == 0 && col < ncolsW) {
    T s = part[0][lane];
    for (int q = 1; q < 8; ++q) s += part[q][lane];
    W[(int64_t)(c0 + c) * ldw + col] += s;
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

// ---------------------------------------------------------------------------------------------
// Staged forms.  Every operand a CTA needs (its D block, its acc rows of W, the update blocks and
// source values, the gathered ancestor rows of W) is copied into shared memory with cp.async, so
// a CTA waits for memory about once instead of once per dependent load; the update blocks go
// through a ring of LS_R buffers, LS_R - 1 chunks in flight while one is applied.  Each CTA is
// one warp; shared memory is sized per level (small supernodes at the bottom of the tree keep
// many CTAs per SM).
constexpr int LS_R = 4;

__device__ __forceinline__ void cpa8(void *s, const void *g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(s)),
               "l"(g)
               : "memory");
}
__device__ __forceinline__ void cpa4(void *s, const void *g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((unsigned)__cvta_generic_to_shared(s)),
               "l"(g)
               : "memory");
}
template <class T>
__device__ __forceinline__ void cpaT(void *s, const void *g) {
  if constexpr (sizeof(T) == 8) cpa8(s, g);
  else cpa4(s, g);
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cpa_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__host__ __device__ inline int al16(int b) { return (b + 15) & ~15; }

struct FwdLayout {
  int acc, ds, meta, hdr, buf, bufsz, total;
};
// nc: ncol bound, cw/np: update chunk width / rows bound (cw = 0: no updates), with_d: D block
__host__ __device__ inline FwdLayout fwd_layout(int nc, int cw, int np, bool with_d, int es) {
  FwdLayout L;
  int o = 0;
  L.acc = o;
  o += al16(nc * 32 * es);
  L.ds = o;
  o += with_d ? al16(nc * nc * es) : 0;
  L.meta = o;
  o += cw > 0 ? 64 * (int)sizeof(UpdMeta) : 0;
  L.hdr = o;  // per ring slot: (row count, source column count) of the chunk it holds
  o += cw > 0 ? al16(LS_R * 8) : 0;
  L.buf = o;
  L.bufsz = cw > 0 ? al16(cw * 32 * es) + al16(cw * np * es) + al16(np * 4) : 0;
  o += LS_R * L.bufsz;
  L.total = o;
  return L;
}

struct BwdLayout {
  int ls, ds, acc, wv, rws, total;
};
__host__ __device__ inline BwdLayout bwd_layout(int nr, int nc, int es) {
  BwdLayout L;
  int o = 0;
  L.ls = o;
  o += al16(nr * nc * es);
  L.ds = o;
  o += al16(nc * nc * es);
  L.acc = o;
  o += al16(nc * 32 * es);
  L.wv = o;
  o += al16(nr * 32 * es);
  L.rws = o;
  o += al16(nr * 4);
  L.total = o;
  return L;
}

// acc[srel[p]][lane] -= sum over the updates [ub, ue) of L_d[p1 + p, :] W[S_d], the update
// blocks taken in chunks of <= cw source columns through the ring.  An update whose source
// supernode d the skip rule drops for this tile is passed over: W[S_d] of the tile's right-hand
// sides is zero there (d's own solve was skipped), so the result is the same bit for bit.  The
// producer writes each chunk's (rows, columns) into its slot header, so the consumer needs no
// update index of its own.
template <class T>
__device__ __forceinline__ int pull_staged(const DevSym &S, int ub, int ue, const T *L,
                                            const T *Wc, int64_t ldw, T *acc,
                                            unsigned char *sm, const FwdLayout &lay, int cw, int npb,
                                            int lane, const LsSkip &sk, int tile) {
  UpdMeta *ms = reinterpret_cast<UpdMeta *>(sm + lay.meta);
  int2 *hdr = reinterpret_cast<int2 *>(sm + lay.hdr);
  int meta_end = ub;
  int iu = ub, ij = 0, issued = 0, chunks = 0;
  const int es = (int)sizeof(T);
  const int xs_off = 0, lb_off = al16(cw * 32 * es), sr_off = lb_off + al16(cw * npb * es);
  const int2 kr = sk.bits ? sk.tile_keys[tile] : make_int2(0, -1);
  auto dropped = [&](int d) {
    if (!sk.bits) return false;
    for (int key = kr.x; key <= kr.y; ++key)
      if (sk.bits[(int64_t)key * sk.words + (d >> 5)] & (1u << (d & 31))) return false;
    return true;
  };
  auto issue = [&]() {
    while (iu < ue) {
      while (iu >= meta_end) {  // next 32 records into the metadata ring (64 entries)
        const int v = meta_end + lane;
        if (v < ue) ms[v & 63] = S.upd_meta[v];
        meta_end += 32;
        __syncwarp();
      }
      if (ij > 0 || !dropped(ms[iu & 63].src)) break;
      ++iu;
    }
    if (iu < ue) {
      const UpdMeta m = ms[iu & 63];
      const int slot = issued % LS_R;
      unsigned char *b = sm + lay.buf + slot * lay.bufsz;
      T *xs = reinterpret_cast<T *>(b + xs_off);
      T *Lb = reinterpret_cast<T *>(b + lb_off);
      int *sr = reinterpret_cast<int *>(b + sr_off);
      const int w = min(cw, m.dncol - ij);
      for (int q = 0; q < w; ++q) cpaT<T>(xs + q * 32 + lane, Wc + (int64_t)(m.dc0 + ij + q) * ldw);
      const T *Lsrc = L + m.valp + (int64_t)ij * m.dnrow + m.p1;
      for (int e = lane; e < m.np * w; e += 32) {
        const int q = e / m.np, p = e - q * m.np;
        cpaT<T>(Lb + e, Lsrc + (int64_t)q * m.dnrow + p);
      }
      for (int p = lane; p < m.np; p += 32) cpa4(sr + p, S.upd_rel + m.relptr + p);
      if (lane == 0) hdr[slot] = make_int2(m.np, w);
      ++chunks;
      ij += w;
      if (ij >= m.dncol) {
        ++iu;
        ij = 0;
      }
    }
    cpa_commit();
    ++issued;
  };
  for (int k = 0; k < LS_R - 1; ++k) issue();
  int done = 0;
  while (done < chunks) {  // chunks == done here only once the producer has reached ue
    issue();
    cpa_wait<LS_R - 1>();
    __syncwarp();
    const int2 h = hdr[done % LS_R];
    const unsigned char *b = sm + lay.buf + (done % LS_R) * lay.bufsz;
    const T *xs = reinterpret_cast<const T *>(b + xs_off);
    const T *Lb = reinterpret_cast<const T *>(b + lb_off);
    const int *sr = reinterpret_cast<const int *>(b + sr_off);
    const int np = h.x, w = h.y;
    int p = 0;
    for (; p + 3 < np; p += 4) {
      T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
      for (int q = 0; q < w; ++q) {
        const T x = xs[q * 32 + lane];
        const T *lq = Lb + q * np + p;
        a0 = fma(lq[0], x, a0);
        a1 = fma(lq[1], x, a1);
        a2 = fma(lq[2], x, a2);
        a3 = fma(lq[3], x, a3);
      }
      acc[sr[p] * 32 + lane] -= a0;
      acc[sr[p + 1] * 32 + lane] -= a1;
      acc[sr[p + 2] * 32 + lane] -= a2;
      acc[sr[p + 3] * 32 + lane] -= a3;
    }
    for (; p < np; ++p) {
      T a0 = T(0);
      for (int q = 0; q < w; ++q) a0 = fma(Lb[q * np + p], xs[q * 32 + lane], a0);
      acc[sr[p] * 32 + lane] -= a0;
    }
    __syncwarp();
    ++done;
  }
  return chunks;  // update chunks pulled (0: every update was passed over)
}

// NW warps per CTA: NW = 1 for wide levels (many CTAs per SM already use every SM
// sub-partition); NW = 2 for middling levels and NW = 4 for narrow levels near the root, where
// one CTA per SM would leave FP64 sub-partitions idle: warp 0 applies the updates, then the
// product with D is split by rows over the warps.
template <class T, int NW>
__global__ void __launch_bounds__(32 * NW)
    k_lfwd2(DevSym S, int lvl_begin, int ntiles, const T *__restrict__ L,
            const T *__restrict__ Dall, T *W, int64_t ldw, int ncolsW, LsSkip sk, int nc,
            int cw, int npb) {
  extern __shared__ __align__(16) unsigned char smf[];
  const FwdLayout lay = fwd_layout(nc, cw, npb, true, (int)sizeof(T));
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int t = S.lvl_sn[lvl_begin + blockIdx.x / ntiles];
  const int tile = blockIdx.x % ntiles;
  if (ls_skip(sk, t, tile)) return;
  const int col = tile * 32 + lane;
  const bool act = col < ncolsW;
  const int c0 = S.sn_col[t];
  const int ncol = S.sn_col[t + 1] - c0;
  T *acc = reinterpret_cast<T *>(smf + lay.acc);
  T *Ds = reinterpret_cast<T *>(smf + lay.ds);
  T *Wc = W + (act ? col : 0);
  for (int j = warp; j < ncol; j += NW) cpaT<T>(acc + j * 32 + lane, Wc + (int64_t)(c0 + j) * ldw);
  const T *D = Dall + S.sn_dptr[t];
  for (int e = tid; e < ncol * ncol; e += 32 * NW) cpaT<T>(Ds + e, D + e);
  cpa_commit();
  if (NW > 1) {
    cpa_wait<0>();
    __syncthreads();
  }
  if (warp == 0) {
    pull_staged(S, S.upd_ptr[t], S.upd_c0end[t], L, Wc, ldw, acc, smf, lay, cw, npb, lane, sk,
                tile);
    cpa_wait<0>();
  }
  __syncthreads();
  // W[S_t] <- D acc  (D lower: D[i][j] = Ds[i + j ncol], zero above the diagonal), 4 rows at once
  for (int i0 = 4 * warp; i0 < ncol; i0 += 4 * NW) {
    T a[4] = {T(0), T(0), T(0), T(0)};
    const int jend = min(i0 + 4, ncol);
    for (int j = 0; j < jend; ++j) {
      const T x = acc[j * 32 + lane];
#pragma unroll
      for (int r = 0; r < 4; ++r)
        if (i0 + r < ncol) a[r] = fma(Ds[(i0 + r) + j * ncol], x, a[r]);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
      if (act && i0 + r < ncol) Wc[(int64_t)(c0 + i0 + r) * ldw] = a[r];
  }
}

template <class T>
__global__ void k_lfwd_partial2(DevSym S, int x0, int ntiles, const T *__restrict__ L,
                                const T *__restrict__ W, int64_t ldw, int ncolsW, LsSkip sk,
                                T *Pw, int nc, int cw, int npb) {
  extern __shared__ __align__(16) unsigned char smp[];
  const FwdLayout lay = fwd_layout(nc, cw, npb, false, (int)sizeof(T));
  const int lane = threadIdx.x;
  const int x = x0 + blockIdx.x / ntiles;
  const int tile = blockIdx.x % ntiles;
  const int t = S.xch_t[x];
  if (ls_skip(sk, t, tile)) return;
  const int col = tile * 32 + lane;
  const bool act = col < ncolsW;
  const int ncol = S.sn_col[t + 1] - S.sn_col[t];
  T *acc = reinterpret_cast<T *>(smp + lay.acc);
  for (int c = 0; c < ncol; ++c) acc[c * 32 + lane] = T(0);
  const int pulled = pull_staged(S, S.xch_ub[x], S.xch_ue[x], L, W + (act ? col : 0), ldw, acc,
                                 smp, lay, cw, npb, lane, sk, tile);
  cpa_wait<0>();
  __syncwarp();
  if (lane == 0) S.xvalid[(int64_t)x * S.xv_stride + tile] = pulled > 0;
  if (pulled == 0) return;  // nothing reached this chunk: the reduce passes the slot over
  T *P = Pw + S.xch_slotw[x] * ldw + (act ? col : 0);
  if (act)
    for (int c = 0; c < ncol; ++c) P[(int64_t)c * ldw] = acc[c * 32 + lane];
}

template <class T, int NW>
__global__ void __launch_bounds__(32 * NW)
    k_lbwd2(DevSym S, int lvl_begin, int ntiles, const T *__restrict__ L,
            const T *__restrict__ Dall, T *W, int64_t ldw, int ncolsW, LsSkip sk,
            int nr_b, int nc_b) {
  extern __shared__ __align__(16) unsigned char smb[];
  const BwdLayout lay = bwd_layout(nr_b, nc_b, (int)sizeof(T));
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int t = S.lvl_sn[lvl_begin + blockIdx.x / ntiles];
  const int tile = blockIdx.x % ntiles;
  if (ls_skip(sk, t, tile)) return;
  const int col = tile * 32 + lane;
  const bool act = col < ncolsW;
  const int c0 = S.sn_col[t];
  const int ncol = S.sn_col[t + 1] - c0;
  const int64_t r0 = S.sn_rowptr[t];
  const int nrow = (int)(S.sn_rowptr[t + 1] - r0);
  T *Ls = reinterpret_cast<T *>(smb + lay.ls);
  T *Ds = reinterpret_cast<T *>(smb + lay.ds);
  T *acc = reinterpret_cast<T *>(smb + lay.acc);
  T *wv = reinterpret_cast<T *>(smb + lay.wv);
  int *rws = reinterpret_cast<int *>(smb + lay.rws);
  const T *Lt = L + S.sn_valptr[t];
  const T *D = Dall + S.sn_dptr[t];
  T *Wc = W + (act ? col : 0);
  for (int p = ncol + tid; p < nrow; p += 32 * NW) rws[p] = S.rows[r0 + p];
  for (int e = tid; e < nrow * ncol; e += 32 * NW) cpaT<T>(Ls + e, Lt + e);
  for (int e = tid; e < ncol * ncol; e += 32 * NW) cpaT<T>(Ds + e, D + e);
  for (int j = warp; j < ncol; j += NW) cpaT<T>(acc + j * 32 + lane, Wc + (int64_t)(c0 + j) * ldw);
  __syncthreads();
  for (int p = ncol + warp; p < nrow; p += NW)
    cpaT<T>(wv + (p - ncol) * 32 + lane, Wc + (int64_t)rws[p] * ldw);
  cpa_commit();
  cpa_wait<0>();
  __syncthreads();
  // acc[j] -= sum_{p >= ncol} L[p][j] W[rows[p]], 4 columns j at once (column blocks over warps)
  for (int j0 = 4 * warp; j0 < ncol; j0 += 4 * NW) {
    T a[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) a[r] = (j0 + r < ncol) ? acc[(j0 + r) * 32 + lane] : T(0);
    for (int p = ncol; p < nrow; ++p) {
      const T w = wv[(p - ncol) * 32 + lane];
#pragma unroll
      for (int r = 0; r < 4; ++r)
        if (j0 + r < ncol) a[r] = fma(-Ls[p + (j0 + r) * nrow], w, a[r]);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
      if (j0 + r < ncol) acc[(j0 + r) * 32 + lane] = a[r];
  }
  __syncthreads();
  // W[S_t] <- D^T acc: out[i] = sum_{j >= i} D[j][i] acc[j], 4 rows at once (row blocks over warps)
  for (int i0 = 4 * warp; i0 < ncol; i0 += 4 * NW) {
    T a[4] = {T(0), T(0), T(0), T(0)};
    for (int j = i0; j < ncol; ++j) {
      const T x = acc[j * 32 + lane];
#pragma unroll
      for (int r = 0; r < 4; ++r)
        if (i0 + r < ncol) a[r] = fma(Ds[j + (i0 + r) * ncol], x, a[r]);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
      if (act && i0 + r < ncol) Wc[(int64_t)(c0 + i0 + r) * ldw] = a[r];
  }
}

constexpr int LS_SMEM_CAP = 200 * 1024;

bool lsolve_staged_fits(const LsLevel *lvl_info, int height, int elem_size) {
  for (int l = 0; l < height; ++l) {
    const LsLevel &lv = lvl_info[l];
    if (fwd_layout(lv.nc, lv.cw, lv.np, true, elem_size).total > LS_SMEM_CAP) return false;
    if (bwd_layout(lv.nr, lv.nc, elem_size).total > LS_SMEM_CAP) return false;
  }
  return true;
}
constexpr int LS_NARROW_PER_SM = 8;  // CTAs per SM of a level below which a CTA gets four warps
constexpr int LS_MEDIUM_PER_SM = 48;  // ... and below which a CTA gets two

template <class T>
int lsolve(const DevSym &S, const int *lvl_ptr_host, const int *lvl_xptr_host,
           const int *lvl_fptr_host, const LsLevel *lvl_info, int height, bool fwd,
           const T *L, const T *D, T *W, int64_t ldw, int ncolsW, const LsSkip &sk,
           T *Pw, const int64_t *active, cudaStream_t st) {
  if (ncolsW <= 0) return 0;
  const int ntiles = (ncolsW + 31) / 32;
  const size_t smem = (size_t)S.max_ncol * 32 * 8 + (size_t)LS_CH * S.max_nrow * 8 + (size_t)S.max_nrow * 4 + 16;
  if (smem > 48 * 1024) {
    smem_optin((const void *)k_lfwd);
    smem_optin((const void *)k_lbwd);
    smem_optin((const void *)k_lfwd_partial);
  }
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 1;
  }
  smem_optin((const void *)k_lfwd2<T, 1>);
  smem_optin((const void *)k_lbwd2<T, 1>);
  smem_optin((const void *)k_lfwd2<T, 4>);
  smem_optin((const void *)k_lbwd2<T, 4>);
  smem_optin((const void *)k_lbwd2<T, 2>);
  smem_optin((const void *)k_lfwd2<T, 2>);
  smem_optin((const void *)k_lfwd_partial2<T>);
  int launches = 0;
  for (int li = 0; li < height; ++li) {
    const int l = fwd ? li : height - 1 - li;
    const int b = lvl_ptr_host[l], cnt = lvl_ptr_host[l + 1] - b;
    const int64_t blocks = (int64_t)cnt * ntiles;
    if (blocks <= 0) continue;
    const LsLevel &lv = lvl_info[l];
    const int es = (int)sizeof(T);
    const int sf = fwd_layout(lv.nc, lv.cw, lv.np, true, es).total;
    const int sp = fwd_layout(lv.nc, lv.cw, lv.np, false, es).total;
    const int sb = bwd_layout(lv.nr, lv.nc, es).total;
    // CTAs the skip rule drops return at once: the shape follows the pairs that do work
    const int64_t work = active ? active[l] : blocks;
    const bool narrow = work <= (int64_t)LS_NARROW_PER_SM * nsm;
    const bool medium = work <= (int64_t)LS_MEDIUM_PER_SM * nsm;
    if (fwd && sf <= LS_SMEM_CAP) {
      const int xb = lvl_xptr_host[l], xc = lvl_xptr_host[l + 1] - xb;
      if (xc > 0) {
        k_lfwd_partial2<T><<<(unsigned)((int64_t)xc * ntiles), 32, sp, st>>>(
            S, xb, ntiles, L, W, ldw, ncolsW, sk, Pw, lv.nc, lv.cw, lv.np);
        const int f0 = lvl_fptr_host[l], nf = lvl_fptr_host[l + 1] - f0;
        if (nf > 0) k_lfwd_reduce<T><<<dim3(ntiles, lv.nc, nf), 256, 0, st>>>(S, f0, Pw, W, ldw, ncolsW, sk);
        launches += 2;
      }
      if (narrow)
        k_lfwd2<T, 4><<<(unsigned)blocks, 128, sf, st>>>(S, b, ntiles, L, D, W, ldw, ncolsW, sk, lv.nc,
                                                      lv.cw, lv.np);
      else if (medium)
        k_lfwd2<T, 2><<<(unsigned)blocks, 64, sf, st>>>(S, b, ntiles, L, D, W, ldw, ncolsW, sk, lv.nc,
                                                     lv.cw, lv.np);
      else
        k_lfwd2<T, 1><<<(unsigned)blocks, 32, sf, st>>>(S, b, ntiles, L, D, W, ldw, ncolsW, sk, lv.nc,
                                                     lv.cw, lv.np);
    } else if (!fwd && sb <= LS_SMEM_CAP) {
      if (narrow)
        k_lbwd2<T, 4><<<(unsigned)blocks, 128, sb, st>>>(S, b, ntiles, L, D, W, ldw, ncolsW, sk, lv.nr,
                                                      lv.nc);
      else if (medium)
        k_lbwd2<T, 2><<<(unsigned)blocks, 64, sb, st>>>(S, b, ntiles, L, D, W, ldw, ncolsW, sk, lv.nr,
                                                     lv.nc);
      else
        k_lbwd2<T, 1><<<(unsigned)blocks, 32, sb, st>>>(S, b, ntiles, L, D, W, ldw, ncolsW, sk, lv.nr,
                                                     lv.nc);
    } else if constexpr (!std::is_same<T, double>::value) {
      return -1;  // FP32 solves only through the staged kernels
    } else if (fwd) {
      const int xb = lvl_xptr_host[l], xc = lvl_xptr_host[l + 1] - xb;
      if (xc > 0) {
        k_lfwd_partial<<<(unsigned)((int64_t)xc * ntiles), 32, smem, st>>>(S, xb, ntiles, L, W, ldw,
                                                                           ncolsW, sk, Pw);
        const int f0 = lvl_fptr_host[l], nf = lvl_fptr_host[l + 1] - f0;
        if (nf > 0) k_lfwd_reduce<double><<<dim3(ntiles, S.max_ncol, nf), 256, 0, st>>>(S, f0, Pw, W, ldw, ncolsW, sk);
        launches += 2;
      }
      k_lfwd<<<(unsigned)blocks, 32, smem, st>>>(S, b, ntiles, L, D, W, ldw, ncolsW, sk, Pw);
    }
    else k_lbwd<<<(unsigned)blocks, 32, smem, st>>>(S, b, ntiles, L, D, W, ldw, ncolsW, sk);
    ++launches;
  }
  return launches;
}

template int lsolve<double>(const DevSym &, const int *, const int *, const int *, const LsLevel *,
                            int, bool, const double *, const double *, double *, int64_t, int,
                            const LsSkip &, double *, const int64_t *, cudaStream_t);
template int lsolve<float>(const DevSym &, const int *, const int *, const int *, const LsLevel *,
                           int, bool, const float *, const float *, float *, int64_t, int,
                           const LsSkip &, float *, const int64_t *, cudaStream_t);

// W[rowof[j] * ldw + j] = 1 for the unit right-hand sides (W zeroed before)
template <class T>
__global__ void k_rhs_unit(T *W, int64_t ldw, const int *rowof, int nrhs) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < nrhs) W[(int64_t)rowof[j] * ldw + j] = T(1);
}

template <class T>
void launch_rhs_unit(T *W, int64_t ldw, const int *rowof, int nrhs, cudaStream_t st) {
  if (nrhs > 0) k_rhs_unit<T><<<(nrhs + 255) / 256, 256, 0, st>>>(W, ldw, rowof, nrhs);
}
template void launch_rhs_unit<double>(double *, int64_t, const int *, int, cudaStream_t);
template void launch_rhs_unit<float>(float *, int64_t, const int *, int, cudaStream_t);

}  // namespace mcsdp

// Host only: the shared-memory layouts of the staged level solves, so that the host tests can
// check them for every admissible clique size (see include/mcsdp.h).
extern "C" mcsdp_status mcsdp_lsolve_layout(int32_t nc, int32_t nr, int32_t cw, int32_t np,
                                            int32_t with_d, int32_t elem_size, int32_t *fwd,
                                            int32_t *bwd, int32_t *cap) {
  if (nc <= 0 || nr < nc || cw < 0 || np < 0 || (elem_size != 4 && elem_size != 8) || !fwd ||
      !bwd)
    return MCSDP_ERR_ARG;
  const mcsdp::FwdLayout f = mcsdp::fwd_layout(nc, cw, np, with_d != 0, elem_size);
  const int32_t fv[7] = {f.acc, f.ds, f.meta, f.hdr, f.buf, f.bufsz, f.total};
  for (int i = 0; i < 7; ++i) fwd[i] = fv[i];
  const mcsdp::BwdLayout b = mcsdp::bwd_layout(nr, nc, elem_size);
  const int32_t bv[6] = {b.ls, b.ds, b.acc, b.wv, b.rws, b.total};
  for (int i = 0; i < 6; ++i) bwd[i] = bv[i];
  if (cap) *cap = mcsdp::LS_SMEM_CAP;
  return MCSDP_OK;
}
