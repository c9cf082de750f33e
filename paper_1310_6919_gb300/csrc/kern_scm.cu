// K3: SCM assembly, eq. (newSCM2) of Sec. 3.1, S-ELEMENTS.
//
// The paper evaluates column j of B with, for each nonzero column k of A_j, one solve
// v1 = L̂^{-T} L̂^{-1} e_k and one v2 = N^{-T} N^{-1} [A_j]_{*k}, then B_ij += v1^T A_i v2
// (Algorithm 2, Step 3-3).  Here constraints are grouped (group g = constraints J_g whose
// nonzeros lie in the index set P_g) and, per group, the columns X̂ e_k and Y^{-1} e_k for
// k in P_g are computed once by the level-scheduled many-right-hand-side solves of
// kern_lsolve.cu (a chunk of groups at a time, within a memory budget).  Because
// [A_j]_{*k} is supported on P_g, v2 = Y^{-1}[:, P_g] [A_j]_{P_g, k}; substituting, every term
// of eq. (newSCM2) becomes
//     B_ij = sum_{(a,b) in A_i} sum_{(c,d) in A_j} [A_i]_ab [A_j]_cd X̂_ac Y^{-1}_bd,
// which a CTA evaluates for the tile (J_h, J_g) from the blocks X̂[P_h, P_g], Y^{-1}[P_h, P_g]
// staged in shared memory.  Only the lower triangle (h >= g) is formed (B is symmetric).
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"
#include "warp_solve.cuh"

namespace mcsdp {

constexpr int XW_CAP = 6144;  // doubles of shared memory for the X̂-times-A_j products

// T = double: the FP64 form; T = float: the mixed form's assembly (FP32 operands and sums, the
// entries stored into the FP64 B)
template <class T>
__global__ void k_scm_tiles(DevSym S, const int2 *__restrict__ tiles,
                            const T *__restrict__ WX, const T *__restrict__ WY,
                            int64_t ldw, const int *__restrict__ goff, double *B, int64_t ldb,
                            double *hvec, const int *__restrict__ colmap) {
  extern __shared__ __align__(16) unsigned char smr[];
  T *sm = reinterpret_cast<T *>(smr);
  const int2 tl = tiles[blockIdx.x];
  const int h = tl.x, g = tl.y;
  const int pbg = S.grp_pptr[g], pg = S.grp_pptr[g + 1] - pbg;
  const int pbh = S.grp_pptr[h], ph = S.grp_pptr[h + 1] - pbh;
  const int cg = colmap ? 0 : goff[g];
  T *Xs = sm;
  T *Ys = sm + ph * pg;
  const int tid = threadIdx.x, bd = blockDim.x;
  // X̂[P_h, P_g], Y^{-1}[P_h, P_g]: rows P_h of the group's solved columns
  for (int idx = tid; idx < ph * pg; idx += bd) {
    const int a = idx / pg, c = idx % pg;
    const int64_t o = (int64_t)S.grp_cols[pbh + a] * ldw + (colmap ? colmap[S.grp_cols[pbg + c]] : cg + c);
    Xs[a + c * ph] = WX[o];
    Ys[a + c * ph] = WY[o];
  }
  __syncthreads();
  const int i0 = S.grp_cptr[h], nh = S.grp_cptr[h + 1] - i0;
  const int j0 = S.grp_cptr[g], ng = S.grp_cptr[g + 1] - j0;
  // nonzero lists of J_h and J_g in shared memory: (offset into Xs/Ys column, value)
  const int hb = S.anz_ptr[i0], hn = S.anz_ptr[i0 + nh] - hb;
  const int gb = S.anz_ptr[j0], gn = S.anz_ptr[j0 + ng] - gb;
  T *hv = Ys + ph * pg;
  T *gv = hv + hn;
  int *ha = reinterpret_cast<int *>(gv + gn);  // a (row of Xs) | b << 16 (row of Ys)
  int *ga = ha + hn;                           // c * ph | d * ph << 16 packed as two shorts
  int *gd = ga + gn;
  for (int e = tid; e < hn; e += bd) {
    hv[e] = (T)S.anz_v[hb + e];
    ha[e] = S.anz_a[hb + e] | (S.anz_b[hb + e] << 16);
  }
  for (int e = tid; e < gn; e += bd) {
    gv[e] = (T)S.anz_v[gb + e];
    ga[e] = S.anz_a[gb + e] * ph;
    gd[e] = S.anz_b[gb + e] * ph;
  }
  __syncthreads();
  // constraints j of J_g in batches of JB: XW[jb][u][a] = [A_j]_u * X̂[P_h[a], c_u] for the
  // nonzeros u of A_j, then B_ij = sum_t v_t sum_u XW[jb][u][a_t] Y^{-1}[P_h[b_t], d_u]
  // (one multiply-add per pair of nonzeros)
  // the int lists (hn + 2 gn ints) start 8-byte aligned; round their end up to 8 bytes
  T *XW = reinterpret_cast<T *>(ha + ((hn + 2 * gn + 1) & ~1));
  const int cap_nnz = XW_CAP / (ph > 0 ? ph : 1);
  for (int jb0 = 0, nj = 0; jb0 < ng; jb0 += nj) {
    // batch: as many constraints as fit XW_CAP doubles (at least one)
    nj = 1;
    while (jb0 + nj < ng && S.anz_ptr[j0 + jb0 + nj + 1] - S.anz_ptr[j0 + jb0] <= cap_nnz) ++nj;
    // the batch's nonzeros are contiguous: [S.anz_ptr[j0 + jb0], S.anz_ptr[j0 + jb0 + nj])
    const int ub0 = S.anz_ptr[j0 + jb0] - gb, ub1 = S.anz_ptr[j0 + jb0 + nj] - gb;
    for (int e = tid; e < (ub1 - ub0) * ph; e += bd) {
      const int u = ub0 + e / ph, a = e % ph;
      XW[(u - ub0) * ph + a] = gv[u] * Xs[a + ga[u]];
    }
    __syncthreads();
    for (int idx = tid; idx < nh * nj; idx += bd) {
      const int ii = idx % nh, jb = idx / nh;
      const int i = i0 + ii, j = j0 + jb0 + jb;
      if (h == g && i < j) continue;
      const int ub = S.anz_ptr[j] - gb, ue = S.anz_ptr[j + 1] - gb;
      T acc = T(0);
      for (int t = S.anz_ptr[i] - hb; t < S.anz_ptr[i + 1] - hb; ++t) {
        const int a = ha[t] & 0xffff, b = ha[t] >> 16;
        const T *xw = XW + (ub - ub0) * ph + a;
        const T *yr = Ys + b;
        T s0 = T(0), s1 = T(0);
        int u = 0;
        const int nu = ue - ub;
        for (; u + 1 < nu; u += 2) {
          s0 = fma(xw[u * ph], yr[gd[ub + u]], s0);
          s1 = fma(xw[(u + 1) * ph], yr[gd[ub + u + 1]], s1);
        }
        if (u < nu) s0 = fma(xw[u * ph], yr[gd[ub + u]], s0);
        acc = fma(hv[t], s0 + s1, acc);
      }
      B[i + (int64_t)j * ldb] = (double)acc;
    }
    __syncthreads();
  }
  if (h == g) {
    for (int ii = tid; ii < nh; ii += bd) {
      const int i = i0 + ii;
      T hsum = T(0);
      for (int t = S.anz_ptr[i]; t < S.anz_ptr[i + 1]; ++t)
        hsum = fma((T)S.anz_v[t], Ys[S.anz_a[t] + S.anz_b[t] * ph], hsum);
      hvec[i] = (double)hsum;
    }
  }
}

// es: element size (8 for the FP64 form; the FP32 form needs about half, so two CTAs fit an SM)
size_t scm_tiles_smem_bytes(const DevSym &S, int pmax, int es) {
  const size_t xw = std::max<size_t>(XW_CAP, (size_t)S.max_con_nnz * pmax);
  return (size_t)2 * pmax * pmax * es + (size_t)2 * S.max_grp_nnz * (es + 8) + 64 + xw * es;
}
size_t scm_tiles_smem_bytes(const DevSym &S, int pmax) { return scm_tiles_smem_bytes(S, pmax, 8); }

template <class T>
void launch_scm_tiles(const DevSym &S, const int2 *tiles, int ntiles, const T *WX,
                      const T *WY, int64_t ldw, const int *goff, double *B, int64_t ldb,
                      double *hvec, int pmax, cudaStream_t st, const int *colmap) {
  if (ntiles <= 0) return;
  // two |P_h| x |P_g| blocks, the nonzero lists of two groups, and the X̂-times-A_j products of
  // one batch of constraints (XW_CAP doubles, or one constraint's if larger) in shared memory
  const size_t smem = scm_tiles_smem_bytes(S, pmax, (int)sizeof(T));
  smem_optin((const void *)k_scm_tiles<T>);
  k_scm_tiles<T><<<ntiles, 256, smem, st>>>(S, tiles, WX, WY, ldw, goff, B, ldb, hvec, colmap);
}
// Max-cut-shaped constraints (every A_k = e_k e_k^T): eq. newSCM2 reduces to B = X̂ o Y^{-1} on the
// constraints' vertices (the Hadamard product of Sec. 3.1's max-cut discussion).  With X̂ and Y^{-1}
// formed whole (the dense-root path, row-major n x ldw, vertex k's column at colw[k]; both
// symmetric) the lower triangle of B streams: column j of B reads row v_j of both matrices at the
// columns of v_i, i >= j (consecutive i, consecutive columns), and writes B[i + j ldb]; h_i =
// Y^{-1}(v_i, v_i).  Grid: x over the rows i of a column chunk, y over the columns j.
template <class T>
__global__ void __launch_bounds__(256) k_scm_hadamard(DevSym S, const T *__restrict__ WX,
                                                      const T *__restrict__ WY, int64_t ldw,
                                                      const int *__restrict__ colw,
                                                      const int *__restrict__ vtx, double *B,
                                                      int64_t ldb, double *hvec) {
  const int m = S.m;
  for (int j = blockIdx.y; j < m; j += gridDim.y) {
    const int vj = vtx[j];
    const T *xr = WX + (int64_t)vj * ldw, *yr = WY + (int64_t)vj * ldw;
    double *bc = B + (int64_t)j * ldb;
    for (int i = j + blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
      const int c = colw[vtx[i]];
      const T v = xr[c] * yr[c];
      bc[i] = (double)v;
      if (i == j) hvec[i] = (double)yr[c];
    }
  }
}

template <class T>
void launch_scm_hadamard(const DevSym &S, const T *WX, const T *WY, int64_t ldw, const int *colw,
                         const int *vtx, double *B, int64_t ldb, double *hvec, cudaStream_t st) {
  if (S.m <= 0) return;
  dim3 grid(std::max(1, std::min(8, (S.m + 1023) / 1024)), std::min(S.m, 65535));
  k_scm_hadamard<T><<<grid, 256, 0, st>>>(S, WX, WY, ldw, colw, vtx, B, ldb, hvec);
}
template void launch_scm_hadamard<double>(const DevSym &, const double *, const double *, int64_t,
                                          const int *, const int *, double *, int64_t, double *,
                                          cudaStream_t);
template void launch_scm_hadamard<float>(const DevSym &, const float *, const float *, int64_t,
                                         const int *, const int *, double *, int64_t, double *,
                                         cudaStream_t);

template void launch_scm_tiles<double>(const DevSym &, const int2 *, int, const double *,
                                       const double *, int64_t, const int *, double *, int64_t,
                                       double *, int, cudaStream_t, const int *);
template void launch_scm_tiles<float>(const DevSym &, const int2 *, int, const float *,
                                      const float *, int64_t, const int *, double *, int64_t,
                                      double *, int, cudaStream_t, const int *);

}  // namespace mcsdp
