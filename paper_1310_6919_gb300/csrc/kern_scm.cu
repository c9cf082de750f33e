// K3: SCM assembly, eq. (newSCM2) of Sec. 3.1, S-ELEMENTS.
//
// The paper evaluates column j of B with, for each nonzero column k of A_j, one solve
// v1 = L̂^{-T} L̂^{-1} e_k and one v2 = N^{-T} N^{-1} [A_j]_{*k}, then B_ij += v1^T A_i v2
// (Algorithm 2, Step 3-3).  Here constraints are grouped (group g = constraints J_g whose
// nonzeros lie in the index set P_g) and, per group, the columns X̂ e_k and Y^{-1} e_k for
// k in P_g are computed once by warp-per-column supernodal solves (the panel).  Because
// [A_j]_{*k} is supported on P_g, v2 = Y^{-1}[:, P_g] [A_j]_{P_g, k}; substituting, every term
// of eq. (newSCM2) becomes
//     B_ij = sum_{(a,b) in A_i} sum_{(c,d) in A_j} [A_i]_ab [A_j]_cd X̂_ac Y^{-1}_bd,
// which a CTA evaluates for the tile (J_h, J_g) from the blocks X̂[P_h, P_g], Y^{-1}[P_h, P_g]
// staged in shared memory.  Only the lower triangle (h >= g) is formed (B is symmetric).
#include <cuda_runtime.h>

#include "internal.h"
#include "warp_solve.cuh"

namespace mcsdp {

constexpr int PANEL_WPB_MAX = 8;

__global__ void k_scm_panels(DevSym S, int g0, const double *__restrict__ Lh,
                             const double *__restrict__ dinvL, const double *__restrict__ N,
                             const double *__restrict__ dinvN, double *pan,
                             const int64_t *__restrict__ pan_off, const int *__restrict__ rhs,
                             int nrhs, int wpb, int use_global, double *gscratch) {
  extern __shared__ double sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = blockIdx.x * wpb + warp;
  if (q >= nrhs) return;
  const int desc = rhs[q];
  const int g = desc >> 9, which = (desc >> 8) & 1, c = desc & 255;
  const int n = S.n;
  double *W = use_global ? gscratch + (int64_t)q * n : sm + (int64_t)warp * n;
  const int pb = S.grp_pptr[g];
  const int pg = S.grp_pptr[g + 1] - pb;
  const int k = S.grp_cols[pb + c];
  const double *L = which ? N : Lh;
  const double *dv = which ? dinvN : dinvL;
  for (int i = lane; i < n; i += 32) W[i] = (i == k) ? 1.0 : 0.0;
  __syncwarp();
  for (int64_t t = S.reach_ptr[g]; t < S.reach_ptr[g + 1]; ++t)
    warp_fwd_sn(S, L, dv, W, S.reach_sn[t], lane);
  for (int64_t t = S.need_ptr[g + 1] - 1; t >= S.need_ptr[g]; --t)
    warp_bwd_sn(S, L, dv, W, S.need_sn[t], lane);
  const int R = S.grp_pptr[S.ngroup];
  const int64_t ldp = R - pb;
  double *out = pan + pan_off[g - g0] + (int64_t)which * ldp * pg + (int64_t)c * ldp;
  for (int qq = pb + lane; qq < R; qq += 32) out[qq - pb] = W[S.grp_cols[qq]];
}

void launch_scm_panels(const DevSym &S, int g0, int g1, const double *Lh, const double *dinvL,
                       const double *N, const double *dinvN, double *pan, const int64_t *pan_off,
                       const int *rhs, int nrhs, cudaStream_t st) {
  (void)g1;
  size_t per = (size_t)S.n * 8;
  int wpb = (int)((200 * 1024) / per);
  if (wpb > PANEL_WPB_MAX) wpb = PANEL_WPB_MAX;
  if (wpb < 1) wpb = 1;
  int blocks = (nrhs + wpb - 1) / wpb;
  size_t smem = per * wpb;
  static size_t configured = 0;
  if (smem > configured) {
    cudaFuncSetAttribute(k_scm_panels, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    configured = smem;
  }
  k_scm_panels<<<blocks, 32 * wpb, smem, st>>>(S, g0, Lh, dinvL, N, dinvN, pan, pan_off, rhs, nrhs,
                                                wpb, 0, nullptr);
}

__global__ void k_scm_tiles(DevSym S, const int2 *__restrict__ tiles, int g0,
                            const double *__restrict__ pan, const int64_t *__restrict__ pan_off,
                            double *B, int64_t ldb, double *hvec) {
  extern __shared__ double sm[];
  const int2 tl = tiles[blockIdx.x];
  const int h = tl.x, g = tl.y;
  const int pbg = S.grp_pptr[g], pg = S.grp_pptr[g + 1] - pbg;
  const int pbh = S.grp_pptr[h], ph = S.grp_pptr[h + 1] - pbh;
  const int R = S.grp_pptr[S.ngroup];
  const int64_t ldp = R - pbg;
  const int64_t rowst = pbh - pbg;
  const double *Xp = pan + pan_off[g - g0];
  const double *Yp = Xp + ldp * pg;
  double *Xs = sm;
  double *Ys = sm + ph * pg;
  const int tid = threadIdx.x, bd = blockDim.x;
  for (int idx = tid; idx < ph * pg; idx += bd) {
    const int a = idx % ph, c = idx / ph;
    Xs[idx] = Xp[rowst + a + (int64_t)c * ldp];
    Ys[idx] = Yp[rowst + a + (int64_t)c * ldp];
  }
  __syncthreads();
  const int i0 = S.grp_cptr[h], nh = S.grp_cptr[h + 1] - i0;
  const int j0 = S.grp_cptr[g], ng = S.grp_cptr[g + 1] - j0;
  for (int idx = tid; idx < nh * ng; idx += bd) {
    const int i = i0 + idx % nh, j = j0 + idx / nh;
    if (h == g && i < j) continue;
    double acc = 0.0;
    const int ub = S.anz_ptr[j], ue = S.anz_ptr[j + 1];
    for (int t = S.anz_ptr[i]; t < S.anz_ptr[i + 1]; ++t) {
      const int a = S.anz_a[t], b = S.anz_b[t];
      const double *xr = Xs + a;
      const double *yr = Ys + b;
      double s = 0.0;
      for (int u = ub; u < ue; ++u) {
        const int c = S.anz_a[u], d = S.anz_b[u];
        s = fma(S.anz_v[u] * xr[c * ph], yr[d * ph], s);
      }
      acc = fma(S.anz_v[t], s, acc);
    }
    B[i + (int64_t)j * ldb] = acc;
  }
  if (h == g) {
    for (int ii = tid; ii < nh; ii += bd) {
      const int i = i0 + ii;
      double hv = 0.0;
      for (int t = S.anz_ptr[i]; t < S.anz_ptr[i + 1]; ++t)
        hv = fma(S.anz_v[t], Ys[S.anz_a[t] + S.anz_b[t] * ph], hv);
      hvec[i] = hv;
    }
  }
}

void launch_scm_tiles(const DevSym &S, const int2 *tiles, int ntiles, int g0, const double *pan,
                      const int64_t *pan_off, double *B, int64_t ldb, double *hvec, int pmax,
                      cudaStream_t st) {
  if (ntiles <= 0) return;
  // two |P_h| x |P_g| blocks in shared memory; pmax = widest panel (<= 96)
  size_t smem = (size_t)2 * pmax * pmax * 8;
  static size_t configured = 0;
  if (smem > configured) {
    cudaFuncSetAttribute(k_scm_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    configured = smem;
  }
  k_scm_tiles<<<ntiles, 256, smem, st>>>(S, tiles, g0, pan, pan_off, B, ldb, hvec);
}

}  // namespace mcsdp
