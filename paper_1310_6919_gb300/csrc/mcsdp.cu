// libmcsdp: C ABI, context, workspace and the MC-PDIPM driver loop (Sec. 2.2 Steps 0-4 with the
// matrix-completion reformulation of Sec. 3.1).  All arithmetic of the iteration runs in the
// kernels of kern_*.cu; the host only sequences them and reads back a few scalars per iteration.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <thread>
#include <tuple>
#include <type_traits>
#include <vector>

#include "../../include/mcsdp.h"
#include "internal.h"
#include "symbolic.h"
#include "tc.h"
#include "warp_solve.cuh"

using namespace mcsdp;

namespace {

struct Upload {
  size_t off;
  const void *src;
  size_t bytes;
};

struct Chunk {
  int g0, g1;        // groups of the chunk
  int nrhs;          // right-hand sides (= columns of X̂ / Y^{-1}) of the chunk
  int64_t rhs_begin; // into rowof_all / goff offsets
  int64_t tkey_begin;
  int64_t tile_begin;  // SCM tiles (h, g) of the chunk
  int ntiles;
};

constexpr int NCAND = 16;  // candidates per dual step-length round
constexpr int LZ_MAX = 64;  // Lanczos steps of the dense-root step-length bounds
// mixed form: from this m on the SCE is solved by GMRES preconditioned with the FP32 factor
constexpr int MIXED_LONG_M = 4096;
constexpr int GM_K = 40, GM_CYCLES = 8;  // GMRES restart length (<= 128) and cycles
// the largest clique (rows / columns) the shared-memory clique kernels take: Algorithm 1 and the
// primal step stage two k x k FP64 blocks (2 k^2 8 B <= 208 KB at k = 112)
constexpr int SMALL_ROWS = 112, SMALL_COLS = 96;

}  // namespace

struct mcsdp_ctx {
  std::string err;
  mcsdp_options opt;
  ProblemData P;
  Symbolic S;
  cudaStream_t stream = nullptr;
  int device = -1;
  bool host_only = false;
  // workspace plan
  size_t ws_bytes = 0;
  std::vector<Upload> uploads;
  std::map<std::string, size_t> off;
  char *ws = nullptr;
  size_t ws_have = 0;
  DevSym D{};
  int64_t ldb = 0;
  int pmax = 0;
  std::vector<Chunk> chunks;
  std::vector<int> rowof_all;       // SCM right-hand side -> row of its unit vector (per chunk)
  std::vector<int> goff_all;        // per group: first right-hand side within its chunk
  std::vector<int2> tkey_all;       // per SCM tile of 32 right-hand sides: group range
  std::vector<uint32_t> reach_bits, need_bits;  // per group, one bit per supernode
  std::vector<int2> pm_tkey;        // per P-MATRIX tile of 32 columns: (tile, tile)
  std::vector<uint32_t> pm_bits;    // per P-MATRIX tile: supernodes on its columns' paths
  std::vector<uint32_t> pm_need;    // per P-MATRIX tile: supernodes the backward L̂ solve needs
  std::vector<int> pm_rowof;        // P-MATRIX right-hand side j -> row j (identity)
  // update-list chunks (see DevSym)
  std::vector<int> upd_c0end, xch_beg, xch_end, xch_t, xch_ub, xch_ue, lvl_xptr, xfst, lvl_fptr;
  std::vector<UpdMeta> upd_meta;
  std::vector<int64_t> lvl_active;  // scratch: per level, pairs a solve's skip rule keeps
  std::vector<int64_t> cmap_ptr, cmap_off;
  std::vector<LsLevel> lvl_info;
  std::vector<int64_t> xch_slotw, xch_slotf;
  int64_t nslotw = 0, nslotf = 0;
  int bit_words = 1;
  int pm_cols = 0;                  // P-MATRIX columns per chunk (multiple of 32)
  int64_t ldw = 0;                  // leading dimension of the solve buffers
  SolveCfg scfg{};
  int num_sms = 152;
  std::vector<int2> tiles_all;
  // block-diagonal SCM (more than one component, options.scm_blocks = 0): per internal
  // constraint, the row of B that holds its right-hand side (its component's end: a row of that
  // block's columns outside every diagonal block, or m for the last component); per component,
  // the offset of its diagonal-tile inverses in Binv (ncomp + 1 entries)
  bool blocks = false;
  std::vector<int> bord;
  std::vector<int64_t> binv_off;
  // and the blocks' tables for the one-launch factorisation and back substitution
  std::vector<int> bt_off, bt_m, bt_seg_blk, bt_seg_k;
  std::vector<int64_t> bt_soff, bt_seg_start, bt_seg_l0;
  DagBlockTables bt{};
  std::vector<double> z0_default;
  bool z0_ok = false;
  // the input entries as given (caller order), for per-entry gradients
  int form = 1;
  std::vector<int> ue_k, ue_i, ue_j;
  std::vector<int64_t> ent_off;
  std::vector<int> ent_k, ent_pos;
  std::vector<double> ent_f;
  int64_t *ent_off_dev = nullptr;
  int *ent_k_dev = nullptr, *ent_pos_dev = nullptr;
  double *ent_f_dev = nullptr, *zsave = nullptr, *bwd_g = nullptr, *vrhs = nullptr;
  bool iterate_set = false;
  cudaEvent_t ev[8] = {};
  // the graph form of an iteration (options.graph): g = device step-length scalars, the
  // instantiated graph, and the launches it holds (per class) for the statistics
  double *gsc = nullptr;
  cudaGraphExec_t iter_exec = nullptr;
  bool graph_failed = false;  // capture not possible: iterate without the graph
  int64_t graph_launches = 0;
  int64_t graph_kcount[16] = {};
  // the solve graph (options.graph = 2): a WHILE node around the iteration and its loop test;
  // gcnt[0] iterations run, gcnt[1] the launch's iteration limit
  cudaGraphExec_t solve_exec = nullptr;
  bool solve_graph_failed = false;
  int *gcnt = nullptr;
  int64_t sgraph_launches = 0;
  int64_t sgraph_kcount[16] = {};
  cudaStream_t st2 = nullptr;                  // low priority: trailing updates, primal step
  cudaStream_t st1 = nullptr;                  // high priority: the Cholesky's critical path
  cudaStream_t stc = nullptr;                  // the graph iteration's capture (owned: a caller's
                                               // stream may be shared with other contexts)
  cudaStream_t st3 = nullptr;                  // low priority: the P-MATRIX's Y^{-1} columns
  cudaEvent_t ev_yinv = nullptr;               // st3 done with them
  cudaStream_t st4 = nullptr;                  // low priority: the SCM's N solves
  cudaEvent_t ev_n0 = nullptr, ev_n1 = nullptr;  // chunk's right-hand sides set / N solves done
  cudaEvent_t ev_f0 = nullptr, ev_f1 = nullptr;  // Algorithm 1 on st3: may start / done
  CholStreams cs;
  cudaEvent_t ev_next[2] = {}, ev_rest[2] = {};
  // device buffers
  double *Xbar = nullptr, *z = nullptr, *Ylay = nullptr, *N = nullptr, *dinvN = nullptr;
  double *Lh = nullptr, *dinvL = nullptr, *dY = nullptr, *dX = nullptr, *YinvE = nullptr;
  double *W3 = nullptr;  // Y^{-1} columns of the single P-MATRIX block (nullptr: several blocks)
  double *Pw2 = nullptr;          // partial slots and marks of the side streams' solves
  unsigned char *xvalid2 = nullptr;
  double *Pw3 = nullptr;
  unsigned char *xvalid3 = nullptr;
  double *Mlow = nullptr, *Mup = nullptr, *B = nullptr, *hvec = nullptr, *xs = nullptr;
  double *dz = nullptr, *W1 = nullptr, *W2 = nullptr, *Ncand = nullptr;
  double *Pw = nullptr, *Pf = nullptr, *Binv = nullptr;
  // mixed form: FP32 factor of B, FP64 refinement vectors
  float *B32 = nullptr, *Linv32 = nullptr;
  float *L32 = nullptr, *N32 = nullptr, *dL32 = nullptr, *dN32 = nullptr;  // FP32 factor copies
  bool f32_solves = false;      // the FP32 SCM / P-MATRIX solves fit the staged kernels
  double *gref = nullptr, *rref = nullptr, *yref = nullptr, *ayref = nullptr, *nref = nullptr;
  double *dscl = nullptr;  // the mixed factor's equilibration (large m)
  double *gmV = nullptr, *gmH = nullptr;  // GMRES basis and small vectors (large m)
  float *tinv = nullptr;  // the FP32 factor's diagonal-block inverses (large m)
  bool promoted = false;        // the FP64 factor is used for the rest of the solve
  bool fp64_asm = false;        // the SCM and the P-MATRIX are assembled in FP64 (mixed form)
  // mixed form, FP32 assembly stage with a dense root: the root blocks of Y and X̄ are factored
  // (and X̄_RR's factor inverted) in FP32, on the tensor cores for large roots (set per iteration
  // by mcsdp_solve; every other entry point factors in FP64)
  bool root32 = false;
  // mixed form after the FP32 stage: X̄_RR's factor FP64, its inverse (the primal Lanczos
  // operator) FP32 (set per iteration by mcsdp_solve)
  bool inv32 = false;
  int fp64_asm_iter = -1;
  int promoted_iter = -1, refine_steps = 0, cur_iter = 0;
  double *alpha_c = nullptr, *alpha_r = nullptr, *scal = nullptr;
  int *status = nullptr, *rowof_dev = nullptr, *goff_dev = nullptr, *pm_rowof_dev = nullptr;
  int2 *tiles_dev = nullptr, *tkey_dev = nullptr, *pm_tkey_dev = nullptr;
  uint32_t *reach_bits_dev = nullptr, *need_bits_dev = nullptr, *pm_bits_dev = nullptr;
  uint32_t *pm_need_dev = nullptr;
  // dense root (kern_root.cu): the root supernode's columns [nF, n) = R, nR = |R|; the dense
  // completion buffers W1 (X̂), W2 (Y^{-1}), W3 (X̂ dY) are n x ldw row-major with vertex k's
  // column at colw[k] (R first, the forest from column colF0 = nR rounded up to 32)
  bool dense = false;
  int nR = 0, nF = 0, colF0 = 0, nlev = 0;  // nlev: levels the small-clique kernels walk
  std::vector<int> colw, scm_vtx;
  int *scm_vtx_dev = nullptr;
  std::vector<int64_t> rg_ent, rg_ptr;
  std::vector<int> rg_u, rg_ab;
  RootGather rg{};
  // the forest-to-root block L_RF of L̂ (and of N) by root row, for the root's P-MATRIX
  std::vector<int64_t> lrf_ptr, lrf_off;
  std::vector<int> lrf_row;
  const int64_t *lrf_ptr_dev = nullptr, *lrf_off_dev = nullptr;
  const int *lrf_row_dev = nullptr;
  int *colw_dev = nullptr;
  double *RS_X = nullptr, *RS_P = nullptr, *RS_T = nullptr, *RS_M = nullptr;
  double *rLinvN = nullptr, *rLinvX = nullptr, *rLinv2 = nullptr;
  float *rLinv32 = nullptr;
  int *rsyncN = nullptr, *rsyncX = nullptr, *rsync2 = nullptr;
  size_t rsync_words = 0;
  double *lzQ = nullptr, *lzW = nullptr, *lzG = nullptr, *lzU = nullptr, *lzS = nullptr;
  double *Xprev = nullptr, *zprev = nullptr;
  double lz_last[4] = {0, 0, 0, 0};  // diagnostics of the last Lanczos bounds
  int lz_steps[2] = {0, 0};           // steps of the last primal (root) and dual bounds
  const double *Xbar_cur = nullptr;   // the X̄ the factors were last formed from
  double alpha_root_host = 1.0;       // source of the root clique's primal step copy
  float *tcr = nullptr;               // TF32 split operands of the root's tensor-core products
  int64_t tcr_kp = 0;                 // their row length (>= ldw, nR; multiple of 4)
  // kernel statistics
  int64_t launches = 0;
  int64_t kcount[16] = {};
  double kms[16] = {};
  std::vector<cudaEvent_t> evpool;
  std::vector<std::tuple<int, cudaEvent_t, cudaEvent_t>> pending;
};

void mcsdp::smem_optin(const void *kernel) {
  static std::mutex mu;
  static std::set<std::pair<int, const void *>> done;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  if (!done.insert({dev, kernel}).second) return;
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa{};
  cudaFuncGetAttributes(&fa, kernel);
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       optin - (int)fa.sharedSizeBytes);
}

namespace {

mcsdp_status fail(mcsdp_ctx *c, mcsdp_status s, const std::string &msg) {
  if (c) c->err = msg;
  return s;
}

#define CUDA_TRY(ctx, call)                                                                    \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return fail(ctx, MCSDP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));    \
  } while (0)

#define KCHECK(ctx)                                                                            \
  do {                                                                                         \
    cudaError_t e_ = cudaGetLastError();                                                       \
    if (e_ != cudaSuccess)                                                                     \
      return fail(ctx, MCSDP_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)); \
  } while (0)

size_t al(size_t b) { return (b + 255) & ~(size_t)255; }

enum KClass { KC_YCHOL = 0, KC_ALG1, KC_PANEL, KC_TILE, KC_CHOL, KC_BSOLVE, KC_PMAT, KC_PSTEP,
              KC_DSTEP, KC_MISC, KC_PMAT_SIDE, KC_PANEL_SIDE, KC_CHOL32, KC_RGEMM };

cudaEvent_t ev_get(mcsdp_ctx *c) {
  if (c->evpool.empty()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  cudaEvent_t e = c->evpool.back();
  c->evpool.pop_back();
  return e;
}

// Brackets the launches of one kernel class: counts them and, with profiling on, records CUDA
// events on the context's stream around them.
struct KScope {
  mcsdp_ctx *c;
  int cls;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  KScope(mcsdp_ctx *c_, int cls_, cudaStream_t s_ = nullptr) : c(c_), cls(cls_), s(s_ ? s_ : c_->stream) {
    if (c->opt.profile) {
      a = ev_get(c);
      cudaEventRecord(a, s);
    }
  }
  void done(int nlaunch) {
    c->launches += nlaunch;
    c->kcount[cls] += nlaunch;
    if (a) {
      cudaEvent_t b = ev_get(c);
      cudaEventRecord(b, s);
      c->pending.emplace_back(cls, a, b);
      a = nullptr;
    }
  }
};

// resolve recorded event pairs; call only after the stream has been synchronised
// (pairs recorded on the second stream may still be running: they stay pending)
void prof_flush(mcsdp_ctx *c) {
  std::vector<std::tuple<int, cudaEvent_t, cudaEvent_t>> keep;
  for (auto &p : c->pending) {
    if (cudaEventQuery(std::get<2>(p)) == cudaErrorNotReady) {
      if (cudaPeekAtLastError() == cudaErrorNotReady) (void)cudaGetLastError();
      keep.push_back(p);
      continue;
    }
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, std::get<1>(p), std::get<2>(p)) == cudaSuccess)
      c->kms[std::get<0>(p)] += ms;
    c->evpool.push_back(std::get<1>(p));
    c->evpool.push_back(std::get<2>(p));
  }
  c->pending.swap(keep);
}

template <class T>
void plan_table(mcsdp_ctx *c, size_t &cur, const std::string &name, const std::vector<T> &v) {
  c->off[name] = cur;
  if (!v.empty()) c->uploads.push_back({cur, v.data(), v.size() * sizeof(T)});
  cur += al(std::max<size_t>(v.size() * sizeof(T), 8));
}

void plan_buf(mcsdp_ctx *c, size_t &cur, const std::string &name, size_t bytes) {
  c->off[name] = cur;
  cur += al(std::max<size_t>(bytes, 8));
}

void plan_workspace(mcsdp_ctx *c) {
  Symbolic &S = c->S;
  const int64_t nnzL = S.sn_valptr[S.ns];
  const int64_t nnzD = S.sn_dptr[S.ns];
  const int n = S.n, m = S.m;
  size_t cur = 0;
  c->uploads.clear();
  c->dense = S.dense_root;
  c->nR = c->dense ? S.sn_col[S.ns] - S.sn_col[S.ns - 1] : 0;
  c->nF = n - c->nR;
  c->colF0 = (c->nR + 31) / 32 * 32;
  c->nlev = c->dense ? S.height - 1 : S.height;
  c->blocks = S.ncomp > 1 && c->opt.scm_blocks == 0;
  plan_table(c, cur, "sn_col", S.sn_col);
  plan_table(c, cur, "sn_rowptr", S.sn_rowptr);
  plan_table(c, cur, "rows", S.rows);
  plan_table(c, cur, "sn_valptr", S.sn_valptr);
  plan_table(c, cur, "sn_dptr", S.sn_dptr);
  plan_table(c, cur, "sn_parent", S.sn_parent);
  plan_table(c, cur, "col2sn", S.col2sn);
  plan_table(c, cur, "lvl_sn", S.lvl_sn);
  plan_table(c, cur, "upd_ptr", S.upd_ptr);
  plan_table(c, cur, "upd_src", S.upd_src);
  plan_table(c, cur, "upd_p1", S.upd_p1);
  plan_table(c, cur, "upd_p2", S.upd_p2);
  plan_table(c, cur, "upd_relptr", S.upd_relptr);
  plan_table(c, cur, "upd_rel", S.upd_rel);
  plan_table(c, cur, "slot_i", S.slot_i);
  plan_table(c, cur, "slot_j", S.slot_j);
  plan_table(c, cur, "slot_off", S.slot_off);
  plan_table(c, cur, "slot_ptr", S.slot_ptr);
  plan_table(c, cur, "slot_k", S.slot_k);
  plan_table(c, cur, "slot_val", S.slot_val);
  plan_table(c, cur, "slot_a0", S.slot_a0);
  plan_table(c, cur, "con_ptr", S.con_ptr);
  plan_table(c, cur, "con_off", S.con_off);
  plan_table(c, cur, "con_w", S.con_w);
  plan_table(c, cur, "con_v", S.con_v);
  plan_table(c, cur, "arow_ptr", S.arow_ptr);
  plan_table(c, cur, "arow_col", S.arow_col);
  plan_table(c, cur, "arow_off", S.arow_off);
  plan_table(c, cur, "rs_ptr", S.rs_ptr);
  plan_table(c, cur, "rs_col", S.rs_col);
  plan_table(c, cur, "rs_off", S.rs_off);
  plan_table(c, cur, "con_order", S.con_order);
  plan_table(c, cur, "grp_cptr", S.grp_cptr);
  plan_table(c, cur, "grp_pptr", S.grp_pptr);
  plan_table(c, cur, "grp_cols", S.grp_cols);
  plan_table(c, cur, "grp_rowoff", S.grp_rowoff);
  plan_table(c, cur, "anz_ptr", S.anz_ptr);
  plan_table(c, cur, "anz_a", S.anz_a);
  plan_table(c, cur, "anz_b", S.anz_b);
  plan_table(c, cur, "anz_v", S.anz_v);
  plan_table(c, cur, "reach_ptr", S.reach_ptr);
  plan_table(c, cur, "need_ptr", S.need_ptr);
  plan_table(c, cur, "reach_sn", S.reach_sn);
  plan_table(c, cur, "need_sn", S.need_sn);
  plan_table(c, cur, "sn_fdesc", S.sn_fdesc);
  plan_table(c, cur, "b", c->P.b);
  // ---- update lists in chunks: a target with a long list (the root clique of a block-arrow
  // pattern receives an update from nearly every clique) gets its extra chunks summed in
  // parallel by partial kernels, then added in fixed order (deterministic) ----
  {
    const double chunk_work = 256.0;
    c->upd_c0end.assign(S.ns, 0);
    c->xch_beg.assign(S.ns, 0);
    c->xch_end.assign(S.ns, 0);
    c->xch_t.clear(); c->xch_ub.clear(); c->xch_ue.clear();
    c->xch_slotw.clear(); c->xch_slotf.clear();
    c->nslotw = c->nslotf = 0;
    // levels of the targets: chunks are listed level by level
    std::vector<int> lvl_of(S.ns, 0);
    for (int l = 0; l < S.height; ++l)
      for (int q = S.lvl_ptr[l]; q < S.lvl_ptr[l + 1]; ++q) lvl_of[S.lvl_sn[q]] = l;
    c->lvl_xptr.assign(S.height + 1, 0);
    c->lvl_fptr.assign(S.height + 1, 0);
    c->xfst.clear();
    for (int l = 0; l < S.height; ++l) {
      c->lvl_xptr[l] = (int)c->xch_t.size();
      c->lvl_fptr[l] = (int)c->xfst.size();
      for (int q = S.lvl_ptr[l]; q < S.lvl_ptr[l + 1]; ++q) {
        const int t = S.lvl_sn[q];
        const int tncol = S.sn_col[t + 1] - S.sn_col[t];
        const int tnrow = (int)(S.sn_rowptr[t + 1] - S.sn_rowptr[t]);
        if (l >= c->nlev) {  // the dense root: its updates are gathered per entry instead
          c->upd_c0end[t] = S.upd_ptr[t + 1];
          c->xch_beg[t] = c->xch_end[t] = (int)c->xch_t.size();
          continue;
        }
        std::vector<int> cuts{S.upd_ptr[t]};
        double wsum = 0;
        for (int u = S.upd_ptr[t]; u < S.upd_ptr[t + 1]; ++u) {
          const int d = S.upd_src[u];
          const double w = (double)(S.upd_p2[u] - S.upd_p1[u]) * (S.sn_col[d + 1] - S.sn_col[d]);
          if (wsum > 0 && wsum + w > chunk_work) {
            cuts.push_back(u);
            wsum = 0;
          }
          wsum += w;
        }
        cuts.push_back(S.upd_ptr[t + 1]);
        c->upd_c0end[t] = cuts[1];
        c->xch_beg[t] = (int)c->xch_t.size();
        if (cuts.size() > 2) c->xfst.push_back((int)c->xch_t.size());
        for (size_t k = 1; k + 1 < cuts.size(); ++k) {
          c->xch_t.push_back(t);
          c->xch_ub.push_back(cuts[k]);
          c->xch_ue.push_back(cuts[k + 1]);
          c->xch_slotw.push_back(c->nslotw);
          c->xch_slotf.push_back(c->nslotf);
          c->nslotw += tncol;
          c->nslotf += (int64_t)tnrow * tncol;
        }
        c->xch_end[t] = (int)c->xch_t.size();
      }
    }
    c->lvl_xptr[S.height] = (int)c->xch_t.size();
    c->lvl_fptr[S.height] = (int)c->xfst.size();
    // per-update records and per-level bounds of the staged solve kernels
    c->upd_meta.assign(S.upd_src.size(), UpdMeta{});
    for (size_t u = 0; u < S.upd_src.size(); ++u) {
      const int d = S.upd_src[u];
      UpdMeta &q = c->upd_meta[u];
      q.dc0 = S.sn_col[d];
      q.dncol = S.sn_col[d + 1] - S.sn_col[d];
      q.dnrow = (int)(S.sn_rowptr[d + 1] - S.sn_rowptr[d]);
      q.p1 = S.upd_p1[u];
      q.np = S.upd_p2[u] - S.upd_p1[u];
      q.src = d;
      q.relptr = S.upd_relptr[u];
      q.valp = S.sn_valptr[d];
    }
    c->lvl_info.assign(S.height, LsLevel{0, 0, 0, 0});
    for (int l = 0; l < S.height; ++l) {
      LsLevel &lv = c->lvl_info[l];
      for (int q = S.lvl_ptr[l]; q < S.lvl_ptr[l + 1]; ++q) {
        const int t = S.lvl_sn[q];
        lv.nc = std::max(lv.nc, S.sn_col[t + 1] - S.sn_col[t]);
        lv.nr = std::max(lv.nr, (int)(S.sn_rowptr[t + 1] - S.sn_rowptr[t]));
        for (int u = S.upd_ptr[t]; u < S.upd_ptr[t + 1]; ++u) {
          lv.cw = std::max(lv.cw, std::min(8, c->upd_meta[u].dncol));
          lv.np = std::max(lv.np, c->upd_meta[u].np);
        }
      }
    }
    (void)lvl_of;
  }
  // dense root (K2 at the root): per entry of the root block, the contributions of the forest's
  // supernodes, in the order (source update, row a, row b) -- bucketed by root column, then each
  // column's entries ordered by row with a stable sort, so the order of every sum is fixed
  c->rg_ent.clear();
  c->rg_ptr.assign(1, 0);
  c->rg_u.clear();
  c->rg_ab.clear();
  if (c->dense) {
    const int rt = S.ns - 1, nR = c->nR;
    struct Ctb {
      int i, u, ab;
    };
    std::vector<int64_t> colcnt(nR + 1, 0);
    for (int u = S.upd_ptr[rt]; u < S.upd_ptr[rt + 1]; ++u) {
      const int np = S.upd_p2[u] - S.upd_p1[u];
      const int *rel = S.upd_rel.data() + S.upd_relptr[u];
      for (int bb = 0; bb < np; ++bb) colcnt[rel[bb] + 1] += np - bb;
    }
    for (int j = 0; j < nR; ++j) colcnt[j + 1] += colcnt[j];
    std::vector<Ctb> all((size_t)colcnt[nR]);
    std::vector<int64_t> at(colcnt.begin(), colcnt.end() - 1);
    for (int u = S.upd_ptr[rt]; u < S.upd_ptr[rt + 1]; ++u) {
      const int p1 = S.upd_p1[u], np = S.upd_p2[u] - p1;
      const int *rel = S.upd_rel.data() + S.upd_relptr[u];
      for (int aa = 0; aa < np; ++aa)
        for (int bb = 0; bb <= aa; ++bb)
          all[at[rel[bb]]++] = Ctb{rel[aa], u, (p1 + aa) | ((p1 + bb) << 16)};
    }
    for (int j = 0; j < nR; ++j) {
      auto b0 = all.begin() + colcnt[j], b1 = all.begin() + colcnt[j + 1];
      std::stable_sort(b0, b1, [](const Ctb &x, const Ctb &y) { return x.i < y.i; });
      for (auto it = b0; it != b1;) {
        auto e = it;
        while (e != b1 && e->i == it->i) ++e;
        c->rg_ent.push_back((int64_t)it->i + (int64_t)j * nR);
        for (auto q = it; q != e; ++q) {
          c->rg_u.push_back(q->u);
          c->rg_ab.push_back(q->ab);
        }
        c->rg_ptr.push_back((int64_t)c->rg_u.size());
        it = e;
      }
    }
  }
  // L_RF by root row: for every update u of the root from forest supernode d (rows p1 .. p2 of
  // d, at root rows rel[]), the entries L_d[p, q] of d's columns q, in (u, q) order per row
  c->lrf_ptr.assign(1, 0);
  c->lrf_off.clear();
  c->lrf_row.clear();
  if (c->dense) {
    const int rt = S.ns - 1, nR = c->nR;
    std::vector<int64_t> cnt(nR + 1, 0);
    for (int u = S.upd_ptr[rt]; u < S.upd_ptr[rt + 1]; ++u) {
      const int d = S.upd_src[u], ncd = S.sn_col[d + 1] - S.sn_col[d];
      const int *rel = S.upd_rel.data() + S.upd_relptr[u];
      for (int p = 0; p < S.upd_p2[u] - S.upd_p1[u]; ++p) cnt[rel[p] + 1] += ncd;
    }
    for (int r = 0; r < nR; ++r) cnt[r + 1] += cnt[r];
    c->lrf_off.resize((size_t)cnt[nR]);
    c->lrf_row.resize((size_t)cnt[nR]);
    std::vector<int64_t> at(cnt.begin(), cnt.end() - 1);
    for (int u = S.upd_ptr[rt]; u < S.upd_ptr[rt + 1]; ++u) {
      const int d = S.upd_src[u], c0 = S.sn_col[d], ncd = S.sn_col[d + 1] - c0;
      const int64_t nrd = S.sn_rowptr[d + 1] - S.sn_rowptr[d];
      const int *rel = S.upd_rel.data() + S.upd_relptr[u];
      for (int p = S.upd_p1[u]; p < S.upd_p2[u]; ++p) {
        const int r = rel[p - S.upd_p1[u]];
        for (int q = 0; q < ncd; ++q) {
          c->lrf_off[at[r]] = S.sn_valptr[d] + p + (int64_t)q * nrd;
          c->lrf_row[at[r]++] = c0 + q;
        }
      }
    }
    c->lrf_ptr = cnt;
  }
  plan_table(c, cur, "lrf_ptr", c->lrf_ptr);
  plan_table(c, cur, "lrf_off", c->lrf_off);
  plan_table(c, cur, "lrf_row", c->lrf_row);
  plan_table(c, cur, "rg_ent", c->rg_ent);
  plan_table(c, cur, "rg_ptr", c->rg_ptr);
  plan_table(c, cur, "rg_u", c->rg_u);
  plan_table(c, cur, "rg_ab", c->rg_ab);
  plan_table(c, cur, "upd_c0end", c->upd_c0end);
  plan_table(c, cur, "xch_beg", c->xch_beg);
  plan_table(c, cur, "xch_end", c->xch_end);
  plan_table(c, cur, "xch_t", c->xch_t);
  plan_table(c, cur, "xch_ub", c->xch_ub);
  plan_table(c, cur, "xch_ue", c->xch_ue);
  plan_table(c, cur, "xch_slotw", c->xch_slotw);
  plan_table(c, cur, "xch_slotf", c->xch_slotf);
  plan_table(c, cur, "xfst", c->xfst);
  plan_table(c, cur, "upd_meta", c->upd_meta);
  // clique entries outside the own columns of each clique: layout offsets (binary search in the
  // owning supernode's rows, done once here instead of per entry on the device)
  {
    c->cmap_ptr.assign(S.ns + 1, 0);
    c->cmap_off.clear();
    for (int r = 0; r < S.ns; ++r) {
      const int64_t r0 = S.sn_rowptr[r];
      const int k = (int)(S.sn_rowptr[r + 1] - r0);
      const int nsr = S.sn_col[r + 1] - S.sn_col[r];
      for (int i = 0; i < k - nsr; ++i)
        for (int j = 0; j <= i; ++j) {
          const int rr = S.rows[r0 + nsr + i], cc = S.rows[r0 + nsr + j];
          const int t = S.col2sn[cc];
          const int64_t t0 = S.sn_rowptr[t];
          const int tn = (int)(S.sn_rowptr[t + 1] - t0);
          const int lc = cc - S.sn_col[t];
          const int *b = S.rows.data() + t0;
          const int pos = (int)(std::lower_bound(b + lc, b + tn, rr) - b);
          c->cmap_off.push_back(S.sn_valptr[t] + pos + (int64_t)lc * tn);
        }
      c->cmap_ptr[r + 1] = (int64_t)c->cmap_off.size();
    }
  }
  // per input entry: layout offset of its lower position, matrix, index within the gradient
  // output of its kind (matrix 0 / matrices 1..m) and the factor (2 off the diagonal, the sign of
  // the input form for matrix 0)
  {
    const size_t ne = c->ue_k.size();
    c->ent_off.assign(ne, 0);
    c->ent_k.assign(ne, 0);
    c->ent_pos.assign(ne, 0);
    c->ent_f.assign(ne, 0.0);
    int n0 = 0, n1 = 0;
    for (size_t e = 0; e < ne; ++e) {
      const int a = S.iperm[c->ue_i[e]], b2 = S.iperm[c->ue_j[e]];
      const int rr = std::max(a, b2), cc = std::min(a, b2);
      const int t = S.col2sn[cc];
      const int64_t t0 = S.sn_rowptr[t];
      const int tn = (int)(S.sn_rowptr[t + 1] - t0);
      const int lc = cc - S.sn_col[t];
      const int *rb = S.rows.data() + t0;
      const int pos = (int)(std::lower_bound(rb + lc, rb + tn, rr) - rb);
      c->ent_off[e] = S.sn_valptr[t] + pos + (int64_t)lc * tn;
      c->ent_k[e] = c->ue_k[e];
      c->ent_pos[e] = c->ue_k[e] == 0 ? n0++ : n1++;
      c->ent_f[e] = (c->ue_i[e] != c->ue_j[e] ? 2.0 : 1.0) * (c->ue_k[e] == 0 && c->form == 0 ? -1.0 : 1.0);
    }
  }
  plan_table(c, cur, "ent_off", c->ent_off);
  plan_table(c, cur, "ent_k", c->ent_k);
  plan_table(c, cur, "ent_pos", c->ent_pos);
  plan_table(c, cur, "ent_f", c->ent_f);
  plan_table(c, cur, "cmap_ptr", c->cmap_ptr);
  plan_table(c, cur, "cmap_off", c->cmap_off);
  // ---- many-right-hand-side solves (kern_lsolve.cu): skip bitmaps and chunk plan ----
  const double budget = (c->opt.panel_budget_mb > 0 ? c->opt.panel_budget_mb : 1024.0) * 1048576.0;
  c->bit_words = (S.ns + 31) / 32;
  const int words = c->bit_words;
  c->reach_bits.assign((size_t)S.ngroup * words, 0u);
  c->need_bits.assign((size_t)S.ngroup * words, 0u);
  for (int g = 0; g < S.ngroup; ++g) {
    for (int64_t t = S.reach_ptr[g]; t < S.reach_ptr[g + 1]; ++t)
      c->reach_bits[(size_t)g * words + (S.reach_sn[t] >> 5)] |= 1u << (S.reach_sn[t] & 31);
    for (int64_t t = S.need_ptr[g]; t < S.need_ptr[g + 1]; ++t)
      c->need_bits[(size_t)g * words + (S.need_sn[t] >> 5)] |= 1u << (S.need_sn[t] & 31);
  }
  c->chunks.clear();
  c->rowof_all.clear();
  c->tkey_all.clear();
  c->tiles_all.clear();
  c->goff_all.assign(S.ngroup, 0);
  c->pmax = 0;
  int max_rhs = 0;
  // dense root: one chunk of every group (X̂ and Y^{-1} are formed whole)
  const double chunk_budget = c->dense ? std::numeric_limits<double>::infinity() : budget;
  for (int g = 0; g < S.ngroup;) {
    Chunk ch{};
    ch.g0 = g;
    ch.rhs_begin = (int64_t)c->rowof_all.size();
    ch.tkey_begin = (int64_t)c->tkey_all.size();
    ch.tile_begin = (int64_t)c->tiles_all.size();
    int nr = 0;
    std::vector<int> grp_of_rhs;
    while (g < S.ngroup) {
      const int pg = S.grp_pptr[g + 1] - S.grp_pptr[g];
      const double bytes = 2.0 * n * 8.0 * (((nr + pg) + 31) / 32 * 32);
      if (g > ch.g0 && bytes > chunk_budget) break;
      c->goff_all[g] = nr;
      for (int q = 0; q < pg; ++q) {
        c->rowof_all.push_back(S.grp_cols[S.grp_pptr[g] + q]);
        grp_of_rhs.push_back(g);
      }
      nr += pg;
      c->pmax = std::max(c->pmax, pg);
      // groups are contiguous per component: the tiles below the first group of another
      // component are zero blocks of B
      for (int h = g; h < S.ngroup; ++h) {
        if (c->blocks && S.grp_comp[h] != S.grp_comp[g]) break;
        c->tiles_all.push_back(make_int2(h, g));
      }
      ++g;
    }
    ch.g1 = g;
    ch.nrhs = nr;
    for (int t0 = 0; t0 < nr; t0 += 32)
      c->tkey_all.push_back(make_int2(grp_of_rhs[t0], grp_of_rhs[std::min(nr, t0 + 32) - 1]));
    ch.ntiles = (int)((int64_t)c->tiles_all.size() - ch.tile_begin);
    c->chunks.push_back(ch);
    max_rhs = std::max(max_rhs, nr);
  }
  // P-MATRIX: columns in chunks of pm_cols (multiple of 32); per 32-column tile the supernodes on
  // the columns' etree paths (forward reach of the unit right-hand sides)
  {
    // all n columns at once when the budget allows (a ragged last chunk would pay the latency of
    // every level again for a few columns)
    int pmc = (int)std::min<double>((double)n, budget / (2.0 * n * 8.0));
    pmc = pmc >= n ? (n + 31) / 32 * 32 : std::max(32, pmc / 32 * 32);
    c->pm_cols = std::min(pmc, (n + 31) / 32 * 32);
    const int ntile = (n + 31) / 32;
    c->pm_bits.assign((size_t)ntile * words, 0u);
    // M = X̂ dY Y^{-1} is kept only on E: column k needs the rows i >= k of k's clique and the
    // rows i < k with (k, i) in E; the backward substitution for a row needs its supernode and
    // all that supernode's ancestors
    c->pm_need.assign((size_t)ntile * words, 0u);
    auto mark_path = [&](int tl, int s2) {
      for (; s2 >= 0; s2 = S.sn_parent[s2]) {
        uint32_t &wd = c->pm_need[(size_t)tl * words + (s2 >> 5)];
        if (wd & (1u << (s2 & 31))) break;
        wd |= 1u << (s2 & 31);
      }
    };
    for (int tl = 0; tl < ntile; ++tl)
      for (int k = tl * 32; k < std::min(n, tl * 32 + 32); ++k) {
        const int t = S.col2sn[k];
        for (int64_t p = S.sn_rowptr[t]; p < S.sn_rowptr[t + 1]; ++p)
          mark_path(tl, S.col2sn[S.rows[p]]);
        for (int q = S.rs_ptr[k]; q < S.rs_ptr[k + 1]; ++q) mark_path(tl, S.col2sn[S.rs_col[q]]);
      }
    c->pm_tkey.resize(ntile);
    for (int tl = 0; tl < ntile; ++tl) {
      c->pm_tkey[tl] = make_int2(tl, tl);
      for (int k = tl * 32; k < std::min(n, tl * 32 + 32); ++k)
        for (int s2 = S.col2sn[k]; s2 >= 0; s2 = S.sn_parent[s2]) {
          uint32_t &wd = c->pm_bits[(size_t)tl * words + (s2 >> 5)];
          if (wd & (1u << (s2 & 31))) break;
          wd |= 1u << (s2 & 31);
        }
    }
    c->pm_rowof.resize(n);
    for (int k = 0; k < n; ++k) c->pm_rowof[k] = k;
  }
  c->ldw = ((int64_t)std::max(max_rhs, c->pm_cols) + 31) / 32 * 32;
  c->colw.clear();
  if (c->dense) {
    c->ldw = c->colF0 + ((int64_t)c->nF + 31) / 32 * 32;
    c->colw.resize(n);
    for (int k = 0; k < n; ++k) c->colw[k] = k < c->nF ? c->colF0 + k : k - c->nF;
  }
  plan_table(c, cur, "colw", c->colw);
  // max-cut-shaped constraints on the dense path: the vertex (new index) of each internal
  // constraint, for the streamed Hadamard SCM
  c->scm_vtx.clear();
  if (c->dense && S.unit_diag_constraints) {
    c->scm_vtx.resize(m);
    for (int i = 0; i < m; ++i) c->scm_vtx[i] = S.iperm[S.con_order[i]];
  }
  plan_table(c, cur, "scm_vtx", c->scm_vtx);
  plan_table(c, cur, "rowof", c->rowof_all);
  plan_table(c, cur, "goff", c->goff_all);
  plan_table(c, cur, "tkey", c->tkey_all);
  plan_table(c, cur, "tiles", c->tiles_all);
  plan_table(c, cur, "reach_bits", c->reach_bits);
  plan_table(c, cur, "need_bits", c->need_bits);
  plan_table(c, cur, "pm_bits", c->pm_bits);
  plan_table(c, cur, "pm_need", c->pm_need);
  plan_table(c, cur, "pm_tkey", c->pm_tkey);
  plan_table(c, cur, "pm_rowof", c->pm_rowof);
  // iteration buffers
  c->ldb = ((int64_t)m + 1 + 31) / 32 * 32;
  plan_buf(c, cur, "Xbar", nnzL * 8);
  plan_buf(c, cur, "zsave", (size_t)m * 8);
  plan_buf(c, cur, "bwd_g", nnzL * 8);
  plan_buf(c, cur, "vrhs", (size_t)m * 8);
  plan_buf(c, cur, "z", (size_t)m * 8);
  plan_buf(c, cur, "Ylay", nnzL * 8);
  plan_buf(c, cur, "N", nnzL * 8);
  plan_buf(c, cur, "dinvN", (size_t)nnzD * 8);
  plan_buf(c, cur, "Lh", nnzL * 8);
  plan_buf(c, cur, "dinvL", (size_t)nnzD * 8);
  plan_buf(c, cur, "dY", nnzL * 8);
  plan_buf(c, cur, "dX", nnzL * 8);
  plan_buf(c, cur, "YinvE", nnzL * 8);
  plan_buf(c, cur, "Mlow", nnzL * 8);
  plan_buf(c, cur, "Mup", nnzL * 8);
  plan_buf(c, cur, "B", (size_t)c->ldb * m * 8);
  plan_buf(c, cur, "hvec", (size_t)m * 8);
  c->binv_off.assign(1, 0);
  c->bord.clear();
  for (int q = 0; q < (c->blocks ? S.ncomp : 1); ++q) {
    const int o = c->blocks ? S.comp_cptr[q] : 0, e = c->blocks ? S.comp_cptr[q + 1] : m;
    if (c->blocks)
      for (int i = o; i < e; ++i) c->bord.push_back(e);
    c->binv_off.push_back(c->binv_off.back() + (int64_t)((e - o + 63) / 64) * 64 * 64);
  }
  plan_table(c, cur, "bord", c->bord);
  plan_buf(c, cur, "Binv", (size_t)c->binv_off.back() * 8);
  c->bt = DagBlockTables{};
  c->bt_off.clear();
  c->bt_m.clear();
  c->bt_soff.clear();
  c->bt_seg_blk.clear();
  c->bt_seg_k.clear();
  c->bt_seg_start.clear();
  c->bt_seg_l0.clear();
  if (c->blocks) {
    for (int q = 0; q < S.ncomp; ++q) {
      c->bt_off.push_back(S.comp_cptr[q]);
      c->bt_m.push_back(S.comp_cptr[q + 1] - S.comp_cptr[q]);
      c->bt.max_m = std::max(c->bt.max_m, c->bt_m.back());
    }
    DagBlockPlan pl;
    chol_dag_block_plan(c->bt_m, pl);
    c->bt_soff = pl.soff;
    c->bt_seg_start = pl.seg_start;
    c->bt_seg_l0 = pl.seg_l0;
    c->bt_seg_blk = pl.seg_blk;
    c->bt_seg_k = pl.seg_k;
    c->bt.nblk = S.ncomp;
    c->bt.nseg = (int)pl.seg_blk.size();
    c->bt.total = pl.total;
    c->bt.tile_words = pl.tile_words;
    c->bt.words = pl.words;
    c->bt.useful_ctas = pl.useful_ctas;
  }
  plan_table(c, cur, "bt_off", c->bt_off);
  plan_table(c, cur, "bt_m", c->bt_m);
  plan_table(c, cur, "bt_soff", c->bt_soff);
  plan_table(c, cur, "bt_loff", c->binv_off);
  plan_table(c, cur, "bt_seg_start", c->bt_seg_start);
  plan_table(c, cur, "bt_seg_l0", c->bt_seg_l0);
  plan_table(c, cur, "bt_seg_blk", c->bt_seg_blk);
  plan_table(c, cur, "bt_seg_k", c->bt_seg_k);
  plan_buf(c, cur, "xs", (size_t)m * 8);
  plan_buf(c, cur, "dz", (size_t)m * 8);
  plan_buf(c, cur, "W1", (size_t)n * c->ldw * 8);
  plan_buf(c, cur, "W2", (size_t)n * c->ldw * 8);
  // one P-MATRIX block: its Y^{-1} columns get a buffer of their own, so they can be formed
  // while the SCE is solved
  plan_buf(c, cur, "W3", (c->pm_cols >= n || c->dense) ? (size_t)n * c->ldw * 8 : 0);
  plan_buf(c, cur, "Pw", (size_t)std::max<int64_t>(1, c->nslotw) * c->ldw * 8);
  plan_buf(c, cur, "Pf", (size_t)std::max<int64_t>(1, c->nslotf) * NCAND * 8);
  plan_buf(c, cur, "xvalid", std::max<size_t>(1, c->xch_t.size()) * (size_t)(c->ldw / 32));
  // the side stream's own partial slots and marks (single P-MATRIX block: its Y^{-1} columns
  // are solved beside the SCM solves)
  const bool side = c->pm_cols >= n && !c->dense;
  plan_buf(c, cur, "Pw2", side ? (size_t)std::max<int64_t>(1, c->nslotw) * c->ldw * 8 : 0);
  plan_buf(c, cur, "xvalid2", side ? std::max<size_t>(1, c->xch_t.size()) * (size_t)(c->ldw / 32) : 0);
  plan_buf(c, cur, "Pw3", (size_t)std::max<int64_t>(1, c->nslotw) * c->ldw * 8);
  plan_buf(c, cur, "xvalid3", std::max<size_t>(1, c->xch_t.size()) * (size_t)(c->ldw / 32));
  plan_buf(c, cur, "Ncand", c->dense ? 0 : (size_t)NCAND * nnzL * 8);
  {
    const size_t r2 = (size_t)c->nR * c->nR * 8, rl = (size_t)((c->nR + 31) / 32) * 1024;
    c->rsync_words = c->dense ? chol_dag_words(c->nR, c->nR) : 0;
    plan_buf(c, cur, "RS_X", r2);
    plan_buf(c, cur, "RS_P", r2);
    plan_buf(c, cur, "RS_T", r2);
    // RS_M is also the triangular inverse's work area: 256 (nR + 256) values
    plan_buf(c, cur, "RS_M", c->dense ? std::max(r2, (size_t)256 * (c->nR + 256) * 8) : 0);
    plan_buf(c, cur, "rLinvN", rl * 8);
    plan_buf(c, cur, "rLinvX", rl * 8);
    plan_buf(c, cur, "rLinv2", rl * 8);
    plan_buf(c, cur, "rLinv32", rl * 4);
    plan_buf(c, cur, "rsyncN", c->rsync_words * 4);
    plan_buf(c, cur, "rsyncX", c->rsync_words * 4);
    plan_buf(c, cur, "rsync2", c->rsync_words * 4);
    const size_t nv = c->dense ? (size_t)n : 0;
    plan_buf(c, cur, "lzQ", 2 * nv * (LZ_MAX + 1) * 8);
    plan_buf(c, cur, "lzW", nv * 8);
    plan_buf(c, cur, "lzG", nv * 8);
    plan_buf(c, cur, "lzU", 2 * std::max<size_t>(nv, c->ldw) * 8);
    plan_buf(c, cur, "lzS", (4 * LZ_MAX + 8) * 8);
    plan_buf(c, cur, "Xprev", c->dense ? nnzL * 8 : 0);
    // mixed form with a dense root: the TF32 hi / lo parts of the root's product operands (the
    // P-MATRIX's rows of X̂ dY and Y^{-1}, or the inverse factor for Y^{-1}_RR)
    const bool rtc = c->dense && c->opt.precision == 1 && c->opt.tensor_cores != 0;
    const size_t kp = ((size_t)std::max<int64_t>(c->ldw, c->nR) + 3) / 4 * 4;
    c->tcr_kp = (int64_t)kp;
    plan_buf(c, cur, "tcr", rtc ? 4 * (size_t)c->nR * kp * 4 + 256 : 0);
    plan_buf(c, cur, "zprev", c->dense ? (size_t)m * 8 : 0);
  }
  plan_buf(c, cur, "alpha_c", NCAND * 8);
  plan_buf(c, cur, "gsc", 16 * 8);
  plan_buf(c, cur, "gcnt", 16);
  plan_buf(c, cur, "alpha_r", (size_t)S.ns * 8);
  plan_buf(c, cur, "scal", (16 + 6 * 64) * 8);  // scalars, then the measures' partials
  plan_buf(c, cur, "chol_sync", std::max(chol_dag_words(m, m + 1), c->bt.words) * 4);
  plan_buf(c, cur, "status", (8 + NCAND) * 4);  // [0..3] phases, [4] FP32 factor, [8..8+NCAND) dual candidates
  {
    const bool mx = c->opt.precision == 1;
    const size_t nblk = (size_t)(m + 31) / 32;
    plan_buf(c, cur, "B32", mx ? (size_t)m * m * 4 : 0);
    plan_buf(c, cur, "Linv32", mx ? nblk * 32 * 32 * 4 : 0);
    plan_buf(c, cur, "gref", mx ? (size_t)m * 8 : 0);
    plan_buf(c, cur, "rref", mx ? (size_t)m * 8 : 0);
    plan_buf(c, cur, "yref", mx ? (size_t)mixed_chunks(m) * m * 8 : 0);
    plan_buf(c, cur, "ayref", mx ? (size_t)mixed_chunks(m) * m * 8 : 0);
    plan_buf(c, cur, "nref", 4 * 8);
    plan_buf(c, cur, "dscl", mx ? (size_t)m * 8 : 0);
    const bool gm = mx && m >= MIXED_LONG_M;
    plan_buf(c, cur, "gmV", gm ? (size_t)(GM_K + 2) * m * 8 : 0);
    plan_buf(c, cur, "gmH", gm ? (size_t)6 * (GM_K + 2) * 8 : 0);
    plan_buf(c, cur, "tinv", gm ? (size_t)trsv_tinv_buffer_floats(m) * 4 : 0);
    const bool tc = mx && c->opt.tensor_cores != 0 && m >= 2 * TC_PANEL;
    // two buffers each: the chain splits panel k + 1 while panel k's update still reads k's
    plan_buf(c, cur, "tc_hi", tc ? (size_t)2 * tc_panel(m) * m * 4 : 0);
    plan_buf(c, cur, "tc_lo", tc ? (size_t)2 * tc_panel(m) * m * 4 : 0);
    plan_buf(c, cur, "L32", mx ? (size_t)nnzL * 4 : 0);
    plan_buf(c, cur, "N32", mx ? (size_t)nnzL * 4 : 0);
    plan_buf(c, cur, "dL32", mx ? (size_t)nnzD * 4 : 0);
    plan_buf(c, cur, "dN32", mx ? (size_t)nnzD * 4 : 0);
    c->f32_solves = mx && lsolve_staged_fits(c->lvl_info.data(), c->nlev, 4);
  }  // [0..3] phases, [8..8+NCAND) dual candidates
  c->ws_bytes = cur;
}

template <class T>
T *wsp(mcsdp_ctx *c, const char *name) {
  return reinterpret_cast<T *>(c->ws + c->off.at(name));
}

void bind_pointers(mcsdp_ctx *c) {
  Symbolic &S = c->S;
  DevSym &D = c->D;
  D.n = S.n;
  D.m = S.m;
  D.ns = S.ns;
  D.ngroup = S.ngroup;
  // the small-clique kernels size their shared memory from the forest's cliques (the dense
  // root has kernels of its own)
  D.nforest = c->dense ? S.ns - 1 : S.ns;
  D.nR = c->nR;
  D.root_valp = c->dense ? S.sn_valptr[S.ns - 1] : 0;
  D.max_nrow = D.max_ncol = 0;
  for (int t = 0; t < D.nforest; ++t) {
    D.max_nrow = std::max(D.max_nrow, (int)(S.sn_rowptr[t + 1] - S.sn_rowptr[t]));
    D.max_ncol = std::max(D.max_ncol, S.sn_col[t + 1] - S.sn_col[t]);
  }
  D.max_grp_nnz = 0;
  for (int g = 0; g < S.ngroup; ++g)
    D.max_grp_nnz = std::max(D.max_grp_nnz, S.anz_ptr[S.grp_cptr[g + 1]] - S.anz_ptr[S.grp_cptr[g]]);
  D.max_con_nnz = 0;
  for (int i = 0; i < S.m; ++i) D.max_con_nnz = std::max(D.max_con_nnz, S.anz_ptr[i + 1] - S.anz_ptr[i]);
  D.nnzL = S.sn_valptr[S.ns];
  D.nslot = S.nslot;
  D.nnzD = S.sn_dptr[S.ns];
  D.sn_col = wsp<int>(c, "sn_col");
  D.sn_dptr = wsp<int64_t>(c, "sn_dptr");
  D.sn_rowptr = wsp<int64_t>(c, "sn_rowptr");
  D.rows = wsp<int>(c, "rows");
  D.sn_valptr = wsp<int64_t>(c, "sn_valptr");
  D.sn_parent = wsp<int>(c, "sn_parent");
  D.col2sn = wsp<int>(c, "col2sn");
  D.lvl_sn = wsp<int>(c, "lvl_sn");
  D.upd_ptr = wsp<int>(c, "upd_ptr");
  D.upd_src = wsp<int>(c, "upd_src");
  D.upd_p1 = wsp<int>(c, "upd_p1");
  D.upd_p2 = wsp<int>(c, "upd_p2");
  D.upd_relptr = wsp<int64_t>(c, "upd_relptr");
  D.upd_rel = wsp<int>(c, "upd_rel");
  D.slot_i = wsp<int>(c, "slot_i");
  D.slot_j = wsp<int>(c, "slot_j");
  D.slot_off = wsp<int64_t>(c, "slot_off");
  D.slot_ptr = wsp<int>(c, "slot_ptr");
  D.slot_k = wsp<int>(c, "slot_k");
  D.slot_val = wsp<double>(c, "slot_val");
  D.slot_a0 = wsp<double>(c, "slot_a0");
  D.con_ptr = wsp<int>(c, "con_ptr");
  D.con_off = wsp<int64_t>(c, "con_off");
  D.con_w = wsp<double>(c, "con_w");
  D.con_v = wsp<double>(c, "con_v");
  D.arow_ptr = wsp<int>(c, "arow_ptr");
  D.arow_col = wsp<int>(c, "arow_col");
  D.arow_off = wsp<int64_t>(c, "arow_off");
  D.rs_ptr = wsp<int>(c, "rs_ptr");
  D.rs_col = wsp<int>(c, "rs_col");
  D.rs_off = wsp<int64_t>(c, "rs_off");
  D.con_order = wsp<int>(c, "con_order");
  D.bord = c->blocks ? wsp<int>(c, "bord") : nullptr;
  D.grp_cptr = wsp<int>(c, "grp_cptr");
  D.grp_pptr = wsp<int>(c, "grp_pptr");
  D.grp_cols = wsp<int>(c, "grp_cols");
  D.grp_rowoff = wsp<int64_t>(c, "grp_rowoff");
  D.anz_ptr = wsp<int>(c, "anz_ptr");
  D.anz_a = wsp<int16_t>(c, "anz_a");
  D.anz_b = wsp<int16_t>(c, "anz_b");
  D.anz_v = wsp<double>(c, "anz_v");
  D.reach_ptr = wsp<int64_t>(c, "reach_ptr");
  D.need_ptr = wsp<int64_t>(c, "need_ptr");
  D.reach_sn = wsp<int>(c, "reach_sn");
  D.need_sn = wsp<int>(c, "need_sn");
  D.sn_fdesc = wsp<int>(c, "sn_fdesc");

  D.b = wsp<double>(c, "b");
  c->Xbar = wsp<double>(c, "Xbar");
  c->zsave = wsp<double>(c, "zsave");
  c->bwd_g = wsp<double>(c, "bwd_g");
  c->vrhs = wsp<double>(c, "vrhs");
  c->ent_off_dev = wsp<int64_t>(c, "ent_off");
  c->ent_k_dev = wsp<int>(c, "ent_k");
  c->ent_pos_dev = wsp<int>(c, "ent_pos");
  c->ent_f_dev = wsp<double>(c, "ent_f");
  c->z = wsp<double>(c, "z");
  c->Ylay = wsp<double>(c, "Ylay");
  c->N = wsp<double>(c, "N");
  c->dinvN = wsp<double>(c, "dinvN");
  c->Lh = wsp<double>(c, "Lh");
  c->dinvL = wsp<double>(c, "dinvL");
  c->dY = wsp<double>(c, "dY");
  c->dX = wsp<double>(c, "dX");
  c->YinvE = wsp<double>(c, "YinvE");
  c->Mlow = wsp<double>(c, "Mlow");
  c->Mup = wsp<double>(c, "Mup");
  c->B = wsp<double>(c, "B");
  c->hvec = wsp<double>(c, "hvec");
  c->Binv = wsp<double>(c, "Binv");
  c->xs = wsp<double>(c, "xs");
  c->dz = wsp<double>(c, "dz");
  c->W1 = wsp<double>(c, "W1");
  c->W2 = wsp<double>(c, "W2");
  c->W3 = (c->pm_cols >= c->S.n || c->dense) ? wsp<double>(c, "W3") : nullptr;
  c->Pw = wsp<double>(c, "Pw");
  const bool side = c->pm_cols >= c->S.n && !c->dense;
  c->Pw2 = side ? wsp<double>(c, "Pw2") : nullptr;
  c->xvalid2 = side ? wsp<unsigned char>(c, "xvalid2") : nullptr;
  c->Pw3 = wsp<double>(c, "Pw3");
  c->xvalid3 = wsp<unsigned char>(c, "xvalid3");
  c->Pf = wsp<double>(c, "Pf");
  D.upd_c0end = wsp<int>(c, "upd_c0end");
  D.xch_beg = wsp<int>(c, "xch_beg");
  D.xch_end = wsp<int>(c, "xch_end");
  D.xch_t = wsp<int>(c, "xch_t");
  D.xch_ub = wsp<int>(c, "xch_ub");
  D.xch_ue = wsp<int>(c, "xch_ue");
  D.xch_slotw = wsp<int64_t>(c, "xch_slotw");
  D.xch_slotf = wsp<int64_t>(c, "xch_slotf");
  D.xfst = wsp<int>(c, "xfst");
  D.xvalid = wsp<unsigned char>(c, "xvalid");
  D.xv_stride = (int)(c->ldw / 32);
  D.upd_meta = wsp<UpdMeta>(c, "upd_meta");
  D.cmap_ptr = wsp<int64_t>(c, "cmap_ptr");
  D.cmap_off = wsp<int64_t>(c, "cmap_off");
  D.nslotw = c->nslotw;
  D.nslotf = c->nslotf;
  c->Ncand = wsp<double>(c, "Ncand");
  c->alpha_c = wsp<double>(c, "alpha_c");
  c->gsc = wsp<double>(c, "gsc");
  c->gcnt = wsp<int>(c, "gcnt");
  c->alpha_r = wsp<double>(c, "alpha_r");
  c->scal = wsp<double>(c, "scal");
  c->status = wsp<int>(c, "status");
  c->cs.dag_sync = wsp<int>(c, "chol_sync");
  c->cs.dag_words = std::max(chol_dag_words(c->S.m, c->S.m + 1), c->bt.words);
  if (c->blocks) {
    c->bt.off = wsp<int>(c, "bt_off");
    c->bt.mb = wsp<int>(c, "bt_m");
    c->bt.soff = wsp<int64_t>(c, "bt_soff");
    c->bt.loff = wsp<int64_t>(c, "bt_loff");
    c->bt.seg_start = wsp<int64_t>(c, "bt_seg_start");
    c->bt.seg_l0 = wsp<int64_t>(c, "bt_seg_l0");
    c->bt.seg_blk = wsp<int>(c, "bt_seg_blk");
    c->bt.seg_k = wsp<int>(c, "bt_seg_k");
  }
  c->cs.dag_budget = c->opt.timeout_cycles;
  c->B32 = wsp<float>(c, "B32");
  c->Linv32 = wsp<float>(c, "Linv32");
  c->gref = wsp<double>(c, "gref");
  c->rref = wsp<double>(c, "rref");
  c->yref = wsp<double>(c, "yref");
  c->ayref = wsp<double>(c, "ayref");
  c->nref = wsp<double>(c, "nref");
  c->dscl = wsp<double>(c, "dscl");
  c->gmV = wsp<double>(c, "gmV");
  c->gmH = wsp<double>(c, "gmH");
  c->tinv = c->gmV ? wsp<float>(c, "tinv") : nullptr;
  {
    const bool tc = c->opt.precision == 1 && c->opt.tensor_cores != 0 && c->S.m >= 2 * TC_PANEL;
    c->cs.tc_hi = tc ? wsp<float>(c, "tc_hi") : nullptr;
    c->cs.tc_lo = tc ? wsp<float>(c, "tc_lo") : nullptr;
    c->cs.tc_rows = tc ? c->S.m : 0;
    c->cs.tc_err = nullptr;  // the factorisation's own status word
  }
  c->L32 = wsp<float>(c, "L32");
  c->N32 = wsp<float>(c, "N32");
  c->dL32 = wsp<float>(c, "dL32");
  c->dN32 = wsp<float>(c, "dN32");

  c->rowof_dev = wsp<int>(c, "rowof");
  c->goff_dev = wsp<int>(c, "goff");
  c->tkey_dev = wsp<int2>(c, "tkey");
  c->tiles_dev = wsp<int2>(c, "tiles");
  c->reach_bits_dev = wsp<uint32_t>(c, "reach_bits");
  c->need_bits_dev = wsp<uint32_t>(c, "need_bits");
  c->pm_bits_dev = wsp<uint32_t>(c, "pm_bits");
  c->pm_need_dev = wsp<uint32_t>(c, "pm_need");
  c->pm_tkey_dev = wsp<int2>(c, "pm_tkey");
  c->pm_rowof_dev = wsp<int>(c, "pm_rowof");
  c->colw_dev = wsp<int>(c, "colw");
  c->scm_vtx_dev = c->scm_vtx.empty() ? nullptr : wsp<int>(c, "scm_vtx");
  c->rg.nent = (int64_t)c->rg_ent.size();
  c->rg.ent = wsp<int64_t>(c, "rg_ent");
  c->rg.ptr = wsp<int64_t>(c, "rg_ptr");
  c->rg.u = wsp<int>(c, "rg_u");
  c->rg.ab = wsp<int>(c, "rg_ab");
  c->lrf_ptr_dev = wsp<int64_t>(c, "lrf_ptr");
  c->lrf_off_dev = wsp<int64_t>(c, "lrf_off");
  c->lrf_row_dev = wsp<int>(c, "lrf_row");
  c->RS_X = wsp<double>(c, "RS_X");
  c->RS_P = wsp<double>(c, "RS_P");
  c->RS_T = wsp<double>(c, "RS_T");
  c->RS_M = wsp<double>(c, "RS_M");
  c->rLinvN = wsp<double>(c, "rLinvN");
  c->rLinvX = wsp<double>(c, "rLinvX");
  c->rLinv2 = wsp<double>(c, "rLinv2");
  c->rLinv32 = wsp<float>(c, "rLinv32");
  c->rsyncN = wsp<int>(c, "rsyncN");
  c->rsyncX = wsp<int>(c, "rsyncX");
  c->rsync2 = wsp<int>(c, "rsync2");
  c->lzQ = wsp<double>(c, "lzQ");
  c->lzW = wsp<double>(c, "lzW");
  c->lzG = wsp<double>(c, "lzG");
  c->lzU = wsp<double>(c, "lzU");
  c->lzS = wsp<double>(c, "lzS");
  c->Xprev = wsp<double>(c, "Xprev");
  c->tcr = (c->dense && c->opt.precision == 1 && c->opt.tensor_cores != 0) ? wsp<float>(c, "tcr")
                                                                            : nullptr;
  c->zprev = wsp<double>(c, "zprev");
}

mcsdp_status ready(mcsdp_ctx *c) {
  if (!c) return MCSDP_ERR_ARG;
  if (c->host_only) return fail(c, MCSDP_ERR_STATE, "host-only context: no device work");
  if (!c->ws) return fail(c, MCSDP_ERR_STATE, "no workspace: call mcsdp_set_workspace first");
  CUDA_TRY(c, cudaSetDevice(c->device));
  return MCSDP_OK;
}

mcsdp_status read_status(mcsdp_ctx *c, int *h, int count) {
  CUDA_TRY(c, cudaMemcpyAsync(h, c->status, count * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  prof_flush(c);
  return MCSDP_OK;
}

// ---- phases ----

mcsdp_status phase_Y(mcsdp_ctx *c, const double *z) {
  CUDA_TRY(c, cudaMemsetAsync(c->Ylay, 0, c->D.nnzL * 8, c->stream));
  KScope ks(c, KC_MISC);
  launch_slot_combine(c->D, c->Ylay, z, 1.0, -1.0, c->stream);
  ks.done(1);
  KCHECK(c);
  return MCSDP_OK;
}

// K2 on ncand candidates Y + alpha_c dY (ncand = 1 and dY = NULL for Y itself).
mcsdp_status phase_ychol(mcsdp_ctx *c, int ncand, const double *alpha, const double *Yb,
                         const double *dY, double *Nbuf, double *dinv, int *status) {
  const Symbolic &S = c->S;
  if (ychol_smem_bytes(c->D) > 220 * 1024)
    return fail(c, MCSDP_ERR_ARG, "supernode too large for the shared-memory Cholesky kernel");
  if (c->dense && (ncand != 1 || dY))
    return fail(c, MCSDP_ERR_STATE, "internal: candidate factorisations with a dense root");
  KScope ks(c, ncand > 1 ? KC_DSTEP : KC_YCHOL);
  int nl = 0;
  for (int l = 0; l < c->nlev; ++l) {
    const int xb = c->lvl_xptr[l], xc = c->lvl_xptr[l + 1] - xb;
    if (xc > 0) {
      launch_ychol_partials(c->D, xb, xc, c->lvl_fptr[l], c->lvl_fptr[l + 1] - c->lvl_fptr[l], ncand,
                            Nbuf, c->Pf, status, c->stream);
      ++nl;
    }
    launch_ychol_level(c->D, S.lvl_ptr[l], S.lvl_ptr[l + 1] - S.lvl_ptr[l], ncand, alpha, Yb, dY,
                       Nbuf, dinv, status, c->Pf, c->stream);
    ++nl;
  }
  if (c->dense) {
    // the root: its block of Y less the forest's contributions, then the dense Cholesky
    launch_root_assemble(c->D, c->rg, Yb, nullptr, 0.0, Nbuf, c->stream);
    nl += c->rg.nent > 0 ? 2 : 1;
    const int nR = c->nR;
    double *NR = Nbuf + c->D.root_valp;
    if (c->root32) {
      // FP32 factor (its rows mirrored above the diagonal, as the FP64 one), stored back as FP64
      // values with its diagonal-block inverses, so the FP32 assembly reads it as before
      float *N32 = reinterpret_cast<float *>(c->RS_T);
      copy_square<double, float>(NR, nR, N32, nR, nR, c->stream);
      nl += 3 + dense_chol_f32(N32, nR, nR, status, c->rLinv32, c->stream, &c->cs);
      copy_square<float, double>(N32, nR, NR, nR, nR, c->stream);
      cast_f64(c->rLinv32, c->rLinvN, (int64_t)((nR + 31) / 32) * 1024, c->stream);
    } else {
      nl += dense_potrf(NR, nR, nR, status, c->rLinvN, c->stream, c->rsyncN, c->opt.timeout_cycles);
    }
  }
  ks.done(nl);
  KCHECK(c);
  return MCSDP_OK;
}

// the dense root's clique of X̄ (Algorithm 1 at the root needs X̄_RR^{-1}; the primal step needs
// a factor of X̄_RR): RS_X <- Cholesky factor of X̄_RR (positive definite, else status bit),
// RS_P <- its inverse with the inverse's rows mirrored above the diagonal
int factor_X_root(mcsdp_ctx *c, const double *Xbar, int *status, cudaStream_t st) {
  const int nR = c->nR;
  if (c->root32) {
    // FP32: the factor and its inverse in RS_X (two FP32 squares), the diagonal-block inverses in
    // rLinvX, the inverse widened into RS_P
    float *L32 = reinterpret_cast<float *>(c->RS_X), *X32 = L32 + (size_t)nR * nR;
    float *lin32 = reinterpret_cast<float *>(c->rLinvX);
    copy_square<double, float>(Xbar + c->D.root_valp, nR, L32, nR, nR, st);
    int nl = 1 + dense_chol_f32(L32, nR, nR, status, lin32, st, &c->cs);
    nl += dense_trtri<float>(L32, nR, lin32, X32, nR, nR, reinterpret_cast<float *>(c->RS_M), st);
    copy_square<float, double>(X32, nR, c->RS_P, nR, nR, st);
    mirror_lower<double>(c->RS_P, nR, nR, st);
    return nl + 2;
  }
  copy_square<double, double>(Xbar + c->D.root_valp, nR, c->RS_X, nR, nR, st);
  int nl = 1 + dense_potrf(c->RS_X, nR, nR, status, c->rLinvX, st, c->rsyncX, c->opt.timeout_cycles);
  if (c->inv32) {
    // FP64 factor (the iterate's PD certificate), its inverse in FP32: the inverse only applies
    // the Lanczos operator of the step-length bound
    float *L32 = reinterpret_cast<float *>(c->RS_T), *X32 = L32 + (size_t)nR * nR;
    copy_square<double, float>(c->RS_X, nR, L32, nR, nR, st);
    launch_cast_f32(c->rLinvX, c->rLinv32, (int64_t)((nR + 31) / 32) * 1024, st);
    nl += 2 + dense_trtri<float>(L32, nR, c->rLinv32, X32, nR, nR,
                                 reinterpret_cast<float *>(c->RS_M), st);
    copy_square<float, double>(X32, nR, c->RS_P, nR, nR, st);
  } else {
    nl += dense_trtri<double>(c->RS_X, nR, c->rLinvX, c->RS_P, nR, nR, c->RS_M, st);
  }
  mirror_lower<double>(c->RS_P, nR, nR, st);
  return nl + 1;
}

mcsdp_status factor_X(mcsdp_ctx *c, const double *Xbar) {
  if (alg1_smem_bytes(c->D) > 220 * 1024)
    return fail(c, MCSDP_ERR_ARG, "clique too large for the shared-memory Algorithm 1 kernel");
  c->Xbar_cur = Xbar;
  KScope ks(c, KC_ALG1);
  launch_alg1(c->D, Xbar, c->Lh, c->dinvL, c->status + 1, c->stream);
  int nl = 1;
  if (c->dense) nl += factor_X_root(c, Xbar, c->status + 1, c->stream);
  ks.done(nl);
  KCHECK(c);
  return MCSDP_OK;
}

// Y = N N^T and Algorithm 1 (L̂ from X̄) share nothing: Algorithm 1 runs on the side stream st3
// beside the Y factorisation (the status words are cleared before either starts)
mcsdp_status factor_YX(mcsdp_ctx *c, const double *Xbar) {
  if (alg1_smem_bytes(c->D) > 220 * 1024)
    return fail(c, MCSDP_ERR_ARG, "clique too large for the shared-memory Algorithm 1 kernel");
  c->Xbar_cur = Xbar;
  CUDA_TRY(c, cudaMemsetAsync(c->status, 0, 8 * sizeof(int), c->stream));
  CUDA_TRY(c, cudaEventRecord(c->ev_f0, c->stream));
  CUDA_TRY(c, cudaStreamWaitEvent(c->st3, c->ev_f0, 0));
  {
    KScope ks(c, KC_ALG1, c->st3);
    launch_alg1(c->D, Xbar, c->Lh, c->dinvL, c->status + 1, c->st3);
    int nl = 1;
    if (c->dense && !c->root32) nl += factor_X_root(c, Xbar, c->status + 1, c->st3);
    ks.done(nl);
  }
  CUDA_TRY(c, cudaEventRecord(c->ev_f1, c->st3));
  mcsdp_status s = phase_ychol(c, 1, nullptr, c->Ylay, nullptr, c->N, c->dinvN, c->status);
  CUDA_TRY(c, cudaStreamWaitEvent(c->stream, c->ev_f1, 0));
  if (s) return s;
  if (c->dense && c->root32) {
    // the FP32 root factorisations share the tensor-core Cholesky's working storage: X̄_RR's
    // after Y's, on the main stream
    KScope ks(c, KC_ALG1);
    ks.done(factor_X_root(c, Xbar, c->status + 1, c->stream));
  }
  KCHECK(c);
  return MCSDP_OK;
}

// factors in the element type of the solves: FP64 originals, or the FP32 copies of the mixed form
template <class T>
struct SolveFactors {
  const T *Lh, *dinvL, *N, *dinvN;
};
SolveFactors<double> factors_of(const mcsdp_ctx *c, double) {
  return {c->Lh, c->dinvL, c->N, c->dinvN};
}
SolveFactors<float> factors_of(const mcsdp_ctx *c, float) {
  return {c->L32, c->dL32, c->N32, c->dN32};
}

// FP32 copies of L̂, N and their diagonal-block inverses (mixed form)
void cast_factors(mcsdp_ctx *c) {
  KScope ks(c, KC_MISC);
  launch_cast_f32(c->Lh, c->L32, c->D.nnzL, c->stream);
  launch_cast_f32(c->N, c->N32, c->D.nnzL, c->stream);
  launch_cast_f32(c->dinvL, c->dL32, c->D.nnzD, c->stream);
  launch_cast_f32(c->dinvN, c->dN32, c->D.nnzD, c->stream);
  ks.done(4);
}

// Host copy of a skip rule (the bit rows and the key range of each tile of 32 right-hand sides);
// bits == nullptr keeps every (supernode, tile) pair.
struct SkipHost {
  const uint32_t *bits;
  const int2 *tile_keys;
};

template <class T>
int lsolve_c(mcsdp_ctx *c, bool fwd, const T *L, const T *Dinv, T *W, int ncols, const LsSkip &sk,
             const SkipHost &hk) {
  const Symbolic &S = c->S;
  // per level, the (supernode, tile) pairs the skip rule keeps: the launch shape depends on them
  int64_t *active = nullptr;
  if (hk.bits) {
    const int ntiles = (ncols + 31) / 32;
    c->lvl_active.assign(S.height, 0);
    for (int l = 0; l < c->nlev; ++l)
      for (int q = S.lvl_ptr[l]; q < S.lvl_ptr[l + 1]; ++q) {
        const int t = S.lvl_sn[q];
        for (int tl = 0; tl < ntiles; ++tl) {
          const int2 kr = hk.tile_keys[tl];
          for (int key = kr.x; key <= kr.y; ++key)
            if (hk.bits[(size_t)key * c->bit_words + (t >> 5)] & (1u << (t & 31))) {
              ++c->lvl_active[l];
              break;
            }
        }
      }
    active = c->lvl_active.data();
  }
  if (c->nlev <= 0) return 0;
  return lsolve<T>(c->D, S.lvl_ptr.data(), c->lvl_xptr.data(), c->lvl_fptr.data(),
                   c->lvl_info.data(), c->nlev, fwd, L, Dinv, W, c->ldw, ncols, sk,
                   reinterpret_cast<T *>(c->Pw), active, c->stream);
}

// C = alpha A^T B + beta C on the tensor cores for the dense root's FP32 products: operand rows
// A(:, i) = A[i a_r + l a_c] (l < K), likewise B; both split into TF32 hi / lo copies in c->tcr
// (one copy when A and B are the same operand), then the tcgen05 product
void root_tc_gemm(mcsdp_ctx *c, const float *A, int64_t a_r, int64_t a_c, int M, const float *B,
                  int64_t b_r, int64_t b_c, int N, int K, float *C, int64_t cs_i, int64_t cs_j,
                  float alpha, float beta, bool lower, bool mirror) {
  const int64_t kp = c->tcr_kp;
  float *ah = c->tcr, *al = ah + (size_t)c->nR * kp;
  float *bh = al + (size_t)c->nR * kp, *bl = bh + (size_t)c->nR * kp;
  const bool same = A == B && a_r == b_r && a_c == b_c && M == N;
  split_tf32(A, a_r, a_c, M, K, ah, al, kp, nullptr, 0, c->stream);
  if (!same) split_tf32(B, b_r, b_c, N, K, bh, bl, kp, nullptr, 0, c->stream);
  TcOperand oa, ob;
  oa.x = oa.y = ob.x = ob.y = 0;
  const bool ok = make_tmap_kmajor(&oa.hi, ah, kp, K, M) && make_tmap_kmajor(&oa.lo, al, kp, K, M) &&
                  make_tmap_kmajor(&ob.hi, same ? ah : bh, kp, K, N) &&
                  make_tmap_kmajor(&ob.lo, same ? al : bl, kp, K, N);
  if (!ok) {
    cudaMemsetAsync(c->status + 7, 0xff, sizeof(int), c->stream);  // reported by the caller
    return;
  }
  gemm_3xtf32(oa, ob, M, N, K, C, cs_i, cs_j, alpha, beta, lower, mirror, c->status + 7, c->stream);
}

// K3 with a dense root: X̂ and Y^{-1} formed whole in W1 and W2 (n x ldw, the column of vertex k
// at colw[k]).  Their root blocks first: X̂_RR = X̄_RR (a clique block of E, so the completion
// keeps it) and Y^{-1}_RR = (N_RR N_RR^T)^{-1} = X^T X with X = N_RR^{-1} (the trailing block of
// the inverse of Y = N N^T).  The root's columns of the forest's rows then follow from one
// backward level-scheduled solve each (Y^{-1}[:, R] = N^{-T} N^{-1} [:, R] has no forest part
// before the backward step: N^{-1} maps R's unit vectors into R's rows); the forest's columns
// from a forward solve over the forest, the root rows taken from the root columns already formed
// (symmetry), and a backward solve.  No solve passes through the dense root.  Then the SCM tiles
// (eq. newSCM2) read both matrices through the column map.
template <class T>
mcsdp_status phase_scm_dense(mcsdp_ctx *c) {
  const int n = c->S.n, nR = c->nR, nF = c->nF;
  const int64_t ldw = c->ldw;
  const int64_t rv = c->D.root_valp;
  const SolveFactors<T> f = factors_of(c, T());
  T *W1 = reinterpret_cast<T *>(c->W1), *W2 = reinterpret_cast<T *>(c->W2);
  const LsSkip none{nullptr, nullptr, 0};
  const SkipHost hnone{nullptr, nullptr};
  KScope k1(c, KC_PANEL);
  int nl = 0;
  CUDA_TRY(c, cudaMemsetAsync(W1, 0, (size_t)n * ldw * sizeof(T), c->stream));
  CUDA_TRY(c, cudaMemsetAsync(W2, 0, (size_t)n * ldw * sizeof(T), c->stream));
  symmetrize<double, T>(c->Xbar_cur + rv, nR, W1 + (size_t)nF * ldw, ldw, nR, c->stream);
  ++nl;
  if constexpr (std::is_same<T, double>::value) {
    nl += dense_trtri<double>(c->N + rv, nR, c->rLinvN, c->RS_T, nR, nR, c->RS_M, c->stream);
    nl += dense_lauum<double>(c->RS_T, nR, nR, W2 + (size_t)nF * ldw, ldw, 1, true, c->stream);
  } else {
    float *L32 = reinterpret_cast<float *>(c->RS_T), *X32 = L32 + (size_t)nR * nR;
    copy_square<double, float>(c->N + rv, nR, L32, nR, nR, c->stream);
    launch_cast_f32(c->rLinvN, c->rLinv32, (int64_t)((nR + 31) / 32) * 1024, c->stream);
    nl += 2 + dense_trtri<float>(L32, nR, c->rLinv32, X32, nR, nR,
                                 reinterpret_cast<float *>(c->RS_M), c->stream);
    if (c->tcr) {  // X^T X on the tensor cores (the full square: K = nR for every tile)
      root_tc_gemm(c, X32, nR, 1, nR, X32, nR, 1, nR, nR, reinterpret_cast<float *>(W2) + (size_t)nF * ldw,
                   ldw, 1, 1.f, 0.f, true, true);
      nl += 2;
    } else {
      nl += dense_lauum<float>(X32, nR, nR, W2 + (size_t)nF * ldw, ldw, 1, true, c->stream);
    }
  }
  int r[6] = {0, 0, 0, 0, 0, 0};
  if (nF > 0) {
    LsSkip fw{c->pm_bits_dev, c->pm_tkey_dev, c->bit_words};
    const SkipHost hfw{c->pm_bits.data(), c->pm_tkey.data()};
    T *W1F = W1 + c->colF0, *W2F = W2 + c->colF0;
    launch_unit_cols<T>(W1, ldw, c->colw_dev, 0, nF, c->stream);
    launch_unit_cols<T>(W2, ldw, c->colw_dev, 0, nF, c->stream);
    nl += 2;
    // Y^{-1} on the side stream st4 (own partial slots and marks), X̂ here
    CUDA_TRY(c, cudaEventRecord(c->ev_n0, c->stream));
    CUDA_TRY(c, cudaStreamWaitEvent(c->st4, c->ev_n0, 0));
    {
      cudaStream_t main_st = c->stream;
      double *pw = c->Pw;
      unsigned char *xv = c->D.xvalid;
      c->stream = c->st4;
      c->Pw = c->Pw3;
      c->D.xvalid = c->xvalid3;
      KScope kn(c, KC_PANEL_SIDE, c->st4);
      r[3] = lsolve_c<T>(c, false, f.N, f.dinvN, W2, nR, none, hnone);
      r[4] = lsolve_c<T>(c, true, f.N, f.dinvN, W2F, nF, fw, hfw);
      launch_root_rows_from_cols<T>(W2, ldw, c->colw_dev, nR, nF, c->st4);
      r[5] = lsolve_c<T>(c, false, f.N, f.dinvN, W2F, nF, none, hnone);
      kn.done(1 + std::max(0, r[3]) + std::max(0, r[4]) + std::max(0, r[5]));
      c->stream = main_st;
      c->Pw = pw;
      c->D.xvalid = xv;
      CUDA_TRY(c, cudaEventRecord(c->ev_n1, c->st4));
    }
    r[0] = lsolve_c<T>(c, false, f.Lh, f.dinvL, W1, nR, none, hnone);
    r[1] = lsolve_c<T>(c, true, f.Lh, f.dinvL, W1F, nF, fw, hfw);
    launch_root_rows_from_cols<T>(W1, ldw, c->colw_dev, nR, nF, c->stream);
    r[2] = lsolve_c<T>(c, false, f.Lh, f.dinvL, W1F, nF, none, hnone);
    nl += 1 + std::max(0, r[0]) + std::max(0, r[1]) + std::max(0, r[2]);
    CUDA_TRY(c, cudaStreamWaitEvent(c->stream, c->ev_n1, 0));
  }
  k1.done(nl);
  for (int q = 0; q < 6; ++q)
    if (r[q] < 0) return fail(c, MCSDP_ERR_ARG, "solve shape not supported in this precision");
  KCHECK(c);
  KScope k2(c, KC_TILE);
  if (c->scm_vtx_dev) {
    launch_scm_hadamard<T>(c->D, W1, W2, ldw, c->colw_dev, c->scm_vtx_dev, c->B, c->ldb, c->hvec,
                           c->stream);
  } else {
    const Chunk &ch = c->chunks[0];
    launch_scm_tiles(c->D, c->tiles_dev + ch.tile_begin, ch.ntiles, (const T *)W1, (const T *)W2,
                     ldw, c->goff_dev, c->B, c->ldb, c->hvec, c->pmax, c->stream, c->colw_dev);
  }
  k2.done(1);
  KCHECK(c);
  return MCSDP_OK;
}

// K3 with solves in T (the W buffers and partial slots hold T; as FP32 they use half their size)
template <class T>
mcsdp_status phase_scm(mcsdp_ctx *c) {
  if (c->dense) return phase_scm_dense<T>(c);
  const Symbolic &S = c->S;
  const int n = S.n;
  const SolveFactors<T> f = factors_of(c, T());
  T *W1 = reinterpret_cast<T *>(c->W1), *W2 = reinterpret_cast<T *>(c->W2);
  for (const Chunk &ch : c->chunks) {
    KScope k1(c, KC_PANEL);
    int nl = 0;
    CUDA_TRY(c, cudaMemsetAsync(W1, 0, (size_t)n * c->ldw * sizeof(T), c->stream));
    CUDA_TRY(c, cudaMemsetAsync(W2, 0, (size_t)n * c->ldw * sizeof(T), c->stream));
    launch_rhs_unit(W1, c->ldw, c->rowof_dev + ch.rhs_begin, ch.nrhs, c->stream);
    launch_rhs_unit(W2, c->ldw, c->rowof_dev + ch.rhs_begin, ch.nrhs, c->stream);
    nl += 2;
    LsSkip fw{c->reach_bits_dev, c->tkey_dev + ch.tkey_begin, c->bit_words};
    LsSkip bw{c->need_bits_dev, c->tkey_dev + ch.tkey_begin, c->bit_words};
    const SkipHost hfw{c->reach_bits.data(), c->tkey_all.data() + ch.tkey_begin};
    const SkipHost hbw{c->need_bits.data(), c->tkey_all.data() + ch.tkey_begin};
    // X̂[:, P_g] = L̂^{-T} L̂^{-1} E (here) and Y^{-1}[:, P_g] = N^{-T} N^{-1} E (on the side
    // stream st4, with its own partial slots and marks: the two pairs of level-scheduled solves
    // are independent and latency-bound, so they share the SMs)
    CUDA_TRY(c, cudaEventRecord(c->ev_n0, c->stream));
    CUDA_TRY(c, cudaStreamWaitEvent(c->st4, c->ev_n0, 0));
    int r[4];
    {
      cudaStream_t main_st = c->stream;
      double *pw = c->Pw;
      unsigned char *xv = c->D.xvalid;
      c->stream = c->st4;
      c->Pw = c->Pw3;
      c->D.xvalid = c->xvalid3;
      KScope kn(c, KC_PANEL_SIDE, c->st4);
      r[2] = lsolve_c<T>(c, true, f.N, f.dinvN, W2, ch.nrhs, fw, hfw);
      r[3] = lsolve_c<T>(c, false, f.N, f.dinvN, W2, ch.nrhs, bw, hbw);
      kn.done(std::max(0, r[2]) + std::max(0, r[3]));
      c->stream = main_st;
      c->Pw = pw;
      c->D.xvalid = xv;
      CUDA_TRY(c, cudaEventRecord(c->ev_n1, c->st4));
    }
    r[0] = lsolve_c<T>(c, true, f.Lh, f.dinvL, W1, ch.nrhs, fw, hfw);
    r[1] = lsolve_c<T>(c, false, f.Lh, f.dinvL, W1, ch.nrhs, bw, hbw);
    for (int q = 0; q < 2; ++q) nl += std::max(0, r[q]);
    k1.done(nl);
    CUDA_TRY(c, cudaStreamWaitEvent(c->stream, c->ev_n1, 0));
    for (int q = 0; q < 4; ++q)
      if (r[q] < 0) return fail(c, MCSDP_ERR_ARG, "solve shape not supported in this precision");
    KCHECK(c);
    KScope k2(c, KC_TILE);
    launch_scm_tiles(c->D, c->tiles_dev + ch.tile_begin, ch.ntiles, (const T *)W1, (const T *)W2,
                     c->ldw, c->goff_dev, c->B, c->ldb, c->hvec, c->pmax, c->stream);
    k2.done(1);
    KCHECK(c);
  }
  return MCSDP_OK;
}

// P-MATRIX (eq. newdX2) with a dense root, from the dense X̂ (W1) and Y^{-1} (W2) of the SCM
// phase.  Forest entries of E: V = X̂ dY (W3, rows of X̂ times the aggregate-pattern dY), and
// M = X̂ dY Y^{-1} at (r, k) is the dot product of row r of V with row k of Y^{-1} (Mlow at (r, k)
// and, transposed, Mup); Y^{-1} on E read from W2.  Root block: with U = dY Y^{-1}[:, R] (W3 again)
// and the completion's X̂_FR = -L_FF^{-T} L_RF^T X̂_RR, M_RR = X̂_RR (U_RR - L_RF L_FF^{-1} U_F):
// a forward solve over the forest (n_R right-hand sides), the sparse L_RF product, and one
// n_R x n_R x n_R GEMM, where the product over all n columns, X̂_R dY Y^{-1}_{:R}, would take
// n / n_R times the flops.  Then dX on E.
template <class T>
mcsdp_status phase_pmatrix_dense(mcsdp_ctx *c, double betamu, const double *Xbar) {
  const int n = c->S.n, nR = c->nR, nF = c->nF;
  const int64_t ldw = c->ldw, rv = c->D.root_valp;
  const T *W1 = reinterpret_cast<const T *>(c->W1), *W2 = reinterpret_cast<const T *>(c->W2);
  T *V = reinterpret_cast<T *>(c->W3);
  T *M = reinterpret_cast<T *>(c->RS_M);
  T *Tt = reinterpret_cast<T *>(c->RS_T);
  const SolveFactors<T> f = factors_of(c, T());
  KScope k1(c, KC_PMAT);
  int nl = 0;
  if (nF > 0) {
    CUDA_TRY(c, cudaMemsetAsync(V, 0, (size_t)n * ldw * sizeof(T), c->stream));
    if (c->S.diag_constraints)  // dY = -sum dz_k A_k is diagonal: V = X̂ dY scales columns
      launch_times_diag<T>(c->D, c->dY, W1, V, ldw, c->colw_dev, reinterpret_cast<T *>(c->lzU),
                           c->stream);
    else
      launch_times_pattern<T>(c->D, c->dY, W1, V, ldw, c->colw_dev, c->stream);
    launch_forest_M<T>(c->D, V, W2, ldw, (int)ldw, c->Mlow, c->Mup, c->stream);
    nl += 4;
  }
  launch_extract_dense<T>(c->D, W2, ldw, c->colw_dev, c->YinvE, c->stream);
  // U = dY Y^{-1}[:, R] over the root's columns (the forest's use of W3 above is complete)
  T *U = V;
  launch_dY_times<T>(c->D, c->dY, W2, U, ldw, nR, c->stream);
  nl += 2;
  if (nF > 0) {
    const LsSkip none{nullptr, nullptr, 0};
    const SkipHost hnone{nullptr, nullptr};
    const int r = lsolve_c<T>(c, true, f.Lh, f.dinvL, U, nR, none, hnone);
    if (r < 0) return fail(c, MCSDP_ERR_ARG, "solve shape not supported in this precision");
    nl += r;
  }
  launch_root_pull<T>(c->lrf_ptr_dev, c->lrf_off_dev, c->lrf_row_dev, f.Lh, U, ldw, nF, nR, Tt,
                      c->stream);
  ++nl;
  if constexpr (std::is_same<T, float>::value) {
    if (c->tcr) {
      root_tc_gemm(c, W1 + (size_t)nF * ldw, ldw, 1, nR, Tt, nR, 1, nR, nR, M, 1, nR, 1.f, 0.f,
                   false, false);
      nl += 3;
    }
  }
  k1.done(nl);
  nl = 0;
  if (!(std::is_same<T, float>::value && c->tcr)) {
    // the root block's GEMM on its own class (the FP64 form's largest product)
    KScope kg(c, std::is_same<T, double>::value ? KC_RGEMM : KC_PMAT);
    GemmArgs<T> g{};
    g.M = g.N = g.K = nR;
    g.A = W1 + (size_t)nF * ldw;
    g.lda = ldw;
    g.B = Tt;
    g.ldb = nR;
    g.C = M;
    g.cs_i = 1;
    g.cs_j = nR;
    g.alpha = T(1);
    g.beta = T(0);
    gemm_tn<T>(g, c->stream, true);
    kg.done(1);
  }
  KScope k3(c, KC_PMAT);
  launch_root_M<T>(M, nR, c->Mlow + rv, c->Mup + rv, c->stream);
  k3.done(1);
  KScope k2(c, KC_MISC);
  launch_dx_combine(c->D, betamu, Xbar, c->YinvE, c->Mlow, c->Mup, c->dX, c->stream);
  launch_root_dx(nR, betamu, Xbar + rv, c->YinvE + rv, c->Mlow + rv, c->Mup + rv, c->dX + rv,
                 c->stream);
  k2.done(2);
  KCHECK(c);
  return MCSDP_OK;
}

// P-MATRIX (eq. newdX2): for column blocks of the identity, Y^{-1} E (N solves), dY Y^{-1} E,
// X̂ dY Y^{-1} E (L̂ solves), keeping the entries on E.
// Dlay == nullptr: dY (on the aggregate pattern); else a symmetric D on lower(E).  yinv_only:
// only Y^{-1} on E (into YinvE).
template <class T>
// Wy (single block only): the block's Y^{-1} columns and Y^{-1} on E were already formed by
// phase_pmatrix_yinv into Wy; only the dY product and the L̂ solves remain.
mcsdp_status phase_pmatrix(mcsdp_ctx *c, int *nlaunch, const double *Dlay = nullptr,
                           bool yinv_only = false, const T *Wy = nullptr) {
  const Symbolic &S = c->S;
  const int n = S.n;
  int nl = 0;
  const LsSkip none{nullptr, nullptr, 0};
  const SolveFactors<T> f = factors_of(c, T());
  T *W1 = reinterpret_cast<T *>(c->W1), *W2 = reinterpret_cast<T *>(c->W2);
  for (int k0 = 0; k0 < n; k0 += c->pm_cols) {
    const int nc = std::min(c->pm_cols, n - k0);
    LsSkip fw{c->pm_bits_dev, c->pm_tkey_dev + k0 / 32, c->bit_words};
    LsSkip bwL{c->pm_need_dev, c->pm_tkey_dev + k0 / 32, c->bit_words};
    const SkipHost hfw{c->pm_bits.data(), c->pm_tkey.data() + k0 / 32};
    const SkipHost hbwL{c->pm_need.data(), c->pm_tkey.data() + k0 / 32};
    const SkipHost hnone{nullptr, nullptr};
    int r[4] = {0, 0, 0, 0};
    if (Wy) {
      W1 = const_cast<T *>(Wy);
    } else {
      CUDA_TRY(c, cudaMemsetAsync(W1, 0, (size_t)n * c->ldw * sizeof(T), c->stream));
      launch_rhs_unit(W1, c->ldw, c->pm_rowof_dev + k0, nc, c->stream);
      nl += 1;
      r[0] = lsolve_c<T>(c, true, f.N, f.dinvN, W1, nc, fw, hfw);
      r[1] = lsolve_c<T>(c, false, f.N, f.dinvN, W1, nc, none, hnone);
      launch_extract_lowerE(c->D, (const T *)W1, c->ldw, k0, nc, c->YinvE, c->stream);
      nl += 1;
    }
    if (yinv_only) {
      for (int q = 0; q < 2; ++q) {
        if (r[q] < 0) return fail(c, MCSDP_ERR_ARG, "solve shape not supported in this precision");
        nl += r[q];
      }
      continue;
    }
    if constexpr (std::is_same<T, double>::value) {
      if (Dlay) launch_E_times(c->D, Dlay, (const double *)W1, (double *)W2, c->ldw, nc, c->stream);
      else launch_dY_times(c->D, c->dY, (const T *)W1, W2, c->ldw, nc, c->stream);
    } else {
      launch_dY_times(c->D, c->dY, (const T *)W1, W2, c->ldw, nc, c->stream);
    }
    nl += 1;
    r[2] = lsolve_c<T>(c, true, f.Lh, f.dinvL, W2, nc, none, hnone);
    r[3] = lsolve_c<T>(c, false, f.Lh, f.dinvL, W2, nc, bwL, hbwL);
    launch_extract_lowerE(c->D, (const T *)W2, c->ldw, k0, nc, c->Mlow, c->stream);
    launch_extract_upperE(c->D, (const T *)W2, c->ldw, k0, nc, c->Mup, c->stream);
    nl += 2;
    for (int q = 0; q < 4; ++q) {
      if (r[q] < 0) return fail(c, MCSDP_ERR_ARG, "solve shape not supported in this precision");
      nl += r[q];
    }
  }
  KCHECK(c);
  *nlaunch = nl;
  return MCSDP_OK;
}

// The first half of the single P-MATRIX block, Y^{-1} E and Y^{-1} on E, into W3 (needs only
// N, so it can run beside the SCE solve; it uses the solves' partial slots, so not beside the
// SCM solves).  All on c->stream, which the caller points at the side stream.
template <class T>
mcsdp_status phase_pmatrix_yinv(mcsdp_ctx *c, int *nlaunch) {
  const Symbolic &S = c->S;
  const int n = S.n;
  const LsSkip none{nullptr, nullptr, 0};
  const SolveFactors<T> f = factors_of(c, T());
  T *W = reinterpret_cast<T *>(c->W3);
  LsSkip fw{c->pm_bits_dev, c->pm_tkey_dev, c->bit_words};
  const SkipHost hfw{c->pm_bits.data(), c->pm_tkey.data()};
  const SkipHost hnone{nullptr, nullptr};
  CUDA_TRY(c, cudaMemsetAsync(W, 0, (size_t)n * c->ldw * sizeof(T), c->stream));
  launch_rhs_unit(W, c->ldw, c->pm_rowof_dev, n, c->stream);
  const int r0 = lsolve_c<T>(c, true, f.N, f.dinvN, W, n, fw, hfw);
  const int r1 = lsolve_c<T>(c, false, f.N, f.dinvN, W, n, none, hnone);
  if (r0 < 0 || r1 < 0) return fail(c, MCSDP_ERR_ARG, "solve shape not supported in this precision");
  launch_extract_lowerE(c->D, (const T *)W, c->ldw, 0, n, c->YinvE, c->stream);
  *nlaunch = 2 + r0 + r1;
  return MCSDP_OK;
}

// Smallest eigenvalue of the symmetric tridiagonal matrix with diagonal a[0..k) and off-diagonal
// b[0..k-1), and the last component of its unit eigenvector, by cyclic Jacobi rotations on the
// dense k x k matrix (k <= LZ_MAX: host work of microseconds)
void tridiag_min(int k, const double *a, const double *b, double *lam, double *last) {
  std::vector<double> A((size_t)k * k, 0.0), V((size_t)k * k, 0.0);
  for (int i = 0; i < k; ++i) {
    A[(size_t)i * k + i] = a[i];
    if (i + 1 < k) A[(size_t)i * k + i + 1] = A[(size_t)(i + 1) * k + i] = b[i];
    V[(size_t)i * k + i] = 1.0;
  }
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int p = 0; p < k; ++p)
      for (int q = 0; q < k; ++q) {
        const double v = A[(size_t)p * k + q] * A[(size_t)p * k + q];
        tot += v;
        if (p != q) off += v;
      }
    if (off <= 1e-32 * tot) break;
    for (int p = 0; p < k; ++p)
      for (int q = p + 1; q < k; ++q) {
        const double apq = A[(size_t)p * k + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double th = (A[(size_t)q * k + q] - A[(size_t)p * k + p]) / (2.0 * apq);
        const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
        const double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
        for (int r = 0; r < k; ++r) {  // columns p, q
          const double x = A[(size_t)r * k + p], y = A[(size_t)r * k + q];
          A[(size_t)r * k + p] = cs * x - sn * y;
          A[(size_t)r * k + q] = sn * x + cs * y;
        }
        for (int r = 0; r < k; ++r) {  // rows p, q
          const double x = A[(size_t)p * k + r], y = A[(size_t)q * k + r];
          A[(size_t)p * k + r] = cs * x - sn * y;
          A[(size_t)q * k + r] = sn * x + cs * y;
        }
        for (int r = 0; r < k; ++r) {
          const double x = V[(size_t)r * k + p], y = V[(size_t)r * k + q];
          V[(size_t)r * k + p] = cs * x - sn * y;
          V[(size_t)r * k + q] = sn * x + cs * y;
        }
      }
  }
  int im = 0;
  for (int i = 1; i < k; ++i)
    if (A[(size_t)i * k + i] < A[(size_t)im * k + im]) im = i;
  *lam = A[(size_t)im * k + im];
  *last = V[(size_t)(k - 1) * k + im];
}

// Smallest eigenvalue of an operator self-adjoint in the inner product <u, v>_G = u^T G v, by
// Lanczos with full reorthogonalisation from a fixed pseudo-random start: op(v, w) forms w = op v,
// gmul(v, gv) forms gv = G v (has_g false: G = I), both on c->stream, vectors of length dim.
// Stops at LZ_MAX steps, at an invariant subspace, or once the Ritz value's residual bound is
// below tol max(1, |theta|) (tested every 8 steps).  *theta = smallest Ritz value, *bound = its
// residual bound (an eigenvalue lies within bound of theta).
template <class Op, class Gm>
mcsdp_status lanczos_min(mcsdp_ctx *c, int dim, Op op, Gm gmul, bool has_g, double tol,
                         unsigned seed, double *theta, double *bound, int *steps) {
  double *Q = c->lzQ, *GQ = has_g ? c->lzQ + (size_t)dim * (LZ_MAX + 1) : c->lzQ;
  double *w = c->lzW, *gw = has_g ? c->lzG : c->lzW;
  const cudaStream_t st = c->stream;
  fill_hash(Q, dim, seed, st);
  if (has_g) gmul(Q, GQ);
  lz_normalise(dim, Q, GQ, st);
  double hs[2 * LZ_MAX + 2];
  int k = 0;
  *theta = 0.0;
  *bound = 0.0;
  for (int j = 0; j < LZ_MAX; ++j) {
    double *vj = Q + (size_t)j * dim, *gvj = GQ + (size_t)j * dim;
    op(vj, w);
    lz_alpha(dim, w, gvj, vj, j > 0 ? vj - dim : nullptr, c->lzS, j, st);
    lz_reorth(dim, j + 1, w, GQ, Q, c->lzS + 2 * LZ_MAX + 2, st);
    if (has_g) gmul(w, gw);
    lz_beta(dim, w, gw, vj + dim, has_g ? gvj + dim : nullptr, c->lzS, j, st);
    k = j + 1;
    if (k % 8 == 0 || k == LZ_MAX || k == dim) {
      CUDA_TRY(c, cudaMemcpyAsync(hs, c->lzS, 2 * k * 8, cudaMemcpyDeviceToHost, st));
      CUDA_TRY(c, cudaStreamSynchronize(st));
      prof_flush(c);
      double a[LZ_MAX], b[LZ_MAX];
      for (int i = 0; i < k; ++i) {
        a[i] = hs[2 * i];
        b[i] = hs[2 * i + 1];
      }
      double lam, last;
      tridiag_min(k, a, b, &lam, &last);
      *theta = lam;
      *bound = std::fabs(b[k - 1] * last);
      if (!std::isfinite(lam)) return fail(c, MCSDP_ERR_NUMERIC, "NaN in a Lanczos step-length bound");
      if (b[k - 1] <= 1e-14 * std::max(1.0, std::fabs(lam)) || k == dim) break;
      if (*bound <= tol * std::max(1.0, std::fabs(lam))) break;
    }
  }
  *steps = k;
  return MCSDP_OK;
}

// max alpha in (0, 1] with I + alpha T psd for lambda_min(T) >= theta - bound
double step_from_bound(double theta, double bound) {
  const double lam = theta - bound;
  return lam < -1.0 ? -1.0 / lam : 1.0;
}

// Step lengths with a dense root (Lanczos bounds of eq. primal_length2).  Primal, root clique:
// lambda_min(L^{-1} dX_RR L^{-T}) with X̄_RR = L L^T (RS_P holds L^{-1} and its rows mirrored),
// dX_RR made full in RS_M.  Dual: lambda_min(Y^{-1} dY), self-adjoint in the Y-inner product, with
// the dense Y^{-1} of the SCM phase (W2) and Y on the aggregate pattern.  Both are confirmed by
// the next iteration's factorisations (a failure backtracks the step).
template <class T>
mcsdp_status dense_steps(mcsdp_ctx *c, double *alpha_root, double *alpha_dual) {
  const int n = c->S.n, nR = c->nR;
  const int64_t rv = c->D.root_valp;
  double th, bd;
  int steps = 0;
  mcsdp_status s;
  {
    KScope ks(c, KC_PSTEP);
    symmetrize<double, double>(c->dX + rv, nR, c->RS_M, nR, nR, c->stream);
    double *u1 = c->lzU, *u2 = c->lzU + nR;
    auto op = [&](const double *v, double *w) {
      dotcols<double>(c->RS_P, nR, nR, nR, 1, v, u1, 1.0, 0.0, c->stream);
      dotcols<double>(c->RS_M, nR, nR, nR, 0, u1, u2, 1.0, 0.0, c->stream);
      dotcols<double>(c->RS_P, nR, nR, nR, 2, u2, w, 1.0, 0.0, c->stream);
    };
    auto gnone = [&](const double *, double *) {};
    s = lanczos_min(c, nR, op, gnone, false, 1e-3, 7u, &th, &bd, &steps);
    ks.done(1 + 8 * steps);
    if (s) return s;
    *alpha_root = step_from_bound(th, bd);
    c->lz_steps[0] = steps;
    c->lz_last[0] = th;
    c->lz_last[1] = bd;
  }
  {
    KScope ks(c, KC_DSTEP);
    const T *W2 = reinterpret_cast<const T *>(c->W2);
    const int64_t ldw = c->ldw;
    double *u = c->lzU, *ut = c->lzU + std::max<int64_t>(n, ldw);
    CUDA_TRY(c, cudaMemsetAsync(ut, 0, ldw * 8, c->stream));
    auto op = [&](const double *v, double *w) {
      launch_dY_times<double>(c->D, c->dY, v, u, 1, 1, c->stream);
      permute_to_cols(u, c->colw_dev, ut, n, c->stream);
      dotcols<T>(W2, ldw, n, (int)ldw, 0, ut, w, 1.0, 0.0, c->stream);
    };
    auto gmul = [&](const double *v, double *gv) {
      launch_dY_times<double>(c->D, c->Ylay, v, gv, 1, 1, c->stream);
    };
    s = lanczos_min(c, n, op, gmul, true, 1e-3, 11u, &th, &bd, &steps);
    ks.done(1 + 9 * steps);
    if (s) return s;
    *alpha_dual = step_from_bound(th, bd);
    c->lz_steps[1] = steps;
    c->lz_last[2] = th;
    c->lz_last[3] = bd;
  }
  return MCSDP_OK;
}

struct IterOut {
  double mu, pobj, dobj, gap, pinf, ap, ad;
};

// Mixed form of the SCE solve B dz = g (eq. SCE): Cholesky factor of B rounded to FP32 (for
// m >= MIXED_LONG_M of the equilibrated S B S, S = diag(B_ii^{-1/2}), on the tensor cores), then an
// FP64 correction against the stored B.  Measure of convergence: omega = max|r| / max(|B||x| + |g|)
// with r = g - B x formed in FP64.  Success when omega <= sqrt(m) eps64 (FP64-assembled B) or
// 1e-10 (b32: B was assembled in FP32, entries accurate to about 1e-6 relative, so the solve
// error is then far below the assembly error); otherwise (*solved = false, B untouched) the
// caller promotes to the FP64 factorisation, as it does when the FP32 factorisation breaks down.
//   small m: iterative refinement (the scheme of LAPACK's dsposv), abandoned when omega fails to
//   halve in two consecutive steps while above m eps64 (the worst-case backward error of the FP64
//   factorisation itself), or after MIXED_MAX_STEPS steps;
//   large m: refinement contracts by about cond(B) eps32 per step, slowly near the optimum, so the
//   correction is restarted GMRES(GM_K) on B x = g left-preconditioned by the FP32 factor (the
//   GMRES-based refinement of Carson and Higham), Arnoldi in FP64 with classical Gram-Schmidt
//   applied twice, the small least-squares problem by Givens rotations on the host, omega from
//   the true residual after each cycle (a cycle stops once the preconditioned residual has
//   fallen by 1e-7: the FP32 preconditioner bounds what one cycle gains); abandoned when a cycle
//   fails to halve omega above m eps64 or after GM_CYCLES cycles.  When the FP32 factor of S B S
//   breaks down near the optimum, the factor of S B S + sigma I (sigma = 1e-5, 1e-4, then 1e-3)
//   preconditions the same GMRES on B (such a preconditioner leaves the eigenvalues of S B S below
//   sigma to the Krylov space: a longer restart, 100, was measured no better on config 3).  An Arnoldi step (the substitutions over all SMs and one
//   FP64 product with B, O(m^2)) costs about a thousandth of the FP64 factorisation (O(m^3)).
// Leaves x in c->xs (internal order).
constexpr int MIXED_MAX_STEPS = 10;
// default relative gap for the mixed form's switch to FP64 assembly with a dense root
constexpr double MIXED_ASM_GAP_ROOT = 1e-2;

mcsdp_status mixed_gmres(mcsdp_ctx *c, double tol_ok, double tol_stall, bool *solved);

// K4 and K5 in FP64: the bordered Cholesky factorisation of B (the right-hand side in its border
// row) and the backward substitution; x in c->xs (internal order).  A block-diagonal B
// (c->blocks): one of each per component q, on the diagonal block at (o, o), o = comp_cptr[q],
// whose right-hand side k_rhs_border put in row comp_cptr[q + 1] of the block's columns (the row
// after the block, outside every diagonal block), so that the block is itself a bordered matrix of
// leading dimension ldb.  The blocks are independent: all their factorisations share one
// task-queue launch (their tickets concatenated), all their substitutions one launch of a
// cluster per block.
void scm_chol_solve(mcsdp_ctx *c) {
  const Symbolic &S = c->S;
  const int nblk = c->blocks ? S.ncomp : 1;
  auto range = [&](int q, int *o, int *mc) {
    *o = c->blocks ? S.comp_cptr[q] : 0;
    *mc = (c->blocks ? S.comp_cptr[q + 1] : S.m) - *o;
  };
  int o, mc, nl = 0;
  {
    KScope k1(c, KC_CHOL);
    if (c->blocks && c->cs.dag_sync) {
      // every block in one task-queue launch: the blocks' chains overlap instead of running one
      // after another
      nl = dense_chol_dag_blocks(c->B, c->ldb, c->bt, c->status + 2, c->Binv, c->stream,
                                 c->cs.dag_sync, c->cs.dag_budget);
    } else {
      for (int q = 0; q < nblk; ++q) {
        range(q, &o, &mc);
        nl += dense_chol_bordered(c->B + o + (int64_t)o * c->ldb, c->ldb, mc, c->status + 2,
                                  c->Binv + c->binv_off[q], c->stream, &c->cs);
      }
    }
    k1.done(nl);
  }
  KScope k2(c, KC_BSOLVE);
  // one cluster per block in one launch, unless a block exceeds the cluster kernel's vector
  nl = c->blocks ? dense_backsolve_blocks(c->B, c->ldb, c->bt, c->Binv, c->xs, c->stream) : -1;
  if (nl < 0) {
    nl = 0;
    for (int q = 0; q < nblk; ++q) {
      range(q, &o, &mc);
      nl += dense_backsolve(c->B + o + (int64_t)o * c->ldb, c->ldb, mc, c->Binv + c->binv_off[q],
                            c->xs + o, c->stream);
    }
  }
  k2.done(nl);
}

mcsdp_status mixed_sce(mcsdp_ctx *c, bool b32, bool *solved) {
  const int m = c->S.m;
  *solved = false;
  const double eps = std::ldexp(1.0, -53);
  const double tol_ok = b32 ? 1e-10 : std::sqrt((double)m) * eps;
  const double tol_stall = b32 ? 1e-10 : (double)m * eps;
  if (m >= MIXED_LONG_M && c->gmV) {
    // GMRES form: when the FP32 factor of S B S breaks down, that of S B S + sigma I (unit
    // diagonal, sigma = 1e-5, 1e-4, then 1e-3) still preconditions GMRES on B itself
    const double shifts[4] = {0.0, 1e-5, 1e-4, 1e-3};
    for (double sigma : shifts) {
      CUDA_TRY(c, cudaMemsetAsync(c->status + 4, 0, sizeof(int), c->stream));
      {
        KScope k1(c, KC_CHOL32);
        k1.done(mixed_factor(c->B, c->ldb, m, c->B32, c->Linv32, c->status + 4, c->gref, c->rref,
                             c->xs, c->dscl, sigma, c->tinv, c->stream, &c->cs));
      }
      KCHECK(c);
      int fst = 0;
      CUDA_TRY(c, cudaMemcpyAsync(&fst, c->status + 4, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
      CUDA_TRY(c, cudaStreamSynchronize(c->stream));
      prof_flush(c);
      if (fst & ST_TIMEOUT) return fail(c, MCSDP_ERR_TIMEOUT, "FP32 factorisation: a bounded wait gave up");
      if (fst & ST_NUMERIC) return fail(c, MCSDP_ERR_CUDA, "FP32 factorisation: a tensor map could not be made");
      if (fst & ST_NOT_PD) {
        if (c->opt.verbose > 1) std::fprintf(stderr, "  FP32 factor (shift %.0e) broke down\n", sigma);
        continue;
      }
      return mixed_gmres(c, tol_ok, tol_stall, solved);
    }
    return MCSDP_OK;  // every FP32 factor broke down: promote
  }
  CUDA_TRY(c, cudaMemsetAsync(c->status + 4, 0, sizeof(int), c->stream));
  {
    KScope k1(c, KC_CHOL32);
    k1.done(mixed_factor(c->B, c->ldb, m, c->B32, c->Linv32, c->status + 4, c->gref, c->rref,
                         c->xs, c->dscl, 0.0, c->tinv, c->stream, &c->cs));
  }
  KCHECK(c);
  double prev = 1.0;
  int slow = 0;
  for (int k = 0; k < MIXED_MAX_STEPS; ++k) {
    {
      KScope k2(c, KC_BSOLVE);
      k2.done(mixed_refine_step(c->B, c->ldb, m, c->B32, c->Linv32, c->gref, c->xs, c->rref,
                                c->yref, c->ayref, c->nref, c->dscl, c->tinv, c->stream));
    }
    KCHECK(c);
    double nr[2];
    int fst = 0;
    CUDA_TRY(c, cudaMemcpyAsync(nr, c->nref, 2 * 8, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(&fst, c->status + 4, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    prof_flush(c);
    ++c->refine_steps;
    if (fst & ST_TIMEOUT) return fail(c, MCSDP_ERR_TIMEOUT, "FP32 factorisation: a bounded wait gave up");
    if (fst & ST_NUMERIC) return fail(c, MCSDP_ERR_CUDA, "FP32 factorisation: a tensor map could not be made");
    if (fst & ST_NOT_PD) return MCSDP_OK;  // FP32 factor broke down: promote
    const double omega = nr[0] / std::max(nr[1], std::numeric_limits<double>::min());
    if (!std::isfinite(omega)) return MCSDP_OK;
    if (c->opt.verbose > 1) std::fprintf(stderr, "  refine %d omega %.3e\n", k, omega);
    if (omega <= tol_ok) {
      *solved = true;
      return MCSDP_OK;
    }
    slow = (omega > 0.5 * prev) ? slow + 1 : 0;
    if (slow >= 2) {
      *solved = omega <= tol_stall;
      return MCSDP_OK;
    }
    prev = omega;
  }
  return MCSDP_OK;
}

// the GMRES form (see mixed_sce).  On entry x = 0, r = g.  Device vectors: V holds the basis
// (GM_K + 1 vectors of m) and a work vector; H the two Gram-Schmidt passes' coefficients, the
// norms and the update's coefficients.
mcsdp_status mixed_gmres(mcsdp_ctx *c, double tol_ok, double tol_stall, bool *solved) {
  const int m = c->S.m;
  const cudaStream_t st = c->stream;
  double *V = c->gmV, *tv = c->gmV + (size_t)(GM_K + 1) * m;
  double *h1 = c->gmH, *h2 = h1 + (GM_K + 2), *sn = h2 + (GM_K + 2), *yd = sn + 2 * (GM_K + 2);
  double prev = -1.0;
  for (int cyc = 0; cyc < GM_CYCLES; ++cyc) {
    // v_0 = M^{-1} r / beta_0
    double Hc[GM_K + 1][GM_K], gv[GM_K + 1], cs[GM_K], snr[GM_K];
    double beta0 = 0.0;
    int k = 0;
    {
      KScope kb(c, KC_BSOLVE);
      int nl = mixed_precond(c->B32, m, c->Linv32, c->rref, V, c->yref, c->dscl, c->tinv, st);
      lz_beta(m, V, V, V, nullptr, sn, GM_K, st);
      double b = 0.0;
      CUDA_TRY(c, cudaMemcpyAsync(&b, sn + 2 * GM_K + 1, 8, cudaMemcpyDeviceToHost, st));
      CUDA_TRY(c, cudaStreamSynchronize(st));
      beta0 = b;
      gv[0] = beta0;
      for (int j = 0; j < GM_K && beta0 > 0.0; ++j) {
        double *vj = V + (size_t)j * m, *w = V + (size_t)(j + 1) * m;
        nl += mixed_matvec(c->B, c->ldb, m, vj, tv, c->yref, c->ayref, st);
        nl += mixed_precond(c->B32, m, c->Linv32, tv, w, c->yref, c->dscl, c->tinv, st);
        lz_reorth(m, j + 1, w, V, V, h1, st);
        lz_reorth(m, j + 1, w, V, V, h2, st);
        lz_beta(m, w, w, w, nullptr, sn, j, st);
        nl += 5;
        double hh[3 * (GM_K + 2)];
        CUDA_TRY(c, cudaMemcpyAsync(hh, h1, 2 * (GM_K + 2) * 8, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(c, cudaMemcpyAsync(hh + 2 * (GM_K + 2), sn + 2 * j + 1, 8, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(c, cudaStreamSynchronize(st));
        ++c->refine_steps;
        double col[GM_K + 1];
        for (int i = 0; i <= j; ++i) col[i] = hh[i] + hh[(GM_K + 2) + i];
        col[j + 1] = hh[2 * (GM_K + 2)];
        // previous rotations, then the new one zeroing col[j + 1]
        for (int i = 0; i < j; ++i) {
          const double a = cs[i] * col[i] + snr[i] * col[i + 1];
          col[i + 1] = -snr[i] * col[i] + cs[i] * col[i + 1];
          col[i] = a;
        }
        const double rr = std::hypot(col[j], col[j + 1]);
        cs[j] = rr > 0.0 ? col[j] / rr : 1.0;
        snr[j] = rr > 0.0 ? col[j + 1] / rr : 0.0;
        col[j] = rr;
        gv[j + 1] = -snr[j] * gv[j];
        gv[j] = cs[j] * gv[j];
        for (int i = 0; i <= j; ++i) Hc[i][j] = col[i];
        k = j + 1;
        if (!std::isfinite(rr)) return MCSDP_OK;
        // the preconditioned residual: far enough below for this cycle, or a breakdown
        // (the preconditioner runs in FP32, so a cycle gains about that much on the true
        // residual; the restarts refine further)
        if (std::fabs(gv[j + 1]) <= 1e-7 * beta0 || hh[2 * (GM_K + 2)] <= 1e-14 * beta0) break;
      }
      // y = H^{-1} gv (upper triangular), x += V y
      double y[GM_K];
      for (int i = k - 1; i >= 0; --i) {
        double a = gv[i];
        for (int q = i + 1; q < k; ++q) a -= Hc[i][q] * y[q];
        y[i] = Hc[i][i] != 0.0 ? a / Hc[i][i] : 0.0;
      }
      double ny[GM_K];
      for (int i = 0; i < k; ++i) ny[i] = -y[i];
      if (k > 0) {
        CUDA_TRY(c, cudaMemcpyAsync(yd, ny, k * 8, cudaMemcpyHostToDevice, st));
        lz_sub(m, k, c->xs, V, yd, st);
      }
      nl += 1 + mixed_residual(c->B, c->ldb, m, c->gref, c->xs, c->rref, c->yref, c->ayref,
                               c->nref, st);
      kb.done(nl);
    }
    KCHECK(c);
    double nr[2];
    CUDA_TRY(c, cudaMemcpyAsync(nr, c->nref, 2 * 8, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(c, cudaStreamSynchronize(st));
    prof_flush(c);
    const double omega = nr[0] / std::max(nr[1], std::numeric_limits<double>::min());
    if (c->opt.verbose > 1)
      std::fprintf(stderr, "  gmres cycle %d: %d steps, omega %.3e\n", cyc, k, omega);
    if (!std::isfinite(omega)) return MCSDP_OK;
    if (omega <= tol_ok) {
      *solved = true;
      return MCSDP_OK;
    }
    if (prev >= 0.0 && omega > 0.5 * prev) {
      *solved = omega <= tol_stall;
      return MCSDP_OK;
    }
    prev = omega;
  }
  return MCSDP_OK;
}

// Computes the Newton direction at (Xbar, z) into c->dz, c->dY, c->dX and the step lengths.
// Requires Ylay/N/Lh already factored at the iterate.
mcsdp_status direction(mcsdp_ctx *c, const double *Xbar, double mu, IterOut &o, float *tms) {
  const double beta = c->opt.beta;
  const int m = c->S.m;
  cudaEventRecord(c->ev[0], c->stream);
  CUDA_TRY(c, cudaMemsetAsync(c->status + 7, 0, sizeof(int), c->stream));
  // mixed form before promotion: FP32 solves and contraction from FP32 copies of the factors
  bool f32 = c->opt.precision == 1 && !c->promoted && !c->fp64_asm && c->f32_solves;
  if (f32) cast_factors(c);
  // the P-MATRIX's Y^{-1} columns need only N: with a single block they are formed on the side
  // stream st3 (own solve buffer, partial slots and marks) beside the SCM solves, which are
  // latency-bound and leave most SMs idle
  const bool yinv_early = c->W3 != nullptr && !c->dense;
  const bool yinv_f32 = f32;
  mcsdp_status s = MCSDP_OK;
  if (yinv_early) {
    CUDA_TRY(c, cudaEventRecord(c->ev_yinv, c->stream));
    CUDA_TRY(c, cudaStreamWaitEvent(c->st3, c->ev_yinv, 0));
    cudaStream_t main_st = c->stream;
    double *pw = c->Pw;
    unsigned char *xv = c->D.xvalid;
    c->stream = c->st3;
    c->Pw = c->Pw2;
    c->D.xvalid = c->xvalid2;
    KScope ky(c, KC_PMAT_SIDE, c->st3);
    int nly = 0;
    s = f32 ? phase_pmatrix_yinv<float>(c, &nly) : phase_pmatrix_yinv<double>(c, &nly);
    ky.done(nly);
    c->stream = main_st;
    c->Pw = pw;
    c->D.xvalid = xv;
    if (s) return s;
    CUDA_TRY(c, cudaEventRecord(c->ev_yinv, c->st3));
  }
  s = f32 ? phase_scm<float>(c) : phase_scm<double>(c);
  if (s) return s;
  cudaEventRecord(c->ev[1], c->stream);
  {
    KScope k0(c, KC_MISC);
    launch_rhs_border(c->D, c->B, c->ldb, c->hvec, beta * mu, c->stream);
    k0.done(1);
    bool solved = false;
    if (c->opt.precision == 1 && !c->promoted) {
      if (c->blocks) {
        // a block-diagonal B keeps the FP64 factor (its blocks are small); an FP32-assembled B
        // that it finds not positive definite promotes the solve, as a broken-down FP32 factor
        // does
        scm_chol_solve(c);
        int st2 = 0;
        CUDA_TRY(c, cudaMemcpyAsync(&st2, c->status + 2, sizeof(int), cudaMemcpyDeviceToHost,
                                    c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        solved = !(f32 && (st2 & ST_NOT_PD));
        if (!solved) CUDA_TRY(c, cudaMemsetAsync(c->status + 2, 0, sizeof(int), c->stream));
      } else {
        s = mixed_sce(c, f32, &solved);
        if (s) return s;
      }
      if (!solved) {
        // promotion: from here on everything in FP64, starting with this iteration's SCM (an
        // FP32-assembled B can be singular where the FP64 one is not)
        c->promoted = true;
        c->promoted_iter = c->cur_iter;
        if (!c->fp64_asm) {
          c->fp64_asm = true;
          c->fp64_asm_iter = c->cur_iter;
        }
        if (f32) {
          f32 = false;
          s = phase_scm<double>(c);  // (the side stream's FP32 Y^{-1} is redone below)
          if (s) return s;
          KScope k4(c, KC_MISC);
          launch_rhs_border(c->D, c->B, c->ldb, c->hvec, beta * mu, c->stream);
          k4.done(1);
        }
      }
    }
    if (!solved) scm_chol_solve(c);
    KScope k3(c, KC_MISC);
    launch_dz_to_user(c->D, c->xs, c->dz, c->stream);
    k3.done(1);
  }
  KCHECK(c);
  cudaEventRecord(c->ev[2], c->stream);
  CUDA_TRY(c, cudaMemsetAsync(c->dY, 0, c->D.nnzL * 8, c->stream));
  if (c->dense) {
    KScope k0(c, KC_MISC);
    launch_slot_combine(c->D, c->dY, c->dz, 0.0, -1.0, c->stream);
    k0.done(1);
    s = f32 ? phase_pmatrix_dense<float>(c, beta * mu, Xbar)
            : phase_pmatrix_dense<double>(c, beta * mu, Xbar);
    if (s) return s;
  } else {
    KScope k0(c, KC_MISC);
    launch_slot_combine(c->D, c->dY, c->dz, 0.0, -1.0, c->stream);
    k0.done(1);
    KScope k1(c, KC_PMAT);
    int nl = 0;
    mcsdp_status ps;
    if (yinv_early) CUDA_TRY(c, cudaStreamWaitEvent(c->stream, c->ev_yinv, 0));
    if (yinv_early && yinv_f32 == f32)
      ps = f32 ? phase_pmatrix<float>(c, &nl, nullptr, false, reinterpret_cast<const float *>(c->W3))
               : phase_pmatrix<double>(c, &nl, nullptr, false, c->W3);
    else
      ps = f32 ? phase_pmatrix<float>(c, &nl) : phase_pmatrix<double>(c, &nl);
    if (ps) return ps;
    k1.done(nl);
    KScope k2(c, KC_MISC);
    launch_dx_combine(c->D, beta * mu, Xbar, c->YinvE, c->Mlow, c->Mup, c->dX, c->stream);
    k2.done(1);
  }
  // mixed form, FP32 phase: the FP32 products leave A(dX) off b - A(X̄) by their rounding (about
  // 1e-6 relative), which the iterations would accumulate in the primal residual; with disjoint
  // constraint supports (A A^* diagonal, e.g. max-cut) the direction is projected back onto the
  // primal affine set in FP64
  if (f32 && c->S.con_disjoint) {
    KScope kp(c, KC_MISC);
    launch_project_primal(c->D, Xbar, c->dX, c->stream);
    kp.done(1);
  }
  KCHECK(c);
  cudaEventRecord(c->ev[3], c->stream);
  // primal step (eq. primal_length2) on the second stream: it needs only X̄ and dX, so it runs
  // while the dual step's candidate factorisations run on the main stream
  CUDA_TRY(c, cudaStreamWaitEvent(c->st2, c->ev[3], 0));
  {
    KScope k1(c, KC_PSTEP, c->st2);
    launch_primal_step(c->D, Xbar, c->dX, c->alpha_r, c->status + 3, c->st2);
    k1.done(1);
  }
  CUDA_TRY(c, cudaEventRecord(c->ev[5], c->st2));
  KCHECK(c);
  double lo = 0.0, hi = -1.0;  // dual step: largest passing, smallest failing candidate
  if (c->dense) {
    double ar = 1.0, ad = 1.0;
    s = f32 ? dense_steps<float>(c, &ar, &ad) : dense_steps<double>(c, &ar, &ad);
    if (s) return s;
    c->alpha_root_host = ar;
    CUDA_TRY(c, cudaMemcpyAsync(c->alpha_r + (c->S.ns - 1), &c->alpha_root_host, 8,
                                cudaMemcpyHostToDevice, c->stream));
    lo = ad;
    hi = 2.0;
  }
  // dual step: bisection on the success of Y + alpha dY = N N^T (K2 on candidates)
  double cand[NCAND];
  const double first[NCAND] = {1.0, 0.95, 0.9, 0.85, 0.8, 0.7, 0.6, 0.5,
                               0.4, 0.3, 0.2, 0.1, 0.05, 0.02, 0.01, 0.003};
  for (int round = 0; round < (c->dense ? 0 : 6); ++round) {
    if (round == 0) {
      for (int i = 0; i < NCAND; ++i) cand[i] = first[i];
    } else {
      const double L = lo, H = (hi < 0 ? 1.0 : hi);
      if (lo == 0.0 && hi > 0) {  // everything failed so far: go geometric below hi
        for (int i = 0; i < NCAND; ++i) cand[i] = hi * std::pow(0.3, i + 1);
      } else {
        for (int i = 0; i < NCAND; ++i) cand[i] = L + (H - L) * (double)(i + 1) / (NCAND + 1);
      }
    }
    CUDA_TRY(c, cudaMemcpyAsync(c->alpha_c, cand, NCAND * 8, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(c->status + 8, 0, NCAND * sizeof(int), c->stream));
    s = phase_ychol(c, NCAND, c->alpha_c, c->Ylay, c->dY, c->Ncand, nullptr, c->status + 8);
    if (s) return s;
    int cs[NCAND];
    CUDA_TRY(c, cudaMemcpyAsync(cs, c->status + 8, NCAND * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  prof_flush(c);
    for (int i = 0; i < NCAND; ++i) {
      if (cs[i] == 0) lo = std::max(lo, cand[i]);
      else hi = (hi < 0) ? cand[i] : std::min(hi, cand[i]);
    }
    if (lo >= 1.0) break;
    if (lo > 0 && hi > 0 && (hi - lo) <= 1e-3 * lo) break;
  }
  CUDA_TRY(c, cudaStreamWaitEvent(c->stream, c->ev[5], 0));
  {
    KScope k2(c, KC_MISC);
    launch_measures(c->D, Xbar, c->Ylay, c->z, c->alpha_r, c->scal, c->stream);
    k2.done(2);
  }
  KCHECK(c);
  double sc[8];
  int st[8];
  CUDA_TRY(c, cudaMemcpyAsync(sc, c->scal, 6 * 8, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(st, c->status, 8 * 4, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  prof_flush(c);
  if (st[7] == -1) return fail(c, MCSDP_ERR_CUDA, "a tensor map of the root's products could not be made");
  if (st[7] & ST_TIMEOUT) return fail(c, MCSDP_ERR_TIMEOUT, "tensor-core product: a bounded wait gave up");
  if (st[2] & ST_TIMEOUT) return fail(c, MCSDP_ERR_TIMEOUT, "SCM factorisation: a bounded wait gave up");
  if (st[2] & ST_NOT_PD) return fail(c, MCSDP_ERR_NOT_PD, "Schur complement matrix is not positive definite");
  o.ap = sc[5];
  if (lo <= 0.0) return fail(c, MCSDP_ERR_STALL, "dual step length collapsed");
  o.ad = std::min(lo, 1.0);
  cudaEventRecord(c->ev[4], c->stream);
  if (tms) {
    CUDA_TRY(c, cudaEventSynchronize(c->ev[4]));
    float a, b, d, e;
    cudaEventElapsedTime(&a, c->ev[0], c->ev[1]);
    cudaEventElapsedTime(&b, c->ev[1], c->ev[2]);
    cudaEventElapsedTime(&d, c->ev[2], c->ev[3]);
    cudaEventElapsedTime(&e, c->ev[3], c->ev[4]);
    tms[0] += a;
    tms[1] += b;
    tms[2] += d;
    tms[3] += e;
  }
  return MCSDP_OK;
}

mcsdp_status factor_YX(mcsdp_ctx *c, const double *Xbar);
mcsdp_status phase_Y(mcsdp_ctx *c, const double *z);

// The graph form of one iteration (options.graph; FP64, no dense root), recorded on c->stream
// with no host synchronisation: the direction at the current iterate as in direction() with
// beta mu read from the device, the primal step beside it, the dual step's candidate rounds
// with the bracket kept on the device (the host loop's rule, frozen where the host loop would
// stop, so the steps are the same), the update with gamma alpha_p and gamma alpha_d from the
// device (skipped after a failure), then Y, N, L̂ and the scalars at the new iterate.
mcsdp_status graph_body(mcsdp_ctx *c) {
  const int n = c->S.n, m = c->S.m;
  double *g = c->gsc;
  mcsdp_status s;
  launch_graph_betamu(c->scal, n, c->opt.beta, g, c->stream);
  CUDA_TRY(c, cudaMemsetAsync(c->status + 7, 0, sizeof(int), c->stream));
  const bool yinv_early = c->W3 != nullptr;
  if (yinv_early) {
    CUDA_TRY(c, cudaEventRecord(c->ev_yinv, c->stream));
    CUDA_TRY(c, cudaStreamWaitEvent(c->st3, c->ev_yinv, 0));
    cudaStream_t main_st = c->stream;
    double *pw = c->Pw;
    unsigned char *xv = c->D.xvalid;
    c->stream = c->st3;
    c->Pw = c->Pw2;
    c->D.xvalid = c->xvalid2;
    KScope ky(c, KC_PMAT_SIDE, c->st3);
    int nly = 0;
    s = phase_pmatrix_yinv<double>(c, &nly);
    ky.done(nly);
    c->stream = main_st;
    c->Pw = pw;
    c->D.xvalid = xv;
    if (s) return s;
    CUDA_TRY(c, cudaEventRecord(c->ev_yinv, c->st3));
  }
  s = phase_scm<double>(c);
  if (s) return s;
  {
    KScope k0(c, KC_MISC);
    launch_rhs_border(c->D, c->B, c->ldb, c->hvec, 0.0, c->stream, g);
    k0.done(1);
    scm_chol_solve(c);
    KScope k3(c, KC_MISC);
    launch_dz_to_user(c->D, c->xs, c->dz, c->stream);
    k3.done(1);
  }
  CUDA_TRY(c, cudaMemsetAsync(c->dY, 0, c->D.nnzL * 8, c->stream));
  {
    KScope k0(c, KC_MISC);
    launch_slot_combine(c->D, c->dY, c->dz, 0.0, -1.0, c->stream);
    k0.done(1);
    KScope k1(c, KC_PMAT);
    int nl = 0;
    if (yinv_early) CUDA_TRY(c, cudaStreamWaitEvent(c->stream, c->ev_yinv, 0));
    s = yinv_early ? phase_pmatrix<double>(c, &nl, nullptr, false, c->W3)
                   : phase_pmatrix<double>(c, &nl);
    if (s) return s;
    k1.done(nl);
    KScope k2(c, KC_MISC);
    launch_dx_combine(c->D, 0.0, c->Xbar, c->YinvE, c->Mlow, c->Mup, c->dX, c->stream, g);
    k2.done(1);
  }
  CUDA_TRY(c, cudaEventRecord(c->ev[3], c->stream));
  CUDA_TRY(c, cudaStreamWaitEvent(c->st2, c->ev[3], 0));
  {
    KScope k1(c, KC_PSTEP, c->st2);
    launch_primal_step(c->D, c->Xbar, c->dX, c->alpha_r, c->status + 3, c->st2);
    k1.done(1);
  }
  CUDA_TRY(c, cudaEventRecord(c->ev[5], c->st2));
  DualTables tab;
  const double first[NCAND] = {1.0, 0.95, 0.9, 0.85, 0.8, 0.7, 0.6, 0.5,
                               0.4, 0.3, 0.2, 0.1, 0.05, 0.02, 0.01, 0.003};
  for (int i = 0; i < NCAND; ++i) {
    tab.first[i] = first[i];
    tab.geo[i] = std::pow(0.3, i + 1);
  }
  for (int round = 0; round < 6; ++round) {
    launch_dual_cands(g, round, c->alpha_c, NCAND, tab, c->status + 8, c->stream);
    s = phase_ychol(c, NCAND, c->alpha_c, c->Ylay, c->dY, c->Ncand, nullptr, c->status + 8);
    if (s) return s;
    launch_dual_update(c->status + 8, c->alpha_c, NCAND, g, c->stream);
  }
  CUDA_TRY(c, cudaStreamWaitEvent(c->stream, c->ev[5], 0));
  {
    KScope k2(c, KC_MISC);
    launch_measures(c->D, c->Xbar, c->Ylay, c->z, c->alpha_r, c->scal, c->stream);
    launch_graph_steps(c->scal, c->status, c->opt.gamma, g, c->stream);
    launch_update(c->D, c->Xbar, c->dX, 0.0, c->z, c->dz, 0.0, c->stream, g + 6);
    k2.done(4 + 6 * 2);
  }
  s = phase_Y(c, c->z);
  if (s) return s;
  s = factor_YX(c, c->Xbar);
  if (s) return s;
  KScope k3(c, KC_MISC);
  launch_measures(c->D, c->Xbar, c->Ylay, c->z, nullptr, c->scal, c->stream);
  k3.done(2);
  return MCSDP_OK;
}

// Runs one iteration through the graph (captured on first use); false when it cannot be
// captured (the caller then iterates without it)
bool graph_iteration(mcsdp_ctx *c, mcsdp_status *s) {
  *s = MCSDP_OK;
  if (!c->iter_exec) {
    const int64_t l0 = c->launches;
    int64_t k0[16];
    for (int q = 0; q < 16; ++q) k0[q] = c->kcount[q];
    const int prof = c->opt.profile;
    c->opt.profile = 0;  // no timing events inside the graph
    // captured on the context's own stream: work other contexts put on a shared caller stream
    // meanwhile must not enter the graph
    cudaStream_t user = c->stream;
    c->stream = c->stc;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(c->stc, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      (void)cudaGetLastError();
      c->opt.profile = prof;
      c->stream = user;
      return false;
    }
    const mcsdp_status bs = graph_body(c);
    const cudaError_t ec = cudaStreamEndCapture(c->stc, &graph);
    c->stream = user;
    c->opt.profile = prof;
    c->graph_launches = c->launches - l0;
    for (int q = 0; q < 16; ++q) {
      c->graph_kcount[q] = c->kcount[q] - k0[q];
      c->kcount[q] = k0[q];
    }
    c->launches = l0;
    if (bs != MCSDP_OK || ec != cudaSuccess || !graph ||
        cudaGraphInstantiate(&c->iter_exec, graph, cudaGraphInstantiateFlagUseNodePriority) !=
            cudaSuccess) {
      (void)cudaGetLastError();
      if (graph) cudaGraphDestroy(graph);
      c->iter_exec = nullptr;
      c->err.clear();
      return false;
    }
    cudaGraphDestroy(graph);
  }
  if (cudaGraphLaunch(c->iter_exec, c->stream) != cudaSuccess) {
    *s = fail(c, MCSDP_ERR_CUDA, "graph launch failed");
    return true;
  }
  c->launches += c->graph_launches;
  for (int q = 0; q < 16; ++q) c->kcount[q] += c->graph_kcount[q];
  return true;
}

// Runs iterations through the solve graph (built on first use): a WHILE conditional node whose
// body is the iteration of graph_body followed by k_graph_cond, which applies the host loop's
// tests to the new iterate and ends the loop, so that one graph launch and one synchronisation
// run the solve to its end (at most it_left iterations).  *ran: the iterations run.  False when
// the graph cannot be built (the caller then uses the per-iteration graph).
bool solve_graph(mcsdp_ctx *c, int it_left, int *ran, mcsdp_status *s) {
  *s = MCSDP_OK;
  *ran = 0;
  if (!c->solve_exec) {
    const int64_t l0 = c->launches;
    int64_t k0[16];
    for (int q = 0; q < 16; ++q) k0[q] = c->kcount[q];
    cudaGraph_t outer = nullptr;
    cudaGraphConditionalHandle h{};
    cudaGraphNodeParams np{};
    cudaGraphNode_t node = nullptr;
    bool ok = cudaGraphCreate(&outer, 0) == cudaSuccess &&
              cudaGraphConditionalHandleCreate(&h, outer, 1, cudaGraphCondAssignDefault) ==
                  cudaSuccess;
    if (ok) {
      np.type = cudaGraphNodeTypeConditional;
      np.conditional.handle = h;
      np.conditional.type = cudaGraphCondTypeWhile;
      np.conditional.size = 1;
      ok = cudaGraphAddNode(&node, outer, nullptr, nullptr, 0, &np) == cudaSuccess;
    }
    if (ok) {
      const int prof = c->opt.profile;
      c->opt.profile = 0;
      cudaStream_t user = c->stream;
      c->stream = c->stc;
      ok = cudaStreamBeginCaptureToGraph(c->stc, np.conditional.phGraph_out[0], nullptr, nullptr,
                                         0, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (ok) {
        const mcsdp_status bs = graph_body(c);
        launch_graph_cond(h, c->scal, c->status, c->gsc, c->gcnt, c->S.n, c->opt.gap_tol,
                          c->opt.feas_tol, c->stc);
        ++c->launches;
        cudaGraph_t body = nullptr;
        ok = cudaStreamEndCapture(c->stc, &body) == cudaSuccess && bs == MCSDP_OK;
      }
      c->stream = user;
      c->opt.profile = prof;
    }
    c->sgraph_launches = c->launches - l0;
    for (int q = 0; q < 16; ++q) {
      c->sgraph_kcount[q] = c->kcount[q] - k0[q];
      c->kcount[q] = k0[q];
    }
    c->launches = l0;
    if (ok)
      ok = cudaGraphInstantiate(&c->solve_exec, outer, cudaGraphInstantiateFlagUseNodePriority) ==
           cudaSuccess;
    if (outer) cudaGraphDestroy(outer);
    if (!ok) {
      (void)cudaGetLastError();
      c->solve_exec = nullptr;
      c->err.clear();
      return false;
    }
  }
  const int lim[2] = {0, it_left};
  int cnt[2] = {0, 0};
  if (cudaMemcpyAsync(c->gcnt, lim, sizeof(lim), cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
      cudaGraphLaunch(c->solve_exec, c->stream) != cudaSuccess ||
      cudaMemcpyAsync(cnt, c->gcnt, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess) {
    *s = fail(c, MCSDP_ERR_CUDA, "solve graph launch failed");
    return true;
  }
  *ran = cnt[0];
  c->launches += c->sgraph_launches * cnt[0];
  for (int q = 0; q < 16; ++q) c->kcount[q] += c->sgraph_kcount[q] * cnt[0];
  if (cnt[0] < 1) *s = fail(c, MCSDP_ERR_CUDA, "solve graph ran no iteration");
  return true;
}

// Y, N, L̂ and the scalars at the current iterate (c->Xbar, c->z)
mcsdp_status prepare_read(mcsdp_ctx *c, double *scal_host, int *failed);

mcsdp_status prepare(mcsdp_ctx *c, const double *Xbar, const double *z, double *scal_host,
                     int *failed = nullptr) {
  mcsdp_status s = phase_Y(c, z);
  if (s) return s;
  s = factor_YX(c, Xbar);
  if (s) return s;
  {
    KScope k2(c, KC_MISC);
    launch_measures(c->D, Xbar, c->Ylay, z, nullptr, c->scal, c->stream);
    k2.done(2);
  }
  KCHECK(c);
  return prepare_read(c, scal_host, failed);
}

// the host side of prepare: the scalars and the factorisations' statuses
mcsdp_status prepare_read(mcsdp_ctx *c, double *scal_host, int *failed) {
  int st[4];
  if (scal_host) CUDA_TRY(c, cudaMemcpyAsync(scal_host, c->scal, 6 * 8, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(st, c->status, 4 * 4, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  prof_flush(c);
  if (failed) *failed = ((st[0] & ST_NOT_PD) ? 1 : 0) | ((st[1] & ST_NOT_PD) ? 2 : 0);
  if ((st[0] | st[1]) & ST_TIMEOUT) return fail(c, MCSDP_ERR_TIMEOUT, "a dense factorisation: a bounded wait gave up");
  if ((st[0] | st[1]) & ST_NUMERIC) return fail(c, MCSDP_ERR_CUDA, "FP32 root factorisation: a tensor map could not be made");
  if (st[0] & ST_NOT_PD) return fail(c, MCSDP_ERR_NOT_PD, "Y = A_0 - sum z_k A_k is not positive definite");
  if (st[1] & ST_NOT_PD) return fail(c, MCSDP_ERR_NOT_PD, "a clique block of X̄ is not positive definite");
  return MCSDP_OK;
}

mcsdp_status set_default_start(mcsdp_ctx *c) {
  CUDA_TRY(c, cudaMemsetAsync(c->Xbar, 0, c->D.nnzL * 8, c->stream));
  KScope ks(c, KC_MISC);
  launch_set_identity(c->D, c->Xbar, c->stream);
  ks.done(1);
  KCHECK(c);
  CUDA_TRY(c, cudaMemcpyAsync(c->z, c->z0_default.data(), (size_t)c->S.m * 8, cudaMemcpyHostToDevice,
                              c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  prof_flush(c);
  return MCSDP_OK;
}

}  // namespace

// =============================================================================================
extern "C" {

void mcsdp_default_options(mcsdp_options *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->beta = 0.1;
  o->gamma = 0.9;
  o->gap_tol = 1e-7;
  o->feas_tol = 1e-7;
  o->max_iter = 60;
  o->precision = 0;
  o->timeout_cycles = 0;
  o->device = 0;
  o->verbose = 0;
  o->panel_max = 80;
  o->group_max = 64;
  o->panel_budget_mb = 1024.0;
  o->profile = 0;
  o->relax = 1;
  o->solve_warps = 0;
  o->mixed_gap = 0.0;
  o->root_rows = 0;
  o->tensor_cores = 1;
  o->mixed_asm_gap = 0.0;
  o->scm_blocks = 0;
}

const char *mcsdp_last_error(const mcsdp_ctx *c) { return c ? c->err.c_str() : "null context"; }

mcsdp_status mcsdp_create(const mcsdp_problem *p, const mcsdp_options *opt, void *stream,
                          mcsdp_ctx **out) {
  if (!out) return MCSDP_ERR_ARG;
  *out = nullptr;
  mcsdp_ctx *c = new mcsdp_ctx();
  if (opt) c->opt = *opt;
  else mcsdp_default_options(&c->opt);
  *out = c;
  if (!p) return fail(c, MCSDP_ERR_ARG, "problem is NULL");
  if (p->n <= 0 || p->m <= 0) return fail(c, MCSDP_ERR_ARG, "n and m must be positive");
  if (p->nnz < 0 || (p->nnz > 0 && (!p->mat || !p->row || !p->col || !p->val)))
    return fail(c, MCSDP_ERR_ARG, "entry arrays missing");
  if (!p->c) return fail(c, MCSDP_ERR_ARG, "c/b vector missing");
  if (p->form != 0 && p->form != 1) return fail(c, MCSDP_ERR_ARG, "form must be 0 (SDPA) or 1 (paper)");
  if (c->opt.precision != 0 && c->opt.precision != 1)
    return fail(c, MCSDP_ERR_ARG, "precision must be 0 (FP64) or 1 (mixed)");
  if (c->opt.precision == 1 && p->m > 50000)
    return fail(c, MCSDP_ERR_ARG, "the mixed form supports m <= 50000");
  if (c->opt.panel_max <= 0) c->opt.panel_max = 80;
  if (c->opt.panel_max > 96) return fail(c, MCSDP_ERR_ARG, "panel_max must be <= 96");
  if (c->opt.group_max <= 0) c->opt.group_max = 64;
  if (c->opt.group_max > 64) return fail(c, MCSDP_ERR_ARG, "group_max must be <= 64");
  if (!(c->opt.beta > 0 && c->opt.beta < 1) || !(c->opt.gamma > 0 && c->opt.gamma < 1))
    return fail(c, MCSDP_ERR_ARG, "beta and gamma must lie in (0, 1)");
  ProblemData &P = c->P;
  c->form = p->form;
  c->ue_k.clear();
  c->ue_i.clear();
  c->ue_j.clear();
  P.n = p->n;
  P.m = p->m;
  P.b.assign(p->c, p->c + p->m);
  // duplicates: sort (mat, row, col, input index); the first repeat in input order is reported
  int64_t dup = -1;
  {
    std::vector<std::array<int64_t, 4>> keys((size_t)p->nnz);
    for (int64_t t = 0; t < p->nnz; ++t) keys[t] = {p->mat[t], p->row[t], p->col[t], t};
    std::sort(keys.begin(), keys.end());
    for (size_t u = 1; u < keys.size(); ++u)
      if (keys[u][0] == keys[u - 1][0] && keys[u][1] == keys[u - 1][1] &&
          keys[u][2] == keys[u - 1][2] && (dup < 0 || keys[u][3] < dup))
        dup = keys[u][3];
  }
  for (int64_t t = 0; t < p->nnz; ++t) {
    int k = p->mat[t], i = p->row[t], j = p->col[t];
    double v = p->val[t];
    if (k < 0 || k > p->m || i < 0 || j < 0 || i >= p->n || j >= p->n)
      return fail(c, MCSDP_ERR_ARG, "entry " + std::to_string(t) + ": index out of range");
    if (i > j) return fail(c, MCSDP_ERR_ARG, "entry " + std::to_string(t) + ": row > col (give the upper triangle)");
    if (!std::isfinite(v)) return fail(c, MCSDP_ERR_ARG, "entry " + std::to_string(t) + ": not finite");
    if (t == dup)
      return fail(c, MCSDP_ERR_ARG, "entry " + std::to_string(t) + ": duplicate (mat,row,col)");
    c->ue_k.push_back(k);
    c->ue_i.push_back(i);
    c->ue_j.push_back(j);
    if (k == 0 && p->form == 0) v = -v;  // A_0 = -F_0
    P.mat.push_back(k);
    P.row.push_back(i);
    P.col.push_back(j);
    P.val.push_back(v);
  }
  for (double v : P.b)
    if (!std::isfinite(v)) return fail(c, MCSDP_ERR_ARG, "b/c not finite");
  SymbolicOptions so;
  so.panel_max = c->opt.panel_max;
  so.group_max = c->opt.group_max;
  so.relax = c->opt.relax;
  if (c->opt.root_rows < 0) {
    so.root_rows = so.root_cols = 0;
  } else {
    so.root_rows = c->opt.root_rows > 0 ? std::min(c->opt.root_rows, SMALL_ROWS) : SMALL_ROWS;
    so.root_cols = SMALL_COLS;
  }
  std::string e = analyze(P, so, c->S);
  if (!e.empty()) return fail(c, MCSDP_ERR_ARG, e);
  {
    // every clique but a dense root must fit the shared-memory clique kernels
    const Symbolic &S = c->S;
    const int nsmall = S.dense_root ? S.ns - 1 : S.ns;
    int mr = 0, mc = 0;
    for (int t = 0; t < nsmall; ++t) {
      mr = std::max(mr, (int)(S.sn_rowptr[t + 1] - S.sn_rowptr[t]));
      mc = std::max(mc, S.sn_col[t + 1] - S.sn_col[t]);
    }
    if (mc > SMALL_COLS || mr > SMALL_ROWS)
      return fail(c, MCSDP_ERR_ARG, "a clique of " + std::to_string(mr) + " rows / " +
                                        std::to_string(mc) +
                                        " columns exceeds the library's shared-memory clique kernels (" +
                                        std::to_string(SMALL_ROWS) + " / " + std::to_string(SMALL_COLS) + ")");
  }
  // default dual start
  c->z0_default.assign(P.m, 0.0);
  if (c->S.unit_diag_constraints) {
    std::vector<double> rowabs(P.n, 0.0);
    for (size_t t = 0; t < P.row.size(); ++t)
      if (P.mat[t] == 0) {
        rowabs[P.row[t]] += std::fabs(P.val[t]);
        if (P.row[t] != P.col[t]) rowabs[P.col[t]] += std::fabs(P.val[t]);
      }
    for (size_t t = 0; t < P.row.size(); ++t)
      if (P.mat[t] > 0) c->z0_default[P.mat[t] - 1] = -rowabs[P.row[t]] - 1.0;
  }
  c->host_only = c->opt.device < 0;
  if (!c->host_only) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->opt.device) == cudaSuccess &&
        sms > 0)
      c->num_sms = sms;
  }
  plan_workspace(c);
  c->stream = (cudaStream_t)stream;
  if (!c->host_only) {
    c->device = c->opt.device;
    CUDA_TRY(c, cudaSetDevice(c->device));
    for (int i = 0; i < 8; ++i) CUDA_TRY(c, cudaEventCreate(&c->ev[i]));
    int prio_lo = 0, prio_hi = 0;
    CUDA_TRY(c, cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
    CUDA_TRY(c, cudaStreamCreateWithPriority(&c->st2, cudaStreamNonBlocking, prio_lo));
    CUDA_TRY(c, cudaStreamCreateWithPriority(&c->st1, cudaStreamNonBlocking, prio_hi));
    CUDA_TRY(c, cudaStreamCreateWithPriority(&c->st3, cudaStreamNonBlocking, prio_lo));
    CUDA_TRY(c, cudaStreamCreateWithFlags(&c->stc, cudaStreamNonBlocking));
    CUDA_TRY(c, cudaEventCreateWithFlags(&c->ev_yinv, cudaEventDisableTiming));
    CUDA_TRY(c, cudaStreamCreateWithPriority(&c->st4, cudaStreamNonBlocking, prio_lo));
    CUDA_TRY(c, cudaEventCreateWithFlags(&c->ev_n0, cudaEventDisableTiming));
    CUDA_TRY(c, cudaEventCreateWithFlags(&c->ev_n1, cudaEventDisableTiming));
    CUDA_TRY(c, cudaEventCreateWithFlags(&c->ev_f0, cudaEventDisableTiming));
    CUDA_TRY(c, cudaEventCreateWithFlags(&c->ev_f1, cudaEventDisableTiming));
    for (int i = 0; i < 2; ++i) {
      CUDA_TRY(c, cudaEventCreateWithFlags(&c->ev_next[i], cudaEventDisableTiming));
      CUDA_TRY(c, cudaEventCreateWithFlags(&c->ev_rest[i], cudaEventDisableTiming));
      c->cs.next[i] = c->ev_next[i];
      c->cs.rest_ev[i] = c->ev_rest[i];
    }
    CUDA_TRY(c, cudaEventCreateWithFlags(&c->cs.fork, cudaEventDisableTiming));
    CUDA_TRY(c, cudaEventCreateWithFlags(&c->cs.chain_done, cudaEventDisableTiming));
    CUDA_TRY(c, cudaEventCreateWithFlags(&c->cs.entry, cudaEventDisableTiming));
    CUDA_TRY(c, cudaEventCreateWithFlags(&c->cs.exit, cudaEventDisableTiming));
    c->cs.chain = c->st1;
    c->cs.rest = c->st2;
  }
  c->err.clear();
  return MCSDP_OK;
}

void mcsdp_destroy(mcsdp_ctx *c) {
  if (!c) return;
  if (!c->host_only && c->device >= 0) {
    cudaSetDevice(c->device);
    if (c->iter_exec) cudaGraphExecDestroy(c->iter_exec);
    if (c->solve_exec) cudaGraphExecDestroy(c->solve_exec);
    for (int i = 0; i < 8; ++i)
      if (c->ev[i]) cudaEventDestroy(c->ev[i]);
    if (!c->pending.empty()) {
      cudaStreamSynchronize(c->stream);
      prof_flush(c);
    }
    for (cudaEvent_t e : c->evpool) cudaEventDestroy(e);
    for (int i = 0; i < 2; ++i) {
      if (c->ev_next[i]) cudaEventDestroy(c->ev_next[i]);
      if (c->ev_rest[i]) cudaEventDestroy(c->ev_rest[i]);
    }
    if (c->st2) cudaStreamDestroy(c->st2);
    if (c->st1) cudaStreamDestroy(c->st1);
    if (c->st3) cudaStreamDestroy(c->st3);
    if (c->stc) cudaStreamDestroy(c->stc);
    if (c->ev_yinv) cudaEventDestroy(c->ev_yinv);
    if (c->st4) cudaStreamDestroy(c->st4);
    if (c->ev_n0) cudaEventDestroy(c->ev_n0);
    if (c->ev_n1) cudaEventDestroy(c->ev_n1);
    if (c->ev_f0) cudaEventDestroy(c->ev_f0);
    if (c->ev_f1) cudaEventDestroy(c->ev_f1);
    chol_graphs_destroy(&c->cs);
    if (c->cs.fork) cudaEventDestroy(c->cs.fork);
    if (c->cs.chain_done) cudaEventDestroy(c->cs.chain_done);
    if (c->cs.entry) cudaEventDestroy(c->cs.entry);
    if (c->cs.exit) cudaEventDestroy(c->cs.exit);
  }
  delete c;
}

mcsdp_status mcsdp_workspace_size(const mcsdp_ctx *c, size_t *bytes) {
  if (!c || !bytes) return MCSDP_ERR_ARG;
  *bytes = c->ws_bytes;
  return MCSDP_OK;
}

mcsdp_status mcsdp_set_workspace(mcsdp_ctx *c, void *ptr, size_t bytes) {
  if (!c) return MCSDP_ERR_ARG;
  if (c->host_only) return fail(c, MCSDP_ERR_STATE, "host-only context");
  if (!ptr || bytes < c->ws_bytes) return fail(c, MCSDP_ERR_OOM, "workspace smaller than mcsdp_workspace_size");
  if (((uintptr_t)ptr & 255) != 0) return fail(c, MCSDP_ERR_ARG, "workspace must be 256-byte aligned");
  CUDA_TRY(c, cudaSetDevice(c->device));
  c->ws = (char *)ptr;
  c->ws_have = bytes;
  bind_pointers(c);
  if (scm_tiles_smem_bytes(c->D, c->pmax) > 227 * 1024)
    return fail(c, MCSDP_ERR_ARG, "SCM groups too large for the shared-memory tile kernel");
  for (const Upload &u : c->uploads)
    CUDA_TRY(c, cudaMemcpyAsync(c->ws + u.off, u.src, u.bytes, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemsetAsync(c->B, 0, (size_t)c->ldb * c->S.m * 8, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  prof_flush(c);
  c->iterate_set = false;
  return MCSDP_OK;
}

mcsdp_status mcsdp_sym_info_get(const mcsdp_ctx *c, mcsdp_sym_info *info) {
  if (!c || !info) return MCSDP_ERR_ARG;
  const Symbolic &S = c->S;
  info->n = S.n;
  info->m = S.m;
  info->nsuper = S.ns;
  info->ngroup = S.ngroup;
  info->max_nrow = S.max_nrow;
  info->max_ncol = S.max_ncol;
  info->tree_height = S.height;
  info->nnz_layout = S.ns ? S.sn_valptr[S.ns] : 0;
  info->nnz_lower_E = S.nnz_lower_E;
  info->nslot = S.nslot;
  info->table_bytes = 0;
  for (const Upload &u : c->uploads) info->table_bytes += (int64_t)u.bytes;
  info->ncomp = S.ncomp;
  info->scm_blocks = c->blocks ? 1 : 0;
  return MCSDP_OK;
}

mcsdp_status mcsdp_sym_export(const mcsdp_ctx *c, int32_t *perm, int32_t *sn_col, int64_t *sn_rowptr,
                              int32_t *sn_rows, int64_t *sn_valptr, int32_t *con_order) {
  if (!c) return MCSDP_ERR_ARG;
  const Symbolic &S = c->S;
  if (perm) std::copy(S.perm.begin(), S.perm.end(), perm);
  if (sn_col) std::copy(S.sn_col.begin(), S.sn_col.end(), sn_col);
  if (sn_rowptr) std::copy(S.sn_rowptr.begin(), S.sn_rowptr.end(), sn_rowptr);
  if (sn_rows) std::copy(S.rows.begin(), S.rows.end(), sn_rows);
  if (sn_valptr) std::copy(S.sn_valptr.begin(), S.sn_valptr.end(), sn_valptr);
  if (con_order) std::copy(S.con_order.begin(), S.con_order.end(), con_order);
  return MCSDP_OK;
}

mcsdp_status mcsdp_set_iterate(mcsdp_ctx *c, const double *Xbar, const double *z) {
  mcsdp_status s = ready(c);
  if (s) return s;
  if (!c->iterate_set) {
    s = set_default_start(c);
    if (s) return s;
  }
  if (Xbar) CUDA_TRY(c, cudaMemcpyAsync(c->Xbar, Xbar, c->D.nnzL * 8, cudaMemcpyDeviceToDevice, c->stream));
  if (z) CUDA_TRY(c, cudaMemcpyAsync(c->z, z, (size_t)c->S.m * 8, cudaMemcpyDeviceToDevice, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  prof_flush(c);
  c->iterate_set = true;
  return MCSDP_OK;
}

mcsdp_status mcsdp_get_iterate(const mcsdp_ctx *cc, double *Xbar, double *z, double *Y) {
  mcsdp_ctx *c = const_cast<mcsdp_ctx *>(cc);
  mcsdp_status s = ready(c);
  if (s) return s;
  if (Xbar) CUDA_TRY(c, cudaMemcpyAsync(Xbar, c->Xbar, c->D.nnzL * 8, cudaMemcpyDeviceToDevice, c->stream));
  if (z) CUDA_TRY(c, cudaMemcpyAsync(z, c->z, (size_t)c->S.m * 8, cudaMemcpyDeviceToDevice, c->stream));
  if (Y) CUDA_TRY(c, cudaMemcpyAsync(Y, c->Ylay, c->D.nnzL * 8, cudaMemcpyDeviceToDevice, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  prof_flush(c);
  return MCSDP_OK;
}

mcsdp_status mcsdp_factors(mcsdp_ctx *c, const double *Xbar, const double *z, double *Lh, double *N) {
  mcsdp_status s = ready(c);
  if (s) return s;
  s = prepare(c, Xbar, z, nullptr);
  if (s) return s;
  if (Lh) CUDA_TRY(c, cudaMemcpyAsync(Lh, c->Lh, c->D.nnzL * 8, cudaMemcpyDeviceToDevice, c->stream));
  if (N) CUDA_TRY(c, cudaMemcpyAsync(N, c->N, c->D.nnzL * 8, cudaMemcpyDeviceToDevice, c->stream));
  if (c->dense) {
    // Algorithm 1 at the root clique C = S = R: L̂_RR is the Cholesky factor of X̄_RR^{-1}
    // (unique), X̄_RR^{-1} = X^T X with X = L^{-1} of X̄_RR = L L^T (RS_P, from prepare)
    const int nR = c->nR;
    const int64_t rv = c->D.root_valp;
    CUDA_TRY(c, cudaMemsetAsync(c->status + 6, 0, sizeof(int), c->stream));
    KScope ks(c, KC_ALG1);
    // RS_P's upper triangle holds the mirror of its rows: the product must read a zero there
    copy_lower(c->RS_P, nR, c->RS_T, nR, nR, c->stream);
    int nl = 1 + dense_lauum<double>(c->RS_T, nR, nR, c->RS_M, 1, nR, true, c->stream);
    nl += dense_potrf(c->RS_M, nR, nR, c->status + 6, c->rLinv2, c->stream, c->rsync2,
                      c->opt.timeout_cycles);
    if (Lh) copy_lower(c->RS_M, nR, Lh + rv, nR, nR, c->stream);
    // the dense Cholesky keeps the factor's rows mirrored above the diagonal: export zeros there
    if (N) copy_lower(c->N + rv, nR, N + rv, nR, nR, c->stream);
    ks.done(nl + 2);
    int st[8];
    s = read_status(c, st, 8);
    if (s) return s;
    if (st[6] & ST_NOT_PD) return fail(c, MCSDP_ERR_NOT_PD, "X̄_RR^{-1} not positive definite");
  }
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  prof_flush(c);
  return MCSDP_OK;
}

mcsdp_status mcsdp_scm_assemble(mcsdp_ctx *c, const double *Xbar, const double *z, double *Bout,
                                int64_t ldb, double *h, int32_t precision) {
  mcsdp_status s = ready(c);
  if (s) return s;
  if (precision != 0 && precision != 1) return fail(c, MCSDP_ERR_ARG, "precision must be 0 or 1");
  if (!Xbar || !z || !Bout || ldb < c->S.m) return fail(c, MCSDP_ERR_ARG, "bad arguments");
  s = phase_Y(c, z);
  if (s) return s;
  s = factor_YX(c, Xbar);
  if (s) return s;
  if (precision == 1 && !(c->opt.precision == 1 && c->f32_solves))
    return fail(c, MCSDP_ERR_ARG, "precision 1 needs a context created with precision 1");
  CUDA_TRY(c, cudaMemsetAsync(c->status + 7, 0, sizeof(int), c->stream));
  if (precision == 1) {
    cast_factors(c);
    s = phase_scm<float>(c);
  } else {
    s = phase_scm<double>(c);
  }
  if (s) return s;
  KScope ks(c, KC_MISC);
  launch_B_to_user(c->D, c->B, c->ldb, Bout, ldb, c->hvec, h, c->stream);
  ks.done(1);
  KCHECK(c);
  int st[8];
  s = read_status(c, st, 8);
  if (s) return s;
  if (st[7] == -1) return fail(c, MCSDP_ERR_CUDA, "a tensor map of the root's products could not be made");
  if (st[7] & ST_TIMEOUT) return fail(c, MCSDP_ERR_TIMEOUT, "tensor-core product: a bounded wait gave up");
  if (st[0] & ST_NOT_PD) return fail(c, MCSDP_ERR_NOT_PD, "Y is not positive definite");
  if (st[1] & ST_NOT_PD) return fail(c, MCSDP_ERR_NOT_PD, "a clique block of X̄ is not positive definite");
  return MCSDP_OK;
}

mcsdp_status mcsdp_newton_step(mcsdp_ctx *c, const double *Xbar, const double *z, double *dz,
                               double *dX, double *dY, double *ap, double *ad, double *mu) {
  mcsdp_status s = ready(c);
  if (s) return s;
  if (!Xbar || !z) return fail(c, MCSDP_ERR_ARG, "Xbar and z are required");
  // the iterate lives in the context buffers during the step
  CUDA_TRY(c, cudaMemcpyAsync(c->z, z, (size_t)c->S.m * 8, cudaMemcpyDeviceToDevice, c->stream));
  double sc[8];
  s = prepare(c, Xbar, c->z, sc);
  if (s) return s;
  const double muv = sc[0] / c->S.n;
  IterOut o{};
  c->promoted = false;  // each call decides on its own
  c->promoted_iter = -1;
  c->cur_iter = 0;
  s = direction(c, Xbar, muv, o, nullptr);
  if (s) return s;
  if (dz) CUDA_TRY(c, cudaMemcpyAsync(dz, c->dz, (size_t)c->S.m * 8, cudaMemcpyDeviceToDevice, c->stream));
  if (dX) CUDA_TRY(c, cudaMemcpyAsync(dX, c->dX, c->D.nnzL * 8, cudaMemcpyDeviceToDevice, c->stream));
  if (dY) CUDA_TRY(c, cudaMemcpyAsync(dY, c->dY, c->D.nnzL * 8, cudaMemcpyDeviceToDevice, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  prof_flush(c);
  if (ap) *ap = o.ap;
  if (ad) *ad = o.ad;
  if (mu) *mu = muv;
  return MCSDP_OK;
}

mcsdp_status mcsdp_solve(mcsdp_ctx *c, mcsdp_result *res) {
  mcsdp_status s = ready(c);
  if (s) return s;
  if (!c->iterate_set) {
    s = set_default_start(c);
    if (s) return s;
    c->iterate_set = true;
  }
  mcsdp_result r{};
  c->promoted = false;
  c->promoted_iter = -1;
  c->fp64_asm = false;
  c->fp64_asm_iter = -1;
  c->refine_steps = 0;
  // the root's FP32 factorisations belong to this loop only
  struct Root32Off {
    mcsdp_ctx *c;
    ~Root32Off() { c->root32 = c->inv32 = false; }
  } root32_off{c};
  // the gap below which the mixed form runs in FP64 throughout: for large m the refinement of
  // the FP32 factor (long form, see mixed_sce) stays far cheaper than the FP64 factorisation
  // until it stalls, so no gap threshold applies by default
  const double mixed_gap = c->opt.mixed_gap > 0 ? c->opt.mixed_gap
                           : c->opt.mixed_gap < 0 || c->S.m >= MIXED_LONG_M ? 0.0 : 1e-5;
  // the mixed form's FP64-assembly threshold: with a dense root the FP32 products and factors of
  // the root, relative to the shrinking direction, decide the root clique's primal step well
  // before the FP32 factor of B stops refining
  const double asm_gap = c->opt.mixed_asm_gap > 0 ? c->opt.mixed_asm_gap
                        : (c->dense ? MIXED_ASM_GAP_ROOT : (mixed_gap > 0 ? mixed_gap : 1e-5));
  double prev_pinf = -1.0;
  float tms[4] = {0, 0, 0, 0};
  cudaEvent_t t0 = c->ev[6], t1 = c->ev[7];
  cudaEventRecord(t0, c->stream);
  const int n = c->S.n;
  mcsdp_status final_status = MCSDP_ERR_MAXITER;
  double last_ap = 0.0, last_ad = 0.0;
  const bool use_graph = c->opt.graph >= 1 && !c->dense && c->opt.precision == 0;
  bool graph_prepared = false;
  for (int it = 0; it <= c->opt.max_iter; ++it) {
    double sc[8];
    int failed = 0;
    c->root32 = c->opt.precision == 1 && c->dense && !c->fp64_asm && !c->promoted;
    c->inv32 = c->opt.precision == 1 && c->dense && !c->root32;
    if (graph_prepared) {
      // the graph ran the previous iteration's direction and update and these factors
      double gh[12];
      CUDA_TRY(c, cudaMemcpyAsync(gh, c->gsc, 12 * 8, cudaMemcpyDeviceToHost, c->stream));
      s = prepare_read(c, sc, &failed);
      if (s == MCSDP_OK && gh[8] == 2.0)
        s = fail(c, (((int)gh[11]) & ST_TIMEOUT) ? MCSDP_ERR_TIMEOUT : MCSDP_ERR_NOT_PD,
                 "Schur complement matrix is not positive definite");
      if (s == MCSDP_OK && gh[8] == 1.0) s = fail(c, MCSDP_ERR_STALL, "dual step length collapsed");
      if (s) {
        final_status = s;
        break;
      }
      if (c->opt.verbose)
        std::fprintf(stderr, "it %3d (graph) ap %.3f ad %.3f\n", it - 1, gh[9], gh[10]);
    } else {
      s = prepare(c, c->Xbar, c->z, sc, &failed);
    }
    graph_prepared = false;
    // dense root: the step lengths are Lanczos estimates, confirmed here by the factorisations at
    // the new iterate; a failure halves the failing step (from the saved iterate) and retries
    for (int bt = 0; s == MCSDP_ERR_NOT_PD && c->dense && it > 0 && bt < 10; ++bt) {
      if (failed & 2) last_ap *= 0.5;
      if (failed & 1) last_ad *= 0.5;
      CUDA_TRY(c, cudaMemcpyAsync(c->Xbar, c->Xprev, c->D.nnzL * 8, cudaMemcpyDeviceToDevice, c->stream));
      CUDA_TRY(c, cudaMemcpyAsync(c->z, c->zprev, (size_t)c->S.m * 8, cudaMemcpyDeviceToDevice, c->stream));
      launch_update(c->D, c->Xbar, c->dX, c->opt.gamma * last_ap, c->z, c->dz, c->opt.gamma * last_ad,
                    c->stream);
      if (c->opt.verbose)
        std::fprintf(stderr, "  backtrack: ap %.3e ad %.3e\n", last_ap, last_ad);
      failed = 0;
      s = prepare(c, c->Xbar, c->z, sc, &failed);
    }
    if (s) {
      if (it == 0 && s == MCSDP_ERR_NOT_PD && c->err.find("Y =") != std::string::npos)
        c->err += " at the start: give a dual-feasible z with mcsdp_set_iterate";
      return s;
    }
    const double mu = sc[0] / n, pobj = sc[1], dobj = sc[2];
    const double gap = std::fabs(pobj - dobj) / std::max(1.0, (std::fabs(pobj) + std::fabs(dobj)) / 2);
    const double pinf = sc[3] / std::max(1.0, sc[4]);
    // mixed form: FP64 throughout once the gap is small, or if the primal residual grows well
    // above the level the FP32 solves leave (about 1e-6 relative; it contracts by
    // (1 - gamma alpha_p) per iteration in exact arithmetic)
    if (c->opt.precision == 1 && !c->promoted &&
        ((prev_pinf > 0 && pinf > 2.0 * prev_pinf && pinf > 1e-4) || gap < mixed_gap)) {
      c->promoted = true;
      c->promoted_iter = it;
    }
    if (c->opt.precision == 1 && !c->fp64_asm && (c->promoted || gap < asm_gap)) {
      c->fp64_asm = true;
      c->fp64_asm_iter = it;
      if (c->root32) {  // this iteration's root factors were FP32: again in FP64
        c->root32 = false;
        c->inv32 = true;
        s = prepare(c, c->Xbar, c->z, sc, &failed);
        if (s) return s;
      }
    }
    prev_pinf = pinf;
    c->cur_iter = it;
    r.pobj = pobj;
    r.dobj = dobj;
    r.gap = gap;
    r.pinf = pinf;
    r.dinf = 0.0;
    r.mu = mu;
    r.iters = it;
    if (!std::isfinite(pobj) || !std::isfinite(dobj) || !std::isfinite(mu)) {
      final_status = MCSDP_ERR_NUMERIC;
      c->err = "NaN/Inf in the iterate";
      break;
    }
    if (gap <= c->opt.gap_tol && pinf <= c->opt.feas_tol) {
      final_status = MCSDP_OK;
      break;
    }
    if (it == c->opt.max_iter) break;
    if (use_graph && it >= 1 && c->opt.graph == 2 && !c->solve_graph_failed) {
      int ran = 0;
      if (solve_graph(c, c->opt.max_iter - it, &ran, &s)) {
        if (s) {
          final_status = s;
          break;
        }
        it += ran - 1;  // the loop's top reads the state the graph left, as after one iteration
        graph_prepared = true;
        continue;
      }
      c->solve_graph_failed = true;  // not buildable here: the per-iteration graph
    }
    if (use_graph && it >= 1 && !c->graph_failed) {
      if (graph_iteration(c, &s)) {
        if (s) {
          final_status = s;
          break;
        }
        graph_prepared = true;
        continue;
      }
      c->graph_failed = true;  // not capturable here: the iteration runs without the graph
    }
    IterOut o{};
    s = direction(c, c->Xbar, mu, o, tms);
    if (s) {
      final_status = s;
      break;
    }
    if (c->opt.verbose)
      std::fprintf(stderr, "it %3d pobj %+.10e dobj %+.10e gap %.2e pinf %.2e mu %.2e ap %.3f ad %.3f\n",
                   it, pobj, dobj, gap, pinf, mu, o.ap, o.ad);
    if (c->opt.verbose > 1 && c->dense) {
      // the step-length bounds: the root clique's and the dual Lanczos values, the forest's
      // smallest clique step
      std::vector<double> ar(c->S.ns);
      CUDA_TRY(c, cudaMemcpy(ar.data(), c->alpha_r, c->S.ns * 8, cudaMemcpyDeviceToHost));
      double fmin = 1.0;
      for (int r = 0; r + 1 < c->S.ns; ++r) fmin = std::min(fmin, ar[r]);
      std::fprintf(stderr, "    root: theta %.4e bound %.2e alpha %.4f | forest min alpha %.4f | "
                   "dual: theta %.4e bound %.2e\n", c->lz_last[0], c->lz_last[1], ar[c->S.ns - 1],
                   fmin, c->lz_last[2], c->lz_last[3]);
    }
    if (c->dense) {
      CUDA_TRY(c, cudaMemcpyAsync(c->Xprev, c->Xbar, c->D.nnzL * 8, cudaMemcpyDeviceToDevice, c->stream));
      CUDA_TRY(c, cudaMemcpyAsync(c->zprev, c->z, (size_t)c->S.m * 8, cudaMemcpyDeviceToDevice, c->stream));
    }
    last_ap = o.ap;
    last_ad = o.ad;
    KScope ks(c, KC_MISC);
    launch_update(c->D, c->Xbar, c->dX, c->opt.gamma * o.ap, c->z, c->dz, c->opt.gamma * o.ad, c->stream);
    ks.done(1);
    KCHECK(c);
  }
  cudaEventRecord(t1, c->stream);
  CUDA_TRY(c, cudaEventSynchronize(t1));
  prof_flush(c);
  float ms = 0;
  cudaEventElapsedTime(&ms, t0, t1);
  r.seconds = ms * 1e-3;
  r.t_scm = tms[0] * 1e-3;
  r.t_chol = tms[1] * 1e-3;
  r.t_pmat = tms[2] * 1e-3;
  r.t_other = r.seconds - r.t_scm - r.t_chol - r.t_pmat;
  r.status = final_status;
  r.precision = c->opt.precision;
  r.promoted_iter = c->opt.precision == 1 ? c->promoted_iter : -1;
  r.assembly_iter = c->opt.precision == 1 ? c->fp64_asm_iter : -1;
  r.refine_steps = c->refine_steps;
  if (res) *res = r;
  return final_status;
}

mcsdp_status mcsdp_solve_batch(mcsdp_ctx *const *ctxs, int32_t count, int32_t nthreads,
                               mcsdp_result *results) {
  if (count < 0 || (count > 0 && !ctxs)) return MCSDP_ERR_ARG;
  if (count == 0) return MCSDP_OK;
  std::vector<mcsdp_status> st(count, MCSDP_OK);
  auto run = [&](int i) {
    mcsdp_ctx *c = ctxs[i];
    mcsdp_result r{};
    if (!c) {
      st[i] = MCSDP_ERR_ARG;
    } else {
      if (!c->host_only) cudaSetDevice(c->device);
      st[i] = mcsdp_solve(c, &r);
    }
    if (results) results[i] = r;
  };
  // the largest problem first, alone: it sets every kernel's shared-memory attribute to the
  // largest value any of the others needs
  int big = 0;
  size_t bigsz = 0;
  for (int i = 0; i < count; ++i)
    if (ctxs[i] && ctxs[i]->ws_bytes >= bigsz) {
      bigsz = ctxs[i]->ws_bytes;
      big = i;
    }
  run(big);
  std::atomic<int> next{0};
  const int nt = nthreads > 0 ? nthreads : std::min(count, 16);
  auto worker = [&]() {
    for (;;) {
      const int i = next.fetch_add(1);
      if (i >= count) break;
      if (i != big) run(i);
    }
  };
  std::vector<std::thread> pool;
  for (int t = 0; t < nt; ++t) pool.emplace_back(worker);
  for (auto &t : pool) t.join();
  for (int i = 0; i < count; ++i)
    if (st[i] != MCSDP_OK) return st[i];
  return MCSDP_OK;
}

mcsdp_status mcsdp_stats_get(const mcsdp_ctx *c, mcsdp_stats *st) {
  if (!c || !st) return MCSDP_ERR_ARG;
  std::memset(st, 0, sizeof(*st));
  st->launches = c->launches;
  for (int i = 0; i < 16; ++i) {
    st->count[i] = c->kcount[i];
    st->ms[i] = c->kms[i];
  }
  return MCSDP_OK;
}

mcsdp_status mcsdp_work_model(const mcsdp_ctx *c, mcsdp_work *w) {
  if (!c || !w) return MCSDP_ERR_ARG;
  std::memset(w, 0, sizeof(*w));
  const Symbolic &S = c->S;
  const int ns = S.ns;
  auto nrow_of = [&](int s) { return (double)(S.sn_rowptr[s + 1] - S.sn_rowptr[s]); };
  auto ncol_of = [&](int s) { return (double)(S.sn_col[s + 1] - S.sn_col[s]); };
  // stored lower entries of a supernode = multiply-adds of one triangular pass, one RHS
  std::vector<double> ent(ns);
  double nnzE = 0;
  for (int s = 0; s < ns; ++s) {
    const double k = ncol_of(s), r = nrow_of(s);
    ent[s] = k * (k + 1) / 2 + (r - k) * k;
    nnzE += ent[s];
  }
  // path entries from column j upward (forward solve with e_j)
  auto path_entries = [&](int j) {
    int s = S.col2sn[j];
    const double k = ncol_of(s), r = nrow_of(s);
    const double lc = j - S.sn_col[s];
    double e = 0;
    for (double cc = lc; cc < k; cc += 1) e += r - cc;
    for (s = S.sn_parent[s]; s >= 0; s = S.sn_parent[s]) e += ent[s];
    return e;
  };
  // K2: supernodal Cholesky
  double fy = 0;
  for (int s = 0; s < ns; ++s) {
    const double k = ncol_of(s), r = nrow_of(s);
    fy += k * k * k / 3 + (r - k) * k * k;
  }
  for (int t = 0; t < ns; ++t)
    for (int u = S.upd_ptr[t]; u < S.upd_ptr[t + 1]; ++u) {
      const int src = S.upd_src[u];
      const double na = nrow_of(src) - S.upd_p1[u], nb = S.upd_p2[u] - S.upd_p1[u];
      fy += 2 * ncol_of(src) * (na * nb - nb * (nb - 1) / 2);
    }
  w->flops[0] = fy;
  w->bytes[0] = 8 * (2 * nnzE);
  // K1: per clique Cholesky (k^3/3) + triangular inverse (k^3/3)
  double f1 = 0, b1 = 0;
  for (int s = 0; s < ns; ++s) {
    const double k = nrow_of(s);
    f1 += 2 * k * k * k / 3;
  }
  b1 = 8 * 2 * nnzE;
  w->flops[1] = f1;
  w->bytes[1] = b1;
  // K3 panels: 2 |P_g| right-hand sides per group, forward along each column's own path,
  // backward over the supernodes needed by the rows of P_h, h >= g
  // (a block-diagonal B: the tiles, factorisations and substitutions of each diagonal block)
  const int nblk = c->blocks ? S.ncomp : 1;
  std::vector<int> gend(S.ngroup, S.ngroup);  // first group after g's block
  for (int g = S.ngroup - 1; g >= 0; --g)
    if (c->blocks && g + 1 < S.ngroup && S.grp_comp[g + 1] == S.grp_comp[g]) gend[g] = gend[g + 1];
    else if (c->blocks) gend[g] = g + 1;
  double fp = 0, bp = 0;
  for (int g = 0; g < S.ngroup; ++g) {
    double need = 0;
    for (int64_t t = S.need_ptr[g]; t < S.need_ptr[g + 1]; ++t) need += ent[S.need_sn[t]];
    for (int p = S.grp_pptr[g]; p < S.grp_pptr[g + 1]; ++p) fp += 2 * 2 * (path_entries(S.grp_cols[p]) + need);
    bp += 8.0 * 2 * (S.grp_pptr[gend[g]] - S.grp_pptr[g]) * (S.grp_pptr[g + 1] - S.grp_pptr[g]);
  }
  w->flops[2] = fp;
  w->bytes[2] = bp + 8 * 2 * nnzE;  // panels written once, both factors read once
  // K3 tiles: one multiply-add per pair of nonzeros of (A_i, A_j), i >= j
  double ft = 0, lowB = 0;
  std::vector<double> cnt(S.m);
  for (int i = 0; i < S.m; ++i) cnt[i] = S.anz_ptr[i + 1] - S.anz_ptr[i];
  std::vector<double> suffix(S.m + 1, 0.0);
  for (int i = S.m - 1; i >= 0; --i) suffix[i] = suffix[i + 1] + cnt[i];
  double f4 = 0, b4 = 0, f5 = 0;
  for (int q = 0; q < nblk; ++q) {
    const int o = c->blocks ? S.comp_cptr[q] : 0, e = c->blocks ? S.comp_cptr[q + 1] : S.m;
    for (int j = o; j < e; ++j) ft += 2 * cnt[j] * (suffix[j] - suffix[e]);
    // K4: dense Cholesky with the bordered right-hand side; K5: back substitution
    const double mc = e - o;
    lowB += mc * (mc + 1) / 2;
    f4 += mc * mc * mc / 3 + mc * mc;
    b4 += 8 * 2 * (mc * (mc + 1) / 2);
    f5 += mc * mc;
  }
  w->flops[3] = ft;
  w->bytes[3] = bp + 8.0 * lowB;  // panels read once, lower(B) written once
  w->flops[4] = f4;
  w->bytes[4] = b4;
  w->flops[5] = f5;
  w->bytes[5] = 8 * lowB;
  // K6: per column: N forward along the path, N backward, dY product, L̂ forward and backward
  double fpm = 0;
  const double arow = (double)S.arow_col.size();
  for (int j = 0; j < S.n; ++j) fpm += 2 * (path_entries(j) + 3 * nnzE);
  fpm += 2 * arow * S.n;
  w->flops[6] = fpm;
  w->bytes[6] = 8 * (2 * nnzE + (double)S.nslot + 4 * nnzE);
  // K7: per clique Cholesky (k^3/3), two triangular solves with k right-hand sides (k^3 each),
  // Householder tridiagonalisation (4k^3/3)
  double fps = 0;
  for (int s = 0; s < ns; ++s) {
    const double k = nrow_of(s);
    fps += (1.0 / 3 + 2.0 + 4.0 / 3) * k * k * k;
  }
  w->flops[7] = fps;
  w->bytes[7] = 8 * 2 * nnzE;
  w->flops[8] = fy;
  w->bytes[8] = 8 * 3 * nnzE;
  if (!c->dense) return MCSDP_OK;
  // dense root R (nR = |R|): the forest's small-clique work plus the root's dense kernels; the
  // dense completion forms X̂ and Y^{-1} whole (n x n, FP64 or FP32)
  const double nR = c->nR, nF = c->nF, n = S.n;
  const int rt = ns - 1;
  double entF = 0;  // stored lower entries of the forest's blocks
  for (int t = 0; t < rt; ++t) entF += ent[t];
  double pathF = 0;  // forest part of the forward paths of the forest's unit columns
  for (int j = 0; j < c->nF; ++j) {
    int t = S.col2sn[j];
    for (double cc = j - S.sn_col[t]; cc < ncol_of(t); cc += 1) pathF += nrow_of(t) - cc;
    for (t = S.sn_parent[t]; t >= 0 && t != rt; t = S.sn_parent[t]) pathF += ent[t];
  }
  // K2: the forest's supernodal Cholesky, the gathered contributions, the root's Cholesky
  double fy2 = 0;
  for (int t = 0; t < rt; ++t) {
    const double k = ncol_of(t), r = nrow_of(t);
    fy2 += k * k * k / 3 + (r - k) * k * k;
    for (int u = S.upd_ptr[t]; u < S.upd_ptr[t + 1]; ++u) {
      const int src = S.upd_src[u];
      const double na = nrow_of(src) - S.upd_p1[u], nb = S.upd_p2[u] - S.upd_p1[u];
      fy2 += 2 * ncol_of(src) * (na * nb - nb * (nb - 1) / 2);
    }
  }
  double gath = 0;
  for (size_t q = 0; q < c->rg_u.size(); ++q) gath += 2 * c->upd_meta[c->rg_u[q]].dncol;
  w->flops[0] = fy2 + gath + nR * nR * nR / 3;
  w->bytes[0] = 8 * (2 * entF + nR * nR);
  // K1: the forest's cliques (Algorithm 1), the root's Cholesky and triangular inverse
  double f12 = 0;
  for (int t = 0; t < rt; ++t) f12 += 2 * nrow_of(t) * nrow_of(t) * nrow_of(t) / 3;
  w->flops[1] = f12 + 2 * nR * nR * nR / 3;
  w->bytes[1] = 8 * (2 * entF + 2 * nR * nR);
  // K3 panels: Y^{-1}_RR (triangular inverse + X^T X, 2 nR^3 / 3), then per factor the backward
  // forest solves of the nR root columns and the forward + backward solves of the nF forest
  // columns; X̂ and Y^{-1} written once
  w->flops[2] = 2 * nR * nR * nR / 3 + 2 * (2 * nR * entF + 2 * (pathF + nF * entF));
  w->bytes[2] = 8 * (2 * n * n + 2 * nnzE);
  // K3 tiles: both dense matrices read once, lower(B) written once
  w->bytes[3] = 8 * (2 * n * n + S.m * (S.m + 1.0) / 2);
  // K6: V = X̂ dY and the forest's row dot products; for the root block U = dY Y^{-1}[:, R],
  // the forest's forward solve with nR right-hand sides, the L_RF product and the GEMM
  // X̂_RR T (2 nR^3)
  double fM = 0;
  for (int t = 0; t < rt; ++t) fM += 2 * 2 * ent[t] * n;
  const double lrf = (double)c->lrf_off.size();
  w->flops[6] = 2 * arow * n + fM + 2 * arow * nR + 2 * nR * entF + 2 * lrf * nR +
                2 * nR * nR * nR;
  w->bytes[6] = 8 * (3 * n * n + 4 * nnzE + 3 * n * nR + 2 * nR * nR);
  // K7: the forest's cliques as above; the root's Lanczos bound, 3 products with nR x nR
  // matrices per step (the step count of the last bound)
  double fps2 = 0;
  for (int t = 0; t < rt; ++t) fps2 += (1.0 / 3 + 2.0 + 4.0 / 3) * nrow_of(t) * nrow_of(t) * nrow_of(t);
  w->flops[7] = fps2 + 2 * 3 * nR * nR * std::max(1, c->lz_steps[0]);
  w->bytes[7] = 8 * (2 * entF + 3 * nR * nR * std::max(1, c->lz_steps[0]));
  // K8: the dual Lanczos bound, one n x n product per step
  w->flops[8] = 2 * n * n * std::max(1, c->lz_steps[1]);
  w->bytes[8] = 8 * n * n * std::max(1, c->lz_steps[1]);
  return MCSDP_OK;
}

mcsdp_status mcsdp_stats_reset(mcsdp_ctx *c) {
  if (!c) return MCSDP_ERR_ARG;
  if (!c->pending.empty() && !c->host_only) {
    cudaStreamSynchronize(c->stream);
    prof_flush(c);
  }
  c->launches = 0;
  for (int i = 0; i < 16; ++i) {
    c->kcount[i] = 0;
    c->kms[i] = 0.0;
  }
  return MCSDP_OK;
}

mcsdp_status mcsdp_backward(mcsdp_ctx *c, const double *gX, const double *gz, double *gC,
                            double *gb, double *gA) {
  mcsdp_status s = ready(c);
  if (s) return s;
  if (c->dense)
    return fail(c, MCSDP_ERR_STATE, "differentiation is not available with a dense root clique");
  if (!c->iterate_set) return fail(c, MCSDP_ERR_STATE, "no iterate: solve (or set an iterate) first");
  const Symbolic &S = c->S;
  const int n = S.n, m = S.m;
  const int64_t nnzL = c->D.nnzL;
  double sc[8];
  // mu of the current iterate
  s = prepare(c, c->Xbar, c->z, sc);
  if (s) return s;
  const double mu = sc[0] / n;
  if (!(mu > 0)) return fail(c, MCSDP_ERR_NUMERIC, "mu is not positive at the iterate");
  // centring: Newton on F(z) = A(mu Y(z)^{-1}) - b, X̄ = mu Y^{-1} on E (the max-det completion of
  // which is mu Y^{-1}); the Jacobian is the SCM at that X̄ and -F = b - mu h
  bool centred = false;
  double prev_res = -1.0;
  int stalled = 0;
  bool full = false;
  for (int it = 0; it < 60 && !centred; ++it) {
    int nl = 0;
    s = phase_pmatrix<double>(c, &nl, nullptr, true);
    if (s) return s;
    CUDA_TRY(c, cudaMemsetAsync(c->Xbar, 0, nnzL * 8, c->stream));
    launch_axpy(nnzL, mu, c->YinvE, c->Xbar, c->stream);
    launch_measures(c->D, c->Xbar, c->Ylay, c->z, nullptr, c->scal, c->stream);
    launch_diag_range(c->D, c->N, c->scal + 8, c->stream);
    KCHECK(c);
    CUDA_TRY(c, cudaMemcpyAsync(sc, c->scal, 8 * 8, cudaMemcpyDeviceToHost, c->stream));
    double piv[2];
    CUDA_TRY(c, cudaMemcpyAsync(piv, c->scal + 8, 2 * 8, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    prof_flush(c);
    // done at 1e-13 relative; or once Newton stops gaining (three full steps in a row that do
    // not halve the residual) at the rounding level of the residual's evaluation, rho =
    // 64 eps cond(Y), cond(Y) estimated from below by the pivot range (max_j N_jj / min_j N_jj)^2
    // (X = mu Y^{-1} is formed with relative error about eps cond(Y); near the optimum cond(Y)
    // grows like 1/mu)
    const double res = sc[3] / std::max(1.0, sc[4]);
    const bool slow = prev_res >= 0 && full && res > 0.5 * prev_res;
    stalled = slow ? stalled + 1 : 0;
    const double cnd = piv[1] > 0 ? (piv[0] / piv[1]) * (piv[0] / piv[1]) : 1e300;
    const double rho = 64.0 * 2.220446049250313e-16 * cnd;
    if (c->opt.verbose > 1)
      std::fprintf(stderr, "  centring %d: residual %.3e (rounding level %.1e, full step %d)\n", it,
                   res, rho, full ? 1 : 0);
    if (res <= 1e-13 || (stalled >= 3 && res <= rho)) {
      centred = true;
      break;
    }
    prev_res = res;
    s = factor_X(c, c->Xbar);
    if (s) return s;
    s = phase_scm<double>(c);
    if (s) return s;
    launch_rhs_border(c->D, c->B, c->ldb, c->hvec, mu, c->stream);
    scm_chol_solve(c);
    launch_dz_to_user(c->D, c->xs, c->dz, c->stream);
    CUDA_TRY(c, cudaMemcpyAsync(c->zsave, c->z, (size_t)m * 8, cudaMemcpyDeviceToDevice, c->stream));
    double t = 1.0;
    for (int h = 0;; ++h) {
      CUDA_TRY(c, cudaMemcpyAsync(c->z, c->zsave, (size_t)m * 8, cudaMemcpyDeviceToDevice, c->stream));
      launch_axpy(m, t, c->dz, c->z, c->stream);
      CUDA_TRY(c, cudaMemsetAsync(c->status, 0, 4 * sizeof(int), c->stream));
      s = phase_Y(c, c->z);
      if (s) return s;
      s = phase_ychol(c, 1, nullptr, c->Ylay, nullptr, c->N, c->dinvN, c->status);
      if (s) return s;
      int st[4];
      s = read_status(c, st, 4);
      if (s) return s;
      if (st[2] & ST_TIMEOUT) return fail(c, MCSDP_ERR_TIMEOUT, "SCM factorisation: a bounded wait gave up");
  if (st[2] & ST_NOT_PD) return fail(c, MCSDP_ERR_NOT_PD, "Schur complement matrix is not positive definite");
      if (!(st[0] & ST_NOT_PD)) break;
      t *= 0.5;
      if (h > 40) return fail(c, MCSDP_ERR_STALL, "centring step collapsed");
    }
    full = t == 1.0;
  }
  if (!centred) return fail(c, MCSDP_ERR_STALL, "centring did not converge");
  // at the central point: L̂ (Algorithm 1 on X̄ = mu Y^{-1} on E) and the SCM
  s = factor_X(c, c->Xbar);
  if (s) return s;
  s = phase_scm<double>(c);
  if (s) return s;
  // G (symmetric) from the layout weights of the loss on X̄; R = sym(X̂ G Y^{-1}) on E
  double *G = c->dX;
  if (gX) launch_layout_sym(c->D, gX, G, c->stream);
  else CUDA_TRY(c, cudaMemsetAsync(G, 0, nnzL * 8, c->stream));
  int nl = 0;
  s = phase_pmatrix<double>(c, &nl, G);
  if (s) return s;
  launch_sym_combine(c->D, c->Mlow, c->Mup, c->bwd_g, c->stream);  // R
  // v = B^{-1} (A(R) + g_z)
  launch_con_apply(c->D, c->bwd_g, gz, c->vrhs, c->stream);
  launch_border_from_user(c->D, c->B, c->ldb, c->vrhs, c->stream);
  scm_chol_solve(c);
  launch_dz_to_user(c->D, c->xs, c->dz, c->stream);  // v, caller order
  // g_{A_0} = sym(X̂ (A^*(v) - G) Y^{-1}) on E
  CUDA_TRY(c, cudaMemsetAsync(c->dY, 0, nnzL * 8, c->stream));
  launch_slot_combine(c->D, c->dY, c->dz, 0.0, 1.0, c->stream);
  launch_axpy(nnzL, -1.0, G, c->dY, c->stream);
  s = phase_pmatrix<double>(c, &nl, c->dY);
  if (s) return s;
  launch_sym_combine(c->D, c->Mlow, c->Mup, c->bwd_g, c->stream);
  if (gb) CUDA_TRY(c, cudaMemcpyAsync(gb, c->dz, (size_t)m * 8, cudaMemcpyDeviceToDevice, c->stream));
  launch_entry_grads((int64_t)c->ent_k.size(), c->ent_off_dev, c->ent_k_dev, c->ent_pos_dev,
                     c->ent_f_dev, c->bwd_g, c->Xbar, c->z, c->dz, gC, gA, c->stream);
  KCHECK(c);
  int st[4];
  s = read_status(c, st, 4);
  if (s) return s;
  if (st[2] & ST_TIMEOUT) return fail(c, MCSDP_ERR_TIMEOUT, "SCM factorisation: a bounded wait gave up");
  if (st[2] & ST_NOT_PD) return fail(c, MCSDP_ERR_NOT_PD, "Schur complement matrix is not positive definite");
  return MCSDP_OK;
}

// ---- tile-shape tuner (batched form) ----
static const int TUNE_CAND[5][2] = {{64, 80}, {32, 80}, {16, 80}, {64, 96}, {32, 48}};
static std::mutex g_tune_mu;
static std::map<std::array<int64_t, 3>, std::array<int, 2>> g_tune_cache;

static int64_t tune_pow2(int64_t v) {
  int64_t p = 1;
  while (p < v) p <<= 1;
  return p;
}

mcsdp_status mcsdp_tune_workspace_size(const mcsdp_problem *prob, const mcsdp_options *opt,
                                       size_t *bytes) {
  if (!prob || !bytes) return MCSDP_ERR_ARG;
  mcsdp_options o;
  if (opt) o = *opt;
  else mcsdp_default_options(&o);
  o.device = -1;
  size_t need = 0;
  bool any = false;
  for (const auto &cand : TUNE_CAND) {
    o.group_max = cand[0];
    o.panel_max = cand[1];
    mcsdp_ctx *c = nullptr;
    if (mcsdp_create(prob, &o, nullptr, &c) == MCSDP_OK) {
      need = std::max(need, c->ws_bytes);
      any = true;
    }
    mcsdp_destroy(c);
  }
  if (!any) return MCSDP_ERR_ARG;
  *bytes = need;
  return MCSDP_OK;
}

mcsdp_status mcsdp_tune(const mcsdp_problem *prob, mcsdp_options *opt, const double *z0_dev,
                        void *cuda_stream, void *ws, size_t ws_bytes, int32_t iters,
                        mcsdp_tune_info *info) {
  if (!prob || !opt || !ws || iters <= 0 || opt->device < 0) return MCSDP_ERR_ARG;
  mcsdp_tune_info inf{};
  for (double &v : inf.ms_per_iter) v = -1.0;
  {  // the key: the clique structure does not depend on the SCM grouping
    mcsdp_options o = *opt;
    o.device = -1;
    o.group_max = 64;
    o.panel_max = 96;
    mcsdp_ctx *c = nullptr;
    const mcsdp_status s = mcsdp_create(prob, &o, nullptr, &c);
    if (s == MCSDP_OK) {
      inf.key[0] = tune_pow2(prob->n);
      inf.key[1] = tune_pow2(prob->m);
      inf.key[2] = tune_pow2(c->S.max_nrow);
    }
    mcsdp_destroy(c);
    if (s != MCSDP_OK) return s;
  }
  const std::array<int64_t, 3> key{inf.key[0], inf.key[1], inf.key[2]};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      opt->group_max = inf.group_max = it->second[0];
      opt->panel_max = inf.panel_max = it->second[1];
      inf.cached = 1;
      if (info) *info = inf;
      return MCSDP_OK;
    }
  }
  int best = -1;
  mcsdp_status last = MCSDP_ERR_ARG;
  for (int q = 0; q < 5; ++q) {
    mcsdp_options o = *opt;
    o.group_max = TUNE_CAND[q][0];
    o.panel_max = TUNE_CAND[q][1];
    o.max_iter = iters;
    o.profile = 0;
    o.verbose = 0;
    mcsdp_ctx *c = nullptr;
    double ms = -1.0;
    mcsdp_status s = mcsdp_create(prob, &o, cuda_stream, &c);
    if (s == MCSDP_OK && c->ws_bytes > ws_bytes) s = MCSDP_ERR_OOM;
    if (s == MCSDP_OK) s = mcsdp_set_workspace(c, ws, ws_bytes);
    // one untimed run (first-use work: shared-memory attributes, graph capture), one timed
    for (int rep = 0; rep < 2 && s == MCSDP_OK; ++rep) {
      s = set_default_start(c);
      if (s == MCSDP_OK && z0_dev)
        s = cudaMemcpyAsync(c->z, z0_dev, (size_t)c->S.m * 8, cudaMemcpyDeviceToDevice,
                            c->stream) == cudaSuccess ? MCSDP_OK : MCSDP_ERR_CUDA;
      if (s != MCSDP_OK) break;
      c->iterate_set = true;
      mcsdp_result r{};
      s = mcsdp_solve(c, &r);
      if (s == MCSDP_ERR_MAXITER) s = MCSDP_OK;
      if (s == MCSDP_OK && rep == 1) ms = r.seconds * 1e3 / std::max(1, (int)r.iters);
    }
    if (s != MCSDP_OK) last = s;
    mcsdp_destroy(c);
    inf.ms_per_iter[q] = ms;
    if (ms > 0) {
      ++inf.ncand;
      if (best < 0 || ms < inf.ms_per_iter[best]) best = q;
    }
  }
  if (best < 0) return last;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = {TUNE_CAND[best][0], TUNE_CAND[best][1]};
  }
  opt->group_max = inf.group_max = TUNE_CAND[best][0];
  opt->panel_max = inf.panel_max = TUNE_CAND[best][1];
  if (info) *info = inf;
  return MCSDP_OK;
}

void mcsdp_tune_cache_clear(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache.clear();
}

}  // extern "C"
