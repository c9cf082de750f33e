"""Python binding of libmcsdp: argument marshalling only.  Device memory and streams come from
PyTorch; every step of the method runs in the library's CUDA kernels.  There is no CPU path: if
the library or a GPU is missing the calls raise."""
import ctypes as C

import numpy as np
import torch

from . import _lib
from .build import build as build_library


class MCSDPError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_lib.STATUS.get(status, status)}: {msg}")
        self.status = status


def _ptr(t):
    return C.c_void_p(0) if t is None else C.c_void_p(t.data_ptr())


class Problem:
    """One SDP (paper notation: A_0 objective, A_k constraints, b) bound to a CUDA device.

    mat/row/col/val list the upper triangle (row <= col) of A_0..A_m (mat 0 = A_0) when
    form=1, or of SDPA's F_0..F_m with c = b when form=0."""

    def __init__(self, n, m, b, mat, row, col, val, form=1, device=0, stream=None, **options):
        self._L = _lib.load()
        self._ctx = C.c_void_p()
        self.n, self.m = int(n), int(m)
        self._b = np.ascontiguousarray(b, dtype=np.float64)
        self._mat = np.ascontiguousarray(mat, dtype=np.int32)
        self._row = np.ascontiguousarray(row, dtype=np.int32)
        self._col = np.ascontiguousarray(col, dtype=np.int32)
        self._val = np.ascontiguousarray(val, dtype=np.float64)
        prob = _lib.Problem_t(self.n, self.m, int(form),
                              self._b.ctypes.data_as(C.POINTER(C.c_double)), len(self._val),
                              self._mat.ctypes.data_as(C.POINTER(C.c_int32)),
                              self._row.ctypes.data_as(C.POINTER(C.c_int32)),
                              self._col.ctypes.data_as(C.POINTER(C.c_int32)),
                              self._val.ctypes.data_as(C.POINTER(C.c_double)))
        opt = _lib.Options_t()
        self._L.mcsdp_default_options(C.byref(opt))
        for k, v in options.items():
            setattr(opt, k, v)
        opt.device = int(device)
        self.device = int(device)
        cs = None
        if self.device >= 0:
            self.torch_device = torch.device("cuda", self.device)
            s = stream if stream is not None else torch.cuda.current_stream(self.torch_device)
            self.stream = s
            cs = C.c_void_p(s.cuda_stream)
        st = self._L.mcsdp_create(C.byref(prob), C.byref(opt), cs, C.byref(self._ctx))
        self._check(st)
        self.info = self.sym_info()
        if self.device >= 0:
            nbytes = C.c_size_t()
            self._check(self._L.mcsdp_workspace_size(self._ctx, C.byref(nbytes)))
            self.workspace = torch.empty(max(int(nbytes.value), 256), dtype=torch.uint8,
                                         device=self.torch_device)
            self._check(self._L.mcsdp_set_workspace(self._ctx, _ptr(self.workspace),
                                                    self.workspace.numel()))

    @classmethod
    def from_instance(cls, inst, device=0, **options):
        return cls(inst.n, inst.m, inst.b, inst.mat, inst.row, inst.col, inst.val, form=1,
                   device=device, **options)

    def _check(self, st):
        if st != 0:
            msg = self._L.mcsdp_last_error(self._ctx).decode() if self._ctx else ""
            raise MCSDPError(st, msg)

    def __del__(self):
        try:
            if getattr(self, "_ctx", None) and self._ctx.value:
                self._L.mcsdp_destroy(self._ctx)
                self._ctx = C.c_void_p()
        except Exception:
            pass

    # ---- structure ----
    def sym_info(self):
        info = _lib.SymInfo_t()
        self._check(self._L.mcsdp_sym_info_get(self._ctx, C.byref(info)))
        return {f: getattr(info, f) for f, _ in info._fields_}

    def sym_export(self):
        i = self.info
        perm = np.zeros(i["n"], np.int32)
        sn_col = np.zeros(i["nsuper"] + 1, np.int32)
        sn_rowptr = np.zeros(i["nsuper"] + 1, np.int64)
        self._check(self._L.mcsdp_sym_export(self._ctx, None, None, sn_rowptr.ctypes.data_as(C.c_void_p),
                                             None, None, None))
        sn_rows = np.zeros(int(sn_rowptr[-1]), np.int32)
        sn_valptr = np.zeros(i["nsuper"] + 1, np.int64)
        con_order = np.zeros(i["m"], np.int32)
        self._check(self._L.mcsdp_sym_export(
            self._ctx, perm.ctypes.data_as(C.c_void_p), sn_col.ctypes.data_as(C.c_void_p),
            sn_rowptr.ctypes.data_as(C.c_void_p), sn_rows.ctypes.data_as(C.c_void_p),
            sn_valptr.ctypes.data_as(C.c_void_p), con_order.ctypes.data_as(C.c_void_p)))
        return dict(perm=perm, sn_col=sn_col, sn_rowptr=sn_rowptr, sn_rows=sn_rows,
                    sn_valptr=sn_valptr, con_order=con_order)

    def layout_index(self):
        """For every layout value: (row, col) in the caller's indices and a mask of the stored
        lower entries (index bookkeeping only)."""
        s = self.sym_export()
        nnz = int(s["sn_valptr"][-1])
        r_new = np.full(nnz, -1, np.int64)
        c_new = np.full(nnz, -1, np.int64)
        for t in range(len(s["sn_col"]) - 1):
            rows = s["sn_rows"][s["sn_rowptr"][t]:s["sn_rowptr"][t + 1]]
            c0, c1 = s["sn_col"][t], s["sn_col"][t + 1]
            nr = len(rows)
            base = int(s["sn_valptr"][t])
            for lc in range(c1 - c0):
                r_new[base + lc * nr: base + (lc + 1) * nr] = rows
                c_new[base + lc * nr: base + (lc + 1) * nr] = c0 + lc
        valid = r_new >= c_new
        perm = s["perm"].astype(np.int64)
        return perm[np.where(valid, r_new, 0)], perm[np.where(valid, c_new, 0)], valid, s

    # ---- device calls ----
    def _dev(self, a, n):
        if a is None:
            return None
        t = torch.as_tensor(a, dtype=torch.float64, device=self.torch_device).contiguous()
        assert t.numel() == n, (t.numel(), n)
        return t

    def zeros_layout(self):
        return torch.zeros(self.info["nnz_layout"], dtype=torch.float64, device=self.torch_device)

    def set_iterate(self, Xbar_layout=None, z=None):
        X = self._dev(Xbar_layout, self.info["nnz_layout"])
        zz = self._dev(z, self.m)
        self._check(self._L.mcsdp_set_iterate(self._ctx, _ptr(X), _ptr(zz)))

    def get_iterate(self):
        X = self.zeros_layout()
        Y = self.zeros_layout()
        z = torch.zeros(self.m, dtype=torch.float64, device=self.torch_device)
        self._check(self._L.mcsdp_get_iterate(self._ctx, _ptr(X), _ptr(z), _ptr(Y)))
        return X, z, Y

    def solve(self):
        r = _lib.Result_t()
        st = self._L.mcsdp_solve(self._ctx, C.byref(r))
        out = {f: getattr(r, f) for f, _ in r._fields_}
        out["status_name"] = _lib.STATUS.get(st, st)
        if st not in (0, 3):
            self._check(st)
        return out

    def backward(self, gX_layout=None, gz=None):
        """Gradients of l = gX . X̄ (layout) + gz . z at the re-centred central-path point for the
        iterate's mu (mcsdp_backward).  Returns gb (m), gC (entries of matrix 0, input order),
        gA (entries of matrices 1..m, input order) and g_entries (all input entries, input
        order)."""
        n0 = int(np.count_nonzero(self._mat == 0))
        n1 = len(self._mat) - n0
        gX = None if gX_layout is None else self._dev(gX_layout, self.info["nnz_layout"])
        gzz = None if gz is None else self._dev(gz, self.m)
        gb = torch.zeros(self.m, dtype=torch.float64, device=self.torch_device)
        gC = torch.zeros(max(n0, 1), dtype=torch.float64, device=self.torch_device)
        gA = torch.zeros(max(n1, 1), dtype=torch.float64, device=self.torch_device)
        self._check(self._L.mcsdp_backward(self._ctx, _ptr(gX), _ptr(gzz), _ptr(gC), _ptr(gb),
                                           _ptr(gA)))
        gC, gA = gC[:n0], gA[:n1]
        ge = torch.zeros(len(self._mat), dtype=torch.float64, device=self.torch_device)
        sel0 = torch.from_numpy(np.nonzero(self._mat == 0)[0]).to(self.torch_device)
        sel1 = torch.from_numpy(np.nonzero(self._mat != 0)[0]).to(self.torch_device)
        ge[sel0] = gC
        ge[sel1] = gA
        return {"gb": gb, "gC": gC, "gA": gA, "g_entries": ge}

    def scm_assemble(self, Xbar_layout, z, out=None, precision=0):
        X = self._dev(Xbar_layout, self.info["nnz_layout"])
        zz = self._dev(z, self.m)
        B = out if out is not None else torch.zeros(self.m, self.m, dtype=torch.float64,
                                                    device=self.torch_device)
        h = torch.zeros(self.m, dtype=torch.float64, device=self.torch_device)
        # B is filled column-major (lower triangle, i >= j): a row-major torch tensor viewed
        # transposed has that layout
        Bt = B.t()
        assert Bt.stride(0) == 1
        self._check(self._L.mcsdp_scm_assemble(self._ctx, _ptr(X), _ptr(zz), _ptr(B), self.m,
                                               _ptr(h), int(precision)))
        return Bt, h

    def newton_step(self, Xbar_layout, z):
        X = self._dev(Xbar_layout, self.info["nnz_layout"])
        zz = self._dev(z, self.m)
        dz = torch.zeros(self.m, dtype=torch.float64, device=self.torch_device)
        dX = self.zeros_layout()
        dY = self.zeros_layout()
        ap, ad, mu = C.c_double(), C.c_double(), C.c_double()
        self._check(self._L.mcsdp_newton_step(self._ctx, _ptr(X), _ptr(zz), _ptr(dz), _ptr(dX),
                                              _ptr(dY), C.byref(ap), C.byref(ad), C.byref(mu)))
        return dict(dz=dz, dX=dX, dY=dY, alpha_p=ap.value, alpha_d=ad.value, mu=mu.value)

    def stats(self):
        st = _lib.Stats_t()
        self._check(self._L.mcsdp_stats_get(self._ctx, C.byref(st)))
        return dict(launches=st.launches,
                    count={k: st.count[i] for i, k in enumerate(_lib.KCLASS)},
                    ms={k: st.ms[i] for i, k in enumerate(_lib.KCLASS)})

    def work_model(self):
        w = _lib.Work_t()
        self._check(self._L.mcsdp_work_model(self._ctx, C.byref(w)))
        return dict(flops={k: w.flops[i] for i, k in enumerate(_lib.KCLASS)},
                    bytes={k: w.bytes[i] for i, k in enumerate(_lib.KCLASS)})

    def identity_layout(self):
        ro, co, valid, _ = self.layout_index()
        v = np.where(valid & (ro == co), 1.0, 0.0)
        return torch.tensor(v, dtype=torch.float64, device=self.torch_device)

    def stats_reset(self):
        self._check(self._L.mcsdp_stats_reset(self._ctx))

    def factors(self, Xbar_layout, z):
        X = self._dev(Xbar_layout, self.info["nnz_layout"])
        zz = self._dev(z, self.m)
        Lh = self.zeros_layout()
        N = self.zeros_layout()
        self._check(self._L.mcsdp_factors(self._ctx, _ptr(X), _ptr(zz), _ptr(Lh), _ptr(N)))
        return Lh, N


def _problem_t(n, m, b, mat, row, col, val, form):
    """The host arrays (kept alive by the caller through the returned tuple) and Problem_t."""
    arrs = (np.ascontiguousarray(b, dtype=np.float64), np.ascontiguousarray(mat, dtype=np.int32),
            np.ascontiguousarray(row, dtype=np.int32), np.ascontiguousarray(col, dtype=np.int32),
            np.ascontiguousarray(val, dtype=np.float64))
    prob = _lib.Problem_t(int(n), int(m), int(form), arrs[0].ctypes.data_as(C.POINTER(C.c_double)),
                          len(arrs[4]), arrs[1].ctypes.data_as(C.POINTER(C.c_int32)),
                          arrs[2].ctypes.data_as(C.POINTER(C.c_int32)),
                          arrs[3].ctypes.data_as(C.POINTER(C.c_int32)),
                          arrs[4].ctypes.data_as(C.POINTER(C.c_double)))
    return arrs, prob


def tune(inst, z0=None, iters=3, device=0, form=1, **options):
    """mcsdp_tune on an instance (n, m, b, mat, row, col, val): the (group_max, panel_max) the
    library's tile-shape tuner picks, cached by the library per (n, m, largest clique) rounded up
    to powers of two.  Returns (options dict with the choice, info dict).  Marshalling only."""
    L = _lib.load()
    arrs, prob = _problem_t(inst.n, inst.m, inst.b, inst.mat, inst.row, inst.col, inst.val, form)
    opt = _lib.Options_t()
    L.mcsdp_default_options(C.byref(opt))
    for k, v in options.items():
        setattr(opt, k, v)
    opt.device = int(device)
    nb = C.c_size_t()
    st = L.mcsdp_tune_workspace_size(C.byref(prob), C.byref(opt), C.byref(nb))
    if st != 0:
        raise MCSDPError(st, "tune: no candidate fits the problem")
    dev = torch.device("cuda", int(device))
    ws = torch.empty(max(int(nb.value), 256), dtype=torch.uint8, device=dev)
    z = None if z0 is None else torch.as_tensor(z0, dtype=torch.float64, device=dev)
    info = _lib.TuneInfo_t()
    stream = torch.cuda.current_stream(dev).cuda_stream
    st = L.mcsdp_tune(C.byref(prob), C.byref(opt), _ptr(z), C.c_void_p(stream), _ptr(ws),
                      ws.numel(), int(iters), C.byref(info))
    if st != 0:
        raise MCSDPError(st, "tune failed")
    out = dict(options)
    out["group_max"], out["panel_max"] = int(opt.group_max), int(opt.panel_max)
    return out, {"group_max": info.group_max, "panel_max": info.panel_max,
                 "cached": bool(info.cached), "ncand": info.ncand,
                 "ms_per_iter": list(info.ms_per_iter)[:5], "key": list(info.key)}


def tune_cache_clear():
    _lib.load().mcsdp_tune_cache_clear()


def solve_batch(problems, nthreads=0):
    """Solves the problems concurrently (mcsdp_solve_batch): host threads each take the next
    unsolved problem; create each Problem with its own stream (stream=torch.cuda.Stream()) for
    the solves to overlap on the device.  Returns the result dicts in order."""
    if not problems:
        return []
    L = problems[0]._L
    arr = (C.c_void_p * len(problems))(*[p._ctx.value for p in problems])
    res = (_lib.Result_t * len(problems))()
    torch.cuda.synchronize()
    L.mcsdp_solve_batch(arr, len(problems), int(nthreads), res)
    out = []
    for r in res:
        d = {f: getattr(r, f) for f, _ in r._fields_}
        d["status_name"] = _lib.STATUS.get(d["status"], d["status"])
        out.append(d)
    return out


def gemm_tc(A, B, C_out=None, alpha=1.0, beta=0.0):
    """C = alpha A^T B + beta C on the tensor cores (mcsdp_gemm_tc): A (K x M) and B (K x N) FP32
    CUDA tensors whose columns are contiguous (A.t() of a row-major M x K tensor), C (M x N)
    column-major.  Argument marshalling only."""
    L = _lib.load()
    K, M = A.shape
    N = B.shape[1]
    assert A.dtype == torch.float32 and B.dtype == torch.float32 and B.shape[0] == K
    assert A.stride(0) == 1 and B.stride(0) == 1
    if C_out is None:
        C_out = torch.zeros((N, M), dtype=torch.float32, device=A.device).t()
    assert C_out.stride(0) == 1
    nb = C.c_size_t()
    st = L.mcsdp_gemm_tc_work_size(M, N, K, C.byref(nb))
    if st != 0:
        raise MCSDPError(st, "gemm_tc: bad sizes")
    work = torch.empty(int(nb.value), dtype=torch.uint8, device=A.device)
    stream = torch.cuda.current_stream(A.device).cuda_stream
    st = L.mcsdp_gemm_tc(M, N, K, _ptr(A), A.stride(1), _ptr(B), B.stride(1), _ptr(C_out),
                         C_out.stride(1), alpha, beta, _ptr(work), work.numel(), C.c_void_p(stream))
    if st != 0:
        raise MCSDPError(st, "gemm_tc failed")
    return C_out

