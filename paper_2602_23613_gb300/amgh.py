"""Python binding of libamgh (argument marshalling only; every step runs in the library).

Functions carry the names of the C entry points declared in include/amgh.h.  Matrices are passed
as scipy CSR matrices (host) or as (row_ptr, col, val, shape) tuples of CUDA torch tensors
(device); vectors as numpy arrays (host) or torch tensors (host or CUDA).  The library must have
been built (``paper_2602_23613_gb300.build.build()``); there is no fallback.
"""
import ctypes
import os

import numpy as np

from . import build as _build

AMGH_OK, AMGH_ERR_INVALID_ARG, AMGH_ERR_NOT_SPD, AMGH_ERR_NOT_CONVERGED = 0, 1, 2, 3
AMGH_ERR_CUDA, AMGH_ERR_OOM, AMGH_ERR_TIMEOUT, AMGH_ERR_SETUP_STALL, AMGH_ERR_UNSUPPORTED = 4, 5, 6, 7, 8
AMGH_F64, AMGH_F32, AMGH_BF16 = 0, 1, 2
AMGH_INTERP_LOCAL, AMGH_INTERP_LEARNED, AMGH_INTERP_GEOMETRIC, AMGH_INTERP_CONSTRAINED = 0, 1, 2, 3
AMGH_COARSEN_ALGEBRAIC, AMGH_COARSEN_REFINEMENT = 0, 1
KIND = {"schwarz": 0, "l1": 1, "residual": 2, "restrict": 3, "prolong": 4, "coarse": 5, "spmv": 6, "rr": 7}


class amgh_csr(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_int64), ("ncols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("val", ctypes.c_void_p),
                ("on_device", ctypes.c_int)]


class amgh_params(ctypes.Structure):
    _fields_ = [("max_levels", ctypes.c_int), ("coarse_size", ctypes.c_int), ("precision", ctypes.c_int),
                ("interp", ctypes.c_int), ("ring", ctypes.c_int), ("p_max", ctypes.c_int),
                ("theta", ctypes.c_double), ("stall_ratio", ctypes.c_double), ("stream", ctypes.c_void_p),
                ("dense_tail", ctypes.c_int), ("mlp", ctypes.c_void_p), ("rho_ref", ctypes.c_double),
                ("fuse_restrict", ctypes.c_int), ("coarsening", ctypes.c_int), ("mesh_n", ctypes.c_int)]


class amgh_hier_info(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("n", ctypes.c_int64 * 32), ("nnz", ctypes.c_int64 * 32),
                ("nnz_p", ctypes.c_int64 * 32), ("ncolours", ctypes.c_int * 32), ("max_block", ctypes.c_int * 32),
                ("max_patch", ctypes.c_int * 32), ("op_complexity", ctypes.c_double),
                ("grid_complexity", ctypes.c_double), ("setup_host_ms", ctypes.c_double),
                ("setup_device_ms", ctypes.c_double), ("precision", ctypes.c_int * 32),
                ("lanes", ctypes.c_int * 32), ("fused", ctypes.c_int * 32), ("block_kappa", ctypes.c_double * 32),
                ("dense_tail", ctypes.c_int), ("interp_used", ctypes.c_int), ("rho", ctypes.c_double),
                ("rho_exact", ctypes.c_double), ("interp_ms", ctypes.c_double),
                ("fused_rr", ctypes.c_int * 32)]


_LIB = None
EXPORTS = ["amgh_default_params", "amgh_setup", "amgh_batch_setup", "amgh_setup_host_structure", "amgh_vcycle", "amgh_pcg_solve",
           "amgh_batch_pcg_solve", "amgh_pcg_solve_noalloc", "amgh_pcg_solve_multi", "amgh_vcycle_multi",
           "amgh_amg_solve", "amgh_info",
           "amgh_level_structure", "amgh_level_matrix", "amgh_level_apply", "amgh_profile", "amgh_kernel_stats",
           "amgh_launch_count", "amgh_last_error", "amgh_destroy",
           "amgh_mlp_create", "amgh_mlp_set_precision", "amgh_mlp_add_samples", "amgh_mlp_num_samples", "amgh_mlp_train", "amgh_mlp_params",
           "amgh_mlp_loss_grad", "amgh_mlp_predict", "amgh_mlp_features", "amgh_mlp_last_error", "amgh_mlp_destroy",
           "amgh_selftest_wait_timeout"]
_NOT_STATUS = ("amgh_default_params", "amgh_launch_count", "amgh_last_error", "amgh_destroy", "amgh_mlp_num_samples",
               "amgh_mlp_last_error", "amgh_mlp_destroy")


def lib_path():
    return _build.LIB


def load():
    """Load libamgh.so (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError("libamgh.so is not built (%s); run paper_2602_23613_gb300.build.build()" % path)
    L = ctypes.CDLL(path)
    P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    L.amgh_default_params.argtypes = [ctypes.POINTER(amgh_params)]
    L.amgh_default_params.restype = None
    L.amgh_setup.argtypes = [ctypes.POINTER(amgh_csr), ctypes.POINTER(amgh_csr), ctypes.POINTER(amgh_params), ctypes.POINTER(P)]
    L.amgh_setup_host_structure.argtypes = L.amgh_setup.argtypes
    L.amgh_batch_setup.argtypes = [I, ctypes.POINTER(amgh_csr), ctypes.POINTER(amgh_csr), ctypes.POINTER(amgh_params),
                                   ctypes.POINTER(P)]
    L.amgh_vcycle.argtypes = [P, P, P]
    L.amgh_pcg_solve.argtypes = [P, P, P, D, I, ctypes.POINTER(I), ctypes.POINTER(D)]
    L.amgh_amg_solve.argtypes = [P, P, P, D, I, ctypes.POINTER(I), ctypes.POINTER(D)]
    L.amgh_pcg_solve_noalloc.argtypes = [P, P, P, D, I, ctypes.POINTER(I), ctypes.POINTER(D)]
    L.amgh_pcg_solve_multi.argtypes = [P, P, P, I, D, I, ctypes.POINTER(I), ctypes.POINTER(D)]
    L.amgh_vcycle_multi.argtypes = [P, P, P, I]
    L.amgh_batch_pcg_solve.argtypes = [I, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P), D, I,
                                       ctypes.POINTER(I), ctypes.POINTER(D)]
    L.amgh_info.argtypes = [P, ctypes.POINTER(amgh_hier_info)]
    L.amgh_level_structure.argtypes = [P, I] + [ctypes.POINTER(I64)] * 5 + [P] * 6
    L.amgh_level_matrix.argtypes = [P, I, I] + [ctypes.POINTER(I64)] * 3 + [P, P, P]
    L.amgh_level_apply.argtypes = [P, I, I, P, P, P]
    L.amgh_profile.argtypes = [P, I, I, I]
    L.amgh_kernel_stats.argtypes = [P, ctypes.POINTER(I64), ctypes.POINTER(D), ctypes.POINTER(D)]
    L.amgh_launch_count.argtypes = [P]
    L.amgh_launch_count.restype = I64
    L.amgh_last_error.argtypes = [P]
    L.amgh_last_error.restype = ctypes.c_char_p
    L.amgh_destroy.argtypes = [P]
    L.amgh_destroy.restype = None
    U64 = ctypes.c_uint64
    L.amgh_mlp_create.argtypes = [U64, ctypes.POINTER(P)]
    L.amgh_mlp_set_precision.argtypes = [P, I]
    L.amgh_mlp_add_samples.argtypes = [P, P]
    L.amgh_mlp_num_samples.argtypes = [P]
    L.amgh_mlp_num_samples.restype = I64
    L.amgh_mlp_train.argtypes = [P, I, I, D, U64, ctypes.POINTER(D)]
    L.amgh_mlp_params.argtypes = [P, P, P, ctypes.POINTER(I64)]
    L.amgh_mlp_loss_grad.argtypes = [P, P, P, P, I, ctypes.POINTER(D), P]
    L.amgh_mlp_predict.argtypes = [P, P, I64, P]
    L.amgh_mlp_features.argtypes = [P, P, P, P, ctypes.POINTER(I64)]
    L.amgh_mlp_last_error.argtypes = [P]
    L.amgh_mlp_last_error.restype = ctypes.c_char_p
    L.amgh_mlp_destroy.argtypes = [P]
    L.amgh_mlp_destroy.restype = None
    L.amgh_selftest_wait_timeout.argtypes = [ctypes.POINTER(D)]
    for name in EXPORTS:
        if name not in _NOT_STATUS:
            getattr(L, name).restype = I
    _LIB = L
    return L


class AmghError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("amgh status %d: %s" % (status, msg))
        self.status = status


def _check(st, h=None):
    if st != AMGH_OK:
        msg = load().amgh_last_error(h).decode(errors="replace")
        raise AmghError(st, msg)


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _vec_ptr(x, keep):
    """Pointer of a float64 vector (numpy, or torch host/CUDA), contiguous, kept alive in keep."""
    if _is_torch(x):
        import torch
        if x.dtype != torch.float64 or not x.is_contiguous():
            raise TypeError("vectors must be contiguous float64")
        return x.data_ptr()
    a = np.ascontiguousarray(x, dtype=np.float64)
    keep.append(a)
    return a.ctypes.data


def _csr(M, keep):
    c = amgh_csr()
    if isinstance(M, tuple):           # (row_ptr, col, val, (nrows, ncols)) of CUDA torch tensors
        rp, ci, va, shape = M
        c.nrows, c.ncols, c.nnz = shape[0], shape[1], int(ci.numel())
        c.row_ptr, c.col, c.val, c.on_device = rp.data_ptr(), ci.data_ptr(), va.data_ptr(), 1 if rp.is_cuda else 0
        keep.extend([rp, ci, va])
        return c
    import scipy.sparse as sp
    M = sp.csr_matrix(M)
    M.sort_indices()
    rp = np.ascontiguousarray(M.indptr, dtype=np.int32)
    ci = np.ascontiguousarray(M.indices, dtype=np.int32)
    va = np.ascontiguousarray(M.data, dtype=np.float64)
    keep.extend([rp, ci, va])
    c.nrows, c.ncols, c.nnz = M.shape[0], M.shape[1], M.nnz
    c.row_ptr, c.col, c.val, c.on_device = rp.ctypes.data, ci.ctypes.data, va.ctypes.data, 0
    return c


class Handle:
    """Owns an amgh_handle; destroyed with amgh_destroy."""

    def __init__(self, ptr, n):
        self.ptr = ptr
        self.n = n

    def __del__(self):
        if getattr(self, "ptr", None):
            load().amgh_destroy(self.ptr)
            self.ptr = None


def amgh_default_params():
    p = amgh_params()
    load().amgh_default_params(ctypes.byref(p))
    return p


def amgh_setup(A, G, params=None, **kw):
    """Build the hierarchy for (A, G); keyword arguments override fields of amgh_params."""
    L = load()
    p = params if params is not None else amgh_default_params()
    for k, v in kw.items():
        setattr(p, k, v.ptr if isinstance(v, Mlp) else v)
    keep = []
    a, g = _csr(A, keep), _csr(G, keep)
    out = ctypes.c_void_p()
    _check(L.amgh_setup(ctypes.byref(a), ctypes.byref(g), ctypes.byref(p), ctypes.byref(out)))
    return Handle(out.value, a.nrows)


def amgh_batch_setup(As, Gs, params=None, **kw):
    """Set up many systems at once (see include/amgh.h); returns one Handle per system."""
    L = load()
    p = params if params is not None else amgh_default_params()
    for k, v in kw.items():
        setattr(p, k, v.ptr if isinstance(v, Mlp) else v)
    keep = []
    n = len(As)
    arrA = (amgh_csr * n)(*[_csr(A, keep) for A in As])
    arrG = (amgh_csr * n)(*[_csr(G, keep) for G in Gs])
    out = (ctypes.c_void_p * n)()
    _check(L.amgh_batch_setup(n, arrA, arrG, ctypes.byref(p), out))
    return [Handle(out[i], arrA[i].nrows) for i in range(n)]


def amgh_setup_host_structure(A, G, params=None, **kw):
    """Level-0 graph steps on the host only (no GPU needed); see include/amgh.h."""
    L = load()
    p = params if params is not None else amgh_default_params()
    for k, v in kw.items():
        setattr(p, k, v)
    keep = []
    a, g = _csr(A, keep), _csr(G, keep)
    out = ctypes.c_void_p()
    _check(L.amgh_setup_host_structure(ctypes.byref(a), ctypes.byref(g), ctypes.byref(p), ctypes.byref(out)))
    return Handle(out.value, a.nrows)


def amgh_vcycle(h, r, z):
    keep = []
    _check(load().amgh_vcycle(h.ptr, _vec_ptr(r, keep), _z_ptr(z)), h.ptr)


def _z_ptr(z):
    if _is_torch(z):
        import torch
        if z.dtype != torch.float64 or not z.is_contiguous():
            raise TypeError("output vectors must be contiguous float64")
        return z.data_ptr()
    if not (isinstance(z, np.ndarray) and z.dtype == np.float64 and z.flags.c_contiguous and z.flags.writeable):
        raise TypeError("output vectors must be writeable contiguous float64 arrays")
    return z.ctypes.data


def _solve(fn, h, f, x, tol, maxit):
    keep = []
    it = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    st = fn(h.ptr, _vec_ptr(f, keep), _z_ptr(x), tol, maxit, ctypes.byref(it), ctypes.byref(rel))
    if st not in (AMGH_OK, AMGH_ERR_NOT_CONVERGED):
        _check(st, h.ptr)
    return it.value, rel.value, st == AMGH_OK


def amgh_pcg_solve(h, f, x, tol=1e-8, maxit=500):
    """PCG with the V-cycle; x holds x0 on entry.  Returns (iterations, relres, converged)."""
    return _solve(load().amgh_pcg_solve, h, f, x, tol, maxit)


def amgh_batch_pcg_solve(hs, fs, xs, tol=1e-8, maxit=500):
    """All systems in one graph launch (CUDA tensors).  Returns (iterations, relres, converged) lists."""
    n = len(hs)
    P = ctypes.c_void_p
    ha = (P * n)(*[h.ptr for h in hs])
    fa = (P * n)(*[f.data_ptr() for f in fs])
    xa = (P * n)(*[x.data_ptr() for x in xs])
    it = (ctypes.c_int * n)()
    rel = (ctypes.c_double * n)()
    st = load().amgh_batch_pcg_solve(n, ha, fa, xa, tol, maxit, it, rel)
    if st not in (AMGH_OK, AMGH_ERR_NOT_CONVERGED):
        _check(st, hs[0].ptr)
    return list(it), list(rel), st == AMGH_OK


def amgh_pcg_solve_noalloc(h, f, x, tol=1e-8, maxit=500):
    """PCG that allocates nothing (Krylov buffers in the library's fixed device array); CUDA
    tensors only, at most 262144 rows.  Returns (iterations, relres, converged)."""
    return _solve(load().amgh_pcg_solve_noalloc, h, f, x, tol, maxit)


def amgh_pcg_solve_multi(h, F, X, tol=1e-8, maxit=500):
    """k right-hand sides: F, X are (k, n) float64 arrays/tensors (row c = right-hand side c, i.e.
    n x k column-major).  Returns (iterations[k], relres[k], converged)."""
    keep = []
    k = int(F.shape[0])
    it = (ctypes.c_int * k)()
    rel = (ctypes.c_double * k)()
    st = load().amgh_pcg_solve_multi(h.ptr, _vec_ptr(F, keep), _z_ptr(X), k, tol, maxit, it, rel)
    if st not in (AMGH_OK, AMGH_ERR_NOT_CONVERGED):
        _check(st, h.ptr)
    return list(it), list(rel), st == AMGH_OK


def amgh_vcycle_multi(h, R, Z):
    """Z = B R for (k, n) CUDA tensors."""
    _check(load().amgh_vcycle_multi(h.ptr, R.data_ptr(), Z.data_ptr(), int(R.shape[0])), h.ptr)


def amgh_amg_solve(h, f, x, tol=1e-8, maxit=500):
    """Stand-alone V-cycle iteration.  Returns (iterations, relres, converged)."""
    return _solve(load().amgh_amg_solve, h, f, x, tol, maxit)


def amgh_info(h):
    info = amgh_hier_info()
    _check(load().amgh_info(h.ptr, ctypes.byref(info)), h.ptr)
    L = info.levels
    return dict(levels=L, n=list(info.n[:L]), nnz=list(info.nnz[:L]), nnz_p=list(info.nnz_p[:L]),
                ncolours=list(info.ncolours[:L]), max_block=list(info.max_block[:L]),
                max_patch=list(info.max_patch[:L]), op_complexity=info.op_complexity,
                grid_complexity=info.grid_complexity, setup_host_ms=info.setup_host_ms,
                setup_device_ms=info.setup_device_ms, precision=list(info.precision[:L]),
                lanes=list(info.lanes[:L]), fused=list(info.fused[:L]), block_kappa=list(info.block_kappa[:L]),
                dense_tail=info.dense_tail, interp_used=info.interp_used, rho=info.rho, rho_exact=info.rho_exact,
                interp_ms=info.interp_ms, fused_rr=list(info.fused_rr[:L]))


def amgh_level_structure(h, l):
    """Structural outputs of level l as numpy arrays (see include/amgh.h)."""
    Lb = load()
    cnt = [ctypes.c_int64(0) for _ in range(5)]
    nul = [None] * 6
    _check(Lb.amgh_level_structure(h.ptr, l, *[ctypes.byref(c) for c in cnt], *nul), h.ptr)
    nna, ne, ncn, pnz, ns = [c.value for c in cnt]
    cf = np.zeros(nna, np.int8)
    edges = np.zeros((ne, 7), np.int32)
    cnodes = np.zeros(ncn, np.int32)
    pptr = np.zeros(ne + 1, np.int32)
    pidx = np.zeros(pnz, np.int32)
    col = np.zeros(ns, np.int32)
    _check(Lb.amgh_level_structure(h.ptr, l, *[ctypes.byref(c) for c in cnt], cf.ctypes.data, edges.ctypes.data,
                                   cnodes.ctypes.data, pptr.ctypes.data, pidx.ctypes.data, col.ctypes.data), h.ptr)
    return dict(cf_state=cf, edges=edges, coarse_nodes=cnodes, patch_ptr=pptr, patch_idx=pidx, colour=col)


def amgh_level_matrix(h, l, which):
    """Level matrix as scipy CSR: which = 0 A_l, 1 P_l, 2 G_l, 3 P_l^T A_l P_l (symbolic pattern),
    4 the nodal interpolation of the commuting correction (interp CONSTRAINED)."""
    import scipy.sparse as sp
    Lb = load()
    nr, nc, nz = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
    _check(Lb.amgh_level_matrix(h.ptr, l, which, ctypes.byref(nr), ctypes.byref(nc), ctypes.byref(nz),
                                None, None, None), h.ptr)
    rp = np.zeros(nr.value + 1, np.int32)
    ci = np.zeros(nz.value, np.int32)
    va = np.zeros(nz.value, np.float64)
    _check(Lb.amgh_level_matrix(h.ptr, l, which, ctypes.byref(nr), ctypes.byref(nc), ctypes.byref(nz),
                                rp.ctypes.data, ci.ctypes.data, va.ctypes.data), h.ptr)
    return sp.csr_matrix((va, ci, rp), shape=(nr.value, nc.value))


def amgh_level_apply(h, l, op, f, x, y):
    """One V-cycle step on level l with CUDA float64 tensors (see include/amgh.h for op)."""
    _check(load().amgh_level_apply(h.ptr, l, op, f.data_ptr() if f is not None else None, x.data_ptr(),
                                   y.data_ptr()), h.ptr)


def amgh_profile(h, enable, kind="schwarz", level=0):
    _check(load().amgh_profile(h.ptr, int(enable), KIND.get(kind, kind), level), h.ptr)


def amgh_kernel_stats(h):
    n, ms, by = ctypes.c_int64(0), ctypes.c_double(0), ctypes.c_double(0)
    _check(load().amgh_kernel_stats(h.ptr, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by)), h.ptr)
    return dict(launches=n.value, total_ms=ms.value, algorithmic_bytes=by.value)


def amgh_launch_count(h):
    return int(load().amgh_launch_count(h.ptr))


def amgh_selftest_wait_timeout():
    """Run the bounded-wait self-test; returns (status, seconds).  AMGH_ERR_TIMEOUT is the pass."""
    sec = ctypes.c_double(0.0)
    st = load().amgh_selftest_wait_timeout(ctypes.byref(sec))
    return st, sec.value


def amgh_last_error(h=None):
    return load().amgh_last_error(h.ptr if h is not None else None).decode(errors="replace")


def amgh_destroy(h):
    if h.ptr:
        load().amgh_destroy(h.ptr)
        h.ptr = None


# ---- learned interpolation weights ----------------------------------------------------------------
MLP_SLOTS, MLP_DIN = 64, 3 * 64 + 2


class Mlp:
    """Owns an amgh_mlp; destroyed with amgh_mlp_destroy."""

    def __init__(self, ptr):
        self.ptr = ptr

    def __del__(self):
        if getattr(self, "ptr", None):
            load().amgh_mlp_destroy(self.ptr)
            self.ptr = None


def _mcheck(st, m):
    if st != AMGH_OK:
        raise AmghError(st, load().amgh_mlp_last_error(m.ptr if m is not None else None).decode(errors="replace"))


def _f32(x):
    return np.ascontiguousarray(x, dtype=np.float32)


def amgh_mlp_create(seed=0):
    out = ctypes.c_void_p()
    _mcheck(load().amgh_mlp_create(seed, ctypes.byref(out)), None)
    return Mlp(out.value)


def amgh_mlp_set_precision(m, precision):
    """AMGH_F32 or AMGH_BF16 storage of the network's products (see include/amgh.h)."""
    _mcheck(load().amgh_mlp_set_precision(m.ptr, precision), m)


def amgh_mlp_add_samples(m, h):
    _mcheck(load().amgh_mlp_add_samples(m.ptr, h.ptr), m)


def amgh_mlp_num_samples(m):
    return int(load().amgh_mlp_num_samples(m.ptr))


def amgh_mlp_train(m, epochs, batch=256, lr=1e-3, seed=0):
    L = ctypes.c_double(0)
    _mcheck(load().amgh_mlp_train(m.ptr, epochs, batch, lr, seed, ctypes.byref(L)), m)
    return L.value


def amgh_mlp_params(m, new=None):
    """Current parameters (W1, b1, W2, b2, W3, b3 flattened, FP32); loads `new` first if given."""
    Lb = load()
    n = ctypes.c_int64(0)
    _mcheck(Lb.amgh_mlp_params(m.ptr, None, None, ctypes.byref(n)), m)
    out = np.zeros(n.value, np.float32)
    src = None
    if new is not None:
        src = _f32(new)
        if src.size != n.value:
            raise ValueError("expected %d parameters" % n.value)
    _mcheck(Lb.amgh_mlp_params(m.ptr, out.ctypes.data, src.ctypes.data if src is not None else None,
                               ctypes.byref(n)), m)
    return out


def amgh_mlp_loss_grad(m, X, T, M):
    X, T, M = _f32(X), _f32(T), _f32(M)
    n = ctypes.c_int64(0)
    load().amgh_mlp_params(m.ptr, None, None, ctypes.byref(n))
    g = np.zeros(n.value, np.float32)
    L = ctypes.c_double(0)
    _mcheck(load().amgh_mlp_loss_grad(m.ptr, X.ctypes.data, T.ctypes.data, M.ctypes.data, X.shape[0],
                                      ctypes.byref(L), g.ctypes.data), m)
    return L.value, g


def amgh_mlp_predict(m, X):
    X = _f32(X)
    Y = np.zeros((X.shape[0], MLP_SLOTS), np.float32)
    _mcheck(load().amgh_mlp_predict(m.ptr, X.ctypes.data, X.shape[0], Y.ctypes.data), m)
    return Y


def amgh_mlp_features(h):
    """Finest-level (features, exact targets, masks) of a hierarchy as numpy FP32 arrays."""
    Lb = load()
    n = ctypes.c_int64(0)
    _check(Lb.amgh_mlp_features(h.ptr, None, None, None, ctypes.byref(n)), h.ptr)
    X = np.zeros((n.value, MLP_DIN), np.float32)
    T = np.zeros((n.value, MLP_SLOTS), np.float32)
    M = np.zeros((n.value, MLP_SLOTS), np.float32)
    _check(Lb.amgh_mlp_features(h.ptr, X.ctypes.data, T.ctypes.data, M.ctypes.data, ctypes.byref(n)), h.ptr)
    return X, T, M


def amgh_mlp_destroy(m):
    if m.ptr:
        load().amgh_mlp_destroy(m.ptr)
        m.ptr = None
