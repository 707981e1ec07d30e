"""ctypes binding of the C ABI declared in include/snmf.h.

Argument marshalling only: every step of the solver runs in the library's CUDA
kernels.  PyTorch provides device memory and streams.  There is no CPU fallback:
loading fails loudly when the compiled library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libsnmf_gb300.so")

SNMF_OK, SNMF_NOT_CONVERGED = 0, 1
SNMF_ERR_ARG, SNMF_ERR_CUDA, SNMF_ERR_OOM, SNMF_ERR_NUMERIC, SNMF_ERR_TIMEOUT, SNMF_ERR_STATE = -1, -2, -3, -4, -5, -6
SNMF_DENSE, SNMF_CSR, SNMF_DENSE_BATCH = 0, 1, 2
SNMF_F64, SNMF_F32, SNMF_BF16, SNMF_FP8 = 0, 1, 2, 3
SNMF_ON_DEVICE, SNMF_ON_HOST = 0, 1
SNMF_PENALTY, SNMF_DIRECT, SNMF_NAIVE = 0, 1, 2
SNMF_BB1, SNMF_BB2 = 0, 1
SNMF_MLP_IN, SNMF_MLP_HIDDEN = 5, 64
SNMF_MLP_NPARAMS = SNMF_MLP_IN * SNMF_MLP_HIDDEN + 2 * SNMF_MLP_HIDDEN + 1

EXPORTED = (
    "snmf_default_options", "snmf_create", "snmf_set_graph_reg", "snmf_lai_sketch",
    "snmf_solve", "snmf_solve_host", "snmf_restart_stats", "snmf_get_factors",
    "snmf_apply", "snmf_profile_ax", "snmf_apply_dense_noalloc", "snmf_controller_data",
    "snmf_mlp_train", "snmf_tuned_config", "snmf_tuned_tiles", "snmf_profile_steps", "snmf_destroy", "snmf_last_error",
    "snmf_mlp_eval", "snmf_set_timeout", "snmf_step_config", "snmf_svd_init",
    "snmf_get_state", "snmf_set_state", "snmf_stats_ring",
    "snmf_knn_graph", "snmf_cluster_assign", "snmf_cluster_scores",
)
SNMF_RING_VALUES = 8
NOALLOC_SCRATCH_BYTES = 64 << 20
NOALLOC_PARTIAL_BYTES = 4 << 20
NOALLOC_MAX_SLICE_PAIR_BYTES = NOALLOC_SCRATCH_BYTES - NOALLOC_PARTIAL_BYTES
NOALLOC_MAX_ROWS = 64 * ((NOALLOC_PARTIAL_BYTES - 256) // 256)


class snmf_matrix(C.Structure):
    _fields_ = [("kind", C.c_int32), ("dtype", C.c_int32), ("location", C.c_int32),
                ("reserved", C.c_int32), ("n", C.c_int64), ("nnz", C.c_int64), ("ld", C.c_int64),
                ("values", C.c_void_p), ("rowptr", C.c_void_p), ("colidx", C.c_void_p),
                ("nprob", C.c_int32), ("reserved2", C.c_int32), ("batch_desc", C.c_void_p)]


class snmf_options(C.Structure):
    _fields_ = [("formulation", C.c_int32), ("precision", C.c_int32), ("batch", C.c_int32),
                ("nonmonotone_M", C.c_int32), ("bb_variant", C.c_int32), ("max_ls", C.c_int32),
                ("inner_iters", C.c_int32), ("max_iter", C.c_int32), ("power_iters", C.c_int32),
                ("step_controller", C.c_int32), ("lambda_sym", C.c_double), ("theta", C.c_double),
                ("phi", C.c_double), ("eta", C.c_double), ("alpha_min", C.c_double),
                ("alpha_max", C.c_double), ("beta_shrink", C.c_double), ("tol", C.c_double),
                ("direct_rho_factor", C.c_double), ("init_scale", C.c_double), ("seed", C.c_uint64),
                ("mlp_weights", C.c_void_p), ("timeout_cycles", C.c_int64),
                ("autotune", C.c_int32), ("x_parts", C.c_int32), ("tune_cache", C.c_char_p),
                ("sym_half", C.c_int32), ("branch_step", C.c_int32)]


class snmf_stats(C.Structure):
    _fields_ = [("iters", C.c_int32), ("converged", C.c_int32), ("ls_fail", C.c_int32),
                ("clipped_steps", C.c_int32), ("best_restart", C.c_int32), ("ax_products", C.c_int32),
                ("f", C.c_double), ("residual", C.c_double), ("pg_rel", C.c_double),
                ("seconds", C.c_double), ("kernel_launches", C.c_int64), ("graph_replays", C.c_int32),
                ("ctl_proposals", C.c_int32), ("ctl_accepted", C.c_int32), ("reserved", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
# Inputs a handle borrows (a device A in the working precision must outlive the handle): held
# here from snmf_create until snmf_destroy, so a caller's temporary cannot be freed under it.
_BORROWED = {}


def load_library(path: str = LIB_PATH):
    """Load the compiled library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"SNMPBB CUDA library not built ({path}); run __graft_entry__.build()")
    lib = C.CDLL(path)
    H = C.c_void_p
    lib.snmf_default_options.argtypes = [C.POINTER(snmf_options)]
    lib.snmf_default_options.restype = None
    lib.snmf_create.argtypes = [C.POINTER(H), C.POINTER(snmf_matrix), C.c_int, C.POINTER(snmf_options), C.c_void_p]
    lib.snmf_set_graph_reg.argtypes = [H, C.POINTER(snmf_matrix), C.c_double]
    lib.snmf_lai_sketch.argtypes = [H, C.c_int, C.c_int, C.c_int, C.c_uint64]
    lib.snmf_solve.argtypes = [H, C.c_void_p, C.c_void_p, C.POINTER(snmf_stats)]
    lib.snmf_solve_host.argtypes = [H, C.c_void_p, C.c_void_p, C.POINTER(snmf_stats)]
    lib.snmf_restart_stats.argtypes = [H, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.snmf_get_factors.argtypes = [H, C.c_void_p, C.c_void_p]
    lib.snmf_apply.argtypes = [H, C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_double)]
    lib.snmf_profile_ax.argtypes = [H, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    lib.snmf_apply_dense_noalloc.argtypes = [C.c_void_p, C.c_int, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p,
                                             C.c_int, C.POINTER(C.c_double), C.c_void_p]
    lib.snmf_controller_data.argtypes = [H, C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_int32)]
    lib.snmf_mlp_train.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_double,
                                   C.POINTER(C.c_double), C.c_void_p]
    lib.snmf_tuned_config.argtypes = [H, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                      C.POINTER(C.c_double), C.POINTER(C.c_int32)]
    lib.snmf_profile_steps.argtypes = [H, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    lib.snmf_tuned_tiles.argtypes = [H, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    lib.snmf_mlp_eval.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]
    lib.snmf_set_timeout.argtypes = [H, C.c_int64]
    lib.snmf_svd_init.argtypes = [H, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_uint64]
    lib.snmf_get_state.argtypes = [H, C.c_void_p, C.c_int64, C.POINTER(C.c_int64)]
    lib.snmf_set_state.argtypes = [H, C.c_void_p, C.c_int64]
    lib.snmf_stats_ring.argtypes = [H, C.c_void_p, C.c_int, C.POINTER(C.c_int32)]
    lib.snmf_knn_graph.argtypes = [C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_int64), C.c_void_p]
    lib.snmf_cluster_assign.argtypes = [H, C.c_int, C.c_void_p]
    lib.snmf_cluster_scores.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_void_p,
                                        C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_void_p]
    lib.snmf_step_config.argtypes = [H, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int64),
                                     C.POINTER(C.c_int64)]
    lib.snmf_destroy.argtypes = [H]
    lib.snmf_last_error.argtypes = [H]
    lib.snmf_last_error.restype = C.c_char_p
    for name in EXPORTED:
        if name not in ("snmf_default_options", "snmf_last_error"):
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


class SnmfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"snmf status {status}: {msg}")
        self.status = status


def _check(lib, h, st):
    if st < 0:
        raise SnmfError(st, lib.snmf_last_error(h).decode(errors="replace"))
    return st


def snmf_default_options(**overrides) -> snmf_options:
    lib = load_library()
    o = snmf_options()
    lib.snmf_default_options(C.byref(o))
    for k, v in overrides.items():
        if k == "mlp_weights":
            continue
        if k == "tune_cache" and isinstance(v, str):
            v = v.encode()
        setattr(o, k, v)
    return o


def _ptr(t):
    """Data pointer of a torch tensor or numpy array (None -> NULL)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _is_cuda(t):
    return hasattr(t, "is_cuda") and t.is_cuda


def dense_matrix(A) -> tuple:
    """snmf_matrix for a dense n x n torch tensor (device or host) or numpy array."""
    dt = SNMF_F64 if str(A.dtype).endswith("float64") else SNMF_F32
    m = snmf_matrix(kind=SNMF_DENSE, dtype=dt, location=SNMF_ON_DEVICE if _is_cuda(A) else SNMF_ON_HOST,
                    n=A.shape[0], nnz=0, ld=A.shape[1] if A.ndim == 2 else A.shape[0],
                    values=_ptr(A))
    if hasattr(A, "stride") and not isinstance(A, np.ndarray):
        m.ld = A.stride(0)
    return m, (A,)


def csr_matrix(n, rowptr, colidx, values) -> tuple:
    """snmf_matrix for CSR arrays (all torch-on-device or all host numpy/torch)."""
    dt = SNMF_F64 if str(values.dtype).endswith("float64") else SNMF_F32
    m = snmf_matrix(kind=SNMF_CSR, dtype=dt, location=SNMF_ON_DEVICE if _is_cuda(values) else SNMF_ON_HOST,
                    n=n, nnz=int(values.shape[0]), ld=0, values=_ptr(values), rowptr=_ptr(rowptr),
                    colidx=_ptr(colidx))
    return m, (rowptr, colidx, values)


def dense_batch_matrix(values, ns, rs, offsets=None) -> tuple:
    """snmf_matrix of an uneven batch: ``values`` a flat array (device tensor or host) holding
    the n_p x n_p row-major problems back to back (or at ``offsets``), ranks ``rs``."""
    ns = [int(x) for x in ns]
    rs = [int(x) for x in rs]
    if offsets is None:
        offsets = np.concatenate([[0], np.cumsum([n * n for n in ns])[:-1]]).astype(np.int64)
    desc = np.ascontiguousarray(np.stack([np.asarray(ns, np.int64), np.asarray(rs, np.int64),
                                          np.asarray(offsets, np.int64)], 1).reshape(-1))
    dt = SNMF_F64 if str(values.dtype).endswith("float64") else SNMF_F32
    m = snmf_matrix(kind=SNMF_DENSE_BATCH, dtype=dt, location=SNMF_ON_DEVICE if _is_cuda(values) else SNMF_ON_HOST,
                    n=0, nnz=0, ld=0, values=_ptr(values), nprob=len(ns), batch_desc=desc.ctypes.data)
    return m, (values, desc)


def snmf_create(matrix, r: int, options: snmf_options | None = None, stream=None, mlp_weights=None):
    """Create a handle.  ``matrix`` is the (snmf_matrix, keepalive) pair of
    dense_matrix/csr_matrix.  Returns the handle (c_void_p)."""
    lib = load_library()
    m, _keep = matrix
    h = C.c_void_p()
    opt = options if options is not None else snmf_default_options()
    wbuf = None
    if mlp_weights is not None:
        wbuf = np.ascontiguousarray(np.asarray(mlp_weights, dtype=np.float32))
        opt.mlp_weights = wbuf.ctypes.data
    s = None
    if stream is not None:
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    st = lib.snmf_create(C.byref(h), C.byref(m), int(r), C.byref(opt), s)
    _check(lib, None, st)
    _BORROWED[h.value] = _keep
    return h


def snmf_set_graph_reg(h, matrix, gamma: float):
    lib = load_library()
    m = None if matrix is None else C.byref(matrix[0])
    return _check(lib, h, lib.snmf_set_graph_reg(h, m, float(gamma)))


def snmf_lai_sketch(h, k: int, oversample: int, power_iters: int, seed: int):
    lib = load_library()
    return _check(lib, h, lib.snmf_lai_sketch(h, int(k), int(oversample), int(power_iters), int(seed)))


def snmf_svd_init(h, W, Ht=None, oversample: int = 10, power_iters: int = 2, seed: int = 0):
    """SVD start |U E^1/2| (Sec. 4.1 guideline (4)) into device tensors W (and Ht)."""
    lib = load_library()
    return _check(lib, h, lib.snmf_svd_init(h, _ptr(W), _ptr(Ht), int(oversample), int(power_iters), int(seed)))


def snmf_get_state(h) -> bytes:
    """The last solve's per-restart scalar state (for snmf_set_state)."""
    lib = load_library()
    size = C.c_int64()
    _check(lib, h, lib.snmf_get_state(h, None, 0, C.byref(size)))
    buf = (C.c_ubyte * size.value)()
    _check(lib, h, lib.snmf_get_state(h, buf, size.value, C.byref(size)))
    return bytes(buf)


def snmf_set_state(h, blob):
    """Continue the next solve from a state of snmf_get_state (None drops it)."""
    lib = load_library()
    if blob is None:
        return _check(lib, h, lib.snmf_set_state(h, None, 0))
    buf = (C.c_ubyte * len(blob)).from_buffer_copy(blob)
    return _check(lib, h, lib.snmf_set_state(h, buf, len(blob)))


def snmf_stats_ring(h, batch: int, capacity: int = 256):
    """Per-restart statistics records [batch, capacity, 8] of the last solve (see snmf.h)."""
    lib = load_library()
    out = np.zeros((batch, capacity, SNMF_RING_VALUES), dtype=np.float64)
    cnt = C.c_int32()
    _check(lib, h, lib.snmf_stats_ring(h, out.ctypes.data, int(capacity), C.byref(cnt)))
    return out, cnt.value


def snmf_knn_graph(X, k: int = 10, sigma_rank: int = 7, stream=None):
    """kNN similarity graph of device points X (n x d float32): returns (rowptr, colidx, A^ values,
    S values, degrees) as device tensors (see include/snmf.h)."""
    import torch
    lib = load_library()
    if not _is_cuda(X) or X.dim() != 2 or X.dtype != torch.float32 or not X.is_contiguous():
        raise SnmfError(SNMF_ERR_ARG, "X must be a contiguous n x d float32 CUDA tensor")
    n, d = X.shape
    cap = 2 * n * k
    rp = torch.empty(n + 1, dtype=torch.int32, device=X.device)
    ci = torch.empty(cap, dtype=torch.int32, device=X.device)
    ah = torch.empty(cap, dtype=torch.float32, device=X.device)
    sv = torch.empty(cap, dtype=torch.float32, device=X.device)
    dg = torch.empty(n, dtype=torch.float32, device=X.device)
    nnz = C.c_int64()
    s = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(lib, None, lib.snmf_knn_graph(_ptr(X), n, d, int(k), int(sigma_rank), _ptr(rp), _ptr(ci), _ptr(ah),
                                         _ptr(sv), _ptr(dg), cap, C.byref(nnz), s))
    m = nnz.value
    return rp, ci[:m], ah[:m], sv[:m], dg


def snmf_cluster_assign(h, restart: int, n: int):
    """Cluster labels (argmax of the H row) of a restart of the last solve, as a device tensor."""
    import torch
    lib = load_library()
    lab = torch.empty(n, dtype=torch.int32, device="cuda")
    _check(lib, h, lib.snmf_cluster_assign(h, int(restart), _ptr(lab)))
    return lab


def snmf_cluster_scores(truth, pred, k_true: int, k_pred: int, stream=None):
    """(contingency table, ARI, matched accuracy) of two device int32 labelings."""
    lib = load_library()
    n = int(truth.shape[0])
    table = np.zeros((k_true, k_pred), dtype=np.int64)
    ari, acc = C.c_double(), C.c_double()
    s = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(lib, None, lib.snmf_cluster_scores(_ptr(truth), _ptr(pred), n, int(k_true), int(k_pred),
                                              table.ctypes.data, C.byref(ari), C.byref(acc), s))
    return table, ari.value, acc.value


def snmf_solve(h, W=None, Ht=None):
    """Solve in place on device tensors W (and Ht).  Returns (status, stats dict)."""
    lib = load_library()
    out = snmf_stats()
    st = _check(lib, h, lib.snmf_solve(h, _ptr(W), _ptr(Ht), C.byref(out)))
    return st, out.as_dict()


def snmf_solve_host(h, W, Ht=None):
    """Solve with host (pinned or pageable) W / Ht, copied inside the call."""
    lib = load_library()
    out = snmf_stats()
    st = _check(lib, h, lib.snmf_solve_host(h, _ptr(W), _ptr(Ht), C.byref(out)))
    return st, out.as_dict()


def snmf_restart_stats(h, batch: int):
    lib = load_library()
    f = np.zeros(batch)
    res = np.zeros(batch)
    pg = np.zeros(batch)
    it = np.zeros(batch, dtype=np.int32)
    _check(lib, h, lib.snmf_restart_stats(h, f.ctypes.data, res.ctypes.data, pg.ctypes.data, it.ctypes.data))
    return dict(f=f, residual=res, pg_rel=pg, iters=it)


def snmf_get_factors(h, W=None, Ht=None):
    lib = load_library()
    return _check(lib, h, lib.snmf_get_factors(h, _ptr(W), _ptr(Ht)))


def snmf_apply(h, X, Y, cols: int):
    lib = load_library()
    xax = C.c_double()
    _check(lib, h, lib.snmf_apply(h, _ptr(X), _ptr(Y), int(cols), C.byref(xax)))
    return xax.value


def snmf_profile_ax(h, iters: int = 20):
    """Mean ms of one A*X product (kernel + epilogue) and of the product kernel alone."""
    lib = load_library()
    a, b = C.c_double(), C.c_double()
    _check(lib, h, lib.snmf_profile_ax(h, int(iters), C.byref(a), C.byref(b)))
    return a.value, b.value


def snmf_apply_dense_noalloc(A, X, Y, stream=None):
    """Y = A X and <X, A X> without any device allocation (see include/snmf.h).
    A: n x n device tensor (float32/float64, unit column stride), X, Y: contiguous n x cols
    device tensors of A's dtype on A's device.  The C side sees raw pointers only, so the
    shapes, dtypes, strides and devices are checked here before the call."""
    lib = load_library()
    for name, t in (("A", A), ("X", X), ("Y", Y)):
        if not _is_cuda(t) or t.dim() != 2:
            raise SnmfError(SNMF_ERR_ARG, f"{name} must be a 2-D CUDA tensor")
    n, cols = X.shape
    if tuple(A.shape) != (n, n) or A.stride(1) != 1 or A.stride(0) < n:
        raise SnmfError(SNMF_ERR_ARG, f"A must be {n} x {n} with unit column stride (got {tuple(A.shape)})")
    if tuple(Y.shape) != (n, cols) or not X.is_contiguous() or not Y.is_contiguous():
        raise SnmfError(SNMF_ERR_ARG, "X and Y must be contiguous n x cols tensors")
    if not (A.dtype == X.dtype == Y.dtype) or not str(A.dtype).endswith(("float32", "float64")):
        raise SnmfError(SNMF_ERR_ARG, "A, X and Y must share one dtype, float32 or float64")
    if not (A.device == X.device == Y.device):
        raise SnmfError(SNMF_ERR_ARG, "A, X and Y must be on one device")
    dt = SNMF_F64 if str(A.dtype).endswith("float64") else SNMF_F32
    xax = C.c_double()
    s = None
    if stream is not None:
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    st = lib.snmf_apply_dense_noalloc(_ptr(A), dt, n, A.stride(0), _ptr(X), _ptr(Y), cols, C.byref(xax), s)
    if st == SNMF_ERR_ARG:
        raise SnmfError(st, "rejected: needs n <= %d and 2*n*cols*element size <= %d bytes, lda >= n, "
                            "float32/float64" % (NOALLOC_MAX_ROWS, NOALLOC_MAX_SLICE_PAIR_BYTES))
    _check(lib, None, st)
    return xax.value


def snmf_controller_data(h, capacity: int = 1 << 18):
    """Recorded (features, target log2 multiplier) samples of a record-mode handle."""
    lib = load_library()
    feat = np.zeros((capacity, SNMF_MLP_IN), dtype=np.float32)
    targ = np.zeros(capacity, dtype=np.float32)
    cnt = C.c_int32()
    _check(lib, h, lib.snmf_controller_data(h, feat.ctypes.data, targ.ctypes.data, capacity, C.byref(cnt)))
    return feat[:cnt.value].copy(), targ[:cnt.value].copy()


def snmf_mlp_train(feats, targets, weights, steps: int = 1000, lr: float = 1e-2):
    """Train the controller MLP on the GPU.  Returns (weights, final loss, gradient at the
    initial weights)."""
    lib = load_library()
    f = np.ascontiguousarray(feats, dtype=np.float32)
    t = np.ascontiguousarray(targets, dtype=np.float32)
    w = np.array(weights, dtype=np.float32, copy=True)
    g0 = np.zeros(SNMF_MLP_NPARAMS, dtype=np.float32)
    loss = C.c_double()
    _check(lib, None, lib.snmf_mlp_train(f.ctypes.data, t.ctypes.data, len(t), w.ctypes.data, int(steps),
                                         float(lr), C.byref(loss), g0.ctypes.data))
    return w, loss.value, g0


def snmf_mlp_eval(weights, feats):
    """Multipliers 2^(2 tanh o) of the controller network on the device (BF16 weights, as the
    solver uses them) for feature vectors feats[i][5]."""
    lib = load_library()
    w = np.ascontiguousarray(weights, dtype=np.float32)
    f = np.ascontiguousarray(feats, dtype=np.float32).reshape(-1, SNMF_MLP_IN)
    out = np.zeros(len(f), dtype=np.float32)
    _check(lib, None, lib.snmf_mlp_eval(w.ctypes.data, f.ctypes.data, len(f), out.ctypes.data))
    return out


def snmf_set_timeout(h, cycles: int):
    """Bound (clock64 cycles) of the handle's device-side waits; 0 restores the default."""
    lib = load_library()
    return _check(lib, h, lib.snmf_set_timeout(h, int(cycles)))


def snmf_step_config(h) -> dict:
    """Row-kernel body of the D step and update (0 general, 1 tile, 2 recomputing), rows per CTA
    and the algorithmic bytes of one launch of each."""
    lib = load_library()
    body, rows = C.c_int32(), C.c_int32()
    bd, bu = C.c_int64(), C.c_int64()
    _check(lib, h, lib.snmf_step_config(h, C.byref(body), C.byref(rows), C.byref(bd), C.byref(bu)))
    return dict(body=body.value, rows_per_cta=rows.value, dstep_bytes=bd.value, update_bytes=bu.value)


def snmf_profile_steps(h, iters: int = 20):
    """Mean ms of one D-step launch and of one update launch of a W block (after a solve)."""
    lib = load_library()
    a, b = C.c_double(), C.c_double()
    _check(lib, h, lib.snmf_profile_steps(h, int(iters), C.byref(a), C.byref(b)))
    return a.value, b.value


def snmf_tuned_config(h) -> dict:
    """Product launch configuration chosen by the autotuner of this handle."""
    lib = load_library()
    sp, st, ps, fc = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
    ms = C.c_double()
    _check(lib, h, lib.snmf_tuned_config(h, C.byref(sp), C.byref(st), C.byref(ps), C.byref(ms), C.byref(fc)))
    bn, bm = C.c_int32(), C.c_int32()
    _check(lib, h, lib.snmf_tuned_tiles(h, C.byref(bn), C.byref(bm)))
    return dict(splits=sp.value, stages=st.value, per_sm=ps.value, bn=bn.value, row_bm=bm.value, ms=ms.value,
                from_cache=bool(fc.value))


def snmf_destroy(h):
    lib = load_library()
    st = lib.snmf_destroy(h)
    if h is not None:
        _BORROWED.pop(getattr(h, "value", h), None)
    return st


def snmf_last_error(h=None) -> str:
    lib = load_library()
    return lib.snmf_last_error(h).decode(errors="replace")
