"""Python binding of liblogdet (C ABI in include/logdet.h).

Argument marshalling only: every step of the computation runs in the native
library (host set-up in C++, every per-evaluation step in CUDA kernels for
sm_103a).  The functions keep the C names; errors raise LogDetError.

    ctx = ld_create(grid_matrix(LD_STENCIL_2D13_SQ, (1024, 1024), kappa2=0.1),
                    colouring_distance=2, n_shifts=20, tol=1e-8,
                    options=Options(precision=LD_MIXED))
    value, info = ld_logdet(ctx)

`LogDet.apply(ctx, kappa2, tau, scale)` is a torch.autograd.Function whose
backward pass runs the library's gradient kernel on the saved seed solutions
(d log det Q / d eta = tr(Q^{-1} dQ/d eta)).
"""
from __future__ import annotations

import ctypes as C
import os

# The grid engine runs tile groups, and a batch its large instances, on streams of their own;
# the CUDA runtime serves 8 hardware queues unless told otherwise, and streams beyond the
# eighth then wait on one another.  The setting is read when the process creates its CUDA
# context, so it takes effect when this package is imported first.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

import numpy as np

from ._build import OUT as _LIB_PATH

LD_OK, LD_EINVAL, LD_ENOMEM, LD_ECUDA, LD_ENOTSPD, LD_ENOTCONV, LD_ENUMERIC, LD_ETIMEOUT, \
    LD_EUNSUPPORTED, LD_ECALLBACK = range(10)
LD_FP64, LD_MIXED = 0, 1
LD_CSR, LD_STENCIL_2D5, LD_STENCIL_2D13_SQ, LD_STENCIL_3D7, LD_MATFREE = 0, 1, 2, 3, 4
LD_P_KAPPA2, LD_P_TAU, LD_P_SCALE = 0, 1, 2

STATUS_NAMES = {0: "LD_OK", 1: "LD_EINVAL", 2: "LD_ENOMEM", 3: "LD_ECUDA", 4: "LD_ENOTSPD",
                5: "LD_ENOTCONV", 6: "LD_ENUMERIC", 7: "LD_ETIMEOUT", 8: "LD_EUNSUPPORTED",
                9: "LD_ECALLBACK"}


class LogDetError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status


class Matrix(C.Structure):
    _fields_ = [("kind", C.c_int32), ("periodic", C.c_int32), ("n", C.c_int64),
                ("rowptr", C.c_void_p), ("colidx", C.c_void_p), ("val", C.c_void_p),
                ("dims", C.c_int32 * 3), ("kappa2", C.c_double), ("kappa2_field", C.c_void_p),
                ("tau", C.c_double), ("obs_mask", C.c_void_p), ("scale", C.c_double)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("tile_width", C.c_int32), ("max_iter", C.c_int32),
                ("keep_x0", C.c_int32), ("lambda_min", C.c_double), ("lambda_max", C.c_double),
                ("cuda_stream", C.c_void_p), ("colouring", C.c_void_p), ("engine", C.c_int32),
                ("chunk_iters", C.c_int32), ("reliable_delta", C.c_double),
                ("lattice_pass", C.c_int32)]


class Info(C.Structure):
    _fields_ = [("status", C.c_int32), ("n_colours", C.c_int32), ("n_shifts", C.c_int32),
                ("iters", C.c_int32), ("tile_width", C.c_int32), ("engine", C.c_int32),
                ("lambda_min", C.c_double), ("lambda_max", C.c_double), ("quad_cert", C.c_double),
                ("ms", C.c_double), ("iter_ms", C.c_double), ("tile_iters", C.c_int64),
                ("gpu_launches", C.c_int64), ("bulk_rows", C.c_int32),
                ("reliable_updates", C.c_int32), ("rel_resid_max", C.c_double),
                ("pass_words", C.c_int32), ("vertex_tile_iters", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None

# ld_matvec_fn: int (*)(void *user, int64_t n, int32_t ncols, const double *P, double *W, void *stream)
MATVEC_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p)
# ld_dmatvec_fn: int (*)(void *user, int32_t param, int64_t n, int32_t ncols, const double *X, double *Y,
#                        void *stream)
DMATVEC_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_int32, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p,
                         C.c_void_p)


def library(build_if_missing: bool = False):
    """Load liblogdet.so (raises if it is missing: there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        if build_if_missing:
            from ._build import build
            build()
        else:
            raise ImportError("liblogdet.so not built at %s; run __graft_entry__.build()" % _LIB_PATH)
    L = C.CDLL(_LIB_PATH)
    vp, i32, i64, dbl, st = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_int
    P = C.POINTER
    sig = {
        "ld_abi_version": ([], C.c_int),
        "ld_default_options": ([P(Options)], st),
        "ld_create": ([P(Matrix), C.c_int, C.c_int, dbl, P(Options), P(vp)], st),
        "ld_create_matfree": ([i64, MATVEC_FN, vp, vp, dbl, dbl, C.c_int, dbl, P(Options), P(vp)], st),
        "ld_matfree_set_derivative": ([vp, DMATVEC_FN, vp, C.c_int], st),
        "ld_set_params": ([vp, dbl, dbl, dbl], st),
        "ld_logdet": ([vp, P(dbl), P(Info)], st),
        "ld_logdet_grad": ([vp, C.c_int, vp, P(dbl), vp, P(Info)], st),
        "ld_grad": ([vp, C.c_int, vp, vp], st),
        "ld_logdet_partial": ([vp, C.c_int, C.c_int, P(dbl), P(Info)], st),
        "ld_column_terms": ([vp, vp, vp], st),
        "ld_get_colouring": ([vp, vp, P(i32)], st),
        "ld_get_nodes": ([vp, vp, vp, P(i32)], st),
        "ld_apply": ([vp, C.c_int, vp, vp], st),
        "ld_logmv": ([vp, C.c_int, vp, vp, P(Info)], st),
        "ld_select_distance": ([vp, i64, dbl, C.c_int, P(i32), vp, P(Info)], st),
        "ld_hutchinson": ([vp, C.c_int, vp, P(dbl), P(dbl), vp, P(Info)], st),
        "ld_wait_selftest": ([i64], st),
        "ld_invsqrt_mv": ([vp, C.c_int, vp, vp, P(Info)], st),
        "ld_colour_csr": ([i64, vp, vp, C.c_int, vp, P(i32)], st),
        "ld_colour_grid": ([C.c_int, vp, C.c_int, C.c_int, vp, P(i32)], st),
        "ld_hht_nodes": ([dbl, dbl, C.c_int, vp, vp, P(dbl)], st),
        "ld_auto_shifts": ([dbl, dbl, P(i32)], st),
        "ld_grid_bounds": ([P(Matrix), P(dbl), P(dbl)], st),
        "ld_csr_bounds": ([i64, vp, vp, vp, dbl, P(dbl), P(dbl)], st),
        "ld_hht_invsqrt_nodes": ([dbl, dbl, C.c_int, vp, vp], st),
        "ld_spde_fem_csr": ([i64, vp, i64, vp, dbl, C.c_int, dbl, i64, vp, vp, vp, P(i64)], st),
        "ld_batch_create": ([C.c_int, vp, vp, C.c_int, dbl, P(Options), P(vp)], st),
        "ld_batch_logdet": ([vp, vp, vp, vp], st),
        "ld_logdet_static": ([P(Matrix), vp, C.c_int, C.c_int, dbl, C.c_int, vp, P(dbl)], st),
        "ld_last_error": ([], C.c_char_p),
        "ld_destroy": ([vp], None),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _check(status: int):
    if status != LD_OK:
        msg = library().ld_last_error().decode(errors="replace")
        raise LogDetError(status, msg)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class Context:
    """Owns an ld_ctx and the host arrays its matrix description borrowed."""

    def __init__(self, handle, n, keep):
        self.handle = handle
        self.n = n
        self._keep = keep

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            _lib.ld_destroy(h)

    def close(self):
        self.__del__()


def grid_matrix(kind, dims, kappa2, periodic=False, kappa2_field=None, tau=0.0, obs_mask=None,
                scale=1.0):
    """ld_matrix for a grid kind; returns (Matrix, arrays kept alive)."""
    m = Matrix()
    m.kind = kind
    m.periodic = 1 if periodic else 0
    d = list(dims) + [1] * (3 - len(dims))
    m.dims[:] = [int(x) for x in d]
    m.kappa2 = float(kappa2)
    keep = []
    if kappa2_field is not None:
        f = np.ascontiguousarray(kappa2_field, dtype=np.float64)
        keep.append(f)
        m.kappa2_field = _ptr(f)
    if obs_mask is not None:
        mk = np.ascontiguousarray(obs_mask, dtype=np.uint8)
        keep.append(mk)
        m.obs_mask = _ptr(mk)
    m.tau = float(tau)
    m.scale = float(scale)
    return m, keep


def csr_matrix(rowptr, colidx, val, scale=1.0):
    m = Matrix()
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    ci = np.ascontiguousarray(colidx, dtype=np.int32)
    vv = np.ascontiguousarray(val, dtype=np.float64)
    m.kind = LD_CSR
    m.n = rp.size - 1
    m.rowptr, m.colidx, m.val = _ptr(rp), _ptr(ci), _ptr(vv)
    m.dims[:] = [1, 1, 1]
    m.scale = float(scale)
    return m, [rp, ci, vv]


def options(**kw) -> Options:
    o = Options()
    _check(library().ld_default_options(C.byref(o)))
    keep = []
    for k, v in kw.items():
        if k == "colouring" and v is not None:
            a = np.ascontiguousarray(v, dtype=np.int32)
            keep.append(a)
            o.colouring = _ptr(a)
        elif k == "cuda_stream":
            o.cuda_stream = C.c_void_p(int(v)) if v else None
        else:
            setattr(o, k, v)
    o._keep = keep
    return o


def ld_abi_version() -> int:
    return library().ld_abi_version()


def ld_last_error() -> str:
    return library().ld_last_error().decode(errors="replace")


def ld_create(matrix, colouring_distance: int, n_shifts: int, tol: float, opts: Options = None):
    """matrix: (Matrix, keep) from grid_matrix()/csr_matrix()."""
    m, keep = matrix
    h = C.c_void_p()
    o = opts if opts is not None else options()
    _check(library().ld_create(C.byref(m), int(colouring_distance), int(n_shifts), float(tol),
                               C.byref(o), C.byref(h)))
    n = int(m.n) if m.kind == LD_CSR else int(np.prod([max(1, x) for x in m.dims]))
    return Context(h, n, keep)


class _DeviceRows:
    """__cuda_array_interface__ of a library-owned n x ncols float64 device array."""

    def __init__(self, ptr, n, ncols):
        self.__cuda_array_interface__ = {"shape": (int(n), int(ncols)), "typestr": "<f8",
                                         "data": (int(ptr), False), "version": 2, "strides": None}


def ld_create_matfree(n: int, matvec, colouring, lambda_min: float, lambda_max: float, n_shifts: int,
                      tol: float, opts: Options = None):
    """Context for an SPD operator known only through matvec(P, W): P and W are torch
    float64 CUDA tensors (n x ncols views of the library's device buffers, row-major) and
    matvec must write W = Q P; it runs with the library's stream as torch's current stream.
    An exception inside matvec stops the solve with LD_ECALLBACK (the exception is kept in
    ctx.matvec_error)."""
    col = np.ascontiguousarray(colouring, dtype=np.int32)
    ctx_box = {}

    def call(user, n_, ncols, P, W, stream):
        try:
            import torch
            Pt = torch.as_tensor(_DeviceRows(P, n_, ncols), device="cuda")
            Wt = torch.as_tensor(_DeviceRows(W, n_, ncols), device="cuda")
            with torch.cuda.stream(torch.cuda.ExternalStream(int(stream))):
                matvec(Pt, Wt)
            return 0
        except BaseException as e:   # noqa: BLE001 -- reported through LD_ECALLBACK
            if "ctx" in ctx_box:
                ctx_box["ctx"].matvec_error = e
            return 1

    fn = MATVEC_FN(call) if matvec is not None else MATVEC_FN()
    h = C.c_void_p()
    o = opts if opts is not None else options()
    _check(library().ld_create_matfree(int(n), fn, None, _ptr(col) if col.size else None,
                                       float(lambda_min), float(lambda_max), int(n_shifts),
                                       float(tol), C.byref(o), C.byref(h)))
    ctx = Context(h, int(n), [fn, col, o])
    ctx.matvec_error = None
    ctx_box["ctx"] = ctx
    return ctx


def ld_matfree_set_derivative(ctx: Context, dmatvec, n_params: int):
    """Register dQ/d eta_j for a matrix-free context: dmatvec(j, X, Y) must write
    Y = (dQ/d eta_j) X (torch float64 CUDA views, as matvec) for j in [0, n_params); then
    ld_logdet_grad / ld_grad take ids in [0, n_params).  None unregisters.  An exception
    stops the gradient with LD_ECALLBACK (kept in ctx.matvec_error)."""
    def call(user, param, n_, ncols, X, Y, stream):
        try:
            import torch
            Xt = torch.as_tensor(_DeviceRows(X, n_, ncols), device="cuda")
            Yt = torch.as_tensor(_DeviceRows(Y, n_, ncols), device="cuda")
            with torch.cuda.stream(torch.cuda.ExternalStream(int(stream))):
                dmatvec(int(param), Xt, Yt)
            return 0
        except BaseException as e:   # noqa: BLE001 -- reported through LD_ECALLBACK
            ctx.matvec_error = e
            return 1

    fn = DMATVEC_FN(call) if dmatvec is not None else DMATVEC_FN()
    _check(library().ld_matfree_set_derivative(ctx.handle, fn, None, int(n_params) if dmatvec else 0))
    ctx._keep.append(fn)


def ld_set_params(ctx: Context, kappa2: float, tau: float = 0.0, scale: float = 1.0):
    _check(library().ld_set_params(ctx.handle, float(kappa2), float(tau), float(scale)))


def ld_logdet(ctx: Context):
    v = C.c_double()
    info = Info()
    _check(library().ld_logdet(ctx.handle, C.byref(v), C.byref(info)))
    return v.value, info.as_dict()


def ld_logdet_grad(ctx: Context, param_ids):
    ids = np.ascontiguousarray(param_ids, dtype=np.int32)
    g = np.zeros(ids.size)
    v = C.c_double()
    info = Info()
    _check(library().ld_logdet_grad(ctx.handle, ids.size, _ptr(ids), C.byref(v), _ptr(g),
                                    C.byref(info)))
    return v.value, g, info.as_dict()


def ld_grad(ctx: Context, param_ids):
    ids = np.ascontiguousarray(param_ids, dtype=np.int32)
    g = np.zeros(ids.size)
    _check(library().ld_grad(ctx.handle, ids.size, _ptr(ids), _ptr(g)))
    return g


def ld_logdet_partial(ctx: Context, colour_begin: int, colour_end: int):
    v = C.c_double()
    info = Info()
    _check(library().ld_logdet_partial(ctx.handle, int(colour_begin), int(colour_end), C.byref(v),
                                       C.byref(info)))
    return v.value, info.as_dict()


def ld_get_colouring(ctx: Context):
    nc = C.c_int32()
    col = np.zeros(ctx.n, dtype=np.int32)
    _check(library().ld_get_colouring(ctx.handle, _ptr(col), C.byref(nc)))
    return col, nc.value


def ld_column_terms(ctx: Context):
    _, nc = ld_get_colouring(ctx)
    t = np.zeros(nc)
    s = np.zeros(nc)
    _check(library().ld_column_terms(ctx.handle, _ptr(t), _ptr(s)))
    return t, s


def ld_get_nodes(ctx: Context):
    N = C.c_int32()
    _check(library().ld_get_nodes(ctx.handle, None, None, C.byref(N)))
    s = np.zeros(2 * N.value)
    a = np.zeros(2 * N.value)
    _check(library().ld_get_nodes(ctx.handle, _ptr(s), _ptr(a), C.byref(N)))
    return s[0::2] + 1j * s[1::2], a[0::2] + 1j * a[1::2]


def ld_apply(ctx: Context, x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    if x.ndim == 1:
        x = x[:, None]
    y = np.zeros_like(x)
    _check(library().ld_apply(ctx.handle, x.shape[1], _ptr(x), _ptr(y)))
    return y


def ld_logmv(ctx: Context, V: np.ndarray):
    """log(Q) V for an n x k block (vector form of CG-M); returns (Y, info)."""
    V = np.ascontiguousarray(V, dtype=np.float64)
    if V.ndim == 1:
        V = V[:, None]
    Y = np.zeros_like(V)
    info = Info()
    _check(library().ld_logmv(ctx.handle, V.shape[1], _ptr(V), _ptr(Y), C.byref(info)))
    return Y, info.as_dict()


def ld_wait_selftest(limit_ns: int):
    """Bounded-wait self-test: raises LogDetError(LD_ETIMEOUT) when the device wait gave
    up after limit_ns as documented."""
    _check(library().ld_wait_selftest(int(limit_ns)))


def ld_hutchinson(ctx: Context, Z: np.ndarray):
    """Hutchinson estimate of tr log Q from the columns of Z (n x s): returns
    (estimate, standard error, per-column samples, info)."""
    Z = np.ascontiguousarray(Z, dtype=np.float64)
    if Z.ndim == 1:
        Z = Z[:, None]
    est, se = C.c_double(), C.c_double()
    q = np.zeros(Z.shape[1])
    info = Info()
    _check(library().ld_hutchinson(ctx.handle, Z.shape[1], _ptr(Z), C.byref(est), C.byref(se),
                                   _ptr(q), C.byref(info)))
    return est.value, se.value, q, info.as_dict()


def ld_invsqrt_mv(ctx: Context, V: np.ndarray):
    """Q^{-1/2} V for an n x k block; returns (Y, info)."""
    V = np.ascontiguousarray(V, dtype=np.float64)
    if V.ndim == 1:
        V = V[:, None]
    Y = np.zeros_like(V)
    info = Info()
    _check(library().ld_invsqrt_mv(ctx.handle, V.shape[1], _ptr(V), _ptr(Y), C.byref(info)))
    return Y, info.as_dict()


def ld_select_distance(ctx: Context, j: int, eps: float, max_d: int = 32):
    """Colouring distance by decay of log(Q) e_j (Sec. 2.1): returns (distance, profile,
    info); distance -1 when no vertex within max_d falls below eps |y_j|."""
    d = C.c_int32()
    prof = np.zeros(int(max_d) + 1)
    info = Info()
    _check(library().ld_select_distance(ctx.handle, int(j), float(eps), int(max_d), C.byref(d),
                                        _ptr(prof), C.byref(info)))
    return int(d.value), prof, info.as_dict()


def ld_colour_csr(rowptr, colidx, d: int):
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    ci = np.ascontiguousarray(colidx, dtype=np.int32)
    n = rp.size - 1
    col = np.zeros(n, dtype=np.int32)
    nc = C.c_int32()
    _check(library().ld_colour_csr(n, _ptr(rp), _ptr(ci), int(d), _ptr(col), C.byref(nc)))
    return col, nc.value


def ld_colour_grid(kind: int, dims, periodic: bool, d: int):
    dd = np.ones(3, dtype=np.int32)
    dd[:len(dims)] = dims
    n = int(np.prod(dd))
    col = np.zeros(n, dtype=np.int32)
    nc = C.c_int32()
    _check(library().ld_colour_grid(int(kind), _ptr(dd), 1 if periodic else 0, int(d), _ptr(col),
                                    C.byref(nc)))
    return col, nc.value


def ld_hht_nodes(lmin: float, lmax: float, N: int):
    s = np.zeros(2 * N)
    a = np.zeros(2 * N)
    cert = C.c_double()
    _check(library().ld_hht_nodes(float(lmin), float(lmax), int(N), _ptr(s), _ptr(a),
                                  C.byref(cert)))
    return s[0::2] + 1j * s[1::2], a[0::2] + 1j * a[1::2], cert.value


def ld_auto_shifts(lmin: float, lmax: float) -> int:
    """The node count ld_create chooses for n_shifts = 0 on [lmin, lmax]."""
    n = C.c_int32()
    _check(library().ld_auto_shifts(float(lmin), float(lmax), C.byref(n)))
    return n.value


def ld_hht_invsqrt_nodes(lmin: float, lmax: float, N: int):
    s = np.zeros(2 * N)
    b = np.zeros(2 * N)
    _check(library().ld_hht_invsqrt_nodes(float(lmin), float(lmax), int(N), _ptr(s), _ptr(b)))
    return s[0::2] + 1j * s[1::2], b[0::2] + 1j * b[1::2]


def ld_csr_bounds(rowptr, colidx, val, scale=1.0):
    """(lmin, lmax) the library uses for a CSR matrix without user bounds (host only)."""
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    ci = np.ascontiguousarray(colidx, dtype=np.int32)
    vv = np.ascontiguousarray(val, dtype=np.float64)
    lo, hi = C.c_double(), C.c_double()
    _check(library().ld_csr_bounds(rp.size - 1, _ptr(rp), _ptr(ci), _ptr(vv), float(scale), C.byref(lo),
                                   C.byref(hi)))
    return lo.value, hi.value


def ld_grid_bounds(matrix):
    m, _ = matrix
    lo, hi = C.c_double(), C.c_double()
    _check(library().ld_grid_bounds(C.byref(m), C.byref(lo), C.byref(hi)))
    return lo.value, hi.value


def ld_batch_create(matrices, distances, n_shifts: int, tol: float, opts: Options = None):
    arr = (Matrix * len(matrices))(*[m for m, _ in matrices])
    keep = [k for _, k in matrices]
    dist = np.ascontiguousarray(distances, dtype=np.int32)
    h = C.c_void_p()
    o = opts if opts is not None else options()
    _check(library().ld_batch_create(len(matrices), C.cast(arr, C.c_void_p), _ptr(dist),
                                     int(n_shifts), float(tol), C.byref(o), C.byref(h)))
    ctx = Context(h, 0, [arr, keep, dist])
    ctx.count = len(matrices)
    return ctx


def ld_batch_logdet(ctx: Context, with_grad: bool = False):
    out = np.zeros(ctx.count)
    g = np.zeros(ctx.count) if with_grad else None
    info = Info()
    _check(library().ld_batch_logdet(ctx.handle, _ptr(out), _ptr(g), C.byref(info)))
    return out, g, info.as_dict()


def ld_logdet_static(matrix, colour, n_colours: int, n_shifts: int, tol: float,
                     max_iter: int = 100000, cuda_stream=None) -> float:
    """log det with no device allocation (scratch in the library's static device
    array; see the header for limits and for the first-call and overlap rules)."""
    m, _ = matrix
    col = np.ascontiguousarray(colour, dtype=np.int32)
    v = C.c_double()
    _check(library().ld_logdet_static(C.byref(m), _ptr(col), int(n_colours), int(n_shifts),
                                      float(tol), int(max_iter),
                                      C.c_void_p(int(cuda_stream)) if cuda_stream else None,
                                      C.byref(v)))
    return v.value


def ld_destroy(ctx: Context):
    ctx.close()


def _autograd():
    import torch

    class LogDet(torch.autograd.Function):
        """log det Q(kappa2, tau, scale) with a native backward pass.

        forward: ld_set_params + ld_logdet on a keep_x0 context (the seed
        solutions Q^{-1} v_c stay in device memory); backward: ld_grad, the
        gradient kernel sum_c (dQ/d eta v_c)^T Q^{-1} v_c, times grad_out.
        """

        @staticmethod
        def forward(fctx, ctx: Context, kappa2, tau, scale):
            ld_set_params(ctx, float(kappa2), float(tau), float(scale))
            val, info = ld_logdet(ctx)
            fctx.ctx = ctx
            fctx.info = info
            fctx.device = kappa2.device
            return torch.tensor(val, dtype=torch.float64, device=kappa2.device)

        @staticmethod
        def backward(fctx, grad_out):
            ctx = fctx.ctx
            ids = []
            for k, need in zip((LD_P_KAPPA2, LD_P_TAU, LD_P_SCALE), fctx.needs_input_grad[1:]):
                if need:
                    ids.append(k)
            grads = [None, None, None]
            if ids:
                g = ld_grad(ctx, ids)
                for k, v in zip(ids, g):
                    grads[k] = grad_out * torch.tensor(v, dtype=torch.float64, device=fctx.device)
            return (None, *grads)

    return LogDet


def __getattr__(name):
    if name == "LogDet":
        cls = _autograd()
        globals()["LogDet"] = cls
        return cls
    raise AttributeError(name)
