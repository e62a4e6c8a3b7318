"""GB300 (sm_103a) FRAM solver: Python binding of the C ABI in ``include/fram.h``.

This module only marshals arguments: every step of the solve (validation,
prescaling, gradient GEMMs, SDSN, update, assignment, objective) runs in the
CUDA kernels of ``libfram.so``.  There is no CPU fallback: if the library is
missing, :func:`load` raises.

Matrix arguments may be torch tensors (CUDA or CPU), numpy arrays, or raw
integer addresses.  They must be contiguous ``float64`` (``int32`` for
permutations).  Host and device buffers are both accepted by ``fram_solve``
and ``fram_solve_batched``; the step-level calls take device buffers only.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfram.so")

FRAM_OK = 0
FRAM_NOT_READY = 1
FRAM_ERR_INVALID = -1
FRAM_ERR_OOM = -2
FRAM_ERR_CUDA = -3
FRAM_ERR_DEGENERATE = -4
FRAM_ERR_TIMEOUT = -5
FRAM_ERR_BUSY = -6

FRAM_PREC_FP64 = 0
FRAM_PREC_MIXED_TF32 = 1
FRAM_PREC_MIXED_BF16 = 2
FRAM_PROJ_SDSN = 0
FRAM_PROJ_EXACT = 1

STATUS_NAMES = {0: "FRAM_OK", 1: "FRAM_NOT_READY", -1: "FRAM_ERR_INVALID", -2: "FRAM_ERR_OOM",
                -3: "FRAM_ERR_CUDA", -4: "FRAM_ERR_DEGENERATE", -5: "FRAM_ERR_TIMEOUT",
                -6: "FRAM_ERR_BUSY"}


class FramParams(C.Structure):
    _fields_ = [("lam", C.c_double), ("alpha", C.c_double), ("theta", C.c_double),
                ("delta_tol", C.c_double), ("gamma_tol", C.c_double), ("polish_tol", C.c_double),
                ("mixed_delta_tol", C.c_double), ("stall_ratio", C.c_double),
                ("stall_below", C.c_double), ("max_outer", C.c_int), ("max_sweeps", C.c_int), ("max_polish", C.c_int),
                ("precision", C.c_int), ("init", C.c_int), ("projection", C.c_int)]


class FramInfo(C.Structure):
    _fields_ = [("outer_iters", C.c_int), ("total_sweeps", C.c_int), ("polish_sweeps", C.c_int),
                ("sdsn_converged_last", C.c_int), ("lap_augmentations", C.c_int),
                ("lap_auction_phases", C.c_int), ("delta", C.c_double), ("gamma", C.c_double),
                ("objective", C.c_double), ("match_error", C.c_double),
                ("assignment_value", C.c_double), ("ms_total", C.c_double),
                ("ms_gemm", C.c_double), ("ms_sdsn", C.c_double), ("ms_polish", C.c_double),
                ("ms_update", C.c_double), ("ms_rounding", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class FramError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None
_P = C.c_void_p


def load(path: str | None = None):
    """Load ``libfram.so`` (built in-tree by ``paper_2508_00887_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"{path} not found: build it with `python -m paper_2508_00887_gb300.build`")
    lib = C.CDLL(path)
    i, d, u64, sz = C.c_int, C.c_double, C.c_uint64, C.c_size_t
    sig = {
        "fram_create": (i, [C.POINTER(_P), i, sz, _P]),
        "fram_destroy": (i, [_P]),
        "fram_default_params": (None, [C.POINTER(FramParams)]),
        "fram_last_error": (C.c_char_p, [_P]),
        "fram_kernel_launches": (u64, [_P]),
        "fram_set_wait_limit": (i, [_P, i]),
        "fram_selftest_wait_timeout": (i, [_P, i]),
        "fram_solve": (i, [_P, i, _P, _P, _P, C.POINTER(FramParams), _P, _P, C.POINTER(FramInfo)]),
        "fram_solve_batched": (i, [_P, i, _P, _P, _P, C.POINTER(FramParams), _P, _P,
                                   C.POINTER(FramInfo)]),
        "fram_set_batched_kernel": (i, [_P, i]),
        "fram_batched_kernel": (i, [_P, i]),
        "fram_submit": (i, [_P, i, _P, _P, C.POINTER(FramParams), C.POINTER(u64)]),
        "fram_poll": (i, [_P, u64, _P, _P, C.POINTER(FramInfo), i]),
        "fram_serve_ticks": (u64, [_P]),
        "fram_gradient": (i, [_P, i, _P, _P, _P, _P, d, _P]),
        "fram_node_affinity": (i, [_P, i, i, _P, _P, _P]),
        "fram_fra_exact": (i, [_P, i, _P, _P, d, d, i, C.POINTER(i), C.POINTER(d)]),
        "fram_set_sparse_density": (i, [_P, d]),
        "fram_gradient_lowp": (i, [_P, i, _P, _P, _P, _P, d, i, _P]),
        "fram_sdsn": (i, [_P, i, _P, _P, d, d, i, C.POINTER(i), C.POINTER(d)]),
        "fram_sdsn_f32": (i, [_P, i, _P, i, _P, i, d, d, i, C.POINTER(i), C.POINTER(d)]),
        "fram_sdsn_grouped": (i, [_P, i, _P, _P, _P, d, d, i, _P, _P]),
        "fram_assign": (i, [_P, i, _P, _P, C.POINTER(d), C.POINTER(i)]),
        "fram_set_lap_searches": (i, [_P, i]),
        "fram_lap_last_stats": (i, [_P, C.POINTER(i), C.POINTER(i), C.POINTER(C.c_longlong)]),
        "fram_sdsn_static": (i, [i, _P, _P, d, d, i, _P, C.POINTER(i), C.POINTER(d), C.c_char_p,
                                 sz]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    """Names the header declares; used by the ABI test."""
    return ["fram_create", "fram_destroy", "fram_default_params", "fram_last_error",
            "fram_kernel_launches", "fram_set_wait_limit", "fram_selftest_wait_timeout",
            "fram_solve", "fram_solve_batched", "fram_set_batched_kernel", "fram_batched_kernel",
            "fram_submit",
            "fram_poll", "fram_serve_ticks", "fram_node_affinity", "fram_fra_exact", "fram_set_sparse_density", "fram_gradient", "fram_gradient_lowp", "fram_sdsn", "fram_sdsn_f32", "fram_sdsn_grouped",
            "fram_assign", "fram_set_lap_searches", "fram_lap_last_stats", "fram_sdsn_static"]


# ---------------------------------------------------------------- marshalling
_DTYPE_NAMES = {}  # torch dtype object -> "float64", ... (str() of a dtype is slow)


def _dtype_name(dt):
    name = _DTYPE_NAMES.get(dt)
    if name is None:
        name = _DTYPE_NAMES[dt] = str(dt).split(".")[-1]
    return name


def _addr(x, dtype="float64"):
    """Address of a contiguous buffer (torch tensor, numpy array or int)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):            # torch.Tensor
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if _dtype_name(x.dtype) != dtype:
            raise ValueError(f"tensor dtype must be {dtype}, got {x.dtype}")
        return x.data_ptr()
    if hasattr(x, "ctypes"):              # numpy.ndarray
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        if x.dtype.name != dtype:
            raise ValueError(f"array dtype must be {dtype}, got {x.dtype}")
        return x.ctypes.data
    raise TypeError(f"unsupported buffer type {type(x)}")


def _addrs(xs, dtype="float64"):
    """_addr over a list; lists of torch tensors or numpy arrays take a fast
    path (the dtype is checked once per distinct dtype object, by identity)."""
    if not xs:
        return []
    if not hasattr(xs[0], "data_ptr"):
        if not hasattr(xs[0], "ctypes"):
            return [_addr(x, dtype) for x in xs]
        out = []
        seen = None
        for x in xs:
            if x is None or not hasattr(x, "ctypes"):
                out.append(_addr(x, dtype))
                continue
            dt = x.dtype
            if dt is not seen:
                if dt.name != dtype:
                    raise ValueError(f"array dtype must be {dtype}, got {dt}")
                seen = dt
            if not x.flags.c_contiguous:
                raise ValueError("array must be C-contiguous")
            out.append(x.ctypes.data)
        return out
    out = []
    seen = None
    for x in xs:
        if x is None or not hasattr(x, "data_ptr"):
            out.append(_addr(x, dtype))
            continue
        dt = x.dtype
        if dt is not seen:
            if _dtype_name(dt) != dtype:
                raise ValueError(f"tensor dtype must be {dtype}, got {dt}")
            seen = dt
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        out.append(x.data_ptr())
    return out


def _check(ctx, status):
    if status not in (FRAM_OK, FRAM_NOT_READY):
        msg = load().fram_last_error(ctx)
        raise FramError(status, msg.decode() if msg else "")
    return status


def fram_default_params(**overrides) -> FramParams:
    p = FramParams()
    load().fram_default_params(C.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def fram_create(device: int = 0, hbm_budget_bytes: int = 0, stream=None):
    """Create a context; ``stream`` is a cudaStream_t address (e.g.
    ``torch.cuda.current_stream().cuda_stream``) or None."""
    ctx = _P()
    st = load().fram_create(C.byref(ctx), device, hbm_budget_bytes, stream)
    if st != FRAM_OK:
        raise FramError(st, "fram_create failed")
    return ctx


def fram_destroy(ctx):
    return load().fram_destroy(ctx)


def fram_last_error(ctx) -> str:
    m = load().fram_last_error(ctx)
    return m.decode() if m else ""


def fram_kernel_launches(ctx) -> int:
    return int(load().fram_kernel_launches(ctx))


def fram_set_wait_limit(ctx, limit_ms: int, check=True):
    st = load().fram_set_wait_limit(ctx, limit_ms)
    if check:
        _check(ctx, st)
    return st


def fram_selftest_wait_timeout(ctx, blocks: int = 4):
    """Expected to return FRAM_ERR_TIMEOUT (no exception)."""
    return load().fram_selftest_wait_timeout(ctx, blocks)


def fram_solve(ctx, n, A, B, K=None, params=None, X_out=None, perm_out=None, check=True):
    info = FramInfo()
    st = load().fram_solve(ctx, n, _addr(A), _addr(B), _addr(K),
                           C.byref(params) if params is not None else None,
                           _addr(X_out), _addr(perm_out, "int32"), C.byref(info))
    if check:
        _check(ctx, st)
    return st, info


def _is_index_array(x, itemsize):
    """A 1-D C-contiguous numpy integer array with `itemsize`-byte entries."""
    dt = getattr(x, "dtype", None)
    return (dt is not None and hasattr(x, "ctypes") and getattr(dt, "kind", "") in "iu" and
            dt.itemsize == itemsize and x.ndim == 1 and x.flags.c_contiguous)


def _ptr_table(xs, count, dtype):
    """The pointer table of one fram_solve_batched argument: an integer
    address array (numpy, 8-byte entries, one per pair) is passed as it is,
    with no copy and no per-entry check; a list of tensors / arrays / addresses
    goes through _addrs.  Returns (argument, object to keep alive)."""
    if xs is None:
        return None, None
    if _is_index_array(xs, 8):
        if xs.shape[0] != count:
            raise ValueError("an address array needs one entry per pair")
        return xs.ctypes.data, xs
    arr = (_P * count)(*_addrs(xs, dtype))
    return arr, arr


def fram_solve_batched(ctx, ns, As, Bs, params=None, X_outs=None, perm_outs=None, check=True):
    """ns: a list of sizes or a contiguous numpy int32 array.  As, Bs, X_outs,
    perm_outs: lists of matrices / vectors, or numpy integer arrays of their
    addresses (8-byte entries), e.g. base + byte offsets into one packed
    buffer per batch -- the fast path for large batches, which skips the
    per-tensor checks (the library still checks every pointer's memory
    kind)."""
    count = len(ns)
    keep = []
    if _is_index_array(ns, 4):
        n_arr = ns.ctypes.data
        keep.append(ns)
    else:
        n_arr = (C.c_int * count)(*ns)
    a_arr, ka = _ptr_table(As, count, "float64")
    b_arr, kb = _ptr_table(Bs, count, "float64")
    x_arr, kx = _ptr_table(X_outs, count, "float64")
    p_arr, kp = _ptr_table(perm_outs, count, "int32")
    keep += [ka, kb, kx, kp]
    infos = (FramInfo * max(count, 1))()
    st = load().fram_solve_batched(ctx, count, n_arr, a_arr, b_arr,
                                   C.byref(params) if params is not None else None,
                                   x_arr, p_arr, infos)
    if check:
        _check(ctx, st)
    # The ctypes array itself (indexable, iterable, len() == count): copying
    # thousands of structs into a list would cost more than the call.
    return st, (infos if count > 0 else [])


def fram_set_batched_kernel(ctx, variant, check=True):
    st = load().fram_set_batched_kernel(ctx, variant)
    if check:
        _check(ctx, st)
    return st


def fram_batched_kernel(ctx, precision) -> int:
    return int(load().fram_batched_kernel(ctx, precision))


def fram_submit(ctx, n, A, B, params=None, check=True):
    t = C.c_uint64()
    st = load().fram_submit(ctx, n, _addr(A), _addr(B),
                            C.byref(params) if params is not None else None, C.byref(t))
    if check:
        _check(ctx, st)
    return st, t.value


def fram_poll(ctx, ticket, X_out=None, perm_out=None, wait_ms=0, check=True):
    info = FramInfo()
    st = load().fram_poll(ctx, ticket, _addr(X_out), _addr(perm_out, "int32"), C.byref(info),
                          wait_ms)
    if check:
        _check(ctx, st)
    return st, info


def fram_serve_ticks(ctx) -> int:
    return int(load().fram_serve_ticks(ctx))


def fram_node_affinity(ctx, n, d, F, Ft, K, check=True):
    st = load().fram_node_affinity(ctx, n, d, _addr(F), _addr(Ft), _addr(K))
    if check:
        _check(ctx, st)
    return st


def fram_gradient(ctx, n, A, N, B, X, K=None, lam=1.0, check=True):
    st = load().fram_gradient(ctx, n, _addr(A), _addr(N), _addr(B), _addr(K), lam, _addr(X))
    if check:
        _check(ctx, st)
    return st


def fram_gradient_lowp(ctx, n, A, N, B, X, precision, K=None, lam=1.0, check=True):
    st = load().fram_gradient_lowp(ctx, n, _addr(A), _addr(N), _addr(B), _addr(K), lam,
                                   precision, _addr(X, "float32"))
    if check:
        _check(ctx, st)
    return st


def fram_sdsn(ctx, n, X, D, theta, gamma_tol=1e-14, max_sweeps=200, check=True):
    sw = C.c_int()
    g = C.c_double()
    st = load().fram_sdsn(ctx, n, _addr(X), _addr(D), theta, gamma_tol, max_sweeps, C.byref(sw),
                          C.byref(g))
    if check:
        _check(ctx, st)
    return st, sw.value, g.value


def fram_sdsn_f32(ctx, n, X, D, theta, gamma_tol=1e-6, max_sweeps=200, ldx=None, ldd=None,
                  check=True):
    """FP32 SDSN (the mixed paths' kernel) on float32 device buffers with row
    strides ldx / ldd (default n)."""
    sw = C.c_int()
    g = C.c_double()
    st = load().fram_sdsn_f32(ctx, n, _addr(X, "float32"), ldx or n, _addr(D, "float32"),
                              ldd or n, theta, gamma_tol, max_sweeps, C.byref(sw), C.byref(g))
    if check:
        _check(ctx, st)
    return st, sw.value, g.value


FRAM_SDSN_STATIC_MAX_N = 4096


def fram_sdsn_static(n, X, D, theta, gamma_tol=1e-14, max_sweeps=200, stream=None, check=True):
    """Allocation-free SDSN (see include/fram.h): returns (status, sweeps, gamma, message)."""
    sw = C.c_int()
    g = C.c_double()
    buf = C.create_string_buffer(256)
    st = load().fram_sdsn_static(n, _addr(X), _addr(D), theta, gamma_tol, max_sweeps, stream,
                                 C.byref(sw), C.byref(g), buf, 256)
    msg = buf.value.decode()
    if check and st != FRAM_OK:
        raise FramError(st, msg)
    return st, sw.value, g.value, msg


def fram_sdsn_grouped(ctx, ns, Xs, Ds, theta, gamma_tol=1e-14, max_sweeps=200, check=True):
    count = len(ns)
    n_arr = (C.c_int * count)(*ns)
    x_arr = (_P * count)(*[_addr(x) for x in Xs])
    d_arr = (_P * count)(*[_addr(x) for x in Ds])
    sw = (C.c_int * count)()
    g = (C.c_double * count)()
    st = load().fram_sdsn_grouped(ctx, count, n_arr, x_arr, d_arr, theta, gamma_tol, max_sweeps,
                                  C.cast(sw, _P), C.cast(g, _P))
    if check:
        _check(ctx, st)
    return st, list(sw), list(g)


def fram_set_sparse_density(ctx, max_density, check=True):
    st = load().fram_set_sparse_density(ctx, max_density)
    if check:
        _check(ctx, st)
    return st


def fram_fra_exact(ctx, n, X, D, theta, tol=1e-12, max_sweeps=10000, check=True):
    sw = C.c_int()
    res = C.c_double()
    st = load().fram_fra_exact(ctx, n, _addr(X), _addr(D), theta, tol, max_sweeps, C.byref(sw),
                               C.byref(res))
    if check:
        _check(ctx, st)
    return st, sw.value, res.value


def fram_set_lap_searches(ctx, searches, check=True):
    st = load().fram_set_lap_searches(ctx, searches)
    if check:
        _check(ctx, st)
    return st


def fram_lap_last_stats(ctx):
    """(augmenting paths applied, searches repeated, Dijkstra steps) of the
    last assignment."""
    a, r, s = C.c_int(), C.c_int(), C.c_longlong()
    st = load().fram_lap_last_stats(ctx, C.byref(a), C.byref(r), C.byref(s))
    _check(ctx, st)
    return a.value, r.value, s.value


def fram_assign(ctx, n, W, perm, check=True, with_phases=False):
    v = C.c_double()
    ph = C.c_int()
    st = load().fram_assign(ctx, n, _addr(W), _addr(perm, "int32"), C.byref(v), C.byref(ph))
    if check:
        _check(ctx, st)
    return (st, v.value, ph.value) if with_phases else (st, v.value)
