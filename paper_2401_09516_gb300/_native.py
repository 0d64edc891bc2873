"""ctypes binding of libskr.so (the C ABI in include/skr.h).

Argument marshalling only: every computation happens in the CUDA library.
Functions keep the C names.  Arrays may be numpy arrays (host memory,
SKR_MEM_HOST) or CUDA tensors (device memory, SKR_MEM_DEVICE); all arrays
of one call must live in the same place.  If the library has not been
built, importing this module raises: there is no fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libskr.so")

# constants (mirror include/skr.h)
SKR_OK = 0
SKR_NOT_READY = 1
SKR_ERR_INVALID_ARG = -1
SKR_ERR_OOM = -2
SKR_ERR_CUDA = -3
SKR_ERR_TIMEOUT = -4
SKR_ERR_BUSY = -5
SKR_CONVERGED = 0
SKR_NOT_CONVERGED = 1
SKR_BREAKDOWN = 2
SKR_NUMERICAL = 3
SKR_DEVICE_STALL = 4
SKR_FMT_DARCY2D = 1
SKR_FMT_DARCY3D = 2
SKR_FMT_CONVDIFF2D = 3
SKR_FMT_STENCIL5 = 4
SKR_FMT_STENCIL7 = 5
SKR_FMT_HELMHOLTZ2D = 6
SKR_FMT_POISSON2D = 7
SKR_FMT_CSR = 8
SKR_CSR_MAX_ROW = 7
SKR_PC_NONE = 0
SKR_PC_JACOBI = 1
SKR_PC_ILU0 = 2
SKR_PC_SSOR = 3
SKR_PC_BJACOBI = 4
SKR_PREC_FP64 = 0
SKR_PREC_MIXED = 1
SKR_MEM_DEVICE = 0
SKR_MEM_HOST = 1
SKR_MAX_M = 48
SKR_MAX_K = 24

PRECOND = {"none": SKR_PC_NONE, "jacobi": SKR_PC_JACOBI, "ilu0": SKR_PC_ILU0, "ssor": SKR_PC_SSOR,
           "bjacobi": SKR_PC_BJACOBI}
PRECISION = {"fp64": SKR_PREC_FP64, "mixed": SKR_PREC_MIXED}


class SkrSystem(ctypes.Structure):
    _fields_ = [("fmt", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("nz", ctypes.c_int32), ("coef", ctypes.c_void_p), ("rhs", ctypes.c_void_p),
                ("params", ctypes.c_double * 4), ("rowptr", ctypes.c_void_p), ("colind", ctypes.c_void_p)]


class SkrOptions(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("k", ctypes.c_int32), ("maxit", ctypes.c_int32),
                ("max_refine", ctypes.c_int32), ("tol", ctypes.c_double),
                ("inner_tol", ctypes.c_double), ("precond", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("cluster_size", ctypes.c_int32),
                ("max_slots", ctypes.c_int32), ("mem", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("stream", ctypes.c_void_p),
                ("warm_start", ctypes.c_int32), ("diagnostics", ctypes.c_int32),
                ("pc_blocks", ctypes.c_int32), ("eig_fp32", ctypes.c_int32),
                ("recycle_out", ctypes.c_void_p)]


class SkrResult(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int32), ("cycles", ctypes.c_int32), ("matvecs", ctypes.c_int32),
                ("refinements", ctypes.c_int32), ("flag", ctypes.c_int32),
                ("k_final", ctypes.c_int32), ("relres", ctypes.c_double),
                ("seconds", ctypes.c_double), ("delta", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class SkrServerInfo(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("queued", ctypes.c_int64), ("running", ctypes.c_int64), ("chains", ctypes.c_int32),
                ("evicted", ctypes.c_int32), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("mean_ms", ctypes.c_double), ("hbm_bytes", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


if not os.path.exists(LIB_PATH):
    raise ImportError(
        "libskr.so is not built (expected at %s); run __graft_entry__.build() "
        "or python -m paper_2401_09516_gb300.build" % LIB_PATH)

_lib = ctypes.CDLL(LIB_PATH)
_i32, _i64, _vp, _dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_double

_lib.skr_options_default.argtypes = [ctypes.POINTER(SkrOptions)]
_lib.skr_sort.argtypes = [_vp, _i64, _i64, _i64, _i32, _vp, _vp]
_lib.skr_sort_noalloc.argtypes = [_vp, _i64, _i64, _i64, _vp, _vp]
_lib.skr_sort_grouped.argtypes = [_vp, _i64, _i64, _i64, _i32, _vp, _vp, _vp, _vp]
_lib.skr_solve_sequence.argtypes = [ctypes.POINTER(SkrSystem), _i64, _vp, _vp, _i32,
                                    ctypes.POINTER(SkrOptions), ctypes.POINTER(_vp),
                                    ctypes.POINTER(SkrResult)]
_lib.skr_assemble.argtypes = [ctypes.POINTER(SkrSystem), _i32, _vp, _vp, _vp]
_lib.skr_apply.argtypes = [ctypes.POINTER(SkrSystem), _i32, _i32, _i32, _vp, _vp, _i32, _vp]
_lib.skr_last_stats.argtypes = [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i32)]
_lib.skr_last_profile.argtypes = [ctypes.POINTER(ctypes.c_double), _i32]
_lib.skr_last_plan.argtypes = [_vp, _vp, _vp, _i32, ctypes.POINTER(_i32)]
_lib.skr_release_workspace.argtypes = []
_lib.skr_server_create.argtypes = [ctypes.POINTER(SkrOptions), ctypes.c_size_t, _i32, ctypes.POINTER(_vp)]
_lib.skr_submit.argtypes = [_vp, ctypes.POINTER(SkrSystem), _vp, _i64, ctypes.POINTER(ctypes.c_uint64)]
_lib.skr_poll.argtypes = [_vp, ctypes.c_uint64, _vp, ctypes.POINTER(SkrResult)]
_lib.skr_server_stats.argtypes = [_vp, ctypes.POINTER(SkrServerInfo)]
_lib.skr_server_destroy.argtypes = [_vp]
_lib.skr_last_error.argtypes = []
_lib.skr_last_error.restype = ctypes.c_char_p
for _fn in ("skr_options_default", "skr_sort", "skr_sort_noalloc", "skr_sort_grouped", "skr_solve_sequence", "skr_assemble", "skr_apply",
            "skr_last_stats", "skr_last_profile", "skr_last_plan", "skr_release_workspace", "skr_server_create",
            "skr_submit", "skr_poll", "skr_server_stats", "skr_server_destroy"):
    getattr(_lib, _fn).restype = ctypes.c_int32


class SkrError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("skr status %d: %s" % (status, msg))
        self.status = status


def _check(status):
    if status != SKR_OK:
        raise SkrError(status, _lib.skr_last_error().decode())
    return status


def _is_device(x):
    return hasattr(x, "is_cuda") and x.is_cuda


def _ptr(x):
    if x is None:
        return None
    if _is_device(x):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError("expected a numpy array or a CUDA tensor, got %r" % type(x))


def _mem_of(*arrays):
    kinds = {_is_device(a) for a in arrays if a is not None}
    if len(kinds) > 1:
        raise ValueError("all arrays of one call must be on the host or all on the device")
    return SKR_MEM_DEVICE if kinds == {True} else SKR_MEM_HOST


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _f64(a):
    if _is_device(a):
        if str(a.dtype) != "torch.float64" or not a.is_contiguous():
            raise ValueError("device arrays must be contiguous float64")
        return a
    return np.ascontiguousarray(a, dtype=np.float64)


def _int(a, bits):
    if _is_device(a):
        want = "torch.int64" if bits == 64 else "torch.int32"
        if str(a.dtype) != want or not a.is_contiguous():
            raise ValueError("device index arrays must be contiguous int%d" % bits)
        return a
    return np.ascontiguousarray(a, dtype=np.int64 if bits == 64 else np.int32)


def skr_last_error():
    return _lib.skr_last_error().decode()


def skr_options_default(**overrides):
    """SkrOptions with the library defaults, then the given fields overridden.

    precond / precision accept the names "none"/"jacobi"/"ilu0" and
    "fp64"/"mixed"; stream accepts a torch stream or a raw handle.
    """
    opt = SkrOptions()
    _check(_lib.skr_options_default(ctypes.byref(opt)))
    for key, val in overrides.items():
        if key == "precond" and isinstance(val, str):
            val = PRECOND[val]
        if key == "precision" and isinstance(val, str):
            val = PRECISION[val]
        if key == "stream":
            val = _stream_handle(val)
        setattr(opt, key, val)
    return opt


class System:
    """One system of the sequence; keeps its arrays alive for the call."""

    def __init__(self, fmt, nx, ny, nz=1, coef=None, rhs=None, params=(0.0, 0.0, 0.0, 0.0), rowptr=None,
                 colind=None):
        self.coef = None if coef is None else _f64(coef)
        self.rhs = None if rhs is None else _f64(rhs)
        self.rowptr = None if rowptr is None else _int(rowptr, 64)
        self.colind = None if colind is None else _int(colind, 32)
        self.fmt, self.nx, self.ny, self.nz = int(fmt), int(nx), int(ny), int(nz)
        self.params = tuple(float(p) for p in params) + (0.0,) * (4 - len(params))
        self.n = self.nx * self.ny * (self.nz if fmt in (SKR_FMT_DARCY3D, SKR_FMT_STENCIL7) else 1)

    def struct(self):
        s = SkrSystem()
        s.fmt, s.nx, s.ny, s.nz = self.fmt, self.nx, self.ny, self.nz
        s.coef = _ptr(self.coef)
        s.rhs = _ptr(self.rhs)
        s.rowptr = _ptr(self.rowptr)
        s.colind = _ptr(self.colind)
        for i in range(4):
            s.params[i] = self.params[i]
        return s

    def arrays(self):
        return [self.coef, self.rhs, self.rowptr, self.colind]


def darcy2d(loga, rhs=None):
    """System from log a on the (nx+2) x (ny+2) node grid."""
    return System(SKR_FMT_DARCY2D, loga.shape[0] - 2, loga.shape[1] - 2, 1, loga, rhs)


def darcy3d(loga, rhs=None):
    return System(SKR_FMT_DARCY3D, loga.shape[0] - 2, loga.shape[1] - 2, loga.shape[2] - 2, loga, rhs)


def helmholtz2d(k, rhs=None):
    """System -lap u - k^2 u = f from the wavenumber k at the nx x ny interior nodes."""
    return System(SKR_FMT_HELMHOLTZ2D, k.shape[0], k.shape[1], 1, k, rhs)


def poisson2d(f, g):
    """System lap u = f with Dirichlet data (Sec. 3.1 sign).

    f: nx x ny values at the interior nodes; g = (g_x0, g_x1, g_y0, g_y1):
    u on the lines x = 0 and x = 1 (ny values each) and y = 0, y = 1 (nx
    values each).  Host (numpy) or device (torch) arrays, all on one side.
    """
    nx, ny = f.shape
    parts = [f.reshape(-1)] + [gi.reshape(-1) for gi in g]
    if isinstance(f, np.ndarray):
        coef = np.concatenate([np.asarray(t, dtype=np.float64) for t in parts])
    else:
        import torch
        coef = torch.cat([t.to(torch.float64) for t in parts])
    return System(SKR_FMT_POISSON2D, nx, ny, 1, coef, None)


def csr(indptr, indices, data, rhs=None):
    """System from an assembled sparse matrix in CSR form (e.g. a scipy
    csr_matrix's indptr, indices, data): at most SKR_CSR_MAX_ROW entries per
    row, the diagonal among them.  Host (numpy) or device (torch) arrays."""
    n = int(indptr.shape[0]) - 1
    return System(SKR_FMT_CSR, n, 1, 1, data, rhs, rowptr=indptr, colind=indices)


def convdiff2d(nu, beta, nside, rhs=None):
    return System(SKR_FMT_CONVDIFF2D, nside, nside, 1, None, rhs, (nu, beta[0], beta[1], 0.0))


def skr_sort(params, start=0, stream=None):
    """Algorithm 1 order of the rows of params (N x p float64)."""
    P = _f64(params)
    N = int(P.shape[0])
    p = int(np.prod(P.shape[1:])) if N else 1
    mem = _mem_of(P)
    if mem == SKR_MEM_DEVICE:
        import torch
        perm = torch.empty(N, dtype=torch.int32, device=P.device)
    else:
        perm = np.empty(N, dtype=np.int32)
    _check(_lib.skr_sort(_ptr(P) if N else None, N, p, int(start), mem, _stream_handle(stream),
                         _ptr(perm) if N else None))
    return perm


def skr_sort_grouped(params, group_max, stream=None):
    """Large-N order (Sec. 4.1): coordinate groups of at most group_max
    systems, Algorithm 1 inside each, concatenated.

    Returns (perm, offsets): perm like skr_sort's (same memory as params),
    offsets a host int64 array of ngroups + 1 group boundaries in perm.
    """
    P = _f64(params)
    N = int(P.shape[0])
    p = int(np.prod(P.shape[1:])) if N else 1
    mem = _mem_of(P)
    if mem == SKR_MEM_DEVICE:
        import torch
        perm = torch.empty(N, dtype=torch.int32, device=P.device)
    else:
        perm = np.empty(N, dtype=np.int32)
    offs = np.zeros(N + 1, dtype=np.int64)
    ng = ctypes.c_int64(0)
    _check(_lib.skr_sort_grouped(_ptr(P) if N else None, N, p, int(group_max), mem, _stream_handle(stream),
                                 _ptr(perm) if N else None, offs.ctypes.data, ctypes.byref(ng)))
    return perm, offs[:ng.value + 1].copy()


SKR_SORT_NOALLOC_MAX_N = 512


def skr_sort_noalloc(params, start=0, stream=None):
    """skr_sort without device allocation, for callers that cannot allocate.

    params must be a CUDA tensor (N x p float64, N <= SKR_SORT_NOALLOC_MAX_N);
    returns the order as an int32 CUDA tensor.  The scratch is a fixed array
    the library keeps on every device; calls that overlap on the GPU race on
    it, so callers serialise them.
    """
    P = _f64(params)
    if not _is_device(P):
        raise ValueError("skr_sort_noalloc takes device arrays only")
    import torch
    N = int(P.shape[0])
    p = int(np.prod(P.shape[1:])) if N else 1
    perm = torch.empty(N, dtype=torch.int32, device=P.device)
    _check(_lib.skr_sort_noalloc(_ptr(P) if N else None, N, p, int(start), _stream_handle(stream),
                                 _ptr(perm) if N else None))
    return perm


def skr_solve_sequence(systems, order=None, chain_offsets=None, nchains=1, options=None, x_out=None,
                       recycle_out=None):
    """Solve the systems in `order` with recycling along each chain.

    recycle_out: None, or one contiguous float64 CUDA tensor per chain of at
    least 2 k n elements, receiving the chain's final U_k (columns 0..k-1)
    and C_k (columns k..2k-1), column-major (skr_options.recycle_out).
    Returns (x_out, results): x_out is a list of n-vectors (numpy on the
    host path, tensors on the device path), results a list of dicts.
    """
    N = len(systems)
    arrays = [a for s in systems for a in s.arrays()]
    if x_out is not None:
        arrays += list(x_out)
    mem = _mem_of(*arrays)
    opt = options if options is not None else skr_options_default()
    opt.mem = mem
    if x_out is None:
        if mem == SKR_MEM_DEVICE:
            import torch
            dev = next(a.device for a in arrays if a is not None)
            x_out = [torch.empty(s.n, dtype=torch.float64, device=dev) for s in systems]
        else:
            x_out = [np.empty(s.n) for s in systems]
    rec = None
    if recycle_out is not None:
        if len(recycle_out) != int(nchains) or not all(_is_device(t) for t in recycle_out):
            raise ValueError("recycle_out needs one CUDA tensor per chain")
        rec = (_vp * len(recycle_out))(*[_f64(t).data_ptr() for t in recycle_out])
        opt.recycle_out = ctypes.cast(rec, _vp)
    sysarr = (SkrSystem * max(N, 1))(*[s.struct() for s in systems])
    xptr = (_vp * max(N, 1))(*[_ptr(x) for x in x_out])
    res = (SkrResult * max(N, 1))()
    ordv = None if order is None else np.ascontiguousarray(order, dtype=np.int32)
    offv = None if chain_offsets is None else np.ascontiguousarray(chain_offsets, dtype=np.int64)
    try:
        _check(_lib.skr_solve_sequence(sysarr, N, None if ordv is None else ordv.ctypes.data,
                                       None if offv is None else offv.ctypes.data, int(nchains),
                                       ctypes.byref(opt), xptr, res))
    finally:
        if rec is not None:
            opt.recycle_out = None
    return x_out, [res[i].as_dict() for i in range(N)]


def skr_assemble(system, stream=None):
    """(A as nst x n stencil arrays, b) built by the device assembly."""
    mem = _mem_of(*system.arrays())
    nst = 7 if system.fmt in (SKR_FMT_DARCY3D, SKR_FMT_STENCIL7) else 5
    if mem == SKR_MEM_DEVICE:
        import torch
        dev = next(a.device for a in system.arrays() if a is not None)
        coef = torch.empty((nst, system.n), dtype=torch.float64, device=dev)
        rhs = torch.empty(system.n, dtype=torch.float64, device=dev)
    else:
        coef = np.empty((nst, system.n))
        rhs = np.empty(system.n)
    s = system.struct()
    _check(_lib.skr_assemble(ctypes.byref(s), mem, _stream_handle(stream), _ptr(coef), _ptr(rhs)))
    return coef, rhs


def skr_apply(system, v, precond="none", precision="fp64", stream=None, pc_blocks=1):
    """y = A M^-1 v with the solver's operator code (pc_blocks: block-Jacobi's block count)."""
    v = _f64(v)
    mem = _mem_of(v, *system.arrays())
    if mem == SKR_MEM_DEVICE:
        import torch
        y = torch.empty_like(v)
    else:
        y = np.empty_like(v)
    s = system.struct()
    _check(_lib.skr_apply(ctypes.byref(s), PRECOND.get(precond, precond), int(pc_blocks),
                          PRECISION.get(precision, precision), _ptr(v), _ptr(y), mem,
                          _stream_handle(stream)))
    return y


def skr_last_stats():
    b = ctypes.c_uint64()
    ms = ctypes.c_double()
    cs, sl, ln = _i32(), _i32(), _i32()
    _check(_lib.skr_last_stats(ctypes.byref(b), ctypes.byref(ms), ctypes.byref(cs), ctypes.byref(sl),
                               ctypes.byref(ln)))
    return {"bytes": b.value, "kernel_ms": ms.value, "cluster_size": cs.value, "slots": sl.value,
            "launches": ln.value}


def skr_last_plan():
    """Launches of the last skr_solve_sequence call: a list of
    {"cluster_size", "clusters", "chains"} dicts."""
    cap = 16
    cs = (ctypes.c_int32 * cap)()
    cl = (ctypes.c_int32 * cap)()
    ch = (ctypes.c_int32 * cap)()
    n = _i32()
    _check(_lib.skr_last_plan(ctypes.addressof(cs), ctypes.addressof(cl), ctypes.addressof(ch), cap,
                              ctypes.byref(n)))
    return [{"cluster_size": cs[i], "clusters": cl[i], "chains": ch[i]} for i in range(min(cap, n.value))]


PHASES = ["assembly", "refresh", "projection", "operator", "multidot", "update", "gram", "dense",
          "cycle_update", "true_residual", "other", "schur", "eigenvectors", "hessenberg"]


def skr_last_profile():
    """Per-phase device time (ms) of the last profiled skr_solve_sequence call."""
    arr = (ctypes.c_double * len(PHASES))()
    _check(_lib.skr_last_profile(arr, len(PHASES)))
    return {name: arr[i] * 1e-6 for i, name in enumerate(PHASES)}


def skr_release_workspace():
    _check(_lib.skr_release_workspace())


def skr_server_create(options=None, hbm_budget=0, max_chains=0):
    """Start a serving loop; returns an opaque handle (see Server)."""
    opt = options if options is not None else skr_options_default()
    h = _vp()
    _check(_lib.skr_server_create(ctypes.byref(opt), int(hbm_budget), int(max_chains), ctypes.byref(h)))
    return h


def skr_submit(server, system, key=None):
    """Enqueue one system (host arrays); returns its ticket."""
    for a in system.arrays():
        if a is not None and _is_device(a):
            raise ValueError("skr_submit takes host arrays")
    k = None if key is None else np.ascontiguousarray(key, dtype=np.float64).reshape(-1)
    s = system.struct()
    t = ctypes.c_uint64()
    _check(_lib.skr_submit(server, ctypes.byref(s), None if k is None else k.ctypes.data,
                           0 if k is None else k.size, ctypes.byref(t)))
    return t.value


def skr_poll(server, ticket, n):
    """(x, result) once the request is done, else None."""
    x = np.empty(n)
    r = SkrResult()
    st = _lib.skr_poll(server, ctypes.c_uint64(ticket), x.ctypes.data, ctypes.byref(r))
    if st == SKR_NOT_READY:
        return None
    _check(st)
    return x, r.as_dict()


def skr_server_stats(server):
    info = SkrServerInfo()
    _check(_lib.skr_server_stats(server, ctypes.byref(info)))
    return info.as_dict()


def skr_server_destroy(server):
    _check(_lib.skr_server_destroy(server))


class Server:
    """Context-managed serving loop over skr_server_* (marshalling only)."""

    def __init__(self, options=None, hbm_budget=0, max_chains=0):
        self.handle = skr_server_create(options, hbm_budget, max_chains)
        self._n = {}

    def submit(self, system, key=None):
        t = skr_submit(self.handle, system, key)
        self._n[t] = system.n
        return t

    def poll(self, ticket):
        out = skr_poll(self.handle, ticket, self._n[ticket])
        if out is not None:
            del self._n[ticket]
        return out

    def wait(self, ticket, timeout=120.0):
        import time
        t0 = time.time()
        while True:
            out = self.poll(ticket)
            if out is not None:
                return out
            if time.time() - t0 > timeout:
                raise TimeoutError("request %d not done after %.0f s" % (ticket, timeout))
            time.sleep(0.0005)

    def stats(self):
        return skr_server_stats(self.handle)

    def close(self):
        if self.handle is not None:
            skr_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def exported_symbols():
    """Names of the C functions this binding wraps."""
    return ["skr_options_default", "skr_sort", "skr_sort_noalloc", "skr_sort_grouped", "skr_solve_sequence", "skr_assemble", "skr_apply",
            "skr_last_stats", "skr_last_profile", "skr_last_plan", "skr_release_workspace", "skr_last_error",
            "skr_server_create", "skr_submit", "skr_poll", "skr_server_stats", "skr_server_destroy"]


def library():
    return _lib
