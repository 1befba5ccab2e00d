"""Python binding of libilu (include/ilu.h): the GB300 matrix-free surrogate
ILU(0) smoother of arXiv 2210.15280.

Argument marshalling only: every step of set-up and smoothing runs in the
library (host FP64 set-up in C++, sweeps in CUDA kernels for sm_103a).  There
is no Python or CPU fallback: if libilu.so cannot be loaded, every call raises.
Device vectors are torch CUDA tensors (data_ptr is passed through); host
vectors are numpy arrays.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libilu.so")
_lib = None

ILU_OK, ILU_EINVAL, ILU_ENOMEM, ILU_ECUDA, ILU_ESINGULAR, ILU_ENOTCONV, ILU_ETIMEOUT, ILU_EBUSY, ILU_ENODEV = range(9)
F64, F32, MIXED = 0, 1, 2
COEFF_CONST, COEFF_SINPROD, COEFF_KAPPA_I = 0, 1, 2
RICHARDSON, PCG, MG_VCYCLE, MG_PCG = 0, 1, 2, 3
KERNEL_AUTO, KERNEL_SLAB, KERNEL_BAND, KERNEL_PACKED = 0, 1, 2, 3
FACTOR_ILU0, FACTOR_SGS = 0, 1
STENCIL_AUTO, STENCIL_ON_THE_FLY, STENCIL_STORED = 0, 1, 2
VALUES_AUTO, VALUES_ON_THE_FLY, VALUES_TABULATED = 0, 1, 2
ORIENT_GIVEN, ORIENT_LFA = 0, 1
BOUNDARY_V2, BOUNDARY_V1 = 0, 1
STATUS_NAMES = ["ILU_OK", "ILU_EINVAL", "ILU_ENOMEM", "ILU_ECUDA", "ILU_ESINGULAR", "ILU_ENOTCONV",
                "ILU_ETIMEOUT", "ILU_EBUSY", "ILU_ENODEV"]

# every symbol include/ilu.h declares
EXPORTS = [
    "ilu_opts_default", "ilu_setup", "ilu_destroy", "ilu_import_surrogate", "ilu_export_surrogate",
    "ilu_surrogate_size", "ilu_eval_surrogate", "ilu_exact_factor", "ilu_stencil", "ilu_smooth",
    "ilu_smooth_host", "ilu_residual", "ilu_solve", "ilu_batch_create", "ilu_batch_destroy",
    "ilu_batch_smooth", "ilu_batch_launches", "ilu_server_create", "ilu_server_submit", "ilu_server_wait", "ilu_server_release",
    "ilu_server_stats", "ilu_server_destroy", "ilu_num_nodes", "ilu_num_interior", "ilu_index",
    "ilu_last_error", "ilu_version", "ilu_profile_enable", "ilu_profile_read", "ilu_residual_noalloc",
    "ilu_mg_setup", "ilu_mg_destroy", "ilu_mg_level", "ilu_mg_cycle", "ilu_mg_solve", "ilu_mg_rate",
    "ilu_lfa_order", "ilu_vertex_order", "ilu_packed_schedule", "ilu_partition", "ilu_step_floor",
]


class IluError(RuntimeError):
    def __init__(self, status, msg):
        self.status = status
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")


class Coeff(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("c0", ctypes.c_double), ("amp", ctypes.c_double), ("ipow", ctypes.c_int)]


class Opts(ctypes.Structure):
    _fields_ = [("deg", ctypes.c_int * 3), ("sample_level", ctypes.c_int), ("ridge", ctypes.c_double),
                ("precision", ctypes.c_int), ("slabs", ctypes.c_int), ("device", ctypes.c_int),
                ("max_wait_spins", ctypes.c_longlong), ("kernel", ctypes.c_int), ("factor", ctypes.c_int),
                ("stencil", ctypes.c_int), ("orient", ctypes.c_int), ("boundary", ctypes.c_int),
                ("max_cluster", ctypes.c_int), ("values", ctypes.c_int)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_double), ("max_slots", ctypes.c_int), ("device", ctypes.c_int),
                ("precision", ctypes.c_int), ("max_cluster", ctypes.c_int)]


class Request(ctypes.Structure):
    _fields_ = [("macro_tet", ctypes.c_double * 12), ("level", ctypes.c_int), ("coeff", Coeff),
                ("poly_degree", ctypes.c_int), ("method", ctypes.c_int), ("rtol", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("b", ctypes.c_void_p), ("x0", ctypes.c_void_p),
                ("orient", ctypes.c_int), ("boundary", ctypes.c_int)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("rel_res", ctypes.c_double),
                ("latency_ms", ctypes.c_double), ("x", ctypes.c_void_p), ("n", ctypes.c_size_t)]


class Stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong), ("failed", ctypes.c_longlong),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("solves_per_s", ctypes.c_double),
                ("max_concurrent", ctypes.c_int)]


def build(force=False, verbose=False):
    from . import buildlib as _b
    return _b.build(force=force, verbose=verbose)


def lib():
    """Load libilu.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_SO):
            raise RuntimeError(f"libilu.so not built ({_SO}); run paper_2210_15280_gb300.build()")
        L = ctypes.CDLL(_SO)
        vp, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
        P = ctypes.POINTER
        L.ilu_opts_default.argtypes = [P(Opts)]
        L.ilu_setup.argtypes = [P(ctypes.c_double * 12), i, P(Coeff), i, P(Opts), P(vp)]
        L.ilu_destroy.argtypes = [vp]
        L.ilu_import_surrogate.argtypes = [vp, vp, sz]
        L.ilu_export_surrogate.argtypes = [vp, vp, sz]
        L.ilu_surrogate_size.argtypes = [vp]; L.ilu_surrogate_size.restype = sz
        L.ilu_eval_surrogate.argtypes = [vp, i, i, i, vp]
        L.ilu_exact_factor.argtypes = [vp, i, i, i, vp]
        L.ilu_stencil.argtypes = [vp, i, i, i, vp]
        L.ilu_smooth.argtypes = [vp, vp, vp, i, vp, vp]
        L.ilu_smooth_host.argtypes = [vp, vp, vp, i, vp]
        L.ilu_residual.argtypes = [vp, vp, vp, vp, vp, vp]
        L.ilu_residual_noalloc.argtypes = [vp, vp, vp, vp, vp, vp]
        L.ilu_solve.argtypes = [vp, vp, vp, i, d, i, vp, vp, vp]
        L.ilu_batch_create.argtypes = [vp, i, P(Opts), P(vp)]
        L.ilu_batch_destroy.argtypes = [vp]
        L.ilu_batch_smooth.argtypes = [vp, vp, vp, i, vp]
        L.ilu_batch_launches.argtypes = [vp, P(i)]
        L.ilu_server_create.argtypes = [P(ServerOpts), P(vp)]
        L.ilu_server_submit.argtypes = [vp, P(Request), P(ctypes.c_uint64)]
        L.ilu_server_wait.argtypes = [vp, ctypes.c_uint64, i, P(Result)]
        L.ilu_server_release.argtypes = [vp, ctypes.c_uint64]
        L.ilu_server_stats.argtypes = [vp, P(Stats)]
        L.ilu_server_destroy.argtypes = [vp]
        L.ilu_mg_setup.argtypes = [P(ctypes.c_double * 12), i, P(Coeff), i, i, P(Opts), P(vp)]
        L.ilu_mg_destroy.argtypes = [vp]
        L.ilu_mg_level.argtypes = [vp, i, P(vp)]
        L.ilu_mg_cycle.argtypes = [vp, vp, vp, i, vp, vp]
        L.ilu_mg_solve.argtypes = [vp, vp, vp, i, d, i, vp, vp, vp]
        L.ilu_mg_rate.argtypes = [vp, vp, i, vp, vp, vp]
        L.ilu_lfa_order.argtypes = [P(ctypes.c_double * 12), vp, vp, vp]
        L.ilu_vertex_order.argtypes = [vp, vp]
        L.ilu_profile_enable.argtypes = [vp, i]
        L.ilu_profile_read.argtypes = [vp, vp, P(ctypes.c_longlong)]
        L.ilu_num_nodes.argtypes = [i]; L.ilu_num_nodes.restype = sz
        L.ilu_packed_schedule.argtypes = [i, i, i, i, vp, vp, vp, vp]
        L.ilu_partition.argtypes = [i, vp, i, vp, vp]
        L.ilu_step_floor.argtypes = [i, i, i, vp]
        L.ilu_num_interior.argtypes = [i]; L.ilu_num_interior.restype = sz
        L.ilu_index.argtypes = [i, i, i, i]; L.ilu_index.restype = ctypes.c_longlong
        L.ilu_last_error.restype = ctypes.c_char_p
        L.ilu_version.restype = ctypes.c_char_p
        for name in EXPORTS:
            if name not in ("ilu_surrogate_size", "ilu_num_nodes", "ilu_num_interior", "ilu_index",
                            "ilu_last_error", "ilu_version", "ilu_destroy"):
                getattr(L, name).restype = i
        L.ilu_destroy.restype = i
        _lib = L
    return _lib


def _check(st):
    if st != ILU_OK:
        raise IluError(st, lib().ilu_last_error().decode(errors="replace"))


def step_floor(threads=384, steps=4096, device=0):
    """SM cycles per step of the shortest barrier-synchronised substitution
    step (ilu_step_floor)."""
    c = ctypes.c_double(0.0)
    _check(lib().ilu_step_floor(int(device), int(threads), int(steps), ctypes.byref(c)))
    return c.value


def partition(costs, nranks):
    """Split tets of the given costs over nranks GPUs (ilu_partition, longest
    processing time first): (rank of each tet, load of each rank)."""
    c = np.ascontiguousarray(costs, dtype=np.float64)
    rank_of = np.zeros(len(c), dtype=np.int32)
    load = np.zeros(int(nranks))
    _check(lib().ilu_partition(len(c), _ptr(c), int(nranks), _ptr(rank_of), _ptr(load)))
    return rank_of, load


def packed_schedule(level, forward=True, lanes=0, quantum=0):
    """Row schedule of the packed kernels for one substitution at `level`
    (ilu_packed_schedule): (nsteps, lanes, entries[rows, 8], lane_off)."""
    ns, ln = ctypes.c_int(0), ctypes.c_int(0)
    _check(lib().ilu_packed_schedule(int(level), int(bool(forward)), int(lanes), int(quantum), ctypes.byref(ns),
                                     ctypes.byref(ln), None, None))
    n = 2 ** int(level)
    rows = (n - 3) * (n - 2) // 2 if n >= 4 else 0
    ent = np.zeros((rows, 8), dtype=np.int32)
    off = np.zeros(ln.value + 1, dtype=np.int32)
    _check(lib().ilu_packed_schedule(int(level), int(bool(forward)), int(lanes), int(quantum), ctypes.byref(ns),
                                     ctypes.byref(ln), _ptr(ent), _ptr(off)))
    return ns.value, ln.value, ent, off


def num_nodes(level):
    return int(lib().ilu_num_nodes(level))


def num_interior(level):
    return int(lib().ilu_num_interior(level))


def index(level, x, y, z):
    return int(lib().ilu_index(level, x, y, z))


def _ptr(v):
    """Device pointer of a torch tensor, or host pointer of a numpy array."""
    if v is None:
        return None
    if hasattr(v, "data_ptr"):
        return ctypes.c_void_p(v.data_ptr())
    if isinstance(v, np.ndarray):
        assert v.flags.c_contiguous
        return ctypes.c_void_p(v.ctypes.data)
    return ctypes.c_void_p(int(v))


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def make_opts(deg=None, sample_level=-1, ridge=-1.0, precision=MIXED, slabs=0, device=0, max_wait_spins=0,
              kernel=0, factor=0, stencil=0, orient=0, boundary=0, max_cluster=0, values=0):
    o = Opts()
    lib().ilu_opts_default(ctypes.byref(o))
    if deg is not None:
        d = [deg] * 3 if np.isscalar(deg) else list(deg)
        for k in range(3):
            o.deg[k] = int(d[k])
    o.sample_level, o.ridge, o.precision = int(sample_level), float(ridge), int(precision)
    o.slabs, o.device, o.max_wait_spins = int(slabs), int(device), int(max_wait_spins)
    o.kernel = int(kernel)
    o.factor = int(factor)
    o.stencil = int(stencil)
    o.orient = int(orient)
    o.boundary = int(boundary)
    o.max_cluster = int(max_cluster)
    o.values = int(values)
    return o


def make_coeff(kind="const", c0=1.0, amp=0.0, ipow=0):
    k = {"const": COEFF_CONST, "sinprod": COEFF_SINPROD, "kappa_i": COEFF_KAPPA_I}.get(kind, kind)
    return Coeff(int(k), float(c0), float(amp), int(ipow))


def lfa_order(macro_tet):
    """(perm, mu, mu_all): the vertex order with the smallest LFA smoothing
    factor of the ILU(0) smoother (perm[i] = index of the vertex placed at
    position i), its factor and the factors of all 24 orders."""
    P = (ctypes.c_double * 12)(*np.asarray(macro_tet, dtype=np.float64).reshape(12))
    perm = np.zeros(4, dtype=np.int32)
    mu = np.zeros(1)
    mus = np.zeros(24)
    _check(lib().ilu_lfa_order(ctypes.byref(P), _ptr(perm), _ptr(mu), _ptr(mus)))
    return [int(v) for v in perm], float(mu[0]), mus


class _Handle:
    """`with` support for the handle classes: the handle is released on exit."""

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False


class Tet(_Handle):
    """One macro-tetrahedron set up for smoothing (wraps an ilu_tet handle)."""

    def __init__(self, macro_tet, level, coeff=None, poly_degree=4, **opts):
        P = (ctypes.c_double * 12)(*np.asarray(macro_tet, dtype=np.float64).reshape(12))
        self.level, self.N = int(level), 2 ** int(level)
        self.opts = make_opts(**opts)
        self.precision = self.opts.precision
        h = ctypes.c_void_p()
        c = coeff if coeff is not None else make_coeff()
        _check(lib().ilu_setup(ctypes.byref(P), self.level, ctypes.byref(c), int(poly_degree),
                               ctypes.byref(self.opts), ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().ilu_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def dtype(self):
        return np.float32 if self.precision == F32 else np.float64

    def num_nodes(self):
        return num_nodes(self.level)

    def smooth(self, x, b, sweeps=1, stream=None, norms=False):
        out = np.zeros(max(sweeps, 1)) if norms else None
        _check(lib().ilu_smooth(self.h, _ptr(x), _ptr(b), int(sweeps), _stream(stream),
                                _ptr(out) if norms else None))
        return out[:sweeps] if norms else None

    def smooth_host(self, x, b, sweeps=1, norms=False):
        out = np.zeros(max(sweeps, 1)) if norms else None
        _check(lib().ilu_smooth_host(self.h, _ptr(x), _ptr(b), int(sweeps), _ptr(out) if norms else None))
        return out[:sweeps] if norms else None

    def residual(self, x, b, r=None, stream=None):
        nrm = np.zeros(1)
        _check(lib().ilu_residual(self.h, _ptr(x), _ptr(b), _ptr(r), _ptr(nrm), _stream(stream)))
        return float(nrm[0])

    def residual_noalloc(self, x, b, r, norm_dev, stream=None):
        """r = b - A x and ||r|| into the device double norm_dev; no allocation."""
        _check(lib().ilu_residual_noalloc(self.h, _ptr(x), _ptr(b), _ptr(r), _ptr(norm_dev), _stream(stream)))

    def solve(self, x, b, method=RICHARDSON, rtol=1e-8, max_iter=100000, stream=None):
        it = ctypes.c_int(0)
        rel = ctypes.c_double(0.0)
        st = lib().ilu_solve(self.h, _ptr(x), _ptr(b), int(method), float(rtol), int(max_iter), _stream(stream),
                             ctypes.byref(it), ctypes.byref(rel))
        if st not in (ILU_OK, ILU_ENOTCONV):
            _check(st)
        return it.value, rel.value, st == ILU_OK

    def export_surrogate(self):
        n = int(lib().ilu_surrogate_size(self.h))
        out = np.zeros(n)
        _check(lib().ilu_export_surrogate(self.h, _ptr(out), n))
        return out

    def import_surrogate(self, coefs):
        c = np.ascontiguousarray(coefs, dtype=np.float64).reshape(-1)
        _check(lib().ilu_import_surrogate(self.h, _ptr(c), c.size))

    def eval_surrogate(self, x, y, z):
        out = np.zeros(8)
        _check(lib().ilu_eval_surrogate(self.h, int(x), int(y), int(z), _ptr(out)))
        return out

    def exact_factor(self, x, y, z):
        out = np.zeros(8)
        _check(lib().ilu_exact_factor(self.h, int(x), int(y), int(z), _ptr(out)))
        return out

    def profile(self, enable=True):
        _check(lib().ilu_profile_enable(self.h, 1 if enable else 0))

    def profile_read(self):
        """(ms[residual, forward, backward], launches) since the last read."""
        ms = np.zeros(3)
        n = ctypes.c_longlong(0)
        _check(lib().ilu_profile_read(self.h, _ptr(ms), ctypes.byref(n)))
        return ms, n.value

    def vertex_order(self):
        perm = np.zeros(4, dtype=np.int32)
        _check(lib().ilu_vertex_order(self.h, _ptr(perm)))
        return [int(v) for v in perm]

    def stencil(self, x, y, z):
        out = np.zeros(15)
        _check(lib().ilu_stencil(self.h, int(x), int(y), int(z), _ptr(out)))
        return out


class _Borrowed(Tet):
    """A level handle owned by a multigrid hierarchy (never destroyed here)."""

    def __init__(self, h, level, precision, owner):
        self.h, self.level, self.N, self.precision, self._owner = h, level, 2 ** level, precision, owner

    def close(self):
        self.h = None


class Multigrid(_Handle):
    """Geometric multigrid V-cycle on one macro-tet, levels 2..level, with the
    surrogate smoother on levels >= 3 (wraps an ilu_mg handle)."""

    def __init__(self, macro_tet, level, coeff=None, poly_degree=4, nu=3, **opts):
        P = (ctypes.c_double * 12)(*np.asarray(macro_tet, dtype=np.float64).reshape(12))
        self.level, self.nu = int(level), int(nu)
        self.opts = make_opts(**opts)
        self.precision = self.opts.precision
        h = ctypes.c_void_p()
        c = coeff if coeff is not None else make_coeff()
        _check(lib().ilu_mg_setup(ctypes.byref(P), self.level, ctypes.byref(c), int(poly_degree), self.nu,
                                  ctypes.byref(self.opts), ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().ilu_mg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def tet(self, level):
        """The smoother handle of one level (owned by the hierarchy)."""
        h = ctypes.c_void_p()
        _check(lib().ilu_mg_level(self.h, int(level), ctypes.byref(h)))
        return _Borrowed(h, int(level), self.precision, self)

    def cycle(self, x, b, cycles=1, stream=None, norms=False):
        out = np.zeros(max(cycles, 1)) if norms else None
        _check(lib().ilu_mg_cycle(self.h, _ptr(x), _ptr(b), int(cycles), _stream(stream),
                                  _ptr(out) if norms else None))
        return out[:cycles] if norms else None

    def solve(self, x, b, method=RICHARDSON, rtol=1e-8, max_iter=1000, stream=None):
        it = ctypes.c_int(0)
        rel = ctypes.c_double(0.0)
        st = lib().ilu_mg_solve(self.h, _ptr(x), _ptr(b), int(method), float(rtol), int(max_iter),
                                _stream(stream), ctypes.byref(it), ctypes.byref(rel))
        if st not in (ILU_OK, ILU_ENOTCONV):
            _check(st)
        return it.value, rel.value, st == ILU_OK

    def rate(self, e, steps=20, stream=None):
        """(rho, history) of a power iteration from the start error e (device,
        full grid, boundary 0; overwritten)."""
        rho = ctypes.c_double(0.0)
        hist = np.zeros(steps)
        _check(lib().ilu_mg_rate(self.h, _ptr(e), int(steps), _stream(stream), ctypes.byref(rho), _ptr(hist)))
        return rho.value, hist


class Batch(_Handle):
    """Tets smoothed together (wraps an ilu_batch handle).  Keeps the Tet
    objects alive for as long as the batch exists."""

    def __init__(self, tets, slabs=0, max_wait_spins=0):
        self.tets = list(tets)
        arr = (ctypes.c_void_p * len(self.tets))(*[t.h.value for t in self.tets])
        o = make_opts(slabs=slabs, max_wait_spins=max_wait_spins)
        h = ctypes.c_void_p()
        _check(lib().ilu_batch_create(arr, len(self.tets), ctypes.byref(o), ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().ilu_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def smooth(self, xs, bs, sweeps=1, stream=None):
        n = len(self.tets)
        assert len(xs) == n and len(bs) == n
        xa = (ctypes.c_void_p * n)(*[None if v is None else _ptr(v).value for v in xs])
        ba = (ctypes.c_void_p * n)(*[None if v is None else _ptr(v).value for v in bs])
        _check(lib().ilu_batch_smooth(self.h, xa, ba, int(sweeps), _stream(stream)))

    def launches_per_sweep(self):
        """How many kernels one sweep of the batch launches."""
        n = ctypes.c_int(0)
        _check(lib().ilu_batch_launches(self.h, ctypes.byref(n)))
        return n.value


class Server(_Handle):
    """The request loop (wraps an ilu_server handle): submit interior solves,
    wait for their results; the loop admits them by free device memory and
    runs admitted solves concurrently."""

    def __init__(self, budget_bytes=0.0, max_slots=0, device=0, precision=MIXED, max_cluster=0):
        o = ServerOpts(float(budget_bytes), int(max_slots), int(device), int(precision), int(max_cluster))
        h = ctypes.c_void_p()
        _check(lib().ilu_server_create(ctypes.byref(o), ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().ilu_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, macro_tet, level, b, coeff=None, poly_degree=4, method=MG_VCYCLE, rtol=1e-8,
               max_iter=10000, x0=None, orient=ORIENT_GIVEN, boundary=BOUNDARY_V2):
        """Queue an interior solve; returns its ticket.  The default method is
        the V(3,3) multigrid cycle with the surrogate ILU(0) smoother: smoothed
        Richardson alone needs hundreds to thousands of sweeps per request."""
        r = Request()
        r.macro_tet[:] = [float(v) for v in np.asarray(macro_tet, dtype=np.float64).reshape(12)]
        r.level = int(level)
        r.coeff = coeff if coeff is not None else make_coeff()
        r.poly_degree, r.method, r.rtol, r.max_iter = int(poly_degree), int(method), float(rtol), int(max_iter)
        r.orient, r.boundary = int(orient), int(boundary)
        bb = np.ascontiguousarray(b, dtype=np.float64)
        xx = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float64)
        if bb.size != num_nodes(level) or (xx is not None and xx.size != num_nodes(level)):
            raise ValueError("b and x0 must hold num_nodes(level) values")
        r.b = bb.ctypes.data
        r.x0 = None if xx is None else xx.ctypes.data
        tk = ctypes.c_uint64(0)
        _check(lib().ilu_server_submit(self.h, ctypes.byref(r), ctypes.byref(tk)))  # copies b and x0
        return tk.value

    def wait(self, ticket, timeout_ms=-1, release=True):
        """dict(status, iters, rel_res, latency_ms, x); x is a copy (None on failure)."""
        res = Result()
        _check(lib().ilu_server_wait(self.h, ctypes.c_uint64(ticket), int(timeout_ms), ctypes.byref(res)))
        x = None
        if res.x:
            x = np.ctypeslib.as_array(ctypes.cast(res.x, ctypes.POINTER(ctypes.c_double)), shape=(res.n,)).copy()
        out = dict(status=res.status, iters=res.iters, rel_res=res.rel_res, latency_ms=res.latency_ms, x=x)
        if release:
            _check(lib().ilu_server_release(self.h, ctypes.c_uint64(ticket)))
        return out

    def stats(self):
        s = Stats()
        _check(lib().ilu_server_stats(self.h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in Stats._fields_}
