"""Thin Python binding of libgeo.so (include/geo.h): argument marshalling only.

Every step of the likelihood runs in the library's CUDA kernels; torch is used
only to own device memory and to name the current stream.  Importing this
module loads the in-tree shared library and raises if it is missing: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgeo.so")

GEO_OK = 0
GEO_ERR_NOT_SPD = 1
GEO_ERR_TIMEOUT = 2
GEO_ERR_CUDA = 3
GEO_ERR_UNSUPPORTED = 4
GEO_ERR_TOO_LARGE = 5
GEO_NOALLOC_MAX_N = 262144
GEO_NOALLOC_MAX_P = 4096
GEO_LP_SPLIT_BF16 = 0
GEO_LP_FP32 = 1
GEO_FLAG_FP64_OFFBAND_GEN = 1
GEO_FLAG_STEPWISE = 2
GEO_FLAG_FP64_DMMA = 4
GEO_FLAG_DST = 8
GEO_FLAG_TEST_STALL = 16
GEO_DEFAULT_TIMEOUT_NS = 10_000_000_000
GEO_MIN_CTAS = 4             # fewest CTAs of a partial batch launch (Batch(ctas=...))


class GeoError(RuntimeError):
    def __init__(self, code: int, what: str, info: int = 0):
        super().__init__(f"{what} failed with code {code}" + (f" (info={info})" if info else ""))
        self.code = code
        self.info = info


class NotSPDError(GeoError):
    pass


class geo_theta(ctypes.Structure):
    _fields_ = [("sigma2", ctypes.c_double), ("beta", ctypes.c_double),
                ("nu", ctypes.c_double), ("nugget", ctypes.c_double)]


class geo_layout(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("nb", ctypes.c_int), ("p", ctypes.c_int), ("band", ctypes.c_int),
                ("lp_mode", ctypes.c_int), ("pp", ctypes.c_int),
                ("n_dp_tiles", ctypes.c_longlong), ("n_sp_tiles", ctypes.c_longlong),
                ("n_slots", ctypes.c_longlong),
                ("bytes_dp", ctypes.c_size_t), ("bytes_sp", ctypes.c_size_t),
                ("bytes_planes", ctypes.c_size_t), ("bytes_meta", ctypes.c_size_t)]


class geo_tiles(ctypes.Structure):
    _fields_ = [("lay", geo_layout), ("d_dp", ctypes.c_void_p), ("d_sp", ctypes.c_void_p),
                ("d_planes", ctypes.c_void_p), ("d_meta", ctypes.c_void_p),
                ("aux_stream", ctypes.c_void_p), ("ev_fork", ctypes.c_void_p), ("ev_join", ctypes.c_void_p),
                ("tmap", ctypes.c_uint64 * 48), ("flags", ctypes.c_int),
                ("trace", ctypes.c_void_p), ("trace_cap", ctypes.c_longlong),
                ("timeout_ns", ctypes.c_longlong), ("far_products", ctypes.c_int)]


class geo_mle_opts(ctypes.Structure):
    _fields_ = [("max_evals", ctypes.c_int), ("profile", ctypes.c_int), ("fix_nu", ctypes.c_int),
                ("xtol", ctypes.c_double), ("step", ctypes.c_double),
                ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("journal", ctypes.c_void_p), ("journal_cap", ctypes.c_int),
                ("journal_len", ctypes.POINTER(ctypes.c_int))]


class geo_mle_result(ctypes.Structure):
    _fields_ = [("theta", geo_theta), ("loglik", ctypes.c_double), ("evals", ctypes.c_int),
                ("iterations", ctypes.c_int), ("not_spd", ctypes.c_int)]


class geo_batch_item(ctypes.Structure):
    _fields_ = [("t", ctypes.POINTER(geo_tiles)), ("d_x", ctypes.c_void_p), ("d_y", ctypes.c_void_p),
                ("d_z", ctypes.c_void_p)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libgeo.so not built at {LIB_PATH}; run paper_2003_05324_b300/build.py")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "geo_morton_order": [P, P, I, P],
        "geo_layout_init": [I, I, I, I, ctypes.POINTER(geo_layout)],
        "geo_tiles_bind": [ctypes.POINTER(geo_tiles), ctypes.POINTER(geo_layout), P, P, P, P, P],
        "geo_tiles_release": [ctypes.POINTER(geo_tiles)],
        "geo_tiles_set_flags": [ctypes.POINTER(geo_tiles), I],
        "geo_tiles_set_timeout_ns": [ctypes.POINTER(geo_tiles), ctypes.c_longlong],
        "geo_tiles_set_trace": [ctypes.POINTER(geo_tiles), P, ctypes.c_longlong],
        "geo_tiles_set_far": [ctypes.POINTER(geo_tiles), I, P, P, D, I, P],
        "geo_matern_tiles": [ctypes.POINTER(geo_tiles), P, P, geo_theta, P],
        "geo_tiles_load_dense": [ctypes.POINTER(geo_tiles), P, P],
        "geo_tiles_to_dense": [ctypes.POINTER(geo_tiles), P, P],
        "geo_potrf_mp": [ctypes.POINTER(geo_tiles), P],
        "geo_logdet_trsv": [ctypes.POINTER(geo_tiles), P, P, P, P, P],
        "geo_logdet_trsv_noalloc": [ctypes.POINTER(geo_tiles), P, P, P, P],
        "geo_status": [ctypes.POINTER(geo_tiles), ctypes.POINTER(I), ctypes.POINTER(I), P],
        "geo_loglik": [ctypes.POINTER(geo_tiles), P, P, P, geo_theta, ctypes.POINTER(D), ctypes.POINTER(I), P],
        "geo_loglik_async": [ctypes.POINTER(geo_tiles), P, P, P, geo_theta, P, P],
        "geo_krige": [ctypes.POINTER(geo_tiles), P, P, P, geo_theta, P, P, I, P, P, P],
        "geo_batch_workspace": [I, ctypes.POINTER(geo_batch_item), ctypes.POINTER(ctypes.c_size_t)],
        "geo_batch_bind": [I, ctypes.POINTER(geo_batch_item), P, ctypes.c_size_t, P],
        "geo_loglik_batch": [I, ctypes.POINTER(geo_batch_item), P, P, P, P, P],
        "geo_batch_set_ctas": [P, I],
        "geo_batch_release": [P],
        "geo_mle_default_opts": [ctypes.POINTER(geo_mle_opts)],
        "geo_mle": [ctypes.POINTER(geo_tiles), P, P, P, geo_theta, ctypes.POINTER(geo_mle_opts),
                    ctypes.POINTER(geo_mle_result), P],
    }
    sig.update({
        "geo_profile_enable": [I],
        "geo_profile_reset": [],
        "geo_profile_read": [I, ctypes.POINTER(D), ctypes.POINTER(ctypes.c_longlong)],
    })
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.geo_kernel_launches.argtypes = []
    lib.geo_kernel_launches.restype = ctypes.c_ulonglong
    return lib


lib = _load()


def _check(rc: int, what: str, info: int = 0):
    if rc == GEO_OK:
        return
    if rc == GEO_ERR_NOT_SPD:
        raise NotSPDError(rc, what, info)
    raise GeoError(rc, what, info)


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def _stream(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


@dataclass(frozen=True)
class Theta:
    """Matern parameters of Eq. 1 (theta1 = sigma2, theta2 = beta, theta3 = nu) and a nugget."""
    sigma2: float
    beta: float
    nu: float
    nugget: float = 0.0

    def c(self) -> geo_theta:
        return geo_theta(float(self.sigma2), float(self.beta), float(self.nu), float(self.nugget))


def morton_order(x, y) -> np.ndarray:
    """Z-order permutation (host), perm[new] = old index."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    n = x.shape[0]
    perm = np.empty(n, dtype=np.int32)
    _check(lib.geo_morton_order(x.ctypes.data, y.ctypes.data, n, perm.ctypes.data), "geo_morton_order")
    return perm.astype(np.int64)


def layout(n: int, nb: int, band: int, lp_mode: int = GEO_LP_SPLIT_BF16) -> geo_layout:
    lay = geo_layout()
    _check(lib.geo_layout_init(int(n), int(nb), int(band), int(lp_mode), ctypes.byref(lay)), "geo_layout_init")
    return lay


class TileStore:
    """One problem's tile store in device memory (owned by torch tensors)."""

    def __init__(self, n: int, nb: int, band: int, lp_mode: int = GEO_LP_SPLIT_BF16, device="cuda"):
        import torch
        self.lay = layout(n, nb, band, lp_mode)
        dev = torch.device(device)

        def buf(nbytes):
            return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=dev)

        self._dp = buf(self.lay.bytes_dp)
        self._sp = buf(self.lay.bytes_sp)
        self._planes = buf(self.lay.bytes_planes) if self.lay.bytes_planes else None
        self._meta = buf(self.lay.bytes_meta)
        self.t = geo_tiles()
        _check(lib.geo_tiles_bind(ctypes.byref(self.t), ctypes.byref(self.lay), _ptr(self._dp), _ptr(self._sp),
                                  _ptr(self._planes), _ptr(self._meta), _stream()), "geo_tiles_bind")

    def set_flags(self, flags: int):
        _check(lib.geo_tiles_set_flags(ctypes.byref(self.t), int(flags)), "geo_tiles_set_flags")

    def set_far(self, far_band: int = 0, x=None, y=None, far_dist: float = 0.0, products: int = 3, stream=None):
        """The far tier of the three-precision extension (geo_tiles_set_far):
        off-band tiles with i - j >= far_band, or whose locations' bounding
        boxes lie far_dist or more apart, are updated with `products` (1 or 3)
        slice products.  far_band = 0 and far_dist = 0 turn it off."""
        _check(lib.geo_tiles_set_far(ctypes.byref(self.t), int(far_band), _ptr(x), _ptr(y), float(far_dist),
                                     int(products), _stream(stream)), "geo_tiles_set_far")

    def set_timeout_ns(self, ns: int):
        """Bound of every device-side wait of the persistent scheduler (0: default)."""
        _check(lib.geo_tiles_set_timeout_ns(ctypes.byref(self.t), int(ns)), "geo_tiles_set_timeout_ns")

    def enable_trace(self, capacity: int = 1 << 20):
        """Record the scheduler's tasks of the following factorizations."""
        import torch
        self._trace = torch.zeros(64 + 48 * int(capacity), dtype=torch.uint8, device=self._dp.device)
        _check(lib.geo_tiles_set_trace(ctypes.byref(self.t), _ptr(self._trace), int(capacity)), "geo_tiles_set_trace")

    def read_trace(self, reset: bool = True):
        """Records (structured numpy array) of the traced tasks, in completion order."""
        raw = self._trace.cpu().numpy()
        n = int(raw[:8].view(np.uint64)[0])
        cap = (raw.size - 64) // 48
        dt = np.dtype([("type", "i4"), ("sm", "i4"), ("k", "i4"), ("a", "i4"), ("b", "i4"), ("c", "i4"),
                       ("t_claim", "i8"), ("t_ready", "i8"), ("t_end", "i8")])
        recs = raw[64:64 + 48 * min(n, cap)].view(dt).copy()
        if reset:
            self._trace[:8].zero_()
        return recs

    def __del__(self):
        try:
            lib.geo_tiles_release(ctypes.byref(self.t))
        except Exception:
            pass

    @property
    def n(self):
        return self.lay.n

    @property
    def nb(self):
        return self.lay.nb

    @property
    def p(self):
        return self.lay.p

    @property
    def band(self):
        return self.lay.band

    def matern(self, x, y, theta: Theta, stream=None):
        _check(lib.geo_matern_tiles(ctypes.byref(self.t), _ptr(x), _ptr(y), theta.c(), _stream(stream)),
               "geo_matern_tiles")

    def load_dense(self, a, stream=None):
        _check(lib.geo_tiles_load_dense(ctypes.byref(self.t), _ptr(a), _stream(stream)), "geo_tiles_load_dense")

    def to_dense(self, stream=None):
        import torch
        out = torch.empty((self.n, self.n), dtype=torch.float64, device=self._dp.device)
        _check(lib.geo_tiles_to_dense(ctypes.byref(self.t), _ptr(out), _stream(stream)), "geo_tiles_to_dense")
        return out.t()  # stored column-major: transpose the row-major view

    def potrf(self, stream=None, check=True):
        _check(lib.geo_potrf_mp(ctypes.byref(self.t), _stream(stream)), "geo_potrf_mp")
        if check:
            code, info = self.status(stream)
            _check(code, "geo_potrf_mp", info)

    def status(self, stream=None):
        code, info = ctypes.c_int(0), ctypes.c_int(0)
        _check(lib.geo_status(ctypes.byref(self.t), ctypes.byref(code), ctypes.byref(info), _stream(stream)),
               "geo_status")
        return code.value, info.value

    def logdet_trsv(self, z, stream=None, want_y=False):
        import torch
        dev = self._dp.device
        ld = torch.empty(1, dtype=torch.float64, device=dev)
        q = torch.empty(1, dtype=torch.float64, device=dev)
        yv = torch.empty(self.p * self.nb, dtype=torch.float64, device=dev) if want_y else None
        _check(lib.geo_logdet_trsv(ctypes.byref(self.t), _ptr(z), _ptr(ld), _ptr(q), _ptr(yv), _stream(stream)),
               "geo_logdet_trsv")
        return ld, q, yv

    def loglik_async(self, x, y, z, theta: Theta, stream=None, out=None):
        """Generation, factorization, log-det, solve and Eq. 2 enqueued on the
        stream without waiting (geo_loglik_async).  Returns the device FP64[3]
        tensor (log|Sigma|, Z' Sigma^-1 Z, l), written by the library's kernels
        (NaN when the factorization fails); `out` may supply it."""
        import torch
        res = out if out is not None else torch.empty(3, dtype=torch.float64, device=self._dp.device)
        _check(lib.geo_loglik_async(ctypes.byref(self.t), _ptr(x), _ptr(y), _ptr(z), theta.c(), _ptr(res),
                                    _stream(stream)), "geo_loglik_async")
        return res

    def loglik(self, x, y, z, theta: Theta, stream=None):
        """Eq. 2 (blocking): returns (loglik, logdet, quad)."""
        out = (ctypes.c_double * 3)()
        info = ctypes.c_int(0)
        rc = lib.geo_loglik(ctypes.byref(self.t), _ptr(x), _ptr(y), _ptr(z), theta.c(), out,
                            ctypes.byref(info), _stream(stream))
        _check(rc, "geo_loglik", info.value)
        return out[0], out[1], out[2]

    def mle(self, x, y, z, theta0: Theta, max_evals: int = 60, profile: bool = False, fix_nu: bool = False,
            xtol: float = 1e-3, step: float = 0.1, lo=None, hi=None, stream=None, journal=None) -> dict:
        """Maximum likelihood estimate (Nelder-Mead over log-parameters, see geo_mle)
        with every likelihood evaluation on this store.  Returns dict(theta,
        loglik, evals, iterations, not_spd).  journal: optional dict with a
        float64 array "records" (cap x 4) and "len", the evaluation journal of
        geo_mle (replayed, then extended; "len" is updated)."""
        o = geo_mle_opts()
        _check(lib.geo_mle_default_opts(ctypes.byref(o)), "geo_mle_default_opts")
        o.max_evals, o.profile, o.fix_nu = int(max_evals), int(bool(profile)), int(bool(fix_nu))
        o.xtol, o.step = float(xtol), float(step)
        if lo is not None:
            for a in range(3):
                o.lo[a] = float(lo[a])
        if hi is not None:
            for a in range(3):
                o.hi[a] = float(hi[a])
        jl = ctypes.c_int(0)
        if journal is not None:
            rec = journal["records"]
            assert rec.dtype == np.float64 and rec.flags["C_CONTIGUOUS"] and rec.shape[1] == 4
            jl.value = int(journal["len"])
            o.journal, o.journal_cap, o.journal_len = rec.ctypes.data, int(rec.shape[0]), ctypes.pointer(jl)
        r = geo_mle_result()
        _check(lib.geo_mle(ctypes.byref(self.t), _ptr(x), _ptr(y), _ptr(z), theta0.c(), ctypes.byref(o),
                           ctypes.byref(r), _stream(stream)), "geo_mle")
        if journal is not None:
            journal["len"] = jl.value
        th = Theta(r.theta.sigma2, r.theta.beta, r.theta.nu, r.theta.nugget)
        return dict(theta=th, loglik=r.loglik, evals=r.evals, iterations=r.iterations, not_spd=r.not_spd)

    def krige(self, x, y, z, theta: Theta, xnew, ynew, stream=None):
        """Simple-kriging prediction at (xnew, ynew) from the factored store."""
        import torch
        dev = self._dp.device
        m = int(xnew.shape[0])
        zhat = torch.empty(max(m, 1), dtype=torch.float64, device=dev)
        work = torch.empty(2 * self.p * self.nb, dtype=torch.float64, device=dev)
        _check(lib.geo_krige(ctypes.byref(self.t), _ptr(x), _ptr(y), _ptr(z), theta.c(), _ptr(xnew), _ptr(ynew), m,
                             _ptr(zhat), _ptr(work), _stream(stream)), "geo_krige")
        return zhat[:m]


PROF_FP64_UPDATE, PROF_LP_UPDATE, PROF_POTRF, PROF_TRSM = 0, 1, 2, 3


def kernel_launches() -> int:
    """Kernel launches issued by the library in this process."""
    return int(lib.geo_kernel_launches())


def profile_enable(on: bool = True):
    _check(lib.geo_profile_enable(1 if on else 0), "geo_profile_enable")


def profile_reset():
    _check(lib.geo_profile_reset(), "geo_profile_reset")


def profile_read(kind: int):
    """(total ms, launches) of one instrumented kernel kind since the last reset."""
    ms, n = ctypes.c_double(0.0), ctypes.c_longlong(0)
    _check(lib.geo_profile_read(int(kind), ctypes.byref(ms), ctypes.byref(n)), "geo_profile_read")
    return ms.value, n.value


def loglik_flops(n: int) -> float:
    """Algorithmic flop count of one factorization, n^3/3."""
    return n ** 3 / 3.0




def loglik(x, y, z, theta: Theta, nb: int = 500, band: int = 1, lp_mode: int = GEO_LP_SPLIT_BF16,
           flags: int = 0) -> float:
    """geo.loglik(x, y, z, theta, nb, band): Eq. 2 on a fresh tile store (x, y, z:
    Morton-ordered device tensors); raises NotSPDError when the factorization
    meets a non-positive pivot."""
    ts = TileStore(int(z.shape[0]), nb, band, lp_mode, device=z.device)
    if flags:
        ts.set_flags(flags)
    return ts.loglik(x, y, z, theta)[0]


def mle(x, y, z, theta0: Theta, nb: int, band: int, lp_mode: int = GEO_LP_SPLIT_BF16, flags: int = 0, **kw):
    """geo.mle(x, y, z, theta0, nb, band, ...): the estimator on a fresh tile store
    (x, y, z: Morton-ordered device tensors; keywords as TileStore.mle)."""
    ts = TileStore(int(z.shape[0]), nb, band, lp_mode, device=z.device)
    if flags:
        ts.set_flags(flags)
    return ts.mle(x, y, z, theta0, **kw)


class Batch:
    """Many log-likelihood problems evaluated through one generator launch and
    one persistent factorization launch (geo_loglik_batch).

    problems: list of dicts with device tensors x, y, z (Morton-ordered) and
    optional nb (default 128), band (default 1), flags, or an existing
    `store` (TileStore of split-BF16 mode) to evaluate in.  The stores, the
    workspace and the per-problem theta buffer are allocated once; each
    evaluation only enqueues work, so `capture()` can record it in a CUDA graph
    and `replay(thetas)` re-runs it with new parameters.  ctas: run the
    factorization launch on that many SMs (0: all, cooperative; otherwise at
    least GEO_MIN_CTAS), leaving the others to launches on other streams.
    """

    def __init__(self, problems, nb: int = 128, band: int = 1, device="cuda", ctas: int = 0):
        import torch
        self.device = torch.device(device)
        self.stores, self._keep = [], []
        n = len(problems)
        self.items = (geo_batch_item * n)()
        for b, pr in enumerate(problems):
            x, y, z = pr["x"], pr["y"], pr["z"]
            ts = pr.get("store")   # an existing split-BF16 store of this size may be reused
            if ts is None:
                ts = TileStore(int(z.shape[0]), int(pr.get("nb", nb)), int(pr.get("band", band)), GEO_LP_SPLIT_BF16,
                               device=self.device)
                if pr.get("flags"):
                    ts.set_flags(int(pr["flags"]))
            self.stores.append(ts)
            self._keep.append((x, y, z))
            self.items[b].t = ctypes.pointer(ts.t)
            self.items[b].d_x, self.items[b].d_y, self.items[b].d_z = _ptr(x), _ptr(y), _ptr(z)
        self.nprob = n
        nbytes = ctypes.c_size_t(0)
        _check(lib.geo_batch_workspace(n, self.items, ctypes.byref(nbytes)), "geo_batch_workspace")
        self._work = torch.empty(max(int(nbytes.value), 256), dtype=torch.uint8, device=self.device)
        _check(lib.geo_batch_bind(n, self.items, _ptr(self._work), int(nbytes.value), _stream()), "geo_batch_bind")
        if ctas:
            _check(lib.geo_batch_set_ctas(_ptr(self._work), int(ctas)), "geo_batch_set_ctas")
        self.theta = torch.zeros((n, 4), dtype=torch.float64, device=self.device)
        self.out = torch.zeros((n, 3), dtype=torch.float64, device=self.device)
        self.done_ns = torch.zeros(n + 1, dtype=torch.int64, device=self.device)
        self.graph = None

    def __del__(self):
        try:
            lib.geo_batch_release(_ptr(self._work))
        except Exception:
            pass

    def nbytes(self) -> int:
        """Device bytes of the batch workspace (the stores not included)."""
        return int(self._work.numel())

    def set_theta(self, thetas):
        import torch
        t = torch.tensor([[th.sigma2, th.beta, th.nu, th.nugget] for th in thetas], dtype=torch.float64)
        self.theta.copy_(t, non_blocking=False)

    def loglik_async(self, stream=None):
        """Enqueue one evaluation with the parameters in self.theta; results land
        in self.out[b] = (l, log|Sigma|, Z' Sigma^-1 Z), NaN where not SPD, and
        self.done_ns = (launch start, completion of each problem) in ns."""
        _check(lib.geo_loglik_batch(self.nprob, self.items, _ptr(self.theta), _ptr(self._work), _ptr(self.out),
                                    _ptr(self.done_ns), _stream(stream)), "geo_loglik_batch")
        return self.out

    def completion_ms(self):
        """Per-problem completion time of the last evaluation, ms after the
        factorization launch started (NaN for a problem that failed)."""
        t = self.done_ns.cpu().numpy()
        out = (t[1:] - t[0]).astype(np.float64) / 1e6
        out[t[1:] == 0] = np.nan
        return out

    def loglik(self, thetas):
        import torch
        self.set_theta(thetas)
        self.loglik_async()
        torch.cuda.synchronize(self.device)
        return self.out.cpu().numpy().copy()

    def capture(self):
        """Record one evaluation in a CUDA graph (after a warm-up evaluation)."""
        import torch
        s = torch.cuda.Stream(device=self.device)
        s.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(s):
            self.loglik_async(s)
        torch.cuda.current_stream(self.device).wait_stream(s)
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.loglik_async()
        self.graph = g
        return g

    def replay(self, thetas=None):
        import torch
        if thetas is not None:
            self.set_theta(thetas)
        self.graph.replay()
        torch.cuda.synchronize(self.device)
        return self.out.cpu().numpy().copy()

    def status(self):
        return [ts.status() for ts in self.stores]


def __getattr__(name):
    # geo.Server: the serving loop lives in serve.py, which builds on this module
    if name == "Server":
        from .serve import Server
        return Server
    raise AttributeError(name)
