"""Python binding of libfsmlmc.so (the C ABI in include/fsmlmc.h).

Argument marshalling only: every step of the computation runs in the CUDA
library. If the compiled library is missing this module raises at load time;
there is no CPU fallback.
"""

import ctypes
import os

import numpy as np

from . import gamma as _gamma

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfsmlmc.so")

FS_OK, FS_ERR_ARG, FS_ERR_INPUT, FS_ERR_OOM, FS_ERR_BUDGET, FS_ERR_NOCONV, FS_ERR_TIMEOUT, FS_ERR_CUDA, \
    FS_ERR_STATE = range(9)
PREC = {"f64": 0, "f32": 1, "f16": 2, "bf16": 3}
ESTIMATOR = {"diff": 0, "split_even": 1, "product": 2}
SYS_CONVERGED, SYS_NOCONV = 2, 3

EXPORTS = ["fs_ctx_create", "fs_ctx_destroy", "fs_last_error", "fs_set_stream", "fs_ctx_device_bytes",
           "fs_set_gauge", "wilson_dslash", "shifted_solve", "mlmc_level_trace", "fs_mlmc_num_solves",
           "variance_sample", "fs_noise_codes", "fs_profile_enable", "fs_profile_read", "fs_kernel_launches",
           "wilson_dslash_noalloc", "fs_server_create", "fs_server_submit", "fs_server_poll",
           "fs_server_stats", "fs_server_destroy", "fs_interp_variances", "fs_select_shifts",
           "fs_sample_allocation", "fs_eval_grid", "fs_tuned_tile", "fs_probing_colors",
           "variance_sample_probed", "shifted_solve_dev", "fs_hpe_exact_trace",
           "mlmc_level_traces", "fs_server_set_admission", "fs_trace_total", "fs_sampled_level_variances",
           "fs_measure_peak", "fs_profile_read_fp64", "fs_set_iteration_bound", "fs_tuned_shape",
           "fs_set_clover"]
JOB_MAX_LEVELS = 16


class FsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("fsmlmc error %d: %s" % (code, msg))
        self.code = code


class SolveParams(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("prec", ctypes.c_int),
                ("rhs_tile", ctypes.c_int), ("link_compress", ctypes.c_int), ("delta", ctypes.c_double),
                ("verify", ctypes.c_int), ("fallback_iter", ctypes.c_int), ("lanes", ctypes.c_int)]


class SysStats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("status", ctypes.c_int), ("reliable_updates", ctypes.c_int),
                ("restarts", ctypes.c_int), ("true_resid", ctypes.c_double), ("fallback_iters", ctypes.c_int),
                ("pad", ctypes.c_int)]


class MlmcParams(ctypes.Structure):
    _fields_ = [("m", ctypes.c_double), ("nlev", ctypes.c_int), ("p", ctypes.c_int),
                ("sigma", ctypes.POINTER(ctypes.c_double)), ("n_samples", ctypes.POINTER(ctypes.c_int)),
                ("gamma", ctypes.POINTER(ctypes.c_double)), ("seed", ctypes.c_uint64),
                ("job", ctypes.c_uint32), ("estimator", ctypes.c_int), ("solve", SolveParams),
                ("colors", ctypes.POINTER(ctypes.c_int32)), ("ncolors", ctypes.c_int), ("dilute", ctypes.c_int),
                ("hpe_order", ctypes.c_int)]


class Job(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int * 4), ("bc_t", ctypes.c_int), ("U", ctypes.POINTER(ctypes.c_double)),
                ("params", MlmcParams), ("c_sw", ctypes.c_double)]


class JobResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("nlev", ctypes.c_int), ("trace", (ctypes.c_double * 2) * 16),
                ("var", ctypes.c_double * 16), ("solves", ctypes.c_longlong), ("mean_iters", ctypes.c_double),
                ("max_iters", ctypes.c_int), ("noconv", ctypes.c_int), ("restarts", ctypes.c_longlong),
                ("latency_ms", ctypes.c_double), ("queue_ms", ctypes.c_double)]


class ServerReport(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_longlong), ("queued", ctypes.c_longlong), ("active", ctypes.c_longlong),
                ("solves", ctypes.c_longlong), ("reserved_bytes", ctypes.c_size_t), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("solves_per_s", ctypes.c_double), ("gauge_reuses", ctypes.c_longlong)]


_lib = None


def load_library(path=LIB_PATH):
    """Load libfsmlmc.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libfsmlmc.so not found at %s: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`" % path)
    L = ctypes.CDLL(path)
    P, I, D, U64, U32 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    sig = {
        "fs_ctx_create": (I, [ctypes.POINTER(P), ip, I, I]),
        "fs_ctx_destroy": (None, [P]),
        "fs_last_error": (ctypes.c_char_p, [P]),
        "fs_set_stream": (I, [P, P]),
        "fs_ctx_device_bytes": (ctypes.c_size_t, [P]),
        "fs_tuned_tile": (I, [P, I, I]),
        "fs_set_gauge": (I, [P, dp]),
        "fs_set_clover": (I, [P, ctypes.c_double]),
        "wilson_dslash": (I, [P, D, D, dp, dp, I, I, I]),
        "shifted_solve": (I, [P, D, dp, I, dp, I, dp, ctypes.POINTER(SolveParams), ctypes.POINTER(SysStats)]),
        "shifted_solve_dev": (I, [P, D, dp, I, P, I, P, ctypes.POINTER(SolveParams), ctypes.POINTER(SysStats)]),
        "fs_hpe_exact_trace": (I, [P, D, D, dp, I, I, U64, ctypes.POINTER(SolveParams), dp]),
        "mlmc_level_trace": (I, [P, ctypes.POINTER(MlmcParams), dp, dp, dp, ctypes.POINTER(SysStats)]),
        "mlmc_level_traces": (I, [P, ctypes.POINTER(MlmcParams), ip, I, dp, dp, dp, ctypes.POINTER(SysStats)]),
        "fs_mlmc_num_solves": (I, [ctypes.POINTER(MlmcParams)]),
        "variance_sample": (I, [P, D, dp, I, dp, ip, I, I, U64, U32, ctypes.POINTER(SolveParams), dp, dp, dp,
                                dp, dp]),
        "variance_sample_probed": (I, [P, D, dp, I, dp, ip, I, I, U64, U32, ctypes.POINTER(SolveParams),
                                       ctypes.POINTER(ctypes.c_int32), I, I, I, dp, dp, dp, dp, dp]),
        "fs_noise_codes": (I, [P, U64, U32, U32, U32, ctypes.POINTER(ctypes.c_uint8)]),
        "fs_profile_enable": (I, [P, I]),
        "fs_profile_read": (I, [P, ctypes.POINTER(ctypes.c_longlong), dp, dp, dp]),
        "fs_profile_read_fp64": (I, [P, ctypes.POINTER(ctypes.c_longlong), dp, dp]),
        "fs_set_iteration_bound": (I, [P, ctypes.c_longlong]),
        "fs_tuned_shape": (I, [P, I, I, ip, ip, ip]),
        "fs_kernel_launches": (ctypes.c_longlong, []),
        "wilson_dslash_noalloc": (I, [ip, I, D, D, P, P, P, I, P]),
        "fs_server_create": (I, [ctypes.POINTER(P), I, ctypes.c_size_t, I]),
        "fs_server_submit": (I, [P, ctypes.POINTER(Job), ctypes.POINTER(ctypes.c_uint64)]),
        "fs_server_poll": (I, [P, ctypes.c_uint64, ctypes.POINTER(JobResult), I]),
        "fs_server_stats": (I, [P, ctypes.POINTER(ServerReport)]),
        "fs_server_destroy": (None, [P]),
        "fs_server_set_admission": (I, [P, I, D]),
        "fs_interp_variances": (I, [dp, I, dp, dp, dp, I, dp, dp]),
        "fs_select_shifts": (I, [dp, I, dp, dp, dp, dp, I, I, ip, dp, dp, dp]),
        "fs_sample_allocation": (I, [dp, dp, I, D, dp, dp, dp, dp]),
        "fs_eval_grid": (I, [dp, I, dp, I, ip]),
        "fs_trace_total": (I, [dp, dp, ip, I, I, dp, dp]),
        "fs_measure_peak": (I, [I, D, dp, dp]),
        "fs_sampled_level_variances": (I, [dp, I, dp, I, dp]),
        "fs_probing_colors": (I, [ip, I, I, ctypes.POINTER(ctypes.c_int32), ip]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _set_probing(P, colors, ncolors, dilute):
    """Fill the probing / dilution fields of an MlmcParams; returns the array to keep alive."""
    P.dilute = int(bool(dilute))
    if colors is None:
        P.colors = None
        P.ncolors = 0
        return None
    col = np.ascontiguousarray(colors, dtype=np.int32).ravel()
    P.colors = col.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    P.ncolors = int(ncolors) if ncolors is not None else (int(col.max()) + 1 if col.size else 0)
    return col


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _real(a, shape=None):
    """complex array -> contiguous float64 view with a trailing (re, im) axis."""
    a = np.ascontiguousarray(a)
    if np.iscomplexobj(a):
        a = np.ascontiguousarray(a, dtype=np.complex128).view(np.float64)
    else:
        a = np.ascontiguousarray(a, dtype=np.float64)
    return a


def _params(prec="f64", tol=0.0, max_iter=0, rhs_tile=0, link_compress=18, delta=0.0, verify=0, fallback_iter=0,
            lanes=0):
    p = SolveParams()
    p.tol = tol
    p.max_iter = max_iter
    p.prec = PREC[prec] if isinstance(prec, str) else int(prec)
    p.rhs_tile = rhs_tile
    p.link_compress = link_compress
    p.delta = delta
    p.verify = int(verify)
    p.fallback_iter = int(fallback_iter)
    p.lanes = int(lanes)
    return p


class Context:
    """A lattice on one CUDA device (fs_ctx)."""

    def __init__(self, dims, bc_t=-1, device=0):
        self.lib = load_library()
        self.dims = tuple(int(d) for d in dims)
        self.V = int(np.prod(self.dims))
        self.h = ctypes.c_void_p()
        arr = (ctypes.c_int * 4)(*self.dims)
        rc = self.lib.fs_ctx_create(ctypes.byref(self.h), arr, int(bc_t), int(device))
        if rc != FS_OK:
            raise FsError(rc, "fs_ctx_create failed (dims %s, bc_t %d)" % (self.dims, bc_t))

    def close(self):
        if self.h:
            self.lib.fs_ctx_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, allow_noconv=False):
        if rc == FS_OK or (allow_noconv and rc == FS_ERR_NOCONV):
            return rc
        raise FsError(rc, self.lib.fs_last_error(self.h).decode())

    def last_error(self):
        return self.lib.fs_last_error(self.h).decode()

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t integer, or None."""
        handle = getattr(stream, "cuda_stream", stream)
        self._check(self.lib.fs_set_stream(self.h, ctypes.c_void_p(handle or 0)))

    def device_bytes(self):
        return int(self.lib.fs_ctx_device_bytes(self.h))

    def tuned_tile(self, prec="f16", link_compress=18):
        """Systems per tile the autotuner chose for this precision and link format (0: not run)."""
        p = PREC[prec] if isinstance(prec, str) else int(prec)
        return int(self.lib.fs_tuned_tile(self.h, p, int(link_compress)))

    def tuned_shape(self, prec="f16", link_compress=18):
        """(tile, ring depth, resident blocks per SM) the autotuner chose (0: default / not run)."""
        p = PREC[prec] if isinstance(prec, str) else int(prec)
        t, d, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.fs_tuned_shape(self.h, p, int(link_compress), ctypes.byref(t), ctypes.byref(d),
                                            ctypes.byref(b)))
        return t.value, d.value, b.value

    def fs_set_gauge(self, U):
        u = _real(U)
        if u.size != 4 * self.V * 18:
            raise ValueError("gauge field must have 4*V*3*3 complex entries")
        self._check(self.lib.fs_set_gauge(self.h, _dptr(u)))

    set_gauge = fs_set_gauge

    def fs_set_clover(self, c_sw):
        """The Wilson-clover operator with coefficient c_sw for every later operation (0: Wilson)."""
        self._check(self.lib.fs_set_clover(self.h, float(c_sw)))

    set_clover = fs_set_clover

    def wilson_dslash(self, m, sigma, psi, prec="f64", link_compress=18):
        """(D + sigma) psi for psi complex [V][4][3] or [nrhs][V][4][3]."""
        x = _real(psi)
        nrhs = x.size // (self.V * 24)
        if nrhs * self.V * 24 != x.size:
            raise ValueError("spinor size mismatch")
        out = np.empty_like(x)
        p = PREC[prec] if isinstance(prec, str) else int(prec)
        self._check(self.lib.wilson_dslash(self.h, m, sigma, _dptr(x), _dptr(out), nrhs, p, link_compress))
        return out.view(np.complex128).reshape(np.shape(psi))

    def shifted_solve(self, m, sigmas, b, **kw):
        """x[j, k] = (D + sigma_j)^-1 b_k. Returns (x complex [nshift][nrhs][V][4][3], stats list, rc)."""
        sig = np.ascontiguousarray(np.atleast_1d(sigmas), dtype=np.float64)
        bb = _real(b)
        nrhs = bb.size // (self.V * 24)
        x = np.empty((len(sig), nrhs, self.V, 4, 3, 2), dtype=np.float64)
        st = (SysStats * (len(sig) * nrhs))()
        p = _params(**kw)
        rc = self._check(self.lib.shifted_solve(self.h, m, _dptr(sig), len(sig), _dptr(bb), nrhs, _dptr(x),
                                                ctypes.byref(p), st), allow_noconv=True)
        return x.view(np.complex128)[..., 0], [_stats(s) for s in st], rc

    def hpe_exact_trace(self, m, sigma, gamma, p, K, seed=0, **kw):
        """Exact low orders sum_{k<K} Tr(Gamma Omega_p (kappa H)^k) / A of the hopping parameter
        expansion (complex)."""
        g = _gamma.to_abi(gamma)
        out = np.zeros(2)
        prm = _params(**kw)
        self._check(self.lib.fs_hpe_exact_trace(self.h, m, sigma, _dptr(g), int(p), int(K), int(seed),
                                                ctypes.byref(prm), _dptr(out)))
        return complex(out[0], out[1])

    def shifted_solve_dev(self, m, sigmas, b_ptr, nrhs, x_ptr, **kw):
        """shifted_solve on device arrays: b_ptr / x_ptr are device addresses (e.g. a float64 torch
        tensor's data_ptr()) of [nrhs][V][24] and [nshift][nrhs][V][24]; returns the stats."""
        sig = np.ascontiguousarray(sigmas, dtype=np.float64)
        prm = _params(**kw)
        st = (SysStats * max(sig.size * nrhs, 1))()
        self._check(self.lib.shifted_solve_dev(self.h, m, _dptr(sig), sig.size, ctypes.c_void_p(int(b_ptr)),
                                               int(nrhs), ctypes.c_void_p(int(x_ptr)), ctypes.byref(prm), st),
                    allow_noconv=True)
        return [_stats(s) for s in st[:sig.size * nrhs]]

    def mlmc_level_trace(self, m, sigmas, gamma, p, n_samples, seed, job=0, estimator="split_even", colors=None,
                         ncolors=None, dilute=False, hpe_order=0, **kw):
        """Level traces (estimator: "split_even" by default, Eq. (fs_trace_est), measured cheapest on the
        16^3x32 job; "diff" and "product" are the other two); colors ([V] probing colours, canonical order) and dilute (full spin-colour
        dilution) make every sample the sum of the estimator over its pieces; hpe_order = K uses
        the hopping parameter expansion on the last level when m + sigma_L > 0. A sequence p gives
        the traces for every displacement from the same solves (mlmc_level_traces): a list of
        result dicts in the order of p."""
        multi = not np.isscalar(p)
        plist = np.ascontiguousarray(np.atleast_1d(p), dtype=np.int32)
        sig = np.ascontiguousarray(sigmas, dtype=np.float64)
        ns = np.ascontiguousarray(n_samples, dtype=np.int32)
        if ns.size == 1 and sig.size > 1:
            ns = np.full(sig.size, int(ns.ravel()[0]), dtype=np.int32)
        g = _gamma.to_abi(gamma)
        P = MlmcParams()
        P.m = m
        P.nlev = sig.size
        P.p = int(plist[0])
        P.sigma = _dptr(sig)
        P.n_samples = ns.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        P.gamma = _dptr(g)
        P.seed = int(seed)
        P.job = int(job)
        P.estimator = ESTIMATOR[estimator] if isinstance(estimator, str) else int(estimator)
        P.solve = _params(**kw)
        keep = _set_probing(P, colors, ncolors, dilute)  # noqa: F841 (alive through the call)
        P.hpe_order = int(hpe_order)
        nsolve = self.lib.fs_mlmc_num_solves(ctypes.byref(P))
        if nsolve < 0:
            raise FsError(1, "fs_mlmc_num_solves: bad sample counts, ncolors or dilute")
        npl = plist.size
        trace = np.zeros((npl, sig.size, 2))
        var = np.zeros((npl, sig.size))
        samples = np.zeros((npl, int(ns.sum()), 2))
        st = (SysStats * max(nsolve, 1))()
        if multi:
            rc = self._check(self.lib.mlmc_level_traces(self.h, ctypes.byref(P),
                                                        plist.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), npl,
                                                        _dptr(trace), _dptr(var), _dptr(samples), st),
                             allow_noconv=True)
        else:
            rc = self._check(self.lib.mlmc_level_trace(self.h, ctypes.byref(P), _dptr(trace), _dptr(var),
                                                       _dptr(samples), st), allow_noconv=True)
        stats = [_stats(s) for s in st[:nsolve]]
        total, v_fs = fs_trace_total(trace, var, ns)
        offs = np.concatenate([[0], np.cumsum(ns)])
        res = []
        for q in range(npl):
            tr = trace[q, :, 0] + 1j * trace[q, :, 1]
            smp = samples[q, :, 0] + 1j * samples[q, :, 1]
            res.append({"p": int(plist[q]), "trace": tr, "var": var[q],
                        "samples": [smp[offs[l]:offs[l + 1]] for l in range(sig.size)],
                        "total": complex(total[q, 0], total[q, 1]), "v_fs": float(v_fs[q]), "stats": stats,
                        "rc": rc})
        return res if multi else res[0]

    def variance_sample(self, m, s_hat, gamma, p_list, n_s, seed, job=0, colors=None, ncolors=None, dilute=False,
                        hpe_order=0, **kw):
        """Sec. 3.1 variance sampling; colors / dilute select probed and diluted noise and
        hpe_order the hopping parameter expansion of a_i (variance_sample_probed)."""
        sh = np.ascontiguousarray(s_hat, dtype=np.float64)
        pl = np.ascontiguousarray(p_list, dtype=np.int32)
        ms, npl = sh.size, pl.size
        g = _gamma.to_abi(gamma)
        VL = np.zeros((npl, ms))
        Vbar = np.zeros((npl, ms, ms))
        a = np.zeros((n_s, npl, ms, 2))
        b = np.zeros((n_s, npl, ms, ms, 2))
        iters = np.zeros(ms)
        prm = _params(**kw)
        plp = pl.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        if colors is None and not dilute and not hpe_order:
            rc = self._check(self.lib.variance_sample(self.h, m, _dptr(sh), ms, _dptr(g), plp, npl, n_s, int(seed),
                                                      int(job), ctypes.byref(prm), _dptr(VL), _dptr(Vbar),
                                                      _dptr(a), _dptr(b), _dptr(iters)), allow_noconv=True)
        else:
            col = None if colors is None else np.ascontiguousarray(colors, dtype=np.int32).ravel()
            nc = 0 if col is None else (int(ncolors) if ncolors is not None else int(col.max()) + 1)
            cp = None if col is None else col.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
            rc = self._check(self.lib.variance_sample_probed(self.h, m, _dptr(sh), ms, _dptr(g), plp, npl, n_s,
                                                             int(seed), int(job), ctypes.byref(prm), cp, nc,
                                                             int(bool(dilute)), int(hpe_order), _dptr(VL),
                                                             _dptr(Vbar), _dptr(a),
                                                             _dptr(b), _dptr(iters)), allow_noconv=True)
        return {"VL": VL, "Vbar": Vbar, "a": a[..., 0] + 1j * a[..., 1], "b": b[..., 0] + 1j * b[..., 1],
                "Vl": fs_sampled_level_variances(sh, Vbar), "iters": iters, "rc": rc}

    def fs_noise_codes(self, seed, job, level, sample):
        codes = np.empty((self.V, 4, 3), dtype=np.uint8)
        self._check(self.lib.fs_noise_codes(self.h, int(seed), int(job), int(level), int(sample),
                                            codes.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))))
        return codes

    noise_codes = fs_noise_codes

    def profile_enable(self, enable=True):
        self._check(self.lib.fs_profile_enable(self.h, int(enable)))

    def profile_read(self):
        n = ctypes.c_longlong()
        ms = ctypes.c_double()
        by = ctypes.c_double()
        ss = ctypes.c_double()
        self._check(self.lib.fs_profile_read(self.h, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by),
                                             ctypes.byref(ss)))
        return {"launches": n.value, "ms": ms.value, "bytes": by.value, "site_systems": ss.value}

    def set_iteration_bound(self, bound):
        """Watchdog of the host solve loops (0: the built-in bound); FS_ERR_TIMEOUT when exceeded."""
        self._check(self.lib.fs_set_iteration_bound(self.h, int(bound)))

    def profile_read_fp64(self):
        n = ctypes.c_longlong()
        ms = ctypes.c_double()
        ss = ctypes.c_double()
        self._check(self.lib.fs_profile_read_fp64(self.h, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(ss)))
        return {"launches": n.value, "ms": ms.value, "site_systems": ss.value}


def fs_kernel_launches():
    """Kernels launched by the library in this process so far."""
    return int(load_library().fs_kernel_launches())


def wilson_dslash_noalloc(dims, bc_t, m, sigma, U_ptr, in_ptr, out_ptr, nrhs, stream=0):
    """Allocation-free FP64 (D + sigma) on device buffers given as raw device pointers
    (e.g. torch tensor .data_ptr()); stream-ordered on `stream` (raw cudaStream_t).
    Returns the status code (0 = queued)."""
    L = load_library()
    arr = (ctypes.c_int * 4)(*[int(d) for d in dims])
    return int(L.wilson_dslash_noalloc(arr, int(bc_t), float(m), float(sigma), ctypes.c_void_p(U_ptr),
                                       ctypes.c_void_p(in_ptr), ctypes.c_void_p(out_ptr), int(nrhs),
                                       ctypes.c_void_p(stream or 0)))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc, what):
    if rc != FS_OK:
        raise FsError(rc, what + " failed")


def fs_eval_grid(s_hat):
    """The paper's evaluation set of shifts for the sampling shifts s_hat."""
    L = load_library()
    sh = _f64(s_hat)
    n = ctypes.c_int(0)
    _check(L.fs_eval_grid(_dptr(sh), len(sh), None, 0, ctypes.byref(n)), "fs_eval_grid")
    out = np.empty(n.value)
    _check(L.fs_eval_grid(_dptr(sh), len(sh), _dptr(out), len(out), ctypes.byref(n)), "fs_eval_grid")
    return out


def fs_probing_colors(dims, k, p=0):
    """Greedy distance-k (displacement-p along z) probing colours: (int32 [V], ncolors)."""
    L = load_library()
    d = (ctypes.c_int * 4)(*[int(x) for x in dims])
    v = int(np.prod([int(x) for x in dims]))
    out = np.empty(v, dtype=np.int32)
    n = ctypes.c_int(0)
    _check(L.fs_probing_colors(d, int(k), int(p), out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                               ctypes.byref(n)), "fs_probing_colors")
    return out, n.value


def fs_interp_variances(s_hat, VL_hat, Vbar_hat, s):
    """(V_L[n], V_l[n, n]) on the evaluation set s; V_l is NaN for k <= i."""
    L = load_library()
    sh, vl, vb, ss = _f64(s_hat), _f64(VL_hat), _f64(Vbar_hat), _f64(s)
    m, n = len(sh), len(ss)
    VL = np.empty(n)
    Vl = np.empty((n, n))
    _check(L.fs_interp_variances(_dptr(sh), m, _dptr(vl), _dptr(vb), _dptr(ss), n, _dptr(VL), _dptr(Vl)),
           "fs_interp_variances")
    return VL, Vl


def fs_select_shifts(s_hat, VL_hat, Vbar_hat, iters_hat, s, L_shifts):
    """Optimal shifts: dict with idx, sigma, V, C (per level) and F (C_FS = F^2 / eps^2)."""
    L = load_library()
    sh, vl, vb, it, ss = _f64(s_hat), _f64(VL_hat), _f64(Vbar_hat), _f64(iters_hat), _f64(s)
    idx = (ctypes.c_int * (L_shifts + 1))()
    V = np.empty(L_shifts + 1)
    C = np.empty(L_shifts + 1)
    F = ctypes.c_double(0.0)
    _check(L.fs_select_shifts(_dptr(sh), len(sh), _dptr(vl), _dptr(vb), _dptr(it), _dptr(ss), len(ss),
                              int(L_shifts), idx, _dptr(V), _dptr(C), ctypes.byref(F)), "fs_select_shifts")
    ix = list(idx)
    return {"idx": ix, "sigma": ss[ix], "V": V, "C": C, "F": F.value}


def fs_trace_total(trace, var, n_samples):
    """(total [np][2], v_fs [np]) of Eq. (fs_trace_est) summed over levels and Eq. (total_var), from
    mlmc_level_trace(s) output trace [np][nlev][2] (or [nlev][2]) and var [np][nlev]."""
    L = load_library()
    tr = _f64(trace)
    vr = _f64(var)
    ns = np.ascontiguousarray(n_samples, dtype=np.int32)
    nlev = ns.size
    npl = vr.size // nlev
    total = np.empty((npl, 2))
    v_fs = np.empty(npl)
    _check(L.fs_trace_total(_dptr(tr), _dptr(vr), ns.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), nlev, npl,
                            _dptr(total), _dptr(v_fs)), "fs_trace_total")
    return total, v_fs


def fs_sampled_level_variances(s_hat, Vbar):
    """Vl [np][m][m] of Eq. (sampled_prod) from variance_sample's Vbar [np][m][m]."""
    L = load_library()
    sh = _f64(s_hat)
    vb = _f64(Vbar)
    m = sh.size
    out = np.empty(vb.shape)
    _check(L.fs_sampled_level_variances(_dptr(sh), m, _dptr(vb), vb.size // (m * m), _dptr(out)),
           "fs_sampled_level_variances")
    return out


PEAK_KIND = {"f32": 0, "f32x2": 1, "f64": 2}


def fs_measure_peak(kind, seconds=2.0):
    """(TFLOP/s, elapsed ms) of independent FMA chains on the current device: kind "f32" (scalar
    FP32), "f32x2" (packed FP32 pairs) or "f64"."""
    L = load_library()
    tf, ms = ctypes.c_double(), ctypes.c_double()
    _check(L.fs_measure_peak(PEAK_KIND[kind], float(seconds), ctypes.byref(tf), ctypes.byref(ms)),
           "fs_measure_peak")
    return tf.value, ms.value


def fs_sample_allocation(V, C, eps2):
    """(N, mu, V_FS, C_FS) of Eq. (num_samples) / Eq. (total_var)."""
    L = load_library()
    v, c = _f64(V), _f64(C)
    N = np.empty(len(v))
    mu, vfs, cfs = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(L.fs_sample_allocation(_dptr(v), _dptr(c), len(v), float(eps2), _dptr(N), ctypes.byref(mu),
                                  ctypes.byref(vfs), ctypes.byref(cfs)), "fs_sample_allocation")
    return N, mu.value, vfs.value, cfs.value


class Server:
    """fs_server: admission by device-memory budget (least work first by default, with an aging
    limit; first in, first out through set_admission), one worker (context + stream) per active
    job, continuous batching inside each job."""

    def __init__(self, device=0, hbm_budget_bytes=60 << 30, max_active=4):
        self.lib = load_library()
        self.h = ctypes.c_void_p()
        rc = self.lib.fs_server_create(ctypes.byref(self.h), int(device), int(hbm_budget_bytes), int(max_active))
        if rc != FS_OK:
            raise FsError(rc, "fs_server_create failed")

    def submit(self, dims, U, m, sigmas, gamma, p, n_samples, seed, job=0, estimator="split_even", bc_t=-1,
               colors=None, ncolors=None, dilute=False, hpe_order=0, c_sw=0.0, **kw):
        """Queue one trace job (arrays are copied; c_sw: the clover coefficient, 0 = Wilson);
        returns the ticket."""
        u = _real(U)
        sig = np.ascontiguousarray(sigmas, dtype=np.float64)
        ns = np.ascontiguousarray(n_samples, dtype=np.int32)
        g = _gamma.to_abi(gamma)
        J = Job()
        for k in range(4):
            J.dims[k] = int(dims[k])
        J.bc_t = int(bc_t)
        J.U = _dptr(u)
        J.c_sw = float(c_sw)
        P = J.params
        P.m = m
        P.nlev = sig.size
        P.p = int(p)
        P.sigma = _dptr(sig)
        P.n_samples = ns.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        P.gamma = _dptr(g)
        P.seed = int(seed)
        P.job = int(job)
        P.estimator = ESTIMATOR[estimator] if isinstance(estimator, str) else int(estimator)
        P.solve = _params(**kw)
        keep = _set_probing(P, colors, ncolors, dilute)  # noqa: F841 (alive through the call)
        P.hpe_order = int(hpe_order)
        t = ctypes.c_uint64()
        rc = self.lib.fs_server_submit(self.h, ctypes.byref(J), ctypes.byref(t))
        if rc != FS_OK:
            raise FsError(rc, "fs_server_submit failed")
        return t.value

    def set_admission(self, least_work_first=True, max_wait_ms=10000.0):
        """Admission order: least work first with a waiting-time bound (default), or FIFO."""
        rc = self.lib.fs_server_set_admission(self.h, int(bool(least_work_first)), float(max_wait_ms))
        if rc != FS_OK:
            raise FsError(rc, "fs_server_set_admission failed")

    def poll(self, ticket, timeout_ms=-1):
        """Result dict of a finished job, or None on timeout."""
        r = JobResult()
        rc = self.lib.fs_server_poll(self.h, ctypes.c_uint64(ticket), ctypes.byref(r), int(timeout_ms))
        if rc == FS_ERR_TIMEOUT:
            return None
        if rc != FS_OK:
            raise FsError(rc, "fs_server_poll failed")
        n = r.nlev
        return {"status": r.status, "trace": np.array([r.trace[l][0] + 1j * r.trace[l][1] for l in range(n)]),
                "var": np.array([r.var[l] for l in range(n)]), "solves": r.solves, "mean_iters": r.mean_iters,
                "max_iters": r.max_iters, "noconv": r.noconv, "restarts": r.restarts,
                "latency_ms": r.latency_ms, "queue_ms": r.queue_ms}

    def stats(self):
        r = ServerReport()
        if self.lib.fs_server_stats(self.h, ctypes.byref(r)) != FS_OK:
            raise FsError(FS_ERR_ARG, "fs_server_stats failed")
        return {k: getattr(r, k) for k, _ in ServerReport._fields_}

    def close(self):
        if self.h:
            self.lib.fs_server_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _stats(s):
    return {"iters": s.iters, "status": s.status, "reliable_updates": s.reliable_updates,
            "restarts": s.restarts, "true_resid": s.true_resid, "fallback_iters": s.fallback_iters}


# Module-level functions with the C ABI's names.
def fs_ctx_create(dims, bc_t=-1, device=0):
    return Context(dims, bc_t, device)


def fs_set_gauge(ctx, U):
    return ctx.fs_set_gauge(U)


def fs_set_clover(ctx, c_sw):
    return ctx.fs_set_clover(c_sw)


def wilson_dslash(ctx, m, sigma, psi, prec="f64", link_compress=18):
    return ctx.wilson_dslash(m, sigma, psi, prec, link_compress)


def shifted_solve(ctx, m, sigmas, b, **kw):
    return ctx.shifted_solve(m, sigmas, b, **kw)


def mlmc_level_trace(ctx, m, sigmas, gamma, p, n_samples, seed, job=0, estimator="split_even", **kw):
    return ctx.mlmc_level_trace(m, sigmas, gamma, p, n_samples, seed, job, estimator, **kw)


def variance_sample(ctx, m, s_hat, gamma, p_list, n_s, seed, job=0, **kw):
    return ctx.variance_sample(m, s_hat, gamma, p_list, n_s, seed, job, **kw)


def fs_noise_codes(ctx, seed, job, level, sample):
    return ctx.fs_noise_codes(seed, job, level, sample)
