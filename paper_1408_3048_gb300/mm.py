"""Thin ctypes binding of libmm (include/mm.h): argument marshalling only.

Every ``mm_*`` function here has the same name and arguments as its C counterpart;
arrays may be torch tensors (device or host) or numpy arrays (host), passed by pointer.
All arithmetic runs in the library's CUDA kernels.  There is no fallback: if libmm.so
is missing or fails to load, the first call raises.

``Plan`` wraps one ``mm_plan_t`` with torch tensors for the common calls.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "libmm.so")

MM_OK, MM_ERR_ARG, MM_ERR_CUDA, MM_ERR_OOM, MM_ERR_NOT_SPD = 0, 1, 2, 3, 4
MM_ERR_NOT_CONVERGED, MM_ERR_NUMERIC, MM_ERR_TIMEOUT, MM_ERR_STATE = 5, 6, 7, 8
MM_FP64, MM_FP32 = 0, 1
MM_WINDOW_GAUSS, MM_WINDOW_RECT = 0, 1
MM_PREC_BD, MM_PREC_TWOLEVEL, MM_PREC_ADEF2 = 0, 1, 2
MM_SOLVE_FP64, MM_SOLVE_MIXED = 0, 1
MM_BATCH_PAIR, MM_BATCH_REAL, MM_BATCH_TENSOR = 0, 1, 2
MM_RESID_DF32, MM_RESID_FP64 = 0, 1

STATUS_NAMES = {0: "MM_OK", 1: "MM_ERR_ARG", 2: "MM_ERR_CUDA", 3: "MM_ERR_OOM", 4: "MM_ERR_NOT_SPD",
                5: "MM_ERR_NOT_CONVERGED", 6: "MM_ERR_NUMERIC", 7: "MM_ERR_TIMEOUT", 8: "MM_ERR_STATE"}

# every symbol include/mm.h declares (checked by the CPU tests)
EXPORTS = ["mm_plan", "mm_plan_info", "mm_plan_pixels", "mm_plan_row", "mm_gather", "mm_apply_ninv",
           "mm_scatter", "mm_apply_A", "mm_rhs", "mm_precond", "mm_build_coarse", "mm_coarse_info",
           "mm_coarse_vectors", "mm_solve", "mm_profile", "mm_profile_read", "mm_last_error", "mm_destroy",
           "mm_version", "mm_launch_count", "mm_apply_A_static", "mm_solve_ex", "mm_grad", "mm_apply_A_batch",
           "mm_solve_batch", "mm_autotune_read", "mm_batch_config", "mm_build_coarse_apriori",
           "mm_build_coarse_eps", "mm_coarse_import", "mm_build_coarse_arnoldi", "mm_solve_history",
           "mm_pcg_barrier_check", "mm_residual", "mm_scatter_config"]


class mm_psd(ctypes.Structure):
    _fields_ = [("sigma", ctypes.c_double), ("fknee", ctypes.c_double), ("alpha", ctypes.c_double)]


class mm_opts(ctypes.Structure):
    _fields_ = [("ncomp", ctypes.c_int32), ("lambda_", ctypes.c_int32), ("window", ctypes.c_int32),
                ("fft_log2_f64", ctypes.c_int32), ("fft_log2_f32", ctypes.c_int32),
                ("autotune", ctypes.c_int32), ("fsamp", ctypes.c_double), ("rcond_min", ctypes.c_double),
                ("stream", ctypes.c_void_p), ("scatter_lanes", ctypes.c_int32)]


class mm_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("outer", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("fp64_products", ctypes.c_int32), ("rel_resid", ctypes.c_double),
                ("rel_resid_rec", ctypes.c_double), ("ms_total", ctypes.c_double), ("ms_rhs", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class mm_solve_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxit", ctypes.c_int32), ("kind", ctypes.c_int32),
                ("solver", ctypes.c_int32), ("max_outer", ctypes.c_int32), ("inner_tol_min", ctypes.c_double),
                ("first_inner_tol", ctypes.c_double), ("residual", ctypes.c_int32)]


class MMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None
P = ctypes.c_void_p
I32 = ctypes.c_int32
I64 = ctypes.c_int64
D = ctypes.c_double
PP = ctypes.POINTER(ctypes.c_void_p)

_SIGS = {
    "mm_plan": (I32, [PP, P, I64, I32, P, P, I32, P, P, I32, ctypes.POINTER(mm_opts)]),
    "mm_plan_info": (I32, [P, P, P, P, P, P]),
    "mm_plan_pixels": (I32, [P, P, P]),
    "mm_plan_row": (I32, [P, I32, P]),
    "mm_gather": (I32, [P, ctypes.c_int, P, P]),
    "mm_apply_ninv": (I32, [P, ctypes.c_int, P, P]),
    "mm_scatter": (I32, [P, ctypes.c_int, P, P]),
    "mm_apply_A": (I32, [P, ctypes.c_int, P, P]),
    "mm_apply_A_static": (I32, [P, ctypes.c_int, P, P]),
    "mm_rhs": (I32, [P, P, P]),
    "mm_precond": (I32, [P, ctypes.c_int, ctypes.c_int, P, P]),
    "mm_build_coarse": (I32, [P, ctypes.c_int, ctypes.c_int, P, D, ctypes.c_int]),
    "mm_coarse_info": (I32, [P, P, P]),
    "mm_coarse_vectors": (I32, [P, P]),
    "mm_solve": (I32, [P, P, D, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, ctypes.POINTER(mm_stats)]),
    "mm_solve_ex": (I32, [P, P, ctypes.POINTER(mm_solve_opts), P, ctypes.POINTER(mm_stats)]),
    "mm_grad": (I32, [P, P, P, P, P, P, ctypes.POINTER(mm_solve_opts), ctypes.POINTER(mm_stats)]),
    "mm_apply_A_batch": (I32, [P, ctypes.c_int, P, P]),
    "mm_solve_batch": (I32, [P, P, ctypes.c_int, ctypes.POINTER(mm_solve_opts), P, ctypes.POINTER(mm_stats)]),
    "mm_autotune_read": (I32, [P, P, P]),
    "mm_build_coarse_apriori": (I32, [P, ctypes.c_int]),
    "mm_build_coarse_eps": (I32, [P, ctypes.c_int, ctypes.c_double, ctypes.c_int, P, ctypes.c_double, ctypes.c_int]),
    "mm_coarse_import": (I32, [P, P, ctypes.c_int]),
    "mm_build_coarse_arnoldi": (I32, [P, ctypes.c_int, ctypes.c_double, P, ctypes.c_double, ctypes.c_int]),
    "mm_batch_config": (I32, [P, ctypes.c_int32, P, P, P]),
    "mm_profile": (I32, [P, ctypes.c_int]),
    "mm_profile_read": (I32, [P, P, P]),
    "mm_solve_history": (I32, [P, I32, P, P]),
    "mm_pcg_barrier_check": (I32, [P, I32, ctypes.c_double]),
    "mm_residual": (I32, [P, ctypes.c_int, P, P, P]),
    "mm_scatter_config": (I32, [P, P, P]),
    "mm_last_error": (ctypes.c_char_p, [P]),
    "mm_destroy": (None, [P]),
    "mm_version": (ctypes.c_char_p, []),
    "mm_launch_count": (I64, []),
}


def lib():
    """Load libmm.so (built in-tree by ``paper_1408_3048_gb300.build``); raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIBPATH):
            raise RuntimeError(f"libmm.so is not built ({LIBPATH}); run paper_1408_3048_gb300.build.build()")
        L = ctypes.CDLL(LIBPATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


_DT = {MM_FP64: "float64", MM_FP32: "float32"}


def _expect(a, dtype, n, what):
    """Reject, before the C call, an array whose element type or size differs from what the
    call reads or writes: a plain pointer carries neither, and a float32 buffer passed for
    doubles would be read past its end.  dtype None (an unknown precision code) leaves the
    type to the library, which rejects the code itself."""
    if a is None:
        return
    if isinstance(a, np.ndarray):
        dt, cnt = a.dtype.name, a.size
    elif hasattr(a, "data_ptr"):
        dt, cnt = str(a.dtype).rsplit(".", 1)[-1], a.numel()
    else:
        raise TypeError(f"{what}: unsupported array type {type(a)}")
    if dtype is not None and dt != dtype:
        raise TypeError(f"{what}: expected {dtype} elements, got {dt}")
    if cnt != n:
        raise ValueError(f"{what}: expected {n} elements, got {cnt}")


def _check(status, plan=None):
    if status != MM_OK:
        msg = lib().mm_last_error(plan).decode()
        raise MMError(status, msg)


# ---------------------------------------------------------------- C-named wrappers
def mm_version():
    return lib().mm_version().decode()


def mm_launch_count():
    return int(lib().mm_launch_count())


def mm_last_error(plan):
    return lib().mm_last_error(plan).decode()


def mm_plan(pix, nt, npix_sky, weights, interval_off, K, interval_psd, psd, npsd, opts):
    h = ctypes.c_void_p()
    st = lib().mm_plan(ctypes.byref(h), _ptr(pix), int(nt), int(npix_sky), _ptr(weights), _ptr(interval_off),
                       int(K), _ptr(interval_psd), ctypes.cast(psd, ctypes.c_void_p), int(npsd), ctypes.byref(opts))
    _check(st, None)
    return h.value


def mm_plan_info(plan):
    npix = ctypes.c_int32()
    n = ctypes.c_int64()
    nk = ctypes.c_int64()
    b64 = ctypes.c_int32()
    b32 = ctypes.c_int32()
    _check(lib().mm_plan_info(plan, ctypes.byref(npix), ctypes.byref(n), ctypes.byref(nk), ctypes.byref(b64),
                              ctypes.byref(b32)), plan)
    return {"npix_obs": npix.value, "n": n.value, "nkept": nk.value, "fft_block_f64": b64.value,
            "fft_block_f32": b32.value}


def mm_autotune_read(plan):
    """(ms_f64, ms_f32): timed candidate blocks, index log2(B) - 9, 0 where not timed."""
    a = (ctypes.c_float * 16)()
    b = (ctypes.c_float * 16)()
    _check(lib().mm_autotune_read(plan, a, b), plan)
    return list(a), list(b)


def mm_batch_config(plan, R, kind=-1):
    """(kind, log2_block, [ms_pair, ms_real, ms_tensor]) of the batched operator for R columns."""
    kind = ctypes.c_int32(int(kind))
    lb = ctypes.c_int32()
    ms = (ctypes.c_float * 3)()
    _check(lib().mm_batch_config(plan, int(R), ctypes.byref(kind), ctypes.byref(lb), ms), plan)
    return kind.value, lb.value, list(ms)


def mm_plan_pixels(plan, obs2sky, hits):
    _check(lib().mm_plan_pixels(plan, _ptr(obs2sky), _ptr(hits)), plan)


def mm_plan_row(plan, psd_id, row):
    _check(lib().mm_plan_row(plan, int(psd_id), _ptr(row)), plan)


def mm_gather(plan, precision, x, y):
    _check(lib().mm_gather(plan, precision, _ptr(x), _ptr(y)), plan)


def mm_apply_ninv(plan, precision, y, z):
    _check(lib().mm_apply_ninv(plan, precision, _ptr(y), _ptr(z)), plan)


def mm_scatter(plan, precision, z, w):
    _check(lib().mm_scatter(plan, precision, _ptr(z), _ptr(w)), plan)


def mm_apply_A(plan, precision, x, y):
    _check(lib().mm_apply_A(plan, precision, _ptr(x), _ptr(y)), plan)


def mm_apply_A_static(plan, precision, x, y):
    _check(lib().mm_apply_A_static(plan, precision, _ptr(x), _ptr(y)), plan)


def mm_rhs(plan, d, b):
    _check(lib().mm_rhs(plan, _ptr(d), _ptr(b)), plan)


def mm_precond(plan, kind, precision, r, z):
    _check(lib().mm_precond(plan, kind, precision, _ptr(r), _ptr(z)), plan)


def mm_build_coarse(plan, k, precision, bprime, tol, maxit):
    _check(lib().mm_build_coarse(plan, int(k), precision, _ptr(bprime), float(tol), int(maxit)), plan)


def mm_build_coarse_eps(plan, kmax, eps_tol, precision, bprime, tol, maxit):
    _check(lib().mm_build_coarse_eps(plan, int(kmax), float(eps_tol), precision, _ptr(bprime), float(tol),
                                     int(maxit)), plan)


def mm_build_coarse_arnoldi(plan, kmax, eps_tol, bprime, tol, maxit):
    _check(lib().mm_build_coarse_arnoldi(plan, int(kmax), float(eps_tol), _ptr(bprime), float(tol), int(maxit)),
           plan)


def mm_coarse_import(plan, Z, k):
    _check(lib().mm_coarse_import(plan, _ptr(Z), int(k)), plan)


def mm_build_coarse_apriori(plan, r):
    _check(lib().mm_build_coarse_apriori(plan, int(r)), plan)


def mm_coarse_info(plan):
    k = ctypes.c_int32()
    _check(lib().mm_coarse_info(plan, ctypes.byref(k), None), plan)
    vals = np.zeros(max(k.value, 1), dtype=np.float64)
    _check(lib().mm_coarse_info(plan, None, vals.ctypes.data), plan)
    return k.value, vals[: k.value]


def mm_coarse_vectors(plan, Z):
    _check(lib().mm_coarse_vectors(plan, _ptr(Z)), plan)


def mm_solve(plan, d, tol, maxit, kind, solver, m, raise_on_error=True):
    st = mm_stats()
    status = lib().mm_solve(plan, _ptr(d), float(tol), int(maxit), kind, solver, _ptr(m), ctypes.byref(st))
    if raise_on_error:
        _check(status, plan)
    return status, st


def mm_profile(plan, enable):
    _check(lib().mm_profile(plan, int(enable)), plan)


def mm_profile_read(plan):
    ms = np.zeros(8, dtype=np.float64)
    n = np.zeros(8, dtype=np.int64)
    _check(lib().mm_profile_read(plan, ms.ctypes.data, n.ctypes.data), plan)
    return ms, n


def mm_solve_history(plan):
    """||r_j|| / ||b|| after each product A p of the last solve (numpy float64)."""
    cnt = ctypes.c_int32()
    _check(lib().mm_solve_history(plan, 0, None, ctypes.byref(cnt)), plan)
    h = np.zeros(max(cnt.value, 1), dtype=np.float64)
    _check(lib().mm_solve_history(plan, cnt.value, h.ctypes.data, ctypes.byref(cnt)), plan)
    return h[: cnt.value]


def mm_scatter_config(plan):
    """(lanes per pixel of the scatter, [ms at 32, 16, 8 lanes] or zeros)."""
    lpp = ctypes.c_int32()
    ms = (ctypes.c_float * 3)()
    _check(lib().mm_scatter_config(plan, ctypes.byref(lpp), ms), plan)
    return lpp.value, list(ms)


def mm_residual(plan, arith, d, x, r):
    _check(lib().mm_residual(plan, int(arith), _ptr(d), _ptr(x), _ptr(r)), plan)


def mm_pcg_barrier_check(plan, absent_blocks, wait_s):
    """Status of a PCG start whose grid barrier waits for `absent_blocks` blocks that are
    never launched, each wait limited to wait_s seconds (MM_ERR_TIMEOUT when > 0)."""
    return int(lib().mm_pcg_barrier_check(plan, int(absent_blocks), float(wait_s)))


def mm_solve_ex(plan, d, opts, m, raise_on_error=True):
    st = mm_stats()
    status = lib().mm_solve_ex(plan, _ptr(d), ctypes.byref(opts), _ptr(m), ctypes.byref(st))
    if raise_on_error:
        _check(status, plan)
    return status, st


def mm_grad(plan, d, m, g, dL_dd, dL_dpsd, opts):
    st = mm_stats()
    _check(lib().mm_grad(plan, _ptr(d), _ptr(m), _ptr(g), _ptr(dL_dd), _ptr(dL_dpsd), ctypes.byref(opts),
                         ctypes.byref(st)), plan)
    return st


def mm_apply_A_batch(plan, R, X, Y):
    _check(lib().mm_apply_A_batch(plan, int(R), _ptr(X), _ptr(Y)), plan)


def mm_solve_batch(plan, D, R, opts, M, raise_on_error=True):
    st = (mm_stats * int(R))()
    status = lib().mm_solve_batch(plan, _ptr(D), int(R), ctypes.byref(opts), _ptr(M), st)
    if raise_on_error:
        _check(status, plan)
    return status, [x.as_dict() for x in st]


def mm_destroy(plan):
    lib().mm_destroy(plan)


# ------------------------------------------------------------------------ Plan class
def _torch():
    import torch
    return torch


class Plan:
    """One map-making problem on the current CUDA device (torch tensors in and out)."""

    def __init__(self, pix, npix_sky, weights, offsets, interval_psd, psds, lam, fsamp=100.0, ncomp=None,
                 window=MM_WINDOW_GAUSS, rcond_min=1e-6, fft_log2=(0, 0), stream=None, autotune=False,
                 scatter_lanes=0):
        torch = _torch()
        self._torch = torch
        pix = np.ascontiguousarray(np.asarray(pix, dtype=np.int32))
        if ncomp is None:
            ncomp = 1 if weights is None else 3
        w = None if weights is None else np.ascontiguousarray(np.asarray(weights, dtype=np.float64).reshape(-1, 2))
        off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        ipsd = np.ascontiguousarray(np.asarray(interval_psd, dtype=np.int32))
        ps = np.asarray(psds, dtype=np.float64).reshape(-1, 3)
        arr = (mm_psd * len(ps))(*[mm_psd(*map(float, p)) for p in ps])
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        o = mm_opts(ncomp=ncomp, lambda_=int(lam), window=window, fft_log2_f64=int(fft_log2[0]),
                    fft_log2_f32=int(fft_log2[1]), autotune=int(bool(autotune)), fsamp=float(fsamp), rcond_min=float(rcond_min),
                    stream=stream.cuda_stream, scatter_lanes=int(scatter_lanes))
        self.handle = mm_plan(pix, pix.size, npix_sky, w, off, off.size - 1, ipsd, arr, len(ps), o)
        info = mm_plan_info(self.handle)
        self.npix_obs = info["npix_obs"]
        self.n = info["n"]
        self.nkept = info["nkept"]
        self.fft_block_f64 = info["fft_block_f64"]
        self.fft_block_f32 = info["fft_block_f32"]
        self.nt = int(pix.size)
        self.ncomp = ncomp
        self.lam = int(lam)
        self.npsd = len(ps)
        self.psds = ps.copy()     # (sigma, fknee, alpha) per PSD id, as the plan was built

    # helpers
    def _dtype(self, precision):
        return self._torch.float64 if precision == MM_FP64 else self._torch.float32

    def _new(self, size, precision):
        return self._torch.empty(size, dtype=self._dtype(precision), device="cuda")

    def pixels(self):
        o2s = np.zeros(self.npix_obs, dtype=np.int32)
        hits = np.zeros(self.npix_obs, dtype=np.int32)
        mm_plan_pixels(self.handle, o2s, hits)
        return o2s, hits

    def row(self, psd_id):
        r = np.zeros(self.lam + 1, dtype=np.float64)
        mm_plan_row(self.handle, psd_id, r)
        return r

    def gather(self, x, precision=MM_FP64):
        _expect(x, _DT.get(precision), self.n, "x")
        y = self._new(self.nt, precision)
        self._sync_in()
        mm_gather(self.handle, precision, x, y)
        return y

    def apply_ninv(self, y, precision=MM_FP64):
        _expect(y, _DT.get(precision), self.nt, "y")
        z = self._new(self.nt, precision)
        self._sync_in()
        mm_apply_ninv(self.handle, precision, y, z)
        return z

    def scatter(self, z, precision=MM_FP64):
        _expect(z, _DT.get(precision), self.nt, "z")
        w = self._new(self.n, precision)
        self._sync_in()
        mm_scatter(self.handle, precision, z, w)
        return w

    def apply_A(self, x, precision=MM_FP64, out=None):
        _expect(x, _DT.get(precision), self.n, "x")
        _expect(out, _DT.get(precision), self.n, "out")
        y = self._new(self.n, precision) if out is None else out
        self._sync_in()
        mm_apply_A(self.handle, precision, x, y)
        return y

    def rhs(self, d):
        _expect(d, "float64", self.nt, "d")
        b = self._new(self.n, MM_FP64)
        self._sync_in()
        mm_rhs(self.handle, d, b)
        return b

    def precond(self, r, kind=MM_PREC_BD, precision=MM_FP64):
        _expect(r, _DT.get(precision), self.n, "r")
        z = self._new(self.n, precision)
        self._sync_in()
        mm_precond(self.handle, kind, precision, r, z)
        return z

    def build_coarse(self, k, precision=MM_FP64, bprime=None, tol=1e-6, maxit=1000):
        _expect(bprime, "float64", self.n, "bprime")
        self._sync_in()
        mm_build_coarse(self.handle, k, precision, bprime, tol, maxit)
        return mm_coarse_info(self.handle)

    def build_coarse_eps(self, eps_tol, kmax=64, precision=MM_FP64, bprime=None, tol=1e-6, maxit=1000):
        """A posteriori coarse space from the Ritz pairs below eps_tol (at most kmax)."""
        _expect(bprime, "float64", self.n, "bprime")
        self._sync_in()
        mm_build_coarse_eps(self.handle, kmax, eps_tol, precision, bprime, tol, maxit)
        return mm_coarse_info(self.handle)

    def build_coarse_arnoldi(self, eps_tol, kmax=64, bprime=None, tol=1e-6, maxit=1000):
        """A posteriori coarse space from Arnoldi on M_BD A (Algorithm 1); returns (k, values)."""
        _expect(bprime, "float64", self.n, "bprime")
        self._sync_in()
        mm_build_coarse_arnoldi(self.handle, kmax, eps_tol, bprime, tol, maxit)
        return mm_coarse_info(self.handle)

    def coarse_import(self, Z):
        """Install a coarse basis Z (numpy or torch, shape [n, k]); returns k."""
        Zc = np.ascontiguousarray(np.asarray(Z.cpu() if hasattr(Z, "cpu") else Z, dtype=np.float64).T)
        self._sync_in()
        mm_coarse_import(self.handle, Zc, Zc.shape[0])
        return mm_coarse_info(self.handle)[0]

    def build_coarse_apriori(self, r):
        """A priori coarse space Z_S merged into r interval groups; returns the kept k."""
        self._sync_in()
        mm_build_coarse_apriori(self.handle, r)
        return mm_coarse_info(self.handle)[0]

    def coarse_vectors(self):
        k, _ = mm_coarse_info(self.handle)
        Z = np.zeros(k * self.n, dtype=np.float64)
        mm_coarse_vectors(self.handle, Z)
        return Z.reshape(k, self.n).T.copy()

    def solve(self, d, tol=1e-6, maxit=1000, kind=MM_PREC_BD, solver=MM_SOLVE_FP64, out=None,
              raise_on_error=True, **extra):
        """extra: max_outer, inner_tol_min, first_inner_tol, residual (mm_solve_opts)."""
        _expect(d, "float64", self.nt, "d")
        _expect(out, "float64", self.n, "out")
        m = self._new(self.n, MM_FP64) if out is None else out
        if extra:
            o = mm_solve_opts(tol=float(tol), maxit=int(maxit), kind=kind, solver=solver,
                              max_outer=int(extra.get("max_outer", 0)),
                              inner_tol_min=float(extra.get("inner_tol_min", 0.0)),
                              first_inner_tol=float(extra.get("first_inner_tol", 0.0)),
                              residual=int(extra.get("residual", MM_RESID_DF32)))
            self._sync_in()
            status, st = mm_solve_ex(self.handle, d, o, m, raise_on_error)
        else:
            self._sync_in()
            status, st = mm_solve(self.handle, d, tol, maxit, kind, solver, m, raise_on_error)
        return m, st.as_dict(), status

    def grad(self, d, m, g, tol=1e-10, maxit=10000, kind=MM_PREC_BD, solver=MM_SOLVE_FP64, want_d=True,
             want_psd=True):
        """(dL/dd [nt] tensor or None, dL/dtheta [npsd, 3] numpy or None, stats) for g = dL/dm."""
        _expect(d, "float64", self.nt, "d")
        _expect(m, "float64", self.n, "m")
        _expect(g, "float64", self.n, "g")
        o = mm_solve_opts(tol=float(tol), maxit=int(maxit), kind=kind, solver=solver)
        dd = self._new(self.nt, MM_FP64) if want_d else None
        dp = np.zeros((self.npsd, 3), dtype=np.float64) if want_psd else None
        self._sync_in()
        st = mm_grad(self.handle, d, m, g, dd, dp, o)
        return dd, dp, st.as_dict()

    def autotune_ms(self):
        """Timed overlap-save blocks {log2 B: ms} per precision (autotuned plans)."""
        a, b = mm_autotune_read(self.handle)
        return ({i + 9: v for i, v in enumerate(a) if v > 0}, {i + 9: v for i, v in enumerate(b) if v > 0})

    def batch_config(self, R, kind=-1):
        """(kind, log2 block, timings) of the batched operator; fixes it for this plan."""
        self._sync_in()
        return mm_batch_config(self.handle, R, kind)

    def apply_A_batch(self, X, out=None):
        """Y[r] = A X[r] in FP32 for a float32 cuda tensor X [R, n] (R <= 64)."""
        R = X.shape[0]
        _expect(X, "float32", R * self.n, "X")
        _expect(out, "float32", R * self.n, "out")
        Y = self._torch.empty((R, self.n), dtype=self._torch.float32, device="cuda") if out is None else out
        self._sync_in()
        mm_apply_A_batch(self.handle, R, X, Y)
        return Y

    def solve_batch(self, D, tol=1e-6, maxit=5000, out=None, raise_on_error=True, **extra):
        """Maps for D [R, nt] float64 (mixed precision, block-Jacobi); returns (M, stats, status)."""
        R = D.shape[0]
        _expect(D, "float64", R * self.nt, "D")
        _expect(out, "float64", R * self.n, "out")
        M = self._torch.empty((R, self.n), dtype=self._torch.float64, device="cuda") if out is None else out
        o = mm_solve_opts(tol=float(tol), maxit=int(maxit), kind=MM_PREC_BD, solver=MM_SOLVE_MIXED,
                          max_outer=int(extra.get("max_outer", 0)),
                          inner_tol_min=float(extra.get("inner_tol_min", 0.0)),
                          first_inner_tol=float(extra.get("first_inner_tol", 0.0)),
                          residual=int(extra.get("residual", MM_RESID_DF32)))
        self._sync_in()
        status, st = mm_solve_batch(self.handle, D, R, o, M, raise_on_error)
        return M, st, status

    def _sync_in(self):
        """Make work queued on the caller's current stream visible to the plan's stream."""
        cur = self._torch.cuda.current_stream()
        if cur.cuda_stream != self.stream.cuda_stream:
            cur.synchronize()

    def profile(self, enable=True):
        mm_profile(self.handle, enable)

    def solve_history(self):
        """Relative recursive residual after each A p of the last solve (Sec. 5.1)."""
        return mm_solve_history(self.handle)

    def residual(self, d, x, arith=MM_RESID_DF32, out=None):
        """r = P^T N^-1 (d - P x) (FP64 data; band product in double-float or FP64)."""
        _expect(d, "float64", self.nt, "d")
        _expect(x, "float64", self.n, "x")
        _expect(out, "float64", self.n, "out")
        r = self._new(self.n, MM_FP64) if out is None else out
        self._sync_in()
        mm_residual(self.handle, arith, d, x, r)
        return r

    def scatter_config(self):
        """(lanes per pixel of the scatter, timings at 32 / 16 / 8 lanes when autotuned)."""
        return mm_scatter_config(self.handle)

    def barrier_check(self, absent_blocks, wait_s):
        """Status (int) of the bounded-wait diagnostic mm_pcg_barrier_check."""
        self._sync_in()
        return mm_pcg_barrier_check(self.handle, absent_blocks, wait_s)

    def profile_read(self):
        """{stage: (total ms, launches)} per kernel and precision."""
        ms, n = mm_profile_read(self.handle)
        names = ["toeplitz_f64", "toeplitz_f32", "scatter_f64", "scatter_f32", "pcg_f64", "pcg_f32", "toeplitz_df"]
        return {nm: (float(ms[i]), int(n[i])) for i, nm in enumerate(names)}

    def close(self):
        if getattr(self, "handle", None):
            mm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ autograd wrapper
def map_solve(plan, d, theta, tol=1e-10, maxit=10000, kind=MM_PREC_BD, solver=MM_SOLVE_FP64,
              adjoint_tol=None):
    """m = (P^T N^-1 P)^-1 P^T N^-1 d as a differentiable torch op.

    d      cuda float64 tensor [nt] (time-ordered data)
    theta  float64 tensor [npsd, 3] = (sigma, fknee, alpha) per PSD id; it must equal the
           plan's PSDs (plan.psds, the values the plan was built from: ValueError
           otherwise) and only carries their gradient.
    The backward pass runs one adjoint PCG solve (A is symmetric) and the PSD gradient
    products of mm_grad; no Krylov vectors are kept from the forward solve.
    """
    import torch

    th = theta.detach().cpu().numpy().astype(np.float64).reshape(-1, 3)
    ps = np.asarray(plan.psds, dtype=np.float64).reshape(-1, 3)
    if th.shape != ps.shape or not np.array_equal(th, ps):
        raise ValueError("theta must equal the PSD parameters the plan was built from (plan.psds); "
                         "build a new plan for other noise parameters")

    class _MapSolve(torch.autograd.Function):
        @staticmethod
        def forward(ctx, d_, theta_):
            m, st, _ = plan.solve(d_.contiguous(), tol=tol, maxit=maxit, kind=kind, solver=solver)
            ctx.save_for_backward(d_, m)
            return m

        @staticmethod
        def backward(ctx, g):
            d_, m = ctx.saved_tensors
            need_d, need_th = ctx.needs_input_grad
            dd, dp, _ = plan.grad(d_, m, g.contiguous().to(torch.float64),
                                  tol=adjoint_tol if adjoint_tol is not None else tol, maxit=maxit,
                                  kind=kind, solver=solver, want_d=need_d, want_psd=need_th)
            gth = torch.from_numpy(dp).to(theta.device) if need_th else None
            return dd, gth

    return _MapSolve.apply(d, theta)
