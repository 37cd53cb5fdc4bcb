"""Thin ctypes binding of libmgmc.so (include/mgmc.h).

Argument marshalling only: every step of the sampler runs in the CUDA
kernels of the library.  PyTorch provides device memory (its caching
allocator is handed to the library as the mgmc_allocator) and streams.
If the library has not been built, or no CUDA device is present, the calls
raise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmgmc.so")

MGMC_FP64 = 0
MGMC_FP32 = 1
MGMC_FD = 0
MGMC_Q1 = 1
MGMC_SSL = 2
MGMC_MAX_OBS = 64
MGMC_NOALLOC_MAX_SERIES = 65536

STATUS = {0: "MGMC_OK", 1: "MGMC_ERR_ARG", 2: "MGMC_ERR_CUDA", 3: "MGMC_ERR_OOM", 4: "MGMC_ERR_NOT_SPD",
          5: "MGMC_ERR_TIMEOUT", 6: "MGMC_ERR_STATE", 7: "MGMC_ERR_NUMERIC"}


class MGMCError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class mgmc_config(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int), ("n_levels", ctypes.c_int), ("nu1", ctypes.c_int),
                ("nu2", ctypes.c_int), ("precision", ctypes.c_int), ("scale_hd", ctypes.c_int),
                ("coarse_max_n", ctypes.c_int), ("gibbs", ctypes.c_int), ("disc", ctypes.c_int),
                ("band_min_n", ctypes.c_int), ("gamma", ctypes.c_int)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class mgmc_allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", ctypes.c_void_p)]


class mgmc_problem(ctypes.Structure):
    _fields_ = [("kappa2", ctypes.POINTER(ctypes.c_double)), ("kappa2_const", ctypes.c_double), ("m", ctypes.c_int),
                ("obs_site", ctypes.POINTER(ctypes.c_int32)), ("obs_w", ctypes.POINTER(ctypes.c_double)),
                ("nnz_per_obs", ctypes.c_int), ("Gamma", ctypes.POINTER(ctypes.c_double)),
                ("y", ctypes.POINTER(ctypes.c_double)), ("n_qoi", ctypes.c_int),
                ("qoi_site", ctypes.POINTER(ctypes.c_int32)), ("qoi_w", ctypes.POINTER(ctypes.c_double))]


class mgmc_stats(ctypes.Structure):
    _fields_ = [("mean", ctypes.c_double), ("var", ctypes.c_double), ("tau_int", ctypes.c_double),
                ("tau_err", ctypes.c_double), ("ess", ctypes.c_double), ("window", ctypes.c_int64),
                ("n_used", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_I32P = ctypes.POINTER(ctypes.c_int32)
_F64P = ctypes.POINTER(ctypes.c_double)
_lib = None

# every symbol include/mgmc.h declares
EXPORTS = ("mgmc_config_default", "mgmc_create", "mgmc_point_obs_rows", "mgmc_sample", "mgmc_mean_solve",
           "mgmc_qoi_stats", "mgmc_qoi_stats_noalloc", "mgmc_info", "mgmc_level_n", "mgmc_launches_per_cycle", "mgmc_set_profiling",
           "mgmc_profile_times", "mgmc_set_band_min_n", "mgmc_set_coarse_threads", "mgmc_create_batch", "mgmc_sample_batch", "mgmc_get_state", "mgmc_destroy",
           "mgmc_tc_gemm", "mgmc_unet_create", "mgmc_unet_n_params", "mgmc_unet_get_params",
           "mgmc_unet_set_params", "mgmc_unet_inputs", "mgmc_unet_gradient", "mgmc_unet_train",
           "mgmc_unet_predict", "mgmc_unet_destroy", "mgmc_check_status", "mgmc_set_wait_limit",
           "mgmc_fine_operator",
           "mgmc_last_error")


def load():
    """Load libmgmc.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2407_12149_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    L.mgmc_last_error.restype = ctypes.c_char_p
    L.mgmc_config_default.argtypes = [ctypes.POINTER(mgmc_config), ctypes.c_int, ctypes.c_int]
    L.mgmc_create.argtypes = [ctypes.POINTER(mgmc_config), ctypes.POINTER(mgmc_allocator), ctypes.c_void_p,
                              _F64P, ctypes.c_double, ctypes.c_int, _I32P, _F64P, ctypes.c_int, _F64P, _F64P,
                              ctypes.c_int, _I32P, _F64P, ctypes.POINTER(ctypes.c_void_p)]
    L.mgmc_point_obs_rows.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _F64P, _I32P, _F64P]
    L.mgmc_sample.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.mgmc_mean_solve.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_void_p,
                                  ctypes.POINTER(ctypes.c_int), _F64P, ctypes.c_void_p]
    L.mgmc_qoi_stats.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                                 ctypes.POINTER(mgmc_stats), ctypes.c_void_p]
    L.mgmc_qoi_stats_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                                         ctypes.POINTER(mgmc_stats), ctypes.c_void_p]
    L.mgmc_info.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                            ctypes.POINTER(ctypes.c_int)]
    L.mgmc_level_n.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    L.mgmc_launches_per_cycle.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]
    L.mgmc_set_profiling.argtypes = [ctypes.c_void_p, ctypes.c_int]
    L.mgmc_set_band_min_n.argtypes = [ctypes.c_void_p, ctypes.c_int]
    L.mgmc_set_coarse_threads.argtypes = [ctypes.c_void_p, ctypes.c_int]
    L.mgmc_profile_times.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float), ctypes.c_int, ctypes.c_void_p]
    L.mgmc_create_batch.argtypes = [ctypes.c_int, ctypes.POINTER(mgmc_config), ctypes.POINTER(mgmc_problem),
                                    ctypes.POINTER(mgmc_allocator), ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    L.mgmc_sample_batch.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint64,
                                    ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p, ctypes.c_void_p]
    L.mgmc_get_state.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    L.mgmc_tc_gemm.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                               ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                               ctypes.c_void_p]
    L.mgmc_unet_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                   ctypes.POINTER(mgmc_allocator), ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    L.mgmc_unet_n_params.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]
    L.mgmc_unet_get_params.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    L.mgmc_unet_set_params.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    L.mgmc_unet_inputs.argtypes = [ctypes.c_int, _F64P, ctypes.c_double, ctypes.c_int, _I32P, _F64P, ctypes.c_int,
                                   _F64P, ctypes.c_void_p]
    L.mgmc_unet_gradient.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p]
    L.mgmc_unet_train.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                  ctypes.c_int, ctypes.c_float, ctypes.c_uint64, ctypes.c_void_p]
    L.mgmc_unet_predict.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    L.mgmc_unet_destroy.argtypes = [ctypes.c_void_p]
    L.mgmc_destroy.argtypes = [ctypes.c_void_p]
    L.mgmc_check_status.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    L.mgmc_fine_operator.argtypes = [ctypes.POINTER(mgmc_config), _F64P, ctypes.c_double, _F64P]
    L.mgmc_set_wait_limit.argtypes = [ctypes.c_void_p, ctypes.c_int64]
    for name in EXPORTS:
        if name != "mgmc_last_error":
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(rc: int):
    if rc != 0:
        msg = load().mgmc_last_error()
        raise MGMCError(rc, msg.decode() if msg else "")


def _ptr(a, ctype):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctype))


def _torch():
    import torch
    return torch


def _stream_handle(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


class TorchAllocator:
    """mgmc_allocator backed by torch's CUDA caching allocator."""

    def __init__(self, device: int = 0):
        torch = _torch()
        self.device = device

        def _alloc(nbytes, stream, ctx):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), device)
            except Exception:
                return None

        def _free(ptr, stream, ctx):
            torch.cuda.caching_allocator_delete(ptr)

        self._a = ALLOC_FN(_alloc)
        self._f = FREE_FN(_free)
        self.struct = mgmc_allocator(self._a, self._f, None)


# --------------------------------------------------------------------------
# functions with the C names
# --------------------------------------------------------------------------

def mgmc_fine_operator(problem) -> np.ndarray:
    """The finest grid's operator A_L of a problem as the library assembles it:
    float64 [N, W^dim] stencil, W = 5 for the squared shifted Laplacian, else 3 (host only)."""
    p = problem
    disc = getattr(p, "disc", MGMC_FD)
    cfg = mgmc_config(p.dim, p.n, p.n_levels, 1, 1, MGMC_FP64, p.scale_hd, 0, 0, disc)
    k2 = None if p.kappa2 is None else np.ascontiguousarray(p.kappa2, dtype=np.float64).ravel()
    out = np.empty((p.N, (5 if disc == MGMC_SSL else 3) ** p.dim), dtype=np.float64)
    _check(load().mgmc_fine_operator(ctypes.byref(cfg), _ptr(k2, ctypes.c_double), float(p.kappa2_const),
                                     _ptr(out, ctypes.c_double)))
    return out


def mgmc_check_status(h, stream=None):
    _check(load().mgmc_check_status(h, _stream_handle(stream)))


def mgmc_set_wait_limit(h, limit_ns: int):
    _check(load().mgmc_set_wait_limit(h, int(limit_ns)))


def mgmc_point_obs_rows(dim: int, n: int, xyz: np.ndarray):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, dim)
    m = xyz.shape[0]
    site = np.empty((m, 1 << dim), dtype=np.int32)
    w = np.empty((m, 1 << dim), dtype=np.float64)
    _check(load().mgmc_point_obs_rows(dim, n, m, _ptr(xyz, ctypes.c_double), _ptr(site, ctypes.c_int32),
                                      _ptr(w, ctypes.c_double)))
    return site, w


def mgmc_create(dim, n, *, n_levels=0, nu1=1, nu2=1, precision=MGMC_FP64, scale_hd=1, coarse_max_n=0,
                kappa2=None, kappa2_const=10.0, obs_site=None, obs_w=None, Gamma=None, y=None,
                qoi_site=None, qoi_w=None, allocator: Optional[TorchAllocator] = None, stream=None, gibbs=0,
                disc=MGMC_FD, band_min_n=0, gamma=0):
    L = load()
    cfg = mgmc_config(dim, n, n_levels, nu1, nu2, precision, scale_hd, coarse_max_n, gibbs, disc, band_min_n,
                      gamma)
    k2 = None if kappa2 is None else np.ascontiguousarray(kappa2, dtype=np.float64).ravel()
    if obs_site is None:
        m, nnz, os_, ow_, G_, y_ = 0, 1, None, None, None, None
    else:
        os_ = np.ascontiguousarray(obs_site, dtype=np.int32)
        ow_ = np.ascontiguousarray(obs_w, dtype=np.float64)
        m, nnz = os_.shape
        G_ = np.ascontiguousarray(Gamma, dtype=np.float64)
        y_ = np.ascontiguousarray(y, dtype=np.float64)
    if qoi_site is None:
        nq, qs, qw = 0, None, None
    else:
        qs = np.ascontiguousarray(qoi_site, dtype=np.int32)
        qw = np.ascontiguousarray(qoi_w, dtype=np.float64)
        nq = qs.size
    h = ctypes.c_void_p()
    _check(L.mgmc_create(ctypes.byref(cfg), ctypes.byref(allocator.struct) if allocator else None,
                         _stream_handle(stream), _ptr(k2, ctypes.c_double), float(kappa2_const), m,
                         _ptr(os_, ctypes.c_int32), _ptr(ow_, ctypes.c_double), nnz, _ptr(G_, ctypes.c_double),
                         _ptr(y_, ctypes.c_double), nq, _ptr(qs, ctypes.c_int32), _ptr(qw, ctypes.c_double),
                         ctypes.byref(h)))
    return h


EPI_BIAS, EPI_RELU, EPI_BF16 = 1, 2, 4


def tc_gemm(A, B, out=None, splits=1, epilogue=0, bias=None, stream=None):
    """C = A B^T on the tensor cores: A [M][K], B [N][K] bfloat16 CUDA tensors
    (row strides multiples of 8); returns C [M][N] float32 (bfloat16 with EPI_BF16)."""
    torch = _torch()
    M, K = A.shape
    N = B.shape[0]
    if out is None:
        out = torch.empty(M, N, dtype=torch.bfloat16 if epilogue & EPI_BF16 else torch.float32, device=A.device)
    _check(load().mgmc_tc_gemm(ctypes.c_void_p(A.data_ptr()), A.stride(0), ctypes.c_void_p(B.data_ptr()),
                               B.stride(0), ctypes.c_void_p(out.data_ptr()), M, N, K, splits, epilogue,
                               ctypes.c_void_p(bias.data_ptr()) if bias is not None else None,
                               _stream_handle(stream)))
    return out


def mgmc_get_state(h, chain, x_ptr, stream=None):
    _check(load().mgmc_get_state(h, int(chain), ctypes.c_void_p(x_ptr), _stream_handle(stream)))


def mgmc_sample(h, n_steps, seed, step_offset, chain, x_ptr, qoi_ptr, stream=None):
    _check(load().mgmc_sample(h, int(n_steps), int(seed) & (2**64 - 1), int(step_offset), int(chain),
                              ctypes.c_void_p(x_ptr), ctypes.c_void_p(qoi_ptr) if qoi_ptr else None,
                              _stream_handle(stream)))


def mgmc_mean_solve(h, rtol, max_cycles, x_ptr, stream=None):
    c = ctypes.c_int()
    rr = ctypes.c_double()
    _check(load().mgmc_mean_solve(h, float(rtol), int(max_cycles), ctypes.c_void_p(x_ptr), ctypes.byref(c),
                                  ctypes.byref(rr), _stream_handle(stream)))
    return c.value, rr.value


def mgmc_qoi_stats(qoi_ptr, n, burn_in=0, S=1.5, stream=None):
    out = mgmc_stats()
    _check(load().mgmc_qoi_stats(ctypes.c_void_p(qoi_ptr), int(n), int(burn_in), float(S), ctypes.byref(out),
                                 _stream_handle(stream)))
    return out.as_dict()


def mgmc_qoi_stats_noalloc(qoi_ptr, n, burn_in=0, S=1.5, stream=None):
    """mgmc_qoi_stats without any device allocation (fixed library scratch)."""
    out = mgmc_stats()
    _check(load().mgmc_qoi_stats_noalloc(ctypes.c_void_p(qoi_ptr), int(n), int(burn_in), float(S),
                                         ctypes.byref(out), _stream_handle(stream)))
    return out.as_dict()


def mgmc_launches_per_cycle(h):
    v = ctypes.c_int()
    _check(load().mgmc_launches_per_cycle(h, ctypes.byref(v)))
    return v.value


def mgmc_set_profiling(h, enable):
    _check(load().mgmc_set_profiling(h, 1 if enable else 0))


def mgmc_set_band_min_n(h, band_min_n):
    _check(load().mgmc_set_band_min_n(h, int(band_min_n)))


def mgmc_set_coarse_threads(h, threads):
    _check(load().mgmc_set_coarse_threads(h, int(threads)))


def mgmc_profile_times(h, stream=None):
    ms = (ctypes.c_float * 2)()
    _check(load().mgmc_profile_times(h, ms, 2, _stream_handle(stream)))
    return float(ms[0]), float(ms[1])


def mgmc_destroy(h):
    if h:
        _check(load().mgmc_destroy(h))


# --------------------------------------------------------------------------
# convenience object over one problem
# --------------------------------------------------------------------------

class Sampler:
    """MGMC sampler of one posterior problem (paper_2407_12149_gb300.inputs.Problem);
    gibbs=True gives the plain Gibbs sampler of the same posterior (finest-grid sweeps only).
    gamma: cycle index (1 V-cycle, 2 W-cycle; 0 = 2 for the squared shifted Laplacian, else 1)."""

    def __init__(self, problem, precision: str = "fp64", nu1: int = 1, nu2: int = 1, coarse_max_n: int = 0,
                 device: int = 0, use_torch_allocator: bool = True, gibbs: bool = False, band_min_n: int = 0,
                 gamma: int = 0):
        torch = _torch()
        if not torch.cuda.is_available():
            raise MGMCError(2, "no CUDA device available (the sampler has no CPU fallback)")
        self.problem = problem
        self.device = device
        self.precision = MGMC_FP32 if precision == "fp32" else MGMC_FP64
        self.dtype = torch.float32 if self.precision == MGMC_FP32 else torch.float64
        self._alloc = TorchAllocator(device) if use_torch_allocator else None
        p = problem
        self.h = mgmc_create(p.dim, p.n, n_levels=p.n_levels, nu1=nu1, nu2=nu2, precision=self.precision,
                             scale_hd=p.scale_hd, coarse_max_n=coarse_max_n, kappa2=p.kappa2,
                             kappa2_const=p.kappa2_const, obs_site=p.obs_site, obs_w=p.obs_w, Gamma=p.Gamma,
                             y=p.y, qoi_site=p.qoi_site, qoi_w=p.qoi_w, allocator=self._alloc,
                             gibbs=1 if gibbs else 0, disc=getattr(p, "disc", MGMC_FD), band_min_n=band_min_n,
                             gamma=gamma)

    def zeros(self):
        torch = _torch()
        return torch.zeros(self.problem.N, dtype=self.dtype, device=f"cuda:{self.device}")

    def sample(self, x, n_steps: int, seed: int, step_offset: int = 0, chain: int = 0, qoi=None, stream=None):
        """Advance x (torch CUDA tensor or pinned/host tensor, modified in place);
        x = None continues from the state the handle holds (see get_state)."""
        if x is not None and (x.dtype != self.dtype or not x.is_contiguous() or x.numel() != self.problem.N):
            raise ValueError("x must be a contiguous tensor of N entries in the sampler's precision")
        if qoi is not None and (qoi.dtype != _torch().float64 or qoi.numel() < n_steps):
            raise ValueError("qoi must be a float64 tensor with at least n_steps entries")
        mgmc_sample(self.h, n_steps, seed, step_offset, chain, x.data_ptr() if x is not None else None,
                    qoi.data_ptr() if qoi is not None else None, stream)
        return x

    def get_state(self, x, stream=None):
        """Copy the state the handle holds into x (device or host tensor)."""
        if x.dtype != self.dtype or not x.is_contiguous() or x.numel() != self.problem.N:
            raise ValueError("x must be a contiguous tensor of N entries in the sampler's precision")
        mgmc_get_state(self.h, 0, x.data_ptr(), stream)
        return x

    def mean_solve(self, x, rtol=1e-10, max_cycles=200, stream=None):
        return mgmc_mean_solve(self.h, rtol, max_cycles, x.data_ptr(), stream)

    def check_status(self, stream=None):
        """Raise MGMCError if a kernel flagged the chain (wait gave up, non-finite QoI)."""
        mgmc_check_status(self.h, stream)

    def set_wait_limit(self, limit_ns: int):
        """Bound of the kernels' staging waits (0 default, < 0 give up at once: tests)."""
        mgmc_set_wait_limit(self.h, limit_ns)

    def set_band_min_n(self, band_min_n: int):
        """Grids from which the 9-point depths run in the band kernels (mgmc_set_band_min_n)."""
        mgmc_set_band_min_n(self.h, band_min_n)

    def set_coarse_threads(self, threads: int):
        """Threads per CTA of the coarse-grid kernel (mgmc_set_coarse_threads; 0 = automatic)."""
        mgmc_set_coarse_threads(self.h, threads)

    def launches_per_cycle(self):
        return mgmc_launches_per_cycle(self.h)

    def close(self):
        if getattr(self, "h", None):
            mgmc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchSampler:
    """Many independent chains (inputs.Problem list, 2D) advanced by batched launches.

    Chain c uses the Philox chain id c: it reproduces Sampler(problems[c],
    coarse_max_n=coarse_max_n).sample(..., chain=c)."""

    def __init__(self, problems, precision: str = "fp32", coarse_max_n: Optional[int] = None, device: int = 0,
                 use_torch_allocator: bool = True, band_min_n: Optional[int] = None, tune_cache=None,
                 coarse_threads: Optional[int] = None):
        """coarse_max_n / band_min_n / coarse_threads: explicit values win; else, with
        tune_cache (an autotune.TuneCache or a path to its JSON file), the cached choice for
        this batch; else the defaults (31, 0, 0)."""
        torch = _torch()
        if not torch.cuda.is_available():
            raise MGMCError(2, "no CUDA device available (the sampler has no CPU fallback)")
        self.problems = list(problems)
        self.device = device
        self.precision = MGMC_FP32 if precision == "fp32" else MGMC_FP64
        self.dtype = torch.float32 if self.precision == MGMC_FP32 else torch.float64
        self._alloc = TorchAllocator(device) if use_torch_allocator else None
        from . import autotune
        if tune_cache is not None and not isinstance(tune_cache, autotune.TuneCache):
            tune_cache = autotune.TuneCache(str(tune_cache))
        self.settings = autotune.resolve_settings(self.problems, precision, coarse_max_n, band_min_n, tune_cache,
                                                  coarse_threads=coarse_threads)
        coarse_max_n, band_min_n = self.settings["coarse_max_n"], self.settings["band_min_n"]
        n = len(self.problems)
        cfgs = (mgmc_config * n)()
        probs = (mgmc_problem * n)()
        self._keep = []
        for c, p in enumerate(self.problems):
            cfgs[c] = mgmc_config(p.dim, p.n, p.n_levels, 1, 1, self.precision, p.scale_hd, coarse_max_n, 0,
                                  p.disc, band_min_n)
            arrs = {}
            arrs["k2"] = None if p.kappa2 is None else np.ascontiguousarray(p.kappa2, dtype=np.float64)
            if p.obs_site is not None:
                arrs["os"] = np.ascontiguousarray(p.obs_site, dtype=np.int32)
                arrs["ow"] = np.ascontiguousarray(p.obs_w, dtype=np.float64)
                arrs["G"] = np.ascontiguousarray(p.Gamma, dtype=np.float64)
                arrs["y"] = np.ascontiguousarray(p.y, dtype=np.float64)
            if p.qoi_site is not None:
                arrs["qs"] = np.ascontiguousarray(p.qoi_site, dtype=np.int32)
                arrs["qw"] = np.ascontiguousarray(p.qoi_w, dtype=np.float64)
            self._keep.append(arrs)
            probs[c] = mgmc_problem(
                _ptr(arrs["k2"], ctypes.c_double), float(p.kappa2_const), p.m,
                _ptr(arrs.get("os"), ctypes.c_int32), _ptr(arrs.get("ow"), ctypes.c_double),
                int(arrs["os"].shape[1]) if "os" in arrs else 1,
                _ptr(arrs.get("G"), ctypes.c_double), _ptr(arrs.get("y"), ctypes.c_double),
                int(arrs["qs"].size) if "qs" in arrs else 0,
                _ptr(arrs.get("qs"), ctypes.c_int32), _ptr(arrs.get("qw"), ctypes.c_double))
        h = ctypes.c_void_p()
        _check(load().mgmc_create_batch(n, cfgs, probs, ctypes.byref(self._alloc.struct) if self._alloc else None,
                                        _stream_handle(None), ctypes.byref(h)))
        self.h = h
        if self.settings.get("coarse_threads"):
            mgmc_set_coarse_threads(self.h, self.settings["coarse_threads"])

    def zeros(self):
        torch = _torch()
        return [torch.zeros(p.N, dtype=self.dtype, device=f"cuda:{self.device}") for p in self.problems]

    def sample(self, xs, n_steps, seed, step_offset=0, qoi=None, stream=None):
        """xs: one tensor per chain (modified in place), all on the device or all in
        host memory (the library copies them in and out and synchronises), or None
        to continue from the states the handle holds (see get_state)."""
        n = len(self.problems)
        if xs is not None:
            for x, p in zip(xs, self.problems):
                if x.dtype != self.dtype or not x.is_contiguous() or x.numel() != p.N:
                    raise ValueError("each state must be a contiguous tensor of N_c entries in the precision")
        ptrs = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs]) if xs is not None else None
        if qoi is not None and (qoi.dtype != _torch().float64 or qoi.numel() < n * n_steps):
            raise ValueError("qoi must be a float64 tensor with n_chains * n_steps entries")
        _check(load().mgmc_sample_batch(self.h, int(n_steps), int(seed) & (2**64 - 1), int(step_offset), ptrs,
                                        ctypes.c_void_p(qoi.data_ptr()) if qoi is not None else None,
                                        _stream_handle(stream)))
        return xs

    def check_status(self, stream=None):
        """Raise MGMCError if a kernel flagged a chain (wait gave up, non-finite QoI)."""
        mgmc_check_status(self.h, stream)

    def set_wait_limit(self, limit_ns: int):
        """Bound of the kernels' staging waits (0 default, < 0 give up at once: tests)."""
        mgmc_set_wait_limit(self.h, limit_ns)

    def set_band_min_n(self, band_min_n: int):
        """Grids from which the 9-point depths run in the band kernels (mgmc_set_band_min_n)."""
        mgmc_set_band_min_n(self.h, band_min_n)

    def set_coarse_threads(self, threads: int):
        """Threads per CTA of the coarse-grid kernel (mgmc_set_coarse_threads; 0 = by chain count)."""
        mgmc_set_coarse_threads(self.h, threads)

    def get_state(self, c, x, stream=None):
        """Copy chain c's state into x (device or host tensor of N_c entries)."""
        if x.dtype != self.dtype or not x.is_contiguous() or x.numel() != self.problems[c].N:
            raise ValueError("x must be a contiguous tensor of N entries in the sampler's precision")
        mgmc_get_state(self.h, c, x.data_ptr(), stream)
        return x

    def launches_per_cycle(self):
        return mgmc_launches_per_cycle(self.h)

    def close(self):
        if getattr(self, "h", None):
            mgmc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def unet_inputs(p):
    """Input channels [n+1][n+1][3] (BF16 bits as uint16, host numpy) of an inputs.Problem."""
    n = p.n
    out = np.zeros((n + 1) * (n + 1) * 3, dtype=np.uint16)
    k2 = None if p.kappa2 is None else np.ascontiguousarray(p.kappa2, dtype=np.float64)
    if p.obs_site is not None:
        os_ = np.ascontiguousarray(p.obs_site, dtype=np.int32)
        ow = np.ascontiguousarray(p.obs_w, dtype=np.float64)
        y = np.ascontiguousarray(p.y, dtype=np.float64)
        nnz = int(os_.shape[1])
    else:
        os_ = ow = y = None
        nnz = 1
    _check(load().mgmc_unet_inputs(n, _ptr(k2, ctypes.c_double), float(p.kappa2_const), p.m,
                                   _ptr(os_, ctypes.c_int32), _ptr(ow, ctypes.c_double), nnz,
                                   _ptr(y, ctypes.c_double), out.ctypes.data_as(ctypes.c_void_p)))
    return out.reshape(n + 1, n + 1, 3)


class Unet:
    """The learned warm start (mgmc_unet_*).  Inputs: CUDA tensors holding BF16 bits
    (int16 or bfloat16) [samples][n+1][n+1][3]; targets: float32 CUDA [samples][n*n]."""

    def __init__(self, n, c0=32, max_batch=8, seed=0, device=0, use_torch_allocator=True):
        torch = _torch()
        if not torch.cuda.is_available():
            raise MGMCError(2, "no CUDA device available (the U-Net has no CPU fallback)")
        self.n, self.c0, self.max_batch, self.device = n, c0, max_batch, device
        self._alloc = TorchAllocator(device) if use_torch_allocator else None
        h = ctypes.c_void_p()
        _check(load().mgmc_unet_create(n, c0, max_batch, int(seed) & (2**64 - 1),
                                       ctypes.byref(self._alloc.struct) if self._alloc else None,
                                       _stream_handle(None), ctypes.byref(h)))
        self.h = h
        cnt = ctypes.c_int64()
        _check(load().mgmc_unet_n_params(self.h, ctypes.byref(cnt)))
        self.n_params = int(cnt.value)

    def get_params(self):
        out = np.zeros(self.n_params, dtype=np.float32)
        _check(load().mgmc_unet_get_params(self.h, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def set_params(self, theta):
        theta = np.ascontiguousarray(theta, dtype=np.float32)
        _check(load().mgmc_unet_set_params(self.h, theta.ctypes.data_as(ctypes.c_void_p)))

    def gradient(self, inputs, targets, batch):
        loss = ctypes.c_float()
        g = np.zeros(self.n_params, dtype=np.float32)
        _check(load().mgmc_unet_gradient(self.h, batch, ctypes.c_void_p(inputs.data_ptr()),
                                         ctypes.c_void_p(targets.data_ptr()), ctypes.byref(loss),
                                         g.ctypes.data_as(ctypes.c_void_p)))
        return float(loss.value), g

    def train(self, inputs, targets, epochs, batch, lr, shuffle_seed=0):
        losses = np.zeros(max(epochs, 1), dtype=np.float32)
        _check(load().mgmc_unet_train(self.h, targets.shape[0], ctypes.c_void_p(inputs.data_ptr()),
                                      ctypes.c_void_p(targets.data_ptr()), epochs, batch, float(lr),
                                      int(shuffle_seed) & (2**64 - 1), losses.ctypes.data_as(ctypes.c_void_p)))
        return losses[:epochs]

    def predict(self, inputs, precision="fp32"):
        torch = _torch()
        ns = inputs.shape[0]
        dt = torch.float32 if precision == "fp32" else torch.float64
        out = torch.empty(ns, self.n * self.n, dtype=dt, device=inputs.device)
        _check(load().mgmc_unet_predict(self.h, ns, ctypes.c_void_p(inputs.data_ptr()),
                                        ctypes.c_void_p(out.data_ptr()),
                                        MGMC_FP32 if precision == "fp32" else MGMC_FP64))
        return out

    def close(self):
        if getattr(self, "h", None):
            load().mgmc_unet_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
