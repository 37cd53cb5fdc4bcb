"""ctypes wrapper of the plain FP64 CPU oracle (``mgmc_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference arm of ``bench.py`` may import this module.  The
product library (``paper_2407_12149_gb300``) never imports it, and the oracle
shares no code with the CUDA path.

The oracle follows the paper step by step (Alg. 1 V-cycle, Alg. 3 low-rank
Gibbs smoother, Eq. galerkin_triple_product, exact coarsest Cholesky sampler);
see the header of ``mgmc_oracle.c`` for the list of equations it implements
and the readings taken where the paper is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mgmc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

_c_int_p = ctypes.POINTER(ctypes.c_int32)
_c_dbl_p = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to the source (gcc, -ffp-contract=off)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.oracle_create.restype = ctypes.c_int
        L.oracle_create.argtypes = [
            ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
            _c_dbl_p, ctypes.c_double,
            ctypes.c_int, _c_int_p, _c_dbl_p, ctypes.c_int,
            _c_dbl_p, _c_dbl_p,
            ctypes.c_int, _c_int_p, _c_dbl_p,
            ctypes.POINTER(ctypes.c_void_p)]
        L.oracle_destroy.argtypes = [ctypes.c_void_p]
        L.oracle_destroy.restype = None
        L.oracle_level_n.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.oracle_set_gamma.argtypes = [ctypes.c_void_p, ctypes.c_int]
        for name in ("oracle_level_stencil", "oracle_level_B_dense"):
            getattr(L, name).argtypes = [ctypes.c_void_p, ctypes.c_int, _c_dbl_p]
        L.oracle_level_G_dense.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _c_dbl_p]
        L.oracle_level_G_support.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
        L.oracle_coarsest_dense.argtypes = [ctypes.c_void_p, _c_dbl_p]
        L.oracle_smoother_step_given.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                                 _c_dbl_p, _c_dbl_p, _c_dbl_p, _c_dbl_p, _c_dbl_p]
        L.oracle_sample.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint64,
                                    ctypes.c_uint32, ctypes.c_int, _c_dbl_p, _c_dbl_p]
        L.oracle_sample_gibbs.argtypes = L.oracle_sample.argtypes
        L.oracle_mean_solve.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_int, _c_dbl_p,
                                        ctypes.POINTER(ctypes.c_int), _c_dbl_p]
        L.oracle_fine_rhs.argtypes = [ctypes.c_void_p, _c_dbl_p]
        L.oracle_rel_residual.argtypes = [ctypes.c_void_p, _c_dbl_p]
        L.oracle_rel_residual.restype = ctypes.c_double
        L.oracle_philox4x32_10.argtypes = [ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32),
                                           ctypes.POINTER(ctypes.c_uint32)]
        L.oracle_philox4x32_10.restype = None
        L.oracle_normal_pair.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                         ctypes.c_uint32, _c_dbl_p, _c_dbl_p]
        L.oracle_normal_pair.restype = None
        L.oracle_normal_quad.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                         ctypes.c_uint32, _c_dbl_p]
        L.oracle_normal_quad.restype = None
        L.oracle_chain_stats.argtypes = [_c_dbl_p, ctypes.c_int64, ctypes.c_double, _c_dbl_p, _c_dbl_p,
                                         _c_dbl_p, _c_dbl_p, ctypes.POINTER(ctypes.c_int64)]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(_c_dbl_p) if a is not None else None


def _ip(a):
    return a.ctypes.data_as(_c_int_p) if a is not None else None


class OracleError(RuntimeError):
    pass


class Oracle:
    """One posterior problem held by the CPU oracle (FP64)."""

    def __init__(self, dim, n, n_levels, *, kappa2=None, kappa2_const=10.0, scale_hd=1,
                 nu1=1, nu2=1, obs_site=None, obs_w=None, Gamma=None, y=None,
                 qoi_site=None, qoi_w=None, disc=0, gamma=1):
        """disc: 0 finite-difference fine operator, 1 Q1 finite elements (constant kappa^2),
        2 the 13-point finite-difference squared shifted Laplacian (2D, constant kappa^2).
        gamma: cycle index of Alg. 1 (1 V-cycle, 2 W-cycle)."""
        L = lib()
        self.dim, self.n, self.n_levels = dim, n, n_levels
        self.W = 5 if disc == 2 else 3
        self.N = n ** dim
        k2 = None if kappa2 is None else np.ascontiguousarray(kappa2, dtype=np.float64).ravel()
        if obs_site is None:
            m, nnz = 0, 1
            os_ = ow_ = G_ = y_ = None
        else:
            os_ = np.ascontiguousarray(obs_site, dtype=np.int32)
            ow_ = np.ascontiguousarray(obs_w, dtype=np.float64)
            m, nnz = os_.shape
            G_ = np.ascontiguousarray(Gamma, dtype=np.float64)
            y_ = np.ascontiguousarray(y, dtype=np.float64)
        self.m = m
        if qoi_site is None:
            nq, qs, qw = 0, None, None
        else:
            qs = np.ascontiguousarray(qoi_site, dtype=np.int32)
            qw = np.ascontiguousarray(qoi_w, dtype=np.float64)
            nq = qs.size
        h = ctypes.c_void_p()
        rc = L.oracle_create(dim, n, n_levels, scale_hd, int(disc), nu1, nu2, _dp(k2), float(kappa2_const),
                             m, _ip(os_), _dp(ow_), nnz, _dp(G_), _dp(y_),
                             nq, _ip(qs), _dp(qw), ctypes.byref(h))
        if rc != 0:
            raise OracleError(f"oracle_create failed with code {rc}")
        self._h = h
        if gamma != 1 and L.oracle_set_gamma(h, int(gamma)) != 0:
            self.close()
            raise OracleError(f"oracle_set_gamma({gamma}) failed")

    def close(self):
        if getattr(self, "_h", None):
            lib().oracle_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- level queries -------------------------------------------------
    def level_n(self, l):
        return lib().oracle_level_n(self._h, l)

    def level_N(self, l):
        return self.level_n(l) ** self.dim

    def stencil(self, l):
        NS = self.W ** self.dim
        out = np.zeros((self.level_N(l), NS))
        lib().oracle_level_stencil(self._h, l, _dp(out))
        return out

    def B_dense(self, l):
        out = np.zeros((self.level_N(l), max(self.m, 1)))
        lib().oracle_level_B_dense(self._h, l, _dp(out))
        return out[:, : self.m]

    def G_dense(self, l, direction):
        out = np.zeros((self.level_N(l), max(self.m, 1)))
        rc = lib().oracle_level_G_dense(self._h, l, direction, _dp(out))
        if rc:
            raise OracleError(rc)
        return out[:, : self.m]

    def G_support(self, l, direction):
        return lib().oracle_level_G_support(self._h, l, direction)

    def coarsest_dense(self):
        n0 = self.level_N(0)
        out = np.zeros((n0, n0))
        lib().oracle_coarsest_dense(self._h, _dp(out))
        return out

    def fine_rhs(self):
        out = np.zeros(self.N)
        lib().oracle_fine_rhs(self._h, _dp(out))
        return out

    def rel_residual(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        return lib().oracle_rel_residual(self._h, _dp(x))

    # -- method --------------------------------------------------------
    def smoother_step_given(self, l, direction, x, fd, zdiag, zlr, d=None):
        """Alg. 3 on level l for the right-hand side fd + B_l Gamma^-1 d."""
        x = np.array(x, dtype=np.float64, copy=True)
        fd = np.ascontiguousarray(fd, dtype=np.float64)
        zd = np.ascontiguousarray(zdiag, dtype=np.float64)
        zl = np.ascontiguousarray(zlr if zlr is not None else np.zeros(max(self.m, 1)), dtype=np.float64)
        dv = np.ascontiguousarray(d if d is not None else np.zeros(max(self.m, 1)), dtype=np.float64)
        rc = lib().oracle_smoother_step_given(self._h, l, direction, _dp(x), _dp(fd), _dp(dv), _dp(zd), _dp(zl))
        if rc:
            raise OracleError(rc)
        return x

    def sample(self, n_steps, seed, x=None, step_offset=0, chain=0, noise=True, qoi=True, gibbs=False):
        """n_steps MGMC V-cycles, or with gibbs=True steps of the plain Gibbs sampler (Sec. 5.1.3)."""
        x = np.zeros(self.N) if x is None else np.array(x, dtype=np.float64, copy=True).ravel()
        q = np.zeros(max(n_steps, 1)) if qoi else None
        fn = lib().oracle_sample_gibbs if gibbs else lib().oracle_sample
        rc = fn(self._h, int(n_steps), int(seed) & (2**64 - 1), int(step_offset),
                int(chain), 1 if noise else 0, _dp(x), _dp(q))
        if rc:
            raise OracleError(rc)
        return (x, q[:n_steps]) if qoi else x

    def mean_solve(self, rtol=1e-10, max_cycles=200, x=None):
        x = np.zeros(self.N) if x is None else np.array(x, dtype=np.float64, copy=True).ravel()
        cyc = ctypes.c_int()
        rr = ctypes.c_double()
        rc = lib().oracle_mean_solve(self._h, float(rtol), int(max_cycles), _dp(x), ctypes.byref(cyc),
                                     ctypes.byref(rr))
        if rc:
            raise OracleError(rc)
        return x, cyc.value, rr.value


def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().oracle_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def normal_pair(seed, c0, c1, c2, c3):
    z0 = ctypes.c_double()
    z1 = ctypes.c_double()
    lib().oracle_normal_pair(int(seed) & (2**64 - 1), c0, c1, c2, c3, ctypes.byref(z0), ctypes.byref(z1))
    return z0.value, z1.value


def normal_quad(seed, c0, c1, c2, c3):
    """The four normals of one site-noise block (kind 0)."""
    z = np.zeros(4)
    lib().oracle_normal_quad(int(seed) & (2**64 - 1), c0, c1, c2, c3, z.ctypes.data_as(_c_dbl_p))
    return tuple(float(v) for v in z)


def chain_stats(series, S=1.5):
    a = np.ascontiguousarray(series, dtype=np.float64)
    mean, var, tau, err = (ctypes.c_double() for _ in range(4))
    W = ctypes.c_int64()
    rc = lib().oracle_chain_stats(_dp(a), a.size, float(S), ctypes.byref(mean), ctypes.byref(var),
                                  ctypes.byref(tau), ctypes.byref(err), ctypes.byref(W))
    if rc:
        raise OracleError(rc)
    return dict(mean=mean.value, var=var.value, tau=tau.value, tau_err=err.value, window=W.value,
                ess=a.size / tau.value)
