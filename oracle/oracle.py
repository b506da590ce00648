"""ctypes wrapper of the FP64 CPU oracle (test infrastructure only)."""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pflbm_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")

COLL_MRT, COLL_BGK, COLL_MRT_ALL_EQUAL = 0, 1, 2
# order of the two collisions in a step: both at phi^t (the reading used
# everywhere), or the phase field first and the hydrodynamics at phi^{t+1}
SCHED_CONCURRENT, SCHED_SEQUENTIAL = 0, 1

_lib = None


def build_oracle(force=False):
    """Compile the oracle with plain IEEE FP64 flags (no FMA contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp.%d" % os.getpid()
    cmd = ["g++", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           "-std=c++17", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build_oracle()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        lib.ora_new.restype = P
        lib.ora_new.argtypes = [P, P, P, P, P]
        lib.ora_free.argtypes = [P]
        lib.ora_step.argtypes = [P, ctypes.c_int, ctypes.c_int]
        lib.ora_time.restype = ctypes.c_long
        lib.ora_time.argtypes = [P]
        lib.ora_get_pops.argtypes = [P, P, P]
        lib.ora_set_pops.argtypes = [P, P, P]
        lib.ora_fields.argtypes = [P, P, P, P, P]
        lib.ora_tables.restype = ctypes.c_int
        lib.ora_tables.argtypes = [ctypes.c_int, P, P, P, P, P, P]
        lib.ora_mrt_collide.argtypes = [ctypes.c_int, P, P, P, P, P]
        lib.ora_set_solid.argtypes = [P, P]
        lib.ora_tangent.argtypes = [P, P, P, P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int,
                                    P, P]
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a, n=None):
    if a is None:
        return None
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64)).reshape(-1)
    if n is not None and a.size != n:
        raise ValueError("expected %d values, got %d" % (n, a.size))
    return a


class Oracle:
    """One PFLBM domain on the CPU in FP64.

    Arrays are x-fastest: a field of shape (nz, ny, nx) flattened; vector
    fields are SoA (3, nz, ny, nx); populations are (q, nz, ny, nx) in the
    canonical velocity order (cz, cy, cx each looping -1, 0, 1, cx fastest).
    """

    def __init__(self, nx, ny, nz, bc, rho_h, rho_l, nu_h, nu_l, sigma, mobility, xi,
                 gravity=(0.0, 0.0, 0.0), phi0=None, u0=None, p0=None, collision=COLL_MRT, h_lattice=15,
                 schedule=SCHED_CONCURRENT):
        self.lib = _load()
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        self.qh = {27: 27, 9: 9}.get(h_lattice, 15)
        self.qg = 9 if self.qh == 9 else 27
        if schedule not in (SCHED_CONCURRENT, SCHED_SEQUENTIAL):
            raise ValueError("unknown schedule %r" % (schedule,))
        ip = np.array([nx, ny, nz] + list(bc) + [collision, self.qh, schedule], dtype=np.int32)
        dp = np.array([rho_h, rho_l, nu_h, nu_l, sigma, mobility, xi] + list(gravity), dtype=np.float64)
        self._phi0 = _f64(phi0, self.N)
        self._u0 = _f64(u0, 3 * self.N)
        self._p0 = _f64(p0, self.N)
        self.h = self.lib.ora_new(_ptr(ip), _ptr(dp), _ptr(self._phi0), _ptr(self._u0), _ptr(self._p0))

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.ora_free(h)
            self.h = None

    def set_solid(self, mask):
        """Solid cells (nonzero entries of a (nz, ny, nx) mask)."""
        m = np.ascontiguousarray(np.asarray(mask).reshape(-1) != 0, dtype=np.uint8)
        if m.size != self.N:
            raise ValueError("solid mask must hold one byte per cell")
        self.lib.ora_set_solid(self.h, _ptr(m))

    def step(self, n=1, threads=0):
        self.lib.ora_step(self.h, int(n), int(threads))

    @property
    def time(self):
        return self.lib.ora_time(self.h)

    def populations(self):
        h = np.empty((self.qh,) + self.shape)
        g = np.empty((self.qg,) + self.shape)
        self.lib.ora_get_pops(self.h, _ptr(h), _ptr(g))
        return h, g

    def set_populations(self, h, g):
        h = _f64(h, self.qh * self.N)
        g = _f64(g, self.qg * self.N)
        self.lib.ora_set_pops(self.h, _ptr(h), _ptr(g))

    def fields(self):
        """phi, rho, p (= p* rho c_s^2) and u (3, nz, ny, nx) at the current time."""
        phi = np.empty(self.shape)
        rho = np.empty(self.shape)
        p = np.empty(self.shape)
        u = np.empty((3,) + self.shape)
        self.lib.ora_fields(self.h, _ptr(phi), _ptr(rho), _ptr(p), _ptr(u))
        return phi, rho, p, u


def tables(q):
    """Velocities, weights, opposites, moment degrees, M and M^-1 of D3Q15/D3Q27."""
    lib = _load()
    c = np.empty((q, 3), dtype=np.int32)
    w = np.empty(q)
    opp = np.empty(q, dtype=np.int32)
    deg = np.empty(q, dtype=np.int32)
    M = np.empty((q, q))
    Minv = np.empty((q, q))
    got = lib.ora_tables(q, _ptr(c), _ptr(w), _ptr(opp), _ptr(deg), _ptr(M), _ptr(Minv))
    if got != q:
        raise ValueError("unknown lattice q=%d" % q)
    return dict(c=c, w=w, opp=opp, degree=deg, M=M, Minv=Minv)


def mrt_collide(q, f, feq, src, rates):
    lib = _load()
    f, feq, src, rates = (_f64(a, q) for a in (f, feq, src, rates))
    out = np.empty(q)
    lib.ora_mrt_collide(q, _ptr(f), _ptr(feq), _ptr(src), _ptr(rates), _ptr(out))
    return out


def from_params(p, phi0, u0=None, p0=None, schedule=SCHED_CONCURRENT):
    """Oracle built from a ``workloads.Params``-like object (duck-typed)."""
    o = Oracle(p.nx, p.ny, p.nz, p.bc, p.rho_h, p.rho_l, p.nu_h, p.nu_l, p.sigma, p.mobility, p.xi,
               p.gravity, phi0, u0, p0, collision=p.collision, h_lattice=getattr(p, "h_lattice", 15),
               schedule=schedule)
    if getattr(p, "solid", None) is not None:
        o.set_solid(p.solid)
    return o


PARAM_INDEX = {"mobility": 0, "xi": 1, "sigma": 2}


def tangent(p, phi0, u0, p0, n, obs, param, threads=0):
    """Exact dJ/d(param) by forward-mode (dual-number) differentiation of the
    oracle, J = sum over (step, W) in obs of W . phi(step) after n steps;
    param is "mobility", "xi" or "sigma".  Returns (J, dJ)."""
    lib = _load()
    N = p.nx * p.ny * p.nz
    qh = {27: 27, 9: 9}.get(getattr(p, "h_lattice", 15), 15)
    ip = np.array([p.nx, p.ny, p.nz] + list(p.bc) + [p.collision, qh, SCHED_CONCURRENT], dtype=np.int32)
    dp = np.array([p.rho_h, p.rho_l, p.nu_h, p.nu_l, p.sigma, p.mobility, p.xi] + list(p.gravity),
                  dtype=np.float64)
    steps = np.array([int(t) for t, _ in obs], dtype=np.int32)
    if np.any(steps < 0) or np.any(steps > n):
        raise ValueError("observation step outside [0, n]")
    W = np.ascontiguousarray(np.stack([_f64(w, N) for _, w in obs]))
    phi0, u0, p0 = _f64(phi0, N), _f64(u0, 3 * N), _f64(p0, N)
    J = ctypes.c_double(0.0)
    dJ = ctypes.c_double(0.0)
    lib.ora_tangent(_ptr(ip), _ptr(dp), _ptr(phi0), _ptr(u0), _ptr(p0), PARAM_INDEX[param], int(n), len(obs),
                    _ptr(steps), _ptr(W), int(threads), ctypes.byref(J), ctypes.byref(dJ))
    return J.value, dJ.value
