"""ctypes front end of the dense FP64 S_N stepper in dense_sn.c (test infrastructure).

``build()`` compiles dense_sn.c with gcc (OpenMP) into oracle/_build/; ``DenseSolver``
runs steps on a full-grid array I[k, q] (merged row k, angle q = l*N_phi + p).
"""
import ctypes
import os
import subprocess

import numpy as np

from . import problem as _problem

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libdense_sn.so")
_lib = None


def build(force=False):
    src = os.path.join(_HERE, "dense_sn.c")
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=gnu99",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.dense_step.restype = ctypes.c_int
        _lib.dense_step.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        _lib.dense_num_threads.restype = ctypes.c_int
    return _lib


class _Params(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("G", ctypes.c_int), ("nang", ctypes.c_int),
                ("dir", ctypes.c_void_p * 3), ("domega", ctypes.c_void_p),
                ("lam", ctypes.c_double * 3), ("acoef", ctypes.c_void_p),
                ("scoef", ctypes.c_void_p), ("eps", ctypes.c_void_p),
                ("inflow", ctypes.c_void_p * 6), ("flux", ctypes.c_int), ("alpha_local", ctypes.c_int)]


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


class DenseSolver:
    """Full-grid FP64 solver: state I of shape (N_Z, N_theta*N_phi)."""

    def __init__(self, wl, coef=None):
        self.wl = wl
        self.coef = coef if coef is not None else _problem.build(wl)
        c = self.coef
        d = c.dirs
        self._keep = [np.ascontiguousarray(d["nx"], dtype=float), np.ascontiguousarray(d["ny"], dtype=float),
                      np.ascontiguousarray(d["nz"], dtype=float), np.ascontiguousarray(d["domega"], dtype=float),
                      np.ascontiguousarray(c.acoef), np.ascontiguousarray(c.scoef), np.ascontiguousarray(c.eps)]
        self._inflow = [None if x is None else np.ascontiguousarray(x, dtype=float) for x in c.inflow]
        p = _Params()
        p.ndim, p.nx, p.ny, p.nz, p.G = c.ndim, c.nx, c.ny, c.nz, c.G
        p.nang = c.nang
        for a in range(3):
            p.dir[a] = _ptr(self._keep[a])
            p.lam[a] = float(c.lam[a])
        p.domega = _ptr(self._keep[3])
        p.acoef, p.scoef, p.eps = _ptr(self._keep[4]), _ptr(self._keep[5]), _ptr(self._keep[6])
        for f in range(6):
            p.inflow[f] = _ptr(self._inflow[f])
        p.flux = {"upwind": 0, "rusanov": 1, "central": 2}[c.flux]
        p.alpha_local = 1 if c.alpha_local else 0
        self._p = p
        self._lib = _load()

    def initial(self):
        rows = _problem.initial_rows(self.wl, self.coef)
        return np.repeat(rows[:, None], self.coef.nang, axis=1).copy()

    def step(self, I, return_star=False):
        I = np.ascontiguousarray(I, dtype=float)
        out = np.empty_like(I)
        star = np.empty_like(I) if return_star else None
        err = self._lib.dense_step(ctypes.byref(self._p), _ptr(I), _ptr(out), _ptr(star))
        if err:
            raise MemoryError("dense_step: allocation failed")
        return (out, star) if return_star else out

    @staticmethod
    def threads():
        return _load().dense_num_threads()

    # diagnostics -------------------------------------------------------------
    def J(self, I):
        """Group mean intensity per merged row, J = (1/4pi) sum dOmega I (Sec. 2)."""
        return I @ self.coef.dirs["domega"] / (4.0 * np.pi)

    def energy_density(self, I):
        """E_f = (4 pi / c) J_f per merged row (Sec. 2)."""
        return 4.0 * np.pi / self.coef.c * self.J(I)

    def total_energy(self, I):
        return self.coef.dV * float(np.sum(self.energy_density(I)))
