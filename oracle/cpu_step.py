"""ctypes binding of the plain C/OpenMP CPU step (``oracle/lbcg_cpu.c``).

THIS IS TEST INFRASTRUCTURE (see ``oracle/lbcg_oracle.py``): a second, independent CPU
implementation of the step, checked against the PyTorch oracle by ``tests/`` and timed by
``bench.py``'s CPU-baseline leg.  It shares no code with the CUDA library.  ``build()`` compiles
it with gcc (OpenMP when available).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lbcg_cpu.c")
LIB = os.path.join(HERE, "liblbcg_cpu.so")
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
BCX = {"periodic": 0, "closed": 1, "inout": 2}
BCY = {"periodic": 0, "closed": 1}


class _Params(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("nu_R", "nu_B", "sigma", "beta", "s_e", "s_eps", "s_q", "rho0", "u_in",
                                          "rho_out", "grad_eps")] + [("inlet_profile", C.c_int), ("wetting", C.c_int)]


def build(force: bool = False) -> str:
    """Compile liblbcg_cpu.so (portable flags: no -march=native; no FMA contraction)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    base = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off", SRC, "-o", LIB + ".tmp", "-lm"]
    r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
    if r.returncode != 0:
        r = subprocess.run(base, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("gcc failed on lbcg_cpu.c:\n" + r.stderr)
    os.replace(LIB + ".tmp", LIB)
    return LIB


_lib = None


def library():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(LIB)
        lib.lbcg_cpu_create.restype = C.c_void_p
        lib.lbcg_cpu_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.c_double, C.POINTER(_Params)]
        lib.lbcg_cpu_step.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
        lib.lbcg_cpu_open_columns.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        lib.lbcg_cpu_destroy.argtypes = [C.c_void_p]
        lib.lbcg_cpu_max_threads.restype = C.c_int
        lib.lbcg_cpu_has_openmp.restype = C.c_int
        _lib = lib
    return _lib


def max_threads() -> int:
    return int(library().lbcg_cpu_max_threads())


def threads_used(requested: int) -> int:
    """Threads a step run with `requested` threads (0 = all) actually uses."""
    if not library().lbcg_cpu_has_openmp():
        return 1
    return requested if requested > 0 else max_threads()


class CpuLattice:
    """One lattice of the C step; states are float64 arrays [9, ny, nx] per colour."""

    def __init__(self, geom, prm):
        lib = library()
        self.g, self.p = geom, prm
        self._keep = [np.ascontiguousarray(geom.solid, np.uint8)]
        nrm = None if geom.normal is None else np.ascontiguousarray(geom.normal, np.float64)
        th = None if geom.theta_node is None else np.ascontiguousarray(geom.theta_node, np.float64)
        self._keep += [nrm, th]
        P = _Params(prm.nu_R, prm.nu_B, prm.sigma, prm.beta, prm.s_e, prm.s_eps, prm.s_q, prm.rho0, prm.u_in,
                    prm.rho_out, prm.grad_eps, int(prm.inlet_profile), int(prm.wetting))
        self.h = lib.lbcg_cpu_create(geom.nx, geom.ny, BCX[geom.bc_x], BCY[geom.bc_y], self._keep[0].ctypes.data,
                                     None if nrm is None else nrm.ctypes.data, None if th is None else th.ctypes.data,
                                     float(prm.theta), C.byref(P))
        if not self.h:
            raise MemoryError("lbcg_cpu_create")

    def init_state(self):
        """Rest populations of the initial colour field, open columns applied."""
        r = np.asarray(self.g.rhoN0, np.float64)
        fl = (np.asarray(self.g.solid) == 0).astype(np.float64)
        fR = np.ascontiguousarray(W[:, None, None] * self.p.rho0 * (1 + r) / 2 * fl)
        fB = np.ascontiguousarray(W[:, None, None] * self.p.rho0 * (1 - r) / 2 * fl)
        library().lbcg_cpu_open_columns(self.h, fR.ctypes.data, fB.ctypes.data)
        return fR, fB

    def run(self, fR, fB, n: int, threads: int = 0):
        a = (np.ascontiguousarray(fR, np.float64).copy(), np.ascontiguousarray(fB, np.float64).copy())
        b = (np.empty_like(a[0]), np.empty_like(a[1]))
        for _ in range(n):
            library().lbcg_cpu_step(self.h, a[0].ctypes.data, a[1].ctypes.data, b[0].ctypes.data, b[1].ctypes.data,
                                    int(threads))
            a, b = b, a
        return a

    def close(self):
        if self.h:
            library().lbcg_cpu_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
