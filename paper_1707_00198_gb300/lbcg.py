"""ctypes binding of liblbcg.so (the C ABI declared in include/lbcg.h).

Module-level functions carry the names of the C entry points and only marshal arguments;
every step of the method runs in the library's CUDA kernels.  ``Lattice`` is a small
convenience wrapper around one handle.  There is no fallback: if the library is missing or
a call fails, an exception is raised.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

from .inputs import Geometry, Params

_HERE = os.path.dirname(os.path.abspath(__file__))
# the library this binding loads; LBCG_LIBRARY selects another build of it (e.g. the checked
# build, liblbcg_checked.so)
LIB_PATH = os.environ.get("LBCG_LIBRARY") or os.path.join(_HERE, "liblbcg.so")

LBCG_FP64, LBCG_FP32, LBCG_FP16_STORE, LBCG_BF16_STORE = 0, 1, 2, 3
PRECISIONS = {"fp64": LBCG_FP64, "fp32": LBCG_FP32, "fp16": LBCG_FP16_STORE, "bf16": LBCG_BF16_STORE}
STORE_BYTES = {LBCG_FP64: 8, LBCG_FP32: 4, LBCG_FP16_STORE: 2, LBCG_BF16_STORE: 2}
_BCX = {"periodic": 0, "closed": 1, "inout": 2}
_BCY = {"periodic": 0, "closed": 1}
STATUS = {0: "LBCG_OK", 1: "LBCG_E_ARG", 2: "LBCG_E_GEOMETRY", 3: "LBCG_E_UNSTABLE_PARAM", 4: "LBCG_E_CUDA",
          5: "LBCG_E_DIVERGED", 6: "LBCG_E_TIMEOUT", 7: "LBCG_E_UNSUPPORTED", 8: "LBCG_E_NOMEM", 9: "LBCG_E_BOUNDS"}


class lbcg_geometry(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("bc_x", C.c_int32), ("bc_y", C.c_int32),
                ("solid", C.POINTER(C.c_uint8)), ("rhoN0", C.POINTER(C.c_double)),
                ("normal", C.POINTER(C.c_double)), ("theta_node", C.POINTER(C.c_double))]


class lbcg_params(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("nu_R", "nu_B", "sigma", "theta", "beta", "s_e", "s_eps", "s_q",
                                          "rho0", "u_in", "rho_out", "grad_eps")] + [("inlet_profile", C.c_int32), ("wetting", C.c_int32)]


class lbcg_obs_spec(C.Structure):
    _fields_ = [("wall_y", C.c_double), ("cyl_x", C.c_double), ("cyl_y", C.c_double), ("cyl_r", C.c_double),
                ("tip_row0", C.c_int32), ("tip_row1", C.c_int32), ("cl_row0", C.c_int32), ("cl_row1", C.c_int32)]


class lbcg_obs(C.Structure):
    _fields_ = [("step", C.c_int64), ("mass_R", C.c_double), ("mass_B", C.c_double), ("umax", C.c_double),
                ("n_pts", C.c_double), ("xc", C.c_double), ("yc", C.c_double), ("R", C.c_double),
                ("theta_deg", C.c_double), ("dp_laplace", C.c_double), ("x_tip", C.c_double),
                ("x_cl", C.c_double), ("moments", C.c_double * 9), ("nonfinite", C.c_int32)]


class lbcg_adjoint_spec(C.Structure):
    _fields_ = [("nsteps", C.c_int64), ("checkpoint", C.c_int64), ("objective", C.c_int32),
                ("weight", C.POINTER(C.c_double)), ("tip_row0", C.c_int32), ("tip_row1", C.c_int32),
                ("cl_row0", C.c_int32), ("cl_row1", C.c_int32), ("reverse_fp32", C.c_int32)]


class lbcg_grads(C.Structure):
    _fields_ = [("J", C.c_double), ("dJ_dsigma", C.c_double), ("dJ_dnu_R", C.c_double), ("dJ_dnu_B", C.c_double),
                ("dJ_dtheta", C.c_double), ("dJ_dtheta_node", C.POINTER(C.c_double))]


class lbcg_diag_spec(C.Structure):
    _fields_ = [("cx", C.c_double), ("cy", C.c_double), ("r", C.c_double), ("inside_red", C.c_int32)]


class lbcg_diag(C.Structure):
    _fields_ = [("step", C.c_int64), ("prev_step", C.c_int64)] + [
        (n, C.c_double) for n in ("e1", "e_npmt", "m_R_in", "m_R_out", "m_B_in", "m_B_out")]


LBCG_OBJ_WEIGHTED, LBCG_OBJ_FINGER_LENGTH, LBCG_OBJ_RED_MASS = 0, 1, 2
OBJECTIVES = {"weighted": LBCG_OBJ_WEIGHTED, "finger_length": LBCG_OBJ_FINGER_LENGTH, "red_mass": LBCG_OBJ_RED_MASS}


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
RELEASE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class lbcg_allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("release", RELEASE_FN), ("ctx", C.c_void_p)]


class LBCGError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def library():
    """Load liblbcg.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1707_00198_gb300.build.build() "
                           "(or __graft_entry__.build()); there is no CPU fallback")
    lib = C.CDLL(LIB_PATH)
    H = C.c_void_p
    sigs = {
        "lbcg_create": (C.c_int, [C.POINTER(lbcg_geometry), C.POINTER(lbcg_params), C.c_int32, C.c_void_p,
                                  C.POINTER(H)]),
        "lbcg_create_batch": (C.c_int, [C.c_int32, C.POINTER(lbcg_geometry), C.POINTER(lbcg_params), C.c_int32,
                                        C.c_void_p, C.POINTER(H)]),
        "lbcg_step": (C.c_int, [H, C.c_int64]),
        "lbcg_observables": (C.c_int, [H, C.c_int32, C.POINTER(lbcg_obs_spec), C.POINTER(lbcg_obs)]),
        "lbcg_get_populations": (C.c_int, [H, C.c_int32, C.c_void_p]),
        "lbcg_set_populations": (C.c_int, [H, C.c_int32, C.c_void_p]),
        "lbcg_get_fields": (C.c_int, [H, C.c_int32, C.c_void_p]),
        "lbcg_state_bytes": (C.c_size_t, [H]),
        "lbcg_upload_state": (C.c_int, [H, C.c_void_p, C.c_size_t]),
        "lbcg_download_state": (C.c_int, [H, C.c_void_p, C.c_size_t]),
        "lbcg_set_tile": (C.c_int, [H, C.c_int32]),
        "lbcg_set_sweep": (C.c_int, [H, C.c_int32]),
        "lbcg_set_poll_limit": (C.c_int, [H, C.c_int32]),
        "lbcg_set_allocator": (C.c_int, [C.POINTER(lbcg_allocator)]),
        "lbcg_profile": (C.c_int, [H, C.c_int32]),
        "lbcg_kernel_times": (C.c_int, [H, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
        "lbcg_launches_per_step": (C.c_int32, [H]),
        "lbcg_step_host": (C.c_int, [H, C.c_void_p, C.c_void_p, C.c_size_t, C.c_int64]),
        "lbcg_step_launches": (C.c_int64, [H]),
        "lbcg_total_nodes": (C.c_int64, [H]),
        "lbcg_destroy": (C.c_int, [H]),
        "lbcg_last_error": (C.c_char_p, []),
        "lbcg_field_moments_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p,
                                                 C.c_void_p]),
        "lbcg_adjoint": (C.c_int, [H, C.POINTER(lbcg_adjoint_spec), C.POINTER(lbcg_grads)]),
        "lbcg_autotune": (C.c_int, [H, C.c_int32, C.POINTER(C.c_int32)]),
        "lbcg_diagnostics": (C.c_int, [H, C.c_int32, C.POINTER(lbcg_diag_spec), C.POINTER(lbcg_diag)]),
        "lbcg_schedule": (C.c_int, [H, C.POINTER(C.c_int32)]),
        "lbcg_sweep_rows": (C.c_int32, [H]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols() -> list:
    return ["lbcg_create", "lbcg_create_batch", "lbcg_step", "lbcg_observables", "lbcg_get_populations",
            "lbcg_set_populations", "lbcg_get_fields", "lbcg_state_bytes", "lbcg_upload_state",
            "lbcg_download_state", "lbcg_set_sweep", "lbcg_set_tile", "lbcg_profile", "lbcg_kernel_times", "lbcg_launches_per_step", "lbcg_step_host", "lbcg_step_launches", "lbcg_total_nodes", "lbcg_destroy",
            "lbcg_last_error", "lbcg_field_moments_noalloc", "lbcg_adjoint", "lbcg_autotune", "lbcg_schedule", "lbcg_sweep_rows", "lbcg_diagnostics",
            "lbcg_set_poll_limit", "lbcg_set_allocator"]


def _check(status: int):
    if status != 0:
        raise LBCGError(status, library().lbcg_last_error().decode())


def _dptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


def _marshal(geoms: Sequence[Geometry], prms: Sequence[Params]):
    keep = []
    G = (lbcg_geometry * len(geoms))()
    P = (lbcg_params * len(prms))()
    for i, (g, p) in enumerate(zip(geoms, prms)):
        solid = np.ascontiguousarray(g.solid, np.uint8)
        rn = np.ascontiguousarray(g.rhoN0, np.float64)
        nrm = None if g.normal is None else np.ascontiguousarray(g.normal, np.float64)
        th = None if g.theta_node is None else np.ascontiguousarray(g.theta_node, np.float64)
        keep += [solid, rn, nrm, th]
        G[i] = lbcg_geometry(g.nx, g.ny, _BCX[g.bc_x], _BCY[g.bc_y], solid.ctypes.data_as(C.POINTER(C.c_uint8)),
                             _dptr(rn), _dptr(nrm), _dptr(th))
        P[i] = lbcg_params(p.nu_R, p.nu_B, p.sigma, p.theta, p.beta, p.s_e, p.s_eps, p.s_q, p.rho0, p.u_in,
                           p.rho_out, p.grad_eps, int(p.inlet_profile), int(p.wetting))
    return G, P, keep


# ---------------------------------------------------------------- functions with the C names
def lbcg_create_batch(geoms: Sequence[Geometry], prms: Sequence[Params], precision: int = LBCG_FP32,
                      stream: int = 0) -> int:
    G, P, keep = _marshal(geoms, prms)
    h = C.c_void_p()
    _check(library().lbcg_create_batch(len(geoms), G, P, precision, C.c_void_p(stream or None), C.byref(h)))
    return h.value


def lbcg_create(geom: Geometry, prm: Params, precision: int = LBCG_FP32, stream: int = 0) -> int:
    return lbcg_create_batch([geom], [prm], precision, stream)


def lbcg_step(h: int, nsteps: int):
    _check(library().lbcg_step(h, nsteps))


def lbcg_observables(h: int, lattice: int = 0, spec: Optional[lbcg_obs_spec] = None, raise_on_diverged=True) -> dict:
    spec = spec or obs_spec()
    o = lbcg_obs()
    st = library().lbcg_observables(h, lattice, C.byref(spec), C.byref(o))
    if st != 0 and not (st == 5 and not raise_on_diverged):
        _check(st)
    d = {k: getattr(o, k) for k, _ in lbcg_obs._fields_ if k != "moments"}
    d["moments"] = list(o.moments)
    return d


def lbcg_get_populations(h: int, lattice: int, nx: int, ny: int) -> np.ndarray:
    out = np.empty((2, 9, ny, nx), np.float64)
    _check(library().lbcg_get_populations(h, lattice, out.ctypes.data))
    return out


def lbcg_set_populations(h: int, lattice: int, f: np.ndarray):
    f = np.ascontiguousarray(f, np.float64)
    _check(library().lbcg_set_populations(h, lattice, f.ctypes.data))


def lbcg_get_fields(h: int, lattice: int, nx: int, ny: int) -> np.ndarray:
    out = np.empty((4, ny, nx), np.float64)
    _check(library().lbcg_get_fields(h, lattice, out.ctypes.data))
    return out


def lbcg_state_bytes(h: int) -> int:
    return int(library().lbcg_state_bytes(h))


def lbcg_upload_state(h: int, ptr: int, nbytes: int):
    _check(library().lbcg_upload_state(h, ptr, nbytes))


def lbcg_download_state(h: int, ptr: int, nbytes: int):
    _check(library().lbcg_download_state(h, ptr, nbytes))


def lbcg_step_host(h: int, ptr_in: int, ptr_out: int, nbytes: int, nsteps: int):
    _check(library().lbcg_step_host(h, ptr_in, ptr_out, nbytes, nsteps))


def lbcg_set_tile(h: int, ty: int):
    _check(library().lbcg_set_tile(h, ty))


def lbcg_set_sweep(h: int, rows: int = 0):
    _check(library().lbcg_set_sweep(h, rows))


def lbcg_set_poll_limit(h: int, polls: int = -1):
    """Polls of the sweep's bounded wait for a staged row (-1: the default, 0: give up at once)."""
    _check(library().lbcg_set_poll_limit(h, polls))


_allocator_keepalive = []   # every installed allocator: handles keep the one they were created with


def lbcg_set_allocator(alloc=None, release=None):
    """Device allocator of handles created afterwards: alloc(nbytes, stream) -> device pointer
    (int, 256-byte aligned; 0 on failure) and release(ptr, stream); no arguments restores
    cudaMalloc / cudaFree."""
    if alloc is None:
        _check(library().lbcg_set_allocator(None))
        return
    a = ALLOC_FN(lambda nbytes, stream, ctx: alloc(int(nbytes), int(stream or 0)) or None)
    r = RELEASE_FN(lambda ptr, stream, ctx: release(int(ptr), int(stream or 0)))
    spec = lbcg_allocator(a, r, None)
    _check(library().lbcg_set_allocator(C.byref(spec)))
    _allocator_keepalive.append((a, r, spec))   # the callbacks outlive every handle using them


def use_torch_allocator(enable: bool = True):
    """Take the device memory of handles created afterwards from PyTorch's caching allocator
    (so torch.cuda.memory_allocated() counts it); enable=False restores cudaMalloc."""
    if not enable:
        lbcg_set_allocator()
        return
    import torch

    def _alloc(nbytes, stream):
        return torch.cuda.caching_allocator_alloc(nbytes, stream=stream)

    def _release(ptr, stream):
        torch.cuda.caching_allocator_delete(ptr)

    lbcg_set_allocator(_alloc, _release)


def lbcg_autotune(h: int, probe_steps: int = 10) -> int:
    """Time each step schedule on the current state and keep the fastest (0 = sweep, else tile height)."""
    out = C.c_int32(-1)
    _check(library().lbcg_autotune(h, probe_steps, C.byref(out)))
    return out.value


def lbcg_schedule(h: int) -> int:
    out = C.c_int32(-1)
    _check(library().lbcg_schedule(h, C.byref(out)))
    return out.value


def lbcg_diagnostics(h: int, lattice: int, circle, inside_red: bool = True) -> dict:
    """E_1 against the previous call's velocity and E_NPMT for the circle (cx, cy, r)."""
    cx, cy, r = circle
    out = lbcg_diag()
    _check(library().lbcg_diagnostics(h, lattice, C.byref(lbcg_diag_spec(cx, cy, r, 1 if inside_red else 0)),
                                      C.byref(out)))
    return {k: getattr(out, k) for k, _ in lbcg_diag._fields_}


def lbcg_profile(h: int, enable: bool):
    _check(library().lbcg_profile(h, 1 if enable else 0))


def lbcg_kernel_times(h: int):
    """(ms of the wall kernel and the step kernel summed, number of profiled steps)."""
    ms = (C.c_double * 2)()
    n = C.c_int64()
    _check(library().lbcg_kernel_times(h, ms, C.byref(n)))
    return list(ms), n.value


def lbcg_launches_per_step(h: int) -> int:
    return int(library().lbcg_launches_per_step(h))


def lbcg_step_launches(h: int) -> int:
    return int(library().lbcg_step_launches(h))


def lbcg_total_nodes(h: int) -> int:
    return int(library().lbcg_total_nodes(h))


def lbcg_destroy(h: int):
    _check(library().lbcg_destroy(h))


LBCG_MASK_SOLID = 1
LBCG_MASK_NO_FIT = 8


def lbcg_field_moments_noalloc(fields_ptr: int, mask_ptr: int, nx: int, ny: int, stream: int, out_ptr: int):
    """Device pointers in, device pointer out (17 doubles); allocates nothing."""
    _check(library().lbcg_field_moments_noalloc(fields_ptr, mask_ptr, nx, ny, C.c_void_p(stream or None), out_ptr))


def lbcg_adjoint(h: int, nx: int, ny: int, nsteps: int, checkpoint: int, weight: Optional[np.ndarray] = None,
                 tip_rows=None, cl_rows=None, objective: Optional[str] = None, reverse_fp32: bool = False) -> dict:
    """Run nsteps forward, then the reverse sweep; returns J and its gradients.  With `weight`
    ([ny, nx]) J = sum weight * rho^N at the last step; otherwise `objective` selects
    "finger_length" (the default) or "red_mass".  reverse_fp32 runs the reverse kernels in FP32."""
    if weight is not None:
        w = np.ascontiguousarray(weight, dtype=np.float64).reshape(ny, nx)
        obj, wp = LBCG_OBJ_WEIGHTED, _dptr(w)
    else:
        w, obj, wp = None, OBJECTIVES[objective or "finger_length"], None
    o = obs_spec(ny=ny, tip_rows=tip_rows, cl_rows=cl_rows)
    spec = lbcg_adjoint_spec(nsteps, checkpoint, obj, wp, o.tip_row0, o.tip_row1, o.cl_row0, o.cl_row1,
                             1 if reverse_fp32 else 0)
    dth = np.zeros((ny, nx), dtype=np.float64)
    out = lbcg_grads(0, 0, 0, 0, 0, _dptr(dth))
    _check(library().lbcg_adjoint(h, C.byref(spec), C.byref(out)))
    return {"J": out.J, "dsigma": out.dJ_dsigma, "dnu_R": out.dJ_dnu_R, "dnu_B": out.dJ_dnu_B,
            "dtheta": out.dJ_dtheta, "dtheta_node": dth}


def obs_spec(wall_y: float = 0.5, cyl=None, tip_rows=None, cl_rows=None, ny: Optional[int] = None) -> lbcg_obs_spec:
    if tip_rows is None:
        tip_rows = ((ny // 2 - 1, ny // 2) if ny % 2 == 0 else (ny // 2, ny // 2)) if ny else (-1, -1)
    if cl_rows is None:
        cl_rows = (1, ny - 2) if ny else (-1, -1)
    cx, cy, cr = cyl if cyl is not None else (0.0, 0.0, 0.0)
    return lbcg_obs_spec(wall_y, cx, cy, cr, tip_rows[0], tip_rows[1], cl_rows[0], cl_rows[1])


class Lattice:
    """One handle of liblbcg.so holding one or more lattices."""

    def __init__(self, geoms, prms, precision="fp32", stream: int = 0):
        if isinstance(geoms, Geometry):
            geoms, prms = [geoms], [prms]
        self.geoms = list(geoms)
        self.prms = list(prms)
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.h = lbcg_create_batch(self.geoms, self.prms, self.precision, stream)

    def step(self, n: int = 1):
        lbcg_step(self.h, n)

    def observables(self, lattice: int = 0, **kw) -> dict:
        g = self.geoms[lattice]
        return lbcg_observables(self.h, lattice, obs_spec(ny=g.ny, **kw))

    def populations(self, lattice: int = 0) -> np.ndarray:
        g = self.geoms[lattice]
        return lbcg_get_populations(self.h, lattice, g.nx, g.ny)

    def set_populations(self, f: np.ndarray, lattice: int = 0):
        lbcg_set_populations(self.h, lattice, f)

    def fields(self, lattice: int = 0) -> np.ndarray:
        g = self.geoms[lattice]
        return lbcg_get_fields(self.h, lattice, g.nx, g.ny)

    def adjoint(self, nsteps: int, checkpoint: int, weight: Optional[np.ndarray] = None, **kw) -> dict:
        """Gradients of J at step (current + nsteps); see lbcg_adjoint.  FP64 or FP32, one lattice."""
        g = self.geoms[0]
        return lbcg_adjoint(self.h, g.nx, g.ny, nsteps, checkpoint, weight, **kw)

    def set_tile(self, ty: int):
        lbcg_set_tile(self.h, ty)

    def set_sweep(self, rows: int = 0):
        lbcg_set_sweep(self.h, rows)

    def set_poll_limit(self, polls: int = -1):
        lbcg_set_poll_limit(self.h, polls)

    def diagnostics(self, circle, inside_red: bool = True, lattice: int = 0) -> dict:
        return lbcg_diagnostics(self.h, lattice, circle, inside_red)

    def autotune(self, probe_steps: int = 10) -> int:
        return lbcg_autotune(self.h, probe_steps)

    @property
    def schedule(self) -> int:
        return lbcg_schedule(self.h)

    @property
    def sweep_rows(self) -> int:
        return int(library().lbcg_sweep_rows(self.h))

    @property
    def state_bytes(self) -> int:
        return lbcg_state_bytes(self.h)

    @property
    def launches_per_step(self) -> int:
        return lbcg_launches_per_step(self.h)

    @property
    def step_launches(self) -> int:
        return lbcg_step_launches(self.h)

    @property
    def total_nodes(self) -> int:
        return lbcg_total_nodes(self.h)

    def close(self):
        if self.h:
            lbcg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
