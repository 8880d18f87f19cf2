"""Seeded synthetic inputs: lattice geometries, initial colour fields and parameter sets.

This module is shared by the CUDA path (through the C-ABI binding), the FP64 oracle
(through the tests) and ``bench.py``.  It holds no arithmetic of the method itself:
it only lays out solid nodes, initial colour-indicator fields rho^N_0, optional analytic
solid normals and per-node contact angles, and the physical parameters of each workload.

Workloads follow the paper's test problems:

* static droplet on a flat wall (Sec. III.A; the paper's 160x100 case and a 100x50 analogue),
* droplet on a cylinder (Sec. III.B, 200x200, cylinder R=40 at (100, 60)),
* capillary filling between two solid blocks in a periodic box (Sec. III.C),
* displacement in a channel with a velocity inlet and a pressure outlet (Sec. III.D),
* a batch of such channels of uneven size with swept (M, Ca, theta),
* a large two-wall box whose state is far larger than the GPU's L2 cache (roofline runs).

Conventions (used identically by both implementations):

* arrays are row-major ``[ny, nx]`` with x fastest; node (x, y) sits at integer
  coordinates, the half-way bounce-back wall lies half a lattice unit outside the
  outermost fluid node;
* ``solid`` is uint8, 1 = solid, 0 = fluid;
* ``bc_x`` is ``"periodic"``, ``"closed"`` (edge columns must be solid) or ``"inout"``
  (velocity inlet on column 0, pressure outlet on column nx-1); ``bc_y`` is
  ``"periodic"`` or ``"closed"`` (edge rows must be solid);
* contact angles are in radians, measured through the red fluid (red wets for theta < 90 deg);
* the initial colour field is sharp (+1 red / -1 blue by node-centre inside test) plus
  uniform noise of amplitude ``noise`` drawn from ``numpy.random.default_rng(seed)``,
  clamped to [-1, 1].
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

BC_X = ("periodic", "closed", "inout")
BC_Y = ("periodic", "closed")


@dataclasses.dataclass
class Params:
    """Physical and numerical parameters of one lattice (Sec. II.A, Eq. 4-6, 10, 14, 18)."""

    nu_R: float = 1.0 / 6.0      # kinematic viscosity of the red fluid
    nu_B: float = 1.0 / 6.0      # kinematic viscosity of the blue fluid
    sigma: float = 1e-2          # interfacial tension coefficient (Eq. 10)
    theta: float = math.pi / 2   # prescribed contact angle [rad] (Eq. 34)
    beta: float = 0.7            # segregation parameter (Eq. 14)
    s_e: float = 1.64            # Eq. 6
    s_eps: float = 1.54          # Eq. 6
    s_q: float = 1.9             # Eq. 6
    rho0: float = 1.0            # reference density of both fluids
    u_in: float = 0.0            # uniform inlet velocity (bc_x == "inout")
    rho_out: float = 1.0         # outlet density (bc_x == "inout")
    grad_eps: float = 1e-12      # |grad rho^N| at or below which n = 0
    inlet_profile: int = 0       # 0: uniform u_in; 1: Poiseuille profile of maximum u_in
    wetting: int = 0             # 0: improved scheme (a); 1: scheme (b), Eq. 48; 2: surface energy


@dataclasses.dataclass
class Geometry:
    nx: int
    ny: int
    solid: np.ndarray                       # uint8 [ny, nx]
    rhoN0: np.ndarray                       # float64 [ny, nx]
    bc_x: str = "periodic"
    bc_y: str = "closed"
    normal: Optional[np.ndarray] = None     # float64 [2, ny, nx] analytic n_s (into the solid) or None
    theta_node: Optional[np.ndarray] = None # float64 [ny, nx] per-node contact angle [rad] or None
    name: str = ""

    def __post_init__(self):
        assert self.bc_x in BC_X and self.bc_y in BC_Y
        self.solid = np.ascontiguousarray(self.solid, dtype=np.uint8)
        self.rhoN0 = np.ascontiguousarray(self.rhoN0, dtype=np.float64)
        assert self.solid.shape == (self.ny, self.nx) and self.rhoN0.shape == (self.ny, self.nx)
        if self.normal is not None:
            self.normal = np.ascontiguousarray(self.normal, dtype=np.float64)
            assert self.normal.shape == (2, self.ny, self.nx)
        if self.theta_node is not None:
            self.theta_node = np.ascontiguousarray(self.theta_node, dtype=np.float64)
            assert self.theta_node.shape == (self.ny, self.nx)

    @property
    def n_nodes(self) -> int:
        return self.nx * self.ny


def _noisy(sign: np.ndarray, solid: np.ndarray, noise: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    rhoN = sign.astype(np.float64)
    if noise > 0:
        rhoN = rhoN + rng.uniform(-noise, noise, size=rhoN.shape)
    rhoN = np.clip(rhoN, -1.0, 1.0)
    rhoN[solid != 0] = 0.0
    return rhoN


def _grid(nx: int, ny: int):
    y, x = np.mgrid[0:ny, 0:nx]
    return x.astype(np.float64), y.astype(np.float64)


def periodic_box_droplet(nx: int, ny: int, R: float, xc: Optional[float] = None,
                         yc: Optional[float] = None, noise: float = 0.0, seed: int = 0) -> Geometry:
    """Free red droplet of radius R in a blue, fully periodic box (Laplace test)."""
    x, y = _grid(nx, ny)
    xc = nx / 2 if xc is None else xc
    yc = ny / 2 if yc is None else yc
    solid = np.zeros((ny, nx), np.uint8)
    inside = (x - xc) ** 2 + (y - yc) ** 2 < R * R
    return Geometry(nx, ny, solid, _noisy(np.where(inside, 1, -1), solid, noise, seed),
                    bc_x="periodic", bc_y="periodic", name=f"periodic_droplet_{nx}x{ny}_R{R}")


def flat_wall_droplet(nx: int = 100, ny: int = 50, R: float = 20.0, xc: Optional[float] = None,
                      yc: Optional[float] = None, noise: float = 1e-3, seed: int = 0,
                      closed_x: bool = False) -> Geometry:
    """Droplet on the bottom wall of a channel with solid rows 0 and ny-1.

    The default centre lies on the half-way wall (y = 0.5), giving a semicircle.  With
    ``closed_x`` the edge columns are solid too (the paper's closed box, Sec. III.A).
    """
    x, y = _grid(nx, ny)
    xc = nx / 2 if xc is None else xc
    yc = 0.5 if yc is None else yc
    solid = np.zeros((ny, nx), np.uint8)
    solid[0, :] = 1
    solid[ny - 1, :] = 1
    if closed_x:
        solid[:, 0] = 1
        solid[:, nx - 1] = 1
    inside = (x - xc) ** 2 + (y - yc) ** 2 < R * R
    return Geometry(nx, ny, solid, _noisy(np.where(inside, 1, -1), solid, noise, seed),
                    bc_x="closed" if closed_x else "periodic", bc_y="closed",
                    name=f"flat_wall_droplet_{nx}x{ny}_R{R}")


def cylinder_droplet(nx: int = 200, ny: int = 200, Rs: float = 40.0, cx: float = 100.0,
                     cy: float = 60.0, Rd: float = 40.0, theta: float = math.pi / 2,
                     noise: float = 0.0, seed: int = 0, analytic_normal: bool = True) -> Geometry:
    """Red droplet resting on a solid cylinder (Sec. III.B) in a closed box.

    The droplet centre sits at the distance D = sqrt(Rs^2 + Rd^2 - 2 Rs Rd cos(theta)) above
    the cylinder centre, the distance at which two circles meet at angle theta.
    The analytic normal at node (x, y) is the unit vector from (x, y) towards the cylinder
    centre (pointing into the solid).
    """
    x, y = _grid(nx, ny)
    solid = ((x - cx) ** 2 + (y - cy) ** 2 <= Rs * Rs).astype(np.uint8)
    solid[0, :] = 1
    solid[ny - 1, :] = 1
    solid[:, 0] = 1
    solid[:, nx - 1] = 1
    D = math.sqrt(Rs * Rs + Rd * Rd - 2 * Rs * Rd * math.cos(theta))
    inside = (x - cx) ** 2 + (y - (cy + D)) ** 2 < Rd * Rd
    normal = None
    if analytic_normal:
        dx, dy = cx - x, cy - y
        r = np.sqrt(dx * dx + dy * dy)
        r[r == 0] = 1.0
        normal = np.stack([dx / r, dy / r])
    return Geometry(nx, ny, solid, _noisy(np.where(inside, 1, -1), solid, noise, seed),
                    bc_x="closed", bc_y="closed", normal=normal,
                    name=f"cylinder_droplet_{nx}x{ny}")


def capillary_filling(L: int = 800, d: int = 40, reservoir: int = 200, wall: int = 20,
                      red_into: int = 100, noise: float = 0.0, seed: int = 0) -> Geometry:
    """Capillary filling in a periodic box (Sec. III.C layout).

    Two solid blocks of thickness ``wall`` sit above and below a channel of ``d`` fluid rows
    over ``reservoir <= x < reservoir + L``; the reservoirs at both ends span the full
    height.  Red fills x < reservoir + red_into, blue the rest.  Periodic in x and y.
    """
    nx = L + 2 * reservoir
    ny = d + 2 * wall
    x, y = _grid(nx, ny)
    solid = np.zeros((ny, nx), np.uint8)
    in_chan = (x >= reservoir) & (x < reservoir + L)
    solid[(in_chan) & ((y < wall) | (y >= wall + d))] = 1
    red = x < reservoir + red_into
    return Geometry(nx, ny, solid, _noisy(np.where(red, 1, -1), solid, noise, seed),
                    bc_x="periodic", bc_y="periodic", name=f"capillary_{nx}x{ny}")


def displacement_channel(W: int = 100, L: int = 2000, x_I: float = 100.0, amp: float = 0.5,
                         seed: int = 0, noise: float = 0.0) -> Geometry:
    """Channel of W fluid rows between solid rows 0 and W+1, inlet at x=0, outlet at x=L-1.

    Red (the invading fluid) fills x < x_I(y) with
    x_I(y) = x_I + amp*sin(2*pi*y/W + phi0) + amp*xi(y), xi ~ U(-1, 1) per row, phi0 ~ U(0, 2pi).
    """
    rng = np.random.default_rng(seed)
    nx, ny = L, W + 2
    x, y = _grid(nx, ny)
    phi0 = rng.uniform(0.0, 2 * math.pi)
    xi = rng.uniform(-1.0, 1.0, size=ny)
    xI = x_I + amp * np.sin(2 * math.pi * np.arange(ny) / W + phi0) + amp * xi
    solid = np.zeros((ny, nx), np.uint8)
    solid[0, :] = 1
    solid[ny - 1, :] = 1
    red = x < xI[:, None]
    return Geometry(nx, ny, solid, _noisy(np.where(red, 1, -1), solid, noise, seed + 1),
                    bc_x="inout", bc_y="closed", name=f"channel_{nx}x{ny}")


def two_wall_box(nx: int, ny: int, bands: int = 4, noise: float = 1e-3, seed: int = 0) -> Geometry:
    """Periodic-x box with solid rows 0 and ny-1 and alternating red/blue vertical bands."""
    x, y = _grid(nx, ny)
    solid = np.zeros((ny, nx), np.uint8)
    solid[0, :] = 1
    solid[ny - 1, :] = 1
    band = np.floor(x * bands / nx).astype(np.int64) % 2 == 0
    return Geometry(nx, ny, solid, _noisy(np.where(band, 1, -1), solid, noise, seed),
                    bc_x="periodic", bc_y="closed", name=f"two_wall_box_{nx}x{ny}")


# ----------------------------------------------------------------------------- parameter maps

def fingering_params(M: float, Ca: float, theta_deg: float, nu_R: float = 0.5,
                     u_in: float = 0.01) -> Params:
    """Sec. III.D parameter mapping: M = nu_R/nu_B, Ca = nu_R*u0/sigma."""
    return Params(nu_R=nu_R, nu_B=nu_R / M, sigma=nu_R * u_in / Ca,
                  theta=math.radians(theta_deg), u_in=u_in, rho_out=1.0)


M_GRID = (1.0, 5.0, 20.0, 50.0, 100.0)
CA_GRID = (0.01, 0.05, 0.1)
THETA_GRID = (30.0, 60.0, 90.0, 120.0, 150.0)


def channel_sweep(n: int = 64, seed: int = 0, wmin: int = 40, wmax: int = 200,
                  aspect: int = 10, x_I_frac: float = 0.05, param_seed: Optional[int] = None):
    """A batch of displacement channels of uneven size with (M, Ca, theta) drawn from the grids.

    Widths W ~ U{wmin..wmax}, lengths 10*W; returns (geometries, params).  With
    ``param_seed`` the widths still come from ``seed`` but (M, Ca, theta) and the interface
    noise come from ``param_seed``: batches of equal size with different parameters (one
    per rank of a weak-scaling run).
    """
    rng = np.random.default_rng(seed)
    prng = None if param_seed is None else np.random.default_rng(param_seed)
    gseed = seed if param_seed is None else param_seed
    geoms: List[Geometry] = []
    prms: List[Params] = []
    for i in range(n):
        W = int(rng.integers(wmin, wmax + 1))
        M = float(rng.choice(M_GRID))
        Ca = float(rng.choice(CA_GRID))
        th = float(rng.choice(THETA_GRID))
        if prng is not None:
            M, Ca, th = float(prng.choice(M_GRID)), float(prng.choice(CA_GRID)), float(prng.choice(THETA_GRID))
        geoms.append(displacement_channel(W=W, L=aspect * W, x_I=max(4.0, x_I_frac * aspect * W),
                                          seed=gseed * 1000 + i))
        prms.append(fingering_params(M, Ca, th))
    return geoms, prms


def config_static_droplet() -> tuple:
    """Flat bottom wall, 100x50, R=20 semicircle, theta=60 deg, M=1, sigma=1e-2, tau=1."""
    g = flat_wall_droplet(100, 50, R=20.0, noise=1e-3, seed=0)
    p = Params(nu_R=1 / 6, nu_B=1 / 6, sigma=1e-2, theta=math.radians(60.0))
    return g, p


def config_capillary() -> tuple:
    """Capillary filling: 1200x80, channel d=40, L=800, theta=30 deg, M=1, sigma=1e-2."""
    g = capillary_filling(L=800, d=40, reservoir=200, wall=20, red_into=100)
    p = Params(nu_R=1 / 6, nu_B=1 / 6, sigma=1e-2, theta=math.radians(30.0))
    return g, p


def config_fingering(M: float = 1.0, Ca: float = 0.05, theta_deg: float = 90.0, seed: int = 0):
    """Displacement channel: width 100, length 2000, interface at x=100."""
    return displacement_channel(W=100, L=2000, x_I=100.0, seed=seed), fingering_params(M, Ca, theta_deg)


def fingering_grid():
    """The viscous-fingering study as one batch: a 2000x102 channel (width 100, interface at
    x = 100, its own interface noise from seed i) for every (M, Ca, theta) of the grids,
    M x Ca x theta = 5 x 3 x 5 = 75 channels; returns (geometries, params)."""
    pts = [(M, Ca, th) for M in M_GRID for Ca in CA_GRID for th in THETA_GRID]
    geoms, prms = zip(*[config_fingering(M=M, Ca=Ca, theta_deg=th, seed=i) for i, (M, Ca, th) in enumerate(pts)])
    return list(geoms), list(prms)


def config_wettability(theta_deg: float, seed: int = 0):
    """Sec. III.D.2 (wettability): 630x60 domain (58 fluid rows between two wall rows), flat
    initial interface at x = 30, Poiseuille inlet of maximum u0 = 0.1, pressure outlet,
    nu_R = nu_B = 0.3 (M = 1), sigma = 0.06 (Ca = nu_R u0 / sigma = 0.5)."""
    g = displacement_channel(W=58, L=630, x_I=30.0, amp=0.0, seed=seed)
    p = Params(nu_R=0.3, nu_B=0.3, sigma=0.06, theta=math.radians(theta_deg), u_in=0.1, rho_out=1.0,
               inlet_profile=1)
    return g, p


def config_adjoint(seed: int = 0):
    """Adjoint workload: channel width 40, length 400, M=10, Ca=0.05, theta=60 deg."""
    return displacement_channel(W=40, L=400, x_I=40.0, seed=seed), fingering_params(10.0, 0.05, 60.0)
