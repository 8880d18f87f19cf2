"""FP64 CPU oracle of one time step of the two-colour D2Q9 MRT colour-gradient lattice
Boltzmann method with the improved geometric wetting scheme (Yu, Liu, Zhang & Liang,
arXiv 1707.00198, Sec. II).

THIS IS TEST INFRASTRUCTURE.  It exists only to check the CUDA path: only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline leg and ``--impl reference``)
may import it.  It shares no code with the CUDA library and imports nothing from it.

It is written for clarity, not speed: plain PyTorch float64 CPU operations over whole
fields, one lattice direction at a time, in the order of the paper's equations.  Neighbour
values phi(x + e) come from ``torch.roll`` (periodic axes) or an index clamp (open axes,
which doubles as the zero-gradient ghost column).  Every operation is differentiable, so
``torch.autograd`` can run through whole trajectories on tiny lattices.

Readings of places where the paper is silent, garbled or ambiguous (each listed with its
reason in the design notes of this repository):

* Eq. 3: the last row of M is the moment p_xy = e_x e_y, i.e. (0 0 0 0 0 1 -1 1 -1); the
  printed row is not orthogonal to the first row.
* Eq. 14: the blue line carries a minus sign, so that f''_R + f''_B = f'.
* Eq. 14: the perturbation is w_a (e_a . n) with n = grad rho^N / |grad rho^N|, no 1/|e_a|.
* Eq. 15: each colour streams itself.
* Eq. 5 and 18: both fluids have density rho0, so the dynamic and kinematic viscosities
  coincide; tau_v = 3 nu + 1/2 per node.
* u in Eq. 7 and Eq. 9 is the velocity of Eq. 17 (with the F/2 term).
* If |grad rho^N| <= grad_eps, n = 0 (no perturbation, no recolouring bias, F = 0).
* Omega_Fb = fluid nodes with at least one solid D2Q9 neighbour; outermost solid nodes =
  solid nodes with at least one fluid D2Q9 neighbour; alpha_1 runs over the D2Q9
  directions from such a solid node to fluid nodes (Eq. 29).
* The corrected gradient of Eq. 31 replaces the raw one everywhere downstream (n, the
  virtual n, kappa, F and the recolouring direction).
* n_s of Eq. 32 points from the fluid into the solid; theta is measured through the red
  fluid; Eq. 34 multiplies the row vector n_s by the matrix, i.e. (n_f)_1 is n_s rotated
  counter-clockwise by theta; the tie D1 == D2 picks (n_f)_1 (Eq. 36).
* E8 stencil (Eq. 32) beyond the array edge: periodic wrap on periodic axes, solid on
  closed axes, a copy of the edge column on the inlet/outlet axis.
* Inlet/outlet (Sec. III.D, used with bc_x = "inout"): Zou-He velocity inlet carrying pure
  red fluid at x = 0, Zou-He pressure outlet (rho = rho_out) at x = nx-1 whose unknown
  populations take the colour fraction of the outlet node's known populations.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

DT = torch.float64

# ------------------------------------------------------------------ D2Q9 lattice (Sec. II.A)
# e_0 = (0,0), e_{1,3} = (+-1,0), e_{2,4} = (0,+-1), e_{5,6} = (+-1,1), e_{7,8} = (-+1,-1)
E = ((0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1))
W = (4 / 9, 1 / 9, 1 / 9, 1 / 9, 1 / 9, 1 / 36, 1 / 36, 1 / 36, 1 / 36)
OPP = (0, 3, 4, 1, 2, 7, 8, 5, 6)
CS2 = 1.0 / 3.0

# Eq. 3, rows (rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy); last row read as e_x*e_y.
M_ROWS = (
    (1, 1, 1, 1, 1, 1, 1, 1, 1),
    (-4, -1, -1, -1, -1, 2, 2, 2, 2),
    (4, -2, -2, -2, -2, 1, 1, 1, 1),
    (0, 1, 0, -1, 0, 1, -1, -1, 1),
    (0, -2, 0, 2, 0, 1, -1, -1, 1),
    (0, 0, 1, 0, -1, 1, 1, -1, -1),
    (0, 0, -2, 0, 2, 1, 1, -1, -1),
    (0, 1, -1, 1, -1, 0, 0, 0, 0),
    (0, 0, 0, 0, 0, 1, -1, 1, -1),
)


def mrt_matrix() -> torch.Tensor:
    """M of Eq. 3."""
    return torch.tensor(M_ROWS, dtype=DT)


def mrt_inverse() -> torch.Tensor:
    """M^-1 by a library inverse (no closed form is assumed here)."""
    return torch.linalg.inv(mrt_matrix())


# ------------------------------------------------------------------ E8 stencil (Eq. 32-33)
def e8_stencil():
    """The 24 vectors of the eighth-order isotropic stencil with their weights w(|c|^2)."""
    wt = {1: 4 / 21, 2: 4 / 45, 4: 1 / 60, 5: 2 / 315, 8: 1 / 5040}
    out = []
    for cy in range(-2, 3):
        for cx in range(-2, 3):
            c2 = cx * cx + cy * cy
            if c2 in wt:
                out.append((cx, cy, wt[c2]))
    return out


# ------------------------------------------------------------------ neighbour access
def neighbour(phi: torch.Tensor, ex: int, ey: int, periodic_x: bool, periodic_y: bool) -> torch.Tensor:
    """phi(x + e) for a field whose last two dims are [ny, nx].

    Periodic axes wrap; non-periodic axes clamp the index (the ghost row/column copies the
    edge node).
    """
    ny, nx = phi.shape[-2], phi.shape[-1]
    if ex != 0:
        if periodic_x:
            phi = torch.roll(phi, shifts=-ex, dims=-1)
        else:
            idx = torch.clamp(torch.arange(nx) + ex, 0, nx - 1)
            phi = phi.index_select(-1, idx)
    if ey != 0:
        if periodic_y:
            phi = torch.roll(phi, shifts=-ey, dims=-2)
        else:
            idy = torch.clamp(torch.arange(ny) + ey, 0, ny - 1)
            phi = phi.index_select(-2, idy)
    return phi


# ------------------------------------------------------------------ lattice set-up
@dataclass
class OracleLattice:
    nx: int
    ny: int
    px: bool                  # periodic in x
    py: bool                  # periodic in y
    inout: bool               # velocity inlet at x=0, pressure outlet at x=nx-1
    solid: torch.Tensor       # bool [ny, nx]
    fluid: torch.Tensor       # bool [ny, nx]
    fluid_nb: torch.Tensor    # bool [9, ny, nx]: is x + e_a a fluid node
    outer_solid: torch.Tensor # bool [ny, nx]
    omega_fb: torch.Tensor    # bool [ny, nx]
    n_s: torch.Tensor         # float64 [2, ny, nx] solid normal at Omega_Fb nodes (else 0)
    theta: torch.Tensor       # float64 [ny, nx] contact angle at every node
    near_solid: torch.Tensor  # bool [ny, nx]: within Chebyshev distance 3 of a solid node


def solid_normal_e8(solid: torch.Tensor, omega_fb: torch.Tensor, bc_x: str, bc_y: str) -> torch.Tensor:
    """Eq. 32-33: n_s = sum_k w(|c_k|^2) s(x + c_k) c_k / |...| at Omega_Fb nodes.

    The weights of Eq. 33 are k/5040 with integer k (960, 448, 84, 32, 1); the common factor
    cancels in the normalisation, so the sum is taken over the integers k, which is exact.
    Flat walls then give exactly axis-aligned normals, so the tie D1 == D2 of Eq. 36 is an
    exact tie rather than a rounding accident."""
    ny, nx = solid.shape
    s = solid.to(DT)
    # pad by two on each side following the edge rule of the stencil
    pad_x = 2
    if bc_x == "periodic":
        s = torch.cat([s[:, -pad_x:], s, s[:, :pad_x]], dim=1)
    elif bc_x == "closed":
        s = torch.cat([torch.ones(ny, pad_x, dtype=DT), s, torch.ones(ny, pad_x, dtype=DT)], dim=1)
    else:
        s = torch.cat([s[:, :1].expand(ny, pad_x), s, s[:, -1:].expand(ny, pad_x)], dim=1)
    if bc_y == "periodic":
        s = torch.cat([s[-2:, :], s, s[:2, :]], dim=0)
    else:
        s = torch.cat([torch.ones(2, nx + 4, dtype=DT), s, torch.ones(2, nx + 4, dtype=DT)], dim=0)
    vx = torch.zeros(ny, nx, dtype=DT)
    vy = torch.zeros(ny, nx, dtype=DT)
    for cx, cy, w in e8_stencil():
        k = float(round(w * 5040))
        sv = s[2 + cy: 2 + cy + ny, 2 + cx: 2 + cx + nx]
        vx = vx + k * sv * cx
        vy = vy + k * sv * cy
    mag = torch.sqrt(vx * vx + vy * vy)
    ok = omega_fb & (mag > 0)
    safe = torch.where(ok, mag, torch.ones_like(mag))
    return torch.stack([torch.where(ok, vx / safe, 0.0), torch.where(ok, vy / safe, 0.0)])


def make_lattice(geom, theta: float | torch.Tensor) -> OracleLattice:
    """Classify nodes (Sec. II.C) and set up solid normals and contact angles."""
    nx, ny = geom.nx, geom.ny
    px = geom.bc_x == "periodic"
    py = geom.bc_y == "periodic"
    solid = torch.from_numpy(np.asarray(geom.solid) != 0)
    fluid = ~solid
    # neighbour fluid flags; on open (inout) x edges the ghost copies the edge node
    fluid_nb = torch.stack([neighbour(fluid, ex, ey, px, py) for ex, ey in E])
    if geom.bc_x == "closed":
        assert bool(solid[:, 0].all()) and bool(solid[:, -1].all()), "closed x needs solid edge columns"
    if geom.bc_y == "closed":
        assert bool(solid[0, :].all()) and bool(solid[-1, :].all()), "closed y needs solid edge rows"
    any_fluid_nb = fluid_nb[1:].any(dim=0)
    any_solid_nb = (~fluid_nb[1:]).any(dim=0)
    outer_solid = solid & any_fluid_nb
    omega_fb = fluid & any_solid_nb
    if geom.normal is not None:
        n_s = torch.from_numpy(np.asarray(geom.normal)).to(DT) * omega_fb.to(DT)
    else:
        n_s = solid_normal_e8(solid, omega_fb, geom.bc_x, geom.bc_y)
    if geom.theta_node is not None and not torch.is_tensor(theta):
        th = torch.from_numpy(np.asarray(geom.theta_node)).to(DT)
    elif torch.is_tensor(theta):
        th = theta.to(DT) * torch.ones(ny, nx, dtype=DT)
    else:
        th = torch.full((ny, nx), float(theta), dtype=DT)
    # distance-to-solid flag for the contact-angle measurement (Chebyshev radius 3)
    near = solid.clone()
    for dy in range(-3, 4):
        for dx in range(-3, 4):
            near = near | neighbour(solid, dx, dy, px, py)
    return OracleLattice(nx, ny, px, py, geom.bc_x == "inout", solid, fluid, fluid_nb,
                         outer_solid, omega_fb, n_s, th, near)


# ------------------------------------------------------------------ initial state
def init_state(lat: OracleLattice, rhoN0, rho0: float = 1.0, prm=None):
    """Rest equilibrium with the caller's colour field: f_{a,R} = w_a rho0 (1 + rho^N_0)/2,
    f_{a,B} = w_a rho0 (1 - rho^N_0)/2 on fluid nodes, zero on solid nodes.

    On an inlet/outlet lattice the Zou-He conditions of Sec. III.D constrain the
    post-streaming populations of the open columns; the initial state is a post-streaming
    state, so they are imposed on it too (``prm`` supplies u_in and rho_out)."""
    r = torch.as_tensor(np.asarray(rhoN0), dtype=DT)
    fl = lat.fluid.to(DT)
    w = torch.tensor(W, dtype=DT)[:, None, None]
    fR = w * rho0 * (1 + r) / 2 * fl
    fB = w * rho0 * (1 - r) / 2 * fl
    if lat.inout:
        if prm is None:
            raise ValueError("an inlet/outlet lattice needs the parameters to set its initial state")
        fR, fB = inlet_outlet(lat, prm, fR, fB)
    return fR, fB


# ------------------------------------------------------------------ gradients (Eq. 28-36)
def virtual_fill(lat: OracleLattice, phi: torch.Tensor) -> torch.Tensor:
    """Eq. 29: on outermost solid nodes replace phi by the w-weighted mean of phi over the
    D2Q9 neighbours that are fluid; fluid nodes keep phi; other solid nodes get 0."""
    num = torch.zeros_like(phi)
    den = torch.zeros(lat.ny, lat.nx, dtype=DT)
    for a in range(1, 9):
        ex, ey = E[a]
        fl = lat.fluid_nb[a].to(DT)
        num = num + W[a] * neighbour(phi, ex, ey, lat.px, lat.py) * fl
        den = den + W[a] * fl
    safe = torch.where(lat.outer_solid, den, torch.ones_like(den))
    virt = torch.where(lat.outer_solid, num / safe, torch.zeros_like(phi))
    return torch.where(lat.fluid, phi, virt)


def iso_gradient(lat: OracleLattice, phi: torch.Tensor):
    """Eq. 28: d_i phi(x) = (1/c_s^2) sum_a w_a phi(x + e_a) e_{a,i}."""
    gx = torch.zeros_like(phi)
    gy = torch.zeros_like(phi)
    for a in range(1, 9):
        ex, ey = E[a]
        nb = neighbour(phi, ex, ey, lat.px, lat.py)
        gx = gx + W[a] * nb * ex
        gy = gy + W[a] * nb * ey
    return gx / CS2, gy / CS2


def one_sided_gradient(lat: OracleLattice, phi: torch.Tensor):
    """Eq. 48 (scheme (b)): d_i phi(x) = sum_a w_a [phi(x + e_a) - phi(x)] e_ai / sum_a w_a e_ai^2
    over the directions a whose neighbour is fluid.  The paper prints the denominator as
    sum_a w_a; normalising each component by sum_a w_a e_ai^2 makes the estimate exact on
    linear fields, as Eq. 28 is (as printed, a full stencil would return 0.6 of the gradient)."""
    gx = torch.zeros_like(phi)
    gy = torch.zeros_like(phi)
    wx = torch.zeros_like(phi)
    wy = torch.zeros_like(phi)
    for a in range(1, 9):
        ex, ey = E[a]
        fl = lat.fluid_nb[a].to(DT)
        d = neighbour(phi, ex, ey, lat.px, lat.py) - phi
        gx = gx + W[a] * d * ex * fl
        gy = gy + W[a] * d * ey * fl
        wx = wx + W[a] * ex * ex * fl
        wy = wy + W[a] * ey * ey * fl
    return (torch.where(wx > 0, gx / torch.where(wx > 0, wx, torch.ones_like(wx)), torch.zeros_like(gx)),
            torch.where(wy > 0, gy / torch.where(wy > 0, wy, torch.ones_like(wy)), torch.zeros_like(gy)))


def wetting_correction(lat: OracleLattice, gx: torch.Tensor, gy: torch.Tensor, eps: float):
    """Eq. 30-36 on Omega_Fb nodes: keep |grad rho^N|, replace its direction by the rotated
    solid normal (n_f)_1 or (n_f)_2 nearer to the estimated direction."""
    mag = torch.sqrt(gx * gx + gy * gy)
    ok = mag > eps
    safe = torch.where(ok, mag, torch.ones_like(mag))
    esx, esy = gx / safe, gy / safe                       # Eq. 30
    nsx, nsy = lat.n_s[0], lat.n_s[1]
    c, s = torch.cos(lat.theta), torch.sin(lat.theta)
    # Eq. 34: row vector n_s times [[cos, sin], [-sin, cos]] (and the same with -theta)
    f1x, f1y = nsx * c - nsy * s, nsx * s + nsy * c
    f2x, f2y = nsx * c + nsy * s, -nsx * s + nsy * c
    d1 = torch.sqrt((f1x - esx) ** 2 + (f1y - esy) ** 2)  # Eq. 35
    d2 = torch.sqrt((f2x - esx) ** 2 + (f2y - esy) ** 2)
    pick1 = d1 <= d2                                      # Eq. 36
    nfx = torch.where(pick1, f1x, f2x)
    nfy = torch.where(pick1, f1y, f2y)
    sel = lat.omega_fb & ok
    return torch.where(sel, mag * nfx, gx), torch.where(sel, mag * nfy, gy)  # Eq. 31


def unit_normal(gx, gy, eps):
    """n = grad rho^N / |grad rho^N| (Eq. 11), zero where |grad rho^N| <= eps."""
    mag = torch.sqrt(gx * gx + gy * gy)
    ok = mag > eps
    safe = torch.where(ok, mag, torch.ones_like(mag))
    return torch.where(ok, gx / safe, 0.0), torch.where(ok, gy / safe, 0.0)


# ------------------------------------------------------------------ macroscopic fields
def densities(fR, fB):
    """Eq. 16 and Eq. 12."""
    rhoR = fR.sum(0)
    rhoB = fB.sum(0)
    rho = rhoR + rhoB
    return rhoR, rhoB, rho


def interface_fields(lat: OracleLattice, prm, fR, fB):
    """rho_R, rho_B, rho^N, corrected grad rho^N, n, kappa and F at every fluid node."""
    rhoR, rhoB, rho = densities(fR, fB)
    fl = lat.fluid
    rho_safe = torch.where(fl, rho, torch.ones_like(rho))
    rhoN = torch.where(fl, (rhoR - rhoB) / rho_safe, torch.zeros_like(rho))       # Eq. 12
    eps = prm.grad_eps
    wetting = getattr(prm, "wetting", 0)
    if wetting == 2:
        # surface-energy formulation (Sec. III.A.1): rho^N = cos(theta) on the outermost solid
        # nodes, no geometric correction
        filled = torch.where(lat.outer_solid, torch.full_like(rhoN, math.cos(float(prm.theta))), rhoN)
        gx, gy = iso_gradient(lat, filled)
    else:
        gx, gy = iso_gradient(lat, virtual_fill(lat, rhoN))                          # Eq. 28-29
        gx, gy = wetting_correction(lat, gx, gy, eps)                                # Eq. 30-36
    gx = torch.where(fl, gx, torch.zeros_like(gx))
    gy = torch.where(fl, gy, torch.zeros_like(gy))
    nx_, ny_ = unit_normal(gx, gy, eps)
    dnx_dx, dnx_dy = iso_gradient(lat, virtual_fill(lat, nx_))                      # Eq. 29, 28 (second BC)
    dny_dx, dny_dy = iso_gradient(lat, virtual_fill(lat, ny_))
    if wetting == 1:
        # scheme (b) (Sec. III.A.2): grad n on the outermost fluid nodes by Eq. 48
        bx_x, bx_y = one_sided_gradient(lat, nx_)
        by_x, by_y = one_sided_gradient(lat, ny_)
        fb = lat.omega_fb
        dnx_dx, dnx_dy = torch.where(fb, bx_x, dnx_dx), torch.where(fb, bx_y, dnx_dy)
        dny_dx, dny_dy = torch.where(fb, by_x, dny_dx), torch.where(fb, by_y, dny_dy)
    kappa = -nx_ * nx_ * dny_dy - ny_ * ny_ * dnx_dx + nx_ * ny_ * (dnx_dy + dny_dx)  # Eq. 13
    kappa = torch.where(fl, kappa, torch.zeros_like(kappa))
    Fx = 0.5 * prm.sigma * kappa * gx                                                # Eq. 10
    Fy = 0.5 * prm.sigma * kappa * gy
    return dict(rhoR=rhoR, rhoB=rhoB, rho=rho, rhoN=rhoN, gx=gx, gy=gy, nx=nx_, ny=ny_,
                kappa=kappa, Fx=Fx, Fy=Fy)


def velocity(lat, fR, fB, rho, Fx, Fy):
    """Eq. 17: rho u = sum_a f_a e_a + F/2."""
    f = fR + fB
    jx = sum(f[a] * E[a][0] for a in range(9))
    jy = sum(f[a] * E[a][1] for a in range(9))
    rho_safe = torch.where(lat.fluid, rho, torch.ones_like(rho))
    ux = torch.where(lat.fluid, (jx + 0.5 * Fx) / rho_safe, torch.zeros_like(rho))
    uy = torch.where(lat.fluid, (jy + 0.5 * Fy) / rho_safe, torch.zeros_like(rho))
    return ux, uy


def macroscopic(lat: OracleLattice, prm, fR, fB):
    """All per-node quantities of one time step before the collision."""
    d = interface_fields(lat, prm, fR, fB)
    d["ux"], d["uy"] = velocity(lat, fR, fB, d["rho"], d["Fx"], d["Fy"])
    return d


# ------------------------------------------------------------------ collision (Eq. 1-9)
def equilibrium(rho, ux, uy):
    """Eq. 7."""
    usq = ux * ux + uy * uy
    out = []
    for a in range(9):
        eu = E[a][0] * ux + E[a][1] * uy
        out.append(rho * W[a] * (1 + eu / CS2 + eu * eu / (2 * CS2 * CS2) - usq / (2 * CS2)))
    return torch.stack(out)


def guo_source(ux, uy, Fx, Fy):
    """Eq. 9: F~_a = w_a [(e_a - u)/c_s^2 + (e_a . u) e_a / c_s^4] . F."""
    out = []
    for a in range(9):
        ex, ey = E[a]
        eu = ex * ux + ey * uy
        cx = (ex - ux) / CS2 + eu * ex / (CS2 * CS2)
        cy = (ey - uy) / CS2 + eu * ey / (CS2 * CS2)
        out.append(W[a] * (cx * Fx + cy * Fy))
    return torch.stack(out)


def relaxation_rates(prm, rhoN):
    """Eq. 4-6 with tau_v from Eq. 5 and the harmonic viscosity of Eq. 18, per node.
    Returns the 9 diagonal entries of S as a [9, ny, nx] tensor."""
    inv_nu = (1 + rhoN) / (2 * prm.nu_R) + (1 - rhoN) / (2 * prm.nu_B)   # Eq. 18
    nu = 1.0 / inv_nu
    tau_v = nu / CS2 + 0.5                                               # Eq. 5 (delta_t = 1)
    sv = 1.0 / tau_v
    one = torch.ones_like(rhoN)
    return torch.stack([one, prm.s_e * one, prm.s_eps * one, one, prm.s_q * one,
                        one, prm.s_q * one, sv, sv])


def collide(lat, prm, fR, fB, mac):
    """Eq. 1, 2 and 8: f' = f - M^-1 S M (f - f^eq) + M^-1 (I - S/2) M F~ on the total f."""
    Mm = mrt_matrix()
    Minv = mrt_inverse()
    f = fR + fB
    feq = equilibrium(mac["rho"], mac["ux"], mac["uy"])
    Fsrc = guo_source(mac["ux"], mac["uy"], mac["Fx"], mac["Fy"])
    S = relaxation_rates(prm, mac["rhoN"])
    m_neq = torch.einsum("ab,bij->aij", Mm, f - feq)
    m_F = torch.einsum("ab,bij->aij", Mm, Fsrc)
    omega = -torch.einsum("ab,bij->aij", Minv, S * m_neq)
    Fbar = torch.einsum("ab,bij->aij", Minv, (1 - 0.5 * S) * m_F)
    return f + omega + Fbar


def recolour(lat, prm, fpost, mac):
    """Eq. 14 (blue line with the minus sign)."""
    rho = torch.where(lat.fluid, mac["rho"], torch.ones_like(mac["rho"]))
    rhoR, rhoB = mac["rhoR"], mac["rhoB"]
    nxv, nyv = mac["nx"], mac["ny"]
    outR, outB = [], []
    for a in range(9):
        en = E[a][0] * nxv + E[a][1] * nyv
        pert = prm.beta * rhoR * rhoB / rho * W[a] * en
        outR.append(rhoR / rho * fpost[a] + pert)
        outB.append(rhoB / rho * fpost[a] - pert)
    fl = lat.fluid.to(DT)
    return torch.stack(outR) * fl, torch.stack(outB) * fl


# ------------------------------------------------------------------ streaming (Eq. 15)
def stream(lat, prm, pR, pB):
    """Eq. 15 with half-way bounce-back: f_{a,k}(x, t+1) = f''_{a,k}(x - e_a, t) if x - e_a
    is a fluid node, else f''_{opp(a),k}(x, t)."""
    outR, outB = [], []
    for a in range(9):
        ex, ey = E[a]
        src_fluid = lat.fluid_nb[OPP[a]]             # is x - e_a fluid
        fromR = neighbour(pR[a], -ex, -ey, lat.px, lat.py)
        fromB = neighbour(pB[a], -ex, -ey, lat.px, lat.py)
        outR.append(torch.where(src_fluid, fromR, pR[OPP[a]]))
        outB.append(torch.where(src_fluid, fromB, pB[OPP[a]]))
    fl = lat.fluid.to(DT)
    fR, fB = torch.stack(outR) * fl, torch.stack(outB) * fl
    if lat.inout:
        fR, fB = inlet_outlet(lat, prm, fR, fB)
    return fR, fB


def inlet_outlet(lat, prm, fR, fB):
    """Zou-He boundaries on the fluid nodes of columns 0 (velocity u_in, pure red) and nx-1
    (density rho_out, colour fraction of the known populations).  Directions entering from
    outside: 1, 5, 8 at the inlet; 3, 6, 7 at the outlet."""
    fR = fR.clone()
    fB = fB.clone()
    fl_in = lat.fluid[:, 0]
    fl_out = lat.fluid[:, -1]
    # inlet, x = 0: known 0, 2, 3, 4, 6, 7
    f = fR[:, :, 0] + fB[:, :, 0]
    u = prm.u_in
    if getattr(prm, "inlet_profile", 0):
        # Poiseuille profile of maximum u_in across the inlet column's fluid rows, the walls
        # half a node beyond the first and last of them (Sec. III.D)
        rows = torch.nonzero(fl_in, as_tuple=True)[0]
        y0, w = float(rows.min()) - 0.5, float(rows.max() - rows.min() + 1)
        s = (torch.arange(lat.ny, dtype=DT) - y0) / w
        u = 4 * prm.u_in * s * (1 - s)
    rho = (f[0] + f[2] + f[4] + 2 * (f[3] + f[6] + f[7])) / (1 - u)
    f1 = f[3] + 2.0 / 3.0 * rho * u
    f5 = f[7] - 0.5 * (f[2] - f[4]) + rho * u / 6.0
    f8 = f[6] + 0.5 * (f[2] - f[4]) + rho * u / 6.0
    newR = f.clone()
    newR[1], newR[5], newR[8] = f1, f5, f8
    fR[:, :, 0] = torch.where(fl_in[None, :], newR, fR[:, :, 0])
    fB[:, :, 0] = torch.where(fl_in[None, :], torch.zeros_like(newR), fB[:, :, 0])
    # outlet, x = nx-1: known 0, 1, 2, 4, 5, 8
    fRo, fBo = fR[:, :, -1], fB[:, :, -1]
    f = fRo + fBo
    r = prm.rho_out
    ux = -1 + (f[0] + f[2] + f[4] + 2 * (f[1] + f[5] + f[8])) / r
    f3 = f[1] - 2.0 / 3.0 * r * ux
    f7 = f[5] + 0.5 * (f[2] - f[4]) - r * ux / 6.0
    f6 = f[8] - 0.5 * (f[2] - f[4]) - r * ux / 6.0
    known = (0, 1, 2, 4, 5, 8)
    kR = sum(fRo[a] for a in known)
    kT = sum(f[a] for a in known)
    frac = torch.where(kT != 0, kR / torch.where(kT != 0, kT, torch.ones_like(kT)), torch.zeros_like(kT))
    newR, newB = fRo.clone(), fBo.clone()
    for a, v in ((3, f3), (7, f7), (6, f6)):
        newR[a] = frac * v
        newB[a] = (1 - frac) * v
    fR[:, :, -1] = torch.where(fl_out[None, :], newR, fRo)
    fB[:, :, -1] = torch.where(fl_out[None, :], newB, fBo)
    return fR, fB


# ------------------------------------------------------------------ one step
def step(lat: OracleLattice, prm, fR, fB):
    """One time step in the paper's order: macroscopic fields and interface geometry,
    MRT collision with Guo forcing, recolouring, streaming with bounce-back (and the
    inlet/outlet columns when present)."""
    mac = macroscopic(lat, prm, fR, fB)
    fpost = collide(lat, prm, fR, fB, mac)
    pR, pB = recolour(lat, prm, fpost, mac)
    return stream(lat, prm, pR, pB)


def run(lat, prm, fR, fB, nsteps: int):
    for _ in range(nsteps):
        fR, fB = step(lat, prm, fR, fB)
    return fR, fB
