"""Pins of the oracle's constants and per-node algebra against what the paper prints and
what the mathematics fixes (Eq. 3-9, 13, 28-36)."""
import json
import math
import os

import numpy as np
import pytest
import torch

from oracle import lbcg_oracle as O

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def test_lattice_constants_match_paper():
    assert [list(e) for e in O.E] == GOLD["d2q9_velocities"]["value"]
    assert np.allclose(O.W, GOLD["d2q9_weights"]["value"], rtol=0, atol=1e-16)
    assert abs(O.CS2 - 1 / 3) < 1e-16
    for a in range(9):
        assert O.E[O.OPP[a]] == (-O.E[a][0], -O.E[a][1])


def test_lattice_moments_isotropy():
    # sum w = 1, sum w e = 0, sum w e_i e_j = c_s^2 delta_ij, fourth moments of D2Q9
    w = np.array(O.W)
    e = np.array(O.E, dtype=float)
    assert abs(w.sum() - 1) < 1e-15
    assert np.allclose(w @ e, 0, atol=1e-16)
    assert np.allclose(np.einsum("a,ai,aj->ij", w, e, e), np.eye(2) / 3, atol=1e-16)
    assert abs(np.sum(w * e[:, 0] ** 4) - 1 / 3) < 1e-15 and abs(np.sum(w * e[:, 0] ** 2 * e[:, 1] ** 2) - 1 / 9) < 1e-15


def test_mrt_rows_and_inverse_closed_form():
    M = O.mrt_matrix().numpy()
    assert M[:8].tolist() == GOLD["mrt_matrix_rows_1_to_8"]["value"]
    # the printed ninth row is not orthogonal to row 1, which is why it is read as e_x e_y
    printed = np.array(GOLD["mrt_matrix_row_9_printed"]["value"], dtype=float)
    assert abs(printed @ M[0]) == 2.0
    assert np.allclose(M[8], [e[0] * e[1] for e in O.E])
    # orthogonal rows: M^-1 = M^T diag(1/|row|^2), the textbook closed form
    D = np.diag([1 / 9, 1 / 36, 1 / 36, 1 / 6, 1 / 12, 1 / 6, 1 / 12, 1 / 4, 1 / 4])
    assert np.allclose(O.mrt_inverse().numpy(), M.T @ D, atol=1e-14)
    assert np.allclose(M @ M.T, np.linalg.inv(D), atol=1e-12)


def test_equilibrium_moments_closed_form():
    # M f^eq = rho (1, -2+3u^2, 1-3u^2, ux, -ux, uy, -uy, ux^2-uy^2, ux uy) for Eq. 7
    g = torch.Generator().manual_seed(1)
    rho = 0.8 + 0.4 * torch.rand(5, 7, generator=g, dtype=O.DT)
    ux = 0.1 * (torch.rand(5, 7, generator=g, dtype=O.DT) - 0.5)
    uy = 0.1 * (torch.rand(5, 7, generator=g, dtype=O.DT) - 0.5)
    m = torch.einsum("ab,bij->aij", O.mrt_matrix(), O.equilibrium(rho, ux, uy))
    u2 = ux * ux + uy * uy
    ref = torch.stack([rho, rho * (-2 + 3 * u2), rho * (1 - 3 * u2), rho * ux, -rho * ux, rho * uy, -rho * uy,
                       rho * (ux * ux - uy * uy), rho * ux * uy])
    assert torch.allclose(m, ref, atol=1e-14)


def test_guo_source_moments():
    # Guo's scheme: sum F~ = 0, sum F~ e = F, sum F~ e e = u F + F u
    g = torch.Generator().manual_seed(2)
    sh = (4, 6)
    ux, uy, Fx, Fy = [0.05 * (torch.rand(sh, generator=g, dtype=O.DT) - 0.5) for _ in range(4)]
    S = O.guo_source(ux, uy, Fx, Fy)
    e = torch.tensor(O.E, dtype=O.DT)
    assert torch.allclose(S.sum(0), torch.zeros(sh, dtype=O.DT), atol=1e-17)
    assert torch.allclose(torch.einsum("aij,a->ij", S, e[:, 0]), Fx, atol=1e-16)
    assert torch.allclose(torch.einsum("aij,a->ij", S, e[:, 1]), Fy, atol=1e-16)
    assert torch.allclose(torch.einsum("aij,a->ij", S, e[:, 0] * e[:, 0]), 2 * ux * Fx, atol=1e-16)
    assert torch.allclose(torch.einsum("aij,a->ij", S, e[:, 0] * e[:, 1]), ux * Fy + uy * Fx, atol=1e-16)


def test_relaxation_rates_eq6_and_viscosity():
    class P:  # noqa: D401 - plain holder
        nu_R, nu_B, s_e, s_eps, s_q = 0.35, 0.0035, 1.64, 1.54, 1.9
    rhoN = torch.tensor([[1.0, -1.0, 0.0]], dtype=O.DT)
    S = O.relaxation_rates(P, rhoN)
    assert np.allclose(S[:7, 0, 0].numpy(), GOLD["relaxation_rates_fixed"]["value"])
    # pure red: tau = 3 nu_R + 1/2; pure blue: 3 nu_B + 1/2; mixed: harmonic mean (Eq. 18)
    assert abs(1 / S[7, 0, 0].item() - (3 * 0.35 + 0.5)) < 1e-14
    assert abs(1 / S[7, 0, 1].item() - (3 * 0.0035 + 0.5)) < 1e-14
    nu_mid = 1 / (0.5 / 0.35 + 0.5 / 0.0035)
    assert abs(1 / S[8, 0, 2].item() - (3 * nu_mid + 0.5)) < 1e-14


def _lat(nx, ny, solid=None, bc_x="periodic", bc_y="periodic", theta=math.pi / 2):
    from paper_1707_00198_gb300.inputs import Geometry
    s = np.zeros((ny, nx), np.uint8) if solid is None else solid
    g = Geometry(nx, ny, s, np.zeros((ny, nx)), bc_x=bc_x, bc_y=bc_y)
    return O.make_lattice(g, theta)


def test_isotropic_gradient_exact_on_quadratics():
    # Eq. 28 is exact for polynomials up to degree 2
    lat = _lat(12, 10)
    y, x = torch.meshgrid(torch.arange(10, dtype=O.DT), torch.arange(12, dtype=O.DT), indexing="ij")
    phi = 0.3 * x - 0.7 * y + 0.05 * x * x + 0.02 * x * y - 0.03 * y * y
    gx, gy = O.iso_gradient(lat, phi)
    inner = (slice(1, -1), slice(1, -1))
    assert torch.allclose(gx[inner], (0.3 + 0.1 * x + 0.02 * y)[inner], atol=1e-13)
    assert torch.allclose(gy[inner], (-0.7 + 0.02 * x - 0.06 * y)[inner], atol=1e-13)


def test_virtual_fill_weights_flat_wall():
    # Eq. 29 at a bottom-wall solid node: alpha_1 = {6, 2, 5} with weights 1/36, 1/9, 1/36.
    solid = np.zeros((6, 10), np.uint8)
    solid[0] = 1
    solid[-1] = 1
    lat = _lat(10, 6, solid=solid, bc_y="closed")
    y, x = torch.meshgrid(torch.arange(6, dtype=O.DT), torch.arange(10, dtype=O.DT), indexing="ij")
    # linear along the wall: the virtual value equals the value one row up (d_n phi = 0, Eq. 42)
    v = O.virtual_fill(lat, torch.where(lat.fluid, 0.4 * x + 0.1 * y, 0.0))
    assert torch.allclose(v[0, 2:8], (0.4 * x + 0.1)[0, 2:8], atol=1e-14)
    # quadratic along the wall distinguishes the weights: mean over x-1, x, x+1 with (1,4,1)/6
    v = O.virtual_fill(lat, torch.where(lat.fluid, x * x, 0.0))
    assert torch.allclose(v[0, 2:8], (x * x + 1 / 3)[0, 2:8], atol=1e-13)
    # interior solid nodes (none here) and fluid nodes are untouched
    assert torch.allclose(v[1:-1], (x * x)[1:-1])


def test_e8_stencil_weights_and_isotropy():
    st = O.e8_stencil()
    assert len(st) == 24
    gold = {int(k): v for k, v in GOLD["e8_weights"]["value"].items()}
    for cx, cy, w in st:
        assert abs(w - gold[cx * cx + cy * cy]) < 1e-17
    c = np.array([(cx, cy) for cx, cy, _ in st], dtype=float)
    w = np.array([w for *_, w in st])
    assert abs(np.sum(w * c[:, 0] ** 2) - 1) < 1e-15 and abs(np.sum(w * c[:, 0] * c[:, 1])) < 1e-16
    # isotropic fourth moment: sum w cx^4 = 3 sum w cx^2 cy^2
    assert abs(np.sum(w * c[:, 0] ** 4) - 3 * np.sum(w * c[:, 0] ** 2 * c[:, 1] ** 2)) < 1e-15


def test_e8_normal_flat_walls_and_diagonal():
    # flat bottom and top walls: n_s = (0, -1) and (0, +1) exactly (pointing into the solid)
    solid = np.zeros((8, 9), np.uint8)
    solid[0] = 1
    solid[-1] = 1
    lat = _lat(9, 8, solid=solid, bc_y="closed")
    assert torch.allclose(lat.n_s[:, 1, :], torch.tensor([[0.0], [-1.0]], dtype=O.DT).expand(2, 9))
    assert torch.allclose(lat.n_s[:, 6, :], torch.tensor([[0.0], [1.0]], dtype=O.DT).expand(2, 9))
    # a 45-degree staircase (solid where y <= x - 3 in a periodic-free box): normal along (1,-1)/sqrt2
    n = 24
    y, x = np.mgrid[0:n, 0:n]
    solid = (y - x <= -3).astype(np.uint8)
    solid[0, :] = 1
    solid[-1, :] = 1
    solid[:, 0] = 1
    solid[:, -1] = 1
    lat = _lat(n, n, solid=solid, bc_x="closed", bc_y="closed")
    for k in range(8, 14):  # nodes on the staircase far from the box walls
        xx, yy = k, k - 2
        assert bool(lat.omega_fb[yy, xx])
        v = lat.n_s[:, yy, xx].numpy()
        assert np.allclose(v, [1 / math.sqrt(2), -1 / math.sqrt(2)], atol=1e-12), v


def test_contact_angle_rotation_and_selection():
    # |n_f| = 1, n_f . n_s = cos(theta); the chosen candidate is the one nearer to the estimate
    g = np.random.default_rng(3)
    solid = np.zeros((5, 5), np.uint8)
    solid[0] = 1
    solid[-1] = 1
    lat = _lat(5, 5, solid=solid, bc_y="closed")
    for _ in range(20):
        th = g.uniform(0.1, math.pi - 0.1)
        lat.theta = torch.full((5, 5), th, dtype=O.DT)
        phi = g.uniform(0, 2 * math.pi)
        mag = g.uniform(0.01, 1.0)
        gx = torch.full((5, 5), mag * math.cos(phi), dtype=O.DT)
        gy = torch.full((5, 5), mag * math.sin(phi), dtype=O.DT)
        cx, cy = O.wetting_correction(lat, gx, gy, 1e-12)
        v = np.array([cx[1, 2].item(), cy[1, 2].item()]) / mag
        ns = np.array([0.0, -1.0])
        assert abs(np.linalg.norm(v) - 1) < 1e-13
        assert abs(v @ ns - math.cos(th)) < 1e-13
        # the other candidate, mirrored about n_s, is never nearer to the estimate
        other = np.array([-v[0], v[1]])
        est = np.array([math.cos(phi), math.sin(phi)])
        assert np.linalg.norm(v - est) <= np.linalg.norm(other - est) + 1e-13
        # non-boundary nodes keep the raw gradient
        assert abs(cx[2, 2].item() - gx[2, 2].item()) < 1e-16


def test_contact_line_direction_bottom_wall():
    # right contact line of a red droplet on a bottom wall: grad rho^N ~ (-sin th, -cos th),
    # which is the clockwise candidate (n_f)_2 of Eq. 34
    solid = np.zeros((5, 5), np.uint8)
    solid[0] = 1
    solid[-1] = 1
    lat = _lat(5, 5, solid=solid, bc_y="closed", theta=math.radians(60))
    est = torch.tensor([-math.sin(math.radians(50)), -math.cos(math.radians(50))], dtype=O.DT)
    cx, cy = O.wetting_correction(lat, est[0].expand(5, 5).clone(), est[1].expand(5, 5).clone(), 1e-12)
    assert abs(cx[1, 1].item() + math.sin(math.radians(60))) < 1e-14
    assert abs(cy[1, 1].item() + math.cos(math.radians(60))) < 1e-14


def test_curvature_sign_and_size_on_a_circle():
    # a smooth red disc: n points inward, kappa = 1/R at the interface, F points into red
    n, R = 64, 14.0
    lat = _lat(n, n)
    y, x = torch.meshgrid(torch.arange(n, dtype=O.DT), torch.arange(n, dtype=O.DT), indexing="ij")
    r = torch.sqrt((x - 32.3) ** 2 + (y - 31.6) ** 2)
    rhoN = torch.tanh((R - r) / 2.0)
    gx, gy = O.iso_gradient(lat, O.virtual_fill(lat, rhoN))
    nx_, ny_ = O.unit_normal(gx, gy, 1e-12)
    dnx = O.iso_gradient(lat, nx_)
    dny = O.iso_gradient(lat, ny_)
    kappa = -nx_ * nx_ * dny[1] - ny_ * ny_ * dnx[0] + nx_ * ny_ * (dnx[1] + dny[0])
    band = (r > R - 0.5) & (r < R + 0.5)
    k = kappa[band]
    assert abs(k.mean().item() * R - 1) < 0.02, k.mean().item() * R
    # n . (x - c) < 0 (inward, into the red disc)
    assert bool(((nx_ * (x - 32.3) + ny_ * (y - 31.6))[band] < 0).all())


def test_one_sided_gradient_of_scheme_b_is_exact_on_linear_fields():
    """Eq. 48 as read (each component normalised by sum w e_i^2 over the fluid directions):
    exact for phi = a x + b y next to a wall, where only fluid directions count, and in the bulk."""
    import math
    from paper_1707_00198_gb300 import inputs as I
    g = I.flat_wall_droplet(14, 9, R=3.0, noise=0.0)
    lat = O.make_lattice(g, math.radians(60))
    y, x = torch.meshgrid(torch.arange(g.ny, dtype=O.DT), torch.arange(g.nx, dtype=O.DT), indexing="ij")
    phi = 0.37 * x - 1.3 * y
    gx, gy = O.one_sided_gradient(lat, phi)
    # interior columns (periodic x wraps, so skip the two edge columns)
    sel = lat.fluid.clone()
    sel[:, 0] = False
    sel[:, -1] = False
    assert float((gx[sel] - 0.37).abs().max()) < 1e-13
    assert float((gy[sel] + 1.3).abs().max()) < 1e-13


def test_surface_energy_wall_gradient_closed_form():
    """Surface-energy variant: rho^N = c on the fluid above a flat bottom wall, cos(theta) on the
    solid row; on the first fluid row Eq. 28 gives d_y rho^N = (c - cos theta)/2, d_x = 0."""
    import math
    from paper_1707_00198_gb300 import inputs as I
    g = I.flat_wall_droplet(16, 10, R=3.0, noise=0.0)
    g.rhoN0[:] = 0.3
    theta = math.radians(50)
    p = I.Params(theta=theta, wetting=2)
    lat = O.make_lattice(g, theta)
    fR, fB = O.init_state(lat, g.rhoN0, p.rho0, p)
    d = O.interface_fields(lat, p, fR, fB)
    row = d["gy"][1]
    assert float((row - (0.3 - math.cos(theta)) / 2).abs().max()) < 1e-14
    assert float(d["gx"][1].abs().max()) < 1e-14
