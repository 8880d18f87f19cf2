"""Pins of the oracle's whole step against invariants the method must keep (conservation,
symmetry, the direction of streaming) and against an independent node-by-node scalar
implementation on tiny lattices."""
import math

import numpy as np
import pytest
import torch

from oracle import lbcg_oracle as O
from paper_1707_00198_gb300 import inputs as I


def _state(geom, prm):
    lat = O.make_lattice(geom, prm.theta)
    fR, fB = O.init_state(lat, geom.rhoN0, prm.rho0, prm)
    return lat, fR, fB


def test_streaming_moves_each_population_along_its_velocity():
    g = I.periodic_box_droplet(8, 7, R=0.0)
    lat, fR, fB = _state(g, I.Params())
    for a in range(9):
        pR = torch.zeros(9, 7, 8, dtype=O.DT)
        pR[a, 3, 4] = 1.0
        oR, _ = O.stream(lat, I.Params(), pR, torch.zeros_like(pR))
        ex, ey = O.E[a]
        assert oR[a, (3 + ey) % 7, (4 + ex) % 8] == 1.0 and oR.sum() == 1.0


def test_half_way_bounce_back_at_a_wall():
    g = I.flat_wall_droplet(8, 6, R=0.0)
    lat, fR, fB = _state(g, I.Params())
    for a in (4, 7, 8):  # populations leaving row 1 towards the bottom wall
        pR = torch.zeros(9, 6, 8, dtype=O.DT)
        pR[a, 1, 3] = 1.0
        oR, _ = O.stream(lat, I.Params(), pR, torch.zeros_like(pR))
        assert oR[O.OPP[a], 1, 3] == 1.0 and oR.sum() == 1.0


@pytest.mark.parametrize("maker", ["flat", "cyl", "cap"])
def test_per_colour_mass_is_conserved(maker):
    if maker == "flat":
        g, p = I.config_static_droplet()
        g = I.flat_wall_droplet(40, 24, R=9.0, noise=1e-3)
    elif maker == "cyl":
        g = I.cylinder_droplet(48, 48, Rs=10.0, cx=24, cy=16, Rd=9.0, theta=math.radians(60), noise=1e-3)
        p = I.Params(theta=math.radians(60))
    else:
        g = I.capillary_filling(L=30, d=8, reservoir=10, wall=4, red_into=8, noise=1e-3)
        p = I.Params(theta=math.radians(30))
    lat, fR, fB = _state(g, p)
    m0 = (fR.sum().item(), fB.sum().item())
    fR, fB = O.run(lat, p, fR, fB, 60)
    assert abs(fR.sum().item() - m0[0]) < 1e-12 * (m0[0] + m0[1])
    assert abs(fB.sum().item() - m0[1]) < 1e-12 * (m0[0] + m0[1])


def test_momentum_changes_by_the_total_force_in_a_periodic_box():
    g = I.periodic_box_droplet(32, 28, R=8.0, noise=1e-3, seed=4)
    p = I.Params(nu_R=0.2, nu_B=0.05, sigma=0.02)
    lat, fR, fB = _state(g, p)
    e = torch.tensor(O.E, dtype=O.DT)
    for _ in range(5):
        fR, fB = O.run(lat, p, fR, fB, 7)
        mac = O.macroscopic(lat, p, fR, fB)
        f = fR + fB
        j0 = torch.einsum("aij,ak->k", f, e)
        f1R, f1B = O.step(lat, p, fR, fB)
        j1 = torch.einsum("aij,ak->k", f1R + f1B, e)
        F = torch.stack([mac["Fx"].sum(), mac["Fy"].sum()])
        assert torch.allclose(j1 - j0, F, atol=1e-15), (j1 - j0, F)


def test_recolouring_splits_the_post_collision_population():
    g = I.flat_wall_droplet(30, 20, R=8.0, noise=1e-3)
    p = I.Params(theta=math.radians(50), sigma=0.03, nu_B=0.05)
    lat, fR, fB = _state(g, p)
    fR, fB = O.run(lat, p, fR, fB, 10)
    mac = O.macroscopic(lat, p, fR, fB)
    fpost = O.collide(lat, p, fR, fB, mac)
    pR, pB = O.recolour(lat, p, fpost, mac)
    fl = lat.fluid
    assert torch.allclose((pR + pB)[:, fl], fpost[:, fl], atol=1e-16)
    assert torch.allclose(pR.sum(0)[fl], mac["rhoR"][fl], atol=1e-15)
    assert torch.allclose(pB.sum(0)[fl], mac["rhoB"][fl], atol=1e-15)
    # collision conserves mass at every node
    assert torch.allclose(fpost.sum(0)[fl], mac["rho"][fl], atol=1e-15)


# ---------------------------------------------------------------------------- symmetries
MIRROR_X = (0, 3, 2, 1, 4, 6, 5, 8, 7)     # e_a -> (-ex, ey)
TRANSPOSE = (0, 2, 1, 4, 3, 5, 8, 7, 6)    # e_a -> (ey, ex)


def _mirror_geom(g, nx):
    return I.Geometry(g.nx, g.ny, g.solid[:, ::-1], g.rhoN0[:, ::-1], bc_x=g.bc_x, bc_y=g.bc_y)


def _unclamped(g, seed):
    # colour field strictly inside (-1, 1) so that no gradient is exactly wall-normal: an exact
    # tie D1 == D2 in Eq. 36 picks (n_f)_1 in both images and breaks the mirror symmetry
    rng = np.random.default_rng(seed)
    r = 0.99 * np.sign(g.rhoN0) + rng.uniform(-1e-3, 1e-3, g.rhoN0.shape)
    r[g.solid != 0] = 0
    return I.Geometry(g.nx, g.ny, g.solid, r, bc_x=g.bc_x, bc_y=g.bc_y)


def test_mirror_symmetry_in_x():
    # a droplet on a wall between two closed side walls and its mirror image evolve as mirror images
    g = _unclamped(I.flat_wall_droplet(30, 18, R=7.0, xc=11.3, noise=0.0, closed_x=True), 5)
    p = I.Params(theta=math.radians(70), sigma=0.02, nu_B=0.08)
    lat, fR, fB = _state(g, p)
    gm = _mirror_geom(g, g.nx)
    latm, mR, mB = _state(gm, p)
    fR, fB = O.run(lat, p, fR, fB, 25)
    mR, mB = O.run(latm, p, mR, mB, 25)
    perm = list(MIRROR_X)
    assert torch.allclose(fR, mR[perm].flip(-1), atol=1e-13)
    assert torch.allclose(fB, mB[perm].flip(-1), atol=1e-13)


def test_transpose_symmetry_with_a_staircase():
    n = 22
    y, x = np.mgrid[0:n, 0:n]
    solid = ((x + 2 * y) < 14).astype(np.uint8)   # a non-symmetric staircase corner
    solid[0, :] = 1
    solid[-1, :] = 1
    solid[:, 0] = 1
    solid[:, -1] = 1
    rng = np.random.default_rng(6)
    rhoN = np.where((x - 12.2) ** 2 + (y - 9.7) ** 2 < 30, 0.99, -0.99) + rng.uniform(-1e-3, 1e-3, (n, n))
    g = I.Geometry(n, n, solid, rhoN, bc_x="closed", bc_y="closed")
    gt = I.Geometry(n, n, solid.T.copy(), rhoN.T.copy(), bc_x="closed", bc_y="closed")
    p = I.Params(theta=math.radians(40), sigma=0.02)
    lat, fR, fB = _state(g, p)
    latt, tR, tB = _state(gt, p)
    # transposition reverses orientation, so it maps rotation by +theta onto rotation by -theta:
    # the selection rule of Eq. 36 is orientation-free, so the runs must still agree
    fR, fB = O.run(lat, p, fR, fB, 20)
    tR, tB = O.run(latt, p, tR, tB, 20)
    perm = list(TRANSPOSE)
    assert torch.allclose(fR, tR[perm].transpose(-1, -2), atol=1e-13)


def test_translation_invariance_in_periodic_x():
    g = I.flat_wall_droplet(26, 14, R=5.0, noise=1e-3, seed=7)
    p = I.Params(theta=math.radians(110), sigma=0.02)
    gs = I.Geometry(g.nx, g.ny, np.roll(g.solid, 9, 1), np.roll(g.rhoN0, 9, 1), bc_x="periodic", bc_y="closed")
    lat, fR, fB = _state(g, p)
    lats, sR, sB = _state(gs, p)
    fR, fB = O.run(lat, p, fR, fB, 15)
    sR, sB = O.run(lats, p, sR, sB, 15)
    assert torch.allclose(torch.roll(fR, 9, -1), sR, atol=1e-14)


# ---------------------------------------------------------------------------- scalar brute force
def _scalar_step(g, p, fR, fB):
    """Node-by-node push-form step written from Eq. 1-18 and 28-36 with explicit loops."""
    nx, ny = g.nx, g.ny
    E, W, OPP = O.E, O.W, O.OPP
    S = g.solid
    px, py = g.bc_x == "periodic", g.bc_y == "periodic"

    def nb(x, y, ex, ey):
        xx, yy = x + ex, y + ey
        if px:
            xx %= nx
        if py:
            yy %= ny
        if 0 <= xx < nx and 0 <= yy < ny:
            return xx, yy
        return None

    def is_fluid(c):
        return c is not None and S[c[1], c[0]] == 0

    rhoR = {}
    rhoB = {}
    rhoN = {}
    for y in range(ny):
        for x in range(nx):
            if S[y, x] == 0:
                rR = sum(fR[a][y][x] for a in range(9))
                rB = sum(fB[a][y][x] for a in range(9))
                rhoR[x, y], rhoB[x, y] = rR, rB
                rhoN[x, y] = (rR - rB) / (rR + rB)

    def value(field, x, y):
        if S[y, x] == 0:
            return field[x, y]
        num = den = 0.0
        for a in range(1, 9):
            c = nb(x, y, *E[a])
            if is_fluid(c):
                num += W[a] * field[c]
                den += W[a]
        return num / den if den > 0 else 0.0

    def grad(field, x, y):
        gx = gy = 0.0
        for a in range(1, 9):
            c = nb(x, y, *E[a])
            v = value(field, *c)
            gx += 3 * W[a] * v * E[a][0]
            gy += 3 * W[a] * v * E[a][1]
        return gx, gy

    # solid normal (Eq. 32-33) with the edge rule of the stencil
    def s_at(x, y):
        if px:
            x %= nx
        elif g.bc_x == "closed" and not 0 <= x < nx:
            return 1.0
        else:
            x = min(max(x, 0), nx - 1)
        if py:
            y %= ny
        elif not 0 <= y < ny:
            return 1.0
        return float(S[y, x])

    wt = {1: 4 / 21, 2: 4 / 45, 4: 1 / 60, 5: 2 / 315, 8: 1 / 5040}
    theta = p.theta
    G = {}
    nrm = {}
    for (x, y) in rhoN:
        gx, gy = grad(rhoN, x, y)
        boundary = any(not is_fluid(nb(x, y, *E[a])) for a in range(1, 9))
        mag = math.hypot(gx, gy)
        if boundary and mag > p.grad_eps:
            vx = vy = 0.0
            for cy in range(-2, 3):
                for cx in range(-2, 3):
                    if cx * cx + cy * cy in wt:
                        s = s_at(x + cx, y + cy)
                        vx += wt[cx * cx + cy * cy] * s * cx
                        vy += wt[cx * cx + cy * cy] * s * cy
            m = math.hypot(vx, vy)
            nsx, nsy = vx / m, vy / m
            ex_, ey_ = gx / mag, gy / mag
            c, s = math.cos(theta), math.sin(theta)
            c1 = (nsx * c - nsy * s, nsx * s + nsy * c)
            c2 = (nsx * c + nsy * s, -nsx * s + nsy * c)
            d1 = math.hypot(c1[0] - ex_, c1[1] - ey_)
            d2 = math.hypot(c2[0] - ex_, c2[1] - ey_)
            nf = c1 if d1 <= d2 else c2
            gx, gy = mag * nf[0], mag * nf[1]
        G[x, y] = (gx, gy)
        m = math.hypot(gx, gy)
        nrm[x, y] = (gx / m, gy / m) if m > p.grad_eps else (0.0, 0.0)
    nX = {k: v[0] for k, v in nrm.items()}
    nY = {k: v[1] for k, v in nrm.items()}
    Minv = np.linalg.inv(np.array(O.M_ROWS, dtype=float))
    Mm = np.array(O.M_ROWS, dtype=float)
    oR = np.zeros((9, ny, nx))
    oB = np.zeros((9, ny, nx))
    for (x, y) in rhoN:
        dnx = grad(nX, x, y)
        dny = grad(nY, x, y)
        n1, n2 = nrm[x, y]
        kap = -n1 * n1 * dny[1] - n2 * n2 * dnx[0] + n1 * n2 * (dnx[1] + dny[0])
        Fx, Fy = 0.5 * p.sigma * kap * G[x, y][0], 0.5 * p.sigma * kap * G[x, y][1]
        f = [fR[a][y][x] + fB[a][y][x] for a in range(9)]
        rho = rhoR[x, y] + rhoB[x, y]
        ux = (sum(f[a] * E[a][0] for a in range(9)) + Fx / 2) / rho
        uy = (sum(f[a] * E[a][1] for a in range(9)) + Fy / 2) / rho
        nu = 1 / ((1 + rhoN[x, y]) / (2 * p.nu_R) + (1 - rhoN[x, y]) / (2 * p.nu_B))
        sv = 1 / (3 * nu + 0.5)
        Sd = np.array([1, p.s_e, p.s_eps, 1, p.s_q, 1, p.s_q, sv, sv])
        feq = np.zeros(9)
        Ft = np.zeros(9)
        for a in range(9):
            eu = E[a][0] * ux + E[a][1] * uy
            feq[a] = rho * W[a] * (1 + 3 * eu + 4.5 * eu * eu - 1.5 * (ux * ux + uy * uy))
            Ft[a] = W[a] * ((3 * (E[a][0] - ux) + 9 * eu * E[a][0]) * Fx + (3 * (E[a][1] - uy) + 9 * eu * E[a][1]) * Fy)
        fpost = np.array(f) - Minv @ (Sd * (Mm @ (np.array(f) - feq))) + Minv @ ((1 - Sd / 2) * (Mm @ Ft))
        for a in range(9):
            pert = p.beta * rhoR[x, y] * rhoB[x, y] / rho * W[a] * (E[a][0] * n1 + E[a][1] * n2)
            vR = rhoR[x, y] / rho * fpost[a] + pert
            vB = rhoB[x, y] / rho * fpost[a] - pert
            c = nb(x, y, *E[a])
            if is_fluid(c):
                oR[a, c[1], c[0]] = vR
                oB[a, c[1], c[0]] = vB
            else:
                oR[OPP[a], y, x] = vR
                oB[OPP[a], y, x] = vB
    return oR, oB


@pytest.mark.parametrize("case", ["periodic", "walls", "corner"])
def test_scalar_brute_force_agrees(case):
    rng = np.random.default_rng(11)
    if case == "periodic":
        g = I.periodic_box_droplet(7, 6, R=2.2, xc=3.3, yc=2.8, noise=1e-2, seed=1)
    elif case == "walls":
        g = I.flat_wall_droplet(9, 8, R=3.1, xc=4.2, noise=1e-2, seed=2)
    else:
        solid = np.zeros((9, 9), np.uint8)
        solid[0] = solid[-1] = 1
        solid[:, 0] = solid[:, -1] = 1
        solid[1:4, 1:3] = 1
        rhoN = np.clip(np.where(np.arange(9)[None, :] < 5, 1.0, -1.0) + rng.uniform(-0.05, 0.05, (9, 9)), -1, 1)
        g = I.Geometry(9, 9, solid, rhoN, bc_x="closed", bc_y="closed")
    p = I.Params(theta=math.radians(63), sigma=0.05, nu_R=0.2, nu_B=0.07)
    lat, fR, fB = _state(g, p)
    # perturb the populations so that velocities and forces are not trivial
    fl = lat.fluid.to(O.DT)
    fR = fR * (1 + 0.05 * torch.from_numpy(rng.uniform(-1, 1, fR.shape))) * fl
    fB = fB * (1 + 0.05 * torch.from_numpy(rng.uniform(-1, 1, fB.shape))) * fl
    for _ in range(3):
        sR, sB = _scalar_step(g, p, fR.numpy(), fB.numpy())
        fR, fB = O.step(lat, p, fR, fB)
        assert np.allclose(fR.numpy(), sR, atol=1e-14, rtol=0)
        assert np.allclose(fB.numpy(), sB, atol=1e-14, rtol=0)


def test_poiseuille_inlet_imposes_the_profile():
    """The Zou-He velocity inlet with the Poiseuille profile (Sec. III.D): on the inlet column
    sum_a e_ax f_a / rho equals 4 u0 s (1 - s), s = (y - y0) / W across the W fluid rows, for any
    incoming populations; its mean over the rows is u0 (2/3 + 1/(3 W^2))."""
    g = I.displacement_channel(W=9, L=12, x_I=5.0, seed=0, noise=1e-2)
    p = I.Params(u_in=0.05, inlet_profile=1)
    lat = O.make_lattice(g, p.theta)
    rng = np.random.default_rng(1)
    fR = torch.tensor(rng.uniform(0.0, 0.2, (9, g.ny, g.nx)))
    fB = torch.tensor(rng.uniform(0.0, 0.2, (9, g.ny, g.nx)))
    fR, fB = O.inlet_outlet(lat, p, fR, fB)
    f = (fR + fB)[:, :, 0]
    ex = torch.tensor([e[0] for e in O.E], dtype=torch.float64)
    u = (ex[:, None] * f).sum(0) / f.sum(0)
    W = 9
    rows = np.arange(1, W + 1)
    s = (rows - 0.5) / W
    want = 4 * p.u_in * s * (1 - s)
    assert np.abs(u.numpy()[rows] - want).max() <= 1e-15
    assert abs(want.mean() - p.u_in * (2 / 3 + 1 / (3 * W * W))) <= 1e-16
    assert float(fB[:, rows, 0].abs().max()) == 0.0   # the inlet carries red only
