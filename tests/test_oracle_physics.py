"""Pins of the oracle against closed forms of the physics it must reproduce: viscous decay
of a shear wave (Eq. 5, 18), Laplace's law (Eq. 10-13), the prescribed contact angle on a
flat wall (Eq. 28-36, Table I) and Lucas-Washburn capillary filling (Eq. 49)."""
import math

import numpy as np
import pytest
import torch

from oracle import lbcg_oracle as O
from oracle import observables as OB
from paper_1707_00198_gb300 import inputs as I


def _shear_amplitude(lat, p, fR, fB, k):
    mac = O.macroscopic(lat, p, fR, fB)
    ux = mac["ux"].mean(1)
    y = torch.arange(lat.ny, dtype=O.DT)
    s = torch.sin(k * y)
    return float((ux * s).sum() / (s * s).sum())


@pytest.mark.parametrize("colour,nu", [("red", 0.1), ("blue", 0.04)])
def test_shear_wave_decays_at_the_fluid_viscosity(colour, nu):
    # u_x(y, t) = U exp(-nu k^2 t) sin(k y): pins tau_v = 3 nu + 1/2 (Eq. 5) and the pure-fluid
    # limits of Eq. 18 (nu_R for rho^N = 1, nu_B for rho^N = -1)
    nx, ny = 4, 32
    g = I.Geometry(nx, ny, np.zeros((ny, nx), np.uint8), np.ones((ny, nx)) * (1 if colour == "red" else -1),
                   bc_x="periodic", bc_y="periodic")
    p = I.Params(nu_R=nu if colour == "red" else 0.3, nu_B=nu if colour == "blue" else 0.3)
    lat = O.make_lattice(g, p.theta)
    k = 2 * math.pi / ny
    y = torch.arange(ny, dtype=O.DT)[:, None].expand(ny, nx)
    feq = O.equilibrium(torch.ones(ny, nx, dtype=O.DT), 0.01 * torch.sin(k * y), torch.zeros(ny, nx, dtype=O.DT))
    fR, fB = (feq, torch.zeros_like(feq)) if colour == "red" else (torch.zeros_like(feq), feq)
    fR, fB = O.run(lat, p, fR, fB, 20)
    a0 = _shear_amplitude(lat, p, fR, fB, k)
    fR, fB = O.run(lat, p, fR, fB, 300)
    a1 = _shear_amplitude(lat, p, fR, fB, k)
    expect = math.exp(-nu * k * k * 300)
    assert abs(a1 / a0 / expect - 1) < 0.01, (a1 / a0, expect)


def test_laplace_law_for_a_free_droplet():
    # 2-D Laplace law: p_in - p_out = sigma / R, averaged over acoustic oscillations
    for R in (8.0, 12.0):
        g = I.periodic_box_droplet(40, 40, R=R)
        p = I.Params(sigma=0.01)
        lat = O.make_lattice(g, p.theta)
        fR, fB = O.init_state(lat, g.rhoN0, p.rho0, p)
        fR, fB = O.run(lat, p, fR, fB, 300)
        dps, Rs = [], []
        for _ in range(40):
            fR, fB = O.run(lat, p, fR, fB, 7)
            o = OB.observables(lat, p, fR, fB)
            dps.append(o["dp_laplace"])
            Rs.append(o["R"])
        ratio = np.mean(dps) * np.mean(Rs) / p.sigma
        assert abs(ratio - 1) < 0.04, (R, ratio)


@pytest.mark.parametrize("theta_deg", [60.0, 120.0])
def test_static_contact_angle_on_a_flat_wall(theta_deg):
    # Sec. III.A: the droplet is initialised as the equilibrium cap (centre at y_w - R cos theta)
    # and must keep the prescribed angle; Table I reports errors below 2 deg at R = 45, the
    # smaller R = 12 here is allowed 3 deg
    R = 12.0
    th = math.radians(theta_deg)
    g = I.flat_wall_droplet(64, 32, R=R, yc=0.5 - R * math.cos(th), noise=1e-3, seed=0)
    p = I.Params(sigma=1e-2, theta=th)
    lat = O.make_lattice(g, p.theta)
    fR, fB = O.init_state(lat, g.rhoN0, p.rho0, p)
    fR, fB = O.run(lat, p, fR, fB, 1000)
    o = OB.observables(lat, p, fR, fB, wall_y=0.5)
    assert abs(o["theta_deg"] - theta_deg) < 3.0, o["theta_deg"]
    # and the wetting sense is right: theta < 90 flattens the cap (centre below the wall)
    assert (o["yc"] < 0.5) == (theta_deg < 90)


def test_capillary_filling_follows_lucas_washburn():
    # Eq. 49 with M = 1: dx/dt = sigma cos(theta) d / (6 mu L); the closed form neglects the
    # reservoirs and the entrance, which slow the meniscus by a few percent
    d, L = 12, 100
    g = I.capillary_filling(L=L, d=d, reservoir=30, wall=4, red_into=20)
    p = I.Params(sigma=0.05, theta=math.radians(30))
    lat = O.make_lattice(g, p.theta)
    fR, fB = O.init_state(lat, g.rhoN0, p.rho0, p)
    fR, fB = O.run(lat, p, fR, fB, 1000)
    ts, xs = [], []
    for k in range(5):
        fR, fB = O.run(lat, p, fR, fB, 250)
        o = OB.observables(lat, p, fR, fB, tip_rows=(g.ny // 2 - 1, g.ny // 2))
        ts.append(1000 + 250 * (k + 1))
        xs.append(o["x_tip"])
    slope = np.polyfit(ts, xs, 1)[0]
    pred = p.sigma * math.cos(p.theta) * d / (6 * p.nu_R * L)
    assert 0.88 < slope / pred < 1.05, slope / pred
