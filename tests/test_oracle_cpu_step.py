"""The plain C/OpenMP CPU step (oracle/lbcg_cpu.c) against the PyTorch oracle: two independent
CPU implementations of the paper's step agree to 1e-12 after 30 steps on every feature --
walls, the E8 and analytic solid normals, per-node contact angles, periodic, closed and open
boundaries with uniform and Poiseuille inlets, the wetting variants -- and give the same result
on one thread and on several."""
import math

import numpy as np
import pytest
import torch

from oracle import cpu_step as CS
from oracle import lbcg_oracle as O
from paper_1707_00198_gb300 import inputs as I


def _cases():
    th = math.radians
    yield "flat_wall_60x30", I.flat_wall_droplet(60, 30, R=10.0, xc=27.3, noise=1e-3, seed=1), \
        I.Params(theta=th(60), sigma=0.02, nu_B=0.08)
    yield "periodic_40x36", I.periodic_box_droplet(40, 36, R=9.0, xc=19.2, yc=17.6, noise=1e-3, seed=2), \
        I.Params(sigma=0.02, nu_R=0.2, nu_B=0.05)
    g = I.flat_wall_droplet(45, 21, R=7.0, xc=20.7, noise=1e-3, seed=3, closed_x=True)
    yield "closed_box_45x21", g, I.Params(theta=th(130), sigma=0.03, nu_R=0.1, nu_B=0.3)
    g = I.cylinder_droplet(60, 50, Rs=10.0, cx=30.0, cy=18.0, Rd=9.0, theta=th(70), noise=1e-3, seed=4)
    yield "cylinder_analytic_60x50", g, I.Params(theta=th(70), sigma=0.02)
    g = I.cylinder_droplet(60, 50, Rs=10.0, cx=30.0, cy=18.0, Rd=9.0, theta=th(110), noise=1e-3, seed=5,
                           analytic_normal=False)
    yield "cylinder_e8_60x50", g, I.Params(theta=th(110), sigma=0.02)
    g = I.displacement_channel(W=16, L=70, x_I=20.0, seed=6, noise=1e-3)
    yield "channel_uniform_70x18", g, I.fingering_params(M=5.0, Ca=0.1, theta_deg=60.0)
    g = I.displacement_channel(W=16, L=70, x_I=20.0, seed=7, noise=1e-3)
    g.rhoN0[4:12, 60:] = 1.0
    yield "channel_poiseuille_70x18", g, I.Params(**{**I.fingering_params(M=3.0, Ca=0.2, theta_deg=120.0).__dict__,
                                                     "u_in": 0.05, "inlet_profile": 1})
    g = I.flat_wall_droplet(45, 21, R=7.0, xc=20.7, noise=1e-3, seed=8)
    g.theta_node = np.random.default_rng(8).uniform(th(40), th(140), size=(g.ny, g.nx))
    yield "per_node_theta_45x21", g, I.Params(sigma=0.02)
    g = I.flat_wall_droplet(45, 21, R=7.0, xc=20.7, noise=1e-3, seed=9, closed_x=True)
    yield "scheme_b_45x21", g, I.Params(theta=th(50), sigma=0.02, wetting=1)
    g = I.flat_wall_droplet(45, 21, R=7.0, xc=20.7, noise=1e-3, seed=10)
    yield "surface_energy_45x21", g, I.Params(theta=th(70), sigma=0.02, wetting=2)
    g = I.capillary_filling(L=40, d=8, reservoir=12, wall=4, red_into=8, noise=1e-3, seed=11)
    yield "capillary_64x16", g, I.Params(theta=th(30), sigma=0.02)


CASES = list(_cases())


@pytest.mark.parametrize("name,g,p", CASES, ids=[c[0] for c in CASES])
def test_c_step_matches_the_pytorch_oracle(name, g, p):
    lat = O.make_lattice(g, p.theta)
    fR, fB = O.init_state(lat, g.rhoN0, p.rho0, p)
    C = CS.CpuLattice(g, p)
    cR, cB = C.init_state()
    assert np.abs(cR - fR.numpy()).max() <= 1e-15 and np.abs(cB - fB.numpy()).max() <= 1e-15
    oR, oB = O.run(lat, p, fR, fB, 30)
    cR, cB = C.run(cR, cB, 30)
    C.close()
    err = max(np.abs(cR - oR.numpy()).max(), np.abs(cB - oB.numpy()).max())
    assert err <= 1e-12, (name, err)


def test_c_step_is_independent_of_the_thread_count():
    g, p = CASES[5][1], CASES[5][2]
    C = CS.CpuLattice(g, p)
    f0 = C.init_state()
    a = C.run(*f0, 10, threads=1)
    b = C.run(*f0, 10, threads=max(2, CS.max_threads()))
    C.close()
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
