"""Pins of the oracle's open columns (Sec. III.D: velocity inlet, pressure outlet; Zou-He).

What fixes them, independently of how ``inlet_outlet`` computes its unknown populations:

* the inlet's defining moments: at every fluid node of column 0 the populations carry the
  prescribed velocity, sum_a e_ax f_a = u_in sum_a f_a and sum_a e_ay f_a = 0, and (reading r13)
  only red;
* the outlet's defining moments: sum_a f_a = rho_out and sum_a e_ay f_a = 0, and (reading r13)
  the three unknown populations carry the red fraction of the six known ones;
* the known populations of both columns pass through unchanged (in total), and applying the
  conditions to a state that already satisfies them changes nothing (reading r22);
* an exact discrete mass balance of one whole step: the populations that leave through the
  open columns and those the conditions create account for every change of the total, red
  and blue masses.
"""
import copy
import math

import numpy as np
import pytest
import torch

from oracle import lbcg_oracle as O
from paper_1707_00198_gb300 import inputs as I

EX = torch.tensor([e[0] for e in O.E], dtype=O.DT)[:, None]
EY = torch.tensor([e[1] for e in O.E], dtype=O.DT)[:, None]
IN_UNKNOWN = (1, 5, 8)     # populations entering column 0 from outside
OUT_UNKNOWN = (3, 6, 7)    # populations entering column nx-1 from outside
IN_KNOWN = (0, 2, 3, 4, 6, 7)
OUT_KNOWN = (0, 1, 2, 4, 5, 8)


def _channel(seed=3, W=12, L=30, x_I=9.0, noise=1e-3, **kw):
    g = I.displacement_channel(W=W, L=L, x_I=x_I, seed=seed, noise=noise)
    p = I.Params(**{**I.fingering_params(M=4.0, Ca=0.1, theta_deg=70.0, u_in=0.02).__dict__, **kw})
    lat = O.make_lattice(g, p.theta)
    return g, p, lat


def _random_two_colour_state(lat, seed):
    """Positive populations of both colours near rest, everywhere on the fluid nodes."""
    rng = np.random.default_rng(seed)
    w = torch.tensor(O.W, dtype=O.DT)[:, None, None]
    frac = torch.from_numpy(rng.uniform(0.05, 0.95, (lat.ny, lat.nx)))
    pert = torch.from_numpy(rng.uniform(-0.2, 0.2, (9, lat.ny, lat.nx)))
    f = w * (1 + pert)
    fl = lat.fluid.to(O.DT)
    return f * frac * fl, f * (1 - frac) * fl


def _no_open_columns(lat):
    lat2 = copy.copy(lat)
    lat2.inout = False
    return lat2


@pytest.mark.parametrize("profile", [0, 1], ids=["uniform", "poiseuille"])
def test_inlet_imposes_its_velocity_and_colour(profile):
    g, p, lat = _channel(u_in=0.03, inlet_profile=profile)
    fR, fB = _random_two_colour_state(lat, 1)
    oR, oB = O.inlet_outlet(lat, p, fR, fB)
    rows = torch.nonzero(lat.fluid[:, 0], as_tuple=True)[0]
    f = (oR + oB)[:, rows, 0]
    rho = f.sum(0)
    if profile:
        y0, w = float(rows.min()) - 0.5, float(rows.max() - rows.min() + 1)
        s = (rows.to(O.DT) - y0) / w
        u = 4 * p.u_in * s * (1 - s)      # Sec. III.D: maximum u_in, zero half a node beyond
    else:
        u = torch.full_like(rho, p.u_in)
    assert torch.allclose((EX * f).sum(0), u * rho, rtol=0, atol=1e-15)
    assert float((EY * f).sum(0).abs().max()) <= 1e-15
    assert float(oB[:, rows, 0].abs().max()) == 0.0
    # the known populations keep their totals (only their colour changes)
    for a in IN_KNOWN:
        assert torch.allclose(oR[a, rows, 0], fR[a, rows, 0] + fB[a, rows, 0], rtol=0, atol=1e-16)
    # nothing but the two open columns changes
    assert torch.equal(oR[:, :, 1:-1], fR[:, :, 1:-1]) and torch.equal(oB[:, :, 1:-1], fB[:, :, 1:-1])


def test_outlet_imposes_its_density_and_the_known_colour_fraction():
    g, p, lat = _channel(rho_out=0.97)
    fR, fB = _random_two_colour_state(lat, 2)
    oR, oB = O.inlet_outlet(lat, p, fR, fB)
    rows = torch.nonzero(lat.fluid[:, -1], as_tuple=True)[0]
    f = (oR + oB)[:, rows, -1]
    assert float((f.sum(0) - p.rho_out).abs().max()) <= 1e-15
    assert float((EY * f).sum(0).abs().max()) <= 1e-15
    kR = sum(fR[a, rows, -1] for a in OUT_KNOWN)
    kT = sum(fR[a, rows, -1] + fB[a, rows, -1] for a in OUT_KNOWN)
    for a in OUT_UNKNOWN:
        tot = oR[a, rows, -1] + oB[a, rows, -1]
        assert torch.allclose(oR[a, rows, -1], kR / kT * tot, rtol=1e-15, atol=1e-17)
    for a in OUT_KNOWN:
        assert torch.equal(oR[a, rows, -1], fR[a, rows, -1]) and torch.equal(oB[a, rows, -1], fB[a, rows, -1])


def test_open_columns_are_idempotent():
    for profile in (0, 1):
        g, p, lat = _channel(inlet_profile=profile, rho_out=1.01)
        fR, fB = _random_two_colour_state(lat, 3)
        aR, aB = O.inlet_outlet(lat, p, fR, fB)
        bR, bB = O.inlet_outlet(lat, p, aR, aB)
        assert float((bR - aR).abs().max()) <= 1e-16 and float((bB - aB).abs().max()) <= 1e-16


def _one_step_parts(lat, p, fR, fB):
    mac = O.macroscopic(lat, p, fR, fB)
    pR, pB = O.recolour(lat, p, O.collide(lat, p, fR, fB, mac), mac)     # f'' of Eq. 14
    nR, nB = O.stream(lat, p, pR, pB)                                      # next state
    sR, sB = O.stream(_no_open_columns(lat), p, pR, pB)                    # streamed, before Zou-He
    return pR, pB, nR, nB, sR, sB


def _cols(f, col, dirs):
    return sum(float(f[a, :, col].sum()) for a in dirs)


@pytest.mark.parametrize("profile", [0, 1], ids=["uniform", "poiseuille"])
def test_mass_balance_through_the_open_columns(profile):
    """One step changes each mass only through the open columns.  Per node the collision
    keeps rho and the recolouring keeps rho_R and rho_B (Eq. 1-9, 14), so sum f'' = M(t).
    Streaming (Eq. 15) with half-way bounce-back puts every f''_a(x) into exactly one slot of
    the next state, except f''_{3,6,7} of column 0 and f''_{1,5,8} of column nx-1, which
    leave the lattice (or bounce into a slot the conditions overwrite).  The conditions then
    fill the unknown slots (1, 5, 8 at the inlet; 3, 6, 7 at the outlet) and, at the inlet,
    turn the blue of the known slots into red.  Hence, with IN the unknown slots of the new
    state and OUT the leaving f'':
        M(t+1)   = M(t)   + IN   - OUT,
        M_B(t+1) = M_B(t) + IN_B - OUT_B - C,
    C the blue in the inlet column's known slots after streaming; M_R follows as M - M_B."""
    g, p, lat = _channel(inlet_profile=profile, x_I=6.0)
    fR, fB = O.init_state(lat, g.rhoN0, p.rho0, p)
    fR, fB = O.run(lat, p, fR, fB, 25)
    for _ in range(3):
        pR, pB, nR, nB, sR, sB = _one_step_parts(lat, p, fR, fB)
        M0, MB0 = float((fR + fB).sum()), float(fB.sum())
        IN = _cols(nR + nB, 0, IN_UNKNOWN) + _cols(nR + nB, -1, OUT_UNKNOWN)
        OUT = _cols(pR + pB, 0, OUT_UNKNOWN) + _cols(pR + pB, -1, IN_UNKNOWN)
        IN_B = _cols(nB, -1, OUT_UNKNOWN)
        OUT_B = _cols(pB, 0, OUT_UNKNOWN) + _cols(pB, -1, IN_UNKNOWN)
        C = _cols(sB, 0, IN_KNOWN)
        M1, MB1 = float((nR + nB).sum()), float(nB.sum())
        assert abs((M1 - M0) - (IN - OUT)) <= 1e-13 * M0
        assert abs((MB1 - MB0) - (IN_B - OUT_B - C)) <= 1e-13 * M0
        assert abs((M1 - MB1) - (M0 - MB0) - (IN - IN_B - (OUT - OUT_B) + C)) <= 1e-13 * M0
        assert IN > 0 and OUT > 0
        fR, fB = nR, nB


def test_red_enters_only_through_the_inlet_of_a_pure_red_column():
    """With a sharp initial field (no noise) the inlet region stays pure red for the first
    steps, so nothing is recoloured there and the red mass grows by exactly the red the
    inlet's unknown populations bring in minus what leaves through column 0; the outlet,
    pure blue, exchanges no red.  Later, once the start-up pressure waves have passed, the red
    mass grows at the inlet's mass flux sum_y rho(0, y) u_in (the momentum the inlet imposes)
    while the red has not reached the outlet: within 1 % over 200 steps."""
    g, p, lat = _channel(x_I=15.0, noise=0.0, L=40)
    fR, fB = O.init_state(lat, g.rhoN0, p.rho0, p)
    for _ in range(6):
        pR, pB, nR, nB, sR, sB = _one_step_parts(lat, p, fR, fB)
        assert _cols(sB, 0, IN_KNOWN) == 0.0 and _cols(nR, -1, OUT_UNKNOWN) == 0.0
        dMR = float(nR.sum() - fR.sum())
        expect = _cols(nR, 0, IN_UNKNOWN) - _cols(pR, 0, OUT_UNKNOWN) - _cols(pR, -1, IN_UNKNOWN)
        assert abs(dMR - expect) <= 1e-13 * float(fR.sum())
        fR, fB = nR, nB
    fR, fB = O.run(lat, p, fR, fB, 94)
    rows = torch.nonzero(lat.fluid[:, 0], as_tuple=True)[0]
    m0, flux = float(fR.sum()), 0.0
    for _ in range(200):
        flux += float(((fR + fB)[:, rows, 0].sum(0) * p.u_in).sum())
        fR, fB = O.step(lat, p, fR, fB)
    assert float(fR[:, :, -1].sum()) <= 1e-9            # no red at the outlet yet
    assert abs((float(fR.sum()) - m0) / flux - 1.0) <= 0.01
