"""Parity of the open columns (Sec. III.D: Zou-He velocity inlet carrying red, pressure outlet)
on the benchmarked FP32 and 16-bit paths, element by element over every column of the
lattice -- the inlet and outlet columns included -- against the FP64 oracle.

Cases: displacement channels with a uniform and a Poiseuille inlet, and a channel whose
outlet carries both colours (a red blob leaving through it), so that the outlet's colour
split is exercised.  The longer channels span several 124-column sweep strips, the last of
them ragged, so the outlet falls into a partial strip.  Schedules: the y-sweep kernel with
automatic and with 5-row segments, and the 32 x 8 tile kernel.
"""
import math

import numpy as np
import pytest
import torch

from oracle import lbcg_oracle as O
from oracle import observables as OB
from paper_1707_00198_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as ge
    ge.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def _cases():
    g = I.displacement_channel(W=20, L=110, x_I=25.0, seed=6, noise=1e-3)
    yield "uniform_110x22", g, I.fingering_params(M=5.0, Ca=0.1, theta_deg=60.0)
    g = I.displacement_channel(W=24, L=260, x_I=30.0, seed=31, noise=1e-3)
    yield "poiseuille_260x26", g, I.Params(**{**I.fingering_params(M=3.0, Ca=0.2, theta_deg=120.0).__dict__,
                                              "u_in": 0.05, "inlet_profile": 1})
    g = I.displacement_channel(W=20, L=250, x_I=20.0, seed=21, noise=1e-3)
    g.rhoN0[6:16, 238:] = 1.0          # red leaving through the outlet: both colours there
    yield "outlet_two_colour_250x22", g, I.fingering_params(M=0.5, Ca=0.05, theta_deg=80.0)


CASES = list(_cases())
SCHEDULES = [("sweep", None, 0), ("sweep5", None, 5), ("tiles8", 8, None)]


def _oracle(g, p, n, state=None):
    lat = O.make_lattice(g, p.theta)
    if state is None:
        fR, fB = O.init_state(lat, g.rhoN0, p.rho0, p)
    else:
        fR, fB = torch.from_numpy(state[0].copy()), torch.from_numpy(state[1].copy())
    fR, fB = O.run(lat, p, fR, fB, n)
    return lat, np.stack([fR.numpy(), fB.numpy()])


def _gpu(g, p, n, prec, ty=None, rows=None, state=None):
    from paper_1707_00198_gb300.lbcg import Lattice
    L = Lattice(g, p, prec)
    if ty:
        L.set_tile(ty)
    if rows is not None:
        L.set_sweep(rows)
    if state is not None:
        L.set_populations(state)
    L.step(n)
    out = L.populations()
    L.close()
    return out


def _edge_and_all(got, ref):
    err = np.abs(got - ref)
    return float(err.max()), float(max(err[..., 0].max(), err[..., -1].max()))


_CONDITIONING = {}


def _fp32_conditioning(g, p, n):
    """How far the FP64 oracle itself moves in n steps when its initial populations are
    perturbed by half an FP32 ulp (relative 2^-24, random signs): the spread that FP32 rounding
    alone must be allowed to cause.  On channels with noisy initial fields it is far above the
    droplet's: the choice between the two rotated normals of Eq. 36 (D1 <= D2) is
    discontinuous, and on outermost fluid nodes where the noisy gradient is nearly equidistant
    from both, a rounding-level change picks the other candidate and changes n there by O(1)."""
    if (g.name, n) in _CONDITIONING:
        return _CONDITIONING[(g.name, n)]
    lat = O.make_lattice(g, p.theta)
    fR, fB = O.init_state(lat, g.rhoN0, p.rho0, p)
    rng = np.random.default_rng(0)
    sR = torch.from_numpy(rng.choice([-1.0, 1.0], size=tuple(fR.shape)))
    sB = torch.from_numpy(rng.choice([-1.0, 1.0], size=tuple(fB.shape)))
    aR, aB = O.run(lat, p, fR, fB, n)
    bR, bB = O.run(lat, p, fR * (1 + 2.0 ** -24 * sR), fB * (1 + 2.0 ** -24 * sB), n)
    _CONDITIONING[(g.name, n)] = max(float((aR - bR).abs().max()), float((aB - bB).abs().max()))
    return _CONDITIONING[(g.name, n)]


@pytest.mark.parametrize("kind,ty,rows", SCHEDULES, ids=[s[0] for s in SCHEDULES])
@pytest.mark.parametrize("name,g,p", CASES, ids=[c[0] for c in CASES])
def test_fp32_open_columns_one_step_and_100_steps(name, g, p, kind, ty, rows):
    """FP32 one step from the oracle's state at step 50 within 2e-6 of the oracle's step at
    every node of every column; and 100 steps from the initial state within 5e-5 or, where the
    problem amplifies rounding more (see _fp32_conditioning), within twice the oracle's own
    spread under FP32-level perturbations of its initial state."""
    _, s50 = _oracle(g, p, 50)
    _, ref1 = _oracle(g, p, 1, state=s50)
    got1 = _gpu(g, p, 1, "fp32", ty, rows, state=s50)
    err1, edge1 = _edge_and_all(got1, ref1)
    assert err1 <= 2e-6, (name, kind, err1, edge1)
    _, ref = _oracle(g, p, 100)
    got = _gpu(g, p, 100, "fp32", ty, rows)
    err, edge = _edge_and_all(got, ref)
    tol = max(5e-5, 2 * _fp32_conditioning(g, p, 100))
    assert err <= tol, (name, kind, err, edge, tol)
    assert edge <= 5e-5, (name, kind, edge)      # the open columns themselves stay tight


# one step from a common state: within four half-ulps at 4/9 (see the derivation beside the
# same bound in test_gpu_parity.py); on the open columns the unknown populations are formed
# from the stored known ones, whose errors the Zou-He sums carry with weights of order one
STORE16 = [("fp16", 4 * 2.0 ** -13), ("bf16", 4 * 2.0 ** -10)]


@pytest.mark.parametrize("prec,tol", STORE16, ids=[s[0] for s in STORE16])
@pytest.mark.parametrize("kind,ty,rows", [SCHEDULES[0], SCHEDULES[2]], ids=["sweep", "tiles8"])
@pytest.mark.parametrize("name,g,p", CASES, ids=[c[0] for c in CASES])
def test_16bit_open_columns_one_step(name, g, p, kind, ty, rows, prec, tol):
    _, s50 = _oracle(g, p, 50)
    _, ref1 = _oracle(g, p, 1, state=s50)
    got1 = _gpu(g, p, 1, prec, ty, rows, state=s50)
    err1, edge1 = _edge_and_all(got1, ref1)
    assert err1 <= tol, (name, kind, prec, err1, edge1, tol)


@pytest.mark.parametrize("name,g,p", CASES[:2], ids=[c[0] for c in CASES[:2]])
def test_fp64_finger_tip_and_contact_line_match_oracle(name, g, p):
    """The finger tip x_tip, the contact line x_cl and the finger length x_tip - x_cl of
    Sec. III.D, measured by the GPU reductions on a channel, equal the oracle's measurement of
    the oracle's state to 1e-9, at two times."""
    from paper_1707_00198_gb300.lbcg import Lattice
    L = Lattice(g, p, "fp64")
    lat = O.make_lattice(g, p.theta)
    fR, fB = O.init_state(lat, g.rhoN0, p.rho0, p)
    done = 0
    for n in (100, 300):
        L.step(n - done)
        fR, fB = O.run(lat, p, fR, fB, n - done)
        done = n
        o = L.observables()
        ref = OB.observables(lat, p, fR, fB)
        assert ref["x_tip"] > 0 and ref["x_cl"] > 0
        for k in ("x_tip", "x_cl", "mass_R", "mass_B", "umax"):
            assert abs(o[k] - ref[k]) <= 1e-9 * max(1.0, abs(ref[k])), (name, n, k, o[k], ref[k])
        assert abs((o["x_tip"] - o["x_cl"]) - (ref["x_tip"] - ref["x_cl"])) <= 1e-9
    L.close()
