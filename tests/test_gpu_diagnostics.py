"""lbcg_diagnostics (Sec. III: E_1 of Eq. 45 and E_NPMT of Eq. 47) against the oracle's
diagnostics on the same states (static droplet, FP64 and FP32 handles)."""
import math

import numpy as np
import pytest
import torch

from oracle import lbcg_oracle as O
from oracle import observables as OB
from paper_1707_00198_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _steady_circle(R0, theta, xc, wall_y=0.5):
    """The equilibrium cap of a semicircle of radius R0 on a wall at contact angle theta (equal
    area): radius R and centre (xc, wall_y - R cos theta)."""
    R = math.sqrt(math.pi * R0 * R0 / 2 / (theta - math.sin(theta) * math.cos(theta)))
    return xc, wall_y - R * math.cos(theta), R


# FP32: masses to rounding of their sums; E_1 is a difference of velocities of order 1e-3 that
# each carry FP32 rounding of order 1e-7
@pytest.mark.parametrize("prec,tol,e1_tol", [("fp64", 1e-11, 1e-11), ("fp32", 2e-5, 1e-3)])
def test_diagnostics_match_the_oracle(prec, tol, e1_tol):
    import __graft_entry__ as ge
    ge.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1707_00198_gb300.lbcg import Lattice
    g, p = I.config_static_droplet()
    circle = _steady_circle(20.0, p.theta, g.nx / 2)
    lat = O.make_lattice(g, p.theta)
    fR, fB = O.init_state(lat, g.rhoN0, p.rho0, p)
    mac0 = O.macroscopic(lat, p, fR, fB)
    fR, fB = O.run(lat, p, fR, fB, 150)
    mac1 = O.macroscopic(lat, p, fR, fB)
    L = Lattice(g, p, prec)
    d0 = L.diagnostics(circle)
    assert d0["prev_step"] == -1 and math.isnan(d0["e1"]) and d0["step"] == 0
    r0 = OB.npmt(lat, mac0, *circle, inside_red=True)
    for k in ("m_R_in", "m_R_out", "m_B_in", "m_B_out", "e_npmt"):
        assert abs(d0[k] - r0[k]) <= tol * max(1.0, abs(r0[k])), (k, d0[k], r0[k])
    L.step(150)
    d1 = L.diagnostics(circle)
    L.close()
    assert d1["prev_step"] == 0 and d1["step"] == 150
    e1 = OB.velocity_change(lat, mac0, mac1)
    assert e1 > 0 and abs(d1["e1"] - e1) <= e1_tol * e1, (d1["e1"], e1)
    r1 = OB.npmt(lat, mac1, *circle, inside_red=True)
    for k in ("m_R_in", "m_R_out", "m_B_in", "m_B_out", "e_npmt"):
        assert abs(d1[k] - r1[k]) <= tol * max(1.0, abs(r1[k])), (k, d1[k], r1[k])
    # the droplet is red: the wrong-side masses are a small fraction
    assert d1["e_npmt"] < 0.2
