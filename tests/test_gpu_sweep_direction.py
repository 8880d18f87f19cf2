"""The FP32-arithmetic y-sweep walks every other row segment of a strip downwards (mirrored
stencil rows).  The per-node arithmetic of a step does not depend on the order in which the
rows are visited, so any segment height must give the same bits: one segment per strip (all
upwards), and short segments of odd and even heights whose directions alternate, on a channel
with walls and Zou-He columns, on a y-periodic droplet (segments that wrap) and on a cylinder
(curved wall, Eq. 30-36 on slanted normals).  16-bit storage rounds stochastically with keys of
(node, step), so its bits must not depend on the order either."""
import math

import numpy as np
import pytest
import torch

from paper_1707_00198_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as ge
    ge.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def _cases():
    yield "channel_110x22", I.displacement_channel(W=20, L=110, x_I=25.0, seed=6, noise=1e-3), \
        I.fingering_params(5.0, 0.1, 60.0)
    yield "periodic_droplet_70x50", I.periodic_box_droplet(70, 50, R=12.0, xc=33.1, yc=24.6, noise=1e-3, seed=1), \
        I.Params(sigma=0.02, nu_R=0.2, nu_B=0.05)
    yield "cylinder_90x80", I.cylinder_droplet(90, 80, Rs=16.0, cx=45.0, cy=28.0, Rd=14.0, theta=math.radians(120),
                                               noise=1e-3, seed=4, analytic_normal=False), \
        I.Params(theta=math.radians(120), sigma=0.02)


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("name,g,p", list(_cases()), ids=[c[0] for c in _cases()])
def test_segment_height_and_direction_do_not_change_the_bits(prec, name, g, p):
    from paper_1707_00198_gb300.lbcg import Lattice
    out = {}
    for rows in (g.ny, 3, 7, 8, 17):
        L = Lattice(g, p, prec)
        L.set_sweep(rows)
        L.step(50)
        out[rows] = L.populations()
        L.close()
    ref = out[g.ny]
    assert np.isfinite(ref).all()
    for rows, got in out.items():
        assert np.array_equal(got, ref), (name, prec, rows, float(np.abs(got - ref).max()))
