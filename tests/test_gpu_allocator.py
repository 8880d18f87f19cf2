"""Device memory from a caller's allocator (lbcg_set_allocator): with PyTorch's caching allocator
installed, a handle's pools, node arrays and temporaries come from PyTorch (its accounting grows
by at least the two population pools while the handle lives and falls back when it is
destroyed), the step still matches the oracle, and an allocator that fails makes creation fail
with LBCG_E_NOMEM instead of falling back to cudaMalloc."""
import numpy as np
import pytest
import torch

from oracle import lbcg_oracle as O
from paper_1707_00198_gb300 import inputs as I

pytestmark = pytest.mark.gpu

LBCG_E_NOMEM = 8


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as ge
    ge.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def test_torch_caching_allocator_holds_the_handle_memory():
    from paper_1707_00198_gb300 import lbcg
    g = I.displacement_channel(W=20, L=110, x_I=25.0, seed=6, noise=1e-3)
    p = I.fingering_params(M=5.0, Ca=0.1, theta_deg=60.0)
    torch.cuda.synchronize()
    m0 = torch.cuda.memory_allocated()
    lbcg.use_torch_allocator(True)
    try:
        L = lbcg.Lattice(g, p, "fp64")
        pools = 2 * L.state_bytes
        assert torch.cuda.memory_allocated() - m0 >= pools
        L.step(40)
        got = L.populations()            # its staging buffer comes from PyTorch too
        ad = L.adjoint(20, 10, objective="red_mass")
        assert np.isfinite(ad["J"]) and np.isfinite(ad["dsigma"])
        L.close()
    finally:
        lbcg.use_torch_allocator(False)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == m0
    lat = O.make_lattice(g, p.theta)
    fR, fB = O.init_state(lat, g.rhoN0, p.rho0, p)
    fR, fB = O.run(lat, p, fR, fB, 40)
    assert float(np.abs(got - np.stack([fR.numpy(), fB.numpy()])).max()) <= 1e-10


def test_failing_allocator_reports_nomem():
    from paper_1707_00198_gb300 import lbcg
    g, p = I.config_static_droplet()
    lbcg.lbcg_set_allocator(lambda n, s: 0, lambda q, s: None)
    try:
        with pytest.raises(lbcg.LBCGError) as ei:
            lbcg.Lattice(g, p, "fp32")
        assert ei.value.status == LBCG_E_NOMEM
    finally:
        lbcg.lbcg_set_allocator()
    L = lbcg.Lattice(g, p, "fp32")       # cudaMalloc again
    L.step(2)
    L.close()
