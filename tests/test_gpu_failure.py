"""Failure detection of the y-sweep's bounded device wait, without any GPU fault.

The FP32 and 16-bit y-sweep stage each row in shared memory with bulk asynchronous copies and
every thread waits for the row with a bounded number of polls.  With the bound set to 0 every
wait gives up at once (the copies themselves are ordinary and land): each block must stop
before writing anything, wait for the copies it issued, and set the handle's error word, so
that the next synchronising call returns LBCG_E_TIMEOUT.  After that the handle must be
usable again: with the default bound restored, a state set afresh steps exactly as on a new
handle, directly and through the captured CUDA graph.
"""
import numpy as np
import pytest
import torch

from oracle import lbcg_oracle as O
from paper_1707_00198_gb300 import inputs as I

pytestmark = pytest.mark.gpu

LBCG_E_TIMEOUT = 6


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as ge
    ge.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def _state(g, p, n):
    lat = O.make_lattice(g, p.theta)
    fR, fB = O.init_state(lat, g.rhoN0, p.rho0, p)
    fR, fB = O.run(lat, p, fR, fB, n)
    return np.stack([fR.numpy(), fB.numpy()])


# one step from a common state: the tolerance of each storage form against the oracle (FP32:
# as in test_gpu_parity.py; 16-bit: four half-ulps at 4/9, derived there)
TOL1 = {"fp32": 2e-6, "fp16": 4 * 2.0 ** -13}


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_sweep_wait_timeout_is_reported_and_the_handle_recovers(prec):
    from paper_1707_00198_gb300.lbcg import Lattice, LBCGError
    g = I.displacement_channel(W=20, L=250, x_I=20.0, seed=21, noise=1e-3)
    p = I.fingering_params(M=5.0, Ca=0.1, theta_deg=60.0)
    s0 = _state(g, p, 20)
    lat = O.make_lattice(g, p.theta)
    oR, oB = O.step(lat, p, torch.from_numpy(s0[0].copy()), torch.from_numpy(s0[1].copy()))
    want1 = np.stack([oR.numpy(), oB.numpy()])

    ref = Lattice(g, p, prec)
    ref.set_sweep(0)
    ref.set_populations(s0)
    ref.step(41)
    want41 = ref.populations()
    ref.close()

    L = Lattice(g, p, prec)
    L.set_sweep(0)
    L.set_populations(s0)
    # direct launches, then (back on the first pool) the 32-step captured graph
    for n in (1, 1, 32):
        L.set_poll_limit(0)
        L.step(n)
        with pytest.raises(LBCGError) as ei:
            L.populations()
        assert ei.value.status == LBCG_E_TIMEOUT, str(ei.value)
        L.populations()                     # reported once: the word is cleared
    L.set_poll_limit(-1)
    L.set_populations(s0)
    L.step(1)
    assert float(np.abs(L.populations() - want1).max()) <= TOL1[prec]
    L.step(40)                              # a graph replay plus direct steps
    got41 = L.populations()
    if prec == "fp32":
        assert np.array_equal(got41, want41)
    else:                                   # stochastic rounding keys differ by step count
        assert float(np.abs(got41 - want41).max()) <= 1e-2
    assert L.observables()["nonfinite"] == 0
    L.close()
