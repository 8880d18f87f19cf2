"""lbcg_step_host: host state in, steps, host state out, with the copies of lattice groups
overlapping their steps.  Its result must be the bits of lbcg_upload_state + lbcg_step (direct
launches: fewer than 32 steps) + lbcg_download_state, for a batch (several groups) and a single
lattice (one group), in place and between two buffers, in FP32 and in 16-bit storage (whose
stochastic rounding is keyed by lattice offset and step, not by launch order)."""
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


def _batch():
    gs, ps = I.channel_sweep(11, seed=3, wmin=20, wmax=48)
    return gs, ps


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("which", ["batch", "single"])
@pytest.mark.parametrize("nsteps", [0, 1, 5])
def test_step_host_equals_upload_step_download(prec, which, nsteps):
    from paper_1707_00198_gb300 import lbcg
    gs, ps = _batch()
    if which == "single":
        gs, ps = gs[:1], ps[:1]
    A, B, C = (lbcg.Lattice(gs, ps, prec) for _ in range(3))
    for L in (A, B, C):
        L.step(3)   # a state that is not the initial one, on the second pool (odd step count)
    sb = A.state_bytes
    start = torch.empty(sb, dtype=torch.uint8, pin_memory=True)
    lbcg.lbcg_download_state(A.h, start.data_ptr(), sb)
    # reference: upload, direct steps, download
    ref = torch.empty(sb, dtype=torch.uint8, pin_memory=True)
    lbcg.lbcg_upload_state(A.h, start.data_ptr(), sb)
    A.step(nsteps)
    lbcg.lbcg_download_state(A.h, ref.data_ptr(), sb)
    # in place (B) and between two buffers (C)
    buf = start.clone().pin_memory()
    lbcg.lbcg_step_host(B.h, buf.data_ptr(), buf.data_ptr(), sb, nsteps)
    assert torch.equal(buf, ref), (prec, which, nsteps)
    out = torch.empty(sb, dtype=torch.uint8, pin_memory=True)
    lbcg.lbcg_step_host(C.h, start.data_ptr(), out.data_ptr(), sb, nsteps)
    assert torch.equal(out, ref), (prec, which, nsteps)
    # the handles hold the result and its step count, like A
    spec = lbcg.obs_spec(ny=gs[0].ny)
    for L in (B, C):
        assert lbcg.lbcg_observables(L.h, 0, spec)["step"] == lbcg.lbcg_observables(A.h, 0, spec)["step"]
        for i in range(len(gs)):
            assert np.array_equal(A.populations(i), L.populations(i)), (prec, which, nsteps, i)
    for L in (A, B, C):
        L.close()
