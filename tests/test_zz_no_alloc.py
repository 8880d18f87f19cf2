"""lbcg_field_moments_noalloc: the observable sums for callers that cannot call cudaMalloc
(code under a fixed device-memory budget, allocators that forbid new allocations, threads
that must not take the driver's allocation locks).

The entry point keeps its partial sums in a file-scope device array instead of memory owned
by a handle.  Its sums must match those lbcg_observables computes with handle-owned scratch,
on two calls in a row with different lattices (so a stale partial from the first call would
show up in the second) and on a repeat of the first call.
"""
import math

import numpy as np
import pytest
import torch

from paper_1707_00198_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _near_solid(g):
    """Nodes within Chebyshev distance 3 of a solid node (periodic axes wrap, others clamp)."""
    s = g.solid != 0
    out = s.copy()
    for dy in range(-3, 4):
        for dx in range(-3, 4):
            ys = np.arange(g.ny) + dy
            xs = np.arange(g.nx) + dx
            ys = ys % g.ny if g.bc_y == "periodic" else np.clip(ys, 0, g.ny - 1)
            xs = xs % g.nx if g.bc_x == "periodic" else np.clip(xs, 0, g.nx - 1)
            out |= s[np.ix_(ys, xs)]
    return out


def _device_inputs(L, g):
    rho, rn, ux, uy = L.fields()
    solid = g.solid != 0
    rR = np.where(solid, 0.0, rho * (1 + rn) / 2)
    rB = np.where(solid, 0.0, rho * (1 - rn) / 2)
    fields = torch.tensor(np.stack([rR, rB, ux, uy]), dtype=torch.float64, device="cuda").contiguous()
    mask = (solid.astype(np.uint8) * 1) | (_near_solid(g).astype(np.uint8) * 8)
    return fields, torch.tensor(mask, dtype=torch.uint8, device="cuda").contiguous()


def _check(out, o):
    assert abs(out[0] - o["mass_R"]) <= 1e-9 * abs(o["mass_R"])
    assert abs(out[1] - o["mass_B"]) <= 1e-9 * abs(o["mass_B"])
    assert abs(out[2] - o["umax"]) <= 1e-9 * max(1.0, abs(o["umax"]))
    for k in range(9):
        ref = o["moments"][k]
        assert abs(out[3 + k] - ref) <= 1e-9 * max(1.0, abs(ref)), (k, out[3 + k], ref)
    dp = out[12] / out[13] - out[14] / out[15]
    assert abs(dp - o["dp_laplace"]) <= 1e-9 * max(1.0, abs(o["dp_laplace"]))
    assert out[16] == float(o["nonfinite"])


def test_noalloc_moments_match_observables_on_calls_in_a_row():
    import __graft_entry__ as ge
    ge.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1707_00198_gb300 import lbcg

    cases = [
        (I.flat_wall_droplet(100, 50, R=20.0, noise=1e-3, seed=0), I.Params(theta=math.radians(60)), 60),
        (I.periodic_box_droplet(70, 50, R=12.0, xc=33.1, yc=24.6, noise=1e-3, seed=1), I.Params(sigma=0.02), 40),
    ]
    prepared = []
    for g, p, n in cases:
        L = lbcg.Lattice(g, p, "fp64")
        L.step(n)
        o = L.observables(wall_y=0.5)
        fields, mask = _device_inputs(L, g)
        L.close()
        prepared.append((g, o, fields, mask))
    # every buffer the entry point touches is allocated here, by the caller
    outs = [torch.full((17,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(3)]
    stream = torch.cuda.current_stream().cuda_stream
    order = [0, 1, 0]   # two different lattices in a row, then the first again
    for out, i in zip(outs, order):
        g, o, fields, mask = prepared[i]
        lbcg.lbcg_field_moments_noalloc(fields.data_ptr(), mask.data_ptr(), g.nx, g.ny, stream, out.data_ptr())
    torch.cuda.synchronize()
    for out, i in zip(outs, order):
        _check(out.cpu().numpy(), prepared[i][1])
    assert torch.equal(outs[0], outs[2])


def test_noalloc_rejects_sizes_beyond_the_maximum():
    import __graft_entry__ as ge
    ge.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1707_00198_gb300 import lbcg

    buf = torch.zeros(32, dtype=torch.float64, device="cuda")
    with pytest.raises(lbcg.LBCGError, match="nx\\*ny"):
        lbcg.lbcg_field_moments_noalloc(buf.data_ptr(), buf.data_ptr(), 65536, 65536, 0, buf.data_ptr())
    with pytest.raises(lbcg.LBCGError, match="nx\\*ny"):
        lbcg.lbcg_field_moments_noalloc(buf.data_ptr(), buf.data_ptr(), 0, 5, 0, buf.data_ptr())
