"""Read-before-write poison test of the step kernels (stands in for a memory sanitizer).

Before every step, every stored value that belongs to a solid node or to the padding columns of
the 32-aligned rows is overwritten with NaN.  No kernel may use such a value: the half-way
bounce-back keeps a fluid node's populations in its own slots, and the solid rows of a staged
row segment are copied but never decoded.  The poisoned trajectory must stay finite and equal,
bit for bit, to the same trajectory without poison, for every storage form and both schedules
(y-sweep strips and 32-wide tiles).

The raw state (lbcg_download_state / lbcg_upload_state) of a one-lattice handle is the pool
layout: each row is cut into 32-node segments of [direction 0..8][node 0..31][colour 0..1]
values, so element ((y * pitch/32 + x/32) * 576 + a * 64 + (x % 32) * 2 + k) is colour k of
direction a at node (x, y); pitch is nx rounded up to 32.
"""
import math

import numpy as np
import pytest
import torch

from paper_1707_00198_gb300 import inputs as I

pytestmark = pytest.mark.gpu

DTYPES = {"fp64": np.float64, "fp32": np.float32, "fp16": np.float16, "bf16": np.uint16}
NAN_BF16 = np.uint16(0x7FC0)


def _unused_mask(g):
    pitch = (g.nx + 31) // 32 * 32
    x = np.arange(pitch)
    unused = np.ones((g.ny, pitch), dtype=bool)            # padding columns
    unused[:, :g.nx] = g.solid != 0                         # solid nodes
    # [y][segment][direction][lane][colour]
    m = unused.reshape(g.ny, pitch // 32, 1, 32, 1)
    return np.broadcast_to(m, (g.ny, pitch // 32, 9, 32, 2)).reshape(-1)


def _run(g, p, prec, schedule, n, poison):
    from paper_1707_00198_gb300 import lbcg
    L = lbcg.Lattice(g, p, prec)
    if schedule == "sweep":
        L.set_sweep(0)
    else:
        L.set_tile(8)
    nb = L.state_bytes
    buf = torch.empty(nb, dtype=torch.uint8, pin_memory=True)
    raw = buf.numpy().view(DTYPES[prec])
    mask = _unused_mask(g)
    assert raw.size == mask.size
    for _ in range(n):
        if poison:
            lbcg.lbcg_download_state(L.h, buf.data_ptr(), nb)
            raw[mask] = NAN_BF16 if prec == "bf16" else np.nan
            lbcg.lbcg_upload_state(L.h, buf.data_ptr(), nb)
        L.step(1)
    out = L.populations()
    L.close()
    return out


CASES = [
    ("channel_inout", lambda: (I.displacement_channel(W=20, L=110, x_I=25.0, seed=6, noise=1e-3),
                               I.fingering_params(M=5.0, Ca=0.1, theta_deg=60.0))),
    ("cylinder_box", lambda: (I.cylinder_droplet(90, 80, Rs=16.0, cx=45.0, cy=28.0, Rd=14.0,
                                                 theta=math.radians(120), noise=1e-3, seed=4, analytic_normal=False),
                              I.Params(theta=math.radians(120), sigma=0.02))),
]


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16", "bf16"])
@pytest.mark.parametrize("schedule", ["sweep", "tiles"])
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_solid_and_padding_slots_are_never_read(name, make, schedule, prec):
    import __graft_entry__ as ge
    ge.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    g, p = make()
    ref = _run(g, p, prec, schedule, 12, poison=False)
    got = _run(g, p, prec, schedule, 12, poison=True)
    fl = g.solid == 0
    assert np.isfinite(got[:, :, fl]).all()
    assert np.array_equal(got[:, :, fl], ref[:, :, fl])
