"""The checked build (liblbcg_checked.so: range checks on every population, node-array and
staged-row access of the step kernels) on the cases where indices are most at risk -- lattices
smaller than one tile or strip (every node a halo node), periodic wraps, open inlet/outlet
columns, walls, an E8 cylinder, a batch of uneven lattices -- through every schedule (sweep with
automatic and 3-row segments, 32 x 4/8/16 tiles) and storage form, over 40 steps (a graph
replay and direct launches) and an observables call: no check fails, and the results equal the
normal build's bit for bit (the checks change no arithmetic)."""
import json
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RUN = r'''
import json, math, sys
import numpy as np
sys.path.insert(0, ROOT)
from paper_1707_00198_gb300 import inputs as I, lbcg
th = math.radians
cases = {
    "tiny_walls_5x5": ([I.flat_wall_droplet(5, 5, R=1.6, xc=2.2, noise=1e-2, seed=9)], [I.Params(sigma=0.03)]),
    "tiny_periodic_7x6": ([I.periodic_box_droplet(7, 6, R=2.2, xc=3.3, yc=2.8, noise=1e-2, seed=8)],
                          [I.Params(sigma=0.03)]),
    "channel_130x22": ([I.displacement_channel(W=20, L=130, x_I=25.0, seed=6, noise=1e-3)],
                       [I.fingering_params(5.0, 0.1, 60.0)]),
    "cylinder_e8_60x50": ([I.cylinder_droplet(60, 50, Rs=10.0, cx=30.0, cy=18.0, Rd=9.0, theta=th(110),
                                              noise=1e-3, seed=5, analytic_normal=False)],
                          [I.Params(theta=th(110), sigma=0.02)]),
    "batch_uneven": ([I.flat_wall_droplet(45, 21, R=7.0, xc=20.7, noise=1e-3, seed=1),
                      I.displacement_channel(W=12, L=140, x_I=20.0, seed=3, noise=1e-3),
                      I.periodic_box_droplet(33, 40, R=9.0, noise=1e-3, seed=2)],
                     [I.Params(theta=th(70), sigma=0.02), I.fingering_params(5.0, 0.1, 60.0),
                      I.Params(sigma=0.01, nu_B=0.05)]),
}
schedules = [("sweep", 0), ("sweep3", 3), ("tiles4", 4), ("tiles8", 8), ("tiles16", 16)]
out = {}
for name, (gs, ps) in cases.items():
    for form in ("fp64", "fp32", "fp16", "bf16"):
        for sname, v in schedules:
            L = lbcg.Lattice(gs, ps, form)
            if sname.startswith("sweep"):
                L.set_sweep(v)
            else:
                L.set_tile(v)
            L.step(40)
            status = "ok"
            try:
                obs = [L.observables(lattice=i)["mass_R"] for i in range(len(gs))]
                pops = [L.populations(i) for i in range(len(gs))]
            except lbcg.LBCGError as e:
                status, obs, pops = str(e), [], []
            L.close()
            key = f"{name}/{form}/{sname}"
            out[key] = status
            for i, p in enumerate(pops):
                np.save(f"{OUT}/{key.replace('/', '_')}_{i}.npy", p)
            np.save(f"{OUT}/{key.replace('/', '_')}_obs.npy", np.array(obs))
json.dump(out, open(f"{OUT}/status.json", "w"))
'''


def _run(lib: str, out: str):
    env = {**os.environ, "LBCG_LIBRARY": lib}
    code = f"ROOT = {ROOT!r}\nOUT = {out!r}\n" + RUN
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.load(open(os.path.join(out, "status.json")))


def test_checked_build_reports_nothing_and_matches_the_normal_build():
    import __graft_entry__ as ge
    from paper_1707_00198_gb300 import build as B
    ge.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    checked = B.build(checked=True)
    with tempfile.TemporaryDirectory() as d1, tempfile.TemporaryDirectory() as d2:
        s_chk = _run(checked, d1)
        s_ref = _run(B.LIB, d2)
        bad = {k: v for k, v in s_chk.items() if v != "ok"}
        assert not bad, bad
        assert set(s_ref.values()) == {"ok"}
        files = sorted(f for f in os.listdir(d2) if f.endswith(".npy"))
        assert len(files) >= 5 * 4 * 5 * 2
        for f in files:
            a, b = np.load(os.path.join(d1, f)), np.load(os.path.join(d2, f))
            assert np.array_equal(a, b), f
