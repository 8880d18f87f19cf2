"""Pins of the oracle's steady-state diagnostics (Sec. III): E_1 (Eq. 45) and E_NPMT
(Eq. 47), against hand-made fields with known answers and against node-by-node loops."""
import math

import numpy as np
import torch

from oracle import lbcg_oracle as O
from oracle import observables as OB
from paper_1707_00198_gb300 import inputs as I


def _lattice(nx=23, ny=17, walls=True):
    g = I.flat_wall_droplet(nx, ny, R=5.0, noise=0.0) if walls else I.periodic_box_droplet(nx, ny, R=4.0, noise=0.0)
    return g, O.make_lattice(g, math.radians(60))


def test_e1_is_zero_for_identical_states_and_the_largest_component_change():
    g, lat = _lattice()
    rng = np.random.default_rng(0)
    ux, uy = torch.tensor(rng.normal(size=(g.ny, g.nx))), torch.tensor(rng.normal(size=(g.ny, g.nx)))
    a = {"ux": ux, "uy": uy}
    assert OB.velocity_change(lat, a, a) == 0.0
    dux, duy = rng.normal(size=(g.ny, g.nx)) * 1e-3, rng.normal(size=(g.ny, g.nx)) * 1e-3
    b = {"ux": ux + torch.tensor(dux), "uy": uy + torch.tensor(duy)}
    # loop over fluid nodes (solid nodes do not count)
    want = 0.0
    for y in range(g.ny):
        for x in range(g.nx):
            if g.solid[y, x] == 0:
                want = max(want, abs(float(b["ux"][y, x] - ux[y, x])), abs(float(b["uy"][y, x] - uy[y, x])))
    assert OB.velocity_change(lat, a, b) == want
    # a change confined to a solid node is not seen
    c = {"ux": ux.clone(), "uy": uy.clone()}
    c["ux"][0, 3] += 5.0
    assert g.solid[0, 3] != 0 and OB.velocity_change(lat, a, c) == 0.0


def _inside(g, cx, cy, r):
    y, x = np.mgrid[0:g.ny, 0:g.nx]
    return (x - cx) ** 2 + (y - cy) ** 2 < r * r


def test_npmt_zero_for_the_exact_circle_and_sqrt2_for_swapped_colours():
    g, lat = _lattice(41, 33, walls=False)
    cx, cy, r = 20.3, 15.8, 9.2
    ins = _inside(g, cx, cy, r)
    red = {"rhoR": torch.tensor(ins, dtype=torch.float64), "rhoB": torch.tensor(~ins, dtype=torch.float64)}
    assert OB.npmt(lat, red, cx, cy, r, inside_red=True)["e_npmt"] == 0.0
    assert abs(OB.npmt(lat, red, cx, cy, r, inside_red=False)["e_npmt"] - math.sqrt(2)) < 1e-15
    blue = {"rhoR": red["rhoB"], "rhoB": red["rhoR"]}
    assert OB.npmt(lat, blue, cx, cy, r, inside_red=False)["e_npmt"] == 0.0


def test_npmt_matches_a_node_by_node_loop():
    g, lat = _lattice(19, 15, walls=True)
    rng = np.random.default_rng(3)
    rR, rB = rng.uniform(0, 1, (g.ny, g.nx)), rng.uniform(0, 1, (g.ny, g.nx))
    mac = {"rhoR": torch.tensor(rR), "rhoB": torch.tensor(rB)}
    cx, cy, r = 9.1, 2.5, 6.3
    for inside_red in (True, False):
        sums = {"Ri": 0.0, "Ro": 0.0, "Bi": 0.0, "Bo": 0.0}
        for y in range(g.ny):
            for x in range(g.nx):
                if g.solid[y, x]:
                    continue
                k = "i" if (x - cx) ** 2 + (y - cy) ** 2 < r * r else "o"
                sums["R" + k] += rR[y, x]
                sums["B" + k] += rB[y, x]
        if inside_red:
            want = math.hypot(sums["Bi"] / (sums["Bi"] + sums["Bo"]), sums["Ro"] / (sums["Ri"] + sums["Ro"]))
        else:
            want = math.hypot(sums["Ri"] / (sums["Ri"] + sums["Ro"]), sums["Bo"] / (sums["Bi"] + sums["Bo"]))
        got = OB.npmt(lat, mac, cx, cy, r, inside_red)
        assert abs(got["e_npmt"] - want) <= 1e-13 * want
        assert abs(got["m_R_in"] - sums["Ri"]) <= 1e-12 and abs(got["m_B_out"] - sums["Bo"]) <= 1e-12


def test_circle_fit_recovers_an_exact_circle_and_the_interface_points():
    """The algebraic circle fit (contact-angle measurement) recovers the centre and radius of
    points lying exactly on a circle to 1e-12, whatever their spread (a slip in the moment
    algebra or the normal equations shows up here, not only as a few degrees of angle); and
    the interface points of a field rho^N = (R - r) clipped to [-1, 1] around that circle are
    its linear-interpolation crossings, which lie within 0.03 of the circle for R = 9."""
    nx, ny, xc, yc, R = 40, 30, 19.3, 12.7, 9.0
    rng = np.random.default_rng(3)
    for n in (3, 7, 200):
        t = rng.uniform(0.0, 2 * math.pi, n) if n > 3 else np.array([0.1, 2.0, 4.1])
        x, y = xc + R * np.cos(t) - nx / 2, yc + R * np.sin(t) - ny / 2
        z = x * x + y * y
        mom = dict(n=float(n), Sx=x.sum(), Sy=y.sum(), Sxx=(x * x).sum(), Syy=(y * y).sum(), Sxy=(x * y).sum(),
                   Szx=(z * x).sum(), Szy=(z * y).sum(), Sz=z.sum())
        fx, fy, fR = OB.circle_fit(mom, nx, ny)
        assert abs(fx - xc) <= 1e-12 * nx and abs(fy - yc) <= 1e-12 * ny and abs(fR - R) <= 1e-12 * R, (n, fx, fy, fR)
    g = I.periodic_box_droplet(nx, ny, R=0.0)
    lat = O.make_lattice(g, math.radians(90))
    yy, xx = np.mgrid[0:ny, 0:nx].astype(float)
    rn = torch.from_numpy(np.clip(R - np.hypot(xx - xc, yy - yc), -1.0, 1.0))
    mom = OB.interface_moments(lat, rn)
    fx, fy, fR = OB.circle_fit(mom, nx, ny)
    assert mom["n"] > 20
    assert abs(fx - xc) <= 0.03 and abs(fy - yc) <= 0.03 and abs(fR - R) <= 0.03, (fx, fy, fR)
