"""Observables of a colour-gradient LBM state, computed plainly on the CPU in FP64.

THIS IS TEST INFRASTRUCTURE (see ``oracle/lbcg_oracle.py``); it imports only the oracle.

* per-colour mass (Eq. 16 summed over fluid nodes) and |u|_max (Eq. 46, u from Eq. 17);
* interface points: rho^N = 0 crossings, linearly interpolated on the x-links
  (x, y)-(x+1, y) and y-links (x, y)-(x, y+1) between two fluid nodes that are both
  farther than 3 nodes (Chebyshev) from any solid node; links across a periodic seam are
  skipped; a crossing is a link whose end values differ in the sign test rho^N >= 0;
* an algebraic (Kasa) circle fit through those points from their moment sums, taken about
  the lattice centre (nx/2, ny/2);
* the contact angle: flat wall at height y_w below the droplet,
  cos(theta) = (y_w - y_c)/R; cylinder of radius R_s at (c_x, c_y),
  cos(theta) = (R_s^2 + R^2 - D^2)/(2 R_s R) with D the centre distance;
* the Laplace pressure jump: p = rho c_s^2, mean over fluid nodes with rho^N > 0.9 minus
  the mean over fluid nodes with rho^N < -0.9;
* the finger tip and contact line: the first rho^N >= 0 -> rho^N < 0 change scanning
  from x = 0 along the centre row (the mean of the two middle rows when ny is even) and
  along the given contact-line rows (their mean).
"""
from __future__ import annotations

import math

import torch

from . import lbcg_oracle as O


def interface_moments(lat: O.OracleLattice, rhoN: torch.Tensor):
    """Moment sums (n, Sx, Sy, Sxx, Syy, Sxy, Szx, Szy, Sz) of the interface points, with
    coordinates relative to (nx/2, ny/2) and z = x^2 + y^2."""
    rn = rhoN.detach()
    ok = lat.fluid & ~lat.near_solid
    pts = []
    ny, nx = rn.shape
    # x-links
    a, b = rn[:, :-1], rn[:, 1:]
    m = ok[:, :-1] & ok[:, 1:] & ((a >= 0) != (b >= 0))
    t = a / torch.where(m, a - b, torch.ones_like(a))
    ys, xs = torch.nonzero(m, as_tuple=True)
    pts.append(torch.stack([xs.to(O.DT) + t[m], ys.to(O.DT)], 1))
    # y-links
    a, b = rn[:-1, :], rn[1:, :]
    m = ok[:-1, :] & ok[1:, :] & ((a >= 0) != (b >= 0))
    t = a / torch.where(m, a - b, torch.ones_like(a))
    ys, xs = torch.nonzero(m, as_tuple=True)
    pts.append(torch.stack([xs.to(O.DT), ys.to(O.DT) + t[m]], 1))
    p = torch.cat(pts, 0)
    x = p[:, 0] - nx / 2
    y = p[:, 1] - ny / 2
    z = x * x + y * y
    return dict(n=float(p.shape[0]), Sx=float(x.sum()), Sy=float(y.sum()), Sxx=float((x * x).sum()),
                Syy=float((y * y).sum()), Sxy=float((x * y).sum()), Szx=float((z * x).sum()),
                Szy=float((z * y).sum()), Sz=float(z.sum()))


def circle_fit(mom, nx: int, ny: int):
    """Kasa fit: minimise sum (x^2 + y^2 + D x + E y + F)^2; returns (x_c, y_c, R)."""
    if mom["n"] < 3:
        return float("nan"), float("nan"), float("nan")
    A = torch.tensor([[mom["Sxx"], mom["Sxy"], mom["Sx"]],
                      [mom["Sxy"], mom["Syy"], mom["Sy"]],
                      [mom["Sx"], mom["Sy"], mom["n"]]], dtype=O.DT)
    rhs = -torch.tensor([mom["Szx"], mom["Szy"], mom["Sz"]], dtype=O.DT)
    D, E, F = torch.linalg.solve(A, rhs).tolist()
    xc, yc = -D / 2, -E / 2
    R = math.sqrt(max(xc * xc + yc * yc - F, 0.0))
    return xc + nx / 2, yc + ny / 2, R


def first_crossing(profile: torch.Tensor) -> float:
    """x of the first rho^N >= 0 -> rho^N < 0 change along a row, or -1."""
    a, b = profile[:-1], profile[1:]
    m = (a >= 0) & (b < 0)
    idx = torch.nonzero(m, as_tuple=True)[0]
    if idx.numel() == 0:
        return -1.0
    i = int(idx[0])
    return i + float(a[i] / (a[i] - b[i]))


def observables(lat: O.OracleLattice, prm, fR, fB, wall_y: float = 0.5, cyl=None,
                tip_rows=None, cl_rows=None):
    mac = O.macroscopic(lat, prm, fR, fB)
    fl = lat.fluid
    rhoN = mac["rhoN"].detach()
    out = {}
    out["mass_R"] = float(mac["rhoR"][fl].sum())
    out["mass_B"] = float(mac["rhoB"][fl].sum())
    u = torch.sqrt(mac["ux"] ** 2 + mac["uy"] ** 2)
    out["umax"] = float(u[fl].max()) if bool(fl.any()) else 0.0
    mom = interface_moments(lat, rhoN)
    out["moments"] = mom
    xc, yc, R = circle_fit(mom, lat.nx, lat.ny)
    out["xc"], out["yc"], out["R"], out["n_pts"] = xc, yc, R, mom["n"]
    if cyl is not None:
        cx, cy, Rs = cyl
        D = math.hypot(xc - cx, yc - cy)
        c = (Rs * Rs + R * R - D * D) / (2 * Rs * R)
    else:
        c = (wall_y - yc) / R if R == R and R > 0 else float("nan")
    out["theta_deg"] = math.degrees(math.acos(max(-1.0, min(1.0, c)))) if c == c else float("nan")
    p = mac["rho"].detach() * O.CS2
    inn = fl & (rhoN > 0.9)
    outn = fl & (rhoN < -0.9)
    if bool(inn.any()) and bool(outn.any()):
        out["dp_laplace"] = float(p[inn].mean() - p[outn].mean())
    else:
        out["dp_laplace"] = float("nan")
    ny = lat.ny
    if tip_rows is None:
        tip_rows = (ny // 2 - 1, ny // 2) if ny % 2 == 0 else (ny // 2, ny // 2)
    prof = 0.5 * (rhoN[tip_rows[0]] + rhoN[tip_rows[1]])
    out["x_tip"] = first_crossing(prof)
    if cl_rows is None:
        cl_rows = (1, ny - 2)
    xs = [first_crossing(rhoN[r]) for r in cl_rows]
    xs = [v for v in xs if v >= 0]
    out["x_cl"] = sum(xs) / len(xs) if xs else -1.0
    out["nonfinite"] = int(not bool(torch.isfinite(mac["rho"][fl]).all()))
    return out


def velocity_change(lat: O.OracleLattice, mac_then: dict, mac_now: dict) -> float:
    """E_1 of Eq. 45: max over fluid nodes of max(|u_x^now - u_x^then|, |u_y^now - u_y^then|)
    (the paper takes the two states 500 steps apart and stops when E_1 < 1e-7)."""
    fl = lat.fluid
    dx = (mac_now["ux"] - mac_then["ux"]).detach().abs()[fl]
    dy = (mac_now["uy"] - mac_then["uy"]).detach().abs()[fl]
    return float(torch.maximum(dx, dy).max())


def npmt(lat: O.OracleLattice, mac: dict, cx: float, cy: float, r: float, inside_red: bool = True) -> dict:
    """E_NPMT of Eq. 47 with the theoretical steady interface C = circle (cx, cy, r) in node
    coordinates (node (x, y) is inside when (x - cx)^2 + (y - cy)^2 < r^2).  Masses are sums of
    rho_R and rho_B (Eq. 16) over fluid nodes.  Read as each colour's mass on the wrong side of
    C: with D the colour inside C and O the other, E = sqrt((m_O^in / m_O^all)^2 +
    (m_D^out / m_D^all)^2)."""
    fl = lat.fluid
    ny, nx = fl.shape
    y, x = torch.meshgrid(torch.arange(ny, dtype=O.DT), torch.arange(nx, dtype=O.DT), indexing="ij")
    inside = ((x - cx) ** 2 + (y - cy) ** 2 < r * r) & fl
    outside = fl & ~inside
    rR, rB = mac["rhoR"].detach(), mac["rhoB"].detach()
    m = dict(m_R_in=float(rR[inside].sum()), m_R_out=float(rR[outside].sum()),
             m_B_in=float(rB[inside].sum()), m_B_out=float(rB[outside].sum()))
    if inside_red:
        wrong_O, all_O, wrong_D, all_D = m["m_B_in"], m["m_B_in"] + m["m_B_out"], m["m_R_out"], m["m_R_in"] + m["m_R_out"]
    else:
        wrong_O, all_O, wrong_D, all_D = m["m_R_in"], m["m_R_in"] + m["m_R_out"], m["m_B_out"], m["m_B_in"] + m["m_B_out"]
    m["e_npmt"] = math.sqrt((wrong_O / all_O) ** 2 + (wrong_D / all_D) ** 2)
    return m
