"""The hand-written discrete adjoint (lbcg_adjoint) against reverse mode through the FP64
oracle, and against central finite differences of the forward CUDA path.

The oracle's step is written with differentiable torch operations, so torch autograd through
`oracle.run` gives the exact gradient of the same discrete map (the wetting pick of Eq. 36 and
the guard of the unit normal are piecewise constant, so their derivative is zero almost
everywhere, as in the adjoint kernels).  Gradients: the contact angle per outermost fluid node
(Eq. 34), the interfacial tension sigma (Eq. 10) and the two viscosities (Eq. 18).
"""
import math

import numpy as np
import pytest
import torch

from oracle import lbcg_oracle as O
from paper_1707_00198_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _lib():
    import __graft_entry__ as ge
    ge.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1707_00198_gb300 import lbcg
    return lbcg


def _oracle_grads(g, p, c, nsteps):
    """J = sum c * rho^N over fluid nodes after nsteps, and its gradients by autograd."""
    th = torch.tensor(np.full((g.ny, g.nx), p.theta) if g.theta_node is None else g.theta_node,
                      dtype=torch.float64, requires_grad=True)
    sg = torch.tensor(p.sigma, dtype=torch.float64, requires_grad=True)
    nR = torch.tensor(p.nu_R, dtype=torch.float64, requires_grad=True)
    nB = torch.tensor(p.nu_B, dtype=torch.float64, requires_grad=True)
    pp = I.Params(**{**p.__dict__, "sigma": sg, "nu_R": nR, "nu_B": nB})
    lat = O.make_lattice(g, th)
    fR, fB = O.init_state(lat, g.rhoN0, p.rho0, pp)
    fR, fB = O.run(lat, pp, fR, fB, nsteps)
    rn = O.macroscopic(lat, pp, fR, fB)["rhoN"]
    J = (torch.from_numpy(c) * rn * lat.fluid).sum()
    J.backward()
    return {"J": J.item(), "dsigma": sg.grad.item(), "dnu_R": nR.grad.item(), "dnu_B": nB.grad.item(),
            "dtheta_node": th.grad.numpy()}


def _close(a, b, rtol, atol=0.0):
    return abs(a - b) <= rtol * max(abs(a), abs(b)) + atol


CASES = [
    # inlet/outlet channel with closed walls (Zou-He columns inside the adjoint)
    ("channel", lambda: (I.displacement_channel(W=6, L=16, x_I=6.0, seed=3, noise=1e-2),
                         I.fingering_params(M=3.0, Ca=0.1, theta_deg=60.0)), 10, 4),
    # Poiseuille inlet profile (Sec. III.D): the Zou-He transpose with a row-dependent velocity
    ("poiseuille", lambda: (I.displacement_channel(W=7, L=16, x_I=6.0, seed=5, noise=1e-2),
                            I.Params(**{**I.fingering_params(M=2.0, Ca=0.1, theta_deg=70.0).__dict__,
                                        "u_in": 0.04, "inlet_profile": 1})), 10, 4),
    # periodic x, closed y, a sessile droplet: both contact lines on the bottom wall
    ("droplet", lambda: (I.flat_wall_droplet(24, 14, R=6.0, noise=1e-2, seed=2),
                         I.Params(sigma=0.02, nu_R=0.2, nu_B=0.05, theta=math.radians(120.0))), 12, 5),
    # cylinder with the E8 staircase normal: Eq. 32-36 at every orientation of the wall
    ("cylinder", lambda: (I.cylinder_droplet(28, 28, Rs=5.0, Rd=6.0, theta=math.radians(75.0), cx=14.0, cy=9.0,
                                             noise=1e-2, seed=4, analytic_normal=False),
                          I.Params(sigma=0.01, theta=math.radians(75.0))), 8, 3),
]


# FP64 reverse: rounding only (1e-8).  FP32 reverse: single-precision arithmetic along a few
# thousand dependent operations per step, and normals frozen below |grad rho^N| = 1e-5 (where
# the oracle still differentiates them), 2e-3 of the largest per-node value.
REVERSE_TOL = {"fp64": 1e-8, "fp32": 2e-3}


@pytest.mark.parametrize("reverse", ["fp64", "fp32"])
@pytest.mark.parametrize("name,make,nsteps,ckpt", CASES, ids=[c[0] for c in CASES])
def test_adjoint_matches_oracle_autograd(name, make, nsteps, ckpt, reverse):
    lbcg = _lib()
    g, p = make()
    c = np.random.default_rng(7).uniform(-1.0, 1.0, (g.ny, g.nx))
    ref = _oracle_grads(g, p, c, nsteps)
    L = lbcg.Lattice(g, p, "fp64")
    try:
        out = L.adjoint(nsteps, ckpt, weight=c, reverse_fp32=reverse == "fp32")
    finally:
        L.close()
    tol = REVERSE_TOL[reverse]
    assert _close(out["J"], ref["J"], 1e-11, 1e-12), (out["J"], ref["J"])
    for k in ("dsigma", "dnu_R", "dnu_B"):
        assert _close(out[k], ref[k], tol, 1e-12), (k, out[k], ref[k])
    dn, dr = out["dtheta_node"], ref["dtheta_node"]
    scale = max(1e-12, float(np.abs(dr).max()))
    assert float(np.abs(dn - dr).max()) <= tol * scale, float(np.abs(dn - dr).max())
    assert _close(out["dtheta"], float(dr.sum()), tol, 1e-12)
    # the angle enters only at outermost fluid nodes
    assert np.count_nonzero(dn) > 0


def test_adjoint_checkpoint_interval_does_not_change_the_gradient():
    lbcg = _lib()
    g = I.displacement_channel(W=6, L=16, x_I=6.0, seed=3, noise=1e-2)
    p = I.fingering_params(M=3.0, Ca=0.1, theta_deg=60.0)
    c = np.random.default_rng(0).uniform(-1.0, 1.0, (g.ny, g.nx))
    outs = []
    for ck in (1, 3, 9, 20):
        L = lbcg.Lattice(g, p, "fp64")
        outs.append(L.adjoint(9, ck, weight=c))
        L.close()
    for o in outs[1:]:
        assert o["J"] == outs[0]["J"]
        for k in ("dsigma", "dnu_R", "dnu_B", "dtheta"):
            assert _close(o[k], outs[0][k], 1e-12, 1e-15), k   # FP64 atomics: summation order only


def test_adjoint_finger_length_against_finite_differences():
    """J = x_tip - x_cl (Sec. III.D) of a displacement channel; central differences of the
    forward CUDA path (FP64) for sigma, nu_R, nu_B, the global angle and one node's angle."""
    lbcg = _lib()
    g = I.displacement_channel(W=10, L=48, x_I=12.0, seed=1)
    p = I.fingering_params(M=10.0, Ca=0.05, theta_deg=60.0)
    n = 120

    def J(geom, prm):
        L = lbcg.Lattice(geom, prm, "fp64")
        L.step(n)
        o = L.observables()
        L.close()
        return o["x_tip"] - o["x_cl"]

    L = lbcg.Lattice(g, p, "fp64")
    out = L.adjoint(n, 25)
    L.close()
    assert _close(out["J"], J(g, p), 1e-12)
    h = 1e-6
    for key, field, scale in (("dsigma", "sigma", p.sigma), ("dnu_R", "nu_R", p.nu_R), ("dnu_B", "nu_B", p.nu_B),
                              ("dtheta", "theta", 1.0)):
        d = h * scale
        jp = J(g, I.Params(**{**p.__dict__, field: getattr(p, field) + d}))
        jm = J(g, I.Params(**{**p.__dict__, field: getattr(p, field) - d}))
        fd = (jp - jm) / (2 * d)
        assert _close(out[key], fd, 2e-5, 1e-9), (key, out[key], fd)
    # one node's angle: the outermost fluid node with the largest sensitivity
    dn = out["dtheta_node"]
    iy, ix = np.unravel_index(np.argmax(np.abs(dn)), dn.shape)
    base = np.full((g.ny, g.nx), p.theta)

    def with_theta(delta):
        t = base.copy()
        t[iy, ix] += delta
        return I.Geometry(g.nx, g.ny, g.solid, g.rhoN0, g.bc_x, g.bc_y, theta_node=t)

    fd = (J(with_theta(h), p) - J(with_theta(-h), p)) / (2 * h)
    assert _close(dn[iy, ix], fd, 2e-5, 1e-9), (dn[iy, ix], fd)


def test_adjoint_rejects_unsupported_handles():
    lbcg = _lib()
    g = I.displacement_channel(W=6, L=16, x_I=6.0, seed=3)
    p = I.fingering_params(M=3.0, Ca=0.1, theta_deg=60.0)
    L = lbcg.Lattice(g, p, "fp16")
    with pytest.raises(lbcg.LBCGError, match="FP64 or FP32"):
        L.adjoint(2, 1, weight=np.zeros((g.ny, g.nx)))
    L.close()
    L = lbcg.Lattice([g, g], [p, p], "fp64")
    with pytest.raises(lbcg.LBCGError, match="single-lattice"):
        L.adjoint(2, 1, weight=np.zeros((g.ny, g.nx)))
    L.close()
    L = lbcg.Lattice(g, p, "fp64")
    with pytest.raises(lbcg.LBCGError, match="nsteps"):
        L.adjoint(0, 1, weight=np.zeros((g.ny, g.nx)))
    L.close()


def test_red_mass_objective_matches_oracle_autograd():
    """J = the red (invading) fluid's mass at step T -- the displaced mass plus its initial
    value -- against autograd through the oracle."""
    lbcg = _lib()
    g = I.displacement_channel(W=6, L=16, x_I=6.0, seed=3, noise=1e-2)
    p = I.fingering_params(M=3.0, Ca=0.1, theta_deg=60.0)
    n = 10
    th = torch.tensor(np.full((g.ny, g.nx), p.theta), dtype=torch.float64, requires_grad=True)
    sg = torch.tensor(p.sigma, dtype=torch.float64, requires_grad=True)
    nR = torch.tensor(p.nu_R, dtype=torch.float64, requires_grad=True)
    nB = torch.tensor(p.nu_B, dtype=torch.float64, requires_grad=True)
    pp = I.Params(**{**p.__dict__, "sigma": sg, "nu_R": nR, "nu_B": nB})
    lat = O.make_lattice(g, th)
    fR, fB = O.init_state(lat, g.rhoN0, p.rho0, pp)
    fR, fB = O.run(lat, pp, fR, fB, n)
    J = (fR.sum(dim=0) * lat.fluid).sum()
    J.backward()
    L = lbcg.Lattice(g, p, "fp64")
    out = L.adjoint(n, 4, objective="red_mass")
    L.close()
    assert _close(out["J"], J.item(), 1e-12)
    for k, ref in (("dsigma", sg.grad.item()), ("dnu_R", nR.grad.item()), ("dnu_B", nB.grad.item())):
        assert _close(out[k], ref, 1e-8, 1e-13), (k, out[k], ref)
    dr = th.grad.numpy()
    assert float(np.abs(out["dtheta_node"] - dr).max()) <= 1e-8 * max(1e-12, float(np.abs(dr).max()))


def test_autograd_function_viscosity_ratio_and_global_angle():
    """torch.autograd through WettingObjective: the viscosity ratio M = nu_R / nu_B (nu_R
    fixed) and a global contact angle broadcast to every node, each against central finite
    differences of the forward CUDA path."""
    lbcg = _lib()
    from paper_1707_00198_gb300.adjoint import ObjectiveSpec, objective
    g = I.displacement_channel(W=10, L=48, x_I=12.0, seed=1)
    p = I.fingering_params(M=10.0, Ca=0.05, theta_deg=60.0)
    n = 120
    spec = ObjectiveSpec(g, p, nsteps=n, checkpoint=40, objective="finger_length")
    theta = torch.tensor(p.theta, dtype=torch.float64, requires_grad=True)
    M = torch.tensor(10.0, dtype=torch.float64, requires_grad=True)
    nu_R = torch.tensor(p.nu_R, dtype=torch.float64)
    sigma = torch.tensor(p.sigma, dtype=torch.float64, requires_grad=True)
    J = objective(theta * torch.ones(g.ny, g.nx, dtype=torch.float64), sigma, nu_R, nu_R / M, spec)
    J.backward()

    def fwd(M_, th_, sg_=p.sigma):
        q = I.Params(**{**p.__dict__, "nu_B": p.nu_R / M_, "theta": th_, "sigma": sg_})
        L = lbcg.Lattice(g, q, "fp64")
        L.step(n)
        o = L.observables()
        L.close()
        return o["x_tip"] - o["x_cl"]

    assert _close(J.item(), fwd(10.0, p.theta), 1e-12)
    h = 1e-5
    fd_M = (fwd(10.0 + h, p.theta) - fwd(10.0 - h, p.theta)) / (2 * h)
    fd_t = (fwd(10.0, p.theta + 1e-6) - fwd(10.0, p.theta - 1e-6)) / 2e-6
    hs = 1e-5 * p.sigma
    fd_s = (fwd(10.0, p.theta, p.sigma + hs) - fwd(10.0, p.theta, p.sigma - hs)) / (2 * hs)
    assert _close(M.grad.item(), fd_M, 2e-5, 1e-9), (M.grad.item(), fd_M)
    assert _close(theta.grad.item(), fd_t, 2e-5, 1e-9), (theta.grad.item(), fd_t)
    assert _close(sigma.grad.item(), fd_s, 2e-5, 1e-9), (sigma.grad.item(), fd_s)


@pytest.mark.parametrize("reverse", ["fp64", "fp32"])
def test_fp32_adjoint_against_fp32_finite_differences_and_the_fp64_adjoint(reverse):
    """The adjoint of an FP32 forward run (FP32 steps and checkpoints; the reverse sweep in
    FP64 or in FP32) on the finger length of the 400 x 42 channel (M = 10, Ca = 0.05, theta =
    60 deg, 4000 steps, checkpoint every 200): within 1e-3 relative of central finite
    differences of the FP32 forward path with a step of 1e-3 (relative for sigma, nu_R, nu_B;
    radians for theta), and within 2e-3 of the FP64 adjoint (a different map: the
    trajectories differ by rounding)."""
    lbcg = _lib()
    g, p = I.config_adjoint()
    n, k = 4000, 200

    def J(prm):
        L = lbcg.Lattice(g, prm, "fp32")
        L.step(n)
        o = L.observables()
        L.close()
        return o["x_tip"] - o["x_cl"]

    L = lbcg.Lattice(g, p, "fp32")
    out = L.adjoint(n, k, reverse_fp32=reverse == "fp32")
    L.close()
    L = lbcg.Lattice(g, p, "fp64")
    ref = L.adjoint(n, k)
    L.close()
    assert _close(out["J"], J(p), 1e-9)
    for key, field, d in (("dsigma", "sigma", 1e-3 * p.sigma), ("dnu_R", "nu_R", 1e-3 * p.nu_R),
                          ("dnu_B", "nu_B", 1e-3 * p.nu_B), ("dtheta", "theta", 1e-3)):
        fd = (J(I.Params(**{**p.__dict__, field: getattr(p, field) + d}))
              - J(I.Params(**{**p.__dict__, field: getattr(p, field) - d}))) / (2 * d)
        assert _close(out[key], fd, 1e-3), (key, out[key], fd)
        assert _close(out[key], ref[key], 2e-3), (key, out[key], ref[key])
    assert np.isfinite(out["dtheta_node"]).all()


def test_per_node_angle_gradient_at_the_adjoint_configuration():
    """dJ/d theta_i of the finger length on the 400 x 42 channel (M = 10, Ca = 0.05, theta =
    60 deg, 4000 FP64 steps, checkpoint every 200) at the three outermost fluid nodes where it
    is largest, against central finite differences of the forward CUDA path in which only that
    node's angle moves (step 1e-4 rad): within 1e-3 relative.  The per-node values also sum to
    the global-angle derivative."""
    lbcg = _lib()
    g, p = I.config_adjoint()
    n, k = 4000, 200
    L = lbcg.Lattice(g, p, "fp64")
    out = L.adjoint(n, k)
    L.close()
    dth = out["dtheta_node"]
    assert _close(float(dth.sum()), out["dtheta"], 1e-12, 1e-14)
    nodes = np.argsort(-np.abs(dth).ravel())[:3]

    def J(node, d):
        gg = I.Geometry(g.nx, g.ny, g.solid, g.rhoN0, bc_x=g.bc_x, bc_y=g.bc_y)
        th = np.full((g.ny, g.nx), p.theta)
        th.ravel()[node] += d
        gg.theta_node = th
        L = lbcg.Lattice(gg, p, "fp64")
        L.step(n)
        o = L.observables()
        L.close()
        return o["x_tip"] - o["x_cl"]

    h = 1e-4
    for node in nodes:
        fd = (J(node, h) - J(node, -h)) / (2 * h)
        assert _close(dth.ravel()[node], fd, 1e-3, 1e-9), (int(node), dth.ravel()[node], fd)
