"""The synthetic macroscale FE2 driver (host logic, CPU): hexahedral
kinematics and assembly against exact facts, and the outer loop with a
linear-elastic stand-in for the RVEs and with the FP64 oracle's RVE solves."""
import numpy as np

import oracle
import rve_inputs as ri
from paper_2305_07030_gb300 import macro as mc


def _linear(lam, mu):
    """Cauchy stress of a small-strain isotropic solid, per Gauss point."""
    def solve(F, F_uniform, n_gp):
        if F is None:
            F = np.tile(F_uniform, (n_gp, 1, 1))
        H = F - np.eye(3)
        eps = 0.5 * (H + np.transpose(H, (0, 2, 1)))
        tr = np.trace(eps, axis1=1, axis2=2)
        lam_ = np.broadcast_to(lam, (len(F),))
        mu_ = np.broadcast_to(mu, (len(F),))
        return lam_[:, None, None] * tr[:, None, None] * np.eye(3) + 2 * mu_[:, None, None] * eps
    return solve


def test_affine_patch_and_equilibrium_of_uniform_stress():
    m = mc.HexMesh(3, 2, 2, size=(1.5, 1.0, 1.0))
    assert m.n_gp == 96 and m.boundary.sum() == m.n_nodes - 2
    Fm = np.array([[1.02, 0.01, 0.0], [0.0, 0.99, 0.005], [0.003, 0.0, 1.01]])
    F = m.deformation_gradients(m.X @ (Fm - np.eye(3)).T)
    assert np.abs(F - Fm).max() <= 1e-14
    assert abs(m.wdetJ.sum() - 1.5) <= 1e-14  # the box volume
    sig = np.tile(np.array([[1.0, 0.2, 0.0], [0.2, 0.5, 0.1], [0.0, 0.1, 0.3]]), (m.n_gp, 1, 1))
    f = m.internal_forces(F, sig)
    # a uniform stress loads only the boundary; the forces balance
    assert np.abs(f[~m.boundary]).max() <= 1e-14
    assert np.abs(f.sum(axis=0)).max() <= 1e-14
    # traction on the x = 1.5 face: the face's total force is P n times its area
    J = np.linalg.det(Fm)
    P = J * sig[0] @ np.linalg.inv(Fm).T
    face = np.isclose(m.X[:, 0], 1.5)
    assert np.abs(f[face].sum(axis=0) - P[:, 0] * 1.0).max() <= 1e-13


def test_stiffness_is_symmetric_with_six_rigid_modes():
    m = mc.HexMesh(2, 2, 1)
    K = m.stiffness(1.3, 0.7)
    assert np.abs(K - K.T).max() <= 1e-12
    ev = np.linalg.eigvalsh(K)
    assert (np.abs(ev) <= 1e-10 * ev.max()).sum() == 6 and ev.min() > -1e-10


def test_outer_loop_converges_for_heterogeneous_linear_material():
    m = mc.HexMesh(3, 3, 3)
    rng = np.random.default_rng(3)
    lam = rng.uniform(0.5, 2.0, m.n_gp)
    mu = rng.uniform(0.3, 1.0, m.n_gp)
    solve = _linear(lam, mu)
    d = mc.FE2Driver(m, lambda F, Fu: solve(F, Fu, m.n_gp))
    # the fit sees the average response
    assert abs(d.lam - lam.mean()) <= 1e-9 and abs(d.mu - mu.mean()) <= 1e-9
    for k in range(3):
        rec = d.step(np.diag([1.0 + 0.01 * (k + 1), 1.0, 1.0]), tol=1e-10)
        assert rec["converged"], rec["residuals"]
        assert rec["residuals"][-1] < rec["residuals"][0]
    # a homogeneous material needs no correction of the affine field
    solve_h = _linear(np.full(m.n_gp, 1.2), np.full(m.n_gp, 0.6))
    d2 = mc.FE2Driver(m, lambda F, Fu: solve_h(F, Fu, m.n_gp))
    rec = d2.step(np.diag([1.02, 1.0, 1.0]), tol=1e-12)
    assert rec["outer"] == 1


class OracleRVEs:
    """solve_fn of FE2Driver with the FP64 oracle (affine start first, warm
    starts afterwards), for tests."""

    def __init__(self, nets, damping, tol=1e-8):
        self.nets, self.c, self.tol = nets, damping, tol
        self.u = None

    def __call__(self, F, F_uniform):
        if F is None:
            F = np.tile(F_uniform, (len(self.nets), 1, 1))
        out = []
        us = []
        for p, net in enumerate(self.nets):
            r = oracle.solve(net, F[p], self.c[p], tol=self.tol, init=2 if self.u else 1,
                             u_warm=self.u[p] if self.u else None)
            assert r["status"] == "OK"
            out.append(r["sigma"])
            us.append(r["u"])
        self.u = us
        return np.array(out)


def test_fe2_loop_with_oracle_rves():
    """A 2 x 2 x 2 mesh (one free node) whose 64 Gauss points each carry a
    small random fiber network: the macroscale loop converges and the
    interior node moves off the affine position when the RVEs differ."""
    m = mc.HexMesh(2, 2, 2)
    rng = np.random.default_rng(11)
    nets = [ri.random_network(60, rng) for _ in range(m.n_gp)]
    c = np.array([ri.default_damping(60) for _ in nets])
    d = mc.FE2Driver(m, OracleRVEs(nets, c, tol=1e-7))
    rec = d.step(np.diag([1.01, 1.0, 1.0]), tol=1e-5)
    assert rec["converged"], rec["residuals"]
    centre = ~m.boundary
    affine = m.X[centre] @ (np.diag([1.01, 1.0, 1.0]) - np.eye(3)).T
    assert np.abs(d.u[centre] - affine).max() > 1e-6
