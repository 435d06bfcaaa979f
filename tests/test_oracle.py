"""Pins of the FP64 oracle against facts that do not come from the oracle.

Every test here checks the oracle (oracle/dr_oracle.c, Algorithm 1 of the
paper in serial scatter form) against a closed form, an invariant, an exact
rational recurrence or an independent solver, chosen so that a dropped term,
a sign or index slip, or a swapped update order fails at least one of them.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import rve_inputs as ri

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _net(X, elems, EA, fixed):
    return ri.Network(X=np.asarray(X, float), elems=np.asarray(elems, np.int32),
                      EA=np.asarray(EA, float), fixed=np.asarray(fixed, np.uint8))


# ---------------------------------------------------------------------------
# element-level pins: force law, energy, mass, time step
# ---------------------------------------------------------------------------

def test_force_is_negative_energy_gradient():
    """g = -dW/dx with W = sum 1/2 EA L (l/L - 1)^2 (central differences)."""
    rng = np.random.default_rng(1)
    net = ri.random_network(60, rng)
    L = oracle.ref_lengths(net.X, net.elems)
    x = net.X + 0.03 * rng.standard_normal(net.X.shape)
    g = oracle.internal_forces(x, net.elems, net.EA, L)
    h = 1e-6
    fd = np.zeros_like(x)
    for i in range(x.shape[0]):
        for r in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, r] += h
            xm[i, r] -= h
            fd[i, r] = -(oracle.strain_energy(xp, net.elems, net.EA, L) -
                         oracle.strain_energy(xm, net.elems, net.EA, L)) / (2 * h)
    assert np.abs(g - fd).max() <= 1e-7 * np.abs(g).max()


def test_action_reaction_and_rest_state():
    """Internal forces sum to zero at any configuration; zero at rest."""
    rng = np.random.default_rng(2)
    net = ri.random_network(300, rng)
    L = oracle.ref_lengths(net.X, net.elems)
    assert np.all(oracle.internal_forces(net.X, net.elems, net.EA, L) == 0.0)
    x = net.X + 0.05 * rng.standard_normal(net.X.shape)
    g = oracle.internal_forces(x, net.elems, net.EA, L)
    d = x[net.elems[:, 1]] - x[net.elems[:, 0]]
    l = np.linalg.norm(d, axis=1)
    scale = np.abs(net.EA * (l / L - 1)).sum()
    assert np.abs(g.sum(axis=0)).max() <= 1e-14 * scale
    # a rigid rotation and translation of the reference state is force free
    th = 0.3
    R = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    g_rot = oracle.internal_forces(net.X @ R.T + 0.7, net.elems, net.EA, L)
    assert np.abs(g_rot).max() <= 1e-13 * net.EA.max()


def test_two_node_force_by_hand():
    """A single bar stretched from L = 2 to l = 3 along y: N = EA/2, node a is
    pulled toward b with force N, node b toward a."""
    X = np.array([[0.0, 0.0, 0.0], [0.0, 2.0, 0.0]])
    x = np.array([[0.0, 0.0, 0.0], [0.0, 3.0, 0.0]])
    g = oracle.internal_forces(x, np.array([[0, 1]]), np.array([4.0]),
                               oracle.ref_lengths(X, np.array([[0, 1]])))
    assert np.array_equal(g, np.array([[0, 2.0, 0], [0, -2.0, 0]]))


def test_masses_and_time_step():
    """Lumped masses m_i = sum EA/(2L); the critical step of an axial bar with
    rho*A = EA/L^2 is one, so the step is the safety factor."""
    rng = np.random.default_rng(3)
    net = ri.random_network(200, rng)
    L = oracle.ref_lengths(net.X, net.elems)
    m = oracle.masses(net.n_nodes, net.elems, net.EA, L)
    assert math.isclose(m.sum(), float((net.EA / L).sum()), rel_tol=1e-13)
    deg_mass = np.zeros(net.n_nodes)
    for (a, b), ea, l in zip(net.elems, net.EA, L):
        deg_mass[a] += ea / (2 * l)
        deg_mass[b] += ea / (2 * l)
    assert np.allclose(m, deg_mass, rtol=1e-14, atol=0)
    assert math.isclose(oracle.time_step(net.EA, L, 0.9), 0.9, rel_tol=1e-15)
    assert math.isclose(oracle.time_step(net.EA, L, 0.5), 0.5, rel_tol=1e-15)


# ---------------------------------------------------------------------------
# solver pins
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("init", [0, 1])
def test_identity_F_gives_zero_stress(init):
    """F = I: the reference state is force free, so f_ref = 0, the first
    residual is exactly 0 and the stress is exactly 0."""
    rng = np.random.default_rng(4)
    net = ri.random_network(150, rng)
    r = oracle.solve(net, np.eye(3), 0.002, init=init)
    assert r["status"] == "OK" and r["iters"] == 1
    assert r["f_ref"] == 0.0 and r["rel_res"] == 0.0
    assert np.all(r["sigma"] == 0.0)
    assert np.all(r["u"] == 0.0)


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


@pytest.mark.parametrize("init", [0, 1])
def test_cubic_lattice_uniaxial_closed_form(init):
    """Regular m^3 lattice of unit EA bars under F = diag(lam,1,1): the affine
    state is the equilibrium and sigma_xx = m^2 EA (lam - 1), rest zero."""
    case = _golden("cubic_lattice.json")["uniaxial"]
    m, lam = case["m"], case["lambda"]
    net = ri.cubic_lattice(m)
    F = np.diag([lam, 1.0, 1.0])
    r = oracle.solve(net, F, 0.05, init=init)
    assert r["status"] == "OK"
    s = r["sigma"]
    assert math.isclose(s[0, 0], case["sigma_xx"], rel_tol=1e-7)
    assert np.abs(s - np.diag([s[0, 0], 0, 0])).max() <= 1e-7 * case["sigma_xx"]
    # the equilibrium is the affine state
    assert np.abs(net.X + r["u"] - net.X @ F.T).max() <= 1e-7


def test_series_chains_closed_form():
    """Independent x-chains with EA depending on the bar's x-index only.
    An interior chain carries N_c = (lam-1)/(h sum 1/EA_i); a chain lying in a
    fixed face is stretched affinely. sigma_xx = n_int N_c + n_face (lam-1) h
    sum EA_i."""
    case = _golden("cubic_lattice.json")["series_chains"]
    m, lam, EA_x = case["m"], case["lambda"], np.array(case["EA_x"])
    net = ri.cubic_lattice(m, bars="x", EA_x=EA_x)
    F = np.diag([lam, 1.0, 1.0])
    h = 1.0 / (m - 1)
    n_face = m * m - (m - 2) ** 2
    n_int = (m - 2) ** 2
    Nc = (lam - 1) / (h * (1.0 / EA_x).sum())
    expect = n_int * Nc + n_face * (lam - 1) * h * EA_x.sum()
    assert math.isclose(expect, case["sigma_xx"], rel_tol=1e-12)
    for init in (0, 1):
        r = oracle.solve(net, F, 0.1, init=init, tol=1e-10)
        assert r["status"] == "OK"
        s = r["sigma"]
        assert math.isclose(s[0, 0], expect, rel_tol=1e-8), (s[0, 0], expect)
        assert np.abs(s - np.diag([s[0, 0], 0, 0])).max() <= 1e-9 * expect


def _chain_exact(k, lam, EA1, EA2, c, dt):
    """Exact rational trajectory of one free node between two fixed nodes on
    the x-axis (L1 = L2 = 1/2), written as the leapfrog recurrence
    x_{n+1} = x_n + dt w_n, w_{n+1} = (1 - c dt) w_n + dt g(x_{n+1})/m with the
    half-step velocity w_0 = dt/2 g(x_0)/m. Returns positions and residuals."""
    L = Fraction(1, 2)
    x2 = lam
    m = EA1 / (2 * L) + EA2 / (2 * L)

    def g(x1):
        return EA2 * ((x2 - x1) / L - 1) - EA1 * (x1 / L - 1)

    x = lam * Fraction(1, 2)
    w = dt / 2 * g(x) / m
    xs, rs = [], []
    for _ in range(k):
        x = x + dt * w
        gx = g(x)
        xs.append(x)
        rs.append(gx)
        w = (1 - c * dt) * w + dt * gx / m
    return xs, rs


def test_one_dof_chain_exact_trajectory():
    """The oracle's free-node position after k iterations equals the exact
    rational leapfrog recurrence (affine start, damping on the half-step
    velocity), and it stops at the first residual below tol * f_ref."""
    lam, EA1, EA2, c = Fraction(11, 10), Fraction(1), Fraction(2), Fraction(1, 8)
    dt = Fraction(0.9)  # the double nearest 0.9, as the oracle uses it
    X = [[0, 0, 0], [0.5, 0, 0], [1.0, 0, 0]]
    net = _net(X, [[0, 1], [1, 2]], [1.0, 2.0], [1, 0, 1])
    F = np.diag([1.1, 1.0, 1.0])
    xs, rs = _chain_exact(60, lam, EA1, EA2, c, dt)
    for k in (1, 2, 3, 10, 60):
        r = oracle.solve(net, F, 0.125, init=1, max_iter=k, tol=1e-300)
        assert r["iters"] == k
        assert math.isclose(net.X[1, 0] + r["u"][1, 0], float(xs[k - 1]), rel_tol=1e-13,
                            abs_tol=1e-15)
        assert np.all(r["u"][1, 1:] == 0.0)
    # stopping rule: f_ref = ||g(F X)|| over all DOFs = sqrt(0.1^2+0.1^2+0.2^2)
    tol = 1e-6
    fref = math.sqrt(0.06)
    xs, rs = _chain_exact(400, lam, EA1, EA2, c, dt)
    k_stop = next(i + 1 for i, g in enumerate(rs) if abs(float(g)) <= tol * fref)
    r = oracle.solve(net, F, 0.125, init=1, tol=tol)
    assert r["status"] == "OK"
    assert math.isclose(r["f_ref"], fref, rel_tol=1e-14)
    assert r["iters"] == k_stop
    # the converged free node sits where the two bar forces balance
    x_eq = 3.4 / 6.0
    assert abs(net.X[1, 0] + r["u"][1, 0] - x_eq) <= 2e-6


def test_kinetic_energy_exact_on_one_dof_chain():
    """Algorithm 1's optional kinetic energy 1/2 sum m v^2 uses the full-step
    velocity v_k = w + dt/2 a_k, a_k = (g(x_k) - c m w)/m, after the half-step
    velocity w has moved the node to x_k. On the one-DOF chain this is exact
    rational arithmetic; the oracle must match it."""
    lam, EA1, EA2, c = Fraction(11, 10), Fraction(1), Fraction(2), Fraction(1, 8)
    dt = Fraction(0.9)
    L, x2 = Fraction(1, 2), lam
    m = EA1 / (2 * L) + EA2 / (2 * L)

    def g(x1):
        return EA2 * ((x2 - x1) / L - 1) - EA1 * (x1 / L - 1)

    x = lam * Fraction(1, 2)
    w = dt / 2 * g(x) / m
    kes = []
    for _ in range(60):
        x = x + dt * w
        gx = g(x)
        v_full = w + dt / 2 * (gx / m - c * w)
        kes.append(m * v_full * v_full / 2)
        w = (1 - c * dt) * w + dt * gx / m
    X = [[0, 0, 0], [0.5, 0, 0], [1.0, 0, 0]]
    net = _net(X, [[0, 1], [1, 2]], [1.0, 2.0], [1, 0, 1])
    F = np.diag([1.1, 1.0, 1.0])
    for k in (1, 2, 3, 10, 60):
        r = oracle.solve(net, F, 0.125, init=1, max_iter=k, tol=1e-300, want_ke=True)
        assert r["iters"] == k
        assert math.isclose(r["ke"], float(kes[k - 1]), rel_tol=1e-12, abs_tol=1e-300), \
            (k, r["ke"], float(kes[k - 1]))
    # without the flag the energy is not tracked
    assert oracle.solve(net, F, 0.125, init=1, max_iter=3, tol=1e-300)["ke"] == 0.0


def _chain_energy_exact(k, lam, EA1, EA2, c, dt):
    """Exact rational quantities of the one-DOF chain after k iterations: the
    stored elastic energy change W(x_k) - W(x_0) (W = sum 1/2 EA L (l/L - 1)^2;
    the bars stay on the x-axis, so W is quadratic in x and the trapezoid rule
    of the oracle's work sum is exact for it), and the terms of the leapfrog's
    discrete energy identity
        1/2 m w_{k+1}^2 - 1/2 m w_1^2
            = -Wint + Wext + 1/2 (g_k + f_k) du_{k+1} - 1/2 g_0 du_1,
    with w_n the half-step velocity of step n, du_n = dt w_n, f_n = -c m w_n.
    The identity follows from m (w_{n+1} - w_n) = dt (g_n + f_n) times
    (w_{n+1} + w_n)/2, summed by parts; it fixes Wext given Wint."""
    L = Fraction(1, 2)
    x2 = lam
    m = EA1 / (2 * L) + EA2 / (2 * L)

    def g(x1):
        return EA2 * ((x2 - x1) / L - 1) - EA1 * (x1 / L - 1)

    def W(x1):
        return EA1 * L * (x1 / L - 1) ** 2 / 2 + EA2 * L * ((x2 - x1) / L - 1) ** 2 / 2

    x0 = lam * Fraction(1, 2)
    g0 = g(x0)
    w1 = dt / 2 * g0 / m
    x, w = x0, w1
    for _ in range(k):
        x = x + dt * w
        gx = g(x)
        f = -c * m * w
        w_next = w + dt * (gx + f) / m
        w, g_last, f_last = w_next, gx, f
    wint = W(x) - W(x0)
    wext = m * w * w / 2 - m * w1 * w1 / 2 + wint - (g_last + f_last) * dt * w / 2 + g0 * dt * w1 / 2
    return wint, wext


def test_energy_balance_terms_exact_on_one_dof_chain():
    """Algorithm 1's optional energy check, internal and external work: on the
    one-DOF chain the internal work is the exact change of stored energy and
    the damping work closes the leapfrog's discrete energy identity."""
    lam, EA1, EA2, c = Fraction(11, 10), Fraction(1), Fraction(2), Fraction(1, 8)
    dt = Fraction(0.9)
    X = [[0, 0, 0], [0.5, 0, 0], [1.0, 0, 0]]
    net = _net(X, [[0, 1], [1, 2]], [1.0, 2.0], [1, 0, 1])
    F = np.diag([1.1, 1.0, 1.0])
    for k in (1, 2, 3, 10, 60):
        wint, wext = _chain_energy_exact(k, lam, EA1, EA2, c, dt)
        r = oracle.solve(net, F, 0.125, init=1, max_iter=k, tol=1e-300, want_energy=True)
        assert r["iters"] == k
        assert math.isclose(r["wint"], float(wint), rel_tol=1e-11, abs_tol=1e-17), (k, r["wint"], wint)
        assert math.isclose(r["wext"], float(wext), rel_tol=1e-9, abs_tol=1e-17), (k, r["wext"], wext)
        assert r["wext"] < 0.0  # damping only removes energy
    # the work sums are tracked only on request
    r = oracle.solve(net, F, 0.125, init=1, max_iter=3, tol=1e-300, want_ke=True)
    assert r["wint"] == 0.0 and r["wext"] == 0.0


def test_energy_balance_terms_on_a_random_network():
    """Without damping the external work is zero; the internal work follows
    the stored energy sum(1/2 EA L (l/L - 1)^2) of the nonlinear network to
    the trapezoid rule's accuracy at this time step."""
    rng = np.random.default_rng(5)
    net = ri.random_network(300, rng)
    F = ri.symmetric_perturbation(rng)
    a, b = net.elems[:, 0], net.elems[:, 1]
    L = np.linalg.norm(net.X[b] - net.X[a], axis=1)

    def W(x):
        l = np.linalg.norm(x[b] - x[a], axis=1)
        return float(np.sum(0.5 * net.EA * L * (l / L - 1.0) ** 2))

    x0 = net.X @ F.T
    for c, k in ((0.0, 400), (ri.default_damping(300), 3000)):
        r = oracle.solve(net, F, c, init=1, max_iter=k, want_energy=True)
        dW = W(net.X + r["u"]) - W(x0)
        assert abs(r["wint"] - dW) <= 1e-2 * abs(dW), (c, r["wint"], dW)
        if c == 0.0:
            assert r["wext"] == 0.0
        else:
            assert r["wext"] < 0.0


def test_status_maxiter_and_nan():
    rng = np.random.default_rng(5)
    net = ri.random_network(120, rng)
    F = np.diag([1.03, 1.0, 0.99])
    r = oracle.solve(net, F, 0.002, init=1, max_iter=7)
    assert r["status"] == "MAXITER" and r["iters"] == 7
    Fn = F.copy()
    Fn[0, 1] = np.nan
    r = oracle.solve(net, Fn, 0.002, init=1, max_iter=50)
    assert r["status"] == "NAN" and r["iters"] == 1


def test_balance_and_virial_equals_boundary_stress():
    """At convergence the free nodes balance to tol * f_ref; the virial stress
    equals the boundary-reaction stress and is symmetric."""
    rng = np.random.default_rng(6)
    net = ri.random_network(250, rng)
    F = ri.symmetric_perturbation(rng)
    tol = 1e-10
    r = oracle.solve(net, F, ri.default_damping(250), init=1, tol=tol)
    assert r["status"] == "OK"
    L = oracle.ref_lengths(net.X, net.elems)
    x = net.X + r["u"]
    g = oracle.internal_forces(x, net.elems, net.EA, L)
    free = net.fixed == 0
    assert np.linalg.norm(g[free]) <= tol * r["f_ref"] * (1 + 1e-9)
    sv = oracle.stress_virial(x, net.elems, net.EA, L, F)
    sb = oracle.stress_boundary(x, g, net.fixed, F)
    assert np.allclose(sv, r["sigma"], rtol=0, atol=1e-15 * np.abs(sv).max())
    assert np.abs(sv - sv.T).max() <= 1e-15 * np.abs(sv).max()
    assert np.abs(sv - sb).max() <= 1e-6 * np.abs(sv).max()


def test_newton_equilibrium_on_rigid_truss():
    """A braced (triangulated) lattice is rigid: Newton's method from the
    affine state finds its equilibrium independently of the dynamics, and
    dynamic relaxation reaches the same state and stress."""
    net = ri.braced_lattice(4)
    rng = np.random.default_rng(7)
    F = ri.symmetric_perturbation(rng, 0.03)
    u_aff = net.X @ F.T - net.X
    u_n, it, last = oracle.newton(net, u_aff, max_it=30, step_tol=1e-14)
    assert it <= 8 and last <= 1e-14
    L = oracle.ref_lengths(net.X, net.elems)
    g = oracle.internal_forces(net.X + u_n, net.elems, net.EA, L)
    assert np.abs(g[net.fixed == 0]).max() <= 1e-13
    tol = 1e-11
    r = oracle.solve(net, F, 0.05, init=1, tol=tol)
    assert r["status"] == "OK"
    assert np.abs(r["u"] - u_n).max() <= 1e-9
    s_n = oracle.stress_virial(net.X + u_n, net.elems, net.EA, L, F)
    assert np.abs(r["sigma"] - s_n).max() <= 1e-9 * np.abs(s_n).max()
    # Newton started from the relaxed state corrects it by a tolerance-size step
    _, it2, _ = oracle.newton(net, r["u"], max_it=1, step_tol=0.0)
    u_c, _, last2 = oracle.newton(net, r["u"], max_it=1, step_tol=0.0)
    assert last2 <= 1e-9


def test_newton_converges_quadratically_on_random_dense_network():
    """Tiny random network with k = 8 neighbours: Newton converges from the
    relaxed state in a handful of steps (a full-rank free tangent)."""
    rng = np.random.default_rng(8)
    X = rng.random((30, 3))
    el = ri.knn_edges(X, 8)
    net = _net(X, el, np.ones(len(el)), ri.boundary_flags(X, 0.2))
    F = np.diag([1.02, 1.0, 0.99])
    r = oracle.solve(net, F, 0.05, init=1, tol=1e-9)
    assert r["status"] == "OK"
    u_n, it, last = oracle.newton(net, r["u"], max_it=20, step_tol=1e-14)
    assert it <= 6 and last <= 1e-14
    L = oracle.ref_lengths(net.X, net.elems)
    s_n = oracle.stress_virial(net.X + u_n, net.elems, net.EA, L, F)
    assert np.abs(r["sigma"] - s_n).max() <= 1e-7 * np.abs(s_n).max()


def test_objectivity_affine_start():
    """sigma(R F) = R sigma(F) R^T for a rotation R (affine start; the
    trajectories differ only by rounding)."""
    rng = np.random.default_rng(9)
    net = ri.random_network(200, rng)
    F = ri.symmetric_perturbation(rng)
    th = 0.2
    R = np.array([[1, 0, 0], [0, math.cos(th), -math.sin(th)], [0, math.sin(th), math.cos(th)]])
    c = ri.default_damping(200)
    s1 = oracle.solve(net, F, c, init=1)["sigma"]
    s2 = oracle.solve(net, R @ F, c, init=1)["sigma"]
    assert np.abs(s2 - R @ s1 @ R.T).max() <= 1e-6 * np.abs(s1).max()


def test_warm_start_from_converged_state():
    """Restarting from a converged displacement (v = 0) needs few iterations
    and returns the same stress."""
    rng = np.random.default_rng(10)
    net = ri.random_network(200, rng)
    F = ri.symmetric_perturbation(rng)
    c = ri.default_damping(200)
    r1 = oracle.solve(net, F, c, init=1, tol=1e-9)
    r2 = oracle.solve(net, F, c, init=2, u_warm=r1["u"], tol=1e-8)
    assert r2["status"] == "OK" and r2["iters"] < r1["iters"] // 10
    assert np.abs(r2["sigma"] - r1["sigma"]).max() <= 1e-6 * np.abs(r1["sigma"]).max()


def test_batch_matches_single():
    w = ri.uneven_rves(6, 40, 120, workload=4)
    out = oracle.solve_batch(w, init=1, threads=3)
    for p in range(w.n_rve):
        r = oracle.solve(w.nets[p], w.F[p], w.damping[p], init=1)
        assert r["iters"] == out[p]["iters"]
        assert np.array_equal(r["sigma"], out[p]["sigma"])
