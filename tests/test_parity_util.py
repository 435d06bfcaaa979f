"""CPU checks of the parity helpers the GPU tests rely on: the rounding family
of an oracle run and its diameter."""
import numpy as np

from parity_util import PERTURB_ULPS, family_diameter, mixed_bound, perturbations, ulp_steps


def test_perturbations_move_one_input_by_one_to_three_ulps():
    alpha, c = 0.9, 0.0011697
    pairs = perturbations(alpha, c)
    assert len(pairs) == 4 * PERTURB_ULPS == 12
    assert len(set(pairs)) == 12 and (alpha, c) not in pairs
    for a, cc in pairs:
        assert (a == alpha) != (cc == c)  # exactly one input moved
        x, x0 = (a, alpha) if a != alpha else (cc, c)
        k = round(abs(x - x0) / np.spacing(x0))
        assert 1 <= k <= PERTURB_ULPS and ulp_steps(x0, int(np.sign(x - x0)) * k) == x


def test_family_diameter_is_largest_pairwise_distance():
    base = np.diag([2.0, 0.0, 0.0])
    s1 = base + np.diag([1e-3, 0.0, 0.0])
    s2 = base - np.diag([2e-3, 0.0, 0.0])
    # |s1 - s2| = 3e-3 on a base norm of 2
    assert abs(family_diameter([base, s1, s2], base) - 1.5e-3) < 1e-15
    assert family_diameter([base], base) == 0.0


def test_mixed_bound_floor_is_the_stated_tolerance():
    assert mixed_bound(0.0) == 1e-5 and mixed_bound(3e-6) == 1e-5
    assert mixed_bound(4e-4) == 4e-4


def test_within_family_extends_only_when_needed():
    import rve_inputs as ri
    from parity_util import oracle_with_envelope, within_family
    rng = np.random.default_rng(3)
    net = ri.random_network(60, rng)
    F = ri.symmetric_perturbation(rng)
    c = ri.default_damping(60)
    base, diam = oracle_with_envelope(net, F, c)
    ok, err, bound = within_family(net, F, c, base["sigma"], base["sigma"], diam)
    assert ok and err == 0.0 and bound == max(1e-5, diam)
    far = base["sigma"] * (1.0 + 0.05)
    ok, err, bound = within_family(net, F, c, far, base["sigma"], diam)
    assert not ok and abs(err - 0.05) < 1e-12 and bound >= max(1e-5, diam)
