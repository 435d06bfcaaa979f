"""CPU checks of the algebraic identities the mixed-precision kernels rest on
(the kernels evaluate element forces in these rearranged forms; the oracle
uses the plain force law N = EA (l/L - 1), t = (N/l) d):

- displacement form of the lead kernel: with D = X_b - X_a, du = u_b - u_a,
  d = D + du, h = du . (D + d) = l^2 - L^2, the axial force over length is
  N/l = (EA/L) h / (l (l + L)), free of the cancellation in l/L - 1;
- increment form of the FP32 kernel: about a reference vector d_ref with
  q_ref = EA (1/L - 1/l_ref), the force t(d_ref + dd) equals
  t(d_ref) + q_ref dd + dq (d_ref + dd) with dq = EA h / (l l_ref (l + l_ref)),
  h = 2 d_ref . dd + dd . dd, exactly in real arithmetic.
Checked in FP64 on random elements against the plain law, and with h in
exact rationals and the square roots in 60-digit decimals where FP64
rounding would hide a slip."""
from fractions import Fraction

import numpy as np


def _plain(EA, L, d):
    l = np.linalg.norm(d, axis=-1)
    return (EA * (l / L - 1.0) / l)[..., None] * d


def test_displacement_form_matches_the_force_law():
    rng = np.random.default_rng(5)
    n = 2000
    D = rng.normal(size=(n, 3)) * 0.05
    L = np.linalg.norm(D, axis=1)
    EA = rng.lognormal(0.0, 0.3, n)
    for scale in (1e-2, 1e-5, 1e-9):
        du = rng.normal(size=(n, 3)) * scale * L[:, None]
        d = D + du
        l = np.linalg.norm(d, axis=1)
        h = np.einsum("ij,ij->i", du, D + d)
        q = EA / L * h / (l * (l + L))
        t = q[:, None] * d
        ref = _plain(EA, L, d)
        # the plain law loses ~|log10(strain)| digits to cancellation; the
        # displacement form does not, so they agree to the plain law's error
        err = np.abs(t - ref).max() / np.abs(ref).max()
        assert err <= 1e-15 / scale + 1e-12, (scale, err)


def test_increment_form_is_exact_in_rational_arithmetic():
    rng = np.random.default_rng(6)
    for _ in range(20):
        dref = [Fraction(int(x), 1000) for x in rng.integers(-90, 90, 3)]
        dd = [Fraction(int(x), 100000) for x in rng.integers(-90, 90, 3)]
        if all(x == 0 for x in dref):
            continue
        EA, L = Fraction(int(rng.integers(1, 9)), 4), Fraction(int(rng.integers(1, 9)), 100)
        lref2 = sum(x * x for x in dref)
        d = [a + b for a, b in zip(dref, dd)]
        l2 = sum(x * x for x in d)
        h = 2 * sum(a * b for a, b in zip(dref, dd)) + sum(b * b for b in dd)
        assert h == l2 - lref2
        # q(l) - q(l_ref) = EA (1/l_ref - 1/l) = EA h / (l l_ref (l + l_ref))
        import decimal
        decimal.getcontext().prec = 60
        sq = lambda f: decimal.Decimal(f.numerator) / decimal.Decimal(f.denominator)  # noqa: E731
        l, lref = sq(l2).sqrt(), sq(lref2).sqrt()
        EAd, Ld = sq(EA), sq(L)
        qref = EAd * (1 / Ld - 1 / lref)
        q = EAd * (1 / Ld - 1 / l)
        dq = EAd * sq(h) / (l * lref * (l + lref))
        for c in range(3):
            lhs = q * sq(d[c])
            rhs = qref * sq(dref[c]) + qref * sq(dd[c]) + dq * sq(d[c])
            assert abs(lhs - rhs) <= decimal.Decimal(10) ** -50 * (abs(lhs) + 1)
