"""Pins of the oracle's lattice, equilibrium and forced collision against
exact identities (Sec. 2.1, Fig. 1(b), Eqs. 2-3, Eqs. 10-12)."""
from fractions import Fraction
from itertools import product

import numpy as np
import pytest

from oracle import oracle as O


def _frac_weights(w):
    out = []
    for x in w:
        f = Fraction(x).limit_denominator(100)
        assert abs(float(f) - x) < 1e-15
        out.append(f)
    return out


def test_d3q19_velocity_set():
    e, w, opp = O.lattice()
    vecs = {tuple(v) for v in e}
    assert len(vecs) == 19
    expected = {(0, 0, 0)}
    for v in product((-1, 0, 1), repeat=3):
        n = sum(abs(c) for c in v)
        if n in (1, 2):
            expected.add(v)
    assert vecs == expected  # rest + 6 axes + 12 face diagonals, no corners
    for i in range(19):
        assert tuple(e[opp[i]]) == tuple(-e[i])


def test_weights_isotropy_exact():
    """Sum w = 1, sum w e = 0, sum w e_a e_b = c_s^2 delta, fourth-order
    isotropy sum w e_a e_b e_c e_d = c_s^4 (dd + dd + dd), c_s^2 = 1/3."""
    e, w, _ = O.lattice()
    W = _frac_weights(w)
    cs2 = Fraction(1, 3)
    assert sum(W) == 1
    for a in range(3):
        assert sum(W[i] * int(e[i, a]) for i in range(19)) == 0
    d = lambda a, b: 1 if a == b else 0
    for a, b in product(range(3), repeat=2):
        assert sum(W[i] * int(e[i, a]) * int(e[i, b]) for i in range(19)) == cs2 * d(a, b)
    for a, b, c in product(range(3), repeat=3):
        assert sum(W[i] * int(e[i, a]) * int(e[i, b]) * int(e[i, c]) for i in range(19)) == 0
    for a, b, c, dd in product(range(3), repeat=4):
        lhs = sum(W[i] * int(e[i, a] * e[i, b] * e[i, c] * e[i, dd]) for i in range(19))
        rhs = cs2 * cs2 * (d(a, b) * d(c, dd) + d(a, c) * d(b, dd) + d(a, dd) * d(b, c))
        assert lhs == rhs, (a, b, c, dd)


@pytest.mark.parametrize("seed", range(5))
def test_equilibrium_moments(seed):
    """Eq. 2 reproduces rho, rho u and rho (c_s^2 delta + u u) exactly."""
    rng = np.random.default_rng(seed)
    e, _, _ = O.lattice()
    rho = rng.uniform(0.01, 8.0)
    u = rng.uniform(-0.2, 0.2, 3)
    f = O.feq(rho, u)
    assert f.sum() == pytest.approx(rho, rel=1e-14)
    np.testing.assert_allclose(f @ e, rho * u, rtol=0, atol=1e-14 * rho)
    P = np.einsum("i,ia,ib->ab", f, e, e)
    np.testing.assert_allclose(P, rho * (np.eye(3) / 3.0 + np.outer(u, u)), atol=1e-14 * rho)


def test_equilibrium_at_rest_is_weights():
    _, w, _ = O.lattice()
    np.testing.assert_array_equal(O.feq(2.5, [0.0, 0.0, 0.0]), w * 2.5)


@pytest.mark.parametrize("tau", [1.0, 0.8, 1.7])
def test_exact_difference_forcing_moments(tau):
    """Eqs. 10-12: collision keeps the mass and adds exactly F to the
    momentum; at equilibrium input the output is feq(rho, u + F/rho); with
    F = 0 the non-equilibrium part shrinks by (1 - 1/tau)."""
    rng = np.random.default_rng(3)
    e, _, _ = O.lattice()
    for _ in range(20):
        rho = rng.uniform(0.05, 7.0)
        u = rng.uniform(-0.1, 0.1, 3)
        F = rng.uniform(-0.05, 0.05, 3) * rho
        fin = O.feq(rho, u) * (1.0 + rng.uniform(-0.2, 0.2, 19))
        r = fin.sum()
        uu = (fin @ e) / r
        out = O.collide(tau, r, uu, F, fin)
        assert out.sum() == pytest.approx(r, rel=1e-13)
        np.testing.assert_allclose(out @ e, r * uu + F, atol=1e-13 * r)
        eq_in = O.feq(rho, u)
        np.testing.assert_allclose(O.collide(tau, rho, u, F, eq_in), O.feq(rho, u + F / rho),
                                   atol=1e-14 * rho)
        zero = np.zeros(3)
        np.testing.assert_allclose(O.collide(tau, r, uu, zero, fin) - O.feq(r, uu),
                                   (1.0 - 1.0 / tau) * (fin - O.feq(r, uu)), atol=1e-14 * r)


def test_paper_stated_parameters():
    """The numbers the paper states for the method (tests/golden)."""
    import json
    import os
    from paper_1510_03560_gb300 import workloads as W
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_params.json")) as fh:
        g = json.load(fh)
    assert W.PHYSICS["beta"] == g["beta"]["value"]
    e, w, _ = O.lattice()
    assert (w * e[:, 0] ** 2).sum() == pytest.approx(g["cs2"]["value"], rel=1e-15)
    assert g["S"]["value"] == 0.0
