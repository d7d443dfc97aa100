"""Pins of the oracle's single formulas against what the lattice and the
mathematics fix (no GPU).

* the D3Q19 table against the paper's stencil figure caption (tests/golden);
* lattice isotropy (textbook moments of the D3Q19 weights);
* Eq. equilibrium: its moments are exactly rho, rho u, rho/3 I + rho u u;
* Eq. forceterm (Luo): zeroth moment 0, first moment rho a, second moment
  rho (u a + a u) -- this fixes the garbled printed form (a missing c_i factor).
"""
import itertools
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _stencil_fixture():
    rows = []
    for line in open(os.path.join(GOLDEN, "d3q19_stencil.txt")):
        line = line.split("#")[0].strip()
        if not line:
            continue
        i, name, cx, cy, cz, w = line.split()
        rows.append((int(i), name, (int(cx), int(cy), int(cz)), float(Fraction(w))))
    return rows


def test_stencil_matches_caption():
    c, w, opp = oracle.lattice()
    rows = _stencil_fixture()
    assert len(rows) == 19
    for i, name, cv, wv in rows:
        assert tuple(c[i]) == cv, name
        assert w[i] == pytest.approx(wv, abs=0, rel=1e-15), name
    for q in range(19):
        assert tuple(c[opp[q]]) == tuple(-c[q])


def test_lattice_isotropy():
    c, w, _ = oracle.lattice()
    c = c.astype(float)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.abs((w[:, None] * c).sum(0)).max() < 1e-16
    m2 = np.einsum("q,qa,qb->ab", w, c, c)
    assert np.abs(m2 - np.eye(3) / 3.0).max() < 1e-15
    m3 = np.einsum("q,qa,qb,qc->abc", w, c, c, c)
    assert np.abs(m3).max() < 1e-16
    m4 = np.einsum("q,qa,qb,qc,qd->abcd", w, c, c, c, c)
    d = np.eye(3)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) + np.einsum("ad,bc->abcd", d, d)) / 9.0
    assert np.abs(m4 - iso).max() < 1e-15


def _rand_states(n=50, seed=7):
    rng = np.random.default_rng(seed)
    for _ in range(n):
        yield 0.9 + 0.2 * rng.random(), 0.05 * (rng.random(3) - 0.5), 1e-4 * (rng.random(3) - 0.5)


def test_equilibrium_moments():
    c, _, _ = oracle.lattice()
    c = c.astype(float)
    for rho, u, _ in _rand_states():
        f = oracle.feq(rho, u)
        assert abs(f.sum() - rho) <= 4e-16 * rho
        assert np.abs(c.T @ f - rho * u).max() <= 4e-16
        pi = np.einsum("qa,qb,q->ab", c, c, f)
        assert np.abs(pi - (rho / 3.0 * np.eye(3) + rho * np.outer(u, u))).max() <= 4e-16


def test_equilibrium_at_rest_is_weights():
    _, w, _ = oracle.lattice()
    f = oracle.feq(1.25, (0.0, 0.0, 0.0))
    assert np.array_equal(f, 1.25 * w)


def test_force_term_moments():
    c, _, _ = oracle.lattice()
    c = c.astype(float)
    for rho, u, a in _rand_states():
        F = oracle.force_term(rho, u, a)
        assert abs(F.sum()) <= 1e-19
        assert np.abs(c.T @ F - rho * a).max() <= 1e-19
        m2 = np.einsum("qa,qb,q->ab", c, c, F)
        assert np.abs(m2 - rho * (np.outer(u, a) + np.outer(a, u))).max() <= 1e-19


def test_force_term_mutation_is_caught():
    """Dropping the (c.u) c / c_s^4 part (a plausible misreading of the garbled
    Eq. forceterm) breaks the second moment."""
    oracle.set_mutation(3)
    c, _, _ = oracle.lattice()
    c = c.astype(float)
    rho, u, a = 1.0, np.array([0.02, -0.01, 0.03]), np.array([0.0, 0.0, -1e-4])
    F = oracle.force_term(rho, u, a)
    m2 = np.einsum("qa,qb,q->ab", c, c, F)
    assert np.abs(m2 - rho * (np.outer(u, a) + np.outer(a, u))).max() > 1e-7
