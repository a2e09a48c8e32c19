"""Pins for the oracle's matrix sign function (Eq. 13) and Gershgorin bounds.

Each check is independent of the oracle's own formula: a closed form, an
invariant that only the true sign satisfies, or a different algorithm.
"""

import numpy as np
import pytest

import oracle as O
from synth import spectrum_matrix


def _closed_form_sign_2x2(a, c, d):
    # symmetric [[a, c], [c, d]]: eigenvalues m +- r, m = (a+d)/2, r = sqrt(((a-d)/2)^2 + c^2)
    m = 0.5 * (a + d)
    r = np.hypot(0.5 * (a - d), c)
    if abs(m) < r:
        return (np.array([[a, c], [c, d]]) - m * np.eye(2)) / r
    return np.sign(m) * np.eye(2)


def test_sign_2x2_closed_form():
    rng = np.random.default_rng(11)
    n_mixed = 0
    for _ in range(400):
        a, c, d = rng.normal(size=3) * rng.choice([0.1, 1.0, 5.0])
        s, _ = O.sign_eig(np.array([[a, c], [c, d]]))
        ref = _closed_form_sign_2x2(a, c, d)
        n_mixed += abs(0.5 * (a + d)) < np.hypot(0.5 * (a - d), c)
        assert np.max(np.abs(s - ref)) < 1e-13
    assert 50 < n_mixed < 400  # both branches exercised


def test_sign_2x2_hand_values():
    # [[1, 2], [2, 1]] has eigenvalues 3 and -1: sign = [[0, 1], [1, 0]]
    s, lam = O.sign_eig(np.array([[1.0, 2.0], [2.0, 1.0]]))
    assert np.allclose(lam, [-1.0, 3.0])
    assert np.max(np.abs(s - np.array([[0.0, 1.0], [1.0, 0.0]]))) < 1e-15
    # [[2, 0], [0, 3]]: positive definite -> identity
    s, _ = O.sign_eig(np.diag([2.0, 3.0]))
    assert np.array_equal(s, np.eye(2))


def test_sign_diagonal_is_elementwise_with_zero():
    d = np.array([-3.0, -1e-9, 0.0, 2e-7, 5.0])
    s, _ = O.sign_eig(np.diag(d))
    assert np.allclose(s, np.diag(np.sign(d)), atol=1e-15)
    assert s[2, 2] == 0.0  # sign(0) = 0


@pytest.mark.parametrize("n", [3, 17, 64, 150])
def test_sign_invariants(n):
    rng = np.random.default_rng(n)
    eigs = np.concatenate([-rng.uniform(0.2, 2.0, n // 2), rng.uniform(0.2, 2.0, n - n // 2)])
    a = spectrum_matrix(n, eigs, seed=100 + n)
    s, lam = O.sign_eig(a)
    eye = np.eye(n)
    assert np.max(np.abs(s @ s - eye)) < 1e-13  # involution
    assert np.max(np.abs(s @ a - a @ s)) < 1e-13  # commutes with A
    sa = s @ a
    assert np.max(np.abs(sa - sa.T)) < 1e-13
    assert np.min(np.linalg.eigvalsh(0.5 * (sa + sa.T))) > 0.19  # S A = |A| is positive definite
    assert abs(np.trace(s) - (np.count_nonzero(eigs > 0) - np.count_nonzero(eigs < 0))) < 1e-12


@pytest.mark.parametrize("n", [2, 9, 40, 120])
def test_sign_matches_newton_iteration(n):
    rng = np.random.default_rng(1000 + n)
    g = rng.normal(size=(n, n))
    a = g + g.T + np.diag(rng.choice([-1.0, 1.0], n) * 3.0)
    s_eig, _ = O.sign_eig(a)
    s_newton = O.sign_newton(a)
    assert np.max(np.abs(s_eig - s_newton)) < 1e-11


def test_gershgorin_hand_values_and_enclosure():
    a = np.array([[4.0, -1.0, 0.5], [-1.0, -2.0, 0.25], [0.5, 0.25, 1.0]])
    # rows: 4 +- 1.5, -2 +- 1.25, 1 +- 0.75  ->  lo = -3.25, hi = 5.5
    lo, hi = O.gershgorin_bounds(a)
    assert lo == -3.25 and hi == 5.5
    rng = np.random.default_rng(5)
    for n in [5, 30, 100]:
        g = rng.normal(size=(n, n))
        b = g + g.T
        lo, hi = O.gershgorin_bounds(b)
        lam = np.linalg.eigvalsh(b)
        assert lo <= lam[0] and lam[-1] <= hi
    lo, hi = O.gershgorin_bounds(np.diag([-2.0, 7.0]))
    assert (lo, hi) == (-2.0, 7.0)


@pytest.mark.parametrize("n", [1, 4, 23])
def test_block_sign_identity_eq12(n):
    # Eq. 12: for a symmetric positive definite A, sign([[0, A], [I, 0]]) = [[0, A^1/2], [A^-1/2, 0]].
    # The left side goes through the oracle's sign of a (non-symmetric) 2n x 2n matrix by the
    # Newton iteration; the right side is built from A's eigendecomposition (a library routine).
    rng = np.random.default_rng(77 + n)
    g = rng.normal(size=(n, n))
    a = g @ g.T + n * np.eye(n)
    w, v = np.linalg.eigh(a)
    root = (v * np.sqrt(w)) @ v.T
    iroot = (v / np.sqrt(w)) @ v.T
    m = np.block([[np.zeros((n, n)), a], [np.eye(n), np.zeros((n, n))]])
    s = O.sign_newton(m)
    ref = np.block([[np.zeros((n, n)), root], [iroot, np.zeros((n, n))]])
    assert np.max(np.abs(s - ref)) <= 1e-10 * max(1.0, float(np.max(np.abs(ref))))
    assert np.max(np.abs(root @ iroot - np.eye(n))) < 1e-12
