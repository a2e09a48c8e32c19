"""Pins for the oracle's bound model (features, labels, MLP, Adam)."""

import numpy as np
import pytest

import oracle.mlp as M
from synth import spectrum_matrix


def _rand_theta(seed, f=M.F, scale=0.5):
    return np.random.default_rng(seed).normal(0, scale, M.param_count(f))


def test_param_layout_and_forward_closed_form():
    assert M.param_count(9) == 64 * 9 + 64 + 64 * 64 + 64 + 2 * 64 + 2
    theta = np.zeros(M.param_count())
    w1, b1, w2, b2, w3, b3 = M.unpack(theta)
    b1[:] = 0.3          # views into theta
    b2[:] = -0.2
    w3[:] = 0.5
    b3[:] = [0.1, -0.4]
    x = np.random.default_rng(0).normal(size=(5, M.F))
    y, _ = M.forward(theta, x)
    # W1 = W2 = 0: h1 = tanh(0.3), h2 = tanh(-0.2) for every sample
    expect = 64 * 0.5 * np.tanh(-0.2) + np.array([0.1, -0.4])
    assert np.allclose(y, expect[None, :], atol=1e-15)


def test_loss_closed_form_and_bias_gradient():
    theta = np.zeros(M.param_count())
    theta[-2:] = [1.0, 2.0]     # y = b3 for every sample
    x = np.ones((4, M.F))
    t = np.array([[0.0, 0.0], [1.0, 1.0], [2.0, 2.0], [3.0, 3.0]])
    loss, g = M.loss_and_grad(theta, x, t)
    r = np.array([1.0, 2.0])[None, :] - t
    assert abs(loss - 0.5 * np.sum(r * r) / 4) < 1e-15
    assert np.allclose(g[-2:], r.mean(axis=0))
    # W3 gradient is zero because h2 = tanh(0) = 0
    assert np.all(g[-2 - 128:-2] == 0.0)


@pytest.mark.parametrize("seed", [1, 2])
def test_gradient_matches_central_differences(seed):
    rng = np.random.default_rng(seed)
    theta = _rand_theta(seed)
    x = rng.normal(size=(7, M.F))
    t = rng.normal(size=(7, 2))
    _, g = M.loss_and_grad(theta, x, t)
    idx = rng.choice(theta.shape[0], size=60, replace=False)
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        num = (M.loss_and_grad(tp, x, t)[0] - M.loss_and_grad(tm, x, t)[0]) / (2 * h)
        assert abs(num - g[i]) <= 1e-7 * max(1.0, abs(g[i])), (i, num, g[i])


def test_first_adam_step_closed_form():
    theta = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -1e-3, 0.0])
    th1, m, v = M.adam_step(theta, g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    # after one step m_hat = g and v_hat = g^2: the update is lr * g / (|g| + eps)
    assert np.allclose(th1, theta - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_features_and_labels_of_a_diagonal_matrix():
    d = np.array([-0.6, -0.4, 0.3, 0.9])
    a = np.diag(d)
    f = M.features(a, prev_ratio=0.7)
    g = 0.9
    assert np.allclose(f, [np.sqrt(np.sum(d * d) / 4) / g, 0.9 / g, np.mean(np.abs(d)) / g, np.std(d) / g,
                           0.0, 0.0, 4 / 256, np.mean(d) / g, 0.7])
    assert np.allclose(M.labels(a), [1.0, 0.3 / 0.9])
    assert abs(M.square_bound_ratio(a) - 1.0) < 1e-15  # diagonal: the bound from A^2 is exact
    assert abs(M.power_bound_ratio(a) - 1.0) < 1e-15


def test_labels_and_bound_ratios_are_ordered():
    rng = np.random.default_rng(3)
    for n in [10, 60]:
        eigs = np.concatenate([-rng.uniform(0.2, 1.0, n // 2), rng.uniform(0.2, 1.0, n - n // 2)])
        a = spectrum_matrix(n, eigs, seed=n)
        rho, delta = M.labels(a)
        assert abs(rho * M.gershgorin_radius(a) - np.max(np.abs(eigs))) < 1e-12
        assert abs(delta * M.gershgorin_radius(a) - np.min(np.abs(eigs))) < 1e-12
        # rho <= sqrt(||A^2||_inf) <= ||A||_inf
        assert rho <= M.square_bound_ratio(a) + 1e-12 <= 1.0 + 2e-12


def test_init_is_seeded_and_scaled():
    a = M.init_params(5)
    b = M.init_params(5)
    assert np.array_equal(a, b)
    w1, b1, w2, b2, w3, b3 = M.unpack(a)
    assert np.all(np.abs(w1) <= 1 / 3) and np.all(b1 == 0) and np.all(np.abs(w2) <= 1 / 8)


def test_power_bound_is_between_rho_and_the_square_bound():
    rng = np.random.default_rng(8)
    for n in [5, 40, 120]:
        eigs = np.concatenate([-rng.uniform(0.1, 1.0, n // 2), rng.uniform(0.1, 1.0, n - n // 2)])
        a = spectrum_matrix(n, eigs, seed=3 * n)
        g = M.gershgorin_radius(a)
        rho = np.max(np.abs(eigs)) / g
        p0, p2 = M.power_bound_ratio(a, steps=0), M.power_bound_ratio(a)
        assert abs(p0 - M.square_bound_ratio(a)) < 1e-14   # w = 1 alone is the Gershgorin bound of A^2
        assert rho <= p2 * (1 + 1e-12) and p2 <= p0 * (1 + 1e-12)
        # many power steps converge to the Perron root of |A^2| (brute force by eigvalsh)
        perron = np.sqrt(np.max(np.linalg.eigvalsh(np.abs(a @ a)))) / g
        assert abs(M.power_bound_ratio(a, steps=400) - perron) <= 1e-6 * perron
        assert perron <= p2 * (1 + 1e-12)


def test_power_bound_with_a_zero_row():
    a = np.zeros((3, 3))
    a[0, 1] = a[1, 0] = 0.5
    # A^2 = diag(0.25, 0.25, 0): rho(A) = 0.5 = G, the bound is exact
    assert abs(M.power_bound_ratio(a) - 1.0) < 1e-15
