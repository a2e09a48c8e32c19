"""Learned spectral-bound model: features, labels and the MLP, FP64 numpy.

TEST INFRASTRUCTURE ONLY: the reference the GPU model kernels are checked
against (the paper's Section 4 names learning on the fly as a direction; here
a small network predicts each submatrix's spectral bounds from cheap
features, to scale the Newton-Schulz start tighter than the Gershgorin
bound).

Definitions shared with the GPU path (both sides implement them separately):

* A = T_j - mu I (dense, symmetric, n x n), G = max_r sum_c |A_rc| (the
  Gershgorin bound), R_r = sum_{c != r} |A_rc|.
* Features (F = 9), all divided by G except f6, f8:
    f0 = ||A||_F / sqrt(n)        f1 = max_r |A_rr|       f2 = mean_r |A_rr|
    f3 = std_r(A_rr)              f4 = max_r R_r          f5 = mean_r R_r
    f6 = n / 256                  f7 = mean_r A_rr        f8 = previous-step ratio
  where f8 is square_bound_ratio(A) of the same block column at the previous
  snapshot (0 when there is none).  power_bound_ratio is the tighter bound the
  Newton-Schulz start is checked against when the model is on.
* Labels: rho / G and delta / G with rho = max |lambda(A)|, delta = min |lambda(A)|.
* Network: h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2), y = W3 h2 + b3,
  widths F -> 64 -> 64 -> 2; loss L = 1/(2m) sum_i sum_k (y_ik - t_ik)^2.
* Flat parameter layout: W1 (64 x F, row-major), b1 (64), W2 (64 x 64), b2 (64),
  W3 (2 x 64), b3 (2).
* Adam: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
  theta -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).

Parity: pinned by tests/test_oracle_mlp.py (central finite differences of
the gradient, closed-form cases of forward, loss and the first Adam step,
features and labels of diagonal and block-diagonal matrices).
"""

from __future__ import annotations

import numpy as np

F = 9
H = 64
O = 2


def param_count(f: int = F) -> int:
    return H * f + H + H * H + H + O * H + O


def unpack(theta: np.ndarray, f: int = F):
    theta = np.asarray(theta, dtype=np.float64)
    i = 0
    w1 = theta[i:i + H * f].reshape(H, f); i += H * f
    b1 = theta[i:i + H]; i += H
    w2 = theta[i:i + H * H].reshape(H, H); i += H * H
    b2 = theta[i:i + H]; i += H
    w3 = theta[i:i + O * H].reshape(O, H); i += O * H
    b3 = theta[i:i + O]; i += O
    assert i == theta.shape[0]
    return w1, b1, w2, b2, w3, b3


def forward(theta: np.ndarray, x: np.ndarray):
    """x: [m, F] -> (y [m, 2], cache)."""
    w1, b1, w2, b2, w3, b3 = unpack(theta, x.shape[1])
    h1 = np.tanh(x @ w1.T + b1)
    h2 = np.tanh(h1 @ w2.T + b2)
    y = h2 @ w3.T + b3
    return y, (x, h1, h2)


def loss_and_grad(theta: np.ndarray, x: np.ndarray, t: np.ndarray):
    """Mean squared error / 2 and its gradient with respect to the flat parameters."""
    m = x.shape[0]
    w1, b1, w2, b2, w3, b3 = unpack(theta, x.shape[1])
    y, (_, h1, h2) = forward(theta, x)
    r = y - t
    loss = 0.5 * np.sum(r * r) / m
    dy = r / m                                   # dL/dy
    g_w3 = dy.T @ h2
    g_b3 = dy.sum(axis=0)
    dh2 = dy @ w3
    da2 = dh2 * (1.0 - h2 * h2)                  # tanh' = 1 - tanh^2
    g_w2 = da2.T @ h1
    g_b2 = da2.sum(axis=0)
    dh1 = da2 @ w2
    da1 = dh1 * (1.0 - h1 * h1)
    g_w1 = da1.T @ x
    g_b1 = da1.sum(axis=0)
    g = np.concatenate([g_w1.ravel(), g_b1, g_w2.ravel(), g_b2, g_w3.ravel(), g_b3])
    return loss, g


def adam_step(theta, g, m, v, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (t counts from 1); returns (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def gershgorin_radius(a: np.ndarray) -> float:
    return float(np.max(np.sum(np.abs(a), axis=1)))


def features(a: np.ndarray, prev_ratio: float = 0.0) -> np.ndarray:
    """The F = 9 features of the shifted submatrix A (see the module docstring)."""
    n = a.shape[0]
    g = gershgorin_radius(a)
    d = np.diag(a)
    r = np.sum(np.abs(a), axis=1) - np.abs(d)
    return np.array([
        np.sqrt(np.sum(a * a)) / np.sqrt(n) / g,
        np.max(np.abs(d)) / g,
        np.mean(np.abs(d)) / g,
        np.std(d) / g,
        np.max(r) / g,
        np.mean(r) / g,
        n / 256.0,
        np.mean(d) / g,
        prev_ratio,
    ])


def square_bound_ratio(a: np.ndarray) -> float:
    """sqrt(max_r sum_c |(A^2)_rc|) / G: a guaranteed bound on rho / G from A^2."""
    return float(np.sqrt(gershgorin_radius(a @ a)) / gershgorin_radius(a))


def power_bound_ratio(a: np.ndarray, steps: int = 2) -> float:
    """Guaranteed bound on rho(A) / G from Z = A^2 (Collatz-Wielandt).

    For every positive vector w, rho(Z) <= rho(|Z|) <= max_r (|Z| w)_r / w_r.
    The bound is the smallest of these over w = 1 (the row sums: the
    Gershgorin bound of Z) and ``steps`` power steps of |Z| from it; its
    square root over G bounds rho(A) / G.
    """
    z = np.abs(a @ a)
    w = np.ones(a.shape[0])
    best = np.inf
    for _ in range(steps + 1):
        zw = z @ w
        best = min(best, float(np.max(zw / w)))
        w = np.maximum(zw / np.max(zw), 1e-300)  # stays positive where a row of Z is zero
    return float(np.sqrt(best) / gershgorin_radius(a))


def labels(a: np.ndarray) -> np.ndarray:
    """(rho / G, delta / G) from the exact eigenvalues."""
    lam = np.linalg.eigvalsh(a)
    g = gershgorin_radius(a)
    return np.array([np.max(np.abs(lam)) / g, np.min(np.abs(lam)) / g])


def init_params(seed: int, f: int = F) -> np.ndarray:
    """Reference initialisation: U(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_out, fan_in in [(H, f), (H, H), (O, H)]:
        lim = 1.0 / np.sqrt(fan_in)
        parts.append(rng.uniform(-lim, lim, fan_out * fan_in))
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts)
