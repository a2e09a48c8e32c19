"""The scaled Newton-Schulz schedule the kernels follow with a predicted gap (host-side check of
the mathematics the kernels rely on; no GPU).

With every |eigenvalue| of X in [l, 1], the step p(a X), p(x) = x (3 - x^2) / 2, with
a = sqrt(3 / (1 + l + l^2)) maps the interval into [p(a l), 1] (p(a l) = p(a) and p peaks at 1
inside); capped factors (a <= 1.72) and underestimated l keep every eigenvalue in (0, 1]; the
sign is reached from any l in (0, 1]; a step with a factor a moves an eigenvalue at 1 to
p(a) = 1 - 1.5 (a - 1)^2 + O((a - 1)^3), which bounds the factor the last step may use.
"""

import numpy as np
import pytest

CAP = 1.72


def scale(l):
    return 1.0 if l >= 1.0 else min(np.sqrt(3.0 / (1.0 + l + l * l)), CAP)


def p(x):
    return 0.5 * x * (3.0 - x * x)


@pytest.mark.parametrize("l", [1e-6, 1e-3, 0.02, 0.1, 0.37, 0.8, 0.999])
def test_step_maps_the_interval_into_its_image(l):
    a = scale(l)
    x = np.concatenate([np.linspace(l, 1.0, 20001), np.geomspace(l, 1.0, 20001)])
    y = p(a * x)
    assert np.all(y > 0.0) and np.max(y) <= 1.0 + 1e-15
    assert np.min(y) >= p(a * l) * (1 - 1e-12)
    if a < CAP:  # uncapped: equioscillation at the two ends
        assert abs(p(a * l) - p(a)) <= 1e-12


@pytest.mark.parametrize("true_low", [1e-3, 0.05, 0.4])
@pytest.mark.parametrize("guess", [1e-6, 1e-2, 0.3, 1.0])
def test_any_guess_converges_to_the_sign(true_low, guess):
    rng = np.random.default_rng(0)
    lam = np.concatenate([np.geomspace(true_low, 1.0, 50), -np.geomspace(true_low, 0.9, 50), rng.uniform(-1, 1, 50)])
    lam = lam[np.abs(lam) >= true_low]
    x, l = lam.copy(), guess
    for _ in range(60):
        a = scale(l)
        x = p(a * x)
        l = min(p(a * l), 1.0)
        assert np.all(np.abs(x) <= 1.0 + 1e-12) and np.all(np.sign(x) == np.sign(lam))
    assert np.max(np.abs(x - np.sign(lam))) < 1e-12


def test_good_guess_saves_steps():
    lam = np.geomspace(0.01, 1.0, 200)

    def steps(guess):
        x, l = lam.copy(), guess
        for k in range(100):
            if np.max(np.abs(x - 1.0)) < 1e-7:
                return k
            a = scale(l)
            x, l = p(a * x), min(p(a * l), 1.0)
        return 100

    plain = steps(1.0)
    assert steps(0.01) <= plain - 5 and steps(0.005) <= plain - 4


def test_last_step_shift_bound():
    for eps in [1e-2, 3e-4, 1e-5]:
        shift = 1.0 - p(1.0 + eps)
        assert abs(shift - 1.5 * eps**2) <= 0.6 * eps**3
    assert 1.0 - p(1.0 + 3e-4) < 1.4e-7
