"""GPU parity of the learned spectral bound: features, labels, inference,
gradients and Adam against the FP64 oracle of the model, file round trip, and
the gain of the trained network over the method without it.
"""

import numpy as np
import pytest

import oracle as O
import oracle.mlp as M
from synth import make_workload, md_trajectory
from tests.helpers import max_abs_on_columns, oracle_in_input_layout

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _ctx(sysm, prec="fp16x3", eps=0.0):
    from paper_2205_14741_gb300 import SubmatrixDensity

    c = SubmatrixDensity.from_system(sysm)
    c.set_precision(prec)
    c.set_filter_threshold(eps)
    return c


def _oracle_blocks(sysm, mu):
    """A_j = T_j - mu I of every block column (unfiltered pattern)."""
    return [O.gather_submatrix(sysm.block_size, sysm.col_ptr, sysm.row_idx, sysm.values, j, mu=mu)[0]
            for j in range(sysm.block_size.shape[0])]


def _theta(seed):
    """Oracle initialisation plus noise on every parameter (non-zero biases), as FP32."""
    rng = np.random.default_rng(seed)
    return (M.init_params(seed) + rng.normal(0.0, 0.05, M.param_count())).astype(np.float32)


@pytest.mark.parametrize("prec", ["fp64", "fp16x3"])
def test_features_and_labels_match_oracle(prec):
    s = make_workload("water32")
    blocks = _oracle_blocks(s, 0.1)
    with _ctx(s, prec) as c:
        c.set_mu(0.1)
        f, _, lab = c.bound_model_predict(predict=False, labels=True, lanczos_steps=64)
    f_or = np.array([M.features(a, prev_ratio=0.0) for a in blocks])
    lab_or = np.array([M.labels(a) for a in blocks])
    # features: FP32 sums of FP32 (or FP64) entries
    assert np.max(np.abs(f - f_or) / np.maximum(np.abs(f_or), 1e-3)) <= 2e-5
    # labels: Ritz values lie inside the spectrum, so the Lanczos rho never exceeds the
    # true one and the Lanczos delta (from A^2) never falls below it, up to FP32 rounding
    # of the products (relative 1e-5 on rho^2, at most 1e-3 relative on delta); 64 steps
    # give rho to 1e-3 on these sizes
    rho, delta = lab[:, 0], lab[:, 1]
    assert np.all(rho <= lab_or[:, 0] * (1 + 1e-5))
    assert np.all(rho >= lab_or[:, 0] * (1 - 1e-3))
    assert np.all(delta >= lab_or[:, 1] * (1 - 1e-3))
    assert np.all(delta <= rho)


@pytest.mark.parametrize("prec", ["fp64", "fp16x3"])
def test_previous_step_ratio_matches_oracle(prec):
    # f8 after a build and new values: the first-product bound of the build, over G
    s = make_workload("water32")
    blocks = _oracle_blocks(s, -0.05)
    with _ctx(s, prec) as c:
        c.set_mu(-0.05)
        f0, _, _ = c.bound_model_predict(predict=False)
        c.build_density()
        c.set_values(s.values)
        f1, _, _ = c.bound_model_predict(predict=False)
    assert np.all(f0[:, 8] == 0.0)
    ref = np.array([M.square_bound_ratio(a) for a in blocks])
    rel = f1[:, 8] / ref - 1.0
    # FP64 kernel: float rounding of the ratio; tensor-core kernel: the product from
    # split-FP16 operands, FP32 sums and a 1e-5 margin on the bound of A^2
    lo, hi = (-1e-6, 1e-6) if prec == "fp64" else (-2e-5, 3e-5)
    assert lo <= rel.min() and rel.max() <= hi, (rel.min(), rel.max())


def test_inference_matches_oracle_with_fp16_weights():
    s = make_workload("water32")
    theta = _theta(3)
    with _ctx(s) as c:
        c.set_mu(0.0)
        c.bound_model_init(1)
        c.bound_model_set_params(theta)
        assert np.array_equal(c.bound_model_get_params(), theta)
        f, p, _ = c.bound_model_predict()
    theta16 = theta.astype(np.float16).astype(np.float64)  # inference weights are FP16-rounded
    y, _ = M.forward(theta16, f.astype(np.float64))
    assert np.max(np.abs(p - y)) <= 2e-5 * max(1.0, float(np.max(np.abs(y))))


@pytest.mark.parametrize("m", [1, 64, 200])
def test_gradient_matches_oracle(m):
    rng = np.random.default_rng(m)
    x = rng.normal(0.0, 0.5, (m, M.F)).astype(np.float32)
    t = rng.uniform(0.0, 1.0, (m, 2)).astype(np.float32)
    theta = _theta(7)
    with _ctx(make_workload("water32")) as c:
        c.bound_model_init(0)
        c.bound_model_set_params(theta)
        loss, g = c.bound_model_fit(x, t, steps=0)
    loss_or, g_or = M.loss_and_grad(theta.astype(np.float64), x.astype(np.float64), t.astype(np.float64))
    assert abs(loss - loss_or) <= 1e-5 * loss_or
    # FP32 forward/backward and sums over m samples against FP64
    assert np.max(np.abs(g - g_or)) <= 1e-4 * float(np.max(np.abs(g_or)))
    assert np.linalg.norm(g - g_or) <= 2e-5 * np.linalg.norm(g_or)


def test_adam_steps_match_oracle():
    rng = np.random.default_rng(11)
    m = 150
    x = rng.normal(0.0, 0.5, (m, M.F)).astype(np.float32)
    t = rng.uniform(0.0, 1.0, (m, 2)).astype(np.float32)
    theta = _theta(5)
    lr = 1e-3
    with _ctx(make_workload("water32")) as c:
        c.bound_model_init(0)
        c.bound_model_set_params(theta)
        _, g = c.bound_model_fit(x, t, steps=1, lr=lr)
        th1 = c.bound_model_get_params()
        c.bound_model_set_params(theta)  # clears the Adam state
        c.bound_model_fit(x, t, steps=4, lr=lr)
        th4 = c.bound_model_get_params()
    # first step from zero moments: m_hat = g, v_hat = g^2, so the update is lr g / (|g| + eps)
    step1 = -lr * g.astype(np.float64) / (np.abs(g.astype(np.float64)) + 1e-8)
    assert np.max(np.abs((th1.astype(np.float64) - theta) - step1)) <= 1e-6
    # four steps against the FP64 oracle; parameters whose gradient is near zero can take
    # either direction in FP32, so they are held to the size of the step instead
    th = theta.astype(np.float64)
    mo, vo = np.zeros_like(th), np.zeros_like(th)
    gmin = np.full_like(th, np.inf)
    for k in range(1, 5):
        _, go = M.loss_and_grad(th, x.astype(np.float64), t.astype(np.float64))
        gmin = np.minimum(gmin, np.abs(go))
        th, mo, vo = M.adam_step(th, go, mo, vo, k, lr)
    firm = gmin > 1e-4 * np.max(np.abs(g))
    assert firm.mean() > 0.85
    diff = np.abs(th4.astype(np.float64) - th)
    assert np.max(diff[firm]) <= 2e-5
    assert np.max(diff) <= 16 * lr


def test_save_load_round_trip(tmp_path):
    from paper_2205_14741_gb300 import SmxError

    s = make_workload("water32")
    theta = _theta(9)
    path = str(tmp_path / "bound.bin")
    with _ctx(s) as c:
        with pytest.raises(SmxError):
            c.set_bound_model(True)  # never initialised
        c.bound_model_init(2)
        c.bound_model_set_params(theta)
        c.bound_model_save(path)
    raw = open(path, "rb").read()
    assert raw[:8] == b"SMXBNDM1" and len(raw) == 8 + 4 + 4 * M.param_count() + 8
    with _ctx(s) as c:
        c.set_bound_model(True, path)
        assert np.array_equal(c.bound_model_get_params(), theta)
        bad = tmp_path / "bad.bin"
        bad.write_bytes(raw[:100] + bytes([raw[100] ^ 1]) + raw[101:])
        with pytest.raises(SmxError):
            c.set_bound_model(True, str(bad))  # checksum mismatch
        assert np.array_equal(c.bound_model_get_params(), theta)


def test_trained_model_saves_iterations():
    """Train on the first snapshots of a trajectory, compare iterations on later ones."""
    snaps = list(md_trajectory(128, 6, 6.0, 1.5, seed=77, n_snap=14, fixed_pattern=True))
    eps, mu = 1e-5, 0.0
    train, held = snaps[:10], snaps[10:]
    with _ctx(snaps[0], eps=eps) as c:
        c.set_mu(mu)
        c.bound_model_init(4)
        for sysm in train:
            c.set_values(sysm.values)
            c.build_density()          # leaves the bound ratio used as the next snapshot's feature
            c.bound_model_collect(48)
        loss = c.bound_model_train(epochs=300, batch=128, lr=2e-3)
        assert loss < 5e-3

        def run(model_on):
            c.set_bound_model(model_on)
            c.set_values(train[-1].values)
            c.build_density()
            its, fb, ds = [], 0, []
            for sysm in held:
                c.set_values(sysm.values)
                c.build_density()
                its.append(c.get_submatrix_info()[1].copy())
                fb += c.get_stats()["n_bound_fallback"]
                ds.append(c.get_density())
            return np.concatenate(its), fb, ds

        it0, fb0, d0 = run(False)
        it1, fb1, d1 = run(True)
    assert fb0 == 0
    assert fb1 <= 0.1 * it1.shape[0], f"fallback rate {fb1 / it1.shape[0]:.3f}"
    assert it1.mean() <= it0.mean() - 0.3, f"iterations {it0.mean():.3f} -> {it1.mean():.3f}"
    # the density matrix stays within the mixed-precision tolerance of the oracle
    cols = list(range(0, 128, 9))
    d_or, _, _ = oracle_in_input_layout(held[-1], eps, mu, columns=cols)
    assert max_abs_on_columns(d1[-1], d_or, held[-1], cols) <= 1e-5
    assert max_abs_on_columns(d1[-1], d0[-1], held[-1], cols) <= 2e-5
