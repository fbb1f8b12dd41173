"""Pins of the FP64 oracle of the learned proposal (oracle/learned.py): its gradient
against central finite differences, closed forms, and hand-built feature scenes."""
import numpy as np

from oracle import learned as L


def _rand_params(dims, rng, scale=0.5):
    return rng.normal(0.0, scale, size=L.n_params(dims))


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    dims = (6, 7, 5, 4)
    p = _rand_params(dims, rng)
    X = rng.normal(size=(9, 6))
    y = rng.integers(0, 4, size=9)
    loss, g = L.loss_and_grad(p, X, y, dims)
    eps = 1e-6
    fd = np.empty_like(p)
    for i in range(p.size):
        e = np.zeros_like(p)
        e[i] = eps
        fd[i] = (L.loss_and_grad(p + e, X, y, dims)[0] - L.loss_and_grad(p - e, X, y, dims)[0]) / (2 * eps)
    assert np.max(np.abs(fd - g)) < 1e-7 * max(1.0, np.max(np.abs(g))) + 1e-9
    assert loss > 0


def test_masked_outputs_get_no_probability_and_no_gradient():
    rng = np.random.default_rng(1)
    dims = (5, 6, 8)
    p = _rand_params(dims, rng)
    X = rng.normal(size=(4, 5))
    y = np.array([0, 2, 4, 1])
    _, g = L.loss_and_grad(p, X, y, dims, n_valid=5)
    W2g = g[5 * 6 + 6:5 * 6 + 6 + 6 * 8].reshape(6, 8)
    b2g = g[-8:]
    assert np.all(W2g[:, 5:] == 0.0) and np.all(b2g[5:] == 0.0)


def test_zero_network_closed_form():
    X = np.random.default_rng(2).normal(size=(7, 128))
    y = np.arange(7) % 25
    p = np.zeros(L.n_params())
    loss, g = L.loss_and_grad(p, X, y)
    assert abs(loss - np.log(25.0)) < 1e-12
    # only the last bias moves: its gradient is the mean of (uniform - one-hot)
    gb = g[-25:]
    want = np.full(25, 1.0 / 25.0)
    for t in y:
        want[t] -= 1.0 / 7.0
    np.testing.assert_allclose(gb, want, atol=1e-15)
    assert np.all(g[:-25] == 0.0)


def test_forward_hand_example():
    dims = (2, 2, 1)
    # W1 = [[1, -1], [2, 0]], b1 = [0, 1]; W2 = [[3], [-1]], b2 = [0.5]
    p = np.array([1.0, -1.0, 2.0, 0.0, 0.0, 1.0, 3.0, -1.0, 0.5])
    out, _ = L.mlp_forward(p, np.array([[1.0, 1.0], [-1.0, 0.5]]), dims)
    # row 1: z1 = (3, 0) -> relu (3, 0); out = 9 + 0.5. row 2: z1 = (0, 2) -> (0, 2); out = -2 + 0.5
    np.testing.assert_allclose(out[:, 0], [9.5, -1.5])


BOX = (0.0, 0.0, 0.0, 10000.0, 10000.0, 500.0)


def test_one_intruder_lands_in_its_sector():
    s = np.array([5000.0, 5000.0, 200.0])
    p1 = np.array([[5300.0, 5000.0, 210.0]])        # 300 m straight ahead, 10 m above
    p2 = np.array([[5300.0, 5030.0, 210.0]])        # moving left at 30 m/s
    f = L.features(s, 1.0, 0.0, 25.0, (9000.0, 5000.0, 200.0), BOX, p1, p2)
    d = np.sqrt(300.0 ** 2 + 10.0 ** 2)
    w = 1.0 - d / L.R_F
    o = L.N_OWN + 6 * (5 + 10)  # azimuth 0 is sector 5; above: +10
    np.testing.assert_allclose(f[o:o + 6], np.array([0.6, 0.0, 0.02, -25.0 / 50.0, 0.6, 0.0]) * w, rtol=1e-12)
    assert np.count_nonzero(f[L.N_OWN:]) == 4
    assert f[0] == 0.4 and f[6] == 1.0 and f[7] == 0.0 and abs(f[2] - 0.8) < 1e-15


def test_features_ignore_far_or_missing_plans_and_keep_the_nearest_per_sector():
    s = np.array([5000.0, 5000.0, 200.0])
    p1 = np.array([[5000.0, 6100.0, 200.0], [np.nan, np.nan, np.nan], [5100.0, 5010.0, 150.0],
                   [5200.0, 5020.0, 150.0]])
    p2 = p1.copy()
    f = L.features(s, 1.0, 0.0, 30.0, (9000.0, 5000.0, 200.0), BOX, p1, p2)
    o = L.N_OWN + 6 * 5  # ahead, below
    rel = p1[2] - s
    d = np.sqrt(rel @ rel)
    np.testing.assert_allclose(f[o:o + 3], rel / 500.0 * (1 - d / L.R_F), rtol=1e-12)
    assert np.count_nonzero(f[L.N_OWN:]) == 4  # one sector: 3 position terms + the closing speed


def test_features_are_invariant_to_rotating_the_scene():
    rng = np.random.default_rng(3)
    s = np.array([5000.0, 5000.0, 200.0])
    p1 = s + rng.uniform(-900, 900, size=(30, 3)) * np.array([1, 1, 0.1])
    p2 = p1 + rng.uniform(-40, 40, size=(30, 3)) * np.array([1, 1, 0.05])
    goal = np.array([8000.0, 6500.0, 300.0])
    a = 0.7
    R = np.array([[np.cos(a), -np.sin(a), 0.0], [np.sin(a), np.cos(a), 0.0], [0.0, 0.0, 1.0]])
    c = np.array([5000.0, 5000.0, 0.0])
    rot = lambda v: (np.asarray(v) - c) @ R.T + c
    h = 0.3
    f1 = L.features(s, np.cos(h), np.sin(h), 30.0, goal, BOX, p1, p2)
    f2 = L.features(rot(s), np.cos(h + a), np.sin(h + a), 30.0, rot(goal), BOX, rot(p1), rot(p2))
    np.testing.assert_allclose(f1, f2, atol=1e-9)


def test_rounding_mode_reduces_to_the_exact_gradient_and_stays_close():
    rng = np.random.default_rng(6)
    dims = (16, 32, 32, 10)
    p = _rand_params(dims, rng, scale=0.3)
    X = rng.normal(size=(40, 16))
    # labels from a teacher network: a gradient with signal, not just cancelling noise
    teacher = _rand_params(dims, rng, scale=0.3)
    y = np.argmax(L.mlp_forward(teacher, X, dims)[0], axis=1)
    l0, g0 = L.loss_and_grad(p, X, y, dims)
    l1, g1 = L.loss_and_grad(p, X, y, dims, round_fn=lambda v: v)
    assert l0 == l1 and np.array_equal(g0, g1)
    l2, g2 = L.loss_and_grad(p, X, y, dims, round_fn=L.bf16)
    assert abs(l2 - l0) < 1e-2 * l0
    assert np.linalg.norm(g2 - g0) < 2e-2 * np.linalg.norm(g0)
    # bf16: 8 significant bits, ties to even
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -7, -3.14159])
    np.testing.assert_array_equal(L.bf16(v)[:4], [1.0, 1.0, 1.0 + 2 ** -6, 1.0 + 2 ** -7])
    assert abs(L.bf16(v)[4] + 3.140625) < 1e-12
