"""Pin the oracle's MLP gradient (used to check the device's training kernels) by central finite
differences of its own loss, parameter by parameter on a random subset."""
import numpy as np

from oracle import mlp as M


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = rng.normal(0, 0.3, M.COUNT)
    X = rng.normal(0, 1, (40, M.IN))
    t = rng.normal(0, 1, 40)
    norm = np.concatenate([rng.normal(0, 0.2, M.IN), np.exp(rng.normal(0, 0.2, M.IN))])
    _, g = M.loss_and_gradient(p, X, t, norm)
    h = 1e-6
    for e in rng.choice(M.COUNT, 60, replace=False).tolist() + [M.COUNT - 1, 0, 1030]:
        d = np.zeros(M.COUNT)
        d[e] = h
        fd = (M.loss_and_gradient(p + d, X, t, norm)[0] - M.loss_and_gradient(p - d, X, t, norm)[0]) / (2 * h)
        assert abs(fd - g[e]) <= 1e-6 * max(1.0, abs(g[e])), (e, fd, g[e])


def test_parameter_count_matches_layout():
    assert M.COUNT == 128 * 8 + 128 + 128 * 128 + 128 + 128 + 1
