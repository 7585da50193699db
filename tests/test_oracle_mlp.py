"""Pins of the CPU reference of the learned preconditioner network."""
import numpy as np

from oracle import mlp


def random_net(seed):
    rng = np.random.default_rng(seed)
    return mlp.MLP(rng.normal(0, 0.3, (mlp.H, mlp.F)), rng.normal(0, 0.1, mlp.H), rng.normal(0, 0.1, mlp.H),
                   rng.normal(0, 0.1))


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    r = rng.normal(size=300)
    d = rng.normal(size=300) * 3
    f = mlp.features(r, d, -0.4, 5)
    y = rng.normal(size=300) * 0.3
    w = rng.uniform(0.1, 1.0, 300)
    net = random_net(2)
    lam = 0.3
    L0, g = net.loss_and_grad(f, y, w, lam)
    p = net.params()
    h = 1e-5
    idx = np.concatenate([rng.choice(mlp.H * mlp.F, 40, replace=False), mlp.H * mlp.F + np.arange(0, 2 * mlp.H, 7),
                          [p.size - 1]])
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        Lp, _ = mlp.MLP.from_params(pp).loss_and_grad(f, y, w, lam)
        Lm, _ = mlp.MLP.from_params(pm).loss_and_grad(f, y, w, lam)
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (i, fd, g[i])


def test_zero_network_is_the_jacobi_step():
    rng = np.random.default_rng(3)
    r = rng.normal(size=50)
    d = rng.normal(size=50)
    net = mlp.MLP(np.zeros((mlp.H, mlp.F)), np.zeros(mlp.H), np.zeros(mlp.H), 0.0)
    t = mlp.precondition(r, d, 0.2, 1, net)
    assert np.allclose(t, -r / (d - 0.2))


def test_targets_reproduce_an_exact_direction():
    # if e is a multiple of the Jacobi step, every target is 0 with the same weight as tj^2
    rng = np.random.default_rng(4)
    tj = rng.normal(size=20)
    y, w = mlp.targets(tj, 2.5 * tj)
    assert np.allclose(y, 0.0)
    assert np.allclose(w, tj * tj)


def test_prior_term_is_the_mean_square_output():
    rng = np.random.default_rng(6)
    f = mlp.features(rng.normal(size=40), rng.normal(size=40), 0.1, 2)
    net = random_net(7)
    g, _, _ = net.forward(f)
    y = g.copy()                      # data term zero
    L, _ = net.loss_and_grad(f, y, np.ones(40), lam=2.0)
    assert abs(L - 2.0 * np.mean(g * g)) < 1e-12


def test_output_clip_bounds_the_correction():
    rng = np.random.default_rng(8)
    r, d = rng.normal(size=30), rng.normal(size=30) + 3
    big = mlp.MLP(np.zeros((mlp.H, mlp.F)), np.ones(mlp.H), np.full(mlp.H, 10.0), 0.0)   # g = 1280
    t = mlp.precondition(r, d, 0.0, 1, big)
    assert np.allclose(t, mlp.jacobi_step(r, d, 0.0) * 5.0)
