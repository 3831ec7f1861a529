"""The FP64 MLP reference: its analytic gradients equal central finite
differences of its loss; GELU and its derivative match their definitions."""
import math

import numpy as np

from oracle import mlp


def test_gelu_definition_points():
    x = np.array([-3.0, -1.0, 0.0, 0.5, 2.0])
    ref = np.array([v * 0.5 * (1 + math.erf(v / math.sqrt(2))) for v in x])
    assert np.allclose(mlp.gelu(x), ref, rtol=0, atol=1e-15)
    h = 1e-6
    fd = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    assert np.allclose(mlp.gelu_grad(x), fd, rtol=1e-8, atol=1e-9)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = mlp.init_params(1)
    for k in p:
        if k.startswith("b"):
            p[k] = rng.standard_normal(p[k].shape) * 0.1
    x = rng.standard_normal((7, 24))
    y = rng.standard_normal(7) * 2
    L, g = mlp.loss_and_grads(p, x, y)
    h = 1e-6
    for name in p:
        flat = p[name].reshape(-1)
        idx = rng.choice(flat.size, size=min(6, flat.size), replace=False)
        for i in idx:
            old = flat[i]
            flat[i] = old + h
            Lp, _ = mlp.loss_and_grads(p, x, y)
            flat[i] = old - h
            Lm, _ = mlp.loss_and_grads(p, x, y)
            flat[i] = old
            fd = (Lp - Lm) / (2 * h)
            an = g[name].reshape(-1)[i]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (name, i, fd, an)


def test_loss_minimum_is_the_gaussian_fit():
    # for a constant prediction the loss is minimised at mu = mean, s = log var
    rng = np.random.default_rng(2)
    y = rng.normal(1.5, 0.7, 20000)
    out = np.tile([y.mean(), math.log(y.var())], (len(y), 1))
    g = mlp.loss_grad(out, y)
    assert abs(g[:, 0].sum()) < 1e-9 and abs(g[:, 1].sum()) < 1e-9


def test_mean_objective_gradient_and_minimiser():
    rng = np.random.default_rng(4)
    n = 9
    out = rng.standard_normal((n, 2))
    Y = rng.gamma(2.0, 3.0, n)
    B = rng.gamma(2.0, 2.0, n)
    g = mlp.loss_mean_grad(out, Y, B)
    lam0 = mlp.mean_outputs(out, B)
    h = 1e-6
    for i in range(n):
        for j in range(2):
            o = out.copy()
            o[i, j] += h
            Lp = mlp.loss_mean(o, Y, B, lam_fixed=lam0)
            o[i, j] -= 2 * h
            Lm = mlp.loss_mean(o, Y, B, lam_fixed=lam0)
            assert abs((Lp - Lm) / (2 * h) - g[i, j]) < 1e-7
    # the Poisson part is minimised by the mean label: for one feature vector
    # seen with labels Y_k, d/dmu sum_k P_k = 0 at lam = mean(Y)
    Ys = rng.gamma(2.0, 3.0, 1000)
    Bc = 1.7
    mu = np.log(Ys.mean() / (Bc + 1.0))
    o = np.tile([mu, 0.0], (len(Ys), 1))
    assert abs(mlp.loss_mean_grad(o, Ys, np.full(len(Ys), Bc))[:, 0].sum()) < 1e-12
