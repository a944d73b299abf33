"""Pins for the FP64 reference MLP: its analytic gradient against central
finite differences of its own loss (a check independent of the chain-rule
code), its forward pass against an explicit per-sample loop, and the
parameter layout against the count formula.  Copies of the MLP with one
planted slip each must fail these pins."""
import types

import numpy as np
import pytest

from oracle import mlp


def _setup(seed, n_in=5, h=7, B=9):
    rng = np.random.default_rng(seed)
    p = rng.standard_normal(mlp.n_params(n_in, h)) * 0.5
    x = rng.standard_normal((B, n_in)) * 3 + 1
    t = rng.standard_normal(B)
    mean = x.mean(axis=0)
    std = x.std(axis=0) + 0.1
    return p, x, t, mean, std, n_in, h


def _check_gradient(mlp):
    for seed in range(4):
        p, x, t, mean, std, n_in, h = _setup(seed)
        _, g = mlp.loss_and_grad(p, x, t, mean, std, n_in, h)
        eps = 1e-6
        num = np.zeros_like(p)
        for i in range(len(p)):
            q = p.copy()
            q[i] += eps
            lp, _ = mlp.loss_and_grad(q, x, t, mean, std, n_in, h)
            q[i] -= 2 * eps
            lm, _ = mlp.loss_and_grad(q, x, t, mean, std, n_in, h)
            num[i] = (lp - lm) / (2 * eps)
        np.testing.assert_allclose(g, num, rtol=1e-5, atol=1e-7)


def _check_forward(mlp):
    p, x, t, mean, std, n_in, h = _setup(11)
    W1, b1, W2, b2, w3, b3 = mlp.unpack(p, n_in, h)
    y, _ = mlp.forward(p, x, mean, std, n_in, h)
    for b in range(len(x)):
        xn = [(x[b][k] - mean[k]) / std[k] for k in range(n_in)]
        h1 = [max(0.0, sum(xn[k] * W1[k][j] for k in range(n_in)) + b1[j]) for j in range(h)]
        h2 = [max(0.0, sum(h1[k] * W2[k][j] for k in range(h)) + b2[j]) for j in range(h)]
        yy = sum(h2[j] * w3[j] for j in range(h)) + b3
        assert abs(yy - y[b]) <= 1e-12 * (1 + abs(yy))


def test_gradient_matches_finite_differences():
    _check_gradient(mlp)


def test_forward_matches_per_sample_loop():
    _check_forward(mlp)


def test_parameter_count():
    assert mlp.n_params(24, 128) == 24 * 128 + 128 + 128 * 128 + 128 + 128 + 1


MUTANTS = [
    ('mean-square derivative without the 2', 'dy = 2.0 * e / B', 'dy = e / B'),
    ('W2 not transposed in the backward pass', 'dh1 = (dh2 @ W2.T) * (a1 > 0)',
     'dh1 = (dh2 @ W2) * (a1 > 0)'),
    ('ReLU mask dropped in the backward pass', 'dh2 = np.outer(dy, w3) * (a2 > 0)',
     'dh2 = np.outer(dy, w3)'),
    ('input not normalised by std', 'xn = (np.asarray(x, np.float64) - mean) / std',
     'xn = np.asarray(x, np.float64) - mean'),
    ('second bias dropped', 'a2 = h1 @ W2 + b2', 'a2 = h1 @ W2'),
]


@pytest.mark.parametrize('what,old,new', MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(what, old, new):
    with open(mlp.__file__) as f:
        text = f.read()
    assert text.count(old) == 1, what
    mod = types.ModuleType('mlp_copy')
    exec(compile(text.replace(old, new), mlp.__file__, 'exec'), mod.__dict__)
    with pytest.raises(AssertionError):
        _check_gradient(mod)
        _check_forward(mod)
