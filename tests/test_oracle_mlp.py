"""Pins of the ranker network's FP64 oracle: the gradient against central
finite differences of the loss, a closed form at a degenerate point, and the
first Adam step (which moves every parameter by lr * sign(g) up to eps)."""
import numpy as np

from oracle import mlp_oracle as mo


def _rand(F, H, seed):
    rng = np.random.default_rng(seed)
    p = rng.normal(0, 0.5, mo.param_count(F, H))
    X = rng.normal(0, 1, (9, F))
    t = rng.normal(0, 1, 9)
    return p, X, t


def test_gradient_matches_finite_differences():
    F, H = 5, 7
    p, X, t = _rand(F, H, 0)
    loss, g = mo.loss_and_grad(p, F, H, X, t)
    _, (_, a1, _, a2, _) = mo.forward(p, F, H, X)
    assert min(np.abs(a1).min(), np.abs(a2).min()) > 1e-4   # no kink within the step
    h = 1e-6
    fd = np.empty_like(p)
    for i in range(p.size):
        q = p.copy(); q[i] += h
        lp = mo.loss_and_grad(q, F, H, X, t)[0]
        q[i] -= 2 * h
        lm = mo.loss_and_grad(q, F, H, X, t)[0]
        fd[i] = (lp - lm) / (2 * h)
    assert np.allclose(g, fd, rtol=1e-6, atol=1e-8)
    assert loss > 0


def test_closed_form_at_zero_first_layer():
    # W1 = 0, b1 = 0: h1 = 0; W2 = 0, b2 = c > 0: h2 = c; y = c sum(w3) + b3 for every row
    F, H, c = 3, 4, 0.7
    rng = np.random.default_rng(1)
    w3 = rng.normal(size=H)
    b3 = 0.3
    p = mo.pack(np.zeros((H, F)), np.zeros(H), np.zeros((H, H)), np.full(H, c), w3, b3)
    X = rng.normal(size=(6, F))
    t = rng.normal(size=6)
    y, _ = mo.forward(p, F, H, X)
    assert np.allclose(y, c * w3.sum() + b3)
    loss, g = mo.loss_and_grad(p, F, H, X, t)
    W1, b1, W2, b2, dw3, db3 = mo.unpack(g, F, H)
    r = 2 * np.mean(c * w3.sum() + b3 - t)
    assert np.isclose(loss, np.mean((c * w3.sum() + b3 - t) ** 2))
    assert np.isclose(db3, r)
    assert np.allclose(dw3, r * c)
    assert np.allclose(b2, r * w3)
    assert np.allclose(W2, 0) and np.allclose(W1, 0) and np.allclose(b1, 0)   # relu'(0) = 0, h1 = 0


def test_first_adam_step_is_lr_times_sign():
    rng = np.random.default_rng(2)
    p = rng.normal(size=10)
    g = rng.normal(size=10)
    q, m, v = mo.adam(p, g, np.zeros(10), np.zeros(10), 1, 1e-3, 0.9, 0.999, 1e-12)
    assert np.allclose(q, p - 1e-3 * np.sign(g), rtol=0, atol=1e-12)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
