"""The FP64 reference of the surrogate network, pinned by central finite differences
of its own loss (the chain rule written out must agree with the derivative's definition)."""
import numpy as np

from oracle import mlp as M


def _setup(seed=3, n=37):
    g = np.random.default_rng(seed)
    p = g.normal(0.0, 0.3, M.N_PARAMS)
    x = g.normal(size=(n, M.N_IN)) * [1.0, 2.0, 0.5, 3.0] + [1.0, -2.0, 0.0, 5.0]
    t = g.normal(size=(n, M.N_OUT)) * [0.7, 1.5] + [-5.0, 1.0]
    norm = ([1.0, -2.0, 0.0, 5.0], [1.0, 2.0, 0.5, 3.0], [-5.0, 1.0], [0.7, 1.5])
    return p, x, t, norm


def test_backprop_matches_finite_differences():
    p, x, t, norm = _setup()
    _, grad = M.loss_and_grad(p, x, t, norm)
    g = np.random.default_rng(11)
    idx = np.concatenate([np.arange(0, 8), np.arange(256, 264), g.choice(M.N_PARAMS, 60, False),
                          np.arange(M.N_PARAMS - 6, M.N_PARAMS)])
    h = 1e-6
    for i in idx:
        e = np.zeros(M.N_PARAMS)
        e[i] = h
        fd = (M.loss_and_grad(p + e, x, t, norm)[0] - M.loss_and_grad(p - e, x, t, norm)[0]) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-7 * max(1.0, abs(fd)), (i, fd, grad[i])


def test_forward_closed_form_and_layout():
    """With W2 = 0 and b2 = 0 the second layer outputs tanh(0) = 0 and y = b3 in
    standardised units; the flat layout round-trips."""
    p, x, t, norm = _setup()
    w = M.unpack(p)
    w["W2"][:] = 0.0
    w["b2"][:] = 0.0
    y, _ = M.forward(M.pack(w), x, norm)
    np.testing.assert_allclose(y, np.broadcast_to(w["b3"] * norm[3] + norm[2], y.shape), rtol=1e-15)
    assert M.N_PARAMS == 4610
    np.testing.assert_array_equal(M.pack(M.unpack(p)), p)


def test_adam_constant_gradient_closed_form():
    """Adam (Kingma & Ba 2015, Algorithm 1) with a constant gradient g from zero moments:
    after t steps m1 = (1 - beta1^t) g and m2 = (1 - beta2^t) g^2, so the bias-corrected
    moments are exactly g and g^2 and every step moves a parameter by lr g / (|g| + eps),
    whatever t.  A 0-based step count (division by 1 - beta^0 = 0), a missing bias
    correction (steps shrink by 1 - beta1^t at first) or a sign slip all fail it."""
    g = np.array([2.5, -0.75, 1e-3, -40.0, 0.0])
    lr, eps = 1e-2, 1e-8
    p = np.array([0.3, -1.0, 2.0, 0.0, 5.0])
    m1 = np.zeros_like(p)
    m2 = np.zeros_like(p)
    for t in range(1, 31):
        p_new, m1, m2 = M.adam_step(p, g, m1, m2, t, lr, eps=eps)
        np.testing.assert_allclose(p - p_new, lr * g / (np.abs(g) + eps), rtol=1e-12, atol=0)
        np.testing.assert_allclose(m1, (1 - 0.9 ** t) * g, rtol=1e-12)
        np.testing.assert_allclose(m2, (1 - 0.999 ** t) * g * g, rtol=1e-12)
        p = p_new
