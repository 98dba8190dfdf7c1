"""Pins of the FP64 oracle MLP: analytic gradients equal central finite
differences of the loss, SiLU' equals the difference quotient of SiLU, and
Adam reduces the loss of a smooth regression."""
import numpy as np

from oracle import mlp


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    sizes = [7, 16, 16, 1]
    params = mlp.init_params(sizes, seed=1)
    x = rng.normal(size=(40, 7))
    y = rng.normal(size=40)
    _, grads = mlp.loss_and_grads(params, x, y)
    eps = 1e-6
    for li, (W, b) in enumerate(params):
        for arr, g in ((W, grads[li][0]), (b, grads[li][1])):
            flat = arr.reshape(-1)
            gflat = g.reshape(-1)
            for idx in rng.choice(flat.size, size=min(12, flat.size), replace=False):
                old = flat[idx]
                flat[idx] = old + eps
                lp, _ = mlp.loss_and_grads(params, x, y)
                flat[idx] = old - eps
                lm, _ = mlp.loss_and_grads(params, x, y)
                flat[idx] = old
                fd = (lp - lm) / (2 * eps)
                assert abs(fd - gflat[idx]) <= 1e-6 * max(1.0, abs(fd)), (li, idx, fd, gflat[idx])


def test_silu_grad_is_derivative():
    z = np.linspace(-8, 8, 101)
    h = 1e-6
    fd = (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h)
    assert np.allclose(mlp.silu_grad(z), fd, atol=1e-9)


def test_adam_reduces_loss():
    rng = np.random.default_rng(2)
    x = rng.uniform(-1, 1, size=(256, 3))
    y = np.sin(2 * x[:, 0]) + x[:, 1] * x[:, 2]
    params = mlp.init_params([3, 32, 32, 1], seed=3)
    state = mlp.adam_state(params)
    l0, _ = mlp.loss_and_grads(params, x, y)
    for t in range(1, 301):
        _, g = mlp.loss_and_grads(params, x, y)
        params = mlp.adam_step(params, g, state, 3e-3, t)
    l1, _ = mlp.loss_and_grads(params, x, y)
    assert l1 < 0.1 * l0


def test_vector_head_gradients_match_finite_differences():
    """The vector head's loss is the MSE over the first n of its output
    columns (the rates); the rest is padding and must get zero gradient."""
    rng = np.random.default_rng(2)
    n, O = 5, 8
    params = mlp.init_params([6, 12, 12, O], seed=4)
    x = rng.normal(size=(30, 6))
    y = rng.normal(size=(30, O))
    _, grads = mlp.loss_and_grads_vec(params, x, y, n)
    eps = 1e-6
    for li, (W, b) in enumerate(params):
        for arr, g in ((W, grads[li][0]), (b, grads[li][1])):
            flat, gflat = arr.reshape(-1), g.reshape(-1)
            for idx in rng.choice(flat.size, size=min(10, flat.size), replace=False):
                old = flat[idx]
                flat[idx] = old + eps
                lp, _ = mlp.loss_and_grads_vec(params, x, y, n)
                flat[idx] = old - eps
                lm, _ = mlp.loss_and_grads_vec(params, x, y, n)
                flat[idx] = old
                fd = (lp - lm) / (2 * eps)
                assert abs(fd - gflat[idx]) <= 1e-6 * max(1.0, abs(fd)), (li, idx, fd, gflat[idx])
    Wout, bout = grads[-1]
    assert np.all(Wout[n:] == 0) and np.all(bout[n:] == 0)
