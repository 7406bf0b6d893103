"""Pins of the FP64 MLP oracle: activation closed forms and derivatives,
gradients against central finite differences."""
import numpy as np
import pytest

from oracle import mlp as M


def test_activation_values():
    z = np.array([-2.0, -0.5, 0.0, 0.7, 3.0])
    assert np.allclose(M.act(z, M.ELU), [np.exp(-2) - 1, np.exp(-0.5) - 1, 0, 0.7, 3.0], atol=1e-15)
    assert np.allclose(M.act(z, M.SILU), z * (1 / (1 + np.exp(-z))), atol=1e-15)
    assert abs(M.act(np.array([0.0]), M.SILU)[0]) == 0.0
    assert np.allclose(M.act(z, M.TANH), np.tanh(z))


@pytest.mark.parametrize("kind", [M.ELU, M.SILU, M.TANH, M.NONE])
def test_activation_derivatives_match_differences(kind):
    z = np.linspace(-3, 3, 61) + 0.013
    h = 1e-6
    num = (M.act(z + h, kind) - M.act(z - h, kind)) / (2 * h)
    assert np.abs(num - M.act_grad(z, kind)).max() < 1e-8


@pytest.mark.parametrize("dims,hidden,out", [([30, 24, 24, 16], M.SILU, M.NONE), ([20, 32, 16, 3], M.ELU, M.TANH)])
def test_gradients_match_central_differences(dims, hidden, out):
    rng = np.random.default_rng(1)
    params = [(rng.normal(0, 1 / np.sqrt(i), (o, i)), rng.normal(0, 0.1, o)) for i, o in zip(dims[:-1], dims[1:])]
    x = rng.normal(0, 1, (12, dims[0]))
    t = rng.normal(0, 0.5, (12, dims[-1]))
    grads = M.backward(params, x, t, hidden, out)
    h = 1e-6
    for l, (W, b) in enumerate(params):
        for idx in [(0, 0), (W.shape[0] - 1, W.shape[1] - 1), (W.shape[0] // 2, W.shape[1] // 3)]:
            Wp, Wm = W.copy(), W.copy()
            Wp[idx] += h; Wm[idx] -= h
            pp = list(params); pp[l] = (Wp, b)
            pm = list(params); pm[l] = (Wm, b)
            num = (M.mse(M.forward(pp, x, hidden, out), t) - M.mse(M.forward(pm, x, hidden, out), t)) / (2 * h)
            assert abs(num - grads[l][0][idx]) <= 1e-6 * max(1.0, abs(num)) + 1e-9
        bp, bm = b.copy(), b.copy()
        bp[0] += h; bm[0] -= h
        pp = list(params); pp[l] = (W, bp)
        pm = list(params); pm[l] = (W, bm)
        num = (M.mse(M.forward(pp, x, hidden, out), t) - M.mse(M.forward(pm, x, hidden, out), t)) / (2 * h)
        assert abs(num - grads[l][1][0]) <= 1e-6 * max(1.0, abs(num)) + 1e-9
