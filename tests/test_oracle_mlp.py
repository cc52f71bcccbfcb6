"""Pins of the FP64 surrogate-network reference (oracle/mlp_oracle.py): backpropagated
gradients against central finite differences of the loss, the GELU derivative against a
finite difference of GELU, bfloat16 rounding against exhaustive neighbours, and one
Adam step against its closed form."""
import numpy as np
import pytest

from oracle import mlp_oracle as M


def test_gelu_derivative_by_finite_differences():
    z = np.linspace(-6, 6, 241)
    h = 1e-6
    fd = (M.gelu(z + h) - M.gelu(z - h)) / (2 * h)
    assert np.abs(fd - M.gelu_grad(z)).max() < 1e-8
    # GELU(z) -> z for large z, -> 0 for very negative z, GELU(0) = 0
    assert M.gelu(np.array([0.0]))[0] == 0.0
    assert abs(M.gelu(np.array([8.0]))[0] - 8.0) < 1e-12


def test_bf16_rounding_to_nearest_even():
    rng = np.random.default_rng(0)
    x = rng.normal(size=2000) * 10.0 ** rng.integers(-6, 6, size=2000)
    q = M.bf16(x)
    f32 = x.astype(np.float32).view(np.uint32)
    lo = (f32 & 0xFFFF0000).view(np.float32).astype(np.float64)
    hi = ((f32 & 0xFFFF0000) + 0x10000).astype(np.uint32).view(np.float32).astype(np.float64)
    xf = x.astype(np.float32).astype(np.float64)
    # q is one of the two bfloat16 neighbours of the float32 value, and the nearer one
    assert np.all((q == lo) | (q == hi))
    assert np.all(np.abs(q - xf) <= np.minimum(np.abs(lo - xf), np.abs(hi - xf)) + 0.0)


@pytest.mark.parametrize("quantize", [False, True])
def test_backprop_matches_finite_differences(quantize):
    sizes = [5, 7, 6, 4]
    params = M.init_params(sizes, seed=3)
    rng = np.random.default_rng(1)
    x, t = rng.normal(size=(9, 5)), rng.normal(size=(9, 4))
    if quantize:
        # the finite difference must see the same rounding: perturb in FP64 with
        # quantisation off, and compare the unquantised gradient (the quantised one
        # only differs by bf16 rounding of its operands, checked for closeness)
        _, g_q = M.loss_and_grads(params, x, t, quantize=True)
    _, grads = M.loss_and_grads(params, x, t)
    h = 1e-6
    for l in range(len(params)):
        for j in range(2):
            p = params[l][j]
            it = np.nditer(p, flags=["multi_index"])
            for _ in it:
                idx = it.multi_index
                old = p[idx]
                p[idx] = old + h
                lp, _ = M.loss_and_grads(params, x, t)
                p[idx] = old - h
                lm, _ = M.loss_and_grads(params, x, t)
                p[idx] = old
                fd = (lp - lm) / (2 * h)
                assert abs(fd - grads[l][j][idx]) < 1e-7 + 1e-6 * abs(fd), (l, j, idx)
            if quantize:
                rel = np.linalg.norm(g_q[l][j] - grads[l][j]) / max(np.linalg.norm(grads[l][j]), 1e-30)
                assert rel < 3e-2, (l, j, rel)


def test_adam_first_step_closed_form():
    params = [[np.array([[1.0, -2.0]]), np.array([0.5, 0.0])]]
    grads = [[np.array([[0.1, -0.3]]), np.array([2.0, 0.0])]]
    state = {}
    M.adam_step(params, grads, state, lr=0.01)
    # first step: mhat = g, vhat = g^2 -> w -= lr * sign(g) (up to eps)
    assert np.allclose(params[0][0], [[1.0 - 0.01, -2.0 + 0.01]], atol=1e-9)
    assert np.allclose(params[0][1], [0.5 - 0.01, 0.0], atol=1e-9)
