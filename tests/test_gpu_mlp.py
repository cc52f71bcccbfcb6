"""Surrogate network on the GPU (lbm_mlp_*) against the FP64 reference (oracle/mlp_oracle).

With quantize=True the reference rounds to bfloat16 exactly the operands the kernels
hold in bfloat16, so the remaining differences are FP32 accumulation order and the
occasional bfloat16 rounding flip of a value that FP32 and FP64 place on opposite sides
of a rounding boundary (2^-8 on that element): 2e-3 on outputs, 1e-2 on gradient norms.
Against the unquantised FP64 network the bfloat16 operands themselves (2^-8) dominate.
Both product forms are checked: tcgen05 MMAs (the default) and warp-level mma.sync.
"""
import numpy as np
import pytest

from oracle import mlp_oracle as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_1611_02409_gb300 import build
    build.build()
    from paper_1611_02409_gb300 import lbm
    return lbm


def relerr(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-30))


GEMMS = [0, 1]  # LBM_MLP_GEMM_TCGEN05, LBM_MLP_GEMM_MMA_SYNC


@pytest.mark.parametrize("gemm", GEMMS)
@pytest.mark.parametrize("sizes,batch", [([5, 64, 48, 40], 37), ([5, 512, 512, 512, 512, 1024], 256),
                                         ([5, 200, 130, 72], 300), ([5, 1024, 1024], 1100)])
def test_forward_and_gradients_match_reference(L, sizes, batch, gemm):
    # the third case is ragged in every product dimension against the 128-row tcgen05
    # tiles and their 64-wide K steps (batch 300 = 2 x 128 + 44; widths 200, 130, 72); the
    # products of the small cases run on 32-wide tiles (64-wide ones would leave most SMs
    # idle), the 1100 x 1024 x 1024 ones of the last case on 64-wide tiles
    import torch
    rng = np.random.default_rng(5)
    params = M.init_params(sizes, seed=11)
    for W, b in params:  # nonzero biases exercise the bias paths
        b[:] = rng.normal(size=b.shape) * 0.1
    x = rng.normal(size=(batch, sizes[0]))
    t = rng.normal(size=(batch, sizes[-1])) * 0.5
    net = L.MLP(sizes, max_batch=batch, gemm=gemm)
    net.set_params(params)
    params32 = [[W.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64)]
                for W, b in params]
    y = net.forward(torch.tensor(x, dtype=torch.float32)).cpu().numpy()
    loss = net.backward(torch.tensor(t, dtype=torch.float32))
    _, grads = net.get_params(with_grads=True)
    x32 = x.astype(np.float32).astype(np.float64)
    t32 = t.astype(np.float32).astype(np.float64)
    yq, _, _ = M.forward(params32, x32, quantize=True)
    lq, gq = M.loss_and_grads(params32, x32, t32, quantize=True)
    assert relerr(y, yq) < 2e-3
    assert abs(loss - lq) < 2e-3 * lq
    for l in range(len(sizes) - 1):
        assert relerr(grads[l][0], gq[l][0]) < 1e-2, ("W", l, relerr(grads[l][0], gq[l][0]))
        assert relerr(grads[l][1], gq[l][1]) < 1e-2, ("b", l, relerr(grads[l][1], gq[l][1]))
    y64, _, _ = M.forward(params32, x32)
    _, g64 = M.loss_and_grads(params32, x32, t32)
    assert relerr(y, y64) < 3e-2
    for l in range(len(sizes) - 1):
        assert relerr(grads[l][0], g64[l][0]) < 5e-2
    net.close()


def test_gemm_forms_agree(L):
    # the two product forms accumulate the same bfloat16 products in FP32 in different
    # orders: outputs agree to FP32 accumulation roundoff
    import torch
    sizes = [5, 512, 512, 1024]
    rng = np.random.default_rng(3)
    params = M.init_params(sizes, seed=2)
    x = torch.tensor(rng.normal(size=(128, 5)), dtype=torch.float32)
    ys = []
    for gemm in GEMMS:
        net = L.MLP(sizes, max_batch=128, gemm=gemm)
        net.set_params(params)
        ys.append(net.forward(x).cpu().numpy())
        net.close()
    assert relerr(ys[0], ys[1]) < 1e-3


def test_set_gemm_rejects_unknown_kind(L):
    net = L.MLP([5, 8, 4], max_batch=4)
    with pytest.raises(RuntimeError):
        L._check(L.lib().lbm_mlp_set_gemm(net.h, 7))
    net.close()


def test_adam_step_matches_reference(L):
    import torch
    sizes = [5, 32, 16]
    rng = np.random.default_rng(2)
    params = M.init_params(sizes, seed=4)
    net = L.MLP(sizes, max_batch=20)
    net.set_params(params)
    x, t = rng.normal(size=(20, 5)), rng.normal(size=(20, 16))
    net.forward(torch.tensor(x, dtype=torch.float32))
    net.backward(torch.tensor(t, dtype=torch.float32))
    p0, g = net.get_params(with_grads=True)
    net.adam(lr=1e-2)
    p1 = net.get_params()
    ref = [[W.copy(), b.copy()] for W, b in p0]
    M.adam_step(ref, g, {}, lr=1e-2)
    for l in range(2):
        for j in range(2):
            assert np.allclose(p1[l][j], ref[l][j], rtol=1e-5, atol=1e-6)
    net.close()


@pytest.mark.parametrize("gemm", GEMMS)
def test_training_reduces_loss(L, gemm):
    import torch
    sizes = [5, 64, 64, 8]
    rng = np.random.default_rng(9)
    x = rng.uniform(-1, 1, size=(256, 5))
    t = np.stack([np.sin(x @ rng.normal(size=5)) for _ in range(8)], axis=1)
    net = L.MLP(sizes, max_batch=256, gemm=gemm)
    net.set_params(M.init_params(sizes, seed=1))
    xt, tt = torch.tensor(x, dtype=torch.float32), torch.tensor(t, dtype=torch.float32)
    losses = []
    for it in range(600):
        net.forward(xt)
        l = net.backward(tt, want_loss=(it % 100 == 0 or it == 599))
        if l is not None:
            losses.append(l)
        net.adam(lr=3e-3)
    assert losses[-1] < 0.1 * losses[0], losses
    net.close()
