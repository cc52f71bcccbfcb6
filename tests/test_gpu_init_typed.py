"""Initialisation from FP32 fields (lbm_init_fields_typed): the same populations as from
the FP64 fields holding the same values, bit for bit, from device tensors and from host
arrays, with and without the non-equilibrium stress and heat flux."""
import numpy as np
import pytest

from paper_1611_02409_gb300 import inputs

pytestmark = pytest.mark.gpu

CFG = dict(Pr=0.71, gamma=1.4, kappa=0.2, tau=0.7)


@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_1611_02409_gb300 import build
    build.build()
    from paper_1611_02409_gb300 import lbm
    return lbm


@pytest.mark.parametrize("where", ["device", "host"])
@pytest.mark.parametrize("neq", [False, True])
def test_fp32_fields_give_the_fp64_populations(L, where, neq):
    import torch
    ny, nx = 13, 21
    rho, u, T = inputs.random_fields((ny, nx), seed=8)
    rng = np.random.default_rng(8)
    Pi = np.stack([rho * T + 1e-3 * rng.uniform(-1, 1, (ny, nx)), 1e-3 * rng.uniform(-1, 1, (ny, nx)), rho * T])
    q = 1e-3 * rng.uniform(-1, 1, (2, ny, nx))
    fields = [rho, u, T] + ([Pi, q] if neq else [None, None])
    f32 = [None if a is None else np.ascontiguousarray(a, np.float32) for a in fields]
    f64 = [None if a is None else a.astype(np.float64) for a in f32]   # the same values in FP64
    conv = (lambda a: None if a is None else torch.from_numpy(a).cuda()) if where == "device" else (lambda a: a)
    out = []
    for fs in (f32, f64):
        sim = L.Simulation(nx=nx, ny=ny, **CFG)
        L.lbm_init_fields_typed(sim.h, *[conv(a) for a in fs])
        out.append(sim.populations())
        sim.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_typed_init_refuses_mixed_or_unknown_dtypes(L):
    sim = L.Simulation(nx=8, ny=8, **CFG)
    rho, u, T = inputs.random_fields((8, 8), seed=1)
    with pytest.raises(ValueError):
        L.lbm_init_fields_typed(sim.h, rho.astype(np.float32), u, T)
    import ctypes as C
    assert L.lib().lbm_init_fields_typed(sim.h, C.c_void_p(rho.ctypes.data), C.c_void_p(u.ctypes.data),
                                         C.c_void_p(T.ctypes.data), None, None, 7, L.LBM_MEM_HOST) == L.LBM_ERR_ARG
    sim.close()
