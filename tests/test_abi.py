"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/lbm.h declares.  Host-only entry points (lattice derivation, parameter
mapping) are checked against the oracle here; nothing launches a kernel."""
import ctypes as C

import numpy as np
import pytest

from oracle import oracle as O


@pytest.fixture(scope="module")
def L():
    from paper_1611_02409_gb300 import build
    build.build()
    from paper_1611_02409_gb300 import lbm
    return lbm


def test_exports_every_declared_symbol(L):
    names = L.exported_names()
    assert {"lbm_create", "lbm_init_fields", "lbm_step", "lbm_moments", "lbm_destroy",
            "lbm_diagnostics"} <= set(names)
    lib = L.lib()
    for n in names:
        assert hasattr(lib, n), n


@pytest.mark.parametrize("lat,olat", [(1, O.D2Q37), (2, O.D3Q103), (3, O.D2Q33), (4, O.D2Q77)])
def test_library_lattice_matches_oracle(L, lat, olat):
    # two independent FP64 derivations of the same lattice must agree.  D2Q77's degree-12
    # conditions leave its scale r a root known to ~1e-14 in double precision, and its
    # smallest weights (2e-7) move by ~1e-13 with it: compared absolutely there.
    D, r, c, w = L.lbm_lattice_table(lat)
    Do, ro, co, wo = O.lattice(olat)
    assert D == Do and len(c) == len(co)
    assert abs(r - ro) < 1e-13
    key = {tuple(v): wt for v, wt in zip(co, wo)}
    for v, wt in zip(c, w):
        if lat == 4:
            assert abs(wt - key[tuple(v)]) < 2e-13
        else:
            assert wt == pytest.approx(key[tuple(v)], rel=1e-12)
    # the library orders opposite velocities in adjacent pairs after the rest velocity
    assert tuple(c[0]) == (0, 0, 0)
    for k in range(1, len(c), 2):
        assert tuple(c[k + 1]) == tuple(-c[k])


@pytest.mark.parametrize("Pr,gamma,kappa,tau,mode", [(0.71, 1.4, 0.2, 0.528655, 0), (2.0, 1.3, 0.5, 1.0, 0),
                                                      (0.5, 1.67, 0.2, 1.0, 0), (0.71, 1.4, 0.2, 0.8, 1)])
def test_parameter_mapping_matches_oracle(L, Pr, gamma, kappa, tau, mode):
    p = L.make_params(Pr=Pr, gamma=gamma, kappa=kappa, tau=tau, pr_mode=mode)
    m = L.lbm_map_params(p)
    o = O.params(2, Pr, gamma, 0.0, kappa, tau, mode)
    for k in ("Nf", "omega", "nuG", "tau_s", "tau_q"):
        assert m[k] == pytest.approx(o[k], rel=1e-13, abs=1e-15), k
    assert m["warn"] == (m["nuG"] < -0.5)


def test_reference_state_fields_default_and_zero(L):
    # lbm_params ends with the reference state; 0 reads as 1 and the mapping ignores it
    assert [f[0] for f in L.lbm_params._fields_][-2:] == ["rho0", "T0"]
    assert L.make_params().rho0 == 1.0 and L.make_params().T0 == 1.0
    base = L.lbm_map_params(L.make_params())
    for ref in (dict(rho0=0.0, T0=0.0), dict(rho0=1.3, T0=0.8)):
        assert L.lbm_map_params(L.make_params(**ref)) == base


@pytest.mark.parametrize("bad", [dict(lattice=7), dict(tau=0.5), dict(Pr=0.0), dict(kappa=0.0), dict(kappa=1.2),
                                 dict(gamma=2.5), dict(gamma=1.0), dict(nx=0), dict(bc_y=1, ny=4),
                                 dict(storage=9), dict(pr_mode=4),
                                 dict(kappa=1.0, Pr=0.71), dict(pr_mode=1, Pr=2.0, tau=0.9),
                                 dict(bc_y=1, ny=16, wall_T=[1.0, -1.0]), dict(lattice=3, bc_y=1, ny=16),
                                 dict(lattice=4, bc_y=1, ny=16),
                                 dict(bc_x=5), dict(lattice=2, bc_x=2),
                                 dict(nx=4, ny=65536), dict(nx=4, ny=65532, bc_y=1),
                                 dict(lattice=2, nx=4, ny=4, nz=65536),
                                 dict(rho0=-1.0), dict(T0=-0.5), dict(T0=float("nan")), dict(rho0=float("inf"))])
def test_invalid_parameters_rejected_without_gpu(L, bad):
    p = L.make_params(**bad)
    with pytest.raises(L.LbmError) as e:
        L.lbm_map_params(p)
    assert e.value.code == L.LBM_ERR_ARG
    # lbm_create rejects the same set before touching the device
    h = C.c_void_p()
    assert L.lib().lbm_create(C.byref(p), None, C.byref(h)) == L.LBM_ERR_ARG
    assert not h.value
    assert L.lbm_last_error()


@pytest.mark.parametrize("nx,ny,walls", [(6000, 6000, 0), (450, 64489, 0), (450, 64485, 1)])
def test_batch_rejects_instances_beyond_32bit_offsets(L, nx, ny, walls):
    # the batched step forms p * plane + cell (p < 74) in 32-bit integers: an instance
    # whose 74 planes reach 2^31 values (plane > 29,020,049 cells) is refused at creation,
    # before any device work
    p = L.make_params(nx=nx, ny=ny, bc_y=walls, tau=0.8)
    h = C.c_void_p()
    assert L.lib().lbm_batch_create(1, C.byref(p), C.byref(h)) == L.LBM_ERR_ARG
    assert b"2^31" in L.lib().lbm_last_error(None)


@pytest.mark.parametrize("D,Nf,n,null,what", [
    (4, 3.0, 1000, False, "D must be 2 or 3"),
    (1, 3.0, 1000, False, "D must be 2 or 3"),
    (2, -1.0, 1000, False, "N_f"),
    (2, float("nan"), 1000, False, "N_f"),
    (2, 3.0, 1000, True, "null pointer"),
    (2, 3.0, 0, False, "n must be"),
    (3, 3.0, 33554433, False, "33554432"),
])
def test_field_totals_static_refusals_without_gpu(L, D, Nf, n, null, what):
    # every refusal of the allocation-free totals is decided from the arguments alone,
    # before any CUDA call, so it needs no GPU; the pointers are never dereferenced
    fake = None if null else C.c_void_p(0x1000)
    rc = L.lib().lbm_field_totals_static(D, Nf, n, fake, C.c_void_p(0x2000), C.c_void_p(0x3000),
                                         C.c_void_p(0x4000), None)
    assert rc == L.LBM_ERR_ARG
    assert what in L.lbm_last_error()


def test_field_totals_static_wrapper_checks_arguments(L):
    # host arrays or wrong dtypes never reach the library (the kernel would be given a host
    # pointer); on a machine without CUDA the check still refuses before any device call
    torch = pytest.importorskip("torch")
    x = torch.zeros(8, dtype=torch.float64)
    with pytest.raises(ValueError):
        L.lbm_field_totals_static(2, 3.0, x, torch.zeros(16, dtype=torch.float64), x, torch.zeros(6, dtype=torch.float64))
    with pytest.raises(ValueError):
        L.lbm_field_totals_static(2, 3.0, np.zeros(8), np.zeros(16), np.zeros(8), np.zeros(6))


@pytest.mark.parametrize("lat,olat", [(1, O.D2Q37), (2, O.D3Q103), (3, O.D2Q33), (4, O.D2Q77)])
def test_lattice_unit_scale(L, lat, olat):
    # dx = r dt: the same r as the lattice table, and the oracle's independent derivation
    r = L.lbm_lattice_unit_scale(lat)
    assert r == L.lbm_lattice_table(lat)[1]
    assert abs(r - O.lattice(olat)[1]) < 1e-13
    with pytest.raises(L.LbmError):
        L.lbm_lattice_unit_scale(9)


def test_typed_init_refuses_a_null_handle(L):
    assert L.lib().lbm_init_fields_typed(None, None, None, None, None, None, 1, 1) == L.LBM_ERR_ARG
