"""Python binding of the C ABI in ``include/lbm.h`` (argument marshalling only).

Every computation runs in the CUDA library ``liblbm.so``; this module converts
arguments, passes device pointers of torch tensors (or host numpy arrays) and
raises on error codes.  There is no CPU fallback: if the library is missing the
import of :func:`lib` fails loudly.
"""
from __future__ import annotations

import ctypes as C
import os
import re
import threading

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "liblbm.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "lbm.h")

LBM_OK = 0
LBM_ERR_ARG = 1
LBM_ERR_CUDA = 2
LBM_ERR_UNSTABLE = 3
LBM_ERR_NOMEM = 4
LBM_ERR_TIMEOUT = 5
LBM_WARN_PR_RANGE = 100
LBM_D2Q37 = 1
LBM_D3Q103 = 2
LBM_D2Q33 = 3
LBM_D2Q77 = 4
LBM_AUDIT_BATCH = 5
LBM_PR_SHIFTED = 0
LBM_PR_LITERAL = 1
LBM_FP32 = 0
LBM_FP16 = 1
LBM_BF16 = 2
LBM_FP64 = 3
LBM_PERIODIC = 0
LBM_WALLS = 1
LBM_OPEN = 2
LBM_KERNEL_AUTO = 0
LBM_KERNEL_DIRECT = 1
LBM_KERNEL_STAGED = 2
LBM_KERNEL_PAIRED = 3
LBM_KERNEL_TWOPASS = 4
LBM_MLP_GEMM_TCGEN05 = 0
LBM_MLP_GEMM_MMA_SYNC = 1
LBM_MEM_DEVICE = 0
LBM_MEM_HOST = 1

STORAGE = {"fp32": LBM_FP32, "fp16": LBM_FP16, "bf16": LBM_BF16, "fp64": LBM_FP64}


class LbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"lbm error {code}: {msg}")
        self.code = code


class lbm_params(C.Structure):
    _fields_ = [("lattice", C.c_int), ("Pr", C.c_double), ("gamma", C.c_double), ("N_f", C.c_double),
                ("kappa", C.c_double), ("tau", C.c_double), ("pr_mode", C.c_int), ("storage", C.c_int),
                ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("bc_y", C.c_int),
                ("wall_u", (C.c_double * 3) * 2), ("wall_T", C.c_double * 2), ("bc_x", C.c_int),
                ("rho0", C.c_double), ("T0", C.c_double)]


def make_params(lattice=LBM_D2Q37, Pr=0.71, gamma=1.4, N_f=0.0, kappa=0.2, tau=0.6, pr_mode=LBM_PR_SHIFTED,
                storage=LBM_FP32, nx=64, ny=64, nz=1, bc_y=LBM_PERIODIC, wall_u=None, wall_T=None,
                bc_x=LBM_PERIODIC, rho0=1.0, T0=1.0) -> lbm_params:
    p = lbm_params()
    p.lattice, p.Pr, p.gamma, p.N_f, p.kappa, p.tau = lattice, Pr, gamma, N_f, kappa, tau
    p.pr_mode = pr_mode
    p.storage = STORAGE.get(storage, storage) if isinstance(storage, str) else storage
    p.nx, p.ny, p.nz, p.bc_y, p.bc_x = nx, ny, nz, bc_y, bc_x
    p.rho0, p.T0 = rho0, T0
    wu = np.zeros((2, 3)) if wall_u is None else np.asarray(wall_u, float).reshape(2, 3)
    wT = np.ones(2) if wall_T is None else np.asarray(wall_T, float).reshape(2)
    for b in range(2):
        for d in range(3):
            p.wall_u[b][d] = wu[b, d]
        p.wall_T[b] = wT[b]
    return p


_lock = threading.Lock()
_lib = None


def exported_names() -> list[str]:
    """Entry points declared in include/lbm.h."""
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|long long|const char \*|void)\s*\*?\s*(lbm_\w+)\s*\(", src, re.M)))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library {LIB_PATH} is not built; run paper_1611_02409_gb300.build.build()")
            L = C.CDLL(LIB_PATH)
            vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int)
            L.lbm_create.argtypes = [C.POINTER(lbm_params), vp, C.POINTER(vp)]
            L.lbm_destroy.argtypes = [vp]
            L.lbm_last_error.argtypes = [vp]
            L.lbm_last_error.restype = C.c_char_p
            L.lbm_lattice_info.argtypes = [vp, ip, ip, dp, ip, dp]
            L.lbm_lattice_table.argtypes = [C.c_int, ip, ip, dp, ip, dp]
            L.lbm_lattice_unit_scale.argtypes = [C.c_int, dp]
            L.lbm_debug_index_audit.argtypes = [C.POINTER(lbm_params), C.c_int, C.c_int]
            L.lbm_debug_index_audit.restype = C.c_longlong
            L.lbm_debug_reference_state.argtypes = [C.POINTER(lbm_params), dp, dp, dp]
            L.lbm_map_params.argtypes = [C.POINTER(lbm_params), dp]
            L.lbm_coefficients.argtypes = [vp, dp]
            L.lbm_init_fields.argtypes = [vp, vp, vp, vp, C.c_int]
            L.lbm_init_fields_neq.argtypes = [vp, vp, vp, vp, vp, vp, C.c_int]
            L.lbm_init_fields_typed.argtypes = [vp, vp, vp, vp, vp, vp, C.c_int, C.c_int]
            L.lbm_batch_init_fields_neq.argtypes = [vp, C.c_int, vp, vp, vp, vp, vp, C.c_int]
            L.lbm_step.argtypes = [vp, C.c_int]
            L.lbm_moments.argtypes = [vp, vp, vp, vp, vp, vp, C.c_int]
            L.lbm_diagnostics.argtypes = [vp, dp]
            L.lbm_get_populations.argtypes = [vp, vp, vp, C.c_int]
            L.lbm_set_populations.argtypes = [vp, vp, vp, C.c_int]
            L.lbm_set_kernel.argtypes = [vp, C.c_int]
            L.lbm_debug_inject_stall.argtypes = [vp, C.c_int]
            L.lbm_batch_create.argtypes = [C.c_int, C.POINTER(lbm_params), C.POINTER(vp)]
            L.lbm_batch_destroy.argtypes = [vp]
            L.lbm_batch_init_fields.argtypes = [vp, C.c_int, vp, vp, vp, C.c_int]
            L.lbm_batch_run.argtypes = [vp, C.c_int, C.c_double, C.c_int, ip]
            L.lbm_batch_status.argtypes = [vp, ip, dp, ip]
            L.lbm_batch_activate.argtypes = [vp, C.c_int]
            L.lbm_batch_moments.argtypes = [vp, C.c_int, vp, vp, vp, vp, vp, C.c_int]
            L.lbm_batch_autotune.argtypes = [vp, C.c_int, ip]
            L.lbm_mlp_create.argtypes = [C.c_int, ip, C.c_int, vp, C.POINTER(vp)]
            L.lbm_mlp_destroy.argtypes = [vp]
            L.lbm_mlp_num_params.argtypes = [vp]
            L.lbm_mlp_num_params.restype = C.c_longlong
            L.lbm_mlp_set_params.argtypes = [vp, vp]
            L.lbm_mlp_get_params.argtypes = [vp, vp, vp]
            L.lbm_mlp_forward.argtypes = [vp, C.c_int, vp, vp]
            L.lbm_mlp_backward.argtypes = [vp, vp, dp]
            L.lbm_mlp_adam.argtypes = [vp, C.c_float, C.c_float, C.c_float, C.c_float]
            L.lbm_mlp_set_gemm.argtypes = [vp, C.c_int]
            L.lbm_field_totals_static.argtypes = [C.c_int, C.c_double, C.c_longlong, vp, vp, vp, vp, vp]
            L.lbm_autotune.argtypes = [vp, C.c_int, ip]
            _lib = L
    return _lib


def lbm_last_error(h=None) -> str:
    return lib().lbm_last_error(h).decode()


def _check(code, h=None, warn_ok=False):
    if code == LBM_OK or (warn_ok and code == LBM_WARN_PR_RANGE):
        return code
    raise LbmError(code, lbm_last_error(h))


def lbm_lattice_table(lattice=LBM_D2Q37):
    """(D, r, c[Q,3], w[Q]) as derived by the library's host code (no GPU needed)."""
    D, Q, r = C.c_int(), C.c_int(), C.c_double()
    c = np.zeros((128, 3), np.int32)
    w = np.zeros(128)
    _check(lib().lbm_lattice_table(lattice, C.byref(D), C.byref(Q), C.byref(r),
                                   c.ctypes.data_as(C.POINTER(C.c_int)), w.ctypes.data_as(C.POINTER(C.c_double))))
    return D.value, r.value, c[:Q.value].copy(), w[:Q.value].copy()


def lbm_lattice_unit_scale(lattice=LBM_D2Q37) -> float:
    """The lattice's scale r (dx = r dt in the paper's units); no GPU needed."""
    r = C.c_double()
    _check(lib().lbm_lattice_unit_scale(int(lattice), C.byref(r)))
    return r.value


def lbm_debug_index_audit(p: lbm_params, variant: int, wrap_threshold: int = 0) -> int:
    """Out-of-range (or misaligned) accesses of a kernel variant's addressing for the
    configuration p, audited on the host (no GPU needed); raises on invalid arguments."""
    n = lib().lbm_debug_index_audit(C.byref(p), int(variant), int(wrap_threshold))
    if n < 0:
        raise LbmError(int(-n), "index audit: invalid configuration or variant")
    return n


def lbm_debug_reference_state(p: lbm_params):
    """The reference state's per-velocity shifts dg, dh and moment shares as the kernels
    use them (host only); raises on invalid parameters."""
    Q = len(lbm_lattice_table(p.lattice)[2])
    dg, dh, share = np.zeros(Q), np.zeros(Q), np.zeros(5)
    f = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    q = lib().lbm_debug_reference_state(C.byref(p), f(dg), f(dh), f(share))
    if q < 0:
        raise LbmError(int(-q), "reference state: invalid configuration")
    return dg, dh, share


def lbm_map_params(p: lbm_params) -> dict:
    """Mapped coefficients of a parameter set (no GPU needed); raises on invalid sets."""
    out = np.zeros(6)
    code = lib().lbm_map_params(C.byref(p), out.ctypes.data_as(C.POINTER(C.c_double)))
    _check(code, None, warn_ok=True)
    return dict(Nf=out[0], omega=out[1], nuG=out[2], tau_s=out[3], tau_q=out[4], kappa=out[5],
                warn=code == LBM_WARN_PR_RANGE)


def _ptr(x):
    """(pointer, mem) of a torch CUDA tensor or a host numpy array (float64, contiguous)."""
    if x is None:
        return None, None
    if hasattr(x, "data_ptr"):
        if str(x.dtype) != "torch.float64" or not x.is_contiguous():
            raise ValueError("fields must be contiguous float64")
        return C.c_void_p(x.data_ptr()), (LBM_MEM_DEVICE if x.is_cuda else LBM_MEM_HOST)
    if x.dtype != np.float64 or not x.flags.c_contiguous:
        raise ValueError("fields must be contiguous float64")
    return C.c_void_p(x.ctypes.data), LBM_MEM_HOST


def _mem_of(*xs):
    mems = {m for _, m in map(_ptr, xs) if m is not None}
    if len(mems) != 1:
        raise ValueError("all fields must live in the same memory space")
    return mems.pop()


def lbm_create(p: lbm_params, stream=None):
    """Returns (handle, warn) with warn True for LBM_WARN_PR_RANGE."""
    h = C.c_void_p()
    s = C.c_void_p(stream) if isinstance(stream, int) else C.c_void_p(getattr(stream, "cuda_stream", 0) or 0)
    code = lib().lbm_create(C.byref(p), s, C.byref(h))
    _check(code, None, warn_ok=True)
    return h, code == LBM_WARN_PR_RANGE


def lbm_destroy(h):
    return _check(lib().lbm_destroy(h), None)


def lbm_init_fields(h, rho, u, T):
    mem = _mem_of(rho, u, T)
    return _check(lib().lbm_init_fields(h, _ptr(rho)[0], _ptr(u)[0], _ptr(T)[0], mem), h)


def lbm_init_fields_neq(h, rho, u, T, Pi=None, q=None):
    mem = _mem_of(*[x for x in (rho, u, T, Pi, q) if x is not None])
    return _check(lib().lbm_init_fields_neq(h, *(_ptr(x)[0] for x in (rho, u, T, Pi, q)), mem), h)


LBM_DTYPE_F64 = 0
LBM_DTYPE_F32 = 1


def lbm_init_fields_typed(h, rho, u, T, Pi=None, q=None):
    """lbm_init_fields_neq with FP32 or FP64 fields (all of one dtype and one memory space:
    torch tensors on the device or host numpy arrays, contiguous)."""
    xs = [x for x in (rho, u, T, Pi, q) if x is not None]
    names = {str(x.dtype).replace("torch.", "") for x in xs}
    if names == {"float64"}:
        dtype = LBM_DTYPE_F64
    elif names == {"float32"}:
        dtype = LBM_DTYPE_F32
    else:
        raise ValueError(f"fields must all be float32 or all float64, got {sorted(names)}")
    mems = set()
    ptrs = []
    for x in (rho, u, T, Pi, q):
        if x is None:
            ptrs.append(None)
            continue
        if hasattr(x, "data_ptr"):
            if not x.is_contiguous():
                raise ValueError("fields must be contiguous")
            ptrs.append(C.c_void_p(x.data_ptr()))
            mems.add(LBM_MEM_DEVICE if x.is_cuda else LBM_MEM_HOST)
        else:
            if not x.flags.c_contiguous:
                raise ValueError("fields must be contiguous")
            ptrs.append(C.c_void_p(x.ctypes.data))
            mems.add(LBM_MEM_HOST)
    if len(mems) != 1:
        raise ValueError("all fields must live in the same memory space")
    return _check(lib().lbm_init_fields_typed(h, *ptrs, dtype, mems.pop()), h)


def lbm_step(h, nsteps=1):
    return _check(lib().lbm_step(h, int(nsteps)), h)


def lbm_moments(h, rho=None, u=None, T=None, Pi=None, q=None):
    xs = [x for x in (rho, u, T, Pi, q) if x is not None]
    mem = _mem_of(*xs) if xs else LBM_MEM_DEVICE
    return _check(lib().lbm_moments(h, *(_ptr(x)[0] for x in (rho, u, T, Pi, q)), mem), h)


def lbm_diagnostics(h, check=True):
    out = np.zeros(8)
    code = lib().lbm_diagnostics(h, out.ctypes.data_as(C.POINTER(C.c_double)))
    if check:
        _check(code, h)
    return dict(mass=out[0], momentum=out[1:4].copy(), energy=out[4], residual=out[5], bad=int(out[6]),
                steps=int(out[7]), code=code)


def lbm_lattice_info(h):
    D, Q, r = C.c_int(), C.c_int(), C.c_double()
    c = np.zeros((128, 3), np.int32)
    w = np.zeros(128)
    _check(lib().lbm_lattice_info(h, C.byref(D), C.byref(Q), C.byref(r), c.ctypes.data_as(C.POINTER(C.c_int)),
                                  w.ctypes.data_as(C.POINTER(C.c_double))), h)
    return D.value, r.value, c[:Q.value].copy(), w[:Q.value].copy()


def lbm_coefficients(h) -> dict:
    out = np.zeros(6)
    _check(lib().lbm_coefficients(h, out.ctypes.data_as(C.POINTER(C.c_double))), h)
    return dict(Nf=out[0], omega=out[1], nuG=out[2], tau_s=out[3], tau_q=out[4], kappa=out[5])


def lbm_set_kernel(h, variant):
    return _check(lib().lbm_set_kernel(h, int(variant)), h)


def lbm_autotune(h, steps=10) -> int:
    chosen = C.c_int()
    _check(lib().lbm_autotune(h, int(steps), C.byref(chosen)), h)
    return chosen.value


def lbm_field_totals_static(D, N_f, rho, u, T, out, stream=None):
    """Conservation totals of device fields into the device array `out` (6 doubles),
    without any allocation; see include/lbm.h.  The kernel reads rho, u and T and writes
    out through raw device pointers, so each must be a contiguous float64 CUDA tensor on
    the current device, u must hold D n values, T n and out at least 6 (ValueError
    otherwise, before any device work)."""
    import torch
    xs = (("rho", rho), ("u", u), ("T", T), ("out", out))
    for name, x in xs:
        if not isinstance(x, torch.Tensor) or not x.is_cuda or x.dtype != torch.float64 or not x.is_contiguous():
            raise ValueError(f"{name} must be a contiguous float64 CUDA tensor")
    dev = torch.cuda.current_device()
    for name, x in xs:
        if x.device.index != dev:
            raise ValueError(f"{name} lives on cuda:{x.device.index}, not on the current device cuda:{dev}")
    n = rho.numel()
    if u.numel() != int(D) * n or T.numel() != n or out.numel() < 6:
        raise ValueError(f"sizes: u needs D*n = {int(D) * n} values (has {u.numel()}), T n = {n} "
                         f"(has {T.numel()}), out at least 6 (has {out.numel()})")
    s = C.c_void_p(stream) if isinstance(stream, int) else C.c_void_p(getattr(stream, "cuda_stream", 0) or 0)
    return _check(lib().lbm_field_totals_static(int(D), float(N_f), n, _ptr(rho)[0], _ptr(u)[0], _ptr(T)[0],
                                                _ptr(out)[0], s))


def lbm_get_populations(h, g, hh):
    mem = _mem_of(g, hh)
    return _check(lib().lbm_get_populations(h, _ptr(g)[0], _ptr(hh)[0], mem), h)


def lbm_set_populations(h, g, hh):
    mem = _mem_of(g, hh)
    return _check(lib().lbm_set_populations(h, _ptr(g)[0], _ptr(hh)[0], mem), h)


class Simulation:
    """One handle with torch-allocated field tensors (device memory and stream only)."""

    def __init__(self, stream=None, kernel=LBM_KERNEL_AUTO, **kw):
        import torch
        self.torch = torch
        self.p = make_params(**kw)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.h, self.warn = lbm_create(self.p, self.stream)
        if kernel != LBM_KERNEL_AUTO:
            lbm_set_kernel(self.h, kernel)
        self.D, self.r, self.c, self.w = lbm_lattice_info(self.h)
        self.coeffs = lbm_coefficients(self.h)

    @property
    def shape(self):
        p = self.p
        return (p.nz, p.ny, p.nx) if self.D == 3 else (p.ny, p.nx)

    def init(self, rho, u, T):
        t = self.torch
        dev = t.device("cuda")
        f = lambda a: t.as_tensor(np.ascontiguousarray(a, np.float64), device=dev) \
            if not hasattr(a, "data_ptr") else a.to(dev, t.float64).contiguous()
        self._init_keep = (f(rho), f(u), f(T))
        lbm_init_fields(self.h, *self._init_keep)

    def step(self, n=1):
        lbm_step(self.h, n)

    def moments(self, device=False):
        t = self.torch
        s, D = self.shape, self.D
        out = dict(rho=t.empty(s, dtype=t.float64, device="cuda"), u=t.empty((D,) + s, dtype=t.float64, device="cuda"),
                   T=t.empty(s, dtype=t.float64, device="cuda"),
                   Pi=t.empty((D * (D + 1) // 2,) + s, dtype=t.float64, device="cuda"),
                   q=t.empty((D,) + s, dtype=t.float64, device="cuda"))
        lbm_moments(self.h, out["rho"], out["u"], out["T"], out["Pi"], out["q"])
        return out if device else {k: v.cpu().numpy() for k, v in out.items()}

    def diagnostics(self, check=True):
        return lbm_diagnostics(self.h, check)

    def populations(self):
        Q = len(self.c)
        g = np.zeros((Q,) + self.shape)
        hh = np.zeros((Q,) + self.shape)
        lbm_get_populations(self.h, g, hh)
        return g, hh

    def set_populations(self, g, hh):
        lbm_set_populations(self.h, np.ascontiguousarray(g, np.float64), np.ascontiguousarray(hh, np.float64))

    def close(self):
        if getattr(self, "h", None):
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------------------
# Batched instances (lbm_batch_* in include/lbm.h)


def lbm_batch_create(params_list):
    arr = (lbm_params * len(params_list))(*params_list)
    b = C.c_void_p()
    _check(lib().lbm_batch_create(len(params_list), arr, C.byref(b)))
    return b


def lbm_batch_destroy(b):
    return _check(lib().lbm_batch_destroy(b))


def lbm_batch_init_fields(b, i, rho, u, T):
    mem = _mem_of(rho, u, T)
    return _check(lib().lbm_batch_init_fields(b, int(i), _ptr(rho)[0], _ptr(u)[0], _ptr(T)[0], mem))


def lbm_batch_run(b, max_steps, tol, check_every=100) -> int:
    done = C.c_int()
    _check(lib().lbm_batch_run(b, int(max_steps), float(tol), int(check_every), C.byref(done)))
    return done.value


def lbm_batch_status(b, n):
    steps = np.zeros(n, np.int32)
    res = np.zeros(n)
    act = np.zeros(n, np.int32)
    _check(lib().lbm_batch_status(b, steps.ctypes.data_as(C.POINTER(C.c_int)), res.ctypes.data_as(C.POINTER(C.c_double)),
                                  act.ctypes.data_as(C.POINTER(C.c_int))))
    return steps, res, act


def lbm_batch_activate(b, i=-1):
    return _check(lib().lbm_batch_activate(b, int(i)))


def lbm_batch_moments(b, i, rho=None, u=None, T=None, Pi=None, q=None):
    xs = [x for x in (rho, u, T, Pi, q) if x is not None]
    mem = _mem_of(*xs) if xs else LBM_MEM_DEVICE
    return _check(lib().lbm_batch_moments(b, int(i), *(_ptr(x)[0] for x in (rho, u, T, Pi, q)), mem))


def lbm_batch_autotune(b, steps=20) -> int:
    chosen = C.c_int()
    _check(lib().lbm_batch_autotune(b, int(steps), C.byref(chosen)))
    return chosen.value


class Batch:
    """Many independent 2-D D2Q37 FP32 instances stepped together."""

    def __init__(self, param_dicts):
        self.params = [make_params(**d) for d in param_dicts]
        self.n = len(self.params)
        self.b = lbm_batch_create(self.params)

    def init(self, i, rho, u, T):
        lbm_batch_init_fields(self.b, i, np.ascontiguousarray(rho, np.float64), np.ascontiguousarray(u, np.float64),
                              np.ascontiguousarray(T, np.float64))

    def init_neq(self, i, rho, u, T, Pi=None, q=None):
        f = lambda a: None if a is None else np.ascontiguousarray(a, np.float64)
        xs = [f(a) for a in (rho, u, T, Pi, q)]
        _check(lib().lbm_batch_init_fields_neq(self.b, int(i), *(_ptr(x)[0] for x in xs), LBM_MEM_HOST))

    def run(self, max_steps, tol=0.0, check_every=100):
        return lbm_batch_run(self.b, max_steps, tol, check_every)

    def status(self):
        return lbm_batch_status(self.b, self.n)

    def moments(self, i):
        p = self.params[i]
        s = (p.ny, p.nx)
        out = dict(rho=np.zeros(s), u=np.zeros((2,) + s), T=np.zeros(s), Pi=np.zeros((3,) + s), q=np.zeros((2,) + s))
        lbm_batch_moments(self.b, i, out["rho"], out["u"], out["T"], out["Pi"], out["q"])
        return out

    def autotune(self, steps=20):
        return lbm_batch_autotune(self.b, steps)

    def activate(self, i=-1):
        return lbm_batch_activate(self.b, i)

    def close(self):
        if getattr(self, "b", None):
            lbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------------------
# Surrogate network (lbm_mlp_* in include/lbm.h)


class MLP:
    """GELU multilayer perceptron on the tensor cores (bfloat16 products, FP32 master
    weights); parameters exchanged as [[W (k x n), b (n)], ...] float arrays."""

    def __init__(self, sizes, max_batch, stream=None, gemm=None):
        import torch
        self.torch = torch
        self.sizes = list(sizes)
        arr = (C.c_int * len(sizes))(*sizes)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.h = C.c_void_p()
        _check(lib().lbm_mlp_create(len(sizes) - 1, arr, int(max_batch), C.c_void_p(self.stream.cuda_stream),
                                    C.byref(self.h)))
        self.n = lib().lbm_mlp_num_params(self.h)
        if gemm is not None:
            _check(lib().lbm_mlp_set_gemm(self.h, int(gemm)))

    def _pack(self, params):
        return np.concatenate([np.concatenate([np.ravel(W), np.ravel(b)]) for W, b in params]).astype(np.float32)

    def _unpack(self, flat):
        out, o = [], 0
        for k, n in zip(self.sizes[:-1], self.sizes[1:]):
            W = flat[o:o + k * n].reshape(k, n)
            o += k * n
            b = flat[o:o + n]
            o += n
            out.append([W.astype(np.float64), b.astype(np.float64)])
        return out

    def set_params(self, params):
        flat = np.ascontiguousarray(self._pack(params))
        assert flat.size == self.n
        _check(lib().lbm_mlp_set_params(self.h, C.c_void_p(flat.ctypes.data)))

    def get_params(self, with_grads=False):
        p = np.zeros(self.n, np.float32)
        g = np.zeros(self.n, np.float32) if with_grads else None
        _check(lib().lbm_mlp_get_params(self.h, C.c_void_p(p.ctypes.data),
                                        C.c_void_p(g.ctypes.data) if g is not None else None))
        return (self._unpack(p), self._unpack(g)) if with_grads else self._unpack(p)

    def forward(self, x):
        """x: torch CUDA float32 [batch, sizes[0]] -> y [batch, sizes[-1]] (torch)."""
        t = self.torch
        x = x.to(device="cuda", dtype=t.float32).contiguous()
        y = t.empty((x.shape[0], self.sizes[-1]), dtype=t.float32, device="cuda")
        _check(lib().lbm_mlp_forward(self.h, int(x.shape[0]), C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr())))
        return y

    def backward(self, target, want_loss=True):
        t = self.torch
        target = target.to(device="cuda", dtype=t.float32).contiguous()
        loss = C.c_double()
        _check(lib().lbm_mlp_backward(self.h, C.c_void_p(target.data_ptr()), C.byref(loss) if want_loss else None))
        self._keep = target
        return loss.value if want_loss else None

    def adam(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        _check(lib().lbm_mlp_adam(self.h, lr, b1, b2, eps))

    def close(self):
        if getattr(self, "h", None):
            lib().lbm_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
