"""ctypes wrapper of the FP64 CPU oracle (``lbm_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  Nothing in the CUDA library
imports this module, and this module imports nothing from the library.

The oracle is the paper's scheme written out step by step in double precision
(Hu et al., arXiv 1611.02409, Secs. II-VI); the C file's header lists each step's
equation and every reading of the paper it takes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lbm_oracle.c")
LIB = os.path.join(HERE, "liblbm_oracle.so")
# A prebuilt oracle library to load instead (tests that plant a mistake in a copy of the
# oracle point this at the mutant's build); the default is built from SRC.
LIB_OVERRIDE = os.environ.get("LBM_ORACLE_LIB")

D2Q37 = 1
D3Q103 = 2
D2Q33 = 3
D2Q77 = 4
PR_SHIFTED = 0
PR_LITERAL = 1

_lock = threading.Lock()
_lib = None


def build_at(src: str, out: str) -> str:
    """Compile an oracle source file into a shared library (strict IEEE double: no FMA
    contraction)."""
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-shared", "-fPIC", "-o", out, src, "-lm"]
    subprocess.run(cmd, check=True)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (strict IEEE double: no FMA contraction)."""
    if LIB_OVERRIDE:
        return LIB_OVERRIDE
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        build_at(SRC, tmp)
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            ip = C.POINTER(C.c_int)
            L.orc_create.restype = C.c_void_p
            L.orc_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double,
                                     C.c_double, C.c_double, C.c_double, C.c_double, C.c_int, dp, dp]
            L.orc_destroy.argtypes = [C.c_void_p]
            L.orc_set_open_x.argtypes = [C.c_void_p, C.c_int]
            L.orc_init.argtypes = [C.c_void_p, dp, dp, dp]
            L.orc_step.argtypes = [C.c_void_p, C.c_int]
            L.orc_moments.argtypes = [C.c_void_p, dp, dp, dp, dp, dp]
            L.orc_diagnostics.argtypes = [C.c_void_p, dp]
            L.orc_get_pops.argtypes = [C.c_void_p, dp, dp]
            L.orc_set_pops.argtypes = [C.c_void_p, dp, dp]
            L.orc_steps.argtypes = [C.c_void_p]
            L.orc_steps.restype = C.c_long
            L.orc_lattice_info.argtypes = [C.c_int, ip, ip, dp, ip, dp]
            L.orc_hermite_poly.argtypes = [C.c_int, C.c_int, dp, dp]
            L.orc_hermite_coeff.argtypes = [C.c_int, C.c_int, dp, dp, dp]
            L.orc_equilibrium.argtypes = [C.c_int, C.c_int, C.c_double, dp, dp, dp]
            L.orc_params.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
                                     C.c_double, C.c_int, dp]
            L.orc_collide_cell.argtypes = [C.c_void_p, dp, dp, dp, dp]
            L.orc_cell_state.argtypes = [C.c_void_p, dp, dp, dp]
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def lattice(which: int = D2Q37):
    """(D, r, c[Q,3] int, w[Q]) re-solved in FP64 by the oracle."""
    D, Q, r = C.c_int(), C.c_int(), C.c_double()
    c = np.zeros((128, 3), np.int32)
    w = np.zeros(128)
    n = lib().orc_lattice_info(which, C.byref(D), C.byref(Q), C.byref(r),
                               c.ctypes.data_as(C.POINTER(C.c_int)), _dp(w))
    if n < 0:
        raise ValueError("unknown lattice")
    return D.value, r.value, c[:n].copy(), w[:n].copy()


def hermite_poly(n: int, xi) -> np.ndarray:
    """H^(n)(xi) as a D^n tensor (Grad's formula, Sec. IV)."""
    xi = _f64(xi)
    D = xi.size
    out = np.zeros(D ** n)
    if lib().orc_hermite_poly(n, D, _dp(xi), _dp(out)):
        raise ValueError("bad order")
    return out.reshape((D,) * n) if n else out.reshape(())


def hermite_coeff(n: int, u, Lam) -> np.ndarray:
    """a^(n) of the Gaussian N(u, Lambda) by Eq. fESCoe, as a D^n tensor."""
    u = _f64(u)
    Lam = _f64(Lam)
    D = u.size
    if Lam.size != D * D:
        raise ValueError(f"Lambda must be {D}x{D}")
    out = np.zeros(D ** n)
    if lib().orc_hermite_coeff(n, D, _dp(u), _dp(Lam.reshape(-1)), _dp(out)):
        raise ValueError("bad order")
    return out.reshape((D,) * n) if n else out.reshape(())


def equilibrium(which: int, rho: float, u, Lam, order: int = 4) -> np.ndarray:
    """Discrete truncated Gaussian G_i (Eq. GExpansion) on a lattice."""
    D, _, c, _ = lattice(which)
    u = _f64(u)
    Lam = _f64(Lam).reshape(-1)
    if u.shape != (D,) or Lam.shape != (D * D,):
        raise ValueError(f"u needs {D} components and Lambda {D}x{D}")
    G = np.zeros(len(c))
    if lib().orc_equilibrium(which, order, rho, _dp(u), _dp(Lam), _dp(G)):
        raise ValueError("bad args")
    return G


def params(D, Pr, gamma=1.4, Nf=0.0, kappa=0.2, tau=0.6, mode=PR_SHIFTED) -> dict:
    out = np.zeros(5)
    if lib().orc_params(D, Pr, gamma, Nf, kappa, tau, mode, _dp(out)):
        raise ValueError("inadmissible parameters")
    return dict(Nf=out[0], omega=out[1], nuG=out[2], tau_s=out[3], tau_q=out[4])


class Sim:
    """One oracle simulation (periodic box, or 2-D channel with walls in y)."""

    def __init__(self, lattice_id=D2Q37, nx=16, ny=16, nz=1, walls=False, Pr=0.71, gamma=1.4,
                 Nf=0.0, kappa=0.2, tau=0.6, mode=PR_SHIFTED, wall_u=None, wall_T=None, open_x=False):
        self.L = lib()
        self.D, self.r, self.c, self.w = lattice(lattice_id)
        self.nx, self.ny, self.nz = nx, ny, (nz if self.D == 3 else 1)
        self.walls = walls
        wu = _f64(wall_u if wall_u is not None else np.zeros((2, 3))).reshape(6)
        wT = _f64(wall_T if wall_T is not None else np.ones(2)).reshape(2)
        self.h = self.L.orc_create(lattice_id, nx, ny, self.nz, int(walls), Pr, gamma, Nf, kappa, tau,
                                   mode, _dp(wu), _dp(wT))
        if not self.h:
            raise ValueError("oracle rejected the parameters")
        if open_x:
            self.L.orc_set_open_x(self.h, 1)
        self.coeffs = params(self.D, Pr, gamma, Nf, kappa, tau, mode)

    @property
    def ncell(self):
        return self.nx * self.ny * self.nz

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx) if self.D == 3 else (self.ny, self.nx)

    def init(self, rho, u, T):
        rho, u, T = _f64(rho), _f64(u), _f64(T)
        assert rho.size == self.ncell and u.size == self.D * self.ncell and T.size == self.ncell
        self.L.orc_init(self.h, _dp(rho), _dp(u), _dp(T))

    def step(self, n=1):
        self.L.orc_step(self.h, int(n))

    def moments(self):
        n, D = self.ncell, self.D
        rho, u, T = np.zeros(n), np.zeros(D * n), np.zeros(n)
        Pi, q = np.zeros(D * (D + 1) // 2 * n), np.zeros(D * n)
        self.L.orc_moments(self.h, _dp(rho), _dp(u), _dp(T), _dp(Pi), _dp(q))
        s = self.shape
        return dict(rho=rho.reshape(s), u=u.reshape((D,) + s), T=T.reshape(s),
                    Pi=Pi.reshape((D * (D + 1) // 2,) + s), q=q.reshape((D,) + s))

    def diagnostics(self):
        out = np.zeros(5)
        self.L.orc_diagnostics(self.h, _dp(out))
        return dict(mass=out[0], momentum=out[1:4].copy(), energy=out[4])

    def populations(self):
        Q = len(self.c)
        g, h = np.zeros(Q * self.ncell), np.zeros(Q * self.ncell)
        self.L.orc_get_pops(self.h, _dp(g), _dp(h))
        return g.reshape((Q,) + self.shape), h.reshape((Q,) + self.shape)

    def set_populations(self, g, h):
        g, h = _f64(g), _f64(h)
        self.L.orc_set_pops(self.h, _dp(g), _dp(h))

    def collide_cell(self, g, h):
        g, h = _f64(g), _f64(h)
        go, ho = np.zeros_like(g), np.zeros_like(h)
        self.L.orc_collide_cell(self.h, _dp(g), _dp(h), _dp(go), _dp(ho))
        return go, ho

    def cell_state(self, g, h):
        g, h = _f64(g), _f64(h)
        out = np.zeros(17)
        self.L.orc_cell_state(self.h, _dp(g), _dp(h), _dp(out))
        return dict(rho=out[0], u=out[1:1 + self.D].copy(), Ttr=out[4], Tint=out[5], Teq=out[6],
                    Trel=out[7], Lam=out[8:17].reshape(3, 3)[:self.D, :self.D].copy())

    def close(self):
        if self.h:
            self.L.orc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
