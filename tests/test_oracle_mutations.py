"""The oracle's pins are not vacuous: a plausible mistake planted in a copy of the oracle
(a wrong sign, a dropped term, a transposed or reversed index, the wrong temperature in a
relaxation target) must make the pin that guards that part fail.  Each mutant is built
from a textual edit of oracle/lbm_oracle.c in a temporary directory and the pin runs
against it in a child process (LBM_ORACLE_LIB); the unmutated oracle passes the same pins
in the rest of the suite."""
import os
import subprocess
import sys

import pytest

from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (what the mistake is, source text, replacement, the pin that must catch it)
MUTANTS = [
    ("energy populations relax toward T_eq instead of T_rel (reading R1)",
     "ho[i] = h[i] - om * (h[i] - 0.5 * S->k.Nf * st.Trel * G[i]);",
     "ho[i] = h[i] - om * (h[i] - 0.5 * S->k.Nf * st.Teq * G[i]);",
     "tests/test_oracle_equilibrium.py::test_collision_conserves_mass_momentum_energy"),
    ("Grad's Hermite polynomials without the alternating sign (Sec. IV)",
     "double term = (P->npairs & 1) ? -1.0 : 1.0;",
     "double term = 1.0;",
     "tests/test_oracle_hermite.py::test_hermite_poly_vs_numpy"),
    ("Eq. fESCoe without its (-1)^(alpha-beta)",
     "double sign = ((alpha - beta) & 1) ? -1.0 : 1.0;",
     "double sign = 1.0;",
     "tests/test_oracle_hermite.py::test_hermite_coeff_vs_quadrature"),
    ("ES tensor with nu on the isotropic instead of the stress part (Sec. II)",
     "k->nuG * s->sigma[a * D + b])",
     "(1.0 - k->nuG) * s->sigma[a * D + b])",
     "tests/test_oracle_transport.py::test_viscosity_and_conductivity_give_set_Pr"),
    ("shifted mapping with tau_q = tau/Pr (reading R3)",
     "k->tau_q = (tau - 0.5) / Pr + 0.5;",
     "k->tau_q = tau / Pr;",
     "tests/test_oracle_transport.py::test_viscosity_and_conductivity_give_set_Pr"),
    ("pull-stream from x + c_i instead of x - c_i (Sec. V)",
     "int xs = x - S->L.c[i][0];\n                        /* open ends",
     "int xs = x + S->L.c[i][0];\n                        /* open ends",
     "tests/test_oracle_shock_tube.py::test_shock_tube_matches_exact_riemann_solution"),
    ("wall density from the ghost rows instead of the fluid rows (reading R5)",
     "leaving += g[orc_cell(S, xs, yw + n * s + S->gh, zs) * Q + i];",
     "leaving += g[orc_cell(S, xs, yw - n * s + S->gh, zs) * Q + i];",
     "tests/test_oracle_transport.py::test_walls_conserve_fluid_mass"),
    ("D2Q77 expanded to fifth instead of sixth order (reading R19)",
     "orc_build_htab(&S->L, lattice == ORC_D2Q77 ? 6 : 4, &S->T);",
     "orc_build_htab(&S->L, lattice == ORC_D2Q77 ? 5 : 4, &S->T);",
     "tests/test_oracle_transport.py::test_sixth_order_transport_is_galilean_invariant"),
    ("open x ends wrapping instead of clamping at the right end (reading R16)",
     "xs = S->open_x ? (xs < 0 ? 0 : (xs > S->nx - 1 ? S->nx - 1 : xs)) : orc_mod(xs, S->nx);",
     "xs = S->open_x ? (xs < 0 ? 0 : (xs > S->nx - 1 ? 0 : xs)) : orc_mod(xs, S->nx);",
     "tests/test_oracle_shock_tube.py::test_open_ends_keep_an_undisturbed_state"),
    ("a Table D2Q33 shell mistyped, (3,1) for (2,1)",
     "{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {2, 0, 0}, {2, 2, 0}, {3, 0, 0}, {2, 1, 0}, {4, 4, 0}};",
     "{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {2, 0, 0}, {2, 2, 0}, {3, 0, 0}, {3, 1, 0}, {4, 4, 0}};",
     "tests/test_oracle_lattice.py::test_d2q33_matches_printed_table"),
    ("a D2Q77 shell mistyped, (5,2) for (5,3) (reading R19)",
     "{3, 2, 0}, {3, 3, 0}, {4, 0, 0}, {4, 1, 0}, {4, 4, 0}, {5, 0, 0}, {5, 3, 0}};",
     "{3, 2, 0}, {3, 3, 0}, {4, 0, 0}, {4, 1, 0}, {4, 4, 0}, {5, 0, 0}, {5, 2, 0}};",
     "tests/test_oracle_lattice.py::test_d2q77_moments_degree13"),
    ("heat flux without the internal-energy (h) term (reading C-10)",
     "qa[d] += 0.5 * v2 * v[d] * g[i] + v[d] * h[i];",
     "qa[d] += 0.5 * v2 * v[d] * g[i];",
     "tests/test_oracle_moments.py::test_heat_flux_of_a_third_order_hermite_term"),
    ("heat flux without the 1/2 of the kinetic part (reading C-10)",
     "qa[d] += 0.5 * v2 * v[d] * g[i] + v[d] * h[i];",
     "qa[d] += v2 * v[d] * g[i] + v[d] * h[i];",
     "tests/test_oracle_moments.py::test_heat_flux_of_a_third_order_hermite_term"),
    ("heat flux about xi + u instead of the peculiar velocity xi - u",
     "v[d] = S->L.r * S->L.c[i][d] - st.u[d]; v2 += v[d] * v[d]; }\n                        for (int d = 0; d < D; ++d) qa[d]",
     "v[d] = S->L.r * S->L.c[i][d] + st.u[d]; v2 += v[d] * v[d]; }\n                        for (int d = 0; d < D; ++d) qa[d]",
     "tests/test_oracle_moments.py::test_heat_flux_vanishes_for_gaussians_and_pressure_is_rho_lambda"),
    ("initial populations without the wall procedure (reading R6)",
     "    if (S->walls) orc_walls(S, S->g, S->h);\n    S->steps = 0;",
     "    S->steps = 0;",
     "tests/test_oracle_transport.py::test_walls_conserve_fluid_mass_from_any_initial_state"),
    ("total energy without the 1/2 of the kinetic part (Sec. V, rho E)",
     "E += 0.5 * x2 * g + S->h[c * Q + i];",
     "E += x2 * g + S->h[c * Q + i];",
     "tests/test_oracle_moments.py::test_totals_equal_sums_of_the_moment_fields"),
]


@pytest.mark.parametrize("what,old,new,pin", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_its_pin(tmp_path, what, old, new, pin):
    src = open(O.SRC).read()
    assert src.count(old) == 1, "mutation site not unique"
    mut = tmp_path / "lbm_oracle.c"
    mut.write_text(src.replace(old, new))
    so = O.build_at(str(mut), str(tmp_path / "liblbm_oracle.so"))
    env = dict(os.environ, LBM_ORACLE_LIB=so)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", pin],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 1, (what, r.returncode, r.stdout[-2000:])   # 1: tests ran and failed


def test_unmutated_copy_passes_the_same_harness(tmp_path):
    # the harness itself (copy, build, child run) does not make pins fail
    so = O.build_at(O.SRC, str(tmp_path / "liblbm_oracle.so"))
    env = dict(os.environ, LBM_ORACLE_LIB=so)
    pins = sorted({m[3] for m in MUTANTS})
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider"] + pins,
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:]


# mistakes planted in the surrogate network's reference (oracle/mlp_oracle.py)
MLP_MUTANTS = [
    ("GELU derivative without its z phi(z) term",
     "return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)",
     "return 0.5 * (1.0 + erf(z / np.sqrt(2.0)))",
     "test_gelu_derivative_by_finite_differences"),
    ("loss gradient normalised by the batch instead of every output",
     "dz = 2.0 * (y - t) / n",
     "dz = 2.0 * (y - t) / y.shape[0]",
     "test_backprop_matches_finite_differences"),
    ("Adam step divided by v instead of sqrt(v)",
     "p[j] -= lr * mh / (np.sqrt(vh) + eps)",
     "p[j] -= lr * mh / (vh + eps)",
     "test_adam_first_step_closed_form"),
]


@pytest.mark.parametrize("what,old,new,pin", MLP_MUTANTS, ids=[m[0] for m in MLP_MUTANTS])
def test_planted_mlp_mistake_fails_its_pin(tmp_path, what, old, new, pin):
    src_dir = os.path.join(ROOT, "oracle")
    pkg = tmp_path / "oracle"
    pkg.mkdir()
    for f in ("__init__.py", "oracle.py", "mlp_oracle.py", "lbm_oracle.c"):
        text = open(os.path.join(src_dir, f)).read()
        if f == "mlp_oracle.py":
            assert text.count(old) == 1, "mutation site not unique"
            text = text.replace(old, new)
        (pkg / f).write_text(text)
    # the child runs from tmp_path, so `import oracle` resolves to the mutated copy
    env = dict(os.environ, PYTHONPATH=os.pathsep.join([str(tmp_path), ROOT]),
               LBM_ORACLE_LIB=O.build())
    where = subprocess.run([sys.executable, "-c", "import oracle.mlp_oracle as M; print(M.__file__)"],
                           cwd=str(tmp_path), env=env, capture_output=True, text=True, timeout=120)
    assert where.stdout.strip().startswith(str(pkg)), where.stdout      # the copy is the one loaded
    test = os.path.join(ROOT, "tests", "test_oracle_mlp.py") + "::" + pin
    args = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "--rootdir", ROOT, test]
    r = subprocess.run(args, cwd=str(tmp_path), env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1, (what, r.returncode, r.stdout[-2000:])
    # and the same pin passes on an unmutated copy run the same way
    (pkg / "mlp_oracle.py").write_text(open(os.path.join(src_dir, "mlp_oracle.py")).read())
    r0 = subprocess.run(args, cwd=str(tmp_path), env=env, capture_output=True, text=True, timeout=600)
    assert r0.returncode == 0, r0.stdout[-2000:]
