"""Mutation test of the oracle's pins: each case plants one plausible mistake in a copy of the oracle's C
source (a dropped term, a wrong sign, a wrong index or momentum, a transposed or wrongly conjugated operand, a
mistyped integrator coefficient), compiles the copy, and runs the pin tests of tests/test_oracle_pins.py against it in
a subprocess.  At least one pin must fail for every mutant, and all of them must pass for an unmodified copy
built the same way (the control).  The mistakes are planted on the CPU only; the oracle itself is untouched.

The truncated-projection, multi-orbital brute-force and point-group pins (about 45 s together) are left out of
these runs; every mutant below is caught by a faster pin."""
import concurrent.futures
import contextlib
import os
import shutil
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")

# name -> (text in the oracle, replacement): one plausible mistake each
MUTANTS = {
    # Eq. loop_orbital: the projector of the first pair transposed, U*_{t1} U_{t3} for U_{t1} U*_{t3}
    "projector_transposed": ("cplx left = U1[t1 * ns + l1] * conj(U1[t3 * ns + l1]);",
                             "cplx left = U1[t3 * ns + l1] * conj(U1[t1 * ns + l1]);"),
    # Eq. loopplus in the orbital basis: the conjugation on the wrong eigenvector of the second pair
    "crossed_pair_conjugation": ("conj(U2[t2 * ns + l2]) * U2[t4 * ns + l2]",
                                 "U2[t2 * ns + l2] * conj(U2[t4 * ns + l2])"),
    # Eq. loopminus: the partner momentum s + q instead of s - q
    "pp_momentum_sign": ("k1 = imod(sx - qx, Lf) * Lf + imod(sy - qy, Lf);",
                         "k1 = imod(sx + qx, Lf) * Lf + imod(sy + qy, Lf);"),
    # form factors: e^{+iq.(R1-R2)} in the loop k-sum
    "loop_phase_sign": ("= conj(lattice_phase((long)qx * dl[2 * d] + (long)qy * dl[2 * d + 1], Lf));",
                        "= lattice_phase((long)qx * dl[2 * d] + (long)qy * dl[2 * d + 1], Lf);"),
    # Eq. disc_2a: the degenerate branch of d/dT F^- with the wrong sign
    "pp_degenerate_sign": ("return -0.5 * (gp1 + gp2);", "return 0.5 * (gp1 + gp2);"),
    # Eq. disc_2b: the divided difference of d/dT F^+ reversed
    "ph_difference_order": ("if (fabs(d) > OR_DEGEN * T) return (g1 - g2) / d;",
                            "if (fabs(d) > OR_DEGEN * T) return (g2 - g1) / d;"),
    # d g / d e: a dropped term of the derivative of the Fermi weight
    "fermi_derivative_term": ("*gp = h / (T * T) * (1.0 - ax * (1.0 - z) / (1.0 + z));", "*gp = h / (T * T);"),
    # Sec. 3.3: the Fourier transform of the exchange propagators with the wrong sign
    "fourier_sign": ("cplx ph = lattice_phase((long)(u / Lq) * Rx + (long)(u % Lq) * Ry, Lq);",
                     "cplx ph = lattice_phase(-((long)(u / Lq) * Rx + (long)(u % Lq) * Ry), Lq);"),
    # the D -> P gather (second term of Eq. proj_PD's family) dropped
    "dropped_D_to_P": ("val -= ph2 * Cr[(size_t)k * M2 + sr * M + sc];", "(void)ph2;"),
    # the P -> C gather with the legs 3 and 4 of the source exchanged
    "P_to_C_legs": ("size_t sr = (size_t)i1 * ns2 + s1 * ns + s2, sc = (size_t)i2 * ns2 + s4 * ns + s3;",
                    "size_t sr = (size_t)i1 * ns2 + s1 * ns + s2, sc = (size_t)i2 * ns2 + s3 * ns + s4;"),
    # Eq. proj_DC: the D -> C gather added instead of subtracted (D = -C with legs 3, 4 exchanged)
    "D_to_C_sign": ("val -= ph * Cr[(size_t)cm * M2 + sr * M + sc];", "val += ph * Cr[(size_t)cm * M2 + sr * M + sc];"),
    # the P -> C gather with the phase e^{-iu.R''} for e^{iu.R''}
    "P_to_C_phase": ("cplx ph = lattice_phase((long)qx * c->cls[2 * k] + (long)qy * c->cls[2 * k + 1], Lq);",
                     "cplx ph = conj(lattice_phase((long)qx * c->cls[2 * k] + (long)qy * c->cls[2 * k + 1], Lq));"),
    # the bare vertex projected with legs 3 and 4 exchanged (its sign flipped, V0 being antisymmetric)
    "bare_vertex_legs": ("V0[((s1 * ns + s2) * ns + s3) * ns + s4]", "V0[((s1 * ns + s2) * ns + s4) * ns + s3]"),
    # Eq. RGE_spin / the C equation: c_C = 1 instead of 2
    "crossed_prefactor": ("double cx = (ch == 0) ? 1.0 : 2.0;", "double cx = 1.0;"),
    # the Dormand-Prince row that forms the 5th-order solution (the FSAL stage) mistyped, a_71 = 35/385
    "dp45_solution_row": ("{35.0 / 384, 0.0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84}};",
                          "{35.0 / 385, 0.0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84}};"),
    # the substitution x = ln T without its Jacobian: dX/dx = dX/dT instead of T dX/dT
    "lnT_jacobian_dropped": ("for (size_t i = 0; i < n; i++) out[i] *= T;", "(void)n;"),
    # the Jacobi eigensolver: the phase step applied to the eigenvector column with the wrong sign
    "jacobi_vector_phase": ("for (int k = 0; k < n; k++) V[k * n + q] *= conj(ph);",
                            "for (int k = 0; k < n; k++) V[k * n + q] *= ph;"),
    # the Bloch Hamiltonian with e^{-ik.R} for e^{ik.R} (H(-k) for H(k))
    "bloch_phase_sign": ("cplx ph = lattice_phase((long)kx * m->hopR[2 * h] + (long)ky * m->hopR[2 * h + 1], Lf);",
                         "cplx ph = conj(lattice_phase((long)kx * m->hopR[2 * h] + (long)ky * m->hopR[2 * h + 1], Lf));"),
    # the density n(mu) with the sign of mu flipped (the bisection then hits the filling at -mu)
    "density_mu_sign": ("s += fermi(E[(size_t)k * ns + l] - mu, T);", "s += fermi(E[(size_t)k * ns + l] + mu, T);"),
    # Lambda_c reported at the end of the crossing step instead of interpolated in ln T
    "critical_scale_endpoint": ("res->Tc = exp(x_prev + t * (x - x_prev));", "res->Tc = exp(x); (void)t;"),
    # the Fermi function's two branches exchanged (1 - f for f)
    "fermi_branches": ("return e > 0 ? z / (1.0 + z) : 1.0 / (1.0 + z);", "return e > 0 ? 1.0 / (1.0 + z) : z / (1.0 + z);"),
    # Eq. def_lmp with the momentum shell: the product rule of d/dLambda [chi chi] shortened to one doubled term
    "shell_product_rule": ("(or_dchi(e1, lam) * or_chi(e2, lam) + or_chi(e1, lam) * or_dchi(e2, lam)) * or_Fm(e1, e2, T)",
                           "2.0 * or_dchi(e1, lam) * or_chi(e2, lam) * or_Fm(e1, e2, T)"),
    # d chi / d Lambda with the wrong sign
    "shell_dchi_sign": ("return -2.0 * lam * e * e / (d * d);", "return 2.0 * lam * e * e / (d * d);"),
    # Eq. mat_trafo_P: the orbital indices of the two eigenvectors exchanged
    "band_P_pair_swap": ("Ub[(size_t)k2 * ns2 + b * ns + d] * Ub[(size_t)k * ns2 + a * ns + c]",
                         "Ub[(size_t)k2 * ns2 + a * ns + d] * Ub[(size_t)k * ns2 + b * ns + c]"),
    # Eq. mat_trafo_D: the conjugation of the second eigenvector dropped
    "band_C_conjugation": ("Ub[(size_t)k * ns2 + a * ns + c] * conj(Ub[(size_t)k2 * ns2 + b * ns + d])",
                           "Ub[(size_t)k * ns2 + a * ns + c] * Ub[(size_t)k2 * ns2 + b * ns + d]"),
    # the sampled right-hand side (bounded CPU timings): c_C = 1 instead of 2
    "rhs_at_crossed_prefactor": ("double cx = ch == 0 ? 1.0 : 2.0;", "double cx = 1.0;"),
    # the sampled (and sharded) right-hand side projected at the list position instead of the listed momentum
    "rhs_at_momentum_index": ("proj_one(c, s_list[i], Prows + (size_t)i * M2, Crows + (size_t)i * M2, AP, AC);",
                              "proj_one(c, i, Prows + (size_t)i * M2, Crows + (size_t)i * M2, AP, AC);"),
    # the sampled right-hand side with the first product's operands exchanged (L A for A L)
    "rhs_at_operand_order": ("sacc += A[(size_t)r * M + k] * Lm[(size_t)k * M + col];",
                             "sacc += Lm[(size_t)r * M + k] * A[(size_t)k * M + col];"),
    # the band-basis transformation T^T X T instead of T^dagger X T
    "band_transpose_for_adjoint": ("acc += conj(T[(size_t)j * M + r]) * W[(size_t)j * M + c];",
                                   "acc += T[(size_t)j * M + r] * W[(size_t)j * M + c];"),
}
# (A mistyped weight of the error estimate or a mistyped stage time is caught as well, but only after the step
# controller, whose error estimate then no longer shrinks like h^5, has spent minutes on the first adaptive flow.)


def _run_pins(work, name, src_text):
    """Compile one copy of the oracle and run the pins against it (two OpenMP threads per copy)."""
    os.makedirs(work, exist_ok=True)
    src = os.path.join(work, f"{name}.c")
    with open(src, "w") as f:
        f.write(src_text)
    so = oracle.compile_source(src, os.path.join(work, f"lib{name}.so"))
    env = dict(os.environ, **{oracle.MUTANT_ENV: so, "OMP_NUM_THREADS": "2"})
    args = [sys.executable, "-m", "pytest", PINS, "-x", "-q", "-p", "no:cacheprovider", "-k",
            "not truncated_projections and not multiorbital and not point_group"]
    return subprocess.run(args, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)


@pytest.fixture(scope="module")
def runs():
    """The control and every mutant, run concurrently: name -> CompletedProcess.  The copies are built in a
    git-ignored folder of the repository (oracle/_build/mutants), removed afterwards."""
    with open(oracle._SRC) as f:
        src = f.read()
    texts = {"control": src}
    # the integrator mutant runs longest (the pin that catches it comes late): start it first
    for name, (old, new) in sorted(MUTANTS.items(), key=lambda kv: kv[0] != "dp45_solution_row"):
        assert src.count(old) == 1, name
        texts[name] = src.replace(old, new)
    work = os.path.join(ROOT, "oracle", "_build", "mutants")
    workers = max(1, min(len(texts), (os.cpu_count() or 2) // 2))
    try:
        with concurrent.futures.ThreadPoolExecutor(workers) as ex:
            futs = {n: ex.submit(_run_pins, work, n, t) for n, t in texts.items()}
            yield {n: f.result() for n, f in futs.items()}
    finally:
        shutil.rmtree(work, ignore_errors=True)
        with contextlib.suppress(OSError):
            os.rmdir(os.path.dirname(work))   # oracle/_build, when nothing else is in it


def test_control_copy_passes_the_pins(runs):
    r = runs["control"]
    assert r.returncode == 0, r.stdout[-3000:]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(runs, name):
    r = runs[name]
    assert r.returncode == 1, (name, r.returncode, r.stdout[-3000:])   # 1: a test failed
    failed = [ln for ln in r.stdout.splitlines() if ln.startswith("FAILED")]
    assert failed, r.stdout[-3000:]
    print(f"{name}: caught by {failed[0].split()[1]}")
