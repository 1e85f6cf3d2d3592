"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source (a wrong
stencil coefficient, a flipped sign, a dropped term, a transposed axis, a
missing factor), builds it into a temporary library, and runs the pin tests
against it in a subprocess; the pins must fail.  Nothing here touches a GPU.
"""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "mlmd_oracle.c")

MUTANTS = [
    ("laplacian centre coefficient", "lap[0] = -2.5;", "lap[0] = -2.4;"),
    ("gradient outer coefficient sign", "grad[2] = -1.0 / 12.0;", "grad[2] = 1.0 / 12.0;"),
    ("sign of the A.grad term", "- I * ih * ag", "+ I * ih * ag"),
    ("dropped |A|^2/2 term", "(d->V[g] + a2) * c", "(d->V[g]) * c"),
    ("missing dV in the projection", "proj[((int64_t)a * np + i) * no + o] *= dV;", ";"),
    ("missing D in the scatter", "d->D[(int64_t)a * np + i] * proj", "proj"),
    ("Taylor coefficient without 1/j!", "c *= (-I * dt) / (double)j;", "c *= (-I * dt);"),
    ("p projector on the wrong axis", "beta[q * n_proj + 4 * set + 1 + ax] = dl[ax]",
     "beta[q * n_proj + 4 * set + 1 + ax] = dl[(ax + 1) % 3]"),
    ("minimum image without the half shift", "double k = floor(t / L[ax] + 0.5);", "double k = floor(t / L[ax]);"),
    ("current without the A rho term", "jcur[ax * ng + g] = s + A[ax] * rho[g];", "jcur[ax * ng + g] = s;"),
    ("adjoint Taylor with the forward sign", "c *= (I * dt) / (double)j;", "c *= (-I * dt) / (double)j;"),
    ("2nd-order laplacian centre coefficient", "lap[0] = -2.0; lap[1] = 1.0;", "lap[0] = -2.1; lap[1] = 1.0;"),
    ("4th-order laplacian inner coefficient", "lap[1] = 4.0 / 3.0", "lap[1] = 4.0 / 3.1"),
    ("4th-order gradient inner coefficient", "grad[1] = 2.0 / 3.0", "grad[1] = 2.0 / 3.1"),
    ("projector normalised without dV", "s *= dV;", ";"),
    ("split step without the renormalisation", "sqrt(nrm_before[o] / nrm_after[o])", "1.0"),
    ("overlap without dV", "S[(int64_t)n * nb + m] = dV * s;", "S[(int64_t)n * nb + m] = s;"),
    ("sphere membership without the boundary", "if (d2 <= rc2) {", "if (d2 < rc2) {"),
    ("projector Gaussian without the factor 2 in its width", "double s = exp(-d2 / (2.0 * rc * rc));",
     "double s = exp(-d2 / (rc * rc));"),
    ("second projector shell at r_c sqrt(2)", "double rc = set == 0 ? r_c : r_c / sqrt(2.0);",
     "double rc = set == 0 ? r_c : r_c * sqrt(2.0);"),
    ("p projector with the displacement reversed", "beta[q * n_proj + 4 * set + 1 + ax] = dl[ax] / rc * s;",
     "beta[q * n_proj + 4 * set + 1 + ax] = -dl[ax] / rc * s;"),
    ("density without the occupations", "s += f[o] * creal(conj(c) * c);", "s += creal(conj(c) * c);"),
    ("current field with the conjugate on the gradient", "cimag(conj(in[g * no + o]) * gp[g * no + o])",
     "cimag(in[g * no + o] * conj(gp[g * no + o]))"),
    ("energy without the nonlocal part", "orc_apply_h(d, A, psi_in, work, work_proj);\n    for (int64_t g = 0; g < ng; ++g)\n        for (int o = 0; o < no; ++o) {\n            cplx c = in[g * no + o];\n            nrm",
     "orc_apply_hloc(d, A, psi_in, work);\n    for (int64_t g = 0; g < ng; ++g)\n        for (int o = 0; o < no; ++o) {\n            cplx c = in[g * no + o];\n            nrm"),
    ("velocity-gauge phase with the opposite sign", "return cos(th) - I * sin(th);", "return cos(th) + I * sin(th);"),
    ("velocity-gauge phase missing from the scatter",
     "out[(int64_t)d->idx[q] * no + o] += gauge_factor(d, A, a, d->idx[q]) * acc;",
     "out[(int64_t)d->idx[q] * no + o] += acc;"),
    ("velocity-gauge displacement without the minimum image", "dl[ax] = t - L * floor(t / L + 0.5);", "dl[ax] = t;"),
    ("moment projection without the displacement", "wq *= dl[axis];", "wq *= 1.0;"),
    ("moment projection on the wrong axis", "wq *= dl[axis];", "wq *= dl[(axis + 1) % 3];"),
    ("nonlocal current with the opposite sign", "2.0 * creal(I * conj(P[r * no + o])", "2.0 * creal(-I * conj(P[r * no + o])"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(name, old, new, tmp_path):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site not unique: {name}"
    mutated = tmp_path / "mutant.c"
    mutated.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11",
                           "-o", str(so), str(mutated), "-lm"])
    env = dict(os.environ, MLMD_ORACLE_LIB=str(so), OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode != 0, f"pins did not catch: {name}\n{r.stdout[-2000:]}"


KS_MUTANTS = [
    ("overlap transposed", "psi_0 @ C", "psi_0 @ C.T"),
    ("overlap conjugated", "psi_0 @ C", "psi_0 @ C.conj()"),
    ("sign of delta", "psi_t - complex(delta)", "psi_t + complex(delta)"),
    ("missing dV", "C = overlap(psi_0, psi_t, dV)", "C = overlap(psi_0, psi_t, 1.0)"),
]


@pytest.mark.parametrize("name,old,new", KS_MUTANTS, ids=[m[0] for m in KS_MUTANTS])
def test_ks_pin_catches_planted_mistake(name, old, new, monkeypatch):
    """Eq. 5's oracle function with one planted mistake (rebuilt from the
    oracle's own source text) must fail the closed-form pin."""
    import inspect
    import textwrap
    sys.path.insert(0, ROOT)
    import oracle
    src = textwrap.dedent(inspect.getsource(oracle.ks_correction))
    assert src.count(old) == 1, name
    ns = {"np": __import__("numpy"), "overlap": oracle.overlap, "_c128": oracle._c128}
    exec(src.replace(old, new), ns)
    monkeypatch.setattr(oracle, "ks_correction", ns["ks_correction"])
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import test_oracle_pins
    with pytest.raises(AssertionError):
        test_oracle_pins.test_ks_correction_closed_forms()


OCC_MUTANTS = [
    ("overlap transposed", "(np.abs(C) ** 2) @ f", "(np.abs(C) ** 2).T @ f"),
    ("reference and propagated swapped", "C = overlap(psi_ref, psi_t, dV)", "C = overlap(psi_t, psi_ref, dV)"),
    ("missing dV", "C = overlap(psi_ref, psi_t, dV)", "C = overlap(psi_ref, psi_t, 1.0)"),
    ("sign of n_exc", "np.sum(f) - np.sum(f_s)", "np.sum(f_s) - np.sum(f)"),
    ("amplitudes instead of probabilities", "(np.abs(C) ** 2) @ f", "np.abs(C) @ f"),
]


@pytest.mark.parametrize("name,old,new", OCC_MUTANTS, ids=[m[0] for m in OCC_MUTANTS])
def test_occupations_pin_catches_planted_mistake(name, old, new, monkeypatch):
    """The occupation function with one planted mistake must fail its pin."""
    import inspect
    import textwrap
    sys.path.insert(0, ROOT)
    import oracle
    src = textwrap.dedent(inspect.getsource(oracle.occupations))
    assert src.count(old) == 1, name
    ns = {"np": __import__("numpy"), "overlap": oracle.overlap}
    exec(src.replace(old, new), ns)
    monkeypatch.setattr(oracle, "occupations", ns["occupations"])
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import test_oracle_pins
    with pytest.raises(AssertionError):
        test_oracle_pins.test_occupations_closed_forms()
