"""Planted mistakes: each mutant of the oracle (a copy of its C source with
one plausible bug) must fail at least one pin of test_oracle_pins.py.

The mutants are built on the CPU from a temporary copy; the oracle source in
the repository is never modified.
"""
import os
import shutil
import subprocess
import tempfile

import pytest

import oracle
import tests.test_oracle_dome as dome
import tests.test_oracle_enet as enet
import tests.test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "lasso_oracle.c")

# (name, original text, mutated text) -- each original occurs in the source
MUTANTS = [
    ("primal drops lambda", "double P = 0.5 * rr + lambda * l1;", "double P = 0.5 * rr + l1;"),
    ("dual drops lambda", "double d = lambda * (alpha * rho[i]) - y[i];",
     "double d = (alpha * rho[i]) - y[i];"),
    ("soft-threshold sign", "(b > 0.0 ? ab - thr : -(ab - thr))", "(b > 0.0 ? -(ab - thr) : ab - thr)"),
    ("gradient sign", "double b = beta[j] + g / n2;", "double b = beta[j] - g / n2;"),
    ("residual update sign", "for (int64_t i = 0; i < n; ++i) rho[i] -= d * x[i];",
     "for (int64_t i = 0; i < n; ++i) rho[i] += d * x[i];"),
    ("threshold uses norm not squared norm", "double thr = lambda / n2;", "double thr = lambda / sqrt(n2);"),
    ("check correlates y instead of rho", "double cj = in_scope ? dot_col(X, ldx, n, j, rho) : 0.0;",
     "double cj = in_scope ? dot_col(X, ldx, n, j, y) : 0.0;"),
    ("sphere test reversed", "int screen = mu < 1.0;", "int screen = mu > 1.0;"),
    ("radius divided twice by lambda", "double r = sqrt(2.0 * Gs) / lambda;",
     "double r = sqrt(2.0 * Gs) / (lambda * lambda);"),
    ("radius without gap", "double Gs = (G > 0.0 ? G : 0.0) + tau;", "double Gs = tau;"),
    ("dual scaling ignores lambda", "alpha = 1.0 / (lambda > m ? lambda : m);", "alpha = 1.0 / m;"),
    ("grid off by one", "pow(10.0, -delta * (double)t / (double)(T - 1))",
     "pow(10.0, -delta * (double)(t + 1) / (double)(T - 1))"),
    ("column stride transposed", "const double* x = X + j * ldx;\n  double s = 0.0;",
     "const double* x = X + j;\n  double s = 0.0;"),
    ("screened coefficient not removed from residual", "for (int64_t i = 0; i < ns; ++i) rs[i] += b * Xs[i + j * lds];",
     "(void)b;"),
    ("Eq. (8) clipped to the wrong side", "if (a < -lim) a = -lim;", "if (a < -lim) a = lim;"),
    ("lambda_max from the smallest correlation", "if (fabs(c0[j]) > lmax) { lmax = fabs(c0[j]); arg = j; }",
     "if (j == 0 || fabs(c0[j]) < lmax) { lmax = fabs(c0[j]); arg = j; }"),
    ("gap rounding bound dropped", "double tau = 2.0 * (double)(n + p + 8) * u", "double tau = 0.0 * (double)(n + p + 8) * u"),
    # the dome test (Eq. (11), appendix)
    ("dome normal with the main text's sign", "double nx = (xy - xt) / dR;", "double nx = (xt - xy) / dR;"),
    ("dome ratio with the opposite sign", "dal = 2.0 * q - 1.0;", "dal = 1.0 - 2.0 * q;"),
    ("dome radius R instead of R/2", "drad = 0.5 * sqrt(big) / lambda;", "drad = sqrt(big) / lambda;"),
    ("dome support case condition", "if (nx < -alpha * xnorm) return", "if (nx < alpha * xnorm) return"),
    ("dome center without theta", "double cx = 0.5 * (xy + xt);", "double cx = 0.5 * xy;"),
    ("dome ratio from the gap instead of r(beta)", "double small = yy - 2.0 * P - tau;",
     "double small = 2.0 * G;"),
    ("dome rim term without (1 - alpha^2)", "sqrt(w * (1.0 - alpha * alpha))", "sqrt(w)"),
    # the refined radius of Thm. 2
    ("refined radius always R", "if (Rt < r) r = Rt;", "r = Rt;"),
    ("refined radius from the gap term", "double Rt = sqrt(d2 + tau) / lambda;",
     "double Rt = sqrt(2.0 * Gs) / (lambda * lambda);"),
    # the Elastic-Net on the augmented design
    ("Elastic-Net without the ridge rows", "col[n + i] = (i == j) ? sm : 0.0;", "col[n + i] = 0.0;"),
    ("Elastic-Net lambda_max not divided by a", "double lmax = scal[0] / o->enet_alpha", "double lmax = scal[0]"),
    ("Elastic-Net L1 penalty lambda instead of a lambda", "lam1 = o->enet_alpha * lambda;", "lam1 = lambda;"),
    ("Elastic-Net ridge weight a lambda", "double mu = (1.0 - o->enet_alpha) * lambda;",
     "double mu = o->enet_alpha * lambda;"),
    ("Elastic-Net residual tail left at zero", "rhoa[n + j] = -(sm * beta[j]);", "rhoa[n + j] = 0.0;"),
]

PIN_CALLS = [
    (pins.test_grid_is_geometric, {}),
    (pins.test_hand_example_identity_design, {}),
    (pins.test_lambda_max_and_zero_solution, {}),
    (pins.test_first_feature_enters_linearly, {}),
    (pins.test_orthonormal_soft_threshold, {"seed": 3}),
    (pins.test_bad_warm_start_reaches_optimum, {}),
    (pins.test_screening_a_nonzero_coefficient, {}),
    (pins.test_bruteforce_agreement, {"seed": 5, "n": 20, "p": 8}),
    (pins.test_kkt_at_tight_solution, {}),
    (pins.test_every_sphere_contains_dual_optimum, {}),
    (pins.test_screened_features_are_zero, {}),
    (pins.test_finite_identification, {}),
    (pins.test_prop3_sequential_identity, {}),
    (pins.test_dual_point_eq8_is_projection_on_span, {}),
    (pins.test_refined_radius_of_thm2, {}),
    (pins.test_gap_rounding_bound_holds, {}),
    (dome.test_dome_support_matches_sampled_maximum, {"alpha": 0.35}),
    (dome.test_dome_value_is_the_maximum_over_the_safe_set, {"dual_point": 0}),
    (dome.test_dome_lies_inside_the_sphere, {}),
    (dome.test_every_dome_contains_dual_optimum, {}),
    (dome.test_dome_path_reaches_the_exact_solution, {"seed": 44, "n": 20, "p": 8}),
    (enet.test_enet_orthonormal_closed_form, {"a": 0.3}),
    (enet.test_enet_first_feature_enters, {}),
    (enet.test_enet_bruteforce_agreement, {"seed": 32, "n": 20, "p": 8, "a": 0.5}),
    (enet.test_enet_kkt_at_tight_solution, {}),
    (enet.test_enet_hand_examples, {}),
]


@pytest.fixture(scope="module")
def workdir():
    d = tempfile.mkdtemp(prefix="oracle_mut_")
    yield d
    shutil.rmtree(d, ignore_errors=True)


@pytest.mark.parametrize("name,orig,mut", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(workdir, monkeypatch, name, orig, mut):
    src = open(SRC).read()
    assert src.count(orig) >= 1, f"mutation anchor not found: {orig!r}"
    msrc = src.replace(orig, mut, 1)
    idx = MUTANTS.index((name, orig, mut))
    cpath = os.path.join(workdir, f"mut{idx}.c")
    so = os.path.join(workdir, f"libmut{idx}.so")
    open(cpath, "w").write(msrc)
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-std=c99", "-fPIC", "-shared",
                           "-o", so, cpath, "-lm"])
    monkeypatch.setattr(oracle, "_lib", oracle._bind(so))
    caught = None
    # the pins of the mutated part run first (only the order changes: every
    # pin still runs until one fails)
    topic = "dome" if "dome" in name else "enet" if "Elastic" in name else "refined" if "refined" in name else ""
    calls = sorted(PIN_CALLS, key=lambda c: 0 if topic and topic in c[0].__name__ else 1)
    for fn, kw in calls:
        try:
            fn(oracle, **kw)
        except Exception as e:  # noqa: BLE001 -- any failure of a pin counts
            caught = f"{fn.__name__}: {type(e).__name__}"
            break
    assert caught, f"mutant '{name}' passed every pin"
