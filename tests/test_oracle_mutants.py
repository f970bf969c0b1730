"""The oracle's pins have teeth: every plausible mistake planted in a copy of
the oracle (a dropped term, a wrong sign or index, a transposed operand, a
wrong constant) makes at least one pin of ``oracle_pins`` fail.

Each mutant is a one-line textual change of ``oracle/syev3_oracle.cpp``,
compiled to its own library in a temporary directory and loaded in place of
the real oracle for the duration of one test (CPU only).
"""

import concurrent.futures as cf
import os
import shutil

import pytest

import oracle
import oracle_pins

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")

# (name, original text, mutated text)
MUTANTS = [
    ("spike2_sign", "w.b2 = J.c * a[5] - J.s * a[4];", "w.b2 = J.c * a[5] + J.s * a[4];"),
    ("spike1_transposed", "w.b1 = J.c * a[4] + J.s * a[5];", "w.b1 = J.c * a[5] + J.s * a[4];"),
    ("jacobi_half_diff", "T d = (p - r) * T(0.5);", "T d = (r - p) * T(0.5);"),
    ("jacobi_l2", "J.l2 = r - t * q;", "J.l2 = r + t * q;"),
    ("jacobi_s_sign", "J.s = t * k;", "J.s = -t * k;"),
    ("secular_sign", "T f = x - gbar - b1 * r1 - b2 * r2;          // spectral function",
     "T f = x - gbar - b1 * r1 + b2 * r2;          // spectral function"),
    ("derivative_term", "T fp = T(1.0) + b1 * r1 * r1 + b2 * r2 * r2; // Eq. (3)",
     "T fp = T(1.0) + b1 * r1 * r1 + b2 * r2; // Eq. (3)"),
    ("omega0_power", "T w0 = T(1.0) + b2 * abar * r2 * r2 * r2;", "T w0 = T(1.0) + b2 * abar * r2 * r2;"),
    ("increment_factor2", "T q = T(2.0) * f / b;", "T q = f / b;"),
    ("increment_b", "T b = fp + f * r1;", "T b = fp - f * r1;"),
    ("start_conjugate", "T x = (gbar >= T(0.0)) ? hg + rt : bsum / (rt - hg);",
     "T x = (gbar >= T(0.0)) ? hg + rt : bsum / (rt + hg);"),
    ("stop_too_early", "if (f < T(P.c_term * EPS) * x * fp) { converged = 1; break; }",
     "if (f < T(P.c_term * EPS * 1e8) * x * fp) { converged = 1; break; }"),
    ("nu_not_permuted", "nu = bg_zero(abar, bb2, bb1, a2 - g, P, &rn, tn);",
     "nu = bg_zero(abar, bb1, bb2, a2 - g, P, &rn, tn);"),
    ("trace_identity", "lamv[1] = nu - mu + g;", "lamv[1] = mu - nu + g;"),
    ("lambda3_sign", "lamv[2] = a2 - nu;", "lamv[2] = a2 + nu;"),
    ("u1_swapped_spikes", "V[0][0] = b1 * mpa; V[0][1] = b2 * mu;", "V[0][0] = b2 * mpa; V[0][1] = b1 * mu;"),
    ("u2_last", "V[1][2] = b1 * b2 * abar;", "V[1][2] = b1 * b2 * a1;"),
    ("u3_sign", "V[2][2] = T(0.0) - nu * npa;", "V[2][2] = nu * npa;"),
    ("deflated_eigenvalue", "lamv[0] = a1 * gc * gc + a2 * gs * gs;", "lamv[0] = a1 * gs * gs + a2 * gc * gc;"),
    ("deflated_vector", "V[0][0] = gc; V[0][1] = T(0.0) - gs;", "V[0][0] = gs; V[0][1] = T(0.0) - gc;"),
    ("deflation_test_difference", "rhs = T(P.c_defl * EPS) * fabs(a1 + a2) * (h * h);",
     "rhs = T(P.c_defl * EPS) * fabs(a1 - a2) * (h * h);"),
    ("back_transform_sign", "T x0 = w.c * V[k][0] - w.s * V[k][1];", "T x0 = w.c * V[k][0] + w.s * V[k][1];"),
    ("unscale_exponent", "lam_out[k] = std::ldexp(lam[ord[k]], e);", "lam_out[k] = std::ldexp(lam[ord[k]], -e);"),
    ("sign_rule", "double sg = (v[im] < 0.0) ? -1.0 : 1.0;", "double sg = (v[im] > 0.0) ? -1.0 : 1.0;"),
    ("sort_descending", "lam[ord[j]] < lam[ord[j - 1]]", "lam[ord[j]] > lam[ord[j - 1]]"),
    ("normalisation_dropped", "for (int i = 0; i < 3; ++i) V[k][i] = V[k][i] * inv;",
     "for (int i = 0; i < 2; ++i) V[k][i] = V[k][i] * inv;"),
    ("grad_transposed", "C[i][j] = (std::fabs(gap) < tau * nrm) ? 0.0 : M[i][j] / gap;",
     "C[i][j] = (std::fabs(gap) < tau * nrm) ? 0.0 : M[j][i] / gap;"),
    ("grad_gap_sign", "double gap = lam[j] - lam[i];", "double gap = lam[i] - lam[j];"),
    ("grad_mirror_dropped", "gA[3] = Ab[0][1] + Ab[1][0];", "gA[3] = Ab[0][1];"),
    ("grad_mask_ignored", "C[i][j] = (std::fabs(gap) < tau * nrm) ? 0.0 : M[i][j] / gap;",
     "C[i][j] = M[i][j] / gap;"),
    ("newton_step_sign", "T xn = x - f / fp;", "T xn = x + f / fp;"),
    ("direct_step_dropped", "if (delta < x * T(0.5)) {", "if (true) {"),
    ("direct_step_sigma_sign", "T sigma = w0 * x - w1 * r1 - f;", "T sigma = w0 * x - w1 * r1 + f;"),
    ("norm_unscaled", "if (m > 0.0) std::frexp(m, &ev);", "(void)m;"),
    ("tiny_spike_rule_dropped", "constexpr double kTinySpike = 0x1p-480;", "constexpr double kTinySpike = 0.0;"),
]


@pytest.fixture(scope="module")
def mutant_libs(tmp_path_factory):
    base = tmp_path_factory.mktemp("mutants")
    with open(os.path.join(SRC, "syev3_oracle.cpp")) as fh:
        text = fh.read()
    jobs = {}
    for name, old, new in MUTANTS:
        assert text.count(old) == 1, f"mutant {name}: pattern must occur exactly once"
        d = base / name
        d.mkdir()
        (d / "syev3_oracle.cpp").write_text(text.replace(old, new))
        shutil.copy(os.path.join(SRC, "ddjacobi.cpp"), d / "ddjacobi.cpp")
        jobs[name] = str(d)
    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        futs = {name: ex.submit(oracle.build, True, d, os.path.join(d, "liboracle.so")) for name, d in jobs.items()}
        return {name: f.result() for name, f in futs.items()}


def test_unmutated_oracle_passes_every_pin(oracle_mod):
    for name, fn in oracle_pins.PINS.items():
        fn()


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS])
def test_mutant_is_caught(name, mutant_libs):
    oracle.use_library(mutant_libs[name])
    caught = []
    try:
        for pin_name, fn in oracle_pins.PINS.items():
            try:
                fn()
            except (AssertionError, FloatingPointError, ValueError, ZeroDivisionError, OverflowError):
                caught.append(pin_name)
    finally:
        oracle.use_library(None)
    assert caught, f"no pin catches mutant {name}"
