"""The oracle's pins are discriminating: each plausible mistake planted in a
copy of the oracle source (a flipped sign, a wrong index or coefficient, a
swapped operand) makes at least one pin fail -- test_oracle_pins.py for the
forward scheme, test_oracle_adjoint.py for the discrete adjoint,
test_oracle_variants.py for the local dissipation and the variational form.  The first
occurrence of each anchor is mutated (the forward code precedes the adjoint
code that mirrors some of its lines).

Mistakes are planted only in a temporary copy of the C oracle, compiled on
the CPU; the committed oracle is untouched.
"""
import os
import shutil
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle", "lsp_oracle.c")

# name -> (text in the oracle, planted replacement)
MUTANTS = {
    "weno_substencil3_sign": ("double phi3 = v3 / 3.0 + 5.0", "double phi3 = -v3 / 3.0 + 5.0"),
    "weno_optimal_weight3": ("double a3 = 0.3 /", "double a3 = 0.1 /"),
    "weno_sigma2_index": (
        "double s2 = 13.0 / 12.0 * (v2 - 2.0 * v3 + v4) * (v2 - 2.0 * v3 + v4);",
        "double s2 = 13.0 / 12.0 * (v2 - 2.0 * v1 + v4) * (v2 - 2.0 * v1 + v4);"),
    "weno_eps_unsquared": ("double eps = 1e-6 * mx + 1e-99;",
                           "double eps = 1e-6 * sqrt(mx) + 1e-99;"),
    "weno_right_not_mirrored": ("pp[i] = weno5_combine(d[5], d[4], d[3], d[2], d[1]);",
                                "pp[i] = weno5_combine(d[1], d[2], d[3], d[4], d[5]);"),
    "eno2_selection_flipped": ("int first = force2 < 0 ? (fabs(a) <= fabs(b)) : (force2 == 0);",
                               "int first = force2 < 0 ? (fabs(a) > fabs(b)) : (force2 == 0);"),
    "eno3_kstar": ("kstar = k - 1;", "kstar = k;"),
    "eno3_selection_flipped": ("int first3 = force3 < 0 ? (fabs(e) <= fabs(f)) : (force3 == 0);",
                               "int first3 = force3 < 0 ? (fabs(e) > fabs(f)) : (force3 == 0);"),
    "eno2_q2_factor": ("double r = q1 + c * (double)(2 * (i - k) - 1) * dx;",
                       "double r = q1 + c * (double)(2 * (i - k) + 1) * dx;"),
    "second_difference_factor": ("return (D1h(u, j, dx) - D1h(u, j - 1, dx)) / (2.0 * dx);",
                                 "return (D1h(u, j, dx) - D1h(u, j - 1, dx)) / (dx);"),
    "upwind_sides_swapped": (
        "pm[i] = (u[i] - u[i - 1]) / dx;\n        pp[i] = (u[i + 1] - u[i]) / dx;",
        "pp[i] = (u[i] - u[i - 1]) / dx;\n        pm[i] = (u[i + 1] - u[i]) / dx;"),
    "extrapolation_sign": ("ext[G - k] = line[0] + (double)k * (line[0] - line[1]);",
                           "ext[G - k] = line[0] - (double)k * (line[0] - line[1]);"),
    "periodic_wrap_off_by_one": ("ext[G + n - 1 + k] = line[(k - 1) % n];",
                                 "ext[G + n - 1 + k] = line[k % n];"),
    "dissipation_sign": ("diss += ak * 0.5 * (pp[k][i] - pm[k][i]);",
                         "diss -= ak * 0.5 * (pp[k][i] - pm[k][i]);"),
    "rk2_average": ("phi[i] = 0.5 * (phi[i] + p1[i] + dt * L[i]);",
                    "phi[i] = 0.5 * (phi[i] + p1[i]) + dt * L[i];"),
    "rk3_second_stage": ("p2[i] = 0.75 * phi[i] + 0.25 * (p1[i] + dt * L[i]);",
                         "p2[i] = 0.5 * phi[i] + 0.5 * (p1[i] + dt * L[i]);"),
    "cfl_dt_formula": ("s += alpha[k] / orc_dx(P, k);", "s += alpha[k] * orc_dx(P, k);"),
    "tube_max_instead_of_min": ("if (g[i] < phi[i]) phi[i] = g[i];",
                                "if (g[i] > phi[i]) phi[i] = g[i];"),
    "air3d_switching_sign": ("we * fabs(p[0] * Y - p[1] * X - p[2])",
                             "we * fabs(p[0] * Y + p[1] * X - p[2])"),
    "air3d_cos_sin": ("p[0] * (-ve + vp * cos(th))", "p[0] * (-ve + vp * sin(th))"),
    "car4d_bound_axis": ("if (k == 1) return fabs(x[3] * sin(x[2]));",
                         "if (k == 1) return fabs(x[3] * cos(x[2]));"),
    # the switching term as Eq. 32 prints it (the reading derives it from Eq. 31)
    "rockets_switch_as_printed": ("ue * fabs(p[0] * X - p[2])", "ue * fabs(p[0] * X + p[2])"),
    "rockets_gravity_sign": ("p[1] * (a * sin(th) + a - g)", "p[1] * (a * sin(th) + a + g)"),
    "rockets_bound_axis": ("if (k == 0) return a * fabs(cos(x[2])) + ue * fabs(x[0]);",
                           "if (k == 0) return a * fabs(cos(x[2])) + ue * fabs(x[1]);"),
    "double_integrator_input_sign": ("return -(p[0] * x[1] - um * fabs(p[1]));",
                                     "return -(p[0] * x[1] + um * fabs(p[1]));"),
}

# mistakes in the discrete adjoint, caught by the finite-difference pins
ADJOINT_MUTANTS = {
    "adj_weno_eps_term": ("if (m == mstar) gm -= bsum * 2e-6 * v[mstar];",
                          "if (m == mstar) gm += bsum * 2e-6 * v[mstar];"),
    "adj_weno_sigma_factor": ("double ds = 13.0 / 6.0 * a[k] * da[k][m] + 0.5 * b[k] * db[k][m];",
                              "double ds = 13.0 / 12.0 * a[k] * da[k][m] + 0.5 * b[k] * db[k][m];"),
    "adj_eno_q2_coeff": ("c[(j - 1) - i + 3] += f2;", "c[(j - 1) - i + 3] -= f2;"),
    "adj_air3d_dHdp2": ("hp[1] = -(vp * sin(th) - um * g1 * X);",
                        "hp[1] = -(vp * sin(th) + um * g1 * X);"),
    "adj_alpha_dt_path": ("double dL_dalpha = alpha_acc[k] - dt_acc * cfl / (S * S * orc_dx(P, k));",
                          "double dL_dalpha = alpha_acc[k] + dt_acc * cfl / (S * S * orc_dx(P, k));"),
    "adj_ghost_weight": ("wt[0] = 1.0 + k;\n        node[1] = 1;",
                         "wt[0] = 1.0 - k;\n        node[1] = 1;"),
    "adj_tube_branch": ("if (g && g[i] < v) { /* the min took the target */",
                        "if (g && g[i] > v) { /* the min took the target */"),
    "adj_rk3_stage2_weight": ("ln[i] += 0.75 * lb[i];", "ln[i] += 0.25 * lb[i];"),
    "adj_rockets_dHdp3_sign": ("hp[2] = ue * g1 + up * g2;", "hp[2] = ue * g1 - up * g2;"),
    "adj_rockets_dHdg_sign": ("hprm[1] = p[1];", "hprm[1] = -p[1];"),
    "adj_rockets_bound_da": ("g[0] = sgn1(w) * (sin(x[2]) + 1.0);", "g[0] = sgn1(w) * sin(x[2]);"),
    "adj_double_integrator_dHdp1": ("hp[0] = -x[1];", "hp[0] = x[1];"),
}


# mistakes in the local dissipation coefficients and the variational form,
# caught by test_oracle_variants.py
VARIANT_MUTANTS = {
    "varform_clip_wrong_side": ("if (P->varform && rate[i] > 0.0) rate[i] = 0.0;",
                                "if (P->varform && rate[i] < 0.0) rate[i] = 0.0;"),
    "llf_own_dimension_global": ("int local = (P->diss == ORC_DISS_LLLF) || (j == k);",
                                 "int local = (P->diss == ORC_DISS_LLLF) || (j != k);"),
    "box_bound_without_abs": ("if (P->dyn == ORC_DYN_QUADRATIC) return fmax(fabs(clo[k]), fabs(chi[k]));",
                              "if (P->dyn == ORC_DYN_QUADRATIC) return fmax(clo[k], chi[k]);"),
    "normal_speed_bound_signed": ("case ORC_DYN_NORMAL_SPEED: return fabs(c[0]);",
                                  "case ORC_DYN_NORMAL_SPEED: return c[0];"),
}
# mistakes in the loss of the differentiation workload (the oracle's Python
# layer), caught by test_oracle_loss.py
PY_SRC = os.path.join(os.path.dirname(HERE), "oracle", "__init__.py")
PY_MUTANTS = {
    "loss_heaviside_sign": ("vol = np.sum(1.0 / (1.0 + np.exp(f / eps))) * dV",
                            "vol = np.sum(1.0 / (1.0 + np.exp(-f / eps))) * dV"),
    "loss_eps_min_dx": ("eps = float(h.max())", "eps = float(h.min())"),
    "loss_grad_sign": ("g = -Hs * (1.0 - Hs) / eps * dV", "g = Hs * (1.0 - Hs) / eps * dV"),
    "interp_periodic_clamped": ("i1 = np.mod(i0 + 1, n)", "i1 = np.minimum(i0 + 1, n - 1)"),
    "interp_weights_swapped": ("w = w * (frac[k] if b else 1.0 - frac[k])",
                               "w = w * (1.0 - frac[k] if b else frac[k])"),
    "interp_no_clamp": ("t = np.clip(t, 0.0, n - 1.0)", "t = t"),
}

PIN_FILE = {**{k: "test_oracle_pins.py" for k in MUTANTS},
            **{k: "test_oracle_adjoint.py" for k in ADJOINT_MUTANTS},
            **{k: "test_oracle_variants.py" for k in VARIANT_MUTANTS}}


@pytest.mark.slow
@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("name", sorted(MUTANTS) + sorted(ADJOINT_MUTANTS) +
                         sorted(VARIANT_MUTANTS))
def test_planted_mistake_is_caught(tmp_path, name):
    src = open(SRC).read()
    old, new = {**MUTANTS, **ADJOINT_MUTANTS, **VARIANT_MUTANTS}[name]
    old, new = old.replace("\\n", "\n"), new.replace("\\n", "\n")
    assert src.count(old) >= 1, f"mutation anchor for {name} not found"
    c = tmp_path / "mutant.c"
    c.write_text(src.replace(old, new, 1))
    so = tmp_path / "mutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", str(c), "-o", str(so), "-lm"],
                   check=True)
    r = subprocess.run(
        [sys.executable, "-m", "pytest", os.path.join(HERE, PIN_FILE[name]), "-x",
         "-q", "-p", "no:cacheprovider"],
        env=dict(os.environ, LSP_ORACLE_LIB=str(so)), capture_output=True, text=True,
        timeout=600)
    assert r.returncode != 0, f"planted mistake {name} passed every pin:\n{r.stdout[-2000:]}"


@pytest.mark.parametrize("name", sorted(PY_MUTANTS))
def test_planted_loss_mistake_is_caught(tmp_path, orc, name):
    """The same for the loss, which the oracle computes in Python: the
    mutated copy of the module is loaded in place of the oracle by the `orc`
    fixture of a separate pytest run (LSP_ORACLE_PY), on the oracle's
    library as built."""
    src = open(PY_SRC).read()
    old, new = PY_MUTANTS[name]
    assert src.count(old) >= 1, f"mutation anchor for {name} not found"
    m = tmp_path / "oracle_mutant.py"
    m.write_text(src.replace(old, new, 1))
    r = subprocess.run(
        [sys.executable, "-m", "pytest", os.path.join(HERE, "test_oracle_loss.py"), "-x", "-q",
         "-p", "no:cacheprovider"],
        env=dict(os.environ, LSP_ORACLE_PY=str(m), LSP_ORACLE_LIB=orc.build()),
        capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"planted mistake {name} passed every pin:\n{r.stdout[-2000:]}"
