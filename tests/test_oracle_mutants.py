"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a copy of ``oracle/heat_oracle.c`` (a dropped
term, a wrong sign or index, a transposed operand, a wrong factor), compiles it
on the CPU and runs the pin suite against it: the suite must fail.  The
unmodified copy must pass.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "heat_oracle.c")
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")

MUTANTS = {
    "drop_radial_metric": ("o->Arm[c] = o->rf[i] * lf / (ri * hb * o->h[i]);",
                           "o->Arm[c] = lf / (hb * o->h[i]);"),
    "wrong_h_index": ("o->Arm[c] = o->rf[i] * lf / (ri * hb * o->h[i]);",
                      "o->Arm[c] = o->rf[i] * lf / (ri * hb * o->h[i + 1]);"),
    "hbar_not_averaged": ("o->hbar[i] = 0.5 * (o->h[i] + o->h[i + 1]);", "o->hbar[i] = o->h[i + 1];"),
    "axis_face_not_zero": ("o->rf[0] = o->r_lo;", "o->rf[0] = 0.5 * o->rc[0];"),
    "harmonic_weights_swapped": ("return (da + db) / (da / ka + db / kb);",
                                 "return (da + db) / (db / ka + da / kb);"),
    "dirichlet_factor_dropped": ("o->Dzh[c] = 2.0 * lam / (eb * o->eta[Nz]);",
                                 "o->Dzh[c] = lam / (eb * o->eta[Nz]);"),
    "explicit_z_sign": ("if (o->Azp[c] != 0.0) s += o->Azp[c] * (T[IDX(o, i, j + 1)] - t);",
                        "if (o->Azp[c] != 0.0) s += o->Azp[c] * (t - T[IDX(o, i, j + 1)]);"),
    "transposed_offdiagonals": ("                a[i] = -o->Arm[c];\n                cc[i] = -o->Arp[c];",
                                "                a[i] = -o->Arp[c];\n                cc[i] = -o->Arm[c];"),
    "thomas_pivot": ("dw[i] = (d[i] - a[i] * dw[i - 1]) / m;", "dw[i] = (d[i] - a[i] * dw[i - 1]) / b[i];"),
    "full_tau_in_half_step": ("const double half = 0.5 * tau;\n    double *T = o->T, *Tb = o->Tbar;",
                              "const double half = tau;\n    double *T = o->T, *Tb = o->Tbar;"),
    "source_dropped_in_half_step_2": (
        "d[j] = w * Tb[c] + lambda_r(o, Tb, i, j) + xs + o->Dzl[c] * o->Tbc[2] + o->Dzh[c] * o->Tbc[3];",
        "d[j] = w * Tb[c] + lambda_r(o, Tb, i, j) + o->Dzl[c] * o->Tbc[2] + o->Dzh[c] * o->Tbc[3];"),
    "energy_weight_cell_width": ("double wgt = o->rc[i] * o->hbar[i] * o->etabar[j];",
                                 "double wgt = o->rc[i] * o->dr[i] * o->etabar[j];"),
    # the explicit limit (tau_exp): a dropped Dirichlet coupling, dropped z
    # couplings, the half-step length taken for the step
    "tau_exp_drops_dirichlet": ("o->Drl[c] + o->Drh[c] + o->Dzl[c] + o->Dzh[c];\n        if (s > 0.0",
                                "o->Drl[c] + o->Drh[c] + o->Dzl[c];\n        if (s > 0.0"),
    "tau_exp_drops_z_couplings": ("double s = o->Arm[c] + o->Arp[c] + o->Azm[c] + o->Azp[c] +",
                                  "double s = o->Arm[c] + o->Arp[c] +"),
    "tau_exp_half_step": ("if (s > 0.0 && o->cap[c] / s < best) best = o->cap[c] / s;",
                          "if (s > 0.0 && o->cap[c] / s < best) best = 0.5 * o->cap[c] / s;"),
}


# Planted mistakes in the full method (temperature-dependent coefficients,
# the simple iteration, adaptive tau, the pulsed source); the suite run
# against them is the nonlinear pins'.
NL_MUTANTS = {
    "nl_capacity_at_old_layer_in_half_step_1": ("double w = cap_at(o, n, c, Ts[c]) / half;",
                                                "double w = cap_at(o, n, c, T[c]) / half;"),
    "nl_r_operator_at_old_layer_in_half_step_1": (
        "couplings_from(o, n->lam_s, n->face_mean, i, j, ks);  /* r-operator at T^s */",
        "couplings_from(o, n->lam_o, n->face_mean, i, j, ks);  /* r-operator at T^s */"),
    "nl_explicit_z_operator_at_iterate": (
        "couplings_from(o, n->lam_o, n->face_mean, i, j, ko);  /* z-operator at T   */",
        "couplings_from(o, n->lam_s, n->face_mean, i, j, ko);  /* z-operator at T   */"),
    "nl_capacity_iterated_in_half_step_2": ("double w = n->cap_x[c] / half;",
                                            "double w = cap_at(o, n, c, Ts[c]) / half;"),
    "nl_z_operator_at_half_layer_in_half_step_2": (
        "couplings_from(o, n->lam_s, n->face_mean, i, j, ks);  /* z-operator at T^s   */",
        "couplings_from(o, n->lam_o, n->face_mean, i, j, ks);  /* z-operator at T^s   */"),
    "nl_source_at_step_start": ("double pt = orc_pulse(n->model, t + 0.5 * tau,", "double pt = orc_pulse(n->model, t,"),
    "nl_quartered_not_halved": ("tau *= 0.5;", "tau *= 0.25;"),
    "nl_estimates_swapped": ("double tau = trs ? tau_trs : tau_base;", "double tau = trs ? tau_base : tau_trs;"),
    "pulse_erf_sign": ("s += 0.5 * (erf(xi * (zeta * a / t_trs - 1.0)) - erf(xi * (zeta * b / t_trs - 1.0)));",
                       "s += 0.5 * (erf(xi * (zeta * a / t_trs - 1.0)) + erf(xi * (zeta * b / t_trs - 1.0)));"),
    "pulse_no_half": ("s += 0.5 * (erf(xi * (zeta * a / t_trs - 1.0))", "s += (erf(xi * (zeta * a / t_trs - 1.0))"),
    "table_wrong_knot": ("return v[k] + (v[k + 1] - v[k]) * (T - Tk[k]) / (Tk[k + 1] - Tk[k]);",
                         "return v[k] + (v[k + 1] - v[k]) * (T - Tk[k + 1]) / (Tk[k + 1] - Tk[k]);"),
}
NL_PINS = os.path.join(ROOT, "tests", "test_oracle_nl_pins.py")


def _build(tmp_path, name, src_text):
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"lib_{name}.so"
    c.write_text(src_text)
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", str(c), "-o", str(so), "-lm"])
    return str(so)


def _run_pins(so, pins=PINS):
    env = dict(os.environ, HEAT_ORACLE_LIB=so)
    r = subprocess.run([sys.executable, "-m", "pytest", pins, "-x", "-q", "-p", "no:cacheprovider"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    return r.returncode, r.stdout[-2000:]


def test_unmodified_copy_passes(tmp_path):
    so = _build(tmp_path, "orig", open(SRC).read())
    for pins in (PINS, NL_PINS):
        rc, out = _run_pins(so, pins)
        assert rc == 0, out


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation site for {name} not found exactly once"
    so = _build(tmp_path, name, text.replace(old, new))
    rc, out = _run_pins(so)
    assert rc != 0, f"pins did not catch {name}:\n{out}"


@pytest.mark.parametrize("name", sorted(NL_MUTANTS))
def test_planted_mistake_in_the_full_method_is_caught(tmp_path, name):
    old, new = NL_MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation site for {name} not found exactly once"
    so = _build(tmp_path, name, text.replace(old, new))
    rc, out = _run_pins(so, NL_PINS)
    assert rc != 0, f"nonlinear pins did not catch {name}:\n{out}"
