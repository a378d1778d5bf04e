"""The oracle's pins reject planted mistakes.

Each case copies ep_oracle.c, plants one plausible mistake (a dropped term, a
flipped sign, a swapped index, a wrong coefficient), compiles the copy on the
CPU and runs the pin suite against it in a subprocess.  The pins must fail for
every mutant; otherwise the mistake would be invisible to them.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "ep_oracle.c")

MUTANTS = {
    "rhs_dq_drops_self_term": (
        "            for (int c = 0; c < dim; ++c) sq[c] += g * pj[c];\n            if (j != i) {",
        "            if (j != i) for (int c = 0; c < dim; ++c) sq[c] += g * pj[c];\n            if (j != i) {"),
    "rhs_dp_sign": ("sp[c] -= w * (qi[c] - qj[c]);", "sp[c] += w * (qi[c] - qj[c]);"),
    "rhs_dp_uses_pi_twice": ("double w = dot(dim, pi, pj) * orc_phi", "double w = dot(dim, pi, pi) * orc_phi"),
    "gauss_phi_power": ("return -orc_G(kernel, sigma, r) / (sigma * sigma);", "return -orc_G(kernel, sigma, r) / sigma;"),
    "tent_phi_power": ("-1.0 / (sigma * r) : 0.0;", "-1.0 / (sigma * r * r) : 0.0;"),
    "hamiltonian_half": ("    return 0.5 * total;", "    return total;"),
    "rk4_weight": ("(k1q[a] + 2.0 * k2q[a] + 2.0 * k3q[a] + k4q[a])", "(k1q[a] + 2.0 * k2q[a] + 1.0 * k3q[a] + 2.0 * k4q[a])"),
    "rk4_stage3_input": ("yq[a] = q[a] + 0.5 * dt * k2q[a];\n        yp[a] = p[a] + 0.5 * dt * k2p[a];",
                         "yq[a] = q[a] + 0.5 * dt * k1q[a];\n        yp[a] = p[a] + 0.5 * dt * k2p[a];"),
    "match_update_sign": ("p0[a] += h * (Y[a] - q1[a]);", "p0[a] -= h * (Y[a] - q1[a]);"),
    "hvp_drops_psi": ("b * (phi * dv[c] + psi * ddv * d[c])", "b * (phi * dv[c])"),
    "hvp_transposed_cross_term": ("double a = dot(dim, vpi, pj) + dot(dim, pi, vpj);",
                                  "double a = dot(dim, vpj, pj) + dot(dim, pi, vpj);"),
    "adjoint_stage_coeff": ("kb3q[a] += dt * yq[a]; kb3p[a] += dt * yp[a];",
                            "kb3q[a] += 0.5 * dt * yq[a]; kb3p[a] += 0.5 * dt * yp[a];"),
    "adjoint_drops_metric_term": ("grad[a] = k1q[a] + xbp[a];", "grad[a] = xbp[a];"),
    "expcone_psi_term": ("(1.0 / (sigma * sigma * r * r) + 1.0 / (sigma * r * r * r))",
                         "(1.0 / (sigma * sigma * r * r))"),
    "cell_predicate_le": ("if (r2 < 1.0f) {", "if (r2 <= 1.1f) {"),
    "velocity_uses_positions": ("for (int c = 0; c < dim; ++c) s[c] += g * p[j * dim + c];",
                                "for (int c = 0; c < dim; ++c) s[c] += g * q[j * dim + c];"),
    "flow_stage3_input": ("for (a = 0; a < md; ++a) yx[a] = x1[a] + 0.5 * dt * k2x[a];",
                          "for (a = 0; a < md; ++a) yx[a] = x1[a] + 0.5 * dt * k1x[a];"),
    "flow_weights": ("x1[a] += dt / 6.0 * (k1x[a] + 2.0 * k2x[a] + 2.0 * k3x[a] + k4x[a]);",
                     "x1[a] += dt / 6.0 * (k1x[a] + 2.0 * k2x[a] + 1.0 * k3x[a] + 2.0 * k4x[a]);"),
    "inexact_term_sign": ("for (long a = 0; a < n * dim; ++a) dq[a] += s2 * p[a];",
                          "for (long a = 0; a < n * dim; ++a) dq[a] -= s2 * p[a];"),
    "inexact_stop_on_residual": ("if (fabs(d) > dmax) dmax = fabs(d);",
                                 "if (fabs(d) / h > dmax) dmax = fabs(d) / h;"),
    "tangent_dp_sign": ("                dkp[s][a] = -hq[a];", "                dkp[s][a] = hq[a];"),
    "tangent_at_step_start": ("            orc_hvp(dim, kernel, sigma, n, yq, yp, dyq, dyp, hq, hp);",
                              "            orc_hvp(dim, kernel, sigma, n, q1, p1, dyq, dyp, hq, hp);"),
    # (the line break in front keeps each site unique: the inexact loop's inline copy
    # of the gain is indented deeper)
    "default_gain_skips_self": (
        "\n        for (long j = 0; j < n; ++j) row += fabs(",
        "\n        for (long j = 0; j < n; ++j) if (j != i) row += fabs("),
    "default_gain_min_row": ("\n        if (row > best) best = row;", "\n        if (best == 0.0 || row < best) best = row;"),
    "default_gain_mean_row": ("\n        if (row > best) best = row;", "\n        best += row / (double)n;"),
    "flow_stale_velocity_stage": ("orc_velocity(dim, kernel, sigma, n, yq, yp, m, yx, k4x);",
                                  "orc_velocity(dim, kernel, sigma, n, q1, p1, m, yx, k4x);"),
}
# mutations applied at every occurrence: these lines appear both in the full
# function and in its row-sampled variant (orc_rhs_rows, orc_cell_neighbors_rows),
# or in both RK4 integrators (the shoot and the flow)
EVERYWHERE = {"cell_predicate_le", "rhs_dq_drops_self_term", "rhs_dp_sign", "rhs_dp_uses_pi_twice", "rk4_weight"}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    if name in EVERYWHERE:
        assert src.count(old) >= 1, f"mutation site for {name} missing in ep_oracle.c"
    else:
        assert src.count(old) == 1, f"mutation site for {name} not unique in ep_oracle.c"
    mut = tmp_path / "ep_oracle_mut.c"
    mut.write_text(src.replace(old, new))
    lib = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-std=c11", "-shared", "-fPIC",
                    "-o", str(lib), str(mut), "-lm"], check=True)
    env = dict(os.environ, EP_ORACLE_VARIANT_LIB=str(lib), OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"pins accepted the mutant {name}:\n{r.stdout[-2000:]}"


# --------------------------------------------------------------------------- the update rules (Python)
# The velocity update and the Newton loop are Python around library solves; each case
# plants one plausible mistake in a copy of the oracle module (same C library) and runs
# the pins of the rules against it in this process.
import importlib
import inspect
import itertools
import types

ORACLE_PY = os.path.join(ROOT, "oracle", "oracle.py")

PY_MUTANTS = {
    "velocity_multiplies_by_gram": ("p = p + h * np.linalg.solve(GX, r)", "p = p + h * (GX @ r)"),
    "velocity_update_sign": ("p = p + h * np.linalg.solve(GX, r)", "p = p - h * np.linalg.solve(GX, r)"),
    "velocity_drops_gain": ("p = p + h * np.linalg.solve(GX, r)", "p = p + np.linalg.solve(GX, r)"),
    "newton_transposed_jacobian": ("p = p + h * np.linalg.solve(J, r.ravel()).reshape(n, dim)",
                                   "p = p + h * np.linalg.solve(J.T, r.ravel()).reshape(n, dim)"),
    "newton_update_sign": ("p = p + h * np.linalg.solve(J, r.ravel()).reshape(n, dim)",
                           "p = p - h * np.linalg.solve(J, r.ravel()).reshape(n, dim)"),
    "newton_identity_gain": ("p = p + h * np.linalg.solve(J, r.ravel()).reshape(n, dim)",
                             "p = p + h * r"),
}


def _rule_pins():
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    pins = importlib.import_module("test_oracle_pins")
    names = [k for k in dir(pins) if k.startswith("test_") and ("velocity_rule" in k or "newton" in k)]
    return pins, names


def _calls(fn):
    marks = [m for m in getattr(fn, "pytestmark", []) if m.name == "parametrize"]
    if not marks:
        yield {}
        return
    keys, values = [], []
    for m in marks:
        keys.append([s.strip() for s in m.args[0].split(",")])
        values.append(m.args[1])
    for combo in itertools.product(*values):
        kw = {}
        for ks, v in zip(keys, combo):
            kw.update({ks[0]: v} if len(ks) == 1 else dict(zip(ks, v)))
        yield kw


@pytest.mark.parametrize("name", sorted(PY_MUTANTS))
def test_rule_pins_reject_mutant(name):
    old, new = PY_MUTANTS[name]
    src = open(ORACLE_PY).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique in oracle.py"
    mod = types.ModuleType("oracle_mutant")
    mod.__file__ = ORACLE_PY
    exec(compile(src.replace(old, new), ORACLE_PY, "exec"), mod.__dict__)
    pins, names = _rule_pins()
    real = pins.o
    failed = False
    try:
        pins.o = mod
        for nm in names:
            fn = getattr(pins, nm)
            for kw in _calls(fn):
                try:
                    fn(**kw)
                except Exception:
                    failed = True
                    break
            if failed:
                break
    finally:
        pins.o = real
    assert failed, f"the rule pins accepted the mutant {name}"
    assert inspect.ismodule(mod)
