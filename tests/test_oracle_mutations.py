"""The oracle's pins must catch plausible mistakes: each case below plants
one (a flipped sign, a dropped term, a transposed operand, a wrong index or
iterate) in a copy of the oracle source, builds it into a scratch library and
requires the pin suite to fail against it."""
import os
import subprocess
import sys

import pytest

from tests.conftest import ROOT

SRC = os.path.join(ROOT, "oracle", "kin_oracle.c")

MUTATIONS = {
    "volume_term_sign": ("A[i * nn + q] -= tau * vol_weight(P, w, q) * vg;",
                         "A[i * nn + q] += tau * vol_weight(P, w, q) * vg;"),
    "outflow_face_dropped": ("if (vn > 0 && on_face) A[i * nn + i] += tau * vn * face_weight(P, w, i, a);",
                             "if (0) {}"),
    "diff_matrix_transposed": ("vg += V[a] * D[iq[a] * np + ii[a]] / cell_size(P, a);",
                               "vg += V[a] * D[ii[a] * np + iq[a]] / cell_size(P, a);"),
    "interface_uses_current_iterate": ("const double* src = boundary ? prev : cur;",
                                       "const double* src = cur;"),
    "interior_uses_previous_iterate": ("const double* src = boundary ? prev : cur;",
                                       "const double* src = prev;"),
    "crank_nicolson_extrapolation_dropped": ("f[i] = 2.0 * cur[i] - f[i];", "f[i] = cur[i];"),
    "maxwellian_flux_sign": ("M[(2 * a) * m + v] = W[v] / (2.0 * d) + Q[a][v] / (2.0 * P->lambda);",
                             "M[(2 * a) * m + v] = W[v] / (2.0 * d) - Q[a][v] / (2.0 * P->lambda);"),
    "pressure_dropped": ("Q[1 + b] = W[1 + b] * ua + (b == axis ? pr : 0.0);",
                         "Q[1 + b] = W[1 + b] * ua;"),
    "relaxation_sign": ("*fp = P->omega * M[pop] + (1.0 - P->omega) * (*fp);",
                        "*fp = P->omega * M[pop] - (1.0 - P->omega) * (*fp);"),
    "inflow_node_index": ("b[i] += tau * (-vn) * C->facew[a][i] * src[nbase + C->acr[a][i]];",
                          "b[i] += tau * (-vn) * C->facew[a][i] * src[nbase + i];"),
    "half_step_is_full_step": ("double tau = 0.5 * P->dt;\n    size_t base",
                               "double tau = P->dt;\n    size_t base"),
    "kinetic_energy_factor": ("ke *= 0.5 / rho;", "ke *= 1.0 / rho;"),
    "gll_weight_power": ("w[j] = 0.5 * 2.0 / (p * (p + 1.0) * pp * pp);",
                         "w[j] = 0.5 * 2.0 / (p * (p + 1.0) * pp);"),
    "sweep_direction": ("if (C->V[a] < 0) {", "if (C->V[a] > 0) {"),
    "d2q3_angle": ("V[0] = P->lambda * cos(2.0 * M_PI * k / 3.0);",
                   "V[0] = P->lambda * cos(2.0 * M_PI * k / 4.0);"),
    "d3q4_diagonal_sign": ("{{1, 1, 1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}}",
                           "{{1, 1, 1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, -1}}"),
    "moment_row_velocity_component": ("for (int a = 0; a < d; ++a) A[(1 + a) * nv + k] = V[a];",
                                      "for (int a = 0; a < d; ++a) A[(1 + a) * nv + k] = V[d - 1 - a];"),
    "maxwell_cross_product_sign": ("NxE[k] = E[j];", "NxE[k] = -E[j];"),
    "maxwell_source_factor_inverted": ("const double mu = (1.0 - 0.5 * P->sigma * P->dt) / (1.0 + 0.5 * P->sigma * P->dt);",
                                       "const double mu = (1.0 + 0.5 * P->sigma * P->dt) / (1.0 - 0.5 * P->sigma * P->dt);"),
    "maxwell_source_damps_h": ("Wp[v] = v < 3 ? mu * W[v] : W[v];", "Wp[v] = mu * W[v];"),
    "maxwell_literal_relaxation": ("*fp = Mp[pop] + (1.0 - P->omega) * (*fp - M[pop]);",
                                   "*fp = P->omega * Mp[pop] + (1.0 - P->omega) * (*fp);"),
    "inflow_face_swapped": ("C->bval[a][side < 0 ? 0 : 1]", "C->bval[a][side < 0 ? 1 : 0]"),
    "inflow_axis_wraps": ("if (P->inflow[a] && c[a] + side != nb[a]) {",
                          "if (P->inflow[a] && c[a] + side != nb[a] && 0) {"),
    "inflow_value_first_variable": ("C.bval[a][sd] = M[k * ko_num_vars(P) + v];",
                                    "C.bval[a][sd] = M[k * ko_num_vars(P)];"),
}

PIN_FILES = ["tests/test_oracle_basis.py", "tests/test_oracle_relaxation.py",
             "tests/test_oracle_transport.py", "tests/test_oracle_simplex.py",
             "tests/test_oracle_maxwell.py", "tests/test_oracle_inflow.py"]

# the tetrahedral-mesh transport (kin_oracle_tet.c), pinned by test_oracle_tet.py
SRC_TET = os.path.join(ROOT, "oracle", "kin_oracle_tet.c")
MUTATIONS_TET = {
    "tet_volume_term_sign": ("A[i * 4 + j] = mij - tau * vg * g.vol / 4.0;",
                             "A[i * 4 + j] = mij + tau * vg * g.vol / 4.0;"),
    "tet_mass_matrix_lumped": ("const double mij = g.vol / 20.0 * (i == j ? 2.0 : 1.0);",
                               "const double mij = g.vol / 20.0 * (i == j ? 5.0 : 0.0);"),
    "tet_outflow_face_mass_diagonal": ("A[i * 4 + j] += tau * vn * g.area[a] / 12.0 * (i == j ? 2.0 : 1.0);",
                                       "A[i * 4 + j] += tau * vn * g.area[a] / 12.0 * (i == j ? 1.0 : 1.0);"),
    "tet_interface_uses_current_iterate": ("const double* src = is_interface(T, c, a) ? prev : cur;",
                                           "const double* src = cur;"),
    "tet_inflow_node_not_matched": ("fr[j] = src[(size_t)R * 4 + C->match[((size_t)c * 4 + a) * 4 + j]];",
                                    "fr[j] = src[(size_t)R * 4 + j];"),
    "tet_normal_points_inward": ("const double s = dot3(n, to_a) > 0 ? -1.0 : 1.0;",
                                 "const double s = dot3(n, to_a) > 0 ? 1.0 : -1.0;"),
}


def _run_pins(tmp_path, mutated_name, mutated_text, pin_files):
    """Build the oracle with one source replaced by mutated_text and run the
    pins against it; returns pytest's exit code."""
    hdr = os.path.join(ROOT, "oracle", "kin_oracle.h")
    (tmp_path / "kin_oracle.h").write_text(open(hdr).read())
    srcs = []
    for path in (SRC, SRC_TET):
        dst = tmp_path / os.path.basename(path)
        dst.write_text(mutated_text if os.path.basename(path) == mutated_name else open(path).read())
        srcs.append(str(dst))
    lib = tmp_path / "libkin_oracle_mut.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", *srcs, "-o", str(lib), "-lm"])
    env = dict(os.environ, KIN_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider"]
                       + pin_files, cwd=ROOT, env=env, capture_output=True, text=True)
    return r


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path):
    before, after = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(before) >= 1, "mutation anchor vanished from the oracle source"
    r = _run_pins(tmp_path, "kin_oracle.c", src.replace(before, after, 1), PIN_FILES)
    assert r.returncode == 1, f"planted mistake '{name}' passed every pin:\n{r.stdout[-800:]}"


@pytest.mark.parametrize("name", sorted(MUTATIONS_TET))
def test_tet_pins_catch_planted_mistake(name, tmp_path):
    before, after = MUTATIONS_TET[name]
    src = open(SRC_TET).read()
    assert src.count(before) >= 1, "mutation anchor vanished from the tetrahedral oracle source"
    r = _run_pins(tmp_path, "kin_oracle_tet.c", src.replace(before, after, 1), ["tests/test_oracle_tet.py"])
    assert r.returncode == 1, f"planted mistake '{name}' passed every pin:\n{r.stdout[-800:]}"
