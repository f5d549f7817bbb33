"""The oracle's pins bite: each test plants one plausible mistake in a copy of
the oracle's C source (a dropped term, a sign, a transposed operand, swapped
components), builds it, and runs a fast subset of the pins against it
(IDP_ORACLE_LIB); at least one pin must fail.  CPU only."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "idp_oracle.c")

MUTANTS = {
    # energy flux without the pressure work term
    "energy_flux_drops_p": ("F[4][d] = v[d] * (E + p);", "F[4][d] = v[d] * E;"),
    # y and z components of c_ij exchanged in the contraction
    "contraction_transposed": ("out[f] = F[f][0] * c[0] + F[f][1] * c[1] + F[f][2] * c[2];",
                               "out[f] = F[f][0] * c[0] + F[f][2] * c[1] + F[f][1] * c[2];"),
    # c_y read from the c_z row
    "c_component_swapped": ("  c[1] = M->cij[nnz + k];", "  c[1] = M->cij[2 * nnz + k];"),
    # transposed inverse Jacobian in the hexahedral assembly
    "jacobian_transposed": ("grad[v][r] = dphi[v][0] * Jinv[0][r] + dphi[v][1] * Jinv[1][r] + dphi[v][2] * Jinv[2][r];",
                            "grad[v][r] = dphi[v][0] * Jinv[r][0] + dphi[v][1] * Jinv[r][1] + dphi[v][2] * Jinv[r][2];"),
    # wrong sign of the b_ji R_i term of P_ij
    "p_ij_sign": ("(b_ij * rj[f] - b_ji * ri[f] + (dH - d[k]) * (uj[f] - ui[f]))",
                  "(b_ij * rj[f] + b_ji * ri[f] + (dH - d[k]) * (uj[f] - ui[f]))"),
    # second SSP-RK3 stage blended 1/2, 1/2 instead of 3/4, 1/4
    "rk3_stage2_weights": ("U2[q] = 0.75 * U[q] + 0.25 * E[q];", "U2[q] = 0.5 * U[q] + 0.5 * E[q];"),
    # the Psi margin applied with the wrong sign (a stricter test than Psi >= 0)
    "psi_margin_sign": ("const int ok = psi >= -margin * scale;", "const int ok = psi >= margin * scale;"),
    # a wrong factor in the discriminant of Alg. 3's quadratic step
    "newton_discriminant": ("double LamL = dPsiL * dPsiL - 4.0 * PsiL * d112;",
                            "double LamL = dPsiL * dPsiL - 2.0 * PsiL * d112;"),
}

# fast pins first (a mutant run stops at its first failing pin); the
# convergence pin last
PINS = ["tests/test_oracle_margin.py", "tests/test_oracle_stage.py::test_ssprk3_temporal_order",
        "tests/test_oracle_pointwise.py::test_limiter_is_exact_where_psi_is_quadratic",
        "tests/test_oracle_symmetry.py", "tests/test_oracle_matrices.py",
        "tests/test_oracle_2d.py::test_uniform_periodic_closed_forms_2d",
        "tests/test_oracle_2d.py::test_identities_any_quad_mesh",
        "tests/test_oracle_2d.py::test_quad_assembly_is_the_extruded_hex_assembly",
        "tests/test_oracle_2d.py::test_2d_stage_keeps_mz_zero_conserves_and_preserves_free_stream",
        "tests/test_oracle_stage.py::test_conservation_periodic", "tests/test_oracle_stage.py::test_trace_identities",
        "tests/test_oracle_stage.py::test_sod_converges_to_exact"]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(name, tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    old, new = MUTANTS[name]
    with open(SRC) as fh:
        src = fh.read()
    assert src.count(old) == 1, name
    shutil.copy(os.path.join(ROOT, "oracle", "idp_oracle.h"), tmp_path)
    (tmp_path / "idp_oracle.c").write_text(src.replace(old, new))
    lib = str(tmp_path / "libidp_oracle_mutant.so")
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off", "-fopenmp", "-o", lib,
                    str(tmp_path / "idp_oracle.c"), "-lm"], check=True)
    env = dict(os.environ, IDP_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", *PINS], cwd=ROOT,
                       env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"no pin failed for {name}:\n{r.stdout[-2000:]}"


def test_unmodified_copy_passes_the_same_pins(tmp_path):
    """Control: the same procedure on the unmodified source passes, so the
    failures above come from the planted mistakes."""
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    shutil.copy(os.path.join(ROOT, "oracle", "idp_oracle.h"), tmp_path)
    shutil.copy(SRC, tmp_path / "idp_oracle.c")
    lib = str(tmp_path / "libidp_oracle_copy.so")
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off", "-fopenmp", "-o", lib,
                    str(tmp_path / "idp_oracle.c"), "-lm"], check=True)
    env = dict(os.environ, IDP_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider", *PINS], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:]
