"""Mutation check of the oracle pins: plant one plausible mistake at a time in a
copy of the oracle's C source (on the CPU), build it, and require that the pin
suite catches it.  Each mutant is a slip the pins are meant to guard against."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "psolve_oracle.c")

MUTANTS = {
    "stencil_same_h_all_axes": ("- uh) / (h[d] * h[d]);", "- uh) / (h[0] * h[0]);"),
    "stencil_drops_upper_neighbour": ("acc += (-ul + 2.0 * uc - uh)", "acc += (-ul + 2.0 * uc)"),
    "stencil_wrong_centre_weight": ("acc += (-ul + 2.0 * uc - uh)", "acc += (-ul + 2.5 * uc - uh)"),
    "block_restriction_ignored": ("if (bs && (c[d] / bs[d]) != (home[d] / bs[d])) return 0.0;", ""),
    "eig_max_off_by_one": ("mu_dirichlet(n[d], n[d])", "mu_dirichlet(n[d] - 1, n[d])"),
    "eig_min_uses_h_once": ("lo += mu_dirichlet(1, n[d]) / (h[d] * h[d]);", "lo += mu_dirichlet(1, n[d]) / h[d];"),
    "cheb_wrong_rho_in_z_term": ("- rho_old * z[q]);", "- rho_cur * z[q]);"),
    "cheb_first_step_factor": ("y[q] = 2.0 * rho_cur / delta *", "y[q] = rho_cur / delta *"),
    "cheb_sign_in_residual": ("(rhs[q] - Av[q])", "(rhs[q] + Av[q])"),
    "cheb_theta_delta_swapped": ("const double sigma = theta / delta;", "const double sigma = delta / theta;"),
    "bicg_beta_missing_alpha_over_omega": ("(rho_new / rho) * (alpha / omega)", "(rho_new / rho)"),
    "bicg_omega_inverted": ("const double omega = ts / tt;", "const double omega = tt / ts;"),
    "bicg_x_update_drops_omega_term": ("x[q] = x[q] + alpha * ph[q] + omega * rh[q];",
                                       "x[q] = x[q] + alpha * ph[q];"),
    "bicg_p_update_sign": ("p[q] = r[q] + beta * (p[q] - omega * w[q]);",
                           "p[q] = r[q] + beta * (p[q] + omega * w[q]);"),
    "bicg_half_step_skips_x_update": ("x[q] = x[q] + alpha * ph[q];\n            snapshot(",
                                      "x[q] = x[q];\n            snapshot("),
    "bicg_alpha_uses_r_not_rtilde": ("const double sig1 = oracle_dot(N, rt, w);",
                                     "const double sig1 = oracle_dot(N, r, w);"),
    "dot2_drops_product_error": ("s = s + (q + r);", "s = s + q;"),
    "neumann_minus_face_reflects_to_itself": ("if (c[d] < 0 && bc && bc[2 * d] == 1) c[d] = home[d] + 1;",
                                              "if (c[d] < 0 && bc && bc[2 * d] == 1) c[d] = home[d];"),
    "neumann_plus_face_ignored": ("if (c[d] >= n[d] && bc && bc[2 * d + 1] == 1) c[d] = home[d] - 1;", ""),
    "mixed_spectrum_off_by_half": ("const double s1 = sin(pi / (4.0 * (double)m));",
                                   "const double s1 = sin(pi / (2.0 * (double)m));"),
    "bj_interval_skips_last_block": ("mu_range_1d(m, 0, fp, &mn2, &mx2); /* last block */",
                                     "mu_range_1d(m, 0, 0, &mn2, &mx2); /* last block */"),
    "bj_bicgs_blocks_lose_domain_faces": ("bbc[2 * d] = (B[d] == 0) ? pc->bc[2 * d] : 0;", "bbc[2 * d] = 0;"),
    "bj_bicgs_writes_block_back_shifted": ("out[(Bx * m[0] + i) + n[0] *", "out[(Bx * m[0] + (i + 1) % m[0]) + n[0] *"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique/present"
    mpath = tmp_path / "psolve_oracle.c"
    mpath.write_text(src.replace(old, new))
    lib = tmp_path / "liboracle_mutant.so"
    subprocess.run(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-I",
                    os.path.join(ROOT, "oracle"), "-o", str(lib), str(mpath), "-lm"], check=True)
    env = dict(os.environ, PSOLVE_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
