"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a copy of oracle/das_oracle.c (on the CPU,
in a temporary directory), builds it, and runs tests/test_oracle_pins.py
against that build: at least one pin must fail.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "das_oracle.c")

MUTANTS = {
    "transmit_time_zero_dropped": ("if (P->t0_offset) path -= dist3(v, P->t0_ref);", ""),
    "phase_sign_flipped": ("acc[2 * b + 1] += w * (sr * sph + si * cph);",
                           "acc[2 * b + 1] += w * (-sr * sph + si * cph);"),
    "interpolation_taps_swapped": ("double sr = (1.0 - alpha) * r0 + alpha * r1;",
                                   "double sr = alpha * r0 + (1.0 - alpha) * r1;"),
    "f_number_half_width_wrong": ("double half_width = z / (2.0 * P->f_number);",
                                  "double half_width = z / (P->f_number);"),
    "sample_range_off_by_one": ("kf > (double)(P->K - 2)", "kf > (double)(P->K - 1)"),
    "voxel_order_z_fastest": ("long ix = n % P->nx;\n    long iy = (n / P->nx) % P->ny;\n    long iz = n / ((long)P->nx * P->ny);",
                              "long iz = n % P->nz;\n    long iy = (n / P->nz) % P->ny;\n    long ix = n / ((long)P->nz * P->ny);"),
    "adjoint_without_conjugate": ("double cr = w * cos(ph), ci = -w * sin(ph);",
                                  "double cr = w * cos(ph), ci = w * sin(ph);"),
    "adjoint_taps_swapped": ("y[2 * (row + k)] += (1.0 - alpha) * vr;", "y[2 * (row + k)] += alpha * vr;"),
    "grad_sign_flipped": ("double dts = -ts / P->c;", "double dts = ts / P->c;"),
    "grad_phase_term_dropped": ("double gr = (r1 - r0) - theta * si;", "double gr = (r1 - r0);"),
    "sampling_rate_scaled": ("double ts = tau * P->fs; ", "double ts = tau * P->fs * 1.0001; "),
    "aperture_margin_inverted": ("(1.0 + APERTURE_MARGIN) * half_width", "(1.0 - APERTURE_MARGIN) * half_width"),
    "transmit_weight_transposed": ("P->w_tx[(long)q * n_voxels(P) + n]", "P->w_tx[(long)n * P->Q + q]"),
    "plane_wave_sign_flipped": ("return (v[0] * (p[0] - P->t0_ref[0])", "return -(v[0] * (p[0] - P->t0_ref[0])"),
    "count_active_first_transmit_only": ("        for (int q = 0; q < P->Q; ++q)\n            for (int m",
                                         "        for (int q = 0; q < 1; ++q)\n            for (int m"),
    "count_active_drops_first_element": ("if (term(P, q, m, n, p, &k, &alpha, &ts, &w)) ++count;",
                                         "if (term(P, q, m, n, p, &k, &alpha, &ts, &w) && m > 0) ++count;"),
    "near_ties_count_exact_ties": ("if (d > 1e-9 * thr && d <= rel * thr) ++count;", "if (d <= rel * thr) ++count;"),
    "near_ties_half_width_wrong": ("double hw = z / (2.0 * P->f_number);", "double hw = z / (P->f_number);"),
}


@pytest.mark.parametrize("name", list(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    src = open(SRC).read()
    old, new = MUTANTS[name]
    assert old in src, "mutation site moved: " + name
    (tmp_path / "das_oracle.c").write_text(src.replace(old, new, 1))
    (tmp_path / "das_oracle.h").write_text(open(os.path.join(ROOT, "oracle", "das_oracle.h")).read())
    lib = tmp_path / "liboracle_mutant.so"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-D_DEFAULT_SOURCE",
                           "-o", str(lib), str(tmp_path / "das_oracle.c"), "-lm"])
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        "-q", "-x", "-p", "no:cacheprovider"], cwd=ROOT,
                       env=dict(os.environ, DAS_ORACLE_LIB=str(lib)), capture_output=True, text=True)
    assert r.returncode == 1, f"no pin failed for mutant {name}:\n{r.stdout[-2000:]}"
