"""The oracle pins catch plausible mistakes.

Each case plants one mistake (a dropped term, a wrong sign, exponent, index
or factor) in a temporary copy of oracle.c, builds it, and runs the pin suite
against it with GCORECCD_ORACLE_LIB; the suite must fail.  Mistakes are
planted in the oracle only, on the CPU.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = {
    "mobility_exponent_sign": ("pow(T, -2.2)", "pow(T, 2.2)"),
    "mobility_beta_inverse": ("1.0 / beta);", "beta);"),
    "softening_power_1": ("double denom = r2 * sqrt(r2);", "double denom = r2;"),
    "field_sign": ("double rx = x[t] - x[j];", "double rx = x[j] - x[t];"),
    "dropped_z_term": ("rx * rx + ry * ry + rz * rz + eps2", "rx * rx + ry * ry + eps2"),
    "diffusion_factor_2": ("sqrt(2.0 * D * p->dt_s)", "sqrt(D * p->dt_s)"),
    "drift_units": ("double vx = 1e4 * mu * Ex, vy = 1e4 * mu * Ey, vz = 1e4 * mu * Ez;",
                    "double vx = 1e3 * mu * Ex, vy = 1e3 * mu * Ey, vz = 1e3 * mu * Ez;"),
    "static_field_sign": ("double Ez_static = p->a1 * z - p->a2;",
                          "double Ez_static = p->a2 - p->a1 * z;"),
    "philox_multiplier_swap": ("(uint64_t)0xD2511F53u * (uint64_t)x0", "(uint64_t)0xCD9E8D57u * (uint64_t)x0"),
    "philox_weyl": ("k1 += 0xBB67AE85u;", "k1 += 0x9E3779B9u;"),
    "box_muller_sin_cos": ("n[0] = radius * cos(2.0 * ORC_PI * ub);", "n[0] = radius * sin(2.0 * ORC_PI * ub);"),
    "normals_counter_order": ("uint32_t ctr[4] = {id, (uint32_t)step, (uint32_t)(step >> 32), 0u};",
                              "uint32_t ctr[4] = {(uint32_t)step, id, (uint32_t)(step >> 32), 0u};"),
    "pixel_round": ("double fx = floor(", "double fx = round("),
    "image_transposed": ("(e * p->img_h + iy) * p->img_w + ix", "(e * p->img_w + ix) * p->img_h + iy"),
    "reflection_clamp": ("zn = 2.0 * p->thickness_um - zn;", "zn = p->thickness_um;"),
    "coulomb_K_missing_4pi": ("(4.0 * ORC_PI * ORC_EPS0 * eps_rel)", "(ORC_EPS0 * eps_rel)"),
    "thermal_voltage_inverted": ("return ORC_KB * T / ORC_Q;", "return ORC_Q * T / ORC_KB;"),
    "stored_pixel_corner": ("double cx = origin[0] + ((double)ix + 0.5) * p->pixel_um;",
                            "double cx = origin[0] + ((double)ix) * p->pixel_um;"),
    "stored_charge_unweighted": ("sx += (double)q * (rx / denom);", "sx += (rx / denom);"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(os.path.join(ROOT, "oracle", "oracle.c")).read()
    assert src.count(old) >= 1, f"mutation site not found: {old}"
    (tmp_path / "oracle.c").write_text(src.replace(old, new, 1))
    shutil.copy(os.path.join(ROOT, "oracle", "oracle.h"), tmp_path / "oracle.h")
    lib = tmp_path / "liboracle_mutant.so"
    subprocess.run(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
                    str(tmp_path / "oracle.c"), "-o", str(lib), "-lm"], check=True)
    env = dict(os.environ, GCORECCD_ORACLE_LIB=str(lib), OMP_NUM_THREADS="4")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"pins did not catch mutant {name}:\n{r.stdout[-2000:]}"
