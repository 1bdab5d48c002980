"""Mutation check of the oracle's pins (CPU only).

Each case plants one plausible mistake in a copy of the oracle's C source (a
dropped term, a flipped sign, a transposed index, a wrong coefficient or grid
spacing), builds it with the oracle's own compiler flags and runs the pin
suite against the mutant.  The pins are fixed by the paper and the
mathematics, not by the oracle; a mistake that no pin catches would be a
hole in what pins the oracle.  The two self-consistency tests (point vs grid
residual, stage chain vs RK driver) and the stored fixture are left out, so
every mutant has to be caught by a closed form, an invariant, a symmetry or
brute force.
"""
import os
import re
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")
SELECT = "not golden and not point_and_grid and not stage_chain"

# name -> [(exact text in the source, replacement), ...]; every replacement
# is applied once, both where the grid residual and the point residual hold
# their own copy of the step.
MUTANTS = {
    # Eq. 6 / Eq. 7 stencils and the grid
    "d1_outer_weight": [("2.0 * fp1 / 3.0 - fp2 / 12.0) / h;", "2.0 * fp1 / 3.0 - fp2 / 6.0) / h;")],
    "d2_centre_weight": [("- 5.0 * f0 / 2.0", "- 7.0 * f0 / 3.0")],
    "d2_spacing_power": [("- fp2 / 12.0) / (h * h);", "- fp2 / 12.0) / h;")],
    "duplicated_end_point": [("/ (double)p->n[axis];", "/ (double)(p->n[axis] - 1);")],
    "periodic_wrap_off_by_one": [("return r < 0 ? r + n : r;", "return r < 0 ? r + n - 1 : r;")],
    # Eqs. 4-5
    "pressure_half": [("(s.rhoE - 0.5 * s.rho *", "(s.rhoE - 1.0 * s.rho *")],
    "temperature_mach": [("s.T = p->gamma * p->Mach * p->Mach * s.p / s.rho;",
                          "s.T = p->gamma * p->Mach * s.p / s.rho;")],
    # Eq. 1
    "mass_drop_u_drho": [("+ s->u[j] * L->d_rho[j];", ";")],
    # Eq. 2
    "momentum_flux_transposed": [("L->d_rhouu[i][j] + s->rhou[i]", "L->d_rhouu[j][i] + s->rhou[i]")],
    "momentum_flux_axis": [("orc_d1(p, rhouu + (size_t)(3 * i + j) * P, j,", "orc_d1(p, rhouu + (size_t)(3 * i + j) * P, i,"),
                           ("Q_RHOUU + 3 * a + b, b, i, j, k);", "Q_RHOUU + 3 * a + b, a, i, j, k);")],
    "pressure_gradient_sign": [("-0.5 * conv - L->d_p[i]", "-0.5 * conv + L->d_p[i]")],
    "stress_drop_dilatation": [("lap + cross - 2.0 / 3.0 * dil", "lap + cross")],
    "mixed_wrong_component": [("d_u + (size_t)(3 * j + j) * P, i, dd_u", "d_u + (size_t)(3 * i + j) * P, i, dd_u"),
                              ("point_mixed(p, q, Q_U0 + b, a, b, i, j, k)", "point_mixed(p, q, Q_U0 + a, a, b, i, j, k)")],
    # Eq. 3
    "energy_drop_u_drhoE": [("L->d_rhoEu[j] + s->rhoE * L->d_u[j][j] + s->u[j] * L->d_rhoE[j];",
                             "L->d_rhoEu[j] + s->rhoE * L->d_u[j][j];")],
    "energy_drop_pressure_work": [("pwork += L->d_pu[j];", "pwork += 0.0 * L->d_pu[j];")],
    "viscous_work_index": [("s->u[i] * inv_re * stress_div[i]", "s->u[i] * inv_re * stress_div[0]")],
    "dissipation_transposed": [("L->d_u[i][j] + L->d_u[j][i] -", "L->d_u[i][j] + L->d_u[i][j] -")],
    "conductivity_without_prandtl": [("p->Mach * p->Mach * p->Pr)", "p->Mach * p->Mach)")],
    "heat_flux_sign": [("+ kappa * heat;", "- kappa * heat;")],
    "dissipation_dilatation_coefficient": [("2.0 / 3.0 * div_u : 0.0", "1.0 / 3.0 * div_u : 0.0")],
    "viscous_work_sign": [("- pwork + vwork +", "- pwork - vwork +")],
    # Eq. 8 / Fig. 1 coefficients
    "rk_stage_a3": [("{2.0 / 3.0, 5.0 / 12.0, 3.0 / 5.0}", "{2.0 / 3.0, 5.0 / 12.0, 3.0 / 4.0}")],
    "rk_accumulator_b2": [("{1.0 / 4.0, 3.0 / 20.0, 3.0 / 5.0}", "{1.0 / 4.0, 3.0 / 10.0, 3.0 / 5.0}")],
    # §4 initial field and the diagnostics
    "tgv_pressure_amplitude": [("A * A / 16.0", "A * A / 8.0")],
    "tgv_density_mach": [("const double rho = g * M * M * pr;", "const double rho = g * M * pr;")],
    "tgv_internal_energy": [("pr / (g - 1.0) + 0.5 * rho", "pr / g + 0.5 * rho")],
    "ke_half": [("csum_add(&k_sum, 0.5 * rho *", "csum_add(&k_sum, rho *")],
    "ke_normalisation": [("*ke = (k_sum.s + k_sum.c) / (double)P;", "*ke = (k_sum.s + k_sum.c) / (double)(P - 1);")],
    "enstrophy_normalisation": [("*ens = (e_sum.s + e_sum.c) / (double)P;",
                                 "*ens = (e_sum.s + e_sum.c) / (double)(P + 1);")],
    "window_axes_swapped": [("wrap(origin[0] + a, p->n[0]), wrap(origin[1] + b, p->n[1])",
                             "wrap(origin[1] + a, p->n[0]), wrap(origin[0] + b, p->n[1])")],
    "vorticity_sign": [("du[(size_t)(3 * 2 + 1) * P + n] - du[(size_t)(3 * 1 + 2) * P + n]",
                        "du[(size_t)(3 * 2 + 1) * P + n] + du[(size_t)(3 * 1 + 2) * P + n]")],
}


def _compile(src_dir, name, out):
    base = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
            "-o", out, os.path.join(src_dir, name + ".c"), "-lm"]
    r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
    if r.returncode != 0:
        r = subprocess.run(base, capture_output=True, text=True)
    return r


def _run_pins(lib):
    # one thread each: several pin runs share the host, and spinning OpenMP or
    # BLAS pools oversubscribed across processes slow each other down by orders
    # of magnitude
    env = dict(os.environ, ORACLE_LIB=lib, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               OMP_WAIT_POLICY="passive")
    r = subprocess.run([sys.executable, "-m", "pytest", PINS, "-q", "-p", "no:cacheprovider", "-k", SELECT],
                       capture_output=True, text=True, env=env, cwd=ROOT, timeout=600)
    tail = r.stdout.strip().splitlines()[-1] if r.stdout.strip() else r.stderr[-300:]
    m = re.search(r"(\d+) failed", tail)
    return r.returncode, (int(m.group(1)) if m else 0), tail


@pytest.fixture(scope="module")
def sources():
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    with open(os.path.join(ORACLE, "sbli_oracle.c")) as f:
        return f.read()


def test_every_mutant_site_exists_once(sources):
    for name, edits in MUTANTS.items():
        for old, new in edits:
            assert sources.count(old) == 1, (name, old)
            assert old != new, name


def test_unmutated_copy_passes_the_pins(sources, tmp_path):
    shutil.copy(os.path.join(ORACLE, "sbli_oracle.h"), tmp_path)
    (tmp_path / "clean.c").write_text(sources)
    r = _compile(str(tmp_path), "clean", str(tmp_path / "clean.so"))
    assert r.returncode == 0, r.stderr
    rc, failed, tail = _run_pins(str(tmp_path / "clean.so"))
    assert rc == 0 and failed == 0, tail


def test_every_planted_mistake_fails_at_least_two_pins(sources, tmp_path):
    shutil.copy(os.path.join(ORACLE, "sbli_oracle.h"), tmp_path)
    for name, edits in MUTANTS.items():
        s = sources
        for old, new in edits:
            s = s.replace(old, new, 1)
        (tmp_path / (name + ".c")).write_text(s)

    def one(name):
        out = str(tmp_path / (name + ".so"))
        r = _compile(str(tmp_path), name, out)
        if r.returncode != 0:
            return name, None, "compile error: " + r.stderr[-300:]
        rc, failed, tail = _run_pins(out)
        return name, failed, tail

    workers = max(1, min(4, (os.cpu_count() or 2) // 2))
    with ThreadPoolExecutor(workers) as ex:
        results = list(ex.map(one, MUTANTS))
    weak = [(name, failed, tail) for name, failed, tail in results if failed is None or failed < 2]
    assert not weak, weak
