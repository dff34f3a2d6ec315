"""The oracle pins must catch plausible mistakes.

Each case below plants one mistake in a copy of ``oracle/rdcnn_oracle.c``
(on the CPU, in a temporary directory), compiles it, and runs every pin of
``test_oracle_pins.py`` against the mutant.  At least one pin must fail.
The Python-side cases replace ``init_state`` (u = v = k_a x) on an oracle
object with a planted mistake in the same way.
"""
import inspect
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "rdcnn_oracle.c")

MUTANTS = {
    "cubic_over_2": ("(u * u * u) / 3.0", "(u * u * u) / 2.0"),
    "f1_plus_v": ("- (u * u * u) / 3.0 - v;", "- (u * u * u) / 3.0 + v;"),
    "quadratic_f1": ("p[P_C] * u - (u * u * u) / 3.0 - v", "u * (p[P_C] - u * p[P_EPS]) - v"),
    "f2_minus_a": ("p[P_B] * v + p[P_A]", "p[P_B] * v - p[P_A]"),
    "f2_sign": ("return -p[P_EPS] * (u", "return p[P_EPS] * (u"),
    "lap_centre_3": ("- 4.0 * f[i * nm + j]", "- 3.0 * f[i * nm + j]"),
    "lap_north_twice": ("im = neighbour_index(i - 1, nn, boundary)", "im = neighbour_index(i + 1, nn, boundary)"),
    "lap_no_col_wrap": ("jp = neighbour_index(j + 1, nm, boundary)", "jp = (j + 1 < nm ? j + 1 : j)"),
    "du_dv_swapped": ("uc + dt * (r1 + Du * lu)", "uc + dt * (r1 + Dv * lu)"),
    "gauss_seidel": ("r2 = reaction_f2(uc, vc, p);", "r2 = reaction_f2(uc + dt * r1, vc, p);"),
    "dt_squared": ("vn[c] = vc + dt * (r2", "vn[c] = vc + dt * dt * (r2"),
    "adj_jac_uu": ("ru = (c - uk * uk) * luk", "ru = (c - 3.0 * uk * uk) * luk"),
    "adj_eps_sign": ("- eps * lvk;", "+ eps * lvk;"),
    "adj_grad_b": ("g[3] += lvk * (eps * vk);", "g[3] += lvk * vk;"),
    "adj_grad_du_uses_v": ("g[0] += luk * laplacian_bc(u,", "g[0] += luk * laplacian_bc(v,"),
    "adj_dv_term": ("rv + Dv * laplacian_bc(lv", "rv + Du * laplacian_bc(lv"),
    "adj_zf_costate_on_torus": ("Du * laplacian_bc(lu, nn, nm, i, j, boundary)",
                                "Du * laplacian_bc(lu, nn, nm, i, j, ORACLE_PERIODIC)"),
    "adj_cenn_slope_ignored": ("lun[k] = luk + dt * (-luk + cenn_slope(uk) * back);",
                               "lun[k] = luk + dt * (-luk + back);"),
    "adj_cenn_no_leak": ("lun[k] = luk + dt * (-luk + cenn_slope(uk) * back);",
                         "lun[k] = luk + dt * (cenn_slope(uk) * back);"),
    "adj_cenn_offset_dropped": ("lvn[k] = lvk + dt * luk;", "lvn[k] = lvk;"),
    "adj_cenn_grad_c_state": ("g[5] += luk * cenn_output(uk);", "g[5] += luk * uk;"),
    "adj_zf_grad_on_torus": ("g[1] += lvk * laplacian_bc(v, nn, nm, i, j, boundary);",
                             "g[1] += lvk * laplacian_bc(v, nn, nm, i, j, ORACLE_PERIODIC);"),
    "zf_ghost_past_edge": ("return i < 0 ? 0 : (i > n - 1 ? n - 1 : i);", "return i < 0 ? 1 : (i > n - 1 ? n - 2 : i);"),
    "zf_ignored": ("if (boundary == ORACLE_ZEROFLUX) return i < 0", "if (0) return i < 0"),
    "zf_columns_wrap": ("jm = neighbour_index(j - 1, nm, boundary);\n    double vert = f", "jm = wrap_index(j - 1, nm);\n    double vert = f"),
    "cenn_output_halved": ("0.5 * (fabs(x + 1.0) - fabs(x - 1.0))", "0.25 * (fabs(x + 1.0) - fabs(x - 1.0))"),
    "cenn_arms_use_state": ("cenn_output(x[im * nm + j]) + cenn_output(x[ip * nm + j])", "x[im * nm + j] + x[ip * nm + j]"),
    "cenn_no_offset": ("((-uc + feedback) + vc)", "(-uc + feedback)"),
    "cenn_leak_sign": ("((-uc + feedback) + vc)", "((uc + feedback) + vc)"),
    "cenn_arm_missing": ("cenn_output(x[i * nm + jm]) + cenn_output(x[i * nm + jp])", "cenn_output(x[i * nm + jp])"),
}


def _pin_cases():
    cases = []
    for name, fn in inspect.getmembers(pins, inspect.isfunction):
        if not name.startswith("test_"):
            continue
        marks = getattr(fn, "pytestmark", [])
        params = [m for m in marks if m.name == "parametrize"]
        if not params:
            cases.append((fn, {}))
            continue
        argnames, values = params[0].args[0], params[0].args[1]
        names = [a.strip() for a in argnames.split(",")]
        for val in values:
            val = val if len(names) > 1 else (val,)
            cases.append((fn, dict(zip(names, val))))
    return cases


@pytest.fixture(scope="module")
def mutant_dir(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    return tmp_path_factory.mktemp("oracle_mutants")


# Mistakes planted in the Python side of the oracle (init_state, Eq. 1 first line):
# each replaces the function on an oracle object that otherwise uses the real C library.
def _init_v_unscaled(x, ka=1.0):
    x = np.asarray(x, dtype=np.float64)
    return ka * x, x.copy()


def _init_ka_squared(x, ka=1.0):
    x = np.asarray(x, dtype=np.float64)
    return ka * ka * x, ka * ka * x


def _init_ka_ignored(x, ka=1.0):
    x = np.asarray(x, dtype=np.float64)
    return x.copy(), x.copy()


def _init_shared_plane(x, ka=1.0):
    u = ka * np.asarray(x, dtype=np.float64)
    return u, u


PY_MUTANTS = {"init_v_unscaled": _init_v_unscaled, "init_ka_squared": _init_ka_squared,
              "init_ka_ignored": _init_ka_ignored, "init_shared_plane": _init_shared_plane}


def _caught_by_pins(bad):
    caught = []
    for fn, kwargs in _pin_cases():
        if "oracle_mod" not in inspect.signature(fn).parameters:
            continue
        try:
            fn(oracle_mod=bad, **kwargs)
        except (AssertionError, RuntimeError, ValueError):
            caught.append(fn.__name__)
    return caught


@pytest.mark.parametrize("mutant", sorted(PY_MUTANTS))
def test_pins_reject_python_mutant(mutant):
    bad = oracle.Oracle(oracle.build())
    bad.init_state = PY_MUTANTS[mutant]
    assert _caught_by_pins(bad), f"no pin caught mutant {mutant}"


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_pins_reject_mutant(mutant, mutant_dir):
    before, after = MUTANTS[mutant]
    text = open(SRC).read()
    assert text.count(before) >= 1, f"mutation site for {mutant} not found"
    src = mutant_dir / f"{mutant}.c"
    src.write_text(text.replace(before, after, 1))
    lib = str(mutant_dir / f"{mutant}.so")
    oracle.compile_source(str(src), lib)
    bad = oracle.Oracle(lib)
    assert _caught_by_pins(bad), f"no pin caught mutant {mutant}"
