"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source (in a
temporary directory, on the CPU) and runs the pin tests of the update form
it touches (parallel, Eq. 6, or sequential, Eq. 5) against the copy: at
least one pin must fail.  The unmodified copy must pass.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = {
    # Eq. 1 sums over v = 0 too
    "drop_self_term": ("if (q < 0) continue;", "if (q < 0 || centre) continue;"),
    # Eq. 3 weights each merged centroid by its count
    "unweighted_merge": (
        "for (int a = 0; a < d; a++) xacc_add(&acc[a], sp[j * d + a], cc[j]);\n        parent[j] = m2;",
        "for (int a = 0; a < d; a++) xacc_add(&acc[a], sp[j * d + a], 1u);\n        parent[j] = m2;"),
    # floor, not truncation toward zero
    "truncating_floor": ("int64_t gso_floor_div(double x, double h) {\n  double q = floor(x / h);",
                         "int64_t gso_floor_div(double x, double h) {\n  double q = trunc(x / h); return (int64_t)q;"),
    # the neighbourhood is {-1,0,1}^d
    "half_neighbourhood": ("int off = (int)(rest % 3) - 1;", "int off = (int)(rest % 2) - 1;"),
    # the stop test comes before the update is applied
    "stop_after_apply": ("if (!any_nb) { converged = 1; break; }",
                         "if (!any_nb && t > 0) { converged = 1; break; }"),
    # probes follow the cell's own axes
    "wrong_axis": ("probe[a] = ck[j * d + a] + off;", "probe[a] = ck[j * d + (d - 1 - a)] + off;"),
    # round to nearest, ties to even
    "no_ties_to_even": ("if (guard && (sticky || (sig & 1))) sig += 1;", "if (guard) sig += 1;"),
    # clusters numbered by ascending key
    "descending_labels": ("    if (a[i] < b[i]) return -1;\n    if (a[i] > b[i]) return 1;",
                          "    if (a[i] < b[i]) return 1;\n    if (a[i] > b[i]) return -1;"),
    # max_iter counts applied updates
    "step_limit_off_by_one": ("if (t == max_iter) break;", "if (t > max_iter) break;"),
    # tracking window step (Algorithm 2): R's position sums, extent, membership
    "track_sum_y_of_x": ("      sy += y;", "      sy += x;"),
    "track_min_x_as_max": ("if (x < mnx) mnx = x;", "if (x > mnx) mnx = x;"),
    "track_first_bin_always": ("        if (same) {", "        if (same || j == 0) {"),
    # the mode divides the sum by the count
    "mode_off_by_one_count": ("modes[c * d + a] = cs[c * d + a] / (double)cc[c];",
                              "modes[c * d + a] = cs[c * d + a] / (double)(cc[c] + 1);"),
}

# Mistakes in the sequential update (Sec. 2.2, Eq. 5), caught by its own pins
SEQ_MUTANTS = {
    # a neighbour updated earlier in the sweep is read at its new centroid
    "sequential_reads_old_state": (
        "if (done[q]) xacc_add(&acc[a], sp[q * d + a], cc[q]);",
        "if (0 && done[q]) xacc_add(&acc[a], sp[q * d + a], cc[q]);"),
    # ... weighted by its count
    "updated_neighbour_unweighted": ("sp[q * d + a], cc[q]);", "sp[q * d + a], 1u);"),
    # the colour's most significant bit is axis 0
    "colour_axes_reversed": ("for (int a = 0; a < d; a++) c = 2 * c + (k[a] % 2 != 0);",
                             "for (int a = d - 1; a >= 0; a--) c = 2 * c + (k[a] % 2 != 0);"),
    # negative odd keys are odd
    "negative_parity": ("c = 2 * c + (k[a] % 2 != 0);", "c = 2 * c + (k[a] % 2 == 1);"),
    # the sweep goes by colour, not by key alone
    "sweep_in_key_order": ("if (key_colour(ck + j * d, d) == col) sweep[ns++] = j;",
                           "if (col == 0) sweep[ns++] = j;"),
    # colours ascending
    "colours_descending": ("for (int64_t col = 0; col < ncol; col++)",
                           "for (int64_t col = ncol - 1; col >= 0; col--)"),
}

PIN_FILES = {"parallel": "tests/test_oracle_pins.py",
             "sequential": "tests/test_oracle_sequential.py"}


def _copy_tree(dst):
    ign = shutil.ignore_patterns("_build", "__pycache__", "*.so")
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(dst, "oracle"), ignore=ign)
    shutil.copytree(os.path.join(ROOT, "tests"), os.path.join(dst, "tests"), ignore=ign)


def _run_pins(dst, *files):
    return subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                           *files], cwd=dst, capture_output=True, text=True, timeout=600)


def test_unmodified_copy_passes(tmp_path):
    _copy_tree(str(tmp_path))
    r = _run_pins(str(tmp_path), *PIN_FILES.values())
    assert r.returncode == 0, r.stdout[-2000:]


_ALL = sorted([(n, "parallel") for n in MUTANTS] + [(n, "sequential") for n in SEQ_MUTANTS])


@pytest.mark.parametrize("name,form", _ALL, ids=[n for n, _ in _ALL])
def test_planted_mistake_is_caught(tmp_path, name, form):
    old, new = (MUTANTS if form == "parallel" else SEQ_MUTANTS)[name]
    _copy_tree(str(tmp_path))
    src = os.path.join(str(tmp_path), "oracle", "gs_oracle.c")
    text = open(src).read()
    assert text.count(old) == 1, f"mutation site for {name} not found once"
    open(src, "w").write(text.replace(old, new))
    r = _run_pins(str(tmp_path), PIN_FILES[form])
    assert r.returncode != 0, f"no pin caught the mutant {name}:\n{r.stdout[-1500:]}"
