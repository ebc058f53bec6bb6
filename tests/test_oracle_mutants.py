"""The oracle's pins must catch plausible mistakes. Each case plants one mistake in a copy
of the oracle source (on the CPU), builds it, and runs the pin suite against it through
STC_ORACLE_LIB; the suite has to fail."""
import os
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "stc_oracle.cpp")

MUTANTS = {
    "dropped_accumulation": ("acc.sum += p;", "acc.sum = p;"),
    "wrong_sign": ("acc.sum += p;", "acc.sum -= p;"),
    "x_keyed_by_y_modes": ("c[k] = X.at(i, cx[k]);\n    auto hit", "c[k] = X.at(i, cy[k]);\n    auto hit"),
    "reversed_pairing": ("for (int32_t k = 0; k < m; k++) c[k] = Y.at(j, cy[k]);\n    y_by_contract",
                         "for (int32_t k = 0; k < m; k++) c[k] = Y.at(j, cy[m - 1 - k]);\n    y_by_contract"),
    "y_free_before_x_free": ("cat[xfree.size() + b] = Y.at(j, yfree[b]);", "cat[b] = Y.at(j, yfree[b]);"),
    "x_value_squared": ("const double p = xv[i] * yv[j];", "const double p = xv[i] * xv[i];"),
    "out_order_inverted": ("zc[q] = out_order ? cat[out_order[q]] : cat[q];",
                           "zc[out_order ? out_order[q] : q] = cat[q];"),
    "ln_key_little_endian": ("key = key * (unsigned __int128)shape[modes[t]] + (unsigned __int128)c;",
                             "key = key + (unsigned __int128)c * (unsigned __int128)(t ? shape[modes[t - 1]] : 1);"),
    "counting_sort_forward_walk": ("for (int64_t i = n - 1; i >= 0; i--) {", "for (int64_t i = 0; i < n; i++) {"),
    "first_seen_off_by_one": ("const int64_t id = (int64_t)table.size();", "const int64_t id = (int64_t)table.size() + 1;"),
    "bound_counts_entries": ("g.first += w;", "g.first += 1;"),
    "slots_rounded_up": ("return (uint64_t)std::floor(1.3 * (double)bound);", "return (uint64_t)std::ceil(1.3 * (double)bound);"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique or missing"
    mut = tmp_path / "mutant.cpp"
    mut.write_text(src.replace(old, new))
    lib = oracle.compile_source(str(mut), str(tmp_path / "libmutant.so"))
    env = dict(os.environ, STC_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode != 0, f"mutant {name} passed every pin:\n{r.stdout[-2000:]}"
