"""The FP64 oracle against facts the problem fixes: hand-worked examples, closed
forms, exact brute force, a library routine and invariants. Planted mistakes in
copies of the oracle must each fail at least one of these pins."""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
import pins


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda p: p.__name__)
def test_pin(pin, oracle_lib):
    pin(oracle_lib)


# (description, original text, replacement) -- each mutant must be caught
MUTANTS = [
    ("sign of the difference flipped", "(double)x[t] - (double)y[t]", "(double)x[t] + (double)y[t]"),
    ("last coordinate dropped", "t < d; ++t", "t < d - 1; ++t"),
    ("absolute difference instead of square", "s += diff * diff;", "s += diff < 0 ? -diff : diff;"),
    ("ties to the higher index", "if (x->j < y->j) return -1;\n    if (x->j > y->j) return 1;",
     "if (x->j < y->j) return 1;\n    if (x->j > y->j) return -1;"),
    ("self not excluded", "if (exclude_self && j == i) continue;", "if (0) continue;"),
    ("corpus row indexed by the query", "C + (size_t)j * (size_t)d", "C + (size_t)i * (size_t)d"),
    ("query row indexed by output slot", "Q + (size_t)i * (size_t)d", "Q + (size_t)r * (size_t)d"),
    ("descending order", "if (x->d < y->d) return -1;\n    if (x->d > y->d) return 1;",
     "if (x->d < y->d) return 1;\n    if (x->d > y->d) return -1;"),
    ("output shifted by one", "out_idx[r * k + t] = t < n ? pairs[t].j", "out_idx[r * k + t] = t + 1 < n ? pairs[t + 1].j"),
    ("single-precision accumulation", "double s = 0.0;", "float s = 0.0f;"),
    ("similarity: mean added instead of subtracted", "double c = (double)x[t] - m;", "double c = (double)x[t] + m;"),
    ("similarity: centring skipped in the dot product", "((double)x[t] - mx) * ((double)y[t] - my)",
     "((double)x[t]) * ((double)y[t])"),
    ("similarity: mean not divided by d", "m /= (double)d;", "m /= 1.0;"),
    ("similarity: squared norms instead of norms", "*norm = sqrt(ss);", "*norm = ss;"),
    ("similarity: ascending order", "pairs[n].d = -sim_pair(", "pairs[n].d = sim_pair("),
    ("similarity: self not excluded", "                if (exclude_self && j == i) continue;\n                /*",
     "                if (0) continue;\n                /*"),
    ("similarity: query norm dropped", "return dot / (nx * ny);", "return dot / ny;"),
    ("similarity: corpus statistics of the wrong row", "C + (size_t)j * (size_t)d, cm[j], cn[j], d)",
     "C + (size_t)j * (size_t)d, cm[0], cn[0], d)"),
]


@pytest.mark.parametrize("desc,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(desc, old, new, tmp_path):
    src = open(oracle._SRC).read()
    assert old in src, f"mutation anchor missing: {old!r}"
    mutant = tmp_path / "mutant.c"
    mutant.write_text(src.replace(old, new, 1))
    lib_path = str(tmp_path / "libmutant.so")
    oracle.build(force=True, src=str(mutant), out=lib_path)
    lib = oracle.load(lib_path)
    failed = pins.failing_pins(lib)
    assert failed, f"no pin caught the planted mistake: {desc}"


def test_oracle_threads():
    assert oracle.threads() >= 1
