"""Planted mistakes in the oracle are caught by its pins.

Each case copies ``oracle/`` to a temporary directory, plants one plausible
mistake in its C source, builds the copy and runs the compact pin set of
``tests/oracle_checks.py`` on it in a child process: at least one check must
fail (or the copy must crash).  The unmodified copy must pass them all.  The
mistakes cover the vertex order, the filtration order, the id tables, the
boundary, the pivot, the zero-persistence filter, both union-find special
cases, the sandwich's steps and the fast-mode reduction (clearing, the
streamed order, implicit boundaries, the key packing, infinite classes).
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, file, exact text, replacement); the text occurs once in the file
MUTANTS = [
    ("ties broken against the vertex id", "complex.h",
     "if (x->id != y->id) return x->id < y->id ? -1 : 1;",
     "if (x->id != y->id) return x->id < y->id ? 1 : -1;"),
    ("negative floats not flipped", "complex.h",
     "u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);",
     "u = u | 0x80000000u;"),
    ("a coface before its face", "complex.h",
     "if (x->dim != y->dim) return x->dim < y->dim ? -1 : 1;",
     "if (x->dim != y->dim) return x->dim < y->dim ? 1 : -1;"),
    ("two triangle chains swapped in the id table", "complex.h",
     "static const int TRI_A[12] = {1, 2, 1, 4, 2, 4, 1, 2, 3, 4, 5, 6};",
     "static const int TRI_A[12] = {2, 1, 1, 4, 2, 4, 1, 2, 3, 4, 5, 6};"),
    ("a boundary without its last facet", "pairsimplices.c",
     "for (int drop = 0; drop <= dim; drop++) {",
     "for (int drop = 0; drop < dim; drop++) {"),
    ("the lowest row taken as the pivot", "pairsimplices.c",
     "int64_t low = R[j].e[R[j].n - 1];\n            if (owner[low] < 0) break;",
     "int64_t low = R[j].e[0];\n            if (owner[low] < 0) break;"),
    ("zero-persistence filter inverted", "pairsimplices.c",
     "if (dmax == bmax && !keep_zero) continue;",
     "if (dmax != bmax && !keep_zero) continue;"),
    ("D0 union-find keeps the younger minimum", "pairsimplices.c",
     "int64_t young = a > b ? a : b, old = a > b ? b : a;",
     "int64_t young = a > b ? b : a, old = a > b ? a : b;"),
    ("D2 union-find keeps the younger maximum", "pairsimplices.c",
     "int64_t young = a < b ? a : b, old = a < b ? b : a;",
     "int64_t young = a < b ? b : a, old = a < b ? a : b;"),
    ("sandwich: the lowest edge taken as the top", "sandwich.c",
     "tau = B.e[B.n - 1];", "tau = B.e[0];"),
    ("sandwich: the vertex paired with its highest edge", "sandwich.c",
     "for (int64_t q = lo + 1; q < hi && delta < 0; q++) if (w->s[q].dim == 1) delta = q;",
     "for (int64_t q = lo + 1; q < hi; q++) if (w->s[q].dim == 1) delta = q;"),
    ("sandwich: ascent without the gradient step", "sandwich.c",
     "        if (t < 0) return q;\n        int64_t a = w->side[2 * t]",
     "        return q;\n        int64_t a = w->side[2 * t]"),
    ("sandwich: one descent end repeated", "sandwich.c",
     "b = descend(w, w->facet[4 * e + 1]);", "b = descend(w, w->facet[4 * e]);"),
    ("sandwich: the option ignored", "sandwich.c",
     "if (!virtual_max && (end[0] == m || end[1] == m)) continue;", "if (0) continue;"),
    ("sandwich: infinite maxima dropped", "sandwich.c",
     "if (w->grad[p] >= 0 || partner[p] >= 0) continue;",
     "if (w->grad[p] >= 0 || partner[p] >= 0 || w->s[p].dim == 3) continue;"),
    ("fast mode: clearing inverted", "fastpairs.c",
     "if (cleared && cleared[tau] >= 0) continue;",
     "if (cleared && cleared[tau] < 0) continue;"),
    ("fast mode: a lower star visited in decreasing order", "fastpairs.c",
     "for (int j = i; j > 0 && key_lt(keys[j], keys[j - 1]); j--) {",
     "for (int j = i; j > 0 && key_lt(keys[j - 1], keys[j]); j--) {"),
    ("fast mode: a boundary without its last facet", "fastpairs.c",
     "for (int drop = 0; drop <= dim; drop++) {",
     "for (int drop = 0; drop < dim; drop++) {"),
    ("fast mode: a coface before its face", "fastpairs.c",
     "k.lo = ((uint64_t)(r[2] + 1) << 32) | (uint64_t)(r[3] + 1);",
     "k.lo = ((uint64_t)(r[2]) << 32) | (uint64_t)(r[3]);"),
    ("fast mode: zero-persistence filter inverted", "fastpairs.c",
     "if (bmax == dmax && !keep_zero) continue;",
     "if (bmax != dmax && !keep_zero) continue;"),
    ("fast mode: births reported as infinite", "fastpairs.c",
     "int birth = dim < 3 && owner[dim + 1][id] >= 0;",
     "int birth = 0;"),
    ("fast mode: dimensions reduced upward, clearing from pivots not yet found", "fastpairs.c",
     "for (int d = 3; d >= 1 && !st; d--)",
     "for (int d = 1; d <= 3 && !st; d++)"),
]


def _copy(dst):
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(dst, "oracle"),
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))


def _run(directory):
    return subprocess.run([sys.executable, "-m", "tests.oracle_checks", str(directory)],
                          cwd=ROOT, capture_output=True, text=True, timeout=600)


def test_unmodified_copy_passes(tmp_path):
    _copy(tmp_path)
    r = _run(tmp_path)
    assert r.returncode == 0, r.stdout + r.stderr


@pytest.mark.parametrize("name,fname,text,repl", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(tmp_path, name, fname, text, repl):
    _copy(tmp_path)
    path = os.path.join(tmp_path, "oracle", fname)
    src = open(path).read()
    assert src.count(text) == 1, "the planted text must occur once"
    with open(path, "w") as f:
        f.write(src.replace(text, repl))
    r = _run(tmp_path)
    assert r.returncode != 0, f"not caught: {name}"
