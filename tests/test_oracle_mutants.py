"""Plants plausible mistakes in a copy of the oracle, on the CPU, and checks
that the pins catch every one of them."""
import os
import subprocess
import sys
import tempfile

import pytest

import oracle_pins as P
from oracle import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

MUTANTS = [
    ("capacity off by one", "t->live_regular == t->capacity", "t->live_regular > t->capacity"),
    ("map insert overwrites value", "if (lookup(t, k) >= 0) return O_EXISTS;",
     "{ int64_t e_ = lookup(t, k); if (e_ >= 0) { t->nval[e_] = v; return O_EXISTS; } }"),
    ("reserved keys use capacity", "int reserved = is_reserved(t->kind, k);", "int reserved = 0;"),
    ("erase keeps size", "        t->live -= 1;\n", "        t->live -= 0;\n"),
    ("absent find value not zero", "nd >= 0 ? t->nval[nd] : 0", "nd >= 0 ? t->nval[nd] : 1"),
    ("rehash shrinks below live", "new_capacity < t->live_regular", "new_capacity < 0"),
    ("wrong u32 reserved pattern", "k == 0xFFFFFFFEull", "k == 0xFFFFFFFDull"),
    ("erase of absent key succeeds", "    return O_NOT_FOUND;\n}", "    return O_ERASED;\n}"),
    ("clear keeps regular count", "    t->live_regular = 0;\n}", "}"),
    ("int32 value truncated", "(int32_t)(uint32_t)v", "(int32_t)(uint16_t)v"),
    ("chain unlink skips node", "else t->nnext[prev] = t->nnext[n];", "else t->nnext[prev] = t->nnext[prev];"),
    ("find ignores found flag", "if (found) found[i] = (uint8_t)(nd >= 0);", "if (found) found[i] = 1;"),
    ("insert checks capacity before presence",
     "    if (lookup(t, k) >= 0) return O_EXISTS;          /* value left unchanged */\n    int reserved = is_reserved(t->kind, k);\n    if (!reserved && t->live_regular == t->capacity) return O_OVERFLOW;",
     "    int reserved = is_reserved(t->kind, k);\n    if (!reserved && t->live_regular == t->capacity) return O_OVERFLOW;\n    if (lookup(t, k) >= 0) return O_EXISTS;"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(name, old, new):
    src = open(O.SRC).read()
    assert src.count(old) == 1, f"mutation anchor not unique: {old!r}"
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "mut.c")
        open(path, "w").write(src.replace(old, new))
        so = O.build(path, os.path.join(d, "libmut.so"))
        # A mutant may corrupt a chain into a cycle; a run that does not end
        # within the limit counts as caught.
        code = ("import sys; sys.path[:0] = [%r, %r]; import oracle_pins as P; "
                "from oracle import oracle as O; "
                "sys.exit(1 if P.run_all_pins(O.load(%r)) else 0)") % (HERE, ROOT, so)
        try:
            r = subprocess.run([sys.executable, "-c", code], timeout=20, capture_output=True)
            caught = r.returncode != 0
        except subprocess.TimeoutExpired:
            caught = True
        assert caught, f"planted mistake not caught: {name}"


def test_unmutated_passes(oracle_lib):
    assert P.run_all_pins(oracle_lib) == []
