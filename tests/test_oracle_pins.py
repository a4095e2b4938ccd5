"""The CPU oracle against its pins (brute force, the C++ standard library,
container invariants).  CPU only."""
import random

import numpy as np
import pytest

import oracle_pins as P
from oracle import oracle as O


def test_brute_force(oracle_lib):
    assert P.brute_force_pins(oracle_lib, seed=0, n_scripts=40) == []


def test_stl_equivalence(oracle_lib):
    if P.stl_binary() is None:
        pytest.skip("no C++ compiler")
    assert P.stl_pins(oracle_lib, seed=1) == []


def test_invariants(oracle_lib):
    assert P.invariant_pins(oracle_lib) == []


def test_edge_cases(oracle_lib):
    for kind in P.KINDS:
        t = O.OracleTable(kind, 1, oracle_lib)
        empty = P.key_array(kind, [])
        assert len(t.insert(empty, P.val_array(kind, []) if t.is_map else None)) == 0
        assert len(t.erase(empty)) == 0 and len(t.find(empty)[0]) == 0
        # capacity 1: all-equal batch -> one INSERTED, the rest EXISTS
        k = P.key_array(kind, [7] * 33)
        v = P.val_array(kind, list(range(33))) if t.is_map else None
        st = t.insert(k, v)
        assert st[0] == O.INSERTED and (st[1:] == O.EXISTS).all()
        f, fv = t.find(k[:1])
        assert f[0] == 1 and (not t.is_map or int(fv[0]) == 0)
        t.close()
    with pytest.raises(ValueError):
        O.OracleTable(O.SET_U32, 0, oracle_lib)


def test_hypothesis_scripts(oracle_lib):
    hyp = pytest.importorskip("hypothesis")
    st = hyp.strategies

    @hyp.settings(max_examples=150, deadline=None)
    @hyp.given(kind=st.sampled_from(P.KINDS), cap=st.integers(1, 12), seed=st.integers(0, 2**32 - 1))
    def prop(kind, cap, seed):
        rng = random.Random(seed)
        script = P.random_script(rng, kind, 20, P.tiny_domain(kind))
        assert P.check_against_brute_force(oracle_lib, kind, cap, script) == []

    prop()
