"""Golden fixtures: the paper's printed structural facts (tests/golden/paper_facts.txt, each with
its citation) and the stored dense-ED spectrum of the 4-mode workload (written by
tests/golden/make_golden.py from the oracle only)."""
import os

import numpy as np

from oracle import network as N
from paper_2512_15875_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def facts():
    out = {}
    for line in open(os.path.join(GOLDEN, "paper_facts.txt")):
        if line.startswith("#") or not line.strip():
            continue
        key, val, _ = line.split(" ", 2)
        out[key] = int(val)
    return out


def test_generators_match_the_printed_term_counts():
    f = facts()
    assert len(I.uniform_coupled_model(64, d=2).terms) == f["uniform64_terms"]
    h = I.quartic_force_field(0)
    assert h.n_modes == f["qff12_modes"]
    assert len(h.terms) == f["qff12_terms"]
    orders = [sum({"h": 0, "q": 1, "q2": 2, "q3": 3, "q4": 4}[k] for k in
                  [kind for (m, kind), oid in h._op_index.items() if oid in ids])
              for _, ids in h.terms]
    assert orders.count(0) == f["qff12_harmonic_terms"]
    assert orders.count(3) == f["qff12_cubic_terms"]
    assert orders.count(4) == f["qff12_quartic_terms"]


def test_fork4_tree_matches_the_printed_topology():
    f = facts()
    t = I.fork_tree(4, 3, 9)
    aux = [i for i in range(t.n_nodes) if t.phys_dim[i] == 0]
    assert len(aux) == f["fork4_backbone_nodes"]
    for b in aux:
        chain = [c for c in t.children(b) if t.phys_dim[c] > 0]
        assert len(chain) == 1
        n, u = 0, chain[0]
        while True:
            n += 1
            ch = t.children(u)
            if not ch:
                break
            u = ch[0]
        assert n == f["fork4_chain_length"]


def test_uniform_model_bond_three_from_the_golden_fact():
    import pytest
    try:
        from paper_2512_15875_gb300 import ttn as T
        T.load()
    except Exception as e:  # library not built in this environment
        pytest.skip(str(e))
    f = facts()
    ctx = T.ttn_create(-1)
    tree = I.mps_tree(64, 2)
    th = T.ttn_tree_create(ctx, tree)
    _, bonds = T.ttn_build_ttno(ctx, th, I.uniform_coupled_model(64, d=2).flat(tree))
    assert bonds.max() == f["uniform64_ttno_max_bond"]


def test_stored_c1_spectrum_is_reproduced_by_the_oracle():
    stored = np.loadtxt(os.path.join(GOLDEN, "c1_ed.txt"))
    w = I.make_workload("c1", seed=0)
    ev = np.linalg.eigvalsh(N.dense_hamiltonian(w.ham))[:len(stored)]
    assert np.allclose(ev, stored, rtol=1e-12, atol=0)
