"""Host-side checks of libttn that need no GPU: the shared library loads and exports every
entry point declared in include/ttn.h, and the TTNO builder (host C++) produces operators whose
contraction equals the dense Hamiltonian (checked with the oracle's dense contraction)."""
import os
import re

import numpy as np
import pytest

from oracle import network as N
from paper_2512_15875_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ttn():
    from paper_2512_15875_gb300 import build, ttn as T
    if not os.path.exists(T.LIB_PATH):
        build.build()
    T.load()
    return T


@pytest.fixture(scope="module")
def hctx(ttn):
    return ttn.ttn_create(device=-1)


def test_library_exports_every_declared_symbol(ttn):
    header = open(os.path.join(ROOT, "include", "ttn.h")).read()
    declared = set(re.findall(r"\b(ttn_[a-z0-9_]+)\s*\(", header))
    lib = ttn.load()
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert declared == set(ttn.exported_symbols())


def _lib_ttno_dense(ttn, hctx, tree, ham):
    th = ttn.ttn_tree_create(hctx, tree)
    H, bonds = ttn.ttn_build_ttno(hctx, th, ham.flat(tree))
    wb, ents = ttn.ttn_ttno_get_entries(H, tree.n_nodes)
    entries = [[] for _ in range(tree.n_nodes)]
    for node, w, c, op in ents:
        nl = len(N.legs(tree, node))
        entries[node].append((tuple(w[:nl]), op, c))
    T = N.TTNO(np.asarray(wb), entries)
    return N.ttno_to_dense(tree, T), bonds


TREES = [
    ("mps4", lambda d: I.mps_tree(4, d)),
    ("fork2x2", lambda d: I.fork_tree(2, 2, d)),
    ("leafbin2", lambda d: I.leaf_only_binary_tree(2, d)),
    ("physbin5", lambda d: I.all_physical_binary_tree(5, d)),
    ("physbin6", lambda d: I.all_physical_binary_tree(6, d)),
    ("ttree5", lambda d: I.t_tree(5, d)),
    ("fork3x1", lambda d: I.fork_tree(3, 1, d)),
]


@pytest.mark.parametrize("name,mk", TREES)
def test_built_ttno_equals_dense_hamiltonian(ttn, hctx, name, mk):
    tree = mk(3)
    L = int(tree.mode.max()) + 1
    rng = np.random.default_rng(len(name))
    ham = I.Hamiltonian(dims=[3] * L, omega=rng.uniform(1, 2, L))
    for i in range(L):
        ham.add(ham.omega[i], {i: "h"})
    for i in range(L):
        for j in range(i + 1, L):
            ham.add_monomial(rng.normal(0, 0.3), (i, j))
    for _ in range(3 * L):
        ham.add_monomial(rng.normal(0, 0.1), tuple(sorted(rng.integers(0, L, 3))))
        ham.add_monomial(rng.normal(0, 0.05), tuple(sorted(rng.integers(0, L, 4))))
    Hd = N.dense_hamiltonian(ham)
    Ht, bonds = _lib_ttno_dense(ttn, hctx, tree, ham)
    assert np.abs(Ht - Hd).max() <= 1e-12 * np.abs(Hd).max()
    naive = N.build_ttno(tree, ham)
    assert np.all(bonds <= naive.wbond)     # never worse than the uncompressed state diagram


def test_c1_built_ttno_equals_dense(ttn, hctx):
    w = I.make_workload("c1")
    Ht, _ = _lib_ttno_dense(ttn, hctx, w.tree, w.ham)
    Hd = N.dense_hamiltonian(w.ham)
    assert np.abs(Ht - Hd).max() <= 1e-12 * np.abs(Hd).max()


def test_uniform_bilinear_model_has_bond_three(ttn, hctx):
    # Sec. III.A: the 64-mode model with alpha_ij = 0.1 has an optimal TTNO of bond 3 on the MPS
    ham = I.uniform_coupled_model(64, d=2)
    tree = I.mps_tree(64, 2)
    th = ttn.ttn_tree_create(hctx, tree)
    _, bonds = ttn.ttn_build_ttno(hctx, th, ham.flat(tree))
    assert bonds[tree.parent >= 0].max() == 3


def test_uniform_bilinear_model_small_dense(ttn, hctx):
    ham = I.uniform_coupled_model(5, d=3)
    tree = I.mps_tree(5, 3)
    Ht, bonds = _lib_ttno_dense(ttn, hctx, tree, ham)
    assert bonds.max() == 3
    Hd = N.dense_hamiltonian(ham)
    assert np.abs(Ht - Hd).max() <= 1e-12 * np.abs(Hd).max()


def test_qff_bonds_are_reported(ttn, hctx):
    w = I.make_workload("c2")
    th = ttn.ttn_tree_create(hctx, w.tree)
    _, bonds = ttn.ttn_build_ttno(hctx, th, w.ham.flat(w.tree))
    naive = N.build_ttno(w.tree, w.ham)
    assert np.all(bonds <= naive.wbond)
    assert bonds.max() >= 3


def test_invalid_tree_is_rejected(ttn, hctx):
    class Bad:
        parent = np.array([-1, -1], dtype=np.int32)
        phys_dim = np.array([2, 2], dtype=np.int32)
    with pytest.raises(ttn.TTNError) as e:
        ttn.ttn_tree_create(hctx, Bad())
    assert e.value.status == 1


def test_host_only_context_refuses_device_blocks(ttn, hctx):
    tree = I.mps_tree(3, 2)
    th = ttn.ttn_tree_create(hctx, tree)
    with pytest.raises(ttn.TTNError):
        ttn.ttn_block_create(hctx, th, 2, I.uniform_bonds(tree, 2))


def _operator_schmidt_rank(H, dims, sub_modes):
    """Rank of the dense operator realigned as (operators on the subtree's modes) x (operators
    on the other modes): the smallest bond of any exact TTNO across that edge."""
    L = len(dims)
    T = H.reshape(list(dims) + list(dims))
    rest = [m for m in range(L) if m not in sub_modes]
    order = list(sub_modes) + [L + m for m in sub_modes] + rest + [L + m for m in rest]
    rows = int(np.prod([dims[m] ** 2 for m in sub_modes]))
    M = np.transpose(T, order).reshape(rows, -1)
    s = np.linalg.svd(M, compute_uv=False)
    return int(np.sum(s > 1e-10 * s[0]))


@pytest.mark.parametrize("name,mk", TREES[:4])
def test_rank_bound_is_the_operator_schmidt_rank(ttn, hctx, name, mk):
    tree = mk(3)
    rng = np.random.default_rng(11)
    L = int(tree.mode.max()) + 1
    ham = I.Hamiltonian(dims=[3] * L, omega=rng.uniform(1.0, 2.0, L))
    for i in range(L):
        ham.add(ham.omega[i], {i: "h"})
    for i in range(L):
        for j in range(i + 1, L):
            ham.add_monomial(rng.normal(0, 0.3), (i, j))
    for _ in range(L):
        ham.add_monomial(rng.normal(0, 0.1), tuple(sorted(rng.integers(0, L, 3))))
    th = ttn.ttn_tree_create(hctx, tree)
    H, bonds = ttn.ttn_build_ttno(hctx, th, ham.flat(tree))
    rk = ttn.ttn_ttno_rank_bounds(H, tree.n_nodes)
    Hd = N.dense_hamiltonian(ham)
    for c in range(tree.n_nodes):
        if tree.parent[c] < 0:
            continue
        sub = sorted(int(tree.mode[u]) for u in tree.subtree(c) if tree.mode[u] >= 0)
        assert rk[c] == _operator_schmidt_rank(Hd, ham.dims, sub), c
        assert bonds[c] >= rk[c]


def test_rank_bound_of_the_uniform_bilinear_model_is_three(ttn, hctx):
    # Sec. III.A: the uniformly coupled model has an exact TTNO of bond 3 on every MPS edge, and
    # no exact TTNO with a smaller bond exists
    ham = I.uniform_coupled_model(n_modes=16, d=4)
    tree = I.mps_tree(16, 4)
    th = ttn.ttn_tree_create(hctx, tree)
    H, bonds = ttn.ttn_build_ttno(hctx, th, ham.flat(tree))
    rk = ttn.ttn_ttno_rank_bounds(H, tree.n_nodes)
    assert list(rk[1:]) == [3] * 15 and list(bonds[1:]) == [3] * 15


@pytest.mark.parametrize("name", ["c2", "c3", "c4", "c5"])
def test_built_bond_reaches_the_rank_bound_on_the_workloads(ttn, hctx, name):
    # the merged state diagram with a minimum vertex cover per edge is optimal on these
    # Hamiltonians: every edge's bond equals the smallest bond an exact TTNO can have
    w = I.make_workload(name)
    th = ttn.ttn_tree_create(hctx, w.tree)
    H, bonds = ttn.ttn_build_ttno(hctx, th, w.ham.flat(w.tree))
    rk = ttn.ttn_ttno_rank_bounds(H, w.tree.n_nodes)
    for c in range(w.tree.n_nodes):
        if w.tree.parent[c] >= 0:
            assert 1 <= rk[c] == bonds[c], (c, rk[c], bonds[c])
