"""Pins of the oracle's successive randomized compression (Sec. II.C.1, Figs. random tensor and
src) against brute force on tiny systems: the local sketch of a leaf equals the dense product
H|x> contracted with the Khatri-Rao columns of Omega on every other site; with the sketch
dimension at the rank of the exact product the result is H|x> itself; the result is in canonical
form toward the root."""
import numpy as np
import pytest

from oracle import network as N, src as SRC
from paper_2512_15875_gb300 import inputs as I


def _nn_ham(tree, d, seed):
    """Harmonic terms plus q_i q_j couplings along the tree edges between modes (operator bond 3
    on an MPS) and a few on-site quartic terms."""
    L = int(tree.mode.max()) + 1
    rng = np.random.default_rng(seed)
    ham = I.Hamiltonian(dims=[d] * L, omega=rng.uniform(1.0, 2.0, L))
    for i in range(L):
        ham.add(ham.omega[i], {i: "h"})
        ham.add_monomial(rng.normal(0, 0.05), (i, i, i, i))
    for t in range(tree.n_nodes):
        p = int(tree.parent[t])
        if p >= 0 and tree.phys_dim[t] > 0 and tree.phys_dim[p] > 0:
            ham.add_monomial(rng.normal(0, 0.3), (int(tree.mode[t]), int(tree.mode[p])))
    return ham


def _rows(tree, bonds_out, i):
    r = max(int(tree.phys_dim[i]), 1)
    for c in tree.children(i):
        r *= int(bonds_out[c])
    return r


CASES = [
    ("mps6", lambda: I.mps_tree(6, 4), 4, 2),
    ("physbin7", lambda: I.all_physical_binary_tree(7, 3), 3, 2),
]


@pytest.mark.parametrize("name,mk,d,D", CASES, ids=[c[0] for c in CASES])
def test_src_is_exact_at_the_rank_of_the_product(name, mk, d, D):
    tree = mk()
    ham = _nn_ham(tree, d, 3)
    T = N.build_ttno(tree, ham)
    bonds = I.uniform_bonds(tree, D)
    x = [b[0] for b in I.random_block(tree, bonds, 1, seed=5)]
    chi = int(max(int(bonds[i]) * int(T.wbond[i]) for i in range(tree.n_nodes)
                  if tree.parent[i] >= 0))
    out_b = SRC.src_bonds(tree, chi)
    # the sketch and the QR are exercised: some node has more rows than chi
    assert any(_rows(tree, out_b, i) > chi for i in range(tree.n_nodes) if tree.parent[i] >= 0)
    y = SRC.src_apply(tree, T, x, I.src_sketch(tree, chi, seed=9), chi)
    ref = N.dense_hamiltonian(ham) @ N.ttns_to_dense(tree, x)
    assert np.abs(N.ttns_to_dense(tree, y) - ref).max() <= 1e-11 * np.abs(ref).max()
    for i in range(tree.n_nodes):
        if tree.parent[i] >= 0:
            assert y[i].shape[0] == out_b[i]


@pytest.mark.parametrize("name,mk,d,D", CASES, ids=[c[0] for c in CASES])
def test_src_sketch_of_a_leaf_is_the_dense_khatri_rao_sketch(name, mk, d, D):
    tree = mk()
    ham = _nn_ham(tree, d, 4)
    T = N.build_ttno(tree, ham)
    bonds = I.uniform_bonds(tree, D)
    x = [b[0] for b in I.random_block(tree, bonds, 1, seed=6)]
    chi = 5
    omega = I.src_sketch(tree, chi, seed=2)
    _, Ys = SRC.src_apply(tree, T, x, omega, chi, return_sketches=True)
    y = (N.dense_hamiltonian(ham) @ N.ttns_to_dense(tree, x)).reshape([d] * len(ham.dims))
    L = len(ham.dims)
    node_of_mode = tree.node_of_mode()
    leaf = N.postorder(tree)[0]
    m_leaf = int(tree.mode[leaf])
    args = [y, list(range(L))]
    for m in range(L):
        if m != m_leaf:
            args += [omega[node_of_mode[m]], [m, L]]       # c_k^(j)[p_j], column k shared
    ref = np.einsum(*args, [L, m_leaf])
    assert np.abs(Ys[leaf] - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("name,mk,d,D", CASES, ids=[c[0] for c in CASES])
def test_src_result_is_canonical_toward_the_root(name, mk, d, D):
    tree = mk()
    ham = _nn_ham(tree, d, 5)
    T = N.build_ttno(tree, ham)
    bonds = I.uniform_bonds(tree, D)
    x = [b[0] for b in I.random_block(tree, bonds, 1, seed=7)]
    chi = 4
    y = SRC.src_apply(tree, T, x, I.src_sketch(tree, chi, seed=3), chi)
    for i in range(tree.n_nodes):
        if tree.parent[i] >= 0:
            Q = N.with_phys(tree, i, y[i]).reshape(y[i].shape[0], -1)
            assert np.abs(Q @ Q.T - np.eye(Q.shape[0])).max() <= 1e-12
    # a truncated sketch is an approximation, not the product
    ref = N.dense_hamiltonian(ham) @ N.ttns_to_dense(tree, x)
    err = np.linalg.norm(N.ttns_to_dense(tree, y) - ref) / np.linalg.norm(ref)
    assert 1e-8 < err < 1.0
