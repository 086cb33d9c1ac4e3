"""Successive randomized compression (Sec. II.C.1) on the GPU against the FP64 oracle, with the
same seeded sketch matrices Omega^(i) on both sides: node tensors of the result element by
element (both sides orthogonalise with R's diagonal non-negative), on small trees with the
sketch truncating and at the rank of the exact product (where the result is H|x>), and on the
12-mode QFF at D = 24 with chi = 24. The local sketches do not depend on the TTNO's bond basis,
so the library's own TTNO is compared with the oracle's state-diagram TTNO."""
import numpy as np
import pytest

from oracle import network as N, src as SRC
from paper_2512_15875_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 5e-5, "tf32x3": 5e-5}


@pytest.fixture(scope="module")
def T():
    from paper_2512_15875_gb300 import ttn
    ttn.load()
    return ttn


@pytest.fixture(scope="module")
def ctx(T):
    return T.ttn_create(0)


def _ham(tree, d, seed):
    L = int(tree.mode.max()) + 1
    rng = np.random.default_rng(seed)
    ham = I.Hamiltonian(dims=[d] * L, omega=rng.uniform(1.0, 2.0, L))
    for i in range(L):
        ham.add(ham.omega[i], {i: "h"})
    for i in range(L):
        for j in range(i + 1, L):
            ham.add_monomial(rng.normal(0, 0.3), (i, j))
    for _ in range(L):
        ham.add_monomial(rng.normal(0, 0.1), tuple(sorted(rng.integers(0, L, 3))))
    return ham


CASES = [
    ("mps6", lambda: I.mps_tree(6, 4), 4, 3),
    ("fork2x2", lambda: I.fork_tree(2, 2, 3), 3, 3),
    ("leafbin2", lambda: I.leaf_only_binary_tree(2, 3), 3, 3),
    ("physbin7", lambda: I.all_physical_binary_tree(7, 3), 3, 3),
]


def _run(T, ctx, tree, ham, bonds, n, chi, prec, seed, scale=1.0):
    th = T.ttn_tree_create(ctx, tree)
    H, _ = T.ttn_build_ttno(ctx, th, ham.flat(tree))
    blk = I.random_block(tree, bonds, n, seed=seed, scale=scale)
    bx = T.block_from_arrays(ctx, th, bonds, blk)
    omega = I.src_sketch(tree, chi, seed=seed + 1)
    by = T.ttn_src_apply(ctx, H, bx, chi, omega, prec=prec)
    ob = SRC.src_bonds(tree, chi)
    got = [T.ttn_block_get(by, -1, t).reshape((n,) + I.node_shape(tree, ob, t))
           for t in range(tree.n_nodes)]
    otn = N.build_ttno(tree, ham)
    ref = [SRC.src_apply(tree, otn, [b[s] for b in blk], omega, chi) for s in range(n)]
    return blk, got, ref


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_src_matches_the_oracle_when_the_sketch_truncates(T, ctx, case, prec):
    # chi = 4 is below the rank of every local sketch, so each QR factor is unique (R's
    # diagonal non-negative) and the node tensors compare element by element
    name, mk, d, D = case
    tree = mk()
    ham = _ham(tree, d, 21)
    bonds = I.uniform_bonds(tree, D)
    blk, got, ref = _run(T, ctx, tree, ham, bonds, 3, 4, prec, seed=31)
    for s in range(3):
        for t in range(tree.n_nodes):
            r = ref[s][t]
            assert np.abs(got[t][s] - r).max() <= TOL[prec] * max(np.abs(r).max(), 1.0), (s, t)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_src_is_the_exact_product_at_full_sketch(T, ctx, case, prec):
    # chi = 40 reaches the rank of the exact product on every edge: the result is H|x> (the
    # trailing QR columns of rank-deficient sketches are arbitrary, so only the state compares)
    name, mk, d, D = case
    tree = mk()
    ham = _ham(tree, d, 21)
    bonds = I.uniform_bonds(tree, D)
    blk, got, ref = _run(T, ctx, tree, ham, bonds, 3, 40, prec, seed=31)
    Hd = N.dense_hamiltonian(ham)
    for s in range(3):
        y = N.ttns_to_dense(tree, [g[s] for g in got])
        hx = Hd @ N.ttns_to_dense(tree, [b[s] for b in blk])
        assert np.abs(y - hx).max() <= {"fp64": 1e-10, "fp32": 2e-5}[prec] * np.abs(hx).max()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_src_on_the_twelve_mode_qff(T, ctx, prec):
    # full size (fork-4, D = 24, chi = 24): node tensors element by element (float32 errors
    # grow with the conditioning of the local sketches), and the gauge-free <y|y> and <x|y>
    w = I.make_workload("c2")
    blk, got, ref = _run(T, ctx, w.tree, w.ham, w.bonds, 2, 24, prec, seed=41, scale=0.11)
    tol = {"fp64": 1e-10, "fp32": 5e-4}[prec]
    for s in range(2):
        for t in range(w.tree.n_nodes):
            r = ref[s][t]
            assert np.abs(got[t][s] - r).max() <= tol * max(np.abs(r).max(), 1.0), (s, t)
    th = T.ttn_tree_create(ctx, w.tree)
    ob = SRC.src_bonds(w.tree, 24)
    by = T.block_from_arrays(ctx, th, ob, got)
    yy, _ = T.ttn_gram(ctx, None, by, by, want_h=False)
    for s in range(2):
        r = [x for x in ref[s]]
        ref_yy = N.overlap(w.tree, r, r)
        assert abs(yy[s, s] - ref_yy) <= {"fp64": 1e-11, "fp32": 2e-5}[prec] * ref_yy


def test_src_rejects_a_non_finite_sketch(T, ctx):
    tree = I.mps_tree(3, 2)
    ham = _ham(tree, 2, 1)
    th = T.ttn_tree_create(ctx, tree)
    H, _ = T.ttn_build_ttno(ctx, th, ham.flat(tree))
    bonds = I.uniform_bonds(tree, 2)
    bx = T.block_from_arrays(ctx, th, bonds, I.random_block(tree, bonds, 1, seed=1))
    omega = I.src_sketch(tree, 2, seed=1)
    omega[1][0, 0] = np.inf
    with pytest.raises(T.TTNError) as e:
        T.ttn_src_apply(ctx, H, bx, 2, omega)
    assert e.value.status == 4
