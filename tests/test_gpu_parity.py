"""Parity of the CUDA contraction path (through the C ABI) with the FP64 oracle.

Inputs are seeded and identical on both sides. Parity cases use the oracle's own (uncompressed)
TTNO, imported into the library as raw entries, so that both sides contract the same operator;
the library's own TTNO builder is checked against the oracle's term-by-term expectation values,
which do not depend on any TTNO.

Tolerances: FP64 path 1e-12 relative to the largest magnitude of the compared quantity (sums of
at most a few 10^5 products of O(1) numbers in float64); FP32 path 2e-5 relative (float32
accumulation of the same sums: ~1e-7 per operation grown by the contraction depth); the
tensor-core paths (3xTF32 split products, ~2^-21 per product, float32 accumulation; mma.sync or
tcgen05 kernels) use the float32 bound."""
import numpy as np
import pytest

from oracle import network as N
from paper_2512_15875_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-5, "tf32x3": 2e-5, "tf32x3_tc05": 2e-5}


@pytest.fixture(scope="module")
def T():
    from paper_2512_15875_gb300 import ttn
    ttn.load()
    return ttn


@pytest.fixture(scope="module")
def ctx(T):
    return T.ttn_create(0)


def import_ttno(T, ctx, th, tree, otn):
    ops, entries = [], []
    for node in range(tree.n_nodes):
        for w, op, c in otn.entries[node]:
            entries.append((node, tuple(w), len(ops), c))
            ops.append((node, op))
    return T.ttn_ttno_create(ctx, th, otn.wbond, ops, entries)


def rand_ham(tree, d, seed):
    L = int(tree.mode.max()) + 1
    rng = np.random.default_rng(seed)
    ham = I.Hamiltonian(dims=[d] * L, omega=rng.uniform(1, 2, L))
    for i in range(L):
        ham.add(ham.omega[i], {i: "h"})
    for i in range(L):
        for j in range(i + 1, L):
            ham.add_monomial(rng.normal(0, 0.3), (i, j))
    for _ in range(2 * L):
        ham.add_monomial(rng.normal(0, 0.1), tuple(sorted(rng.integers(0, L, 3))))
        ham.add_monomial(rng.normal(0, 0.05), tuple(sorted(rng.integers(0, L, 4))))
    return ham


def shapes(tree, bonds):
    return [I.node_shape(tree, bonds, t) for t in range(tree.n_nodes)]


CASES = [
    # name, tree, d, D  -- bonds span several 64-wide tiles with ragged tails
    ("c1_D36", lambda: I.mps_tree(4, 6), 6, 36),
    ("fork2x2_D24", lambda: I.fork_tree(2, 2, 5), 5, 24),
    ("leafbin2_D20", lambda: I.leaf_only_binary_tree(2, 5), 5, 20),
    ("physbin6_D17", lambda: I.all_physical_binary_tree(6, 4), 4, 17),
    ("ttree6_D16", lambda: I.t_tree(6, 4), 4, 16),
]


def _setup(T, ctx, case, n_bra, n_ket, seed):
    name, mk, d, D = case
    tree = mk()
    ham = rand_ham(tree, d, seed)
    bonds = I.uniform_bonds(tree, D)
    th = T.ttn_tree_create(ctx, tree)
    otn = N.build_ttno(tree, ham)
    H = import_ttno(T, ctx, th, tree, otn)
    A = I.random_block(tree, bonds, n_bra, seed + 1)
    B = I.random_block(tree, bonds, n_ket, seed + 2)
    bA = T.block_from_arrays(ctx, th, bonds, A)
    bB = T.block_from_arrays(ctx, th, bonds, B)
    return tree, ham, bonds, th, otn, H, A, B, bA, bB


def _rel(x, ref):
    return np.abs(x - ref).max() / max(np.abs(ref).max(), 1e-300)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "tf32x3_tc05"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_environments_match_oracle(T, ctx, case, prec):
    tree, ham, bonds, th, otn, H, A, B, bA, bB = _setup(T, ctx, case, 2, 3, seed=7)
    pb = [0, 1, 1, 0]
    pk = [0, 2, 1, 1]
    envs = T.ttn_envs_create(ctx, th)
    T.ttn_env_update(ctx, H, bA, bB, pb, pk, 2, envs, prec)
    for p, (i, j) in enumerate(zip(pb, pk)):
        up, down = N.environments(tree, otn, [x[i] for x in A], [x[j] for x in B])
        for t in range(tree.n_nodes):
            if t == tree.root:
                continue
            ref_up = np.transpose(up[t], (1, 0, 2))        # oracle [a,w,b] -> library [w,a,b]
            ref_dn = np.transpose(down[t], (1, 0, 2))
            got_up = T.ttn_envs_get(envs, t, 0, p, ref_up.shape)
            got_dn = T.ttn_envs_get(envs, t, 1, p, ref_dn.shape)
            assert _rel(got_up, ref_up) <= TOL[prec], (t, "up")
            assert _rel(got_dn, ref_dn) <= TOL[prec], (t, "down")


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "tf32x3_tc05"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_gram_matches_oracle(T, ctx, case, prec):
    tree, ham, bonds, th, otn, H, A, B, bA, bB = _setup(T, ctx, case, 3, 4, seed=11)
    S, Hm = T.ttn_gram(ctx, H, bA, bB, prec=prec)
    for i in range(3):
        for j in range(4):
            a, b = [x[i] for x in A], [x[j] for x in B]
            ref_h = N.expectation(tree, otn, a, b)
            ref_s = N.overlap(tree, a, b)
            assert abs(Hm[i, j] - ref_h) <= 10 * TOL[prec] * np.abs(Hm).max(), (i, j)
            assert abs(S[i, j] - ref_s) <= TOL[prec] * np.abs(S).max() * 10, (i, j)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "tf32x3_tc05"])
def test_symmetric_gram_of_one_block(T, ctx, prec):
    case = CASES[1]
    tree, ham, bonds, th, otn, H, A, B, bA, bB = _setup(T, ctx, case, 5, 1, seed=13)
    S, Hm = T.ttn_gram(ctx, H, bA, bA, prec=prec)
    assert np.array_equal(S, S.T) and np.array_equal(Hm, Hm.T)
    ref = np.array([[N.expectation(tree, otn, [x[i] for x in A], [x[j] for x in A])
                     for j in range(5)] for i in range(5)])
    assert _rel(Hm, ref) <= TOL[prec] * 10
    assert np.all(np.linalg.eigvalsh(S) > -1e-10 * np.abs(S).max())


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "tf32x3_tc05"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_heff_matches_oracle(T, ctx, case, prec):
    tree, ham, bonds, th, otn, H, A, B, bA, bB = _setup(T, ctx, case, 3, 3, seed=17)
    envs = T.ttn_envs_create(ctx, th)
    T.ttn_env_update(ctx, H, bA, bA, [0, 1, 2], [0, 1, 2], 2, envs, prec)
    shp = shapes(tree, bonds)
    bY = T.ttn_block_create(ctx, th, 3, bonds)
    shift = np.array([0.0, 0.5, -1.25])
    for t in range(tree.n_nodes):
        T.ttn_heff_apply(ctx, H, envs, t, bB, bY, shift=shift, prec=prec)
        got = T.ttn_block_get(bY, -1, t).reshape((3,) + shp[t])
        for s in range(3):
            psi = [x[s] for x in A]
            ref = N.heff_apply(tree, otn, t, psi, B[t][s]) - shift[s] * B[t][s]
            assert _rel(got[s], ref) <= TOL[prec] * 10, (t, s)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "tf32x3_tc05"])
@pytest.mark.parametrize("case", CASES[:3], ids=[c[0] for c in CASES[:3]])
def test_exact_apply_matches_oracle(T, ctx, case, prec):
    name, mk, d, D = case
    tree = mk()
    ham = rand_ham(tree, d, 19)
    bonds = I.uniform_bonds(tree, min(D, 6))
    th = T.ttn_tree_create(ctx, tree)
    otn = N.build_ttno(tree, ham)
    H = import_ttno(T, ctx, th, tree, otn)
    A = I.random_block(tree, bonds, 2, 20)
    bA = T.block_from_arrays(ctx, th, bonds, A)
    out = T.ttn_apply_block(ctx, H, bA, prec)
    for s in range(2):
        ref = N.apply_exact(tree, otn, [x[s] for x in A])
        for t in range(tree.n_nodes):
            got = T.ttn_block_get(out, s, t).reshape(ref[t].shape)
            assert _rel(got, ref[t]) <= TOL[prec], t


def test_built_ttno_gram_matches_term_by_term_oracle(T, ctx):
    """The library's compressed TTNO gives the same <A|H|B> as the sum over Hamiltonian terms."""
    w = I.make_workload("c1", D=8)
    th = T.ttn_tree_create(ctx, w.tree)
    H, _ = T.ttn_build_ttno(ctx, th, w.ham.flat(w.tree))
    blk = w.block()
    bX = T.block_from_arrays(ctx, th, w.bonds, blk)
    S, Hm = T.ttn_gram(ctx, H, bX, bX)
    for i in range(w.n_states):
        for j in range(w.n_states):
            ref = N.expectation_terms(w.tree, w.ham, [x[i] for x in blk], [x[j] for x in blk])
            assert abs(Hm[i, j] - ref) <= 1e-12 * np.abs(Hm).max()


def test_empty_pair_list_and_zero_states(T, ctx):
    case = CASES[0]
    tree, ham, bonds, th, otn, H, A, B, bA, bB = _setup(T, ctx, case, 1, 1, seed=3)
    envs = T.ttn_envs_create(ctx, th)
    T.ttn_env_update(ctx, H, bA, bB, [], [], 2, envs)
    b0 = T.ttn_block_create(ctx, th, 0, bonds)
    S, Hm = T.ttn_gram(ctx, H, b0, b0)
    assert S.shape == (0, 0) and Hm.shape == (0, 0)


def test_bond_one_product_states(T, ctx):
    """Degenerate bonds (all 1): the Gram of product states is a product of one-mode numbers."""
    w = I.make_workload("c1", D=1)
    th = T.ttn_tree_create(ctx, w.tree)
    H, _ = T.ttn_build_ttno(ctx, th, w.ham.flat(w.tree))
    blk = w.block(noise=0.0)
    bX = T.block_from_arrays(ctx, th, w.bonds, blk)
    S, Hm = T.ttn_gram(ctx, H, bX, bX)
    assert np.allclose(S, np.eye(w.n_states), atol=1e-14)
    ref = np.array([[N.expectation_terms(w.tree, w.ham, [x[i] for x in blk],
                                         [x[j] for x in blk]) for j in range(w.n_states)]
                    for i in range(w.n_states)])
    assert _rel(Hm, ref) <= 1e-13


def test_bad_arguments_are_reported(T, ctx):
    case = CASES[0]
    tree, ham, bonds, th, otn, H, A, B, bA, bB = _setup(T, ctx, case, 1, 1, seed=5)
    envs = T.ttn_envs_create(ctx, th)
    with pytest.raises(T.TTNError) as e:
        T.ttn_env_update(ctx, H, bA, bB, [0], [7], 2, envs)
    assert e.value.status == 1
    with pytest.raises(T.TTNError):
        T.ttn_block_set(bA, 0, 0, np.zeros(3))


@pytest.mark.slow
@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "tf32x3_tc05"])
def test_full_size_qff_gram_sampled(T, ctx, prec):
    """The 12-mode QFF on the fork-4 tree at D=24 with the 252-state subspace the LOBPCG Gram
    contracts (3 x 84 states): sampled entries against the term-by-term oracle."""
    w = I.make_workload("c2")
    th = T.ttn_tree_create(ctx, w.tree)
    H, _ = T.ttn_build_ttno(ctx, th, w.ham.flat(w.tree))
    blk = I.initial_block(w.tree, w.ham, w.bonds, 252, seed=0, noise=1e-2)
    bS = T.block_from_arrays(ctx, th, w.bonds, blk)
    S, Hm = T.ttn_gram(ctx, H, bS, bS, prec=prec)
    assert np.array_equal(Hm, Hm.T)
    rng = np.random.default_rng(0)
    scale = np.abs(np.diag(Hm)).max()
    for _ in range(4):
        i, j = (int(x) for x in rng.integers(0, 252, 2))
        a, b = [x[i] for x in blk], [x[j] for x in blk]
        assert abs(Hm[i, j] - N.expectation_terms(w.tree, w.ham, a, b)) <= TOL[prec] * scale
        assert abs(S[i, j] - N.overlap(w.tree, a, b)) <= TOL[prec] * np.abs(np.diag(S)).max()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_contractions_in_pair_chunks_match_oracle(T, ctx, prec, monkeypatch):
    """A workspace budget far below one pair's intermediates makes every node contraction run
    in chunks of pairs (each with its own slice of environments and outputs, ragged last
    chunk); environments, H_eff and the Gram still match the oracle."""
    monkeypatch.setenv("TTN_WORKSPACE_GB", "2e-6")
    case = CASES[1]
    tree, ham, bonds, th, otn, H, A, B, bA, bB = _setup(T, ctx, case, 3, 3, seed=23)
    pb, pk = [0, 1, 2, 2, 0], [0, 2, 1, 2, 1]
    envs = T.ttn_envs_create(ctx, th)
    T.ttn_env_update(ctx, H, bA, bB, pb, pk, 2, envs, prec)
    for p, (i, j) in enumerate(zip(pb, pk)):
        up, down = N.environments(tree, otn, [x[i] for x in A], [x[j] for x in B])
        for t in range(tree.n_nodes):
            if t == tree.root:
                continue
            for direction, ref in ((0, up[t]), (1, down[t])):
                ref = np.transpose(ref, (1, 0, 2))
                got = T.ttn_envs_get(envs, t, direction, p, ref.shape)
                assert _rel(got, ref) <= TOL[prec], (t, direction)
    envs_d = T.ttn_envs_create(ctx, th)
    T.ttn_env_update(ctx, H, bA, bA, [0, 1, 2], [0, 1, 2], 2, envs_d, prec)
    bY = T.ttn_block_create(ctx, th, 3, bonds)
    shp = shapes(tree, bonds)
    for t in range(tree.n_nodes):
        T.ttn_heff_apply(ctx, H, envs_d, t, bB, bY, prec=prec)
        got = T.ttn_block_get(bY, -1, t).reshape((3,) + shp[t])
        for s in range(3):
            ref = N.heff_apply(tree, otn, t, [x[s] for x in A], B[t][s])
            assert _rel(got[s], ref) <= TOL[prec] * 10, (t, s)
    S, Hm = T.ttn_gram(ctx, H, bA, bB, prec=prec)
    for i in range(3):
        for j in range(3):
            a, b = [x[i] for x in A], [x[j] for x in B]
            assert abs(Hm[i, j] - N.expectation(tree, otn, a, b)) <= 10 * TOL[prec] * np.abs(Hm).max()
