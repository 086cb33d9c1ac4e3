"""Full-size parity of the block Gram: the 12-mode QFF on the fork-4 tree (D = 24, 84 states, the
benchmark workload), the 64-mode coupled-oscillator model on an MPS (D = 32, 40 states) and on
the leaf-only binary tree (bonds 6..48, 64 states), and the 12-mode QFF on the all-physical
binary tree (D = 32, 84 states). Sampled entries of the
GPU Gram (built with the library's compressed TTNO) against the oracle's environment contraction
with its own, independently constructed state-diagram TTNO; both represent the same Hamiltonian
(Eq. sum_of_tp), so agreement checks the builder and the kernels together.
FP64 1e-11 relative to the largest diagonal entry; FP32 2e-5."""
import os

import numpy as np
import pytest

from oracle import network as N
from paper_2512_15875_gb300 import inputs as I

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def T():
    from paper_2512_15875_gb300 import ttn
    ttn.load()
    return ttn


@pytest.fixture(scope="module")
def ctx(T):
    return T.ttn_create(0)


@pytest.mark.parametrize("name", ["c2", "c3", "c4", "c5"])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "tf32x3_tc05"])
def test_full_size_gram_sampled(T, ctx, name, prec):
    w = I.make_workload(name)
    th = T.ttn_tree_create(ctx, w.tree)
    H, _ = T.ttn_build_ttno(ctx, th, w.ham.flat(w.tree))
    blk = I.initial_block(w.tree, w.ham, w.bonds, w.n_states, seed=2, noise=1e-2)
    b = T.block_from_arrays(ctx, th, w.bonds, blk)
    S, Hm = T.ttn_gram(ctx, H, b, b, prec=prec)
    otn = N.build_ttno(w.tree, w.ham)
    rng = np.random.default_rng(1)
    tol = 1e-11 if prec == "fp64" else 2e-5
    scale_h = np.abs(np.diag(Hm)).max()
    scale_s = np.abs(np.diag(S)).max()
    for i, j in [(0, 0), (0, w.n_states - 1)] + [tuple(int(v) for v in rng.integers(0, w.n_states, 2))]:
        a, c = [x[i] for x in blk], [x[j] for x in blk]
        assert abs(Hm[i, j] - N.expectation(w.tree, otn, a, c)) <= tol * scale_h, (i, j)
        assert abs(S[i, j] - N.overlap(w.tree, a, c)) <= tol * scale_s, (i, j)


# --- element-wise parity at the benchmark size ------------------------------------------------

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c2_gram_252.npz")
TOL = {"fp64": 1e-12, "fp32": 2e-5, "tf32x3": 2e-5, "tf32x3_tc05": 2e-5}


def _c2_gold_block(name):
    """The seeded blocks of tests/golden/make_c2_gram.py (same generator calls)."""
    w = I.make_workload("c2")
    g = np.load(GOLD)
    n = int(g["n_states"])
    if name == "prod":
        blk = I.initial_block(w.tree, w.ham, w.bonds, n, seed=0, noise=1e-2)
    else:
        blk = I.random_block(w.tree, w.bonds, n, seed=7, scale=float(g["rand_scale"]))
    return w, blk, g


@pytest.mark.parametrize("workspace_gb", [None, "1.5"])
@pytest.mark.parametrize("block", ["prod", "rand"])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "tf32x3_tc05"])
def test_c2_gram_every_entry_matches_the_oracle(T, ctx, prec, block, workspace_gb, monkeypatch):
    """All 31 878 pairs of the 252-state subspace of the 12-mode QFF (fork-4, D = 24) against the
    oracle's values stored by tests/golden/make_c2_gram.py, for near-product and dense random
    states; with a 1.5 GB workspace the pairs run in many chunks with a ragged last one."""
    if workspace_gb is not None:
        if prec != "fp32":
            pytest.skip("chunking is checked once, in float32")
        monkeypatch.setenv("TTN_WORKSPACE_GB", workspace_gb)
    w, blk, g = _c2_gold_block(block)
    th = T.ttn_tree_create(ctx, w.tree)
    H, _ = T.ttn_build_ttno(ctx, th, w.ham.flat(w.tree))
    b = T.block_from_arrays(ctx, th, w.bonds, blk)
    S, Hm = T.ttn_gram(ctx, H, b, b, prec=prec)
    iu = np.triu_indices(int(g["n_states"]))
    ref_h, ref_s = g[f"{block}_H"], g[f"{block}_S"]
    n = int(g["n_states"])
    diag = np.arange(n) * n - np.arange(n) * (np.arange(n) - 1) // 2   # (k, k) in the triangle
    scale_h, scale_s = np.abs(ref_h[diag]).max(), np.abs(ref_s[diag]).max()
    assert np.abs(Hm[iu] - ref_h).max() <= TOL[prec] * scale_h
    assert np.abs(S[iu] - ref_s).max() <= TOL[prec] * scale_s


def _import_ttno(T, ctx, th, tree, otn):
    ops, entries = [], []
    for node in range(tree.n_nodes):
        for wv, op, c in otn.entries[node]:
            entries.append((node, tuple(wv), len(ops), c))
            ops.append((node, op))
    return T.ttn_ttno_create(ctx, th, otn.wbond, ops, entries)


@pytest.mark.parametrize("name,nodes", [("c2", (1, 5)), ("c5", (1,))])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "tf32x3_tc05"])
def test_full_size_environments_and_heff(T, ctx, name, nodes, prec):
    """Environments on every leg of a backbone node (two children, no physical leg) and of a
    chain node (one child and a physical leg) of the 12-mode QFF on the fork-4 tree at D = 24,
    and of a node with a parent, two children and a physical leg of the all-physical tree at
    D = 32, for three bra/ket pairs, element by element; and H_eff at those nodes. The oracle's
    state-diagram TTNO is imported so both sides use the same operator bond basis."""
    w = I.make_workload(name)
    tree = w.tree
    th = T.ttn_tree_create(ctx, tree)
    otn = N.build_ttno(tree, w.ham)
    H = _import_ttno(T, ctx, th, tree, otn)
    blk = I.initial_block(tree, w.ham, w.bonds, 3, seed=3, noise=1e-2)
    b = T.block_from_arrays(ctx, th, w.bonds, blk)
    pb, pk = [0, 1, 2], [1, 2, 2]
    envs = T.ttn_envs_create(ctx, th)
    T.ttn_env_update(ctx, H, b, b, pb, pk, 2, envs, prec)
    tol = TOL[prec]
    for p, (i, j) in enumerate(zip(pb, pk)):
        up, down = N.environments(tree, otn, [x[i] for x in blk], [x[j] for x in blk])
        for t in nodes:
            for e in [t] + tree.children(t):
                for direction, ref in ((0, up[e]), (1, down[e])):
                    ref = np.transpose(ref, (1, 0, 2))      # oracle [a,w,b] -> library [w,a,b]
                    got = T.ttn_envs_get(envs, e, direction, p, ref.shape)
                    assert np.abs(got - ref).max() <= tol * np.abs(ref).max(), (t, e, direction)
    envs_d = T.ttn_envs_create(ctx, th)
    T.ttn_env_update(ctx, H, b, b, [0, 1, 2], [0, 1, 2], 2, envs_d, prec)
    bY = T.ttn_block_create(ctx, th, 3, w.bonds)
    for t in nodes:
        T.ttn_heff_apply(ctx, H, envs_d, t, b, bY, prec=prec)
        got = T.ttn_block_get(bY, -1, t).reshape((3,) + I.node_shape(tree, w.bonds, t))
        for s in range(3):
            ref = N.heff_apply(tree, otn, t, [x[s] for x in blk], blk[t][s])
            assert np.abs(got[s] - ref).max() <= 10 * tol * np.abs(ref).max(), (t, s)


# --- fitting and ALS at the benchmark size ------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_full_size_fit_matches_oracle(T, ctx, prec):
    """Variational fitting (Sec. II.C.2) on the 12-mode QFF, fork-4 tree, D = 24, two sweeps, of
    a residual-like target H x_0 - 1.5 x_0 and of a combination of three states, node tensor by
    node tensor against the oracle (same seeded states, same start, the oracle's state-diagram
    TTNO imported). The states are dense random TTNS with unit node tensors, so every node is
    full rank and the gauge (QR with a non-negative R diagonal) is unique; near-product states
    would leave the orthogonal completion of their rank-deficient nodes free. Tolerances as
    for the small trees: float64 1e-10, float32 2e-4 relative per node."""
    from oracle import solvers as S
    w = I.make_workload("c2")
    tree = w.tree
    th = T.ttn_tree_create(ctx, tree)
    otn = N.build_ttno(tree, w.ham)
    idt = N.identity_ttno(tree)
    H = _import_ttno(T, ctx, th, tree, otn)
    n = 5
    blk = I.random_block(tree, w.bonds, n, 4)
    for x in blk:   # unit node tensors: states of norm ~1 (float32 would overflow otherwise)
        x /= np.linalg.norm(x.reshape(n, -1), axis=1).reshape((n,) + (1,) * (x.ndim - 1))
    X = [[x[j] for x in blk] for j in range(n)]
    bX = T.block_from_arrays(ctx, th, w.bonds, blk)
    out = T.ttn_block_create(ctx, th, 2, w.bonds)
    T.ttn_block_copy_states(out, bX, [0, 3])
    coeff = np.zeros((2 * n, 2))
    coeff[0, 0], coeff[n + 0, 0] = 1.0, -1.5
    coeff[n + 1, 1], coeff[n + 3, 1], coeff[n + 4, 1] = 0.3, -0.7, 0.2
    T.ttn_recompress(ctx, coeff, [H] * n + [None] * n, [bX] * (2 * n), list(range(n)) * 2, out,
                     n_sweeps=2, prec=prec)
    shp = [I.node_shape(tree, w.bonds, t) for t in range(tree.n_nodes)]
    got = T.block_to_arrays(out, shp)
    ref0 = S.fit(tree, [(1.0, otn, X[0]), (-1.5, idt, X[0])], X[0], 2)
    ref1 = S.fit(tree, [(0.3, idt, X[1]), (-0.7, idt, X[3]), (0.2, idt, X[4])], X[3], 2)
    tol = 1e-10 if prec == "fp64" else 2e-4
    for t in range(tree.n_nodes):
        for s, ref in ((0, ref0), (1, ref1)):
            assert np.abs(got[t][s] - ref[t]).max() <= tol * np.abs(ref[t]).max(), (t, s)


def test_full_size_als_matches_oracle(T, ctx):
    """One state of the ALS preconditioner solve (H - s) y = r (Sec. II.C.3) on the 12-mode QFF,
    fork-4 tree, D = 24, two sweeps of 10 MINRES steps with no stopping tolerance, float64,
    against the oracle: the represented vector to 1e-8 relative (as for the small trees: the
    rounding of the two implementations is amplified along the dependent Krylov steps)."""
    from oracle import solvers as S
    w = I.make_workload("c2")
    tree = w.tree
    th = T.ttn_tree_create(ctx, tree)
    otn = N.build_ttno(tree, w.ham)
    H = _import_ttno(T, ctx, th, tree, otn)
    blk = I.initial_block(tree, w.ham, w.bonds, 1, seed=6, noise=1e-2)
    X0 = [x[0] for x in blk]
    bR = T.block_from_arrays(ctx, th, w.bonds, blk)
    bY = T.block_from_arrays(ctx, th, w.bonds, blk)
    lam0 = N.expectation(tree, otn, X0, X0) / N.overlap(tree, X0, X0)
    shift = lam0 - 300.0
    T.ttn_als_solve(ctx, H, np.array([shift]), bR, bY, n_sweeps=2, minres_max=10, minres_tol=0.0,
                    prec="fp64")
    shp = [I.node_shape(tree, w.bonds, t) for t in range(tree.n_nodes)]
    got = [g[0] for g in T.block_to_arrays(bY, shp)]
    ref = S.als_solve(tree, otn, shift, X0, X0, 2, 10, 0.0)
    for t in range(tree.n_nodes):
        assert np.abs(got[t] - ref[t]).max() <= 1e-8 * np.abs(ref[t]).max(), t
