"""Block inverse iteration (Alg. 3, Eq. inverse iteration update) on the GPU against the FP64
oracle: one shift per state (the all-physical-tree configuration) and the paper's clustering of
Rayleigh quotients into blocks with a mean shift (Sec. III.B).

MINRES runs with tolerance 0 so both sides take the same Krylov steps. The shifted local systems
are singular to working precision by design (the shift is a Rayleigh quotient, condition numbers
up to ~1e11), so float64 rounding differences grow to ~1e-4 relative in the states; the
Rayleigh quotients, quadratic in the state error, agree to ~1e-8: bound 1e-7 relative."""
import numpy as np
import pytest

from oracle import network as N, solvers as S
from paper_2512_15875_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    from paper_2512_15875_gb300 import ttn
    ttn.load()
    return ttn


@pytest.fixture(scope="module")
def ctx(T):
    return T.ttn_create(0)


def _run(T, ctx, tree, ham, bonds, n, gap, n_iter, noise=1e-2, als_sweeps=1, mr=10):
    th = T.ttn_tree_create(ctx, tree)
    H, _ = T.ttn_build_ttno(ctx, th, ham.flat(tree))
    blk = I.initial_block(tree, ham, bonds, n, seed=1, noise=noise)
    bX = T.block_from_arrays(ctx, th, bonds, blk)
    hist = T.ttn_inverse_iteration(ctx, H, bX, n_iter, cluster_gap=gap, als_sweeps=als_sweeps,
                                   minres_max=mr, minres_tol=0.0, prec="fp64")
    otn = N.build_ttno(tree, ham)
    X0 = [[t[j] for t in blk] for j in range(n)]
    clusters = (lambda l: [[j] for j in range(len(l))]) if gap <= 0 else \
        (lambda l: S.clusters_by_gap(l, gap))
    _, _, ref = S.inverse_iteration(tree, otn, X0, n_iter, clusters, als_sweeps=als_sweeps,
                                    minres_max=mr, minres_tol=0.0)
    return hist, np.array(ref)


@pytest.mark.parametrize("gap", [0.0, 300.0])
def test_inverse_iteration_matches_oracle_on_the_four_mode_model(T, ctx, gap):
    w = I.make_workload("c1", D=8)
    hist, ref = _run(T, ctx, w.tree, w.ham, w.bonds, 5, gap, 2)
    assert np.abs(hist - ref).max() <= 1e-7 * np.abs(ref).max()


def test_inverse_iteration_on_an_all_physical_binary_tree(T, ctx):
    tree = I.all_physical_binary_tree(5, 4)
    rng = np.random.default_rng(3)
    ham = I.Hamiltonian(dims=[4] * 5, omega=rng.uniform(1000, 2000, 5))
    for i in range(5):
        ham.add(ham.omega[i], {i: "h"})
    for i in range(5):
        for j in range(i + 1, 5):
            ham.add_monomial(rng.normal(0, 30), (i, j))
    for _ in range(6):
        ham.add_monomial(rng.normal(0, 5), tuple(sorted(rng.integers(0, 5, 3))))
    bonds = I.uniform_bonds(tree, 8)
    hist, ref = _run(T, ctx, tree, ham, bonds, 6, 0.0, 2)
    assert np.abs(hist - ref).max() <= 1e-7 * np.abs(ref).max()


@pytest.mark.parametrize("gap", [0.0, 300.0])
def test_inverse_iteration_converges_to_eigenvalues_at_full_bond(T, ctx, gap):
    # every Rayleigh quotient reaches one of the five lowest eigenvalues of the dense Hamiltonian
    # to 1e-10 relative, each once (as the pinned oracle does); MINRES stops at the rounding
    # floor once a shift has converged to working precision instead of running to its cap
    w = I.make_workload("c1", D=36)
    ev = np.linalg.eigvalsh(N.dense_hamiltonian(w.ham))
    th = T.ttn_tree_create(ctx, w.tree)
    H, _ = T.ttn_build_ttno(ctx, th, w.ham.flat(w.tree))
    bX = T.block_from_arrays(ctx, th, w.bonds, w.block(noise=1e-2))
    hist = T.ttn_inverse_iteration(ctx, H, bX, 6, cluster_gap=gap, als_sweeps=2, minres_max=300,
                                   minres_tol=1e-12, prec="fp64")
    assert np.abs(np.sort(hist[-1]) - ev[:5]).max() <= 1e-10 * ev[0]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_block_rayleigh_ritz_matches_oracle(T, ctx, prec):
    # the generalized eigenvalue problem Hc = ESc over all states (Sec. III.B) on truncated,
    # non-orthogonal states of the four-mode model
    w = I.make_workload("c1", D=8)
    th = T.ttn_tree_create(ctx, w.tree)
    H, _ = T.ttn_build_ttno(ctx, th, w.ham.flat(w.tree))
    blk = w.block(noise=5e-2)
    bX = T.block_from_arrays(ctx, th, w.bonds, blk)
    theta = T.ttn_block_rayleigh_ritz(ctx, H, bX, eps=1e-12, fit_sweeps=2, prec=prec)
    otn = N.build_ttno(w.tree, w.ham)
    ref, Y = S.block_rayleigh_ritz(w.tree, otn, [[t[j] for t in blk] for j in range(5)], 2)
    tol = {"fp64": 1e-10, "fp32": 2e-6}[prec]
    assert np.abs(theta - ref).max() <= tol * abs(ref[0])
    # the fitted Ritz vectors: same overlaps as the oracle's (not exactly the identity at this
    # truncated bond)
    S2, _ = T.ttn_gram(ctx, H, bX, bX)
    M = np.array([[N.overlap(w.tree, a, b) for b in Y] for a in Y])
    assert np.abs(S2 - M).max() <= {"fp64": 1e-9, "fp32": 1e-5}[prec]
