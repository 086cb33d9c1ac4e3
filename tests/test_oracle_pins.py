"""Pins of the FP64 oracle against facts that do not come from the oracle itself: textbook
identities, closed-form spectra, dense exact diagonalisation on tiny systems, brute force, and
invariants of the algorithms (Sec. II, Sec. III.A)."""
import numpy as np
import pytest

from oracle import closed, network as N, solvers as S
from paper_2512_15875_gb300 import inputs as I


def _rand_ham(tree, d, seed, quartic=True):
    """Small random QFF-like Hamiltonian on the modes of ``tree`` (harmonic + all pairs +
    a few cubic/quartic monomials, with repeated modes)."""
    L = int(tree.mode.max()) + 1
    rng = np.random.default_rng(seed)
    ham = I.Hamiltonian(dims=[d] * L, omega=rng.uniform(1.0, 2.0, L))
    for i in range(L):
        ham.add(ham.omega[i], {i: "h"})
    for i in range(L):
        for j in range(i + 1, L):
            ham.add_monomial(rng.normal(0, 0.2), (i, j))
    for _ in range(2 * L):
        k = 3 if not quartic else int(rng.integers(3, 5))
        ham.add_monomial(rng.normal(0, 0.05), tuple(sorted(rng.integers(0, L, k))))
    return ham


SMALL_TREES = [
    ("mps4", lambda d: I.mps_tree(4, d)),
    ("fork2x2", lambda d: I.fork_tree(2, 2, d)),
    ("leafbin2", lambda d: I.leaf_only_binary_tree(2, d)),
    ("physbin5", lambda d: I.all_physical_binary_tree(5, d)),
    ("ttree5", lambda d: I.t_tree(5, d)),
]


# --- one-mode operators and the dense Hamiltonian ---------------------------------------------

def test_truncated_q_is_the_hermite_jacobi_matrix():
    # eigenvalues of the truncated (a + a^dag)/sqrt(2) in d functions are the roots of H_d:
    # the Gauss-Hermite (DVR) points of the paper's Hermite basis
    for d in (2, 6, 9):
        q = I.ho_matrices(d)["q"]
        roots = np.polynomial.hermite.hermroots([0] * d + [1])
        assert np.allclose(np.sort(np.linalg.eigvalsh(q)), np.sort(roots), atol=1e-12)
        m = I.ho_matrices(d)
        assert np.allclose(m["q3"], q @ q @ q)
        assert np.allclose(np.diag(m["h"]), np.arange(d) + 0.5)


def test_uncoupled_limit_is_exact():
    omega = [1100.0, 1730.0, 2990.0]
    ham = I.Hamiltonian(dims=[5, 4, 6], omega=np.array(omega))
    for i in range(3):
        ham.add(omega[i], {i: "h"})
    ev = np.linalg.eigvalsh(N.dense_hamiltonian(ham))
    assert np.allclose(ev, closed.uncoupled_levels(omega, [5, 4, 6], len(ev)), rtol=1e-14)


def test_bilinear_model_approaches_normal_modes():
    # Eq. (coupled_harmonic_oscillator) with omega_j = sqrt(j/2), alpha = 0.1 on three modes:
    # the error against sum nu_k (n_k + 1/2) shrinks as the basis grows
    errs = []
    for d in (6, 10, 14):
        ham = I.uniform_coupled_model(n_modes=3, d=d, alpha=0.1)
        ev = np.linalg.eigvalsh(N.dense_hamiltonian(ham))[:4]
        nu = closed.normal_mode_frequencies(ham.omega, np.full((3, 3), 0.1))
        errs.append(np.abs(ev - closed.normal_mode_levels(nu, 4)).max())
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-6


def test_term_counts_of_the_paper_models():
    assert len(I.uniform_coupled_model(64, d=2).terms) == 2080          # Sec. III.A: 64 + 2016
    assert len(I.quartic_force_field(0).terms) == 311                   # Sec. III.B: 12+108+191


# --- TTNO and TTNS contractions -------------------------------------------------------------

@pytest.mark.parametrize("name,mk", SMALL_TREES)
def test_ttno_contracts_to_dense_hamiltonian(name, mk):
    tree = mk(3)
    ham = _rand_ham(tree, 3, seed=len(name))
    H = N.dense_hamiltonian(ham)
    T = N.build_ttno(tree, ham)
    assert np.abs(N.ttno_to_dense(tree, T) - H).max() <= 1e-13 * np.abs(H).max()


def test_ttno_pin_detects_a_planted_sign_error():
    tree = I.fork_tree(2, 2, 3)
    ham = _rand_ham(tree, 3, seed=5)
    T = N.build_ttno(tree, ham)
    w, op, c = T.entries[4][-1]
    T.entries[4][-1] = (w, op, -c)
    assert np.abs(N.ttno_to_dense(tree, T) - N.dense_hamiltonian(ham)).max() > 1e-6


def test_c1_ttno_dense_and_symmetric():
    w = I.make_workload("c1", D=8)
    H = N.dense_hamiltonian(w.ham)
    assert H.shape == (1296, 1296)
    assert np.abs(H - H.T).max() == 0.0
    Ht = N.ttno_to_dense(w.tree, N.build_ttno(w.tree, w.ham))
    assert np.abs(Ht - H).max() <= 1e-13 * np.abs(H).max()


@pytest.mark.parametrize("name,mk", SMALL_TREES)
def test_expectation_against_dense_and_terms(name, mk):
    tree = mk(3)
    ham = _rand_ham(tree, 3, seed=11 + len(name))
    H = N.dense_hamiltonian(ham)
    T = N.build_ttno(tree, ham)
    bonds = I.uniform_bonds(tree, 4)
    blk = I.random_block(tree, bonds, 2, seed=3)
    A, B = [t[0] for t in blk], [t[1] for t in blk]
    ref = N.ttns_to_dense(tree, A) @ H @ N.ttns_to_dense(tree, B)
    scale = abs(ref) + 1.0
    for t in range(tree.n_nodes):   # closing at any node exercises every top-down environment
        assert abs(N.expectation(tree, T, A, B, close_at=t) - ref) <= 1e-12 * scale
    assert abs(N.expectation_terms(tree, ham, A, B) - ref) <= 1e-12 * scale
    assert abs(N.overlap(tree, A, B) - N.ttns_to_dense(tree, A) @ N.ttns_to_dense(tree, B)) \
        <= 1e-12 * scale


@pytest.mark.parametrize("name,mk", SMALL_TREES)
def test_heff_is_the_projected_hamiltonian(name, mk):
    """H_eff,t = P^T H P where column k of P is the dense vector of psi with node t replaced by
    the k-th unit tensor."""
    tree = mk(3)
    ham = _rand_ham(tree, 3, seed=21 + len(name))
    H = N.dense_hamiltonian(ham)
    T = N.build_ttno(tree, ham)
    psi = [x[0] for x in I.random_block(tree, I.uniform_bonds(tree, 3), 1, seed=4)]
    for t in range(tree.n_nodes):
        shp = psi[t].shape
        cols = []
        for k in range(int(np.prod(shp))):
            e = np.zeros(psi[t].size)
            e[k] = 1.0
            ps = list(psi)
            ps[t] = e.reshape(shp)
            cols.append(N.ttns_to_dense(tree, ps))
        P = np.array(cols).T
        Heff = np.array([N.heff_apply(tree, T, t, psi, P_col.reshape(shp)).ravel()
                         for P_col in np.eye(psi[t].size)]).T
        ref = P.T @ H @ P
        assert np.abs(Heff - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("name,mk", SMALL_TREES)
def test_exact_apply_against_dense(name, mk):
    tree = mk(3)
    ham = _rand_ham(tree, 3, seed=31 + len(name))
    H = N.dense_hamiltonian(ham)
    T = N.build_ttno(tree, ham)
    psi = [x[0] for x in I.random_block(tree, I.uniform_bonds(tree, 4), 1, seed=5)]
    out = N.apply_exact(tree, T, psi)
    ref = H @ N.ttns_to_dense(tree, psi)
    assert np.abs(N.ttns_to_dense(tree, out) - ref).max() <= 1e-12 * np.abs(ref).max()


def test_gram_invariants():
    w = I.make_workload("c1", D=8)
    T = N.build_ttno(w.tree, w.ham)
    blk = w.block()
    states = [[t[j] for t in blk] for j in range(4)]
    Ht, Mt = S.gram_block(w.tree, T, states)
    assert np.abs(Ht - Ht.T).max() == 0.0
    assert np.linalg.eigvalsh(Mt).min() > 0
    for k, s in enumerate(states):
        v = N.ttns_to_dense(w.tree, s)
        assert abs(Mt[k, k] - v @ v) <= 1e-12 * (v @ v)
    H = N.dense_hamiltonian(w.ham)
    V = np.array([N.ttns_to_dense(w.tree, s) for s in states])
    assert np.abs(Ht - V @ H @ V.T).max() <= 1e-12 * np.abs(Ht).max()


# --- solvers --------------------------------------------------------------------------------

def test_minres_matches_direct_solve_and_is_monotone():
    rng = np.random.default_rng(0)
    for spd in (True, False):
        A = rng.standard_normal((10, 10))
        A = A @ A.T + 10 * np.eye(10) if spd else A + A.T
        b = rng.standard_normal(10)
        x, h = S.minres(lambda v: A @ v, b, maxiter=10, tol=0.0)
        assert np.abs(x - np.linalg.solve(A, b)).max() <= 1e-10 * np.abs(x).max()
        assert np.all(np.diff(h) <= 1e-12 * h[0])
        assert abs(np.linalg.norm(b - A @ x) - h[-1]) <= 1e-10 * h[0]


def test_minres_short_run_residual_matches_history():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((30, 30))
    A = A + A.T
    b = rng.standard_normal(30)
    x0 = rng.standard_normal(30)
    x, h = S.minres(lambda v: A @ v, b, x0=x0, maxiter=5, tol=0.0)
    assert len(h) == 6
    assert abs(np.linalg.norm(b - A @ x) - h[-1]) <= 1e-10 * h[0]


def test_rayleigh_ritz_matches_generalized_eigh():
    import scipy.linalg
    rng = np.random.default_rng(2)
    B = rng.standard_normal((12, 12))
    M = B @ B.T + 0.5 * np.eye(12)
    H = rng.standard_normal((12, 12))
    H = H + H.T
    th, V = S.rayleigh_ritz(H, M, 4)
    assert np.allclose(th, scipy.linalg.eigh(H, M, eigvals_only=True)[:4], atol=1e-10)
    assert np.allclose(V.T @ M @ V, np.eye(4), atol=1e-10)
    assert np.allclose(H @ V, M @ V * th, atol=1e-9)


@pytest.mark.parametrize("name,mk", SMALL_TREES)
def test_canonical_form_preserves_the_state(name, mk):
    tree = mk(3)
    psi = [x[0] for x in I.random_block(tree, I.uniform_bonds(tree, 4), 1, seed=6)]
    v = N.ttns_to_dense(tree, psi)
    c = S.canonicalize(tree, psi)
    assert np.abs(N.ttns_to_dense(tree, psi) - v).max() <= 1e-12 * np.abs(v).max()
    for t in range(tree.n_nodes):      # every non-centre node is an isometry toward the centre
        if t == c:
            continue
        toward = N.path(tree, t, c)[1]
        m = N.legs(tree, t).index(toward)
        M = np.moveaxis(N.with_phys(tree, t, psi[t]), m, -1).reshape(-1, psi[t].shape[m])
        assert np.allclose(M.T @ M, np.eye(M.shape[1]), atol=1e-12)
    for dst in N.preorder(tree)[::-1]:
        c = S.move_center(tree, psi, c, dst)
        assert np.abs(N.ttns_to_dense(tree, psi) - v).max() <= 1e-12 * np.abs(v).max()


def test_fit_is_exact_at_full_bond():
    w = I.make_workload("c1", D=36)
    blk = w.block()
    idt = N.identity_ttno(w.tree)
    X = [[t[j] for t in blk] for j in range(3)]
    terms = [(0.7, idt, X[0]), (-1.3, idt, X[1]), (0.2, idt, X[2])]
    psi = S.fit(w.tree, terms, X[0], 1)
    ref = sum(c * N.ttns_to_dense(w.tree, x) for c, _, x in terms)
    assert np.abs(N.ttns_to_dense(w.tree, psi) - ref).max() <= 1e-12 * np.abs(ref).max()


def test_fit_of_an_operator_term_is_exact_at_full_bond():
    w = I.make_workload("c1", D=36)
    T = N.build_ttno(w.tree, w.ham)
    x = [t[0] for t in w.block()]
    psi = S.fit(w.tree, [(1.0, T, x)], x, 2)
    ref = N.dense_hamiltonian(w.ham) @ N.ttns_to_dense(w.tree, x)
    assert np.abs(N.ttns_to_dense(w.tree, psi) - ref).max() <= 1e-10 * np.abs(ref).max()


def test_als_solves_the_shifted_system_at_full_bond():
    w = I.make_workload("c1", D=36)
    T = N.build_ttno(w.tree, w.ham)
    H = N.dense_hamiltonian(w.ham)
    s = np.linalg.eigvalsh(H)[0] - 100.0
    rhs = [t[2] for t in w.block()]
    y = S.als_solve(w.tree, T, s, rhs, rhs, n_sweeps=3, minres_max=400, minres_tol=1e-14)
    yd, rd = N.ttns_to_dense(w.tree, y), N.ttns_to_dense(w.tree, rhs)
    assert np.linalg.norm((H - s * np.eye(len(H))) @ yd - rd) <= 1e-10 * np.linalg.norm(rd)


@pytest.mark.slow
def test_lobpcg_is_variational_and_monotone():
    w = I.make_workload("c1", D=8)
    T = N.build_ttno(w.tree, w.ham)
    ev = np.linalg.eigvalsh(N.dense_hamiltonian(w.ham))
    blk = w.block()
    X0 = [[t[j] for t in blk] for j in range(w.n_states)]
    lam, X, hist = S.lobpcg(w.tree, T, X0, 3, shift=lambda l: l[0] - 100.0)
    for h in hist[1:]:
        assert np.all(h >= ev[:w.n_states] - 1e-10 * abs(ev[0]))
    for a, b in zip(hist[1:], hist[2:]):
        assert np.all(b <= a + 1e-9 * abs(ev[0]))


@pytest.mark.slow
def test_lobpcg_reaches_the_uncoupled_closed_form():
    omega = np.array([1010.0, 1500.0, 2300.0])
    ham = I.Hamiltonian(dims=[4, 4, 4], omega=omega)
    for i in range(3):
        ham.add(omega[i], {i: "h"})
    tree = I.mps_tree(3, 4)
    bonds = I.uniform_bonds(tree, 16)
    T = N.build_ttno(tree, ham)
    blk = I.initial_block(tree, ham, bonds, 3, seed=0, noise=1e-3)
    X0 = [[t[j] for t in blk] for j in range(3)]
    lam, X, hist = S.lobpcg(tree, T, X0, 4, shift=lambda l: l[0] - 50.0)
    ref = closed.uncoupled_levels(omega, [4, 4, 4], 3)
    assert np.abs(lam - ref).max() <= 1e-10 * ref[0]


def test_minres_stops_at_the_rounding_floor_of_a_converged_shift():
    # (A - s) with s the Rayleigh quotient of a nearly exact eigenvector is singular to working
    # precision: MINRES stops on Paige & Saunders' rounding-level test well before its cap and
    # returns the eigenvector direction to rounding; without the test (eps = 0) the iteration
    # runs to the cap and rounding leaks into the direction
    rng = np.random.default_rng(4)
    n = 60
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = (Q * (3000.0 + np.concatenate([[0.0], np.linspace(50, 5000, n - 1)]))) @ Q.T
    v1 = Q[:, 0]
    worst_without = 0.0
    for noise in (1e-9, 1e-11, 1e-13):
        x = v1 + noise * rng.standard_normal(n)
        x /= np.linalg.norm(x)
        s = x @ A @ x
        for eps in (np.finfo(np.float64).eps, 0.0):
            y, h = S.minres(lambda v: A @ v - s * v, x, x0=x, tol=1e-14, maxiter=300, eps=eps)
            y /= np.linalg.norm(y)
            err = min(np.abs(y - v1).max(), np.abs(y + v1).max())
            if eps > 0:
                assert len(h) < 301 and err <= 1e-13
            else:
                assert len(h) == 301
                worst_without = max(worst_without, err)
    assert worst_without > 1e-11


# --- block inverse iteration (Alg. 3) and its clustering rule (Sec. III.B) --------------------

@pytest.mark.parametrize("lam,gap,blocks", [
    ([0.0, 5.0, 10.0], 5.0, [[0], [1], [2]]),            # a gap equal to the threshold splits
    ([0.0, 4.999, 9.998], 5.0, [[0, 1, 2]]),             # single linkage chains 0 - 4.999 - 9.998
    ([10.0, 0.0, 3.0, 20.0], 5.0, [[1, 2], [0], [3]]),   # unsorted input, blocks in value order
    ([1.0, 1.0, 1.0], 0.5, [[0, 1, 2]]),                 # ties join
    ([1.0, 1.0, 1.0], 0.0, [[0], [1], [2]]),             # gap 0: one state per block
    ([0.0, 1.0, 2.0, 3.0], 10.0, [[0, 1, 2, 3]]),        # one block
    ([7.0, 3.0, 5.0], 1.0, [[1], [2], [0]]),             # all singletons, value order
])
def test_clusters_by_gap_table(lam, gap, blocks):
    assert S.clusters_by_gap(np.array(lam), gap) == blocks


def test_inverse_iteration_is_dense_inverse_iteration_at_full_bond():
    # at full bond (c1, D = 36) one ALS step solves (H - s) y = x exactly, so Alg. 3 with one
    # state is x <- (H - s I)^-1 x / |.| with s the Rayleigh quotient of x, step by step
    w = I.make_workload("c1", D=36)
    H = N.dense_hamiltonian(w.ham)
    T = N.build_ttno(w.tree, w.ham)
    blk = w.block(noise=1e-2)
    for j in (0, 3):
        xs = S.normalize(w.tree, [t[j] for t in blk])
        v = N.ttns_to_dense(w.tree, xs)
        for _ in range(4):
            s = v @ H @ v
            v = np.linalg.solve(H - s * np.eye(len(H)), v)
            v /= np.linalg.norm(v)
            _, X, hist = S.inverse_iteration(w.tree, T, [xs], 1, lambda l: [[0]], als_sweeps=2,
                                             minres_max=400, minres_tol=1e-14)
            xs = X[0]
            xd = N.ttns_to_dense(w.tree, xs)
            assert np.abs(np.sign(xd @ v) * xd - v).max() <= 1e-12
            assert abs(hist[-1][0] - v @ H @ v) <= 1e-13 * abs(v @ H @ v)


@pytest.mark.parametrize("gap", [0.0, 300.0])
def test_inverse_iteration_reaches_the_lowest_dense_eigenvalues(gap):
    # five product-like states at full bond: after six iterations every Rayleigh quotient is one
    # of the five lowest eigenvalues of the dense Hamiltonian to 1e-10 relative, each reached once
    w = I.make_workload("c1", D=36)
    ev = np.linalg.eigvalsh(N.dense_hamiltonian(w.ham))
    T = N.build_ttno(w.tree, w.ham)
    blk = w.block(noise=1e-2)
    X0 = [[t[j] for t in blk] for j in range(5)]
    clusters = (lambda l: [[j] for j in range(len(l))]) if gap <= 0 else \
        (lambda l: S.clusters_by_gap(l, gap))
    lam, _, _ = S.inverse_iteration(w.tree, T, X0, 6, clusters, als_sweeps=2, minres_max=300,
                                    minres_tol=1e-12)
    assert np.abs(np.sort(lam) - ev[:5]).max() <= 1e-10 * ev[0]


def test_block_rayleigh_ritz_is_the_dense_generalized_eigenproblem_at_full_bond():
    # Hc = ESc over five non-orthogonal states (Sec. III.B): at full bond (fitting exact) the
    # Ritz values are the generalized eigenvalues of the dense projections and the new states
    # are orthonormal and diagonalise H
    import scipy.linalg
    w = I.make_workload("c1", D=36)
    T = N.build_ttno(w.tree, w.ham)
    H = N.dense_hamiltonian(w.ham)
    blk = w.block(noise=5e-2)
    X = [[t[j] for t in blk] for j in range(5)]
    V = np.array([N.ttns_to_dense(w.tree, x) for x in X]).T
    ref = scipy.linalg.eigh(V.T @ H @ V, V.T @ V, eigvals_only=True)
    theta, Y = S.block_rayleigh_ritz(w.tree, T, X, fit_sweeps=2)
    assert np.abs(theta - ref).max() <= 1e-10 * abs(ref[0])
    D = np.array([N.ttns_to_dense(w.tree, y) for y in Y]).T
    assert np.abs(D.T @ D - np.eye(5)).max() <= 1e-10
    assert np.abs(D.T @ H @ D - np.diag(theta)).max() <= 1e-9 * abs(ref[0])
