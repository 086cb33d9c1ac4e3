"""FP64 restatement of the TTN eigensolver steps (Sec. II.B, II.C).

Test infrastructure only (see the package docstring). Environments are recomputed from scratch
for every local step: slow, and obviously the definition.

Readings of points the paper leaves open:
* gauge: the solution TTNS is kept in canonical form with the orthogonality centre at the node
  being updated (QR moves, R with a non-negative diagonal), so the fitting metric is I and ALS
  solves (H_eff - s I) y_t = b_t;
* sweep: nodes in depth-first pre-order from the root, the centre moved along the tree path
  between consecutive nodes;
* MINRES warm-starts from the current node tensor and stops at |r| <= tol * |b| or maxiter;
* LOBPCG (Alg. 2): x_j <- sum_{k=1}^{3n} v_kj s_k then normalised, p_j <- sum_{k>n} v_kj s_k,
  iteration 1 uses S = {x} u {r}; the Gram pencil is solved by canonical orthogonalisation
  (drop eigenvalues of M below eps * max);
* fitting starts from the input state with the largest |coefficient| (first one on ties);
* Ritz vectors carry a fixed sign: their largest-magnitude entry is positive.
"""
from __future__ import annotations

import numpy as np

from .network import (environments, expectation, identity_ttno, legs, node_contract,
                      node_envs, overlap, path, postorder, preorder, with_phys)

# ----------------------------------------------------------------------------------------------
# MINRES (Paige & Saunders 1975), used for the local solves (Sec. II.C.2-3)
# ----------------------------------------------------------------------------------------------


def minres(matvec, b, x0=None, tol=1e-5, maxiter=10, eps=np.finfo(np.float64).eps):
    """Minimum-residual Krylov solve of A x = b for symmetric (possibly indefinite) A.

    Lanczos three-term recurrence for T_k, QR of T_k by Givens rotations, and the update of x by
    the direction vectors w_k. Returns (x, residual norms |phibar_k| starting with the initial
    residual), which is non-increasing by construction.

    Stopping (Paige & Saunders 1975): |phibar_k| <= tol * |b|, a Lanczos breakdown
    (beta_{k+1} = 0), maxiter steps, or the residual at the rounding level of the iterate,
    |phibar_k| <= eps * (|T_k|_F * |x_k| + |b|) with |T_k|_F^2 = sum_j (alpha_j^2 + beta_j^2 +
    beta_{j+1}^2): past that point the computed residual no longer describes x_k and further
    steps only add rounding. Inverse iteration with a converged Rayleigh-quotient shift (Alg. 3)
    meets it: (A - s) is then singular to working precision and x_k grows along the eigenvector.
    """
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - matvec(x) if x0 is not None else b.copy()
    bnorm = float(np.linalg.norm(b))
    beta1 = float(np.linalg.norm(r))
    hist = [beta1]
    if beta1 == 0.0 or bnorm == 0.0:
        return x, hist
    v_prev = np.zeros_like(b)
    v = r / beta1
    beta = beta1
    c1, s1, c2, s2 = 1.0, 0.0, 1.0, 0.0
    w_prev = np.zeros_like(b)
    w_prev2 = np.zeros_like(b)
    phibar = beta1
    tnorm2 = 0.0
    for _ in range(maxiter):
        p = matvec(v)
        alpha = float(np.vdot(v, p))
        p = p - alpha * v - beta * v_prev
        beta_next = float(np.linalg.norm(p))
        tnorm2 += alpha * alpha + beta * beta + beta_next * beta_next
        epsk = s2 * beta
        dtil = c2 * beta
        delta = c1 * dtil + s1 * alpha
        gtil = -s1 * dtil + c1 * alpha
        gamma = float(np.hypot(gtil, beta_next))
        if gamma == 0.0:
            break
        c, s = gtil / gamma, beta_next / gamma
        tau = c * phibar
        phibar = -s * phibar
        w = (v - delta * w_prev - epsk * w_prev2) / gamma
        x = x + tau * w
        hist.append(abs(phibar))
        c2, s2, c1, s1 = c1, s1, c, s
        w_prev2, w_prev = w_prev, w
        if beta_next == 0.0 or abs(phibar) <= tol * bnorm:
            break
        if abs(phibar) <= eps * (np.sqrt(tnorm2) * float(np.linalg.norm(x)) + bnorm):
            break
        v_prev, v = v, p / beta_next
        beta = beta_next
    return x, hist


# ----------------------------------------------------------------------------------------------
# gauge: QR moves of the orthogonality centre (Sec. II.A.1 tensor splitting)
# ----------------------------------------------------------------------------------------------


def qr_pos(M):
    """Reduced QR with a non-negative diagonal of R (makes Q unique for full-rank M)."""
    Q, R = np.linalg.qr(M)
    sgn = np.sign(np.diag(R))
    sgn[sgn == 0] = 1.0
    return Q * sgn, R * sgn[:, None]


def qr_toward(tree, psi, u, v):
    """Split node u by QR with the leg toward the neighbour v as the column index; u keeps Q
    (an isometry pointing at v) and R is absorbed into v's leg toward u."""
    m = legs(tree, u).index(v)
    T = np.moveaxis(with_phys(tree, u, psi[u]), m, -1)
    shp = T.shape
    Q, R = qr_pos(T.reshape(-1, shp[-1]))
    if Q.shape[1] != shp[-1]:
        raise ValueError("bond larger than the rest of the node: raise the bond caps")
    Tq = np.moveaxis(Q.reshape(shp), -1, m)
    psi[u] = Tq if tree.phys_dim[u] > 0 else Tq[..., 0]
    mv = legs(tree, v).index(u)
    Tv = np.moveaxis(np.tensordot(R, with_phys(tree, v, psi[v]), axes=([1], [mv])), 0, mv)
    psi[v] = Tv if tree.phys_dim[v] > 0 else Tv[..., 0]


def canonicalize(tree, psi):
    """Bring a TTNS to canonical form with the orthogonality centre at the root (in place)."""
    for c in postorder(tree):
        if tree.parent[c] >= 0:
            qr_toward(tree, psi, c, int(tree.parent[c]))
    return tree.root


def move_center(tree, psi, src, dst):
    p = path(tree, src, dst)
    for a, b in zip(p[:-1], p[1:]):
        qr_toward(tree, psi, a, b)
    return dst


def normalize(tree, psi):
    nrm = np.sqrt(overlap(tree, psi, psi))
    out = [T.copy() for T in psi]
    out[tree.root] = out[tree.root] / nrm
    return out


# ----------------------------------------------------------------------------------------------
# ALS (Sec. II.C.3) and variational fitting (Sec. II.C.2)
# ----------------------------------------------------------------------------------------------


def als_solve(tree, ttno, shift, rhs, y0, n_sweeps=2, minres_max=10, minres_tol=1e-5):
    """Solve (H - shift I) y = rhs with y a TTNS of y0's bonds by alternating local solves.

    At node t (the orthogonality centre) the local system is
        (H_eff,t - shift) y_t = b_t,   b_t = <y without t | rhs>,
    solved by MINRES. Returns the new node tensors."""
    idt = identity_ttno(tree)
    y = [T.copy() for T in y0]
    c = canonicalize(tree, y)
    for _ in range(n_sweeps):
        for t in preorder(tree):
            c = move_center(tree, y, c, t)
            upH, dnH = environments(tree, ttno, y, y)
            envH = node_envs(tree, t, upH, dnH)
            upS, dnS = environments(tree, idt, y, rhs)
            b = node_contract(tree, idt, t, rhs[t], node_envs(tree, t, upS, dnS))

            def mv(v, envH=envH, t=t):
                return node_contract(tree, ttno, t, v, envH) - shift * v
            y[t], _ = minres(mv, b, x0=y[t], tol=minres_tol, maxiter=minres_max)
    return y


def fit(tree, terms, psi0, n_sweeps=2):
    """Variational fitting of psi ~ sum_i c_i O_i phi_i (Sec. II.C.2): in canonical gauge the
    local solution is the right-hand side sum_i c_i <psi without t| O_i |phi_i> itself.

    terms: list of (coefficient, TTNO, phi)."""
    psi = [T.copy() for T in psi0]
    c = canonicalize(tree, psi)
    for _ in range(n_sweeps):
        for t in preorder(tree):
            c = move_center(tree, psi, c, t)
            acc = 0.0
            for coef, op, phi in terms:
                up, dn = environments(tree, op, psi, phi)
                acc = acc + coef * node_contract(tree, op, t, phi[t], node_envs(tree, t, up, dn))
            psi[t] = acc
    return psi


def fit_initial(terms):
    """The input state of the term with the largest |coefficient|."""
    k = int(np.argmax([abs(c) for c, _, _ in terms]))
    return terms[k][2]


# ----------------------------------------------------------------------------------------------
# Rayleigh-Ritz and block LOBPCG (Alg. 2, Eq. lobpcg update)
# ----------------------------------------------------------------------------------------------


def rayleigh_ritz(Ht, Mt, n, eps=1e-12):
    """Smallest n solutions of Ht v = theta Mt v by canonical orthogonalisation of Mt."""
    Ht = 0.5 * (Ht + Ht.T)
    Mt = 0.5 * (Mt + Mt.T)
    mu, U = np.linalg.eigh(Mt)
    keep = mu > eps * mu.max()
    X = U[:, keep] / np.sqrt(mu[keep])
    theta, Y = np.linalg.eigh(X.T @ Ht @ X)
    V = X @ Y
    return theta[:n], _sign_fixed(V[:, :n])


def _sign_fixed(V):
    """Eigenvectors are defined up to sign; fix it so that the entry of largest magnitude
    (first one on ties) of each column is positive."""
    V = V.copy()
    for j in range(V.shape[1]):
        k = int(np.argmax(np.abs(V[:, j])))
        if V[k, j] < 0:
            V[:, j] = -V[:, j]
    return V


def gram_block(tree, ttno, states):
    """H~_kl = <s_k|H|s_l>, M~_kl = <s_k|s_l> over the subspace (Alg. 2)."""
    m = len(states)
    Ht = np.zeros((m, m))
    Mt = np.zeros((m, m))
    for k in range(m):
        for l in range(k, m):
            Ht[k, l] = Ht[l, k] = expectation(tree, ttno, states[k], states[l])
            Mt[k, l] = Mt[l, k] = overlap(tree, states[k], states[l])
    return Ht, Mt


def lobpcg(tree, ttno, X0, n_iter, shift, als_sweeps=2, minres_max=10, minres_tol=1e-5,
           fit_sweeps=2, callback=None):
    """Block LOBPCG on TTNS (Alg. 2) with the ALS preconditioner (Eq. precondition).

    ``shift`` is a function of the current Ritz values returning the preconditioner shift s.
    Returns (Ritz values, states, per-iteration Ritz values)."""
    idt = identity_ttno(tree)
    n = len(X0)
    X = [normalize(tree, x) for x in X0]
    lam = np.array([expectation(tree, ttno, x, x) / overlap(tree, x, x) for x in X])
    P = []
    hist = [lam.copy()]
    for _ in range(n_iter):
        s = shift(lam)
        R = []
        for j in range(n):
            terms = [(1.0, ttno, X[j]), (-lam[j], idt, X[j])]
            r = fit(tree, terms, X[j], fit_sweeps)
            R.append(als_solve(tree, ttno, s, r, r, als_sweeps, minres_max, minres_tol))
        S = X + R + P
        Ht, Mt = gram_block(tree, ttno, S)
        theta, V = rayleigh_ritz(Ht, Mt, n)
        Xn, Pn = [], []
        for j in range(n):
            tx = [(V[k, j], idt, S[k]) for k in range(len(S))]
            Xn.append(normalize(tree, fit(tree, tx, fit_initial(tx), fit_sweeps)))
            tp = [(V[k, j], idt, S[k]) for k in range(n, len(S))]
            Pn.append(fit(tree, tp, fit_initial(tp), fit_sweeps))
        X, P, lam = Xn, Pn, theta
        hist.append(lam.copy())
        if callback is not None:
            callback(lam, X)
    return lam, X, hist


def clusters_by_gap(lam, gap):
    """Single-linkage clusters of the Rayleigh quotients: sorted values closer than ``gap`` join
    (Sec. III.B: states whose Rayleigh quotients differ by less than 5 cm^-1 form one block)."""
    order = [int(i) for i in np.argsort(lam, kind="stable")]
    out = [[order[0]]]
    for a, b in zip(order[:-1], order[1:]):
        if lam[b] - lam[a] < gap:
            out[-1].append(b)
        else:
            out.append([b])
    return [sorted(c) for c in out]


def inverse_iteration(tree, ttno, X0, n_iter, clusters, als_sweeps=1, minres_max=10000,
                      minres_tol=1e-5, fit_sweeps=2):
    """Block inverse iteration (Alg. 3, Eq. inverse iteration update). ``clusters`` maps the
    current Rayleigh quotients to a list of blocks (lists of state indices); each block uses the
    mean Rayleigh quotient of its states as the shift, every state is solved by ALS, and a block
    of more than one state is re-orthogonalised by its own Rayleigh-Ritz step.
    Returns (Rayleigh quotients, states, per-iteration values)."""
    idt = identity_ttno(tree)
    n = len(X0)
    X = [normalize(tree, x) for x in X0]
    lam = np.array([expectation(tree, ttno, x, x) for x in X])
    hist = [lam.copy()]
    for _ in range(n_iter):
        blocks = clusters(lam)
        shift = np.zeros(n)
        for c in blocks:
            shift[c] = np.mean(lam[c])
        Y = [normalize(tree, als_solve(tree, ttno, shift[j], X[j], X[j], als_sweeps, minres_max,
                                       minres_tol)) for j in range(n)]
        Xn, lam_n = list(Y), lam.copy()
        for c in blocks:
            if len(c) == 1:
                j = c[0]
                lam_n[j] = expectation(tree, ttno, Y[j], Y[j])
                continue
            Ht, Mt = gram_block(tree, ttno, [Y[j] for j in c])
            theta, V = rayleigh_ritz(Ht, Mt, len(c))
            for a, j in enumerate(c):
                tx = [(V[b, a], idt, Y[c[b]]) for b in range(len(c))]
                Xn[j] = normalize(tree, fit(tree, tx, fit_initial(tx), fit_sweeps))
                lam_n[j] = theta[a]
        X, lam = Xn, lam_n
        hist.append(lam.copy())
    return lam, X, hist


def block_rayleigh_ritz(tree, ttno, X, fit_sweeps=2, eps=1e-12):
    """The generalized eigenvalue problem Hc = ESc over all states (Sec. III.B): Gram matrices
    over X, canonical orthogonalisation, each state replaced by its fitted and normalised Ritz
    vector (fitting starts from the input state of the largest |coefficient|).
    Returns (Ritz values, states)."""
    idt = identity_ttno(tree)
    Ht, Mt = gram_block(tree, ttno, X)
    theta, V = rayleigh_ritz(Ht, Mt, len(X), eps)
    out = []
    for a in range(len(X)):
        tx = [(V[b, a], idt, X[b]) for b in range(len(X))]
        out.append(normalize(tree, fit(tree, tx, fit_initial(tx), fit_sweeps)))
    return theta, out
