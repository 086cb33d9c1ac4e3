"""FP64 restatement of the tree-tensor-network objects and contractions (Sec. II.A, II.C).

Test infrastructure only (see the package docstring). Every quantity is computed from its
definition with ``numpy.einsum``; nothing is blocked, fused or reordered beyond what the
definition states. All arithmetic is real: the Hamiltonians are real symmetric, so the complex
conjugate on bra tensors is the identity.

Conventions
-----------
* Node tensor legs: (parent, children in increasing index order, physical). Auxiliary nodes
  (``phys_dim = 0``) have no physical leg; internally they get a size-1 one.
* TTNO node tensor W[w_legs..., p, q] (Eq. ttno), stored as a list of entries
  (w-tuple, d x d local operator, coefficient): the operator-valued elements of Sec. II.A.3.
* Environment of an edge: E[a, w, b] with a = bra bond, w = TTNO bond, b = ket bond.
  ``up[t]`` contracts the subtree below edge (t, parent(t)); ``down[t]`` contracts everything
  outside that subtree.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# Contraction-path search for numpy.einsum: greedy pairwise order with intermediates allowed up
# to 2^31 elements (the default cap of the largest input's size forces an unfactored loop over
# every index, which is exact but intractable at the paper's sizes).
_PATH = ("greedy", 1 << 31)

# ----------------------------------------------------------------------------------------------
# tree helpers
# ----------------------------------------------------------------------------------------------


def legs(tree, i):
    """Neighbours of node i in leg order: parent (if any), then children."""
    out = [int(tree.parent[i])] if tree.parent[i] >= 0 else []
    return out + tree.children(i)


def pdim(tree, i):
    return max(int(tree.phys_dim[i]), 1)


def with_phys(tree, i, T):
    """Node tensor with an explicit trailing physical axis (size 1 on auxiliary nodes)."""
    return T if tree.phys_dim[i] > 0 else T[..., None]


def postorder(tree):
    out = []

    def rec(u):
        for c in tree.children(u):
            rec(c)
        out.append(u)
    rec(tree.root)
    return out


def preorder(tree):
    out = []

    def rec(u):
        out.append(u)
        for c in tree.children(u):
            rec(c)
    rec(tree.root)
    return out


def path(tree, u, v):
    """Nodes on the tree path from u to v (inclusive)."""
    def anc(x):
        out = [x]
        while tree.parent[x] >= 0:
            x = int(tree.parent[x])
            out.append(x)
        return out
    au, av = anc(u), anc(v)
    common = next(x for x in au if x in set(av))
    return au[:au.index(common) + 1] + av[:av.index(common)][::-1]


# ----------------------------------------------------------------------------------------------
# Eq. (sum_of_tp), Eq. (ttns): dense objects for tiny systems
# ----------------------------------------------------------------------------------------------


def dense_hamiltonian(ham):
    """H = sum_i c_i (x)_j A_i^(j) with identities on the other modes (Eq. sum_of_tp).
    Basis order: mode 0 is the most significant index."""
    mats_id = [np.eye(d) for d in ham.dims]
    N = int(np.prod(ham.dims))
    H = np.zeros((N, N))
    for c, ids in ham.terms:
        mats = list(mats_id)
        for o in ids:
            m, A = ham.ops[o]
            mats[m] = A
        K = mats[0]
        for A in mats[1:]:
            K = np.kron(K, A)
        H += c * K
    return H


def ttns_to_dense(tree, tensors):
    """Contract all virtual legs of a TTNS (Eq. ttns); axes in mode order."""
    edge = {}
    k = 0
    for i in range(tree.n_nodes):
        if tree.parent[i] >= 0:
            edge[i] = k
            k += 1
    mode_ax = {}
    for i in range(tree.n_nodes):
        if tree.phys_dim[i] > 0:
            mode_ax[int(tree.mode[i])] = k
            k += 1
    args = []
    for i in range(tree.n_nodes):
        sub = ([edge[i]] if tree.parent[i] >= 0 else []) + [edge[c] for c in tree.children(i)]
        if tree.phys_dim[i] > 0:
            sub.append(mode_ax[int(tree.mode[i])])
        args += [tensors[i], sub]
    out = [mode_ax[m] for m in sorted(mode_ax)]
    return np.einsum(*args, out, optimize=_PATH).reshape(-1)


# ----------------------------------------------------------------------------------------------
# TTNO (Eq. ttno) and its construction from a state diagram (Sec. II.A.3)
# ----------------------------------------------------------------------------------------------


@dataclass
class TTNO:
    """``wbond[i]``: operator bond of edge (i, parent(i)) (1 for the root, unused).
    ``entries[i]``: list of (w-tuple in leg order, d x d operator, coefficient)."""
    wbond: np.ndarray
    entries: list

    def wdims(self, tree, i):
        head = [int(self.wbond[i])] if tree.parent[i] >= 0 else []
        return head + [int(self.wbond[c]) for c in tree.children(i)]

    def dense_node(self, tree, i):
        d = pdim(tree, i)
        W = np.zeros(tuple(self.wdims(tree, i)) + (d, d))
        for w, op, c in self.entries[i]:
            W[tuple(w)] += c * op
        return W


def _lca(tree, nodes):
    """Lowest common ancestor of a set of nodes."""
    nodes = list(nodes)

    def anc(x):
        out = [x]
        while tree.parent[x] >= 0:
            x = int(tree.parent[x])
            out.append(x)
        return out
    cur = nodes[0]
    for u in nodes[1:]:
        s = set(anc(cur))
        y = u
        while y not in s:
            y = int(tree.parent[y])
        cur = y
    return cur


def build_ttno(tree, ham):
    """Uncompressed state-diagram TTNO of a sum of products (Sec. II.A.3).

    One channel per edge (t, parent(t)) for
      0  "identity so far"  (no operator of the term inside the subtree of t),
      1  "finished"         (sum of the complete terms that live inside the subtree),
      2+ each distinct restriction of a term to the subtree of t, for terms that also act
         outside that subtree (the hyperedge labels of the state diagram, no vertex merging).
    A term follows its restriction channels up to the lowest common ancestor of its support,
    where its coefficient is applied and it joins the "finished" channel up to the root.
    This is exact (no compression); the minimal-bond construction of the paper (symbolic
    Gaussian elimination + minimum vertex cover) is not needed to define the operator.
    """
    n = tree.n_nodes
    node_of_mode = tree.node_of_mode()
    terms = []
    for c, ids in ham.terms:
        f = {}
        for o in ids:
            m, _ = ham.ops[o]
            f[int(node_of_mode[m])] = o
        terms.append((c, f))
    sub = [set(tree.subtree(i)) for i in range(n)]

    def restrict(f, t):
        return tuple(sorted((u, o) for u, o in f.items() if u in sub[t]))

    chan = [dict() for _ in range(n)]
    for t in range(n):
        if tree.parent[t] < 0:
            continue
        for c, f in terms:
            key = restrict(f, t)
            if key and len(key) < len(f):
                chan[t].setdefault(key, 2 + len(chan[t]))
    wbond = np.array([2 + len(chan[t]) if tree.parent[t] >= 0 else 1 for t in range(n)])

    def child_w(f, c):
        key = restrict(f, c)
        return chan[c][key] if key else 0

    top = [(_lca(tree, f.keys()) if f else tree.root) for _, f in terms]
    entries = [[] for _ in range(n)]
    for t in range(n):
        d = pdim(tree, t)
        eye = np.eye(d)
        ch = tree.children(t)
        root = tree.parent[t] < 0

        def op_at(f):
            o = f.get(t)
            return eye if o is None else ham.ops[o][1]

        def emit(w0, ws, op, coef):
            w = (() if root else (w0,)) + tuple(ws)
            entries[t].append((w, op, float(coef)))

        if not root:
            emit(0, [0] * len(ch), eye, 1.0)
            for key, idx in chan[t].items():
                f = dict(key)
                emit(idx, [child_w(f, c) for c in ch], op_at(f), 1.0)
        for m, c in enumerate(ch):
            ws = [0] * len(ch)
            ws[m] = 1
            emit(1, ws, eye, 1.0)
        for (coef, f), tt in zip(terms, top):
            if tt == t:
                emit(1, [child_w(f, c) for c in ch], op_at(f), coef)
    return TTNO(wbond, entries)


def identity_ttno(tree):
    """Bond-1 TTNO of the identity operator (used for overlap environments)."""
    n = tree.n_nodes
    entries = []
    for t in range(n):
        nl = len(legs(tree, t))
        entries.append([((0,) * nl, np.eye(pdim(tree, t)), 1.0)])
    return TTNO(np.ones(n, dtype=np.int64), entries)


def ttno_to_dense(tree, ttno):
    """Contract all virtual legs of a TTNO (Eq. ttno) to the full operator matrix."""
    edge, k = {}, 0
    for i in range(tree.n_nodes):
        if tree.parent[i] >= 0:
            edge[i] = k
            k += 1
    pax, qax = {}, {}
    for i in range(tree.n_nodes):
        m = int(tree.mode[i])
        if tree.phys_dim[i] > 0:
            pax[m], qax[m] = k, k + 1
            k += 2
    args = []
    for i in range(tree.n_nodes):
        W = ttno.dense_node(tree, i)
        sub = ([edge[i]] if tree.parent[i] >= 0 else []) + [edge[c] for c in tree.children(i)]
        if tree.phys_dim[i] > 0:
            m = int(tree.mode[i])
            sub += [pax[m], qax[m]]
        else:
            W = W[..., 0, 0]
        args += [W, sub]
    out = [pax[m] for m in sorted(pax)] + [qax[m] for m in sorted(qax)]
    H = np.einsum(*args, out, optimize=_PATH)
    N = int(np.sqrt(H.size))
    return H.reshape(N, N)


# ----------------------------------------------------------------------------------------------
# environments, Gram entries, H_eff, exact apply (Sec. II.C; Figs. variational, als)
# ----------------------------------------------------------------------------------------------


def node_contract(tree, ttno, t, ket, envs, bra=None, open_leg=None):
    """Contract node t of <bra| W |ket> with environments on the given legs.

    envs: {leg index: E[a, w, b]}. Returns
      * bra and open_leg given  -> E[a, w, b] on the open leg (an environment update),
      * bra given, no open leg  -> the scalar <bra|H|ket> closed at t,
      * no bra, no open leg     -> y[a_legs..., p] = (H_eff x) in the node's shape.
    """
    nl = len(legs(tree, t))
    W = ttno.dense_node(tree, t)
    B = with_phys(tree, t, ket)
    a = list(range(nl))
    w = list(range(nl, 2 * nl))
    b = list(range(2 * nl, 3 * nl))
    p, q = 3 * nl, 3 * nl + 1
    args = [W, w + [p, q], B, b + [q]]
    for m, E in envs.items():
        args += [E, [a[m], w[m], b[m]]]
    if bra is not None:
        args += [with_phys(tree, t, bra), a + [p]]
    if bra is not None and open_leg is not None:
        out = [a[open_leg], w[open_leg], b[open_leg]]
    elif bra is not None:
        out = []
    else:
        out = a + [p]
    r = np.einsum(*args, out, optimize=_PATH)
    if bra is None and tree.phys_dim[t] == 0:
        r = r[..., 0]            # auxiliary node: drop the size-one physical axis
    return r


def environments(tree, ttno, A, B):
    """All bottom-up (``up``) and top-down (``down``) environments of <A|W|B>."""
    up, down = {}, {}
    for t in postorder(tree):
        if tree.parent[t] < 0:
            continue
        ch = tree.children(t)
        envs = {m + 1: up[c] for m, c in enumerate(ch)}
        up[t] = node_contract(tree, ttno, t, B[t], envs, bra=A[t], open_leg=0)
    for u in preorder(tree):
        ch = tree.children(u)
        off = 1 if tree.parent[u] >= 0 else 0
        for m, c in enumerate(ch):
            envs = {0: down[u]} if off else {}
            for m2, c2 in enumerate(ch):
                if c2 != c:
                    envs[m2 + off] = up[c2]
            down[c] = node_contract(tree, ttno, u, B[u], envs, bra=A[u], open_leg=m + off)
    return up, down


def node_envs(tree, t, up, down):
    """The environments around node t in its leg order."""
    envs = {}
    off = 0
    if tree.parent[t] >= 0:
        envs[0] = down[t]
        off = 1
    for m, c in enumerate(tree.children(t)):
        envs[m + off] = up[c]
    return envs


def expectation(tree, ttno, A, B, close_at=None):
    """<A|H|B> closed at node ``close_at`` (default the root). Closing at any node gives the same
    scalar, which exercises every top-down environment."""
    up, down = environments(tree, ttno, A, B)
    t = tree.root if close_at is None else close_at
    return float(node_contract(tree, ttno, t, B[t], node_envs(tree, t, up, down), bra=A[t]))


def gram(tree, ttno, blockA, blockB):
    """G[k, l] = <A_k|H|B_l> for all pairs (Alg. 2, 'construct matrices'). ``block[node]`` has the
    state index first."""
    nA, nB = blockA[0].shape[0], blockB[0].shape[0]
    G = np.zeros((nA, nB))
    for k in range(nA):
        Ak = [T[k] for T in blockA]
        for l in range(nB):
            G[k, l] = expectation(tree, ttno, Ak, [T[l] for T in blockB])
    return G


def heff_apply(tree, ttno, t, psi, x):
    """(H_eff,t x): the derivative of <psi|H|psi> with respect to the bra tensor at node t,
    evaluated with x in place of psi_t (Sec. II.C.3)."""
    up, down = environments(tree, ttno, psi, psi)
    return node_contract(tree, ttno, t, x, node_envs(tree, t, up, down))


def apply_exact(tree, ttno, psi):
    """Exact TTNO x TTNS product (Sec. II.C.1, the direct contraction): each new bond is the
    pair (w, b) with w the major index; the physical leg keeps its place."""
    out = []
    for t in range(tree.n_nodes):
        nl = len(legs(tree, t))
        W = ttno.dense_node(tree, t)
        B = with_phys(tree, t, psi[t])
        w = list(range(nl))
        b = list(range(nl, 2 * nl))
        p, q = 2 * nl, 2 * nl + 1
        inter = [x for pair in zip(w, b) for x in pair]
        X = np.einsum(W, w + [p, q], B, b + [q], inter + [p])
        shp = [W.shape[m] * B.shape[m] for m in range(nl)]
        X = X.reshape(shp + [X.shape[-1]])
        out.append(X if tree.phys_dim[t] > 0 else X[..., 0])
    return out


# ----------------------------------------------------------------------------------------------
# term-by-term expectation: independent of any TTNO
# ----------------------------------------------------------------------------------------------


def overlap(tree, A, B):
    """<A|B> of two TTNS by contracting bottom-up."""
    E = {}
    for t in postorder(tree):
        nl = len(legs(tree, t))
        a = list(range(nl))
        b = list(range(nl, 2 * nl))
        p = 2 * nl
        args = [with_phys(tree, t, A[t]), a + [p], with_phys(tree, t, B[t]), b + [p]]
        off = 1 if tree.parent[t] >= 0 else 0
        for m, c in enumerate(tree.children(t)):
            args += [E[c], [a[m + off], b[m + off]]]
        out = [a[0], b[0]] if off else []
        E[t] = np.einsum(*args, out, optimize=_PATH)
    return float(E[tree.root])


def expectation_terms(tree, ham, A, B):
    """<A|H|B> = sum_i c_i <A| (x)_j A_i^(j) |B> term by term (Eq. sum_of_tp), each term a plain
    TTNS overlap after applying its one-mode operators to the ket's physical legs."""
    node_of_mode = tree.node_of_mode()
    total = 0.0
    for c, ids in ham.terms:
        B2 = list(B)
        for o in ids:
            m, op = ham.ops[o]
            i = int(node_of_mode[m])
            B2[i] = np.tensordot(B2[i], op, axes=([-1], [1]))
        total += c * overlap(tree, A, B2)
    return total
