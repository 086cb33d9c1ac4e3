"""Successive randomized compression (SRC) of a TTNO x TTNS product (Sec. II.C.1, Figs. random
tensor and src), restated in FP64 NumPy.

Test infrastructure only (see the package docstring). The random sketch is an input: ``omega[i]``
is the d_i x chi matrix Omega^(i) of node i (``None`` for an auxiliary node, which carries no
factor of the Khatri-Rao product), drawn by the seeded generator ``inputs.src_sketch``.

The steps, in the paper's order:

1. Khatri-Rao sketch (Eq. Khatri-Rao): column k of Omega is the Kronecker product of the k-th
   columns c_k^(i) of every Omega^(i), i.e. the product state omega_k with node tensors
   c_k^(i)[p] on bond-one legs. Contracting the TTNO and the TTNS with it over the physical
   output legs gives, per column k, the ordinary environments of <omega_k| H |x>; the top-down
   ones ("down") sketch everything outside the subtree of an edge (Fig. src steps 2-3).
2. Leaves to root: at node i the neighbouring subtrees already processed provide the residual
   environments R_c = <Q| H |x> of its children; with the down sketch of its parent edge they
   give the local sketch Y_i[k, s_children, p] = (A Omega) of the matrix case (Eq. matrix random
   compression). Its QR factor Q_i over (s_children, p) x k (orthonormal columns, R with a
   non-negative diagonal) is the new node tensor, its column index the new parent bond. When
   (s_children, p) has at most chi values the node keeps its full space: Q_i is the identity.
   Contracting Q_i^dagger with the TTNO and TTNS tensors of node i and the children's R_c gives
   R_i, the B = Q^dagger A of the matrix case for the rest of the traversal (Fig. src step 4).
3. At the root the remaining tensors are contracted directly.

The result is a TTNS whose non-root nodes are isometries toward the root (canonical form with
the centre at the root); its bond on edge i is min(chi, rows_i).
"""
from __future__ import annotations

import numpy as np

from .network import environments, node_contract, postorder


def sketch_states(tree, omega, chi):
    """The chi product states omega_k of the Khatri-Rao sketch (node tensors on bond-one legs)."""
    out = []
    for k in range(chi):
        st = []
        for i in range(tree.n_nodes):
            nl = (1 if tree.parent[i] >= 0 else 0) + len(tree.children(i))
            if tree.phys_dim[i] > 0:
                st.append(omega[i][:, k].reshape((1,) * nl + (-1,)).copy())
            else:
                st.append(np.ones((1,) * nl))
        out.append(st)
    return out


def src_apply(tree, ttno, x, omega, chi, return_sketches=False):
    """Approximate H|x> by SRC with sketch dimension chi. Returns the node tensors of the result
    (and, if asked, the local sketches Y_i of the non-root nodes)."""
    sk = sketch_states(tree, omega, chi)
    down = [environments(tree, ttno, w, x)[1] for w in sk]     # per column k: down[k][edge]
    R, out, Ys = {}, [None] * tree.n_nodes, {}
    for i in postorder(tree):
        ch = tree.children(i)
        if tree.parent[i] < 0:
            envs = {m: R[c] for m, c in enumerate(ch)}
            out[i] = node_contract(tree, ttno, i, x[i], envs)
            continue
        # down sketch of the parent edge with the column index k as its bra bond
        D = np.stack([down[k][i][0] for k in range(chi)])          # [k, w, b]
        envs = {0: D}
        envs.update({m + 1: R[c] for m, c in enumerate(ch)})
        Y = node_contract(tree, ttno, i, x[i], envs)                 # [k, s_children..., (p)]
        Ys[i] = Y
        rest = Y.shape[1:]
        rows = int(np.prod(rest))
        if rows <= chi:
            Q = np.eye(rows)
        else:
            Q, Rm = np.linalg.qr(np.moveaxis(Y, 0, -1).reshape(rows, chi))
            sgn = np.sign(np.diag(Rm))
            sgn[sgn == 0] = 1.0
            Q = Q * sgn
        Qi = np.moveaxis(Q.reshape(rest + (Q.shape[1],)), -1, 0)
        out[i] = Qi
        envs = {m + 1: R[c] for m, c in enumerate(ch)}
        R[i] = node_contract(tree, ttno, i, x[i], envs, bra=Qi, open_leg=0)
    return (out, Ys) if return_sketches else out


def src_bonds(tree, chi):
    """Bond of edge i of the SRC result: min(chi, d_i * prod of the children's bonds)."""
    bond = np.ones(tree.n_nodes, dtype=np.int64)
    for i in postorder(tree):
        if tree.parent[i] < 0:
            continue
        rows = max(int(tree.phys_dim[i]), 1)
        for c in tree.children(i):
            rows *= int(bond[c])
        bond[i] = min(chi, rows)
    return bond
