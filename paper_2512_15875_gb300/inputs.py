"""Seeded synthetic workloads: trees, sum-of-products Hamiltonians and initial block states.

This module is the one piece shared by the FP64 oracle and the CUDA path. It only *draws and
lays out inputs*; none of the eigensolver's arithmetic lives here.

Hamiltonians are sums of products of one-mode operators (Sec. II.A.3, Eq. (sum_of_tp)):

    H = sum_t c_t  prod_{k in term t} A_k          (one operator per mode at most)

One-mode operators are written in the harmonic-oscillator finite basis of d functions
(|0>..|d-1>): the harmonic part of mode i is omega_i * diag(n + 1/2), the coordinate is the
truncated q = (a + a^dagger)/sqrt(2) and q^k is the k-th matrix power of that truncated q
(which is what a d-point Gauss-Hermite quadrature gives). With this reading the uncoupled
spectrum sum_i omega_i (n_i + 1/2) is exact for every n_i <= d-1 (Sec. III.A and the basis
paragraph that follows Eq. (coupled_harmonic_oscillator)).

Workloads (all seeded with numpy.random.default_rng):

* ``c1``  4 coupled oscillators, d=6, MPS, D=8 (or 36), n=5  -- the small dense-checkable case.
* ``c2``  12-mode acetonitrile-like quartic force field, d=9, fork-4 tree, D=24, n=84 (Sec. III.B,
          term counts 12 + 108 + 191 = 311).
* ``c3``  64 coupled oscillators with cubic terms, d=6, MPS, D=32, n=40 (Sec. III.A shapes).
* ``c4``  the same Hamiltonian on a leaf-only perfect binary tree, uneven bonds 6..48, n=64.
* ``c5``  the ``c2`` Hamiltonian on an all-physical binary tree, D=32, n=84.
* ``uniform64`` the paper's own 64-D model: omega_j = sqrt(j/2), alpha_ij = 0.1 (Sec. III.A).
"""
from __future__ import annotations

import heapq
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Tree", "Hamiltonian", "Workload",
    "ho_matrices", "mps_tree", "fork_tree", "t_tree", "leaf_only_binary_tree",
    "all_physical_binary_tree",
    "cap_bonds", "uniform_bonds", "coupled_oscillators", "quartic_force_field",
    "uniform_coupled_model", "lowest_harmonic_configurations", "initial_block",
    "make_workload", "WORKLOADS", "src_sketch",
]


# ----------------------------------------------------------------------------------------------
# trees
# ----------------------------------------------------------------------------------------------
@dataclass
class Tree:
    """Rooted tree. ``parent[root] = -1``; ``phys_dim[i] = 0`` marks an auxiliary node.

    ``mode[i]`` is the vibrational mode carried by node i (-1 for auxiliary nodes). Children of a
    node are kept in increasing node-index order; node tensors order their legs as
    (parent, children..., physical).
    """
    parent: np.ndarray
    phys_dim: np.ndarray
    mode: np.ndarray
    name: str = ""

    def __post_init__(self):
        self.parent = np.asarray(self.parent, dtype=np.int32)
        self.phys_dim = np.asarray(self.phys_dim, dtype=np.int32)
        self.mode = np.asarray(self.mode, dtype=np.int32)

    @property
    def n_nodes(self) -> int:
        return int(self.parent.shape[0])

    @property
    def root(self) -> int:
        return int(np.flatnonzero(self.parent < 0)[0])

    def children(self, i: int) -> list[int]:
        return [int(c) for c in np.flatnonzero(self.parent == i)]

    def subtree(self, i: int) -> list[int]:
        out, stack = [], [i]
        while stack:
            u = stack.pop()
            out.append(u)
            stack.extend(self.children(u))
        return sorted(out)

    def node_of_mode(self) -> np.ndarray:
        n_modes = int(self.mode.max()) + 1
        out = np.full(n_modes, -1, dtype=np.int32)
        for i, m in enumerate(self.mode):
            if m >= 0:
                out[m] = i
        return out


def mps_tree(n_modes: int, d: int) -> Tree:
    """Linear chain (MPS); node 0 is the root, node i carries mode i."""
    parent = [-1] + list(range(n_modes - 1))
    return Tree(parent, [d] * n_modes, list(range(n_modes)), name=f"mps{n_modes}")


def fork_tree(n_backbone: int, chain_len: int, d: int) -> Tree:
    """Fork-n tree (comb): a chain of auxiliary backbone nodes, each carrying a chain of
    ``chain_len`` physical nodes (Appendix B, fork-4 figure). Node 0 (first backbone node) is the
    root; backbone node b+1 hangs off backbone node b; chain k's first node hangs off backbone
    node k and each next chain node off the previous one."""
    parent, phys, mode = [], [], []
    for b in range(n_backbone):
        parent.append(b - 1 if b > 0 else -1)
        phys.append(0)
        mode.append(-1)
    m = 0
    for b in range(n_backbone):
        prev = b
        for _ in range(chain_len):
            parent.append(prev)
            phys.append(d)
            mode.append(m)
            prev = len(parent) - 1
            m += 1
    return Tree(parent, phys, mode, name=f"fork{n_backbone}x{chain_len}")


def t_tree(n_modes: int, d: int) -> Tree:
    """T tree (Appendix B): an auxiliary centre node (node 0, the root) with three chains of
    physical nodes hanging off it; the modes are split into three nearly equal consecutive runs
    and each chain starts at the mode next to the centre (the end of its run for the first
    chain, the start for the others, as in the figure of the 64-mode T tree)."""
    sizes = [n_modes // 3 + (1 if k < n_modes % 3 else 0) for k in range(3)]
    runs, m0 = [], 0
    for sz in sizes:
        runs.append(list(range(m0, m0 + sz)))
        m0 += sz
    runs[0] = runs[0][::-1]
    parent, phys, mode = [-1], [0], [-1]
    for run in runs:
        prev = 0
        for m in run:
            parent.append(prev)
            phys.append(d)
            mode.append(m)
            prev = len(parent) - 1
    return Tree(parent, phys, mode, name=f"ttree{n_modes}")


def leaf_only_binary_tree(depth: int, d: int) -> Tree:
    """Perfect binary tree whose 2**depth leaves carry the modes; internal nodes are auxiliary
    (ML-MCTDH-style leaf-only tree). Breadth-first numbering: node k has children 2k+1, 2k+2."""
    n_int = 2 ** depth - 1
    n = 2 ** (depth + 1) - 1
    parent = [-1] + [(k - 1) // 2 for k in range(1, n)]
    phys = [0] * n_int + [d] * (n - n_int)
    mode = [-1] * n_int + list(range(n - n_int))
    return Tree(parent, phys, mode, name=f"leafbin{depth}")


def all_physical_binary_tree(n_modes: int, d: int) -> Tree:
    """Balanced binary tree in breadth-first order where every node carries a mode (node k has
    children 2k+1 and 2k+2 when those exist)."""
    parent = [-1] + [(k - 1) // 2 for k in range(1, n_modes)]
    return Tree(parent, [d] * n_modes, list(range(n_modes)), name=f"physbin{n_modes}")


def _phys_product(tree: Tree, nodes) -> int:
    p = 1
    for u in nodes:
        if tree.phys_dim[u] > 0:
            p *= int(tree.phys_dim[u])
    return p


def cap_bonds(tree: Tree, target: np.ndarray) -> np.ndarray:
    """Bond of edge (i, parent(i)) = min(target[i], phys product below, phys product above).

    Larger bonds than these products cannot carry more information (the exact-rank bound of the
    bipartition). ``bond[root]`` is set to 1 (the root has no parent leg)."""
    n = tree.n_nodes
    out = np.ones(n, dtype=np.int64)
    total = _phys_product(tree, range(n))
    for i in range(n):
        if tree.parent[i] < 0:
            continue
        below = _phys_product(tree, tree.subtree(i))
        out[i] = min(int(target[i]), below, total // below)
    return out.astype(np.int32)


def uniform_bonds(tree: Tree, D: int) -> np.ndarray:
    return cap_bonds(tree, np.full(tree.n_nodes, D))


def depth_bonds(tree: Tree, per_depth: dict[int, int]) -> np.ndarray:
    """Bond by the depth of the child node of each edge (root depth 0)."""
    depth = np.zeros(tree.n_nodes, dtype=np.int64)
    for i in range(tree.n_nodes):
        u, k = i, 0
        while tree.parent[u] >= 0:
            u, k = int(tree.parent[u]), k + 1
        depth[i] = k
    return cap_bonds(tree, np.array([per_depth.get(int(k), 1) for k in depth]))


# ----------------------------------------------------------------------------------------------
# Hamiltonians
# ----------------------------------------------------------------------------------------------
def ho_matrices(d: int) -> dict[str, np.ndarray]:
    """One-mode matrices in the d-function harmonic-oscillator basis (see module docstring)."""
    n = np.arange(d, dtype=np.float64)
    q = np.zeros((d, d))
    off = np.sqrt((n[:-1] + 1.0) / 2.0)
    q[np.arange(d - 1), np.arange(1, d)] = off
    q[np.arange(1, d), np.arange(d - 1)] = off
    out = {"h": np.diag(n + 0.5), "q": q}
    qk = q.copy()
    for k in range(2, 5):
        qk = qk @ q
        out[f"q{k}"] = qk.copy()
    return out


@dataclass
class Hamiltonian:
    """H = sum_t coef[t] * prod_{o in terms[t]} ops[o]; ops[o] = (mode, d x d matrix)."""
    dims: list[int]
    ops: list[tuple[int, np.ndarray]] = field(default_factory=list)
    terms: list[tuple[float, tuple[int, ...]]] = field(default_factory=list)
    omega: np.ndarray | None = None
    name: str = ""
    _op_index: dict = field(default_factory=dict, repr=False)

    @property
    def n_modes(self) -> int:
        return len(self.dims)

    def op(self, mode: int, kind: str) -> int:
        key = (mode, kind)
        if key not in self._op_index:
            self._op_index[key] = len(self.ops)
            self.ops.append((mode, ho_matrices(self.dims[mode])[kind]))
        return self._op_index[key]

    def add(self, coef: float, factors: dict[int, str]):
        ids = tuple(self.op(m, k) for m, k in sorted(factors.items()))
        self.terms.append((float(coef), ids))

    def add_monomial(self, coef: float, modes) -> None:
        """coef * prod q_m over a multiset of modes (repeats become powers of q)."""
        cnt: dict[int, int] = {}
        for m in modes:
            cnt[int(m)] = cnt.get(int(m), 0) + 1
        self.add(coef, {m: ("q" if k == 1 else f"q{k}") for m, k in cnt.items()})

    def flat(self, tree: Tree) -> dict:
        """Flat arrays for the C ABI: ops are attached to tree *nodes* (row-major d x d data)."""
        node_of_mode = tree.node_of_mode()
        op_site = np.array([node_of_mode[m] for m, _ in self.ops], dtype=np.int32)
        sizes = [mat.size for _, mat in self.ops]
        op_offset = np.zeros(len(self.ops) + 1, dtype=np.int64)
        op_offset[1:] = np.cumsum(sizes)
        op_data = np.concatenate([mat.ravel() for _, mat in self.ops]).astype(np.float64)
        coeff = np.array([c for c, _ in self.terms], dtype=np.float64)
        lens = [len(ids) for _, ids in self.terms]
        term_offset = np.zeros(len(self.terms) + 1, dtype=np.int32)
        term_offset[1:] = np.cumsum(lens)
        term_op_ids = np.array([o for _, ids in self.terms for o in ids], dtype=np.int32)
        return dict(op_site=op_site, op_offset=op_offset, op_data=op_data, coeff=coeff,
                    term_offset=term_offset, term_op_ids=term_op_ids)


def coupled_oscillators(n_modes, d, omega, pair_k, cubic=(), name=""):
    """sum_i omega_i (n_i + 1/2) + sum_{i<j} k_ij q_i q_j + sum c * prod q over cubic multisets."""
    h = Hamiltonian(dims=[d] * n_modes, omega=np.asarray(omega, dtype=np.float64), name=name)
    for i in range(n_modes):
        h.add(omega[i], {i: "h"})
    for (i, j), k in pair_k:
        h.add_monomial(k, (i, j))
    for modes, c in cubic:
        h.add_monomial(c, modes)
    return h


def quartic_force_field(seed: int, d: int = 9, n_cubic: int = 108, n_quartic: int = 191):
    """12-mode acetonitrile-like QFF (Sec. III.B shapes): 12 harmonic + 108 cubic + 191 quartic
    product terms in reduced normal coordinates, cm^-1. Frequencies: 4 low U[350,1100],
    4 mid U[1300,1500], 4 high U[2200,3100]; modes 1 and 5 are made degenerate with modes 0 and
    4. Cubic multisets i<=j<=k and quartic multisets i<=j<=k<=l are drawn uniformly without
    replacement; coefficients N(0, 30^2) and N(0, 3^2)."""
    rng = np.random.default_rng(seed)
    omega = np.concatenate([rng.uniform(350, 1100, 4), rng.uniform(1300, 1500, 4),
                            rng.uniform(2200, 3100, 4)])
    omega[1] = omega[0]
    omega[5] = omega[4]
    L = 12
    cub = [(i, j, k) for i in range(L) for j in range(i, L) for k in range(j, L)]
    qua = [(i, j, k, l) for i in range(L) for j in range(i, L) for k in range(j, L)
           for l in range(k, L)]
    ci = rng.choice(len(cub), size=n_cubic, replace=False)
    qi = rng.choice(len(qua), size=n_quartic, replace=False)
    cc = rng.normal(0.0, 30.0, n_cubic)
    qc = rng.normal(0.0, 3.0, n_quartic)
    h = Hamiltonian(dims=[d] * L, omega=omega, name=f"qff12_s{seed}")
    for i in range(L):
        h.add(omega[i], {i: "h"})
    for t, c in zip(sorted(ci), cc):
        h.add_monomial(c, cub[t])
    for t, c in zip(sorted(qi), qc):
        h.add_monomial(c, qua[t])
    return h


def four_mode_model(seed: int, d: int = 6):
    """4 coupled oscillators: omega ~ U[1000,3000] cm^-1, k_ij ~ N(0,50^2) on the 6 pairs,
    c_ijk ~ N(0,5^2) on the 4 triples i<j<k."""
    rng = np.random.default_rng(seed)
    L = 4
    omega = rng.uniform(1000, 3000, L)
    pairs = [(i, j) for i in range(L) for j in range(i + 1, L)]
    k = rng.normal(0.0, 50.0, len(pairs))
    trip = [(i, j, l) for i in range(L) for j in range(i + 1, L) for l in range(j + 1, L)]
    c = rng.normal(0.0, 5.0, len(trip))
    return coupled_oscillators(L, d, omega, list(zip(pairs, k)), list(zip(trip, c)),
                               name=f"osc4_s{seed}")


def sixtyfour_mode_model(seed: int, d: int = 6, n_modes: int = 64):
    """64 coupled oscillators (a.u.): omega ~ U[0.5,2], k_ij ~ N(0,(0.1 wbar)^2) on all pairs,
    one cubic c_iij q_i^2 q_j per mode with a random partner j != i, c ~ N(0,(0.02 wbar)^2)."""
    rng = np.random.default_rng(seed)
    L = n_modes
    omega = rng.uniform(0.5, 2.0, L)
    wbar = float(omega.mean())
    pairs = [(i, j) for i in range(L) for j in range(i + 1, L)]
    k = rng.normal(0.0, 0.1 * wbar, len(pairs))
    partner = [(i + 1 + int(rng.integers(L - 1))) % L for i in range(L)]
    c = rng.normal(0.0, 0.02 * wbar, L)
    cubic = [((i, i, partner[i]), c[i]) for i in range(L)]
    return coupled_oscillators(L, d, omega, list(zip(pairs, k)), cubic,
                               name=f"osc{L}_s{seed}")


def uniform_coupled_model(n_modes: int = 64, d: int = 8, alpha: float = 0.1):
    """The paper's bilinear model: omega_j = sqrt(j/2) (j = 1..L), alpha_ij = alpha (Sec. III.A)."""
    omega = np.sqrt(np.arange(1, n_modes + 1) / 2.0)
    pairs = [((i, j), alpha) for i in range(n_modes) for j in range(i + 1, n_modes)]
    return coupled_oscillators(n_modes, d, omega, pairs, name=f"uniform{n_modes}")


# ----------------------------------------------------------------------------------------------
# initial block
# ----------------------------------------------------------------------------------------------
def lowest_harmonic_configurations(omega, dims, n):
    """The n occupation vectors with the lowest sum_i omega_i (n_i + 1/2) (ties broken by the
    lexicographic order of the occupation vector), by best-first enumeration."""
    omega = np.asarray(omega, dtype=np.float64)
    L = len(dims)
    start = (0,) * L
    key = lambda v: (float(np.dot(omega, np.asarray(v) + 0.5)), v)
    heap = [key(start)]
    seen = {start}
    out = []
    while heap and len(out) < n:
        e, v = heapq.heappop(heap)
        out.append(v)
        for i in range(L):
            if v[i] + 1 < dims[i]:
                w = v[:i] + (v[i] + 1,) + v[i + 1:]
                if w not in seen:
                    seen.add(w)
                    heapq.heappush(heap, key(w))
    return out


def node_shape(tree: Tree, bonds: np.ndarray, i: int) -> tuple[int, ...]:
    """Leg order (parent, children in index order, physical)."""
    shp = []
    if tree.parent[i] >= 0:
        shp.append(int(bonds[i]))
    shp += [int(bonds[c]) for c in tree.children(i)]
    if tree.phys_dim[i] > 0:
        shp.append(int(tree.phys_dim[i]))
    return tuple(shp)


def initial_block(tree: Tree, ham: Hamiltonian, bonds, n, seed, noise=1e-3):
    """Product states of the n lowest harmonic configurations embedded at the full bonds (bond
    index 0 carries the product state, other entries zero), plus seeded N(0, noise^2) entries
    everywhere. Returns ``block[node]`` = array of shape (n, *node_shape)."""
    rng = np.random.default_rng(seed)
    cfgs = lowest_harmonic_configurations(ham.omega, ham.dims, n)
    block = []
    for i in range(tree.n_nodes):
        shp = node_shape(tree, bonds, i)
        t = np.zeros((n,) + shp)
        for s, v in enumerate(cfgs):
            idx = [0] * len(shp)
            if tree.phys_dim[i] > 0:
                idx[-1] = v[tree.mode[i]]
            t[(s,) + tuple(idx)] = 1.0
        t += noise * rng.standard_normal(t.shape)
        block.append(t)
    return block


def random_block(tree: Tree, bonds, n, seed, scale=1.0):
    """Dense N(0, scale^2) node tensors (for contraction tests)."""
    rng = np.random.default_rng(seed)
    return [scale * rng.standard_normal((n,) + node_shape(tree, bonds, i))
            for i in range(tree.n_nodes)]


def src_sketch(tree: Tree, chi: int, seed: int):
    """The random matrices of the Khatri-Rao sketch of SRC (Sec. II.C.1): Omega^(i) of size
    d_i x chi with N(0, 1) entries for every node with a physical leg, None for auxiliary
    nodes."""
    rng = np.random.default_rng(seed)
    return [rng.standard_normal((int(tree.phys_dim[i]), chi)) if tree.phys_dim[i] > 0 else None
            for i in range(tree.n_nodes)]


# ----------------------------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    tree: Tree
    ham: Hamiltonian
    bonds: np.ndarray
    n_states: int
    seed: int
    description: str = ""

    def block(self, noise=1e-3):
        return initial_block(self.tree, self.ham, self.bonds, self.n_states, self.seed, noise)


def make_workload(name: str, seed: int = 0, **kw) -> Workload:
    if name == "c1":
        D = kw.get("D", 8)
        tree = mps_tree(4, 6)
        return Workload(name, tree, four_mode_model(seed), uniform_bonds(tree, D),
                        kw.get("n", 5), seed, f"4 coupled oscillators, d=6, MPS, D={D}")
    if name == "c2":
        D = kw.get("D", 24)
        tree = fork_tree(4, 3, 9)
        return Workload(name, tree, quartic_force_field(seed), uniform_bonds(tree, D),
                        kw.get("n", 84), seed, f"12-mode QFF, d=9, fork-4, D={D}")
    if name == "c3":
        D = kw.get("D", 32)
        L = kw.get("L", 64)
        tree = mps_tree(L, 6)
        return Workload(name, tree, sixtyfour_mode_model(seed, n_modes=L),
                        uniform_bonds(tree, D), kw.get("n", 40), seed,
                        f"{L} coupled oscillators, d=6, MPS, D={D}")
    if name == "c4":
        depth = kw.get("depth", 6)
        tree = leaf_only_binary_tree(depth, 6)
        per_depth = {depth: 6, depth - 1: 8, depth - 2: 16, depth - 3: 24, depth - 4: 32,
                     depth - 5: 48}
        return Workload(name, tree, sixtyfour_mode_model(seed, n_modes=2 ** depth),
                        depth_bonds(tree, per_depth), kw.get("n", 64), seed,
                        "64 coupled oscillators, d=6, leaf-only binary tree, bonds 6..48")
    if name == "c5":
        D = kw.get("D", 32)
        tree = all_physical_binary_tree(12, 9)
        return Workload(name, tree, quartic_force_field(seed), uniform_bonds(tree, D),
                        kw.get("n", 84), seed, f"12-mode QFF, d=9, all-physical binary, D={D}")
    raise KeyError(name)


WORKLOADS = ("c1", "c2", "c3", "c4", "c5")
