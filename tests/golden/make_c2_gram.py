"""Writes tests/golden/c2_gram_252.npz from the FP64 oracle only.

    python tests/golden/make_c2_gram.py [processes]

The complete 252 x 252 Gram matrices H~_kl = <s_k|H|s_l> and M~_kl = <s_k|s_l> (Alg. 2,
"construct matrices") of the 12-mode quartic force field on the fork-4 tree at D = 24, for two
seeded 252-state blocks (the size of the LOBPCG subspace, 3 x 84 states):

* ``prod``: product states of the 252 lowest harmonic configurations plus N(0, 1e-2^2) noise
  (``inputs.initial_block``, seed 0);
* ``rand``: dense N(0, 0.11^2) node tensors (``inputs.random_block``, seed 7), scaled so that
  the norms are of order one.

Each entry is the oracle's bottom-up contraction of the network (environments of Sec. II.C,
closed at the root) with the oracle's own state-diagram TTNO; M~ uses the plain TTNS overlap.
Only the upper triangles (k <= l, row-major) are stored. Pairs are spread over worker processes
(spawn); each worker uses one BLAS thread."""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

N_STATES = 252
RAND_SCALE = 0.11
OUT = os.path.join(HERE, "c2_gram_252.npz")


def blocks():
    from paper_2512_15875_gb300 import inputs as I
    w = I.make_workload("c2")
    prod = I.initial_block(w.tree, w.ham, w.bonds, N_STATES, seed=0, noise=1e-2)
    rand = I.random_block(w.tree, w.bonds, N_STATES, seed=7, scale=RAND_SCALE)
    return w, {"prod": prod, "rand": rand}


def _upward_value(N, tree, ttno, A, B):
    """<A|H|B> from the bottom-up environments only, closed at the root."""
    up = {}
    for t in N.postorder(tree):
        if tree.parent[t] < 0:
            continue
        envs = {m + 1: up[c] for m, c in enumerate(tree.children(t))}
        up[t] = N.node_contract(tree, ttno, t, B[t], envs, bra=A[t], open_leg=0)
    r = tree.root
    envs = {m: up[c] for m, c in enumerate(tree.children(r))}
    return float(N.node_contract(tree, ttno, r, B[r], envs, bra=A[r]))


_STATE = {}


def _init():
    from oracle import network as N
    w, blks = blocks()
    _STATE.update(N=N, w=w, blks=blks, ttno=N.build_ttno(w.tree, w.ham))


def _row(job):
    name, k = job
    N, w, blk, ttno = _STATE["N"], _STATE["w"], _STATE["blks"][name], _STATE["ttno"]
    A = [x[k] for x in blk]
    h, s = [], []
    for l in range(k, N_STATES):
        B = [x[l] for x in blk]
        h.append(_upward_value(N, w.tree, ttno, A, B))
        s.append(N.overlap(w.tree, A, B))
    return name, k, h, s


def main():
    import multiprocessing as mp

    import numpy as np
    procs = int(sys.argv[1]) if len(sys.argv) > 1 else (os.cpu_count() or 1)
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    jobs = [(name, k) for name in ("prod", "rand") for k in range(N_STATES)]
    jobs.sort(key=lambda j: j[1])   # long rows (small k) first
    out = {f"{n}_{m}": np.zeros((N_STATES, N_STATES)) for n in ("prod", "rand") for m in "HS"}
    with mp.get_context("spawn").Pool(procs, initializer=_init) as pool:
        for done, (name, k, h, s) in enumerate(pool.imap_unordered(_row, jobs), 1):
            out[f"{name}_H"][k, k:] = h
            out[f"{name}_S"][k, k:] = s
            if done % 50 == 0:
                print(f"{done}/{len(jobs)} rows", flush=True)
    iu = np.triu_indices(N_STATES)
    np.savez(OUT, n_states=N_STATES, rand_scale=RAND_SCALE,
             **{k: v[iu] for k, v in out.items()})
    print("wrote", OUT)


if __name__ == "__main__":
    main()
