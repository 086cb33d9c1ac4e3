"""Full-size parity of the block Gram: the 12-mode QFF on the fork-4 tree (D = 24, 84 states, the
benchmark workload), the 64-mode coupled-oscillator model on an MPS (D = 32, 40 states) and on
the leaf-only binary tree (bonds 6..48, 64 states), and the 12-mode QFF on the all-physical
binary tree (D = 32, 84 states). Sampled entries of the
GPU Gram (built with the library's compressed TTNO) against the oracle's environment contraction
with its own, independently constructed state-diagram TTNO; both represent the same Hamiltonian
(Eq. sum_of_tp), so agreement checks the builder and the kernels together.
FP64 1e-11 relative to the largest diagonal entry; FP32 2e-5."""
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
@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3"])
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
