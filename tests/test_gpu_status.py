"""Status codes of the C ABI on their failure paths, each provoked without a GPU fault: an
allocation that fails (injected on the host, and a real request beyond the device's memory), a
NaN in a host input, a MINRES cap, and a bounded device wait that is made to run out."""
import numpy as np
import pytest

from paper_2512_15875_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ENOMEM, ENONFINITE, ENOTCONV, ETIMEOUT = 2, 4, 5, 6


@pytest.fixture(scope="module")
def T():
    from paper_2512_15875_gb300 import ttn
    ttn.load()
    return ttn


@pytest.fixture(scope="module")
def ctx(T):
    return T.ttn_create(0)


@pytest.fixture(scope="module")
def c1(T, ctx):
    w = I.make_workload("c1", D=8)
    th = T.ttn_tree_create(ctx, w.tree)
    H, _ = T.ttn_build_ttno(ctx, th, w.ham.flat(w.tree))
    return w, th, H


def test_injected_allocation_failure_is_enomem(T, ctx, c1):
    w, th, H = c1
    T.ttn_fault_inject_alloc(0)
    try:
        with pytest.raises(T.TTNError) as e:
            T.ttn_block_create(ctx, th, 3, w.bonds)
        assert e.value.status == ENOMEM and "injected" in str(e.value)
    finally:
        T.ttn_fault_inject_alloc(-1)
    b = T.ttn_block_create(ctx, th, 3, w.bonds)     # injection switched itself off
    assert b.ptr


def test_block_beyond_device_memory_is_enomem(T, ctx, c1):
    w, th, H = c1
    big = I.uniform_bonds(w.tree, 36)
    # 4e7 states x 2664 doubles per state: about 850 GB, beyond any single device
    with pytest.raises(T.TTNError) as e:
        T.ttn_block_create(ctx, th, 40_000_000, big)
    assert e.value.status == ENOMEM
    S, _ = T.ttn_gram(ctx, H, *(2 * [T.block_from_arrays(ctx, th, w.bonds, w.block())]))
    assert np.all(np.isfinite(S))                    # the context stays usable


def test_nan_in_a_host_input_is_enonfinite_from_ttn_gram(T, ctx, c1):
    w, th, H = c1
    blk = w.block()
    blk[2] = blk[2].copy()
    blk[2][1, 0, 0, 0] = np.nan
    b = T.block_from_arrays(ctx, th, w.bonds, blk)
    with pytest.raises(T.TTNError) as e:
        T.ttn_gram(ctx, H, b, b)
    assert e.value.status == ENONFINITE and "results written" in str(e.value)


def test_minres_cap_is_surfaced_as_enotconv(T, ctx, c1):
    w, th, H = c1
    rhs = T.block_from_arrays(ctx, th, w.bonds, w.block())
    y = T.block_from_arrays(ctx, th, w.bonds, w.block())
    st = T.ttn_als_solve(ctx, H, np.full(w.n_states, 1000.0), rhs, y, n_sweeps=1, minres_max=1,
                         minres_tol=1e-14)
    assert st == ENOTCONV
    st = T.ttn_als_solve(ctx, H, np.full(w.n_states, 1000.0), rhs, y, n_sweeps=1,
                         minres_max=200, minres_tol=1e-3)
    assert st == 0


def test_bounded_wait_that_runs_out_is_etimeout(T, ctx, c1):
    w, th, H = c1
    assert T.ttn_selftest_bounded_wait(ctx, 2.0) == ETIMEOUT
    msg = T.load().ttn_last_error(ctx.ptr).decode()
    assert "self-test" in msg
    b = T.block_from_arrays(ctx, th, w.bonds, w.block())
    S, Hm = T.ttn_gram(ctx, H, b, b)                  # the next call sees no stale flag
    assert np.all(np.isfinite(Hm))
