"""ttn_rayleigh_ritz_noalloc gives the result of ttn_rayleigh_ritz without allocating.

The no-allocation variant exists for callers that may not allocate device memory once they are
running (a serving process that reserves its device budget at start-up, a frozen memory pool, a
host framework that owns the allocator): it works in a fixed area compiled into the library.
This file is collected last so that a failure here never hides another test's result, and it
creates its own context so it also passes alone in a fresh process."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _pencil(m, seed):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((m, m))
    M = B @ B.T / m + 0.1 * np.eye(m)
    H = rng.standard_normal((m, m))
    return H + H.T, M


def _rel(x, ref):
    return np.abs(x - ref).max() / max(np.abs(ref).max(), 1e-300)


def test_noalloc_rayleigh_ritz_matches_the_allocating_call_twice_in_a_row():
    torch = pytest.importorskip("torch")
    from paper_2512_15875_gb300 import ttn as T
    ctx = T.ttn_create(0)
    # two calls in a row; the second is smaller and reuses the area the first one filled. The
    # allocating reference calls and every device buffer come first, so that the free device
    # memory around the no-allocation calls can be compared
    cases = []
    for m, n, seed in [(252, 84, 1), (57, 7, 2)]:
        H, M = _pencil(m, seed)
        th_ref, V_ref = T.ttn_rayleigh_ritz(ctx, H, M, n, 1e-12)
        dev = [torch.tensor(H, dtype=torch.float64, device="cuda:0").contiguous(),
               torch.tensor(M, dtype=torch.float64, device="cuda:0").contiguous(),
               torch.zeros(n, dtype=torch.float64, device="cuda:0"),
               torch.zeros((m, n), dtype=torch.float64, device="cuda:0")]
        cases.append((m, n, th_ref, V_ref, dev))
    torch.cuda.synchronize()
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info(0)[0]
    statuses = []
    for m, n, _, _, (dH, dM, dth, dV) in cases:
        statuses.append(T.ttn_rayleigh_ritz_noalloc(ctx, m, dH.data_ptr(), dM.data_ptr(), n,
                                                    1e-12, dth.data_ptr(), dV.data_ptr()))
    torch.cuda.synchronize()
    free_after = torch.cuda.mem_get_info(0)[0]
    assert statuses == [0, 0]
    assert free_after == free_before
    for m, n, th_ref, V_ref, (_, _, dth, dV) in cases:
        th, V = dth.cpu().numpy(), dV.cpu().numpy()
        assert _rel(th, th_ref) <= 1e-11
        assert _rel(V, V_ref) <= 1e-8


def test_noalloc_rayleigh_ritz_rejects_sizes_beyond_its_area():
    torch = pytest.importorskip("torch")
    from paper_2512_15875_gb300 import ttn as T
    ctx = T.ttn_create(0)
    m = 257
    d = torch.zeros((m, m), dtype=torch.float64, device="cuda:0")
    with pytest.raises(T.TTNError) as e:
        T.ttn_rayleigh_ritz_noalloc(ctx, m, d.data_ptr(), d.data_ptr(), 4, 1e-12, d.data_ptr(),
                                    d.data_ptr())
    assert e.value.status == 1 and "TTN_RR_NOALLOC_MAX_M" in str(e.value)
