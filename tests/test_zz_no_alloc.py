"""The no-allocation cell-list entry point against the allocating one.

hse_cell_list_noalloc serves callers that may not let the library allocate
device memory (their own allocator owns the heap, or their loop may not
allocate).  It must give the same integer cell ids, permutation and cell
starts as hse_cell_list, on consecutive calls that reuse its fixed scratch
array, and reject sizes above its capacity.  This file is collected last so
that a failure here does not hide the rest of the suite.
"""
import numpy as np
import pytest

from workloads import KERNEL_S, problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _run_noalloc(hse, pos, box, ncell):
    n = pos.shape[1]
    cid = torch.empty(n, dtype=torch.int32, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    start = torch.empty(int(np.prod(ncell)) + 1, dtype=torch.int32, device="cuda")
    hse.hse_cell_list_noalloc(n, pos.data_ptr(), box, ncell, cid.data_ptr(), perm.data_ptr(), start.data_ptr(),
                              torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return cid.cpu().numpy(), perm.cpu().numpy(), start.cpu().numpy()


def test_noalloc_cell_list_matches_allocating_entry_point():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1802_07844_gb300 as pkg
    from paper_1802_07844_gb300 import hse
    # two calls in a row with different sizes and cell grids: the second must
    # not see anything the first left in the shared scratch array
    cases = [(200_000, "near_wall", 0.07, 40), (3_001, "uniform", 0.2, 41)]
    for n, dist, rc, seed in cases:
        pr = problem(KERNEL_S, n, 1.0, dist, seed)
        pos = torch.from_numpy(pr.src).cuda()
        plan = pkg.Plan(KERNEL_S, (1.0, 1.0, 1.0), xi=5.0 / rc, rc=rc, P=8, tol=0.0)
        ncell = plan.params["ncell"]
        cid, perm, start = plan.cell_list(pos)
        torch.cuda.synchronize()
        ref = (cid.cpu().numpy(), perm.cpu().numpy(), start.cpu().numpy())
        plan.close()
        got = _run_noalloc(hse, pos, (1.0, 1.0, 1.0), ncell)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b)


def test_noalloc_rejects_sizes_above_capacity():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1802_07844_gb300 import hse
    n = hse.HSE_NOALLOC_MAX_POINTS + 1
    pos = torch.zeros((3, n), dtype=torch.float64, device="cuda")
    with pytest.raises(hse.HseError) as e:
        _run_noalloc(hse, pos, (1.0, 1.0, 1.0), (4, 4, 4))
    assert e.value.status == hse.HSE_ERR_INVALID
    assert "capacity" in hse.hse_last_error(None)
