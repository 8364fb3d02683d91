"""The allocation-free restriction-set entry point (edfa_qsets_noalloc).

Some callers cannot allocate device memory once they are running (a host
program whose own pool or fixed budget owns the GPU, or one that cannot take
the device-wide synchronisation of cudaMalloc mid-run).  This entry point
builds the restriction sets with working memory from a fixed device array
inside the library.  Its sets must equal, bit for bit, the ones the
allocating path (edfa_build) computes, on consecutive calls, and a problem too
large for the fixed array or an output buffer too small must be rejected with
EDFA_ERR_BOUNDS.
"""
import numpy as np
import pytest

import workloads as W
from helpers import gpu_handle

pytestmark = pytest.mark.gpu

EDFA_ERR_INVALID = 1
EDFA_ERR_BOUNDS = 7


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _full_tensor(n, seed):
    s = W.Stream(seed)
    Ne = int(np.prod(n))
    m = np.exp(2.0 * s.normal(Ne))
    q = s.normal(4 * Ne).reshape(Ne, 4)
    return W.assemble(*n, W.rotated_K(m, 0.1, q))


@pytest.mark.parametrize("mode", ["nbr", "thresh", "own", "crow"])
def test_noalloc_sets_equal_allocating_path_on_two_calls(mode):
    torch = _torch()
    import paper_2009_13916_gb300 as P
    cases = [_full_tensor((11, 9, 7), 41), W.config3(20, 16, 5)]
    for sysd in cases:
        h = gpu_handle(sysd, mode=mode)
        ref = h.tensors()
        ref_ptr = ref["qptr"].cpu().numpy()
        ref_idx = ref["qidx"].cpu().numpy()
        h.close()
        A, B, C, D = P.system_to_device(sysd)
        for call in range(2):
            qptr = torch.full((sysd.Ne + 1,), -5, dtype=torch.int64, device="cuda")
            qidx = torch.full((int(ref_ptr[-1]) + 17,), -9, dtype=torch.int32, device="cuda")
            rc, tot = P.qsets_noalloc(A, B, C, sysd.Nf, sysd.Ne, qmode=mode, thresh=0.05, qptr=qptr, qidx=qidx)
            torch.cuda.synchronize()
            assert rc == 0, (call, rc, P.lib().edfa_last_error_detail())
            assert tot == ref_ptr[-1]
            assert np.array_equal(qptr.cpu().numpy(), ref_ptr)
            assert np.array_equal(qidx[:tot].cpu().numpy(), ref_idx)
            assert np.all(qidx[tot:].cpu().numpy() == -9)


def test_noalloc_rejects_small_output_and_oversized_problem():
    torch = _torch()
    import ctypes

    import paper_2009_13916_gb300 as P
    sysd = _full_tensor((6, 5, 4), 42)
    A, B, C, D = P.system_to_device(sysd)
    qptr = torch.empty(sysd.Ne + 1, dtype=torch.int64, device="cuda")
    qidx = torch.full((10,), -9, dtype=torch.int32, device="cuda")
    rc, tot = P.qsets_noalloc(A, B, C, sysd.Nf, sysd.Ne, qmode="nbr", qptr=qptr, qidx=qidx)
    torch.cuda.synchronize()
    assert rc == EDFA_ERR_BOUNDS and tot > 10
    assert P.lib().edfa_last_error_detail() == tot
    assert np.all(qidx.cpu().numpy() == -9)
    # a problem needing more than the fixed array is rejected before any device
    # work (the descriptors claim 20M cells; nothing is read from them)
    big_ne, big_nf = 20_000_000, 61_000_000
    dA = P.Csr(big_nf, big_nf, 1, A[0].data_ptr(), A[1].data_ptr(), A[2].data_ptr())
    dB = P.Csr(big_nf, big_ne, 1, B[0].data_ptr(), B[1].data_ptr(), B[2].data_ptr())
    dC = P.Csr(big_ne, big_nf, 1, C[0].data_ptr(), C[1].data_ptr(), C[2].data_ptr())
    t = ctypes.c_int64(0)
    rc = P.lib().edfa_qsets_noalloc(ctypes.byref(dA), ctypes.byref(dB), ctypes.byref(dC), 1, 0.05,
                                    qptr.data_ptr(), qidx.data_ptr(), 10, ctypes.byref(t), None)
    assert rc == EDFA_ERR_BOUNDS
    assert P.lib().edfa_last_error_detail() > (64 << 20)


def test_noalloc_rejects_invalid_blocks_then_recovers():
    """Blocks whose indices are in range but invalid (columns out of order in a
    row, a row pointer not starting at 0, A without a stored diagonal) are
    rejected with EDFA_ERR_INVALID before any kernel reads through them; the
    next valid call still gives the allocating path's sets."""
    torch = _torch()
    import paper_2009_13916_gb300 as P
    sysd = _full_tensor((7, 6, 5), 43)
    h = gpu_handle(sysd, mode="nbr")
    ref = h.tensors()
    ref_ptr = ref["qptr"].cpu().numpy()
    ref_idx = ref["qidx"].cpu().numpy()
    h.close()
    A, B, C, D = P.system_to_device(sysd)
    qptr = torch.empty(sysd.Ne + 1, dtype=torch.int64, device="cuda")
    qidx = torch.full((int(ref_ptr[-1]),), -9, dtype=torch.int32, device="cuda")

    def call(Ab, Bb, Cb):
        rc, tot = P.qsets_noalloc(Ab, Bb, Cb, sysd.Nf, sysd.Ne, qmode="nbr", qptr=qptr, qidx=qidx)
        torch.cuda.synchronize()
        return rc

    # columns of one row of C swapped (both still inside [0, N_f))
    row = 3
    c_col = C[1].clone()
    a, b = int(sysd.C.rowptr[row]), int(sysd.C.rowptr[row]) + 1
    c_col[a], c_col[b] = C[1][b].item(), C[1][a].item()
    assert call(A, B, (C[0], c_col, C[2])) == EDFA_ERR_INVALID
    assert P.lib().edfa_last_error_detail() == row
    # row pointer of B not starting at 0 (every entry still a valid offset)
    b_ptr = B[0].clone()
    b_ptr[0] = 1
    assert call(A, (b_ptr, B[1], B[2]), C) == EDFA_ERR_INVALID
    # A without a stored diagonal in one row: its diagonal column replaced by a
    # free column between its neighbours, so the row stays ascending and in range
    a_col = None
    for r in range(sysd.Nf):
        p0, p1 = int(sysd.A.rowptr[r]), int(sysd.A.rowptr[r + 1])
        cols = [int(c) for c in sysd.A.col[p0:p1]]
        d = cols.index(r)
        lo = cols[d - 1] if d > 0 else -1
        hi = cols[d + 1] if d + 1 < len(cols) else sysd.Nf
        free = [c for c in range(lo + 1, hi) if c != r]
        if free:
            a_col = A[1].clone()
            a_col[p0 + d] = free[0]
            break
    assert a_col is not None
    assert call((A[0], a_col, A[2]), B, C) == EDFA_ERR_INVALID
    assert P.lib().edfa_last_error_detail() == r
    assert np.all(qidx.cpu().numpy() == -9)
    # a valid call afterwards
    assert call(A, B, C) == 0
    assert np.array_equal(qptr.cpu().numpy(), ref_ptr)
    assert np.array_equal(qidx.cpu().numpy(), ref_idx)
