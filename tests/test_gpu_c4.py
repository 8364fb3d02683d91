"""The batched workload at its full scale: 256 independent systems, grid edges
n ~ U{16..48} (about 10.6M cells and 43M unknowns), one handle over the
block-diagonal concatenation, lock-step FGMRES per system under a CUDA graph
(Sec. 3, Remark 5: the local solves of all systems are independent).

FP64: on a seeded subset of 16 systems, each system's restriction sets and S~
pattern bit-exact, X~ and S~ within 1e-10 and the FGMRES iteration count within
1 of the oracle run on that system alone; every one of the 256 systems at true
relative residual <= 1e-8 on its own right-hand side.  FP32-mixed (FP32 local
solves, S~, factors and application, FP64 Krylov): every system converged to
1e-8, iteration counts close to the FP64 ones."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import TOL_FP64, gpu_handle, normwise_cols_fast

pytestmark = pytest.mark.gpu

NSUB = 16


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def subset(nsys, k, seed=4040):
    """k distinct system indices out of nsys (seeded partial Fisher-Yates)."""
    u = W.Stream(seed).uniform(k)
    perm = np.arange(nsys)
    for j in range(k):
        r = j + int(u[j] * (nsys - j))
        perm[j], perm[r] = perm[r], perm[j]
    return np.sort(perm[:k])


def residuals(systems, fo, co, x):
    out = []
    for i, s in enumerate(systems):
        xi = W.sub_vector(x, systems, fo, co, i)
        out.append(np.linalg.norm(s.full_scipy() @ xi - s.b) / np.linalg.norm(s.b))
    return np.array(out)


def test_config4_full_scale():
    torch = _torch()
    systems = W.config4()
    assert len(systems) == 256
    big, fo, co = W.concat(systems)
    b = torch.as_tensor(big.b, device="cuda")

    h = gpu_handle(big, mode="nbr", precision=0)
    t = h.tensors()
    x, it64, tr64, cycles, rc = h.solve_batched(fo, co, b, restart=50, rtol=1e-8, maxit=2000)
    assert rc == 0
    x64 = x.cpu().numpy()
    res = residuals(systems, fo, co, x64)
    assert res.max() <= 1.05e-8 and tr64.max() <= 1e-8, (res.max(), tr64.max())

    qptr = t["qptr"]
    sptr = t["s_rowptr"]
    for i in subset(len(systems), NSUB):
        s = systems[i]
        ref = O.edfa_pipeline(s, mode="nbr", solve=True)
        c0, c1 = int(co[i]), int(co[i + 1])
        a, e = int(qptr[c0]), int(qptr[c1])
        gptr = (qptr[c0:c1 + 1] - a).cpu().numpy()
        gidx = (t["qidx"][a:e].long() - int(fo[i])).cpu().numpy()
        assert np.array_equal(gptr, ref["qptr"]) and np.array_equal(gidx, ref["qidx"]), i
        assert normwise_cols_fast(t["xval"][a:e].cpu().numpy(), ref["xval"], ref["qptr"]) <= TOL_FP64, i
        sa, se = int(sptr[c0]), int(sptr[c1])
        assert np.array_equal((sptr[c0:c1 + 1] - sa).cpu().numpy(), ref["S"].rowptr), i
        assert np.array_equal((t["s_col"][sa:se].long() - c0).cpu().numpy(), ref["S"].col), i
        assert normwise_cols_fast(t["s_val"][sa:se].cpu().numpy(), ref["S"].val, ref["S"].rowptr) <= TOL_FP64, i
        assert ref["converged"] and abs(int(it64[i]) - ref["iters"]) <= 1, (i, int(it64[i]), ref["iters"])
    del t
    h.close()

    h32 = gpu_handle(big, mode="nbr", precision=1)
    x, it32, tr32, cycles, rc = h32.solve_batched(fo, co, b, restart=50, rtol=1e-8, maxit=2000)
    assert rc == 0
    res32 = residuals(systems, fo, co, x.cpu().numpy())
    assert res32.max() <= 1.05e-8 and tr32.max() <= 1e-8, (res32.max(), tr32.max())
    assert np.all(it32 <= it64 * 1.25 + 2), (it32, it64)
    h32.close()
