"""dgsem_sample_noalloc: receiver sampling for callers that cannot allocate
device memory (inside a stream capture, under a fixed memory budget, or in a
real-time loop).  It must agree with the traces dgsem_run records for the same
points, call after call.  Kept in its own file, collected last."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-4)])
def test_sample_noalloc_matches_run_traces(prec, tol):
    import torch
    from paper_2603_06267_gb300 import dgsem
    w = W.small_two_domain(nx_p=4, nz_p=2, nx_s=2, nz_s=3, n_pmut_side=2, nsteps=60, batch=2, steer=True)
    sol = dgsem.Solver(w)
    traces = sol.run(precision=prec)            # [batch][R][S]; sample S-1 is the final field
    last = traces[:, :, -1]
    recv = np.ascontiguousarray(w.receivers)
    scale = np.abs(last).max()
    assert scale > 0
    for _ in range(2):                         # two calls in a row share the scratch array
        out = torch.full((2, recv.shape[0]), np.nan, dtype=torch.float64, device="cuda")
        dgsem.dgsem_sample_noalloc(sol.ctx, recv, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.abs(got - last).max() <= tol * scale
    with pytest.raises(dgsem.DgsemError) as e:
        dgsem.dgsem_sample_noalloc(sol.ctx, np.zeros((65, 3)), torch.zeros((2, 65), dtype=torch.float64,
                                                                         device="cuda"))
    assert e.value.code == dgsem.DGSEM_EINVAL and "64" in str(e.value)
    sol.close()
