"""dgsem_sample_noalloc: receiver sampling for callers that cannot allocate
device memory (their device memory belongs to another allocator, or to a
fixed budget).  It must agree with the traces dgsem_run records for the same
points, call after call, and refuse bad arguments without writing anything.
Kept in its own file, collected last."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

# The sample and the run's last trace sample interpolate the same stored field
# (FP64 or FP32) with FP64 weights; only the weights' rounding differs (the run
# builds them on the host, the sampling call on the device), so the two agree
# to a few FP64 ulps of the largest term in both precisions.
REL_TOL = 1e-12


def _solver_and_last_sample(prec):
    from paper_2603_06267_gb300 import dgsem
    w = W.small_two_domain(nx_p=4, nz_p=2, nx_s=2, nz_s=3, n_pmut_side=2, nsteps=60, batch=2, steer=True)
    sol = dgsem.Solver(w)
    traces = sol.run(precision=prec)            # [batch][R][S]; sample S-1 is the final field
    return w, sol, traces[:, :, -1]


@pytest.mark.parametrize("prec", [0, 1])
def test_sample_noalloc_matches_run_traces(prec):
    import torch
    from paper_2603_06267_gb300 import dgsem
    w, sol, last = _solver_and_last_sample(prec)
    recv = np.ascontiguousarray(w.receivers)
    scale = np.abs(last).max()
    assert scale > 0
    for _ in range(2):                         # two calls in a row share the scratch array
        out = torch.full((2, recv.shape[0]), np.nan, dtype=torch.float64, device="cuda")
        dgsem.dgsem_sample_noalloc(sol.ctx, recv, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.abs(got - last).max() <= REL_TOL * scale
    sol.close()


def test_sample_noalloc_refusals_leave_context_usable():
    import torch
    from paper_2603_06267_gb300 import dgsem
    w, sol, last = _solver_and_last_sample(1)
    recv = np.ascontiguousarray(w.receivers)
    R = recv.shape[0]
    # more receivers than the table holds
    with pytest.raises(dgsem.DgsemError) as e:
        dgsem.dgsem_sample_noalloc(sol.ctx, np.zeros((65, 3)), torch.zeros((2, 65), dtype=torch.float64,
                                                                         device="cuda"))
    assert e.value.code == dgsem.DGSEM_EINVAL and "64" in str(e.value)
    # an output buffer shorter than [batch][R] is refused before anything is written
    short = torch.full((1, R), 7.0, dtype=torch.float64, device="cuda")
    with pytest.raises(dgsem.DgsemError) as e:
        dgsem.dgsem_sample_noalloc(sol.ctx, recv, short)
    assert e.value.code == dgsem.DGSEM_EINVAL
    torch.cuda.synchronize()
    assert torch.all(short == 7.0)
    # the binding refuses a tensor of the wrong type outright
    with pytest.raises(TypeError):
        dgsem.dgsem_sample_noalloc(sol.ctx, recv, torch.zeros((2, R), dtype=torch.float32, device="cuda"))
    # a receiver outside the mesh: DGSEM_EINVAL naming it
    bad = recv.copy()
    bad[3] = (-1e-3, 0.5e-4, 0.5e-4)
    with pytest.raises(dgsem.DgsemError) as e:
        dgsem.dgsem_sample_noalloc(sol.ctx, bad, torch.zeros((2, R), dtype=torch.float64, device="cuda"))
    assert e.value.code == dgsem.DGSEM_EINVAL and "receiver 3" in str(e.value)
    # ... after which the context and the call still work
    out = torch.full((2, R), np.nan, dtype=torch.float64, device="cuda")
    dgsem.dgsem_sample_noalloc(sol.ctx, recv, out)
    torch.cuda.synchronize()
    assert np.abs(out.cpu().numpy() - last).max() <= REL_TOL * np.abs(last).max()
    tr = sol.run(precision=1)
    assert np.abs(tr[:, :, -1] - last).max() == 0.0
    sol.close()
