"""FP32-mixed against FP64 at the benchmarked sizes, per output.

The FP64 path is itself compared with the oracle element by element (the
other parity tests, including the cropped config-3 run over 8000 steps); at
the full config-3 / config-4 sizes, where the oracle cannot run, the FP32
path is compared with it.  Outputs: the receiver traces (relative L2 overall
and per receiver), the PMUT modal coordinates q(t) and the leapfrog energy
at checkpoints of the run.
"""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import rel_l2

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-4


def _chunked(sol, w, prec, batch, nsteps, chunk, receivers, drive):
    """Run nsteps in chunks (DGSEM_RUN_CONTINUE), returning the traces and, at
    the end of every chunk, q and the leapfrog energy."""
    from paper_2603_06267_gb300 import dgsem
    tr, qs, es = [], [], []
    for c0 in range(0, nsteps, chunk):
        n = min(chunk, nsteps - c0)
        tr.append(sol.run(drive=np.ascontiguousarray(drive[:batch, :, c0:c0 + n]), precision=prec, batch=batch,
                          nsteps=n, receivers=receivers, flags=dgsem.DGSEM_RUN_CONTINUE if c0 else 0))
        qs.append(dgsem.dgsem_get_pmut_state(sol.ctx, batch, w.pmuts.n_pmut, w.pmuts.n_modes)[0])
        es.append(dgsem.dgsem_energy(sol.ctx, batch))
    return np.concatenate(tr, axis=2), np.array(qs), np.array(es)


def test_config3_fp32_vs_fp64_8000_steps():
    """Config 3 (1024 PMUTs, 102.6M nodes), 8000 steps, 64 receivers at
    z = 2 mm: FP32-mixed traces, q(t) and energy against the FP64 path."""
    from paper_2603_06267_gb300 import dgsem
    w = W.config3_array32(nsteps=8000)
    sol = dgsem.Solver(w)
    drive = w.drive(sol.dt, 8000, 1)
    t64, q64, e64 = _chunked(sol, w, dgsem.DGSEM_FP64, 1, 8000, 1000, w.receivers, drive)
    t32, q32, e32 = _chunked(sol, w, dgsem.DGSEM_FP32_MIXED, 1, 8000, 1000, w.receivers, drive)
    sol.close()
    assert np.abs(t64).max() > 0
    err = rel_l2(t32, t64)
    per_r = [rel_l2(t32[0, r], t64[0, r]) for r in range(t64.shape[1])]
    err_q = rel_l2(q32, q64)
    err_e = rel_l2(e32, e64)
    print(f"config 3, 8000 steps, FP32 vs FP64: traces rel-L2 {err:.3e} (per receiver max {max(per_r):.3e}, "
          f"median {np.median(per_r):.3e}); q(t) at 8 checkpoints {err_q:.3e}; energy {err_e:.3e}")
    assert err <= FP32_TOL
    assert max(per_r) <= 10 * FP32_TOL
    assert err_q <= FP32_TOL
    assert err_e <= FP32_TOL


def test_config4_fp32_64_patterns_vs_fp64_per_pattern():
    """Config 4 (64 steering patterns, FP32 in one batch as benchmarked)
    against FP64 runs of its first 8 patterns, 1000 steps, receivers near
    the array (z = 0.15 mm, primary box) and above the interface (z = 0.5 mm,
    secondary box): relative L2 per pattern."""
    from paper_2603_06267_gb300 import dgsem
    w = W.config4_batched(nsteps=1000)
    g = np.linspace(0.2e-3, 3.0e-3, 8)
    X, Y = np.meshgrid(g, g, indexing="ij")
    rec = np.concatenate([np.stack([X.ravel(), Y.ravel(), np.full(64, z)], axis=1) for z in (0.15e-3, 0.5e-3)])
    sol = dgsem.Solver(w)
    drive = w.drive(sol.dt, 1000, 64)
    t32 = sol.run(drive=drive, precision=dgsem.DGSEM_FP32_MIXED, batch=64, nsteps=1000, receivers=rec)
    q32 = dgsem.dgsem_get_pmut_state(sol.ctx, 64, w.pmuts.n_pmut, w.pmuts.n_modes)[0]
    t64 = sol.run(drive=np.ascontiguousarray(drive[:8]), precision=dgsem.DGSEM_FP64, batch=8, nsteps=1000,
                  receivers=rec)
    q64 = dgsem.dgsem_get_pmut_state(sol.ctx, 8, w.pmuts.n_pmut, w.pmuts.n_modes)[0]
    sol.close()
    errs = [rel_l2(t32[b], t64[b]) for b in range(8)]
    errs_q = [rel_l2(q32[b], q64[b]) for b in range(8)]
    assert min(np.abs(t64[b]).max() for b in range(8)) > 0
    print(f"config 4, 1000 steps, FP32 (batch 64) vs FP64 (batch 8): traces rel-L2 per pattern max "
          f"{max(errs):.3e} median {np.median(errs):.3e}; q per pattern max {max(errs_q):.3e}")
    assert max(errs) <= FP32_TOL
    assert max(errs_q) <= FP32_TOL
    # the patterns differ from each other
    assert rel_l2(t64[0], t64[1]) > 1e-2
