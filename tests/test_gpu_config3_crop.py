"""Parity over the full horizon on the cropped config-3 problem.

``workloads.config3_crop``: config 3's first 8x8 block of PMUTs (5 modes,
seeded frequency spread), a 32x32x16 N=4 primary box under a 16x16x96 N=6
secondary box through the 2:1 interface, 6,510,658 nodes, 8000 steps of
Algorithm 1 -- the element types, orders, time step and horizon of the
benchmarked configuration.  The oracle's outputs come from
tests/golden/make_config3_crop_oracle.py (the oracle alone, about an hour of
CPU time) and are compared per output: receiver traces (every 4th step, all
64 receivers), the modal coordinates q every 40 steps, the leapfrog energy
every 400 steps and the final pressure at every 1009th node; FP64 within
1e-10 and FP32-mixed within 1e-4 (relative L2).
"""
import os

import numpy as np
import pytest

import workloads as W
from gpu_helpers import rel_l2

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "config3_crop_oracle.npz")


@pytest.fixture(scope="module")
def golden():
    if not os.path.exists(GOLDEN):
        pytest.fail(f"{GOLDEN} is missing: run tests/golden/make_config3_crop_oracle.py")
    return dict(np.load(GOLDEN))


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-4)])
def test_config3_crop_8000_steps_against_oracle(golden, prec, tol):
    from paper_2603_06267_gb300 import dgsem
    S = int(golden["nsteps"])
    every = int(golden["trace_every"])
    w = W.config3_crop(nsteps=S)
    sol = dgsem.Solver(w)
    dt = float(golden["dt"])
    assert abs(sol.dt - dt) <= 1e-13 * dt
    drive = w.drive(sol.dt, S, 1)
    q_steps = list(golden["q_steps"])
    e_steps = set(int(v) for v in golden["e_steps"])
    chunk = int(q_steps[0])
    K, M = w.pmuts.n_pmut, w.pmuts.n_modes
    tr, qs, es = [], [], []
    for c0 in range(0, S, chunk):
        tr.append(sol.run(drive=np.ascontiguousarray(drive[:, :, c0:c0 + chunk]), precision=prec, nsteps=chunk,
                          flags=dgsem.DGSEM_RUN_CONTINUE if c0 else 0))
        qs.append(dgsem.dgsem_get_pmut_state(sol.ctx, 1, K, M)[0].reshape(-1))
        if c0 + chunk in e_steps:
            es.append(dgsem.dgsem_energy(sol.ctx, 1)[0])
    p = dgsem.dgsem_get_pressure(sol.ctx, 1, sol.ndof)[0]
    sol.close()
    tr = np.concatenate(tr, axis=2)[:, :, every - 1::every]
    ref_tr = golden["traces"]
    assert np.abs(ref_tr).max() > 0
    err_tr = rel_l2(tr, ref_tr)
    per_r = [rel_l2(tr[0, r], ref_tr[0, r]) for r in range(ref_tr.shape[1])]
    err_q = rel_l2(np.array(qs), golden["q"])
    err_e = rel_l2(np.array(es), golden["energy"][:, 0])
    err_p = rel_l2(p[golden["p_nodes"]], golden["p_final"])
    print(f"cropped config 3, {S} steps, precision {prec}: traces {err_tr:.3e} (per receiver max {max(per_r):.3e}), "
          f"q(t) {err_q:.3e}, energy {err_e:.3e}, final field {err_p:.3e}")
    assert err_tr <= tol
    assert err_q <= tol
    assert err_e <= tol
    assert err_p <= tol
