"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and the CPU oracle on the same seeded workload."""
import numpy as np

import workloads as W
from oracle import dgsem_oracle as O


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def gpu_solver(w, dt=0.0):
    from paper_2603_06267_gb300 import dgsem
    return dgsem.Solver(w, dt=dt)


def oracle_problem(w):
    return O.OracleProblem(w)


def run_both(w, precision, drive=None, p0=None, v0=None, nsteps=None, batch=None):
    """Traces of the GPU path and of the oracle for workload w (same dt)."""
    from paper_2603_06267_gb300 import dgsem
    S = w.nsteps if nsteps is None else nsteps
    B = w.batch if batch is None else batch
    P = oracle_problem(w)
    dt = P.stable_dt()
    sol = gpu_solver(w)
    # both sides compute dt from the same CFL reading with their own GLL tables
    assert abs(sol.dt - dt) <= 1e-13 * dt, (sol.dt, dt)
    if drive is None and w.pmuts is not None:
        drive = w.drive(dt, S, B)
    if p0 is not None or v0 is not None:
        dgsem.dgsem_set_state(sol.ctx, p0, v0)
    tg = sol.run(drive=drive, precision=precision, batch=B, nsteps=S)
    pg = dgsem.dgsem_get_pressure(sol.ctx, B, sol.ndof)
    to = P.run(nsteps=S, dt=dt, drive=drive, p0=p0, v0=v0, batch=B)
    po = P.final_state["p"].T
    sol.close()
    return tg, to, pg, po
