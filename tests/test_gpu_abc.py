"""First-order absorbing sides (damping form d of eq. Wf_4) on the GPU path
against the oracle: every tile variant, both precisions, the two-box PMUT
workload, and the argument checks of dgsem_set_absorbing."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import rel_l2, run_both, gpu_solver, oracle_problem

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
FP32_TOL = 1e-4


@pytest.mark.parametrize("prec,tol", [(0, FP64_TOL), (1, FP32_TOL)])
@pytest.mark.parametrize("N,nel", [(4, (40, 9, 3)), (6, (20, 5, 3))])
def test_absorbing_sides_every_tile_variant(prec, tol, N, nel):
    """Five absorbing sides (x-, x+, y-, y+, z+): the x- node, the last-x
    column, edge and corner nodes all carry C/M; seeded initial state."""
    from paper_2603_06267_gb300 import dgsem
    h = 25e-6
    dom = W.Domain((0, 0, 0), tuple(n * h for n in nel), nel, N, absorbing=(1, 1, 1, 1, 0, 1))
    rec = np.random.default_rng(3).uniform(0, 1, size=(5, 3)) * np.array(dom.extent)
    w = W.Workload("abc_box", [dom], 60, rec)
    P = oracle_problem(w)
    x, y, z = P.all_coordinates()
    p0 = W.seeded_field(11, x, y, z)
    v0 = 1e3 * W.seeded_field(12, x, y, z)
    dt = P.stable_dt()
    to = P.run(p0=p0, v0=v0, dt=dt)
    po = P.final_state["p"].T
    sol = gpu_solver(w)
    assert abs(sol.dt - dt) <= 1e-13 * dt
    for v in range(dgsem.dgsem_num_tiles(sol.ctx, prec, 0)):
        dgsem.dgsem_set_tiles(sol.ctx, prec, [v])
        dgsem.dgsem_set_state(sol.ctx, p0, v0)
        tg = sol.run(precision=prec)
        pg = dgsem.dgsem_get_pressure(sol.ctx, 1, sol.ndof)
        assert rel_l2(pg, po) < tol, (v, rel_l2(pg, po))
        assert rel_l2(tg, to) < tol, (v, rel_l2(tg, to))
    sol.close()


@pytest.mark.parametrize("prec,tol", [(0, FP64_TOL), (1, FP32_TOL)])
def test_two_box_pmut_with_absorbing_sides(prec, tol):
    """PMUT array, 2:1 interface, lateral sides of both boxes and the top of
    the secondary absorbing (the open-domain set-up of Sec. 6)."""
    w = W.small_two_domain(nx_p=8, nz_p=2, nx_s=4, nz_s=4, n_pmut_side=2, nsteps=300)
    w.domains[0].absorbing = (1, 1, 1, 1, 0, 0)
    w.domains[1].absorbing = (1, 1, 1, 1, 0, 1)
    tg, to, pg, po = run_both(w, prec)
    assert np.abs(to).max() > 0
    assert rel_l2(tg, to) < tol
    assert rel_l2(pg, po) < tol


def test_absorbing_plane_pulse_leaves_the_box():
    """FP32 path: a plane pulse running along +x passes a receiver and leaves
    through an absorbing x+ side; traces and the final state (which holds
    almost nothing) match the oracle."""
    from paper_2603_06267_gb300 import dgsem
    h, N = 75e-6, 4
    nel = (24, 1, 1)
    dom = W.Domain((0, 0, 0), tuple(n * h for n in nel), nel, N, absorbing=(0, 1, 0, 0, 0, 0))
    Lx = dom.extent[0]
    P0 = oracle_problem(W.Workload("pulse", [dom], 1, np.array([[0.8 * Lx, h / 2, h / 2]])))
    dt = P0.stable_dt()
    S = int((0.4 * Lx + 8 * h) / dom.c / dt)
    w = W.Workload("pulse", [dom], S, np.array([[0.8 * Lx, h / 2, h / 2]]))
    P = oracle_problem(w)
    x, y, z = P.all_coordinates()
    p0, v0 = W.gaussian_pulse_x(dom, x, 0.6 * Lx, 2 * h, +1)
    to = P.run(p0=p0, v0=v0, dt=dt)
    po = P.final_state["p"].T
    sol = gpu_solver(w)
    dgsem.dgsem_set_state(sol.ctx, p0, v0)
    tg = sol.run(precision=1)
    pg = dgsem.dgsem_get_pressure(sol.ctx, 1, sol.ndof)
    sol.close()
    assert np.abs(po).max() < 0.05 * np.abs(p0).max()
    assert np.abs(pg - po).max() < 1e-4 * np.abs(p0).max()
    assert rel_l2(tg, to) < FP32_TOL


def test_set_absorbing_rejects_bad_sides_and_fixed_dt():
    from paper_2603_06267_gb300 import dgsem
    w = W.small_two_domain(nx_p=4, nz_p=2, nx_s=2, nz_s=2, n_pmut_side=2, nsteps=10)
    sol = gpu_solver(w)
    for box, sides in [(0, (0, 0, 0, 0, 1, 0)), (0, (0, 0, 0, 0, 0, 1)), (1, (0, 0, 0, 0, 1, 0)), (2, (1,) * 6)]:
        with pytest.raises(dgsem.DgsemError) as e:
            dgsem.dgsem_set_absorbing(sol.ctx, box, sides)
        assert e.value.code == dgsem.DGSEM_EINVAL
    dt0 = sol.dt
    dgsem.dgsem_set_absorbing(sol.ctx, 1, (1, 1, 1, 1, 0, 1))
    dt1 = dgsem.dgsem_get_dt(sol.ctx)[0]
    assert dt1 < dt0
    dgsem.dgsem_set_absorbing(sol.ctx, 1, (0,) * 6)
    assert dgsem.dgsem_get_dt(sol.ctx)[0] == dt0
    sol.close()
    # a caller-fixed dt above the damping limit is refused
    sol = gpu_solver(w, dt=dt0)
    with pytest.raises(dgsem.DgsemError) as e:
        dgsem.dgsem_set_absorbing(sol.ctx, 1, (1, 1, 1, 1, 0, 1))
    assert e.value.code == dgsem.DGSEM_EUNSTABLE
    sol.close()
