"""Perfectly matched layer (eq. full_problem rows 1-3) on the GPU path against
the oracle: every tile variant with layers on five sides (and absorbing outer
sides), the two-box PMUT workload with layers, a plane pulse entering a
rigid-backed layer, and the argument checks of dgsem_set_pml."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import rel_l2, run_both, gpu_solver, oracle_problem

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
FP32_TOL = 1e-4


@pytest.mark.parametrize("prec,tol", [(0, FP64_TOL), (1, FP32_TOL)])
@pytest.mark.parametrize("N,nel,lay", [(4, (12, 6, 3), (2, 2, 1, 1, 0, 1)), (6, (8, 4, 3), (1, 2, 1, 1, 0, 1))])
def test_pml_every_tile_variant(prec, tol, N, nel, lay):
    from paper_2603_06267_gb300 import dgsem
    h = 25e-6
    dom = W.Domain((0, 0, 0), tuple(n * h for n in nel), nel, N, absorbing=(1, 1, 1, 1, 0, 1),
                   pml=tuple(l * h for l in lay), pml_R=1e-4)
    rec = np.random.default_rng(5).uniform(0, 1, size=(5, 3)) * np.array(dom.extent)
    w = W.Workload("pml_box", [dom], 60, rec)
    P = oracle_problem(w)
    x, y, z = P.all_coordinates()
    p0 = W.seeded_field(21, x, y, z)
    v0 = 1e3 * W.seeded_field(22, x, y, z)
    dt = P.stable_dt()
    to = P.run(p0=p0, v0=v0, dt=dt)
    po = P.final_state["p"].T
    sol = gpu_solver(w)
    assert abs(sol.dt - dt) <= 1e-13 * dt, (sol.dt, dt)
    for v in range(dgsem.dgsem_num_tiles(sol.ctx, prec, 0)):
        dgsem.dgsem_set_tiles(sol.ctx, prec, [v])
        dgsem.dgsem_set_state(sol.ctx, p0, v0)
        tg = sol.run(precision=prec)
        pg = dgsem.dgsem_get_pressure(sol.ctx, 1, sol.ndof)
        assert rel_l2(pg, po) < tol, (v, rel_l2(pg, po))
        assert rel_l2(tg, to) < tol, (v, rel_l2(tg, to))
    sol.close()


@pytest.mark.parametrize("prec,tol", [(0, FP64_TOL), (1, FP32_TOL)])
def test_two_box_pmut_with_pml(prec, tol):
    """Layers on the lateral sides of both boxes and the top of the secondary
    (absorbing outer sides behind them), PMUT array driving, 2:1 interface."""
    w = W.small_two_domain(nx_p=8, nz_p=2, nx_s=4, nz_s=4, n_pmut_side=2, nsteps=300)
    hp = w.domains[0].extent[0] / w.domains[0].nelem[0]
    hs = w.domains[1].extent[0] / w.domains[1].nelem[0]
    w.domains[0].pml = (2 * hp, 2 * hp, 2 * hp, 2 * hp, 0, 0)
    w.domains[0].absorbing = (1, 1, 1, 1, 0, 0)
    w.domains[1].pml = (hs, hs, hs, hs, 0, hs)
    w.domains[1].absorbing = (1, 1, 1, 1, 0, 1)
    tg, to, pg, po = run_both(w, prec)
    assert np.abs(to).max() > 0
    assert rel_l2(tg, to) < tol
    assert rel_l2(pg, po) < tol


def test_pml_plane_pulse_reflection():
    """FP32: a plane pulse runs into a rigid-backed 8-element layer (R = 1e-2):
    traces match the oracle and the reflection is the design coefficient."""
    h = 75e-6
    nin, lay = 16, 8
    dom = W.Domain((0, 0, 0), ((nin + lay) * h, h, h), (nin + lay, 1, 1), 4, pml=(0, lay * h, 0, 0, 0, 0), pml_R=1e-2)
    Li = nin * h
    P0 = oracle_problem(W.Workload("pulse", [dom], 1, np.array([[0.3 * Li, h / 2, h / 2]])))
    dt = P0.stable_dt()
    S = int((0.5 * Li + 2 * lay * h + 0.7 * Li + 10 * h) / dom.c / dt)
    w = W.Workload("pulse", [dom], S, np.array([[0.3 * Li, h / 2, h / 2]]))
    P = oracle_problem(w)
    x, y, z = P.all_coordinates()
    p0, v0 = W.gaussian_pulse_x(dom, x, 0.5 * Li, 1.5 * h, +1)
    to = P.run(p0=p0, v0=v0, dt=dt)
    sol = gpu_solver(w)
    from paper_2603_06267_gb300 import dgsem
    dgsem.dgsem_set_state(sol.ctx, p0, v0)
    tg = sol.run(precision=1)
    sol.close()
    assert np.abs(tg - to).max() < 1e-4
    n0 = int((0.2 * Li + 6 * h) / dom.c / dt)
    refl = np.abs(tg[0, 0, n0:]).max()
    assert abs(refl / 1e-2 - 1.0) < 0.1, refl


def test_set_pml_argument_checks():
    from paper_2603_06267_gb300 import dgsem
    w = W.small_two_domain(nx_p=4, nz_p=2, nx_s=2, nz_s=2, n_pmut_side=2, nsteps=10)
    sol = gpu_solver(w)
    h = w.domains[1].extent[0] / w.domains[1].nelem[0]
    bad = [(0, (0, 0, 0, 0, h, 0), 1e-4), (0, (0, 0, 0, 0, 0, h), 1e-4), (1, (0, 0, 0, 0, h, 0), 1e-4),
           (1, (h, 0, 0, 0, 0, 0), 0.0), (1, (h, 0, 0, 0, 0, 0), 1.0), (1, (-h, 0, 0, 0, 0, 0), 1e-4),
           (1, (2 * h, 2 * h, 0, 0, 0, 0), 1e-4)]
    for box, th, R in bad:
        with pytest.raises(dgsem.DgsemError) as e:
            dgsem.dgsem_set_pml(sol.ctx, box, th, R)
        assert e.value.code == dgsem.DGSEM_EINVAL, (box, th, R)
    dgsem.dgsem_set_pml(sol.ctx, 1, (h, h, h, h, 0, h), 1e-4)
    dgsem.dgsem_set_pml(sol.ctx, 1, (0,) * 6, 1e-4)
    sol.close()
