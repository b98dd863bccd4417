"""TX -> RX switch of the PMUT voltage (eq. ode row 2) on the GPU path against
the oracle: traces, final pressure and the recorded voltages, both sign
conventions, both precisions; and a run continued across the switch."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import rel_l2, gpu_solver, oracle_problem

pytestmark = pytest.mark.gpu


def _rx_case(sign, nsteps=300, rx_switch=140):
    w = W.small_two_domain(nx_p=8, nz_p=2, nx_s=4, nz_s=4, n_pmut_side=2, nsteps=nsteps)
    w.rx_switch = rx_switch
    w.rx_capacitance = np.linspace(0.8e-12, 1.2e-12, w.pmuts.n_pmut)
    w.rx_sign = sign
    return w


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-4)])
@pytest.mark.parametrize("sign", [-1, 1])
def test_rx_switch_matches_oracle(prec, tol, sign):
    from paper_2603_06267_gb300 import dgsem
    w = _rx_case(sign)
    P = oracle_problem(w)
    dt = P.stable_dt()
    drive = w.drive(dt, w.nsteps, 1)
    to = P.run(dt=dt, drive=drive, batch=1)
    po = P.final_state["p"].T
    vo = P.voltages
    sol = gpu_solver(w)
    tg = sol.run(drive=drive, precision=prec)
    pg = dgsem.dgsem_get_pressure(sol.ctx, 1, sol.ndof)
    vg = dgsem.dgsem_get_voltages(sol.ctx, 1, w.pmuts.n_pmut, w.nsteps)
    sol.close()
    assert np.abs(vo[:, :, w.rx_switch:]).max() > 0
    assert rel_l2(tg, to) < tol
    assert rel_l2(pg, po) < tol
    # drive part exact, open-circuit part within the path's tolerance
    np.testing.assert_array_equal(vg[:, :, :w.rx_switch], vo[:, :, :w.rx_switch])
    assert rel_l2(vg[:, :, w.rx_switch:], vo[:, :, w.rx_switch:]) < tol


def test_rx_switch_continued_run_equals_one_run():
    """The switch step counts from rest across DGSEM_RUN_CONTINUE runs."""
    from paper_2603_06267_gb300 import dgsem
    w = _rx_case(-1, nsteps=200, rx_switch=130)
    sol = gpu_solver(w)
    drive = w.drive(sol.dt, 200, 1)
    t_all = sol.run(drive=drive, precision=0, nsteps=200)
    v_all = dgsem.dgsem_get_voltages(sol.ctx, 1, w.pmuts.n_pmut, 200)
    t1 = sol.run(drive=np.ascontiguousarray(drive[:, :, :100]), precision=0, nsteps=100)
    v1 = dgsem.dgsem_get_voltages(sol.ctx, 1, w.pmuts.n_pmut, 100)
    t2 = sol.run(drive=np.ascontiguousarray(drive[:, :, 100:]), precision=0, nsteps=100,
                 flags=dgsem.DGSEM_RUN_CONTINUE)
    v2 = dgsem.dgsem_get_voltages(sol.ctx, 1, w.pmuts.n_pmut, 100)
    sol.close()
    np.testing.assert_array_equal(np.concatenate([t1, t2], axis=2), t_all)
    np.testing.assert_array_equal(np.concatenate([v1, v2], axis=2), v_all)


def test_rx_argument_checks():
    from paper_2603_06267_gb300 import dgsem
    w = W.small_two_domain(nx_p=4, nz_p=2, nx_s=2, nz_s=2, n_pmut_side=2, nsteps=10)
    sol = gpu_solver(w)
    K = w.pmuts.n_pmut
    for cap, sign in [(np.full(K, -1e-12), -1), (np.full(K, 1e-12), 2)]:
        with pytest.raises(dgsem.DgsemError) as e:
            dgsem.pmut_set_receive(sol.ctx, 5, cap, sign)
        assert e.value.code == dgsem.DGSEM_EINVAL
    with pytest.raises(dgsem.DgsemError) as e:
        dgsem.dgsem_get_voltages(sol.ctx, 1, K, 10)       # nothing recorded yet
    assert e.value.code == dgsem.DGSEM_ESTATE
    sol.close()
