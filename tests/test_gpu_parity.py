"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bars: relative L2 of receiver traces (and of the final pressure field)
<= 1e-10 in FP64 and <= 1e-4 in FP32/mixed precision, on the same seeded
inputs; meshes span several CTA tiles with ragged tails.
"""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import rel_l2, run_both, gpu_solver, oracle_problem

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
FP32_TOL = 1e-4


def _standing_field(w, l=(1, 1, 1), seed=None):
    P = oracle_problem(w)
    x, y, z = P.all_coordinates()
    if seed is None:
        p0, _ = W.standing_wave_mode(w.domains[0], l, x, y, z)
    else:
        p0 = W.seeded_field(seed, x, y, z)
    return p0


@pytest.mark.parametrize("N,nel", [(1, (5, 3, 4)), (2, (20, 3, 3)), (3, (13, 4, 3)), (4, (40, 5, 3)),
                                   (5, (19, 3, 2)), (6, (20, 3, 2)), (7, (9, 2, 2)), (8, (18, 2, 1))])
def test_volume_operator_single_box_fp64(N, nel):
    """Rigid box, smooth random initial state, no PMUT: every GLL node of the
    final field and the receiver traces match the oracle (FP64)."""
    h = 25e-6
    dom = W.Domain((0, 0, 0), tuple(n * h for n in nel), nel, N)
    rng = np.random.default_rng(N)
    L = np.array(dom.extent)
    rec = rng.uniform(0, 1, size=(7, 3)) * L
    w = W.Workload("box", [dom], 60, rec)
    p0 = _standing_field(w, seed=N)
    tg, to, pg, po = run_both(w, 0, p0=p0)
    assert rel_l2(pg, po) < FP64_TOL
    assert rel_l2(tg, to) < FP64_TOL


@pytest.mark.parametrize("N,nel", [(4, (40, 5, 3)), (6, (20, 3, 2))])
def test_volume_operator_single_box_fp32(N, nel):
    h = 25e-6
    dom = W.Domain((0, 0, 0), tuple(n * h for n in nel), nel, N)
    rec = np.random.default_rng(1).uniform(0, 1, size=(5, 3)) * np.array(dom.extent)
    w = W.Workload("box", [dom], 80, rec)
    p0 = _standing_field(w, seed=7)
    tg, to, pg, po = run_both(w, 1, p0=p0)
    assert rel_l2(pg, po) < FP32_TOL
    assert rel_l2(tg, to) < FP32_TOL


@pytest.mark.parametrize("prec,tol", [(0, FP64_TOL), (1, FP32_TOL)])
def test_two_domain_interface_initial_state(prec, tol):
    """2:1 non-conforming N=4 | N=6 interface, initial state crossing it."""
    w = W.small_two_domain(nx_p=8, nz_p=2, nx_s=4, nz_s=3, n_pmut_side=2, nsteps=80)
    w.pmuts = None
    p0 = _standing_field(w, seed=3)
    tg, to, pg, po = run_both(w, prec, p0=p0)
    assert rel_l2(pg, po) < tol
    assert rel_l2(tg, to) < tol


@pytest.mark.parametrize("prec,tol", [(0, FP64_TOL), (1, FP32_TOL)])
def test_two_domain_pmut_array(prec, tol):
    """Full step: PMUT array on z = 0, 2:1 interface, receivers in both boxes."""
    w = W.small_two_domain(nx_p=8, nz_p=2, nx_s=4, nz_s=4, n_pmut_side=2, nsteps=300)
    tg, to, pg, po = run_both(w, prec)
    assert np.abs(to).max() > 0
    assert rel_l2(tg, to) < tol
    assert rel_l2(pg, po) < tol


@pytest.mark.parametrize("prec,tol", [(0, FP64_TOL), (1, FP32_TOL)])
def test_two_domain_pmut_every_tile_variant(prec, tol):
    """PMUT forcing and interface terms (the volume kernel's extras planes)
    under every tile variant of each box, the other box at variant 0."""
    from paper_2603_06267_gb300 import dgsem
    w = W.small_two_domain(nx_p=8, nz_p=2, nx_s=4, nz_s=3, n_pmut_side=2, nsteps=160)
    P = oracle_problem(w)
    dt = P.stable_dt()
    drive = w.drive(dt, w.nsteps, 1)
    to = P.run(nsteps=w.nsteps, dt=dt, drive=drive)
    po = P.final_state["p"].T
    sol = gpu_solver(w)
    for box in range(2):
        for v in range(dgsem.dgsem_num_tiles(sol.ctx, prec, box)):
            tiles = [0, 0]
            tiles[box] = v
            dgsem.dgsem_set_tiles(sol.ctx, prec, tiles)
            tg = sol.run(drive=drive, precision=prec)
            pg = dgsem.dgsem_get_pressure(sol.ctx, 1, sol.ndof)
            assert rel_l2(tg, to) < tol, (box, v, rel_l2(tg, to))
            assert rel_l2(pg, po) < tol, (box, v, rel_l2(pg, po))
    sol.close()


def test_two_domain_conforming_interface_fp64():
    """r = 1 (conforming faces), same order on both sides."""
    w = W.small_two_domain(nx_p=4, nz_p=2, nx_s=4, nz_s=2, n_pmut_side=2, nsteps=120, order_s=4)
    tg, to, pg, po = run_both(w, 0)
    assert rel_l2(tg, to) < FP64_TOL


def test_batched_patterns_fp64():
    """B = 3 drive patterns in one launch: each matches its own oracle run."""
    w = W.small_two_domain(nx_p=4, nz_p=2, nx_s=2, nz_s=3, n_pmut_side=2, nsteps=150, batch=3, steer=True)
    tg, to, pg, po = run_both(w, 0)
    for b in range(3):
        assert rel_l2(tg[b], to[b]) < FP64_TOL


def test_config1_full_fp64():
    """Config 1 at full size (8^3 hexes N=4, one PMUT, 2000 steps)."""
    w = W.config1_single_pmut()
    tg, to, pg, po = run_both(w, 0)
    assert rel_l2(tg, to) < FP64_TOL
    for r in range(tg.shape[1]):
        assert rel_l2(tg[0, r], to[0, r]) < FP64_TOL


def test_config1_full_fp32():
    w = W.config1_single_pmut()
    tg, to, pg, po = run_both(w, 1)
    assert rel_l2(tg, to) < FP32_TOL


def test_single_box_pmut_ragged_fp64():
    w = W.small_one_domain(nel=(3, 2, 2), nsteps=200, n_pmut_side=2, order=4)
    tg, to, pg, po = run_both(w, 0)
    assert rel_l2(tg, to) < FP64_TOL


def test_zero_steps_and_no_receivers():
    from paper_2603_06267_gb300 import dgsem
    w = W.small_one_domain(nel=(2, 2, 2), nsteps=5)
    sol = gpu_solver(w)
    tr = sol.run(nsteps=0)
    assert tr.shape == (1, w.receivers.shape[0], 0)
    tr = sol.run(receivers=np.zeros((0, 3)))
    assert tr.shape == (1, 0, 5)
    sol.close()


def test_continue_and_checkpoint_bitwise():
    """run(S) == run(k) + run(S-k, CONTINUE) == run(k) + save/load + run(S-k),
    bit for bit (deterministic kernels, no atomics)."""
    from paper_2603_06267_gb300 import dgsem
    w = W.small_two_domain(nx_p=4, nz_p=2, nx_s=2, nz_s=3, n_pmut_side=2, nsteps=100, batch=2, steer=True)
    for prec in (0, 1):
        sol = gpu_solver(w)
        drive = w.drive(sol.dt, 100, 2)
        full = sol.run(drive=drive, precision=prec)
        a = sol.run(drive=np.ascontiguousarray(drive[:, :, :37]), precision=prec, nsteps=37)
        blob = dgsem.dgsem_state_save(sol.ctx)
        b = sol.run(drive=np.ascontiguousarray(drive[:, :, 37:]), precision=prec, nsteps=63,
                    flags=dgsem.DGSEM_RUN_CONTINUE)
        assert np.array_equal(np.concatenate([a, b], axis=2), full)
        sol2 = gpu_solver(w)
        dgsem.dgsem_state_load(sol2.ctx, blob)
        c = sol2.run(drive=np.ascontiguousarray(drive[:, :, 37:]), precision=prec, nsteps=63,
                     flags=dgsem.DGSEM_RUN_CONTINUE)
        assert np.array_equal(c, b)
        sol.close()
        sol2.close()


def test_linearity_and_time_shift_gpu():
    w = W.small_one_domain(nel=(3, 2, 2), nsteps=90, n_pmut_side=2)
    sol = gpu_solver(w)
    rng = np.random.default_rng(5)
    d1 = rng.normal(size=(1, 4, 90))
    d2 = rng.normal(size=(1, 4, 90))
    t1 = sol.run(drive=d1)
    t2 = sol.run(drive=d2)
    t12 = sol.run(drive=d1 + d2)
    assert rel_l2(t12, t1 + t2) < 1e-12
    k = 11
    ds = np.zeros_like(d1)
    ds[:, :, k:] = d1[:, :, :-k]
    ts = sol.run(drive=ds)
    assert np.array_equal(ts[:, :, k:], t1[:, :, :-k])
    assert np.all(ts[:, :, :k] == 0.0)
    sol.close()


def test_device_pointer_drive_and_traces():
    """drive and traces as torch CUDA tensors (device pointers) give the same
    result as host arrays."""
    import torch
    from paper_2603_06267_gb300 import dgsem
    w = W.small_one_domain(nel=(2, 2, 2), nsteps=50)
    sol = gpu_solver(w)
    drive = w.drive(sol.dt, 50, 1)
    host = sol.run(drive=drive)
    dd = torch.tensor(drive, device="cuda")
    tt = torch.zeros((1, w.receivers.shape[0], 50), dtype=torch.float64, device="cuda")
    sol.run(drive=dd, traces=tt)
    torch.cuda.synchronize()
    assert np.array_equal(tt.cpu().numpy(), host)
    sol.close()


def test_invalid_inputs_return_status():
    from paper_2603_06267_gb300 import dgsem
    w = W.small_one_domain(nel=(2, 2, 2), nsteps=5)
    sol = gpu_solver(w)
    with pytest.raises(dgsem.DgsemError) as e:
        sol.run(receivers=np.array([[1.0, 1.0, 1.0]]))
    assert e.value.code == dgsem.DGSEM_EINVAL
    with pytest.raises(dgsem.DgsemError) as e:
        dgsem.pmut_array_set(sol.ctx, np.array([0, 1]), np.array([10 ** 7]), np.zeros((1, 1)),
                             np.ones((1, 1)), np.zeros((1, 1)), np.zeros((1, 1)))
    assert e.value.code == dgsem.DGSEM_EINVAL
    with pytest.raises(dgsem.DgsemError) as e:
        sol.run(drive=np.zeros((7, sol.K, 5)), flags=dgsem.DGSEM_RUN_CONTINUE, precision=1, batch=7)
    assert e.value.code == dgsem.DGSEM_ESTATE
    sol.close()


@pytest.mark.parametrize("prec,tol", [(0, FP64_TOL), (1, FP32_TOL)])
@pytest.mark.parametrize("N,nel", [(4, (40, 9, 3)), (6, (20, 5, 3))])
def test_every_tile_variant_matches_oracle(prec, tol, N, nel):
    """Each CTA tile shape of the volume kernel (the autotuner's choices) is a
    separate kernel instantiation: every one matches the oracle."""
    from paper_2603_06267_gb300 import dgsem
    h = 25e-6
    dom = W.Domain((0, 0, 0), tuple(n * h for n in nel), nel, N)
    rec = np.random.default_rng(2).uniform(0, 1, size=(5, 3)) * np.array(dom.extent)
    w = W.Workload("box", [dom], 40, rec)
    P = oracle_problem(w)
    x, y, z = P.all_coordinates()
    p0 = W.seeded_field(9, x, y, z)
    to = P.run(p0=p0, dt=P.stable_dt())
    po = P.final_state["p"].T
    sol = gpu_solver(w)
    nv = dgsem.dgsem_num_tiles(sol.ctx, prec, 0)
    assert nv >= 3
    for v in range(nv):
        dgsem.dgsem_set_tiles(sol.ctx, prec, [v])
        dgsem.dgsem_set_state(sol.ctx, p0, None)
        tg = sol.run(precision=prec)
        pg = dgsem.dgsem_get_pressure(sol.ctx, 1, sol.ndof)
        assert rel_l2(pg, po) < tol, (v, rel_l2(pg, po))
        assert rel_l2(tg, to) < tol
    sol.close()


def test_autotune_then_run_matches_oracle():
    from paper_2603_06267_gb300 import dgsem
    w = W.small_two_domain(nx_p=8, nz_p=2, nx_s=4, nz_s=3, n_pmut_side=2, nsteps=120)
    P = oracle_problem(w)
    dt = P.stable_dt()
    drive = w.drive(dt, w.nsteps, 1)
    to = P.run(dt=dt, drive=drive)
    sol = gpu_solver(w)
    for prec, tol in ((1, FP32_TOL), (0, FP64_TOL)):
        chosen = dgsem.dgsem_autotune(sol.ctx, prec, 1, 2, reps=2)
        assert chosen[0] < dgsem.dgsem_num_tiles(sol.ctx, prec, 0)
        assert chosen[1] < dgsem.dgsem_num_tiles(sol.ctx, prec, 1)
        tg = sol.run(drive=drive, precision=prec)
        assert rel_l2(tg, to) < tol
    sol.close()


def test_stability_check_matches_oracle_eigenvalue():
    """dgsem_check_stability's power iteration (M-weighted Rayleigh quotient)
    approaches the largest eigenvalue of M^-1 K from below; a time step above
    the bound is reported as DGSEM_EUNSTABLE (no GPU fault involved)."""
    from paper_2603_06267_gb300 import dgsem
    w = W.small_two_domain(nx_p=4, nz_p=2, nx_s=2, nz_s=2, n_pmut_side=2)
    P = oracle_problem(w)
    D = np.diag(1 / np.sqrt(P.M))
    lmax = np.linalg.eigvalsh(D @ P.K.toarray() @ D)[-1]
    sol = gpu_solver(w)
    code, lam = dgsem.dgsem_check_stability(sol.ctx, 400)
    assert code == dgsem.DGSEM_OK
    assert lam <= lmax * (1 + 1e-9) and lam >= 0.97 * lmax, (lam, lmax)
    _, dts, _ = dgsem.dgsem_get_dt(sol.ctx)
    assert abs(dts - 2 / np.sqrt(lam)) < 1e-12 * dts
    sol.close()
    big = gpu_solver(w, dt=3.0 * 2 / np.sqrt(lmax))
    code, _ = dgsem.dgsem_check_stability(big.ctx, 200)
    assert code == dgsem.DGSEM_EUNSTABLE
    big.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_run_multi_uneven_meshes_equals_separate_runs(prec):
    """Uneven PMUT arrays (different sizes, orders, batches) in one
    graph-captured launch give exactly the traces of separate runs."""
    from paper_2603_06267_gb300 import dgsem
    ws = [W.small_two_domain(nx_p=4, nz_p=2, nx_s=2, nz_s=3, n_pmut_side=2, nsteps=70, batch=2, steer=True),
          W.small_two_domain(nx_p=8, nz_p=2, nx_s=4, nz_s=2, n_pmut_side=4, nsteps=70, batch=1, seed=21),
          W.small_one_domain(nel=(3, 2, 2), nsteps=70, n_pmut_side=2, order=6)]
    sols = [gpu_solver(w) for w in ws]
    drives = [w.drive(s.dt, 70, w.batch) for w, s in zip(ws, sols)]
    sep = [s.run(drive=d, precision=prec) for s, d in zip(sols, drives)]
    multi = dgsem.dgsem_run_multi([s.ctx for s in sols], prec, [w.batch for w in ws], 70, drives,
                                  [w.receivers for w in ws])
    for a, b in zip(sep, multi):
        assert np.array_equal(a, b)
    # the oracle agrees with the multi-mesh run too (FP64)
    if prec == 0:
        P = oracle_problem(ws[1])
        to = P.run(dt=P.stable_dt(), drive=drives[1])
        assert rel_l2(multi[1], to) < FP64_TOL
    for s in sols:
        s.close()


def test_fp32_long_horizon_8000_steps():
    """FP32-mixed stays within 1e-4 of the FP64 oracle over 8000 steps (the
    config-3/4 horizon) on a 2:1 mesh with a PMUT array."""
    w = W.small_two_domain(nx_p=4, nz_p=2, nx_s=2, nz_s=3, n_pmut_side=2, nsteps=8000)
    tg, to, pg, po = run_both(w, 1)
    assert rel_l2(tg, to) < FP32_TOL


def test_config2_full_size_fp32_vs_fp64():
    """Config 2 at full size (18.6M nodes, 256 PMUTs, 64 receivers, 4000 steps):
    FP32-mixed traces within 1e-4 of the FP64 path, receiver by receiver."""
    from paper_2603_06267_gb300 import dgsem
    w = W.config2_array16()
    sol = gpu_solver(w)
    t64 = sol.run(precision=dgsem.DGSEM_FP64)
    t32 = sol.run(precision=dgsem.DGSEM_FP32_MIXED)
    assert np.abs(t64).max() > 0 and np.all(np.isfinite(t32))
    assert rel_l2(t32, t64) < FP32_TOL
    worst = max(rel_l2(t32[0, r], t64[0, r]) for r in range(t64.shape[1]))
    assert worst < 1e-3
    sol.close()


def test_config3_full_size_linearity_and_shift():
    """Config 3 mesh at full size with 64 patterns (the bench's launch
    configuration): linear in the drive, exactly time-shift invariant, and
    each pattern independent of the others in the batch."""
    import torch
    from paper_2603_06267_gb300 import dgsem
    S = 120
    w = W.config4_batched(nsteps=S, batch=64)
    sol = gpu_solver(w)
    dgsem.dgsem_autotune(sol.ctx, 1, 64, 2, reps=1)
    d = w.drive(sol.dt, S, 64)
    # compress the bursts into the window: shift every pattern to start at t = 0
    rng = np.random.default_rng(9)
    d1 = rng.normal(size=d.shape) * 5.0
    d2 = rng.normal(size=d.shape) * 5.0
    t1 = sol.run(drive=d1, precision=1)
    t2 = sol.run(drive=d2, precision=1)
    t12 = sol.run(drive=d1 + d2, precision=1)
    assert rel_l2(t12, t1 + t2) < 1e-5
    k = 7
    ds = np.zeros_like(d1)
    ds[:, :, k:] = d1[:, :, :-k]
    ts = sol.run(drive=ds, precision=1)
    assert np.array_equal(ts[:, :, k:], t1[:, :, :-k])
    # batch independence: pattern 5 of the 64 equals the same drive run alone
    t5 = sol.run(drive=np.ascontiguousarray(d1[5:6]), precision=1, batch=1)
    assert rel_l2(t5[0], t1[5]) < 1e-6
    sol.close()


def test_bounded_wait_gives_up_and_context_stays_usable():
    """A device wait that nothing satisfies gives up within its budget and is
    reported through the status word; the same context then runs normally."""
    from paper_2603_06267_gb300 import dgsem
    w = W.small_two_domain(nx_p=4, nz_p=2, nx_s=2, nz_s=2, n_pmut_side=2, nsteps=40)
    P = oracle_problem(w)
    dt = P.stable_dt()
    drive = w.drive(dt, w.nsteps, 1)
    to = P.run(dt=dt, drive=drive)
    sol = gpu_solver(w)
    dgsem.dgsem_selftest_wait(sol.ctx)
    tg = sol.run(drive=drive, precision=0)
    sol.close()
    assert rel_l2(tg, to) < FP64_TOL


def test_diverging_run_is_reported():
    """A time step far above the stability limit makes the run overflow; the
    run returns DGSEM_EUNSTABLE instead of non-finite traces, and a stable
    context is unaffected."""
    from paper_2603_06267_gb300 import dgsem
    w = W.small_one_domain(nel=(3, 2, 2), order=4, nsteps=600)
    dt = oracle_problem(w).stable_dt()
    bad = dgsem.Solver(w, dt=4.0 * dt)
    for prec in (0, 1):
        with pytest.raises(dgsem.DgsemError) as e:
            bad.run(precision=prec)
        assert e.value.code == dgsem.DGSEM_EUNSTABLE
    bad.close()
    ok = gpu_solver(w)
    tr = ok.run(precision=0, nsteps=50)
    assert np.all(np.isfinite(tr))
    ok.close()


def test_energy_diagnostic_matches_oracle_and_is_conserved():
    """dgsem_energy after a run equals the oracle's leapfrog energy
    1/2 v.M v + 1/2 p^n.K p^{n+1}, and stays constant over a continued run
    (acoustic field, 2:1 interface, no forcing)."""
    from paper_2603_06267_gb300 import dgsem
    w = W.small_two_domain(nx_p=4, nz_p=2, nx_s=2, nz_s=3, nsteps=60)
    w.pmuts = None
    P = oracle_problem(w)
    X = np.column_stack(P.all_coordinates())
    p0 = W.seeded_field(3, X[:, 0], X[:, 1], X[:, 2])
    v0 = 1e6 * W.seeded_field(4, X[:, 0], X[:, 1], X[:, 2])
    sol = gpu_solver(w)
    dgsem.dgsem_set_state(sol.ctx, p0, v0)
    sol.run(precision=0, batch=2)
    e1 = dgsem.dgsem_energy(sol.ctx, 2)
    _, eo = P.run(dt=sol.dt, p0=p0, v0=v0, energy=True, batch=1)
    ref = eo[-1, 0, 0]
    # (the reduction adds with atomics: members agree to rounding, not bit for bit)
    assert abs(e1[0] - ref) < 1e-10 * abs(ref) and abs(e1[1] - e1[0]) < 1e-14 * abs(e1[0])
    sol.run(precision=0, batch=2, nsteps=150, flags=dgsem.DGSEM_RUN_CONTINUE)
    e2 = dgsem.dgsem_energy(sol.ctx, 2)
    assert abs(e2[0] - e1[0]) < 1e-12 * abs(e1[0])
    # an FP32 state: the diagnostic widens it and applies the FP64 operator
    sol.run(precision=1, batch=2)
    e3 = dgsem.dgsem_energy(sol.ctx, 2)
    assert abs(e3[0] - ref) < 1e-4 * abs(ref) and abs(e3[1] - e3[0]) < 1e-12 * abs(e3[0])
    with pytest.raises(dgsem.DgsemError) as e:
        dgsem.dgsem_energy(sol.ctx, 1)
    assert e.value.code == dgsem.DGSEM_EINVAL
    sol.close()


@pytest.mark.parametrize("prec,tol", [(0, FP64_TOL), (1, FP32_TOL)])
def test_pmut_state_getter_matches_oracle(prec, tol):
    """dgsem_get_pmut_state returns q^S, q'^S, q''^S of every pattern, PMUT
    and mode after an S-step run; they equal the oracle's modal state."""
    from paper_2603_06267_gb300 import dgsem
    w = W.small_two_domain(nx_p=4, nz_p=2, nx_s=2, nz_s=3, n_pmut_side=2, nsteps=150, batch=3, steer=True)
    P = oracle_problem(w)
    sol = gpu_solver(w)
    drive = w.drive(sol.dt, w.nsteps, w.batch)
    sol.run(drive=drive, precision=prec)
    q, qd, qdd = dgsem.dgsem_get_pmut_state(sol.ctx, 3, w.pmuts.n_pmut, w.pmuts.n_modes)
    P.run(dt=sol.dt, drive=drive)
    fs = P.final_state
    for got, key in ((q, "q"), (qd, "qd"), (qdd, "qdd")):
        ref = fs[key].T.reshape(3, w.pmuts.n_pmut, w.pmuts.n_modes)
        assert np.abs(ref).max() > 0
        assert rel_l2(got, ref) < tol, key
    sol.close()
