"""Parity with the oracle in the launch configuration of the full-size runs.

At the benchmark's sizes every CTA of a volume launch marches through all of
its box's element layers (16 primary, 96 secondary): the two-stage TMA /
mbarrier ring wraps many times and the z carry stays in registers from layer
to layer.  The interface launch takes 64 patterns in full groups (8 per CTA
in FP32, 4 in FP64).  These tests force the same launch shape on meshes the
oracle finishes: every CTA takes every layer of its box (asserted through
dgsem_vol_launch), 64 steering patterns, each compared with its own oracle
column, element by element on the final field and on every receiver, for
every tile variant of orders 4 and 6 in both precisions.
"""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import oracle_problem, rel_l2

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
FP32_TOL = 1e-4
B = 64
NSTEPS = 240


@pytest.fixture(scope="module")
def case():
    w = W.small_two_domain(nx_p=8, nz_p=6, nx_s=4, nz_s=8, n_pmut_side=4, nsteps=NSTEPS, batch=B, steer=True)
    P = oracle_problem(w)
    dt = P.stable_dt()
    drive = w.drive(dt, NSTEPS, B)
    to = P.run(nsteps=NSTEPS, dt=dt, drive=drive, batch=B)
    po = P.final_state["p"].T                        # [B][ndof]
    return w, dt, drive, to, po


def _variants(prec):
    from paper_2603_06267_gb300 import dgsem
    w = W.small_two_domain(nx_p=4, nz_p=1, nx_s=2, nz_s=1, n_pmut_side=1, nsteps=4)
    sol = dgsem.Solver(w)
    n = [dgsem.dgsem_num_tiles(sol.ctx, prec, d) for d in range(2)]
    sol.close()
    return [(min(i, n[0] - 1), min(i, n[1] - 1)) for i in range(max(n))]


@pytest.mark.parametrize("prec,tol", [(0, FP64_TOL), (1, FP32_TOL)])
def test_all_layers_per_cta_64_patterns_every_tile_variant(case, prec, tol):
    from paper_2603_06267_gb300 import dgsem
    w, dt, drive, to, po = case
    sol = dgsem.Solver(w)
    assert abs(sol.dt - dt) <= 1e-13 * dt
    nz = [d.nelem[2] for d in w.domains]
    dgsem.dgsem_set_layers(sol.ctx, nz)
    for tiles in _variants(prec):
        dgsem.dgsem_set_tiles(sol.ctx, prec, list(tiles))
        tg = sol.run(drive=drive, precision=prec, batch=B, nsteps=NSTEPS)
        for d in range(2):
            sh = dgsem.dgsem_vol_launch(sol.ctx, d)
            assert sh["layers_per_cta"] == nz[d] and sh["nchunks"] == 1, (tiles, d, sh)
            assert sh["grid"][2] == B
        pg = dgsem.dgsem_get_pressure(sol.ctx, B, sol.ndof)
        for b in range(B):
            scale_p = np.abs(po[b]).max()
            assert scale_p > 0
            assert rel_l2(pg[b], po[b]) < tol, (tiles, b)
            assert np.abs(pg[b] - po[b]).max() <= tol * scale_p, (tiles, b)
            assert rel_l2(tg[b], to[b]) < tol, (tiles, b)
            for r in range(tg.shape[1]):
                assert np.abs(tg[b, r] - to[b, r]).max() <= tol * np.abs(to[b]).max(), (tiles, b, r)
    # the patterns really differ (each is checked against its own column)
    assert rel_l2(to[0], to[1]) > 1e-2
    sol.close()


def test_automatic_shape_takes_every_layer_when_the_grid_is_full(case):
    """With 64 patterns a mesh of this size already gives the automatic rule
    (halve the layers per CTA while the grid has fewer than 4 x 152 CTAs)
    enough CTAs per layer chunk only for some boxes; the reported shape is the
    one the rule computes from the grid."""
    from paper_2603_06267_gb300 import dgsem
    w, dt, drive, to, po = case
    sol = dgsem.Solver(w)
    sol.run(drive=drive, precision=1, batch=B, nsteps=8)
    for d in range(2):
        sh = dgsem.dgsem_vol_launch(sol.ctx, d)
        cols = sh["grid"][0] * sh["grid"][1] * B
        nz = w.domains[d].nelem[2]
        layers = nz
        while layers > 1 and cols * ((nz + layers - 1) // layers) < 4 * 152:
            layers = (layers + 1) // 2
        assert sh["layers_per_cta"] == layers
        assert sh["nchunks"] == (nz + layers - 1) // layers
    sol.close()


def test_layer_setter_and_launch_report_edge_cases():
    """Negative layer counts are refused, counts above a box's layers are
    clamped to them, 0 restores the automatic shape, and the launch report
    is refused before the first run."""
    from paper_2603_06267_gb300 import dgsem
    w = W.small_two_domain(nx_p=4, nz_p=3, nx_s=2, nz_s=5, n_pmut_side=2, nsteps=6, batch=2, steer=True)
    sol = dgsem.Solver(w)
    with pytest.raises(dgsem.DgsemError) as e:
        dgsem.dgsem_vol_launch(sol.ctx, 0)
    assert e.value.code == dgsem.DGSEM_ESTATE
    with pytest.raises(dgsem.DgsemError) as e:
        dgsem.dgsem_set_layers(sol.ctx, [-1, 0])
    assert e.value.code == dgsem.DGSEM_EINVAL
    # one value per box: the binding refuses other lengths before the library
    # would read past the array
    with pytest.raises(ValueError):
        dgsem.dgsem_set_layers(sol.ctx, [1])
    with pytest.raises(ValueError):
        dgsem.dgsem_set_tiles(sol.ctx, 1, [0, 0, 0])
    ref = sol.run(precision=1)
    dgsem.dgsem_set_layers(sol.ctx, [1000, 1000])
    tr = sol.run(precision=1)
    for d in range(2):
        sh = dgsem.dgsem_vol_launch(sol.ctx, d)
        assert sh["layers_per_cta"] == w.domains[d].nelem[2] and sh["nchunks"] == 1
    # a different launch shape changes the result by rounding at most
    assert rel_l2(tr, ref) < 1e-6
    dgsem.dgsem_set_layers(sol.ctx, [1, 2])
    tr2 = sol.run(precision=1)
    assert dgsem.dgsem_vol_launch(sol.ctx, 1)["layers_per_cta"] == 2
    assert rel_l2(tr2, ref) < 1e-6
    with pytest.raises(dgsem.DgsemError) as e:
        dgsem.dgsem_vol_launch(sol.ctx, 2)
    assert e.value.code == dgsem.DGSEM_EINVAL
    sol.close()


def test_pmut_state_getter_refusals():
    from paper_2603_06267_gb300 import dgsem
    w = W.small_two_domain(nx_p=4, nz_p=2, nx_s=2, nz_s=3, n_pmut_side=2, nsteps=4)
    sol = dgsem.Solver(w)
    with pytest.raises(dgsem.DgsemError) as e:
        dgsem.dgsem_get_pmut_state(sol.ctx, 1, w.pmuts.n_pmut, w.pmuts.n_modes)
    assert e.value.code == dgsem.DGSEM_ESTATE
    sol.run(precision=0)
    with pytest.raises(dgsem.DgsemError) as e:
        dgsem.dgsem_get_pmut_state(sol.ctx, 1, w.pmuts.n_pmut, w.pmuts.n_modes - 1)
    assert e.value.code == dgsem.DGSEM_EINVAL
    q, qd, qdd = dgsem.dgsem_get_pmut_state(sol.ctx, 1, w.pmuts.n_pmut, w.pmuts.n_modes)
    assert np.all(np.isfinite(q)) and np.abs(qdd).max() > 0
    sol.close()
