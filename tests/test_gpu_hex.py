"""General hexahedra on the GPU (C ABI include/dghex.h) against the
trilinear-element oracle: Algorithm 3 matches, node positions and PMUT face
weights, receiver traces and full fields in FP64 (rel-L2 <= 1e-10) and FP32
(<= 1e-4), element orientation, batching, continued runs, the affine case
against the box path, and the error paths."""
import numpy as np
import pytest

import workloads as W
from workloads import hex as H
from oracle import hex_oracle as HO

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
FP32_TOL = 1e-4


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - b) / max(np.linalg.norm(b), 1e-300))


def _node_map(prob, xyz, first_sec):
    """index into the library's node array of every oracle node (per domain)."""
    from scipy.spatial import cKDTree
    out = []
    bounds = [(0, first_sec), (first_sec, xyz.shape[0])]
    for m, (lo, hi) in zip(prob.meshes, bounds):
        d, idx = cKDTree(xyz[lo:hi]).query(m.coords)
        assert np.max(d) < 1e-12 * 1e-3
        assert np.unique(idx).size == idx.size == hi - lo
        out.append(idx + lo)
    return np.concatenate(out)


@pytest.fixture(scope="module")
def lib():
    from paper_2603_06267_gb300 import dghex
    return dghex.load_library()


@pytest.fixture(scope="module")
def two_dom():
    w = H.distorted_two_domain(nx_p=4, nz_p=2, nx_s=2, nz_s=2, n_pmut_side=2, nsteps=120, scramble=3)
    return w, HO.HexOracleProblem(w)


def test_matching_equals_oracle(lib, two_dom):
    from paper_2603_06267_gb300 import dghex
    w, prob = two_dom
    s = dghex.HexSolver(w)
    q, cf, ref = dghex.dghex_get_matches(s.ctx, len(w.fine_faces))
    assert q == prob.nq
    for f, (F, refp, xq, per) in enumerate(prob.matches):
        for j, (gi, refm) in enumerate(per):
            assert cf[f, j] == gi
            assert np.max(np.abs(ref[f, j] - refm)) < 1e-12
    s.close()


def test_nodes_mass_layout_and_pmut_weights(lib, two_dom):
    from paper_2603_06267_gb300 import dghex
    w, prob = two_dom
    s = dghex.HexSolver(w)
    xyz, first = dghex.dghex_nodes(s.ctx)
    assert xyz.shape[0] == prob.nh and first == prob.meshes[1].offset
    _node_map(prob, xyz, first)
    ids, pxyz, Wf = prob.pmut_face_nodes()
    gx, gw = dghex.dghex_pmut_nodes(s.ctx)
    from scipy.spatial import cKDTree
    d, idx = cKDTree(gx).query(pxyz)
    assert np.max(d) < 1e-15 and gx.shape[0] == pxyz.shape[0]
    np.testing.assert_allclose(gw[idx], Wf, rtol=1e-13)
    dt, ndof = dghex.dghex_get_dt(s.ctx)
    assert ndof == prob.nh and abs(dt - prob.stable_dt()) < 1e-15 * dt
    s.close()


@pytest.mark.parametrize("general", [False, True])
@pytest.mark.parametrize("prec,tol", [(0, FP64_TOL), (1, FP32_TOL)])
def test_two_domain_pmut_parity(lib, two_dom, prec, tol, general):
    """Distorted fine/coarse pair with a bent 2:1 interface, rotated element
    frames and a driven PMUT array: traces and the final field, with the
    face-collapsed and with the full-evaluation interface kernel."""
    from paper_2603_06267_gb300 import dghex
    w, prob = two_dom
    s = dghex.HexSolver(w)
    dghex.dghex_set_interface_kernel(s.ctx, general)
    tr = s.run(precision=prec)
    ref = prob.run(dt=s.dt)
    assert np.max(np.abs(ref)) > 0
    assert _rel(tr, ref) < tol, _rel(tr, ref)
    xyz, first = dghex.dghex_nodes(s.ctx)
    idx = _node_map(prob, xyz, first)
    p = dghex.dghex_get_pressure(s.ctx, 1, s.ndof)[0]
    assert _rel(p[idx], prob.final_state["p"][:, 0]) < tol
    s.close()


@pytest.mark.parametrize("prec,tol", [(0, FP64_TOL), (1, FP32_TOL)])
def test_one_domain_initial_state_parity(lib, prec, tol):
    """Distorted single box, orders 3 and 5, a smooth initial state and no
    PMUT (the set-state start p''0 = -M^-1 K p0)."""
    from paper_2603_06267_gb300 import dghex
    for order, scr in ((3, None), (5, 9)):
        w = H.distorted_one_domain(nel=(3, 2, 2), order=order, nsteps=60, scramble=scr)
        w.pmuts = None
        prob = HO.HexOracleProblem(w)
        s = dghex.HexSolver(w)
        xyz, first = dghex.dghex_nodes(s.ctx)
        idx = _node_map(prob, xyz, first)
        X = prob.meshes[0].coords
        p0 = W.seeded_field(5, X[:, 0], X[:, 1], X[:, 2])
        v0 = 1e6 * W.seeded_field(6, X[:, 0], X[:, 1], X[:, 2])
        g0 = np.zeros(s.ndof); g0[idx] = p0
        gv = np.zeros(s.ndof); gv[idx] = v0
        dghex.dghex_set_state(s.ctx, g0, gv)
        tr = s.run(precision=prec)
        ref = prob.run(dt=s.dt, p0=p0, v0=v0)
        assert _rel(tr, ref) < tol, (order, _rel(tr, ref))
        s.close()


def test_batch_members_are_independent(lib):
    """Drive patterns in one run equal single runs bit for bit, whatever the
    batch width (3: scalar path; 9 FP32 / 5 FP64: padded to the 32-byte
    vector width)."""
    from paper_2603_06267_gb300 import dghex
    w = H.distorted_two_domain(nx_p=4, nz_p=1, nx_s=2, nz_s=2, n_pmut_side=2, nsteps=40, batch=9, steer=True)
    s = dghex.HexSolver(w)
    drive = w.drive(s.dt, w.nsteps, 9)
    for prec, B, general in ((0, 3, False), (1, 3, False), (1, 9, False), (0, 5, False), (1, 9, True)):
        dghex.dghex_set_interface_kernel(s.ctx, general)
        tr = s.run(drive=np.ascontiguousarray(drive[:B]), precision=prec, batch=B)
        for b in range(B):
            one = s.run(drive=np.ascontiguousarray(drive[b:b + 1]), precision=prec, batch=1)
            assert np.array_equal(one[0], tr[b]), (prec, B, b, general)
    s.close()


@pytest.mark.parametrize("orders", [(4, 6), (5, 8), (3, 7)])
def test_volume_variants_agree_bit_for_bit(lib, orders):
    """Every element-stiffness launch variant, and the autotuner's choice,
    gives the default kernel's traces and final field bit for bit: FP32 with
    16 members (8 or 4 per thread, several chunks) and FP64 with 8 members,
    on element counts that leave the last CTA partly filled for several
    elements-per-CTA choices."""
    from paper_2603_06267_gb300 import dghex, dgsem
    w = H.distorted_two_domain(nx_p=6, nz_p=1, nx_s=3, nz_s=2, order_p=orders[0], order_s=orders[1],
                               n_pmut_side=2, nsteps=25, scramble=3, batch=16, steer=True)
    s = dghex.HexSolver(w)
    nv = dghex.dghex_num_volume_variants(s.ctx)
    assert nv >= 2
    for prec, B in ((1, 16), (0, 8)):
        drive = w.drive(s.dt, w.nsteps, B)
        dghex.dghex_set_volume_variant(s.ctx, prec, [0, 0])
        ref_tr = s.run(drive=drive, precision=prec, batch=B)
        ref_p = dghex.dghex_get_pressure(s.ctx, B, s.ndof)
        assert np.max(np.abs(ref_tr)) > 0 and np.all(np.isfinite(ref_p))
        for v in range(1, nv):
            dghex.dghex_set_volume_variant(s.ctx, prec, [v, nv - v])
            tr = s.run(drive=drive, precision=prec, batch=B)
            assert np.array_equal(tr, ref_tr), (orders, prec, v)
            assert np.array_equal(dghex.dghex_get_pressure(s.ctx, B, s.ndof), ref_p), (orders, prec, v)
        chosen = dghex.dghex_autotune(s.ctx, prec, B, 2, reps=1)
        assert all(0 <= c < nv for c in chosen)
        tr = s.run(drive=drive, precision=prec, batch=B)
        assert np.array_equal(tr, ref_tr), (orders, prec, chosen)
    with pytest.raises(dgsem.DgsemError) as e:
        dghex.dghex_set_volume_variant(s.ctx, 1, [0, nv])
    assert e.value.code == dgsem.DGSEM_EINVAL
    s.close()


def test_continued_run_equals_single_run(lib):
    from paper_2603_06267_gb300 import dghex
    w = H.distorted_two_domain(nx_p=4, nz_p=1, nx_s=2, nz_s=2, n_pmut_side=2, nsteps=50)
    s = dghex.HexSolver(w)
    drive = w.drive(s.dt, 50, 1)
    full = s.run(drive=drive, nsteps=50)
    a = s.run(drive=np.ascontiguousarray(drive[:, :, :30]), nsteps=30)
    b = s.run(drive=np.ascontiguousarray(drive[:, :, 30:]), nsteps=20, flags=1)
    assert np.array_equal(np.concatenate([a, b], axis=2), full)
    s.close()


def test_affine_mesh_matches_box_path(lib):
    """The lattice of a box workload given as general hexahedra gives the
    box path's traces (two different GPU implementations of one operator)."""
    from paper_2603_06267_gb300 import dghex, dgsem
    wb = W.small_two_domain(nx_p=4, nz_p=2, nx_s=2, nz_s=3, nsteps=80)
    wh = H.hex_workload_from_box(wb)
    sb = dgsem.Solver(wb)
    sh = dghex.HexSolver(wh)
    assert abs(sb.dt - sh.dt) < 1e-15 * sb.dt
    drive = wb.drive(sb.dt, wb.nsteps, 1)
    tb = sb.run(drive=drive)
    th = sh.run(drive=drive)
    assert _rel(th, tb) < 1e-11, _rel(th, tb)
    sb.close()
    sh.close()


def test_errors_inverted_element_and_unmatched_interface(lib):
    from paper_2603_06267_gb300 import dghex, dgsem
    w = H.distorted_two_domain(nx_p=2, nz_p=1, nx_s=1, nz_s=1, n_pmut_side=1, order_p=2, order_s=2)
    prim, sec = w.domains
    inv = prim.elements.copy()
    inv[0] = inv[0][[1, 0, 3, 2, 5, 4, 7, 6]]         # mirrored: negative Jacobian
    with pytest.raises(dgsem.DgsemError) as e:
        dghex.dghex_mesh_create([H.HexDomain(prim.vertices, inv, 2)])
    assert e.value.code == dgsem.DGSEM_EINVAL and "Jacobian" in str(e.value)
    w4 = H.distorted_two_domain(nx_p=4, nz_p=1, nx_s=2, nz_s=1, n_pmut_side=1, order_p=2, order_s=2)
    with pytest.raises(dgsem.DgsemError) as e:
        dghex.dghex_mesh_create(w4.domains, w4.fine_faces, w4.coarse_faces[:3], w4.pmut_faces)
    assert e.value.code == dgsem.DGSEM_ENOMATCH
    # the library stays usable
    s = dghex.HexSolver(w)
    s.run(nsteps=3)
    s.close()


@pytest.mark.parametrize("general", [False, True])
@pytest.mark.parametrize("orders,dims", [((2, 3), (4, 1, 2, 2)), ((3, 5), (4, 1, 2, 2)), ((4, 8), (2, 1, 1, 1)),
                                         ((1, 2), (4, 2, 2, 2))])
def test_order_pairs_vector_and_scalar_paths(lib, orders, dims, general):
    """Other order pairs across the bent interface, with a batch wide enough
    for the 32-byte vector path (9 FP32 members, 5 FP64 members) and with one
    member (scalar path), against the oracle."""
    from paper_2603_06267_gb300 import dghex
    nxp, nzp, nxs, nzs = dims
    w = H.distorted_two_domain(nx_p=nxp, nz_p=nzp, nx_s=nxs, nz_s=nzs, order_p=orders[0], order_s=orders[1],
                               n_pmut_side=1, nsteps=40, scramble=5, batch=9, steer=True)
    prob = HO.HexOracleProblem(w)
    s = dghex.HexSolver(w)
    dghex.dghex_set_interface_kernel(s.ctx, general)
    for prec, tol, B in ((0, FP64_TOL, 5), (1, FP32_TOL, 9), (0, FP64_TOL, 1)):
        drive = w.drive(s.dt, w.nsteps, B)
        tr = s.run(drive=drive, precision=prec, batch=B)
        ref = prob.run(dt=s.dt, drive=drive, batch=B)
        assert np.max(np.abs(ref)) > 0
        assert _rel(tr, ref) < tol, (orders, prec, B, _rel(tr, ref))
    s.close()


@pytest.mark.parametrize("order", [1, 2, 7, 8])
def test_single_domain_orders(lib, order):
    """Distorted single box at the lowest and highest orders, from a smooth
    initial state, FP64 and FP32 (scalar and vector paths)."""
    from paper_2603_06267_gb300 import dghex
    w = H.distorted_one_domain(nel=(2, 2, 2), order=order, nsteps=40)
    w.pmuts = None
    prob = HO.HexOracleProblem(w)
    s = dghex.HexSolver(w)
    xyz, first = dghex.dghex_nodes(s.ctx)
    idx = _node_map(prob, xyz, first)
    X = prob.meshes[0].coords
    p0 = W.seeded_field(8, X[:, 0], X[:, 1], X[:, 2])
    g0 = np.zeros(s.ndof)
    g0[idx] = p0
    dghex.dghex_set_state(s.ctx, g0, None)
    ref = prob.run(dt=s.dt, p0=p0, batch=1)
    for prec, tol, B in ((0, FP64_TOL, 1), (0, FP64_TOL, 4), (1, FP32_TOL, 1), (1, FP32_TOL, 8)):
        tr = s.run(precision=prec, batch=B)
        for b in range(B):
            assert _rel(tr[b], ref[0]) < tol, (order, prec, B, _rel(tr[b], ref[0]))
    s.close()


def test_stability_check_matches_the_largest_eigenvalue(lib, two_dom):
    """Device power iteration for lambda_max(M^-1 K) against the oracle's
    generalised eigenvalue, and the explicit-scheme limit it enforces."""
    import scipy.sparse as sp
    from scipy.sparse.linalg import eigsh
    from paper_2603_06267_gb300 import dghex, dgsem
    w, prob = two_dom
    Mh = sp.diags(1.0 / np.sqrt(prob.M))
    lam_ref = eigsh(Mh @ prob.K @ Mh, k=1, which="LA", return_eigenvectors=False)[0]
    s = dghex.HexSolver(w)
    code, lam = dghex.dghex_check_stability(s.ctx, 400)
    assert code == 0
    assert abs(lam / lam_ref - 1.0) < 2e-2, (lam, lam_ref)
    assert s.dt < 0.95 * 2.0 / np.sqrt(lam_ref)
    s.close()
    big = dghex.HexSolver(w, dt=1.2 * 2.0 / np.sqrt(lam_ref))
    code, lam2 = dghex.dghex_check_stability(big.ctx, 400)
    assert code == dgsem.DGSEM_EUNSTABLE and abs(lam2 / lam_ref - 1.0) < 2e-2
    big.close()


def _absorbing_workload(nsteps=60):
    w = H.distorted_two_domain(nx_p=4, nz_p=2, nx_s=2, nz_s=2, n_pmut_side=2, nsteps=nsteps)
    prim, sec = w.domains
    w.absorbing_faces = [H.lattice_side_faces(prim.lattice, 0),
                         np.concatenate([H.lattice_side_faces(sec.lattice, 3), H.lattice_side_faces(sec.lattice, 5)])]
    return w


@pytest.mark.parametrize("prec,tol", [(0, FP64_TOL), (1, FP32_TOL)])
def test_absorbing_faces_parity(lib, prec, tol):
    """Absorbing faces on a curved two-domain mesh (primary x-, secondary y+
    and top): driven traces and a run from a state with velocity."""
    from paper_2603_06267_gb300 import dghex
    w = _absorbing_workload()
    prob = HO.HexOracleProblem(w)
    s = dghex.HexSolver(w)
    assert abs(s.dt - prob.stable_dt()) < 1e-15 * s.dt
    tr = s.run(precision=prec)
    ref = prob.run(dt=s.dt)
    assert _rel(tr, ref) < tol, _rel(tr, ref)
    xyz, first = dghex.dghex_nodes(s.ctx)
    idx = _node_map(prob, xyz, first)
    X = np.concatenate([m.coords for m in prob.meshes])
    p0 = W.seeded_field(9, X[:, 0], X[:, 1], X[:, 2])
    v0 = 2e6 * W.seeded_field(10, X[:, 0], X[:, 1], X[:, 2])
    g0 = np.zeros(s.ndof); g0[idx] = p0
    gv = np.zeros(s.ndof); gv[idx] = v0
    dghex.dghex_set_state(s.ctx, g0, gv)
    drive = np.zeros((1, w.pmuts.n_pmut, w.nsteps))
    tr = s.run(drive=drive, precision=prec)
    ref = prob.run(dt=s.dt, drive=drive, p0=p0, v0=v0)
    assert _rel(tr, ref) < tol, _rel(tr, ref)
    s.close()


def test_absorbing_faces_refused_on_the_interface(lib):
    from paper_2603_06267_gb300 import dghex, dgsem
    w = _absorbing_workload()
    s = dghex.HexSolver(w)
    with pytest.raises(dgsem.DgsemError) as e:
        dghex.dghex_set_absorbing_faces(s.ctx, 0, w.fine_faces[:1])
    assert e.value.code == dgsem.DGSEM_EINVAL
    dghex.dghex_set_absorbing_faces(s.ctx, 0, None)
    dghex.dghex_set_absorbing_faces(s.ctx, 1, None)
    dt, _ = dghex.dghex_get_dt(s.ctx)
    assert dt >= s.dt
    s.close()


@pytest.mark.parametrize("prec,tol", [(0, FP64_TOL), (1, FP32_TOL)])
def test_receive_switch_parity(lib, prec, tol):
    """TX -> RX switch at step 25 on the curved mesh: traces and the recorded
    voltages (drive, then open circuit) against the oracle."""
    from paper_2603_06267_gb300 import dghex
    w = H.distorted_two_domain(nx_p=4, nz_p=2, nx_s=2, nz_s=2, n_pmut_side=2, nsteps=60)
    w.rx_switch, w.rx_capacitance, w.rx_sign = 25, np.full(w.pmuts.n_pmut, 2e-12), -1
    prob = HO.HexOracleProblem(w)
    s = dghex.HexSolver(w)
    tr = s.run(precision=prec)
    ref = prob.run(dt=s.dt)
    assert _rel(tr, ref) < tol
    v = dghex.dghex_get_voltages(s.ctx, 1, w.pmuts.n_pmut, w.nsteps)
    assert np.max(np.abs(prob.voltages[:, :, 25:])) > 0
    assert _rel(v, prob.voltages) < tol
    s.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_checkpoint_roundtrip_is_bitwise(lib, prec):
    """30 steps, checkpoint, load into a fresh context, 20 more steps equals
    50 steps in one run bit for bit (reception switching on after the
    checkpoint, so the step count must survive it)."""
    from paper_2603_06267_gb300 import dghex
    w = H.distorted_two_domain(nx_p=4, nz_p=1, nx_s=2, nz_s=2, n_pmut_side=2, nsteps=50, batch=3, steer=True)
    w.rx_switch, w.rx_capacitance, w.rx_sign = 35, np.full(w.pmuts.n_pmut, 2e-12), -1
    a = dghex.HexSolver(w)
    drive = w.drive(a.dt, 50, 3)
    full = a.run(drive=drive, precision=prec, nsteps=50)
    vfull = dghex.dghex_get_voltages(a.ctx, 3, w.pmuts.n_pmut, 50)
    a.run(drive=np.ascontiguousarray(drive[:, :, :30]), precision=prec, nsteps=30)
    blob = dghex.dghex_state_save(a.ctx)
    a.close()
    b = dghex.HexSolver(w)
    dghex.dghex_state_load(b.ctx, blob)
    tail = b.run(drive=np.ascontiguousarray(drive[:, :, 30:]), precision=prec, nsteps=20, flags=1)
    vtail = dghex.dghex_get_voltages(b.ctx, 3, w.pmuts.n_pmut, 20)
    assert np.array_equal(tail, full[:, :, 30:])
    assert np.array_equal(vtail, vfull[:, :, 30:])
    b.close()


def _pml_workload(nsteps=60):
    w = H.distorted_two_domain(nx_p=4, nz_p=2, nx_s=2, nz_s=3, n_pmut_side=2, nsteps=nsteps)
    w.pml = [(0.0, 25e-6, 0.0, 0.0, 0.0, 0.0), (50e-6, 0.0, 0.0, 50e-6, 0.0, 50e-6)]
    w.pml_R = 1e-3
    return w


@pytest.mark.parametrize("prec,tol", [(0, FP64_TOL), (1, FP32_TOL)])
def test_pml_parity(lib, prec, tol):
    """Layers on curved elements (primary x+, secondary x-, y+ and top):
    driven traces and a run from a state with velocity, against the oracle."""
    from paper_2603_06267_gb300 import dghex
    w = _pml_workload()
    prob = HO.HexOracleProblem(w)
    assert prob.pml is not None and len(prob.pml["elems"]) > 0
    s = dghex.HexSolver(w)
    assert abs(s.dt - prob.stable_dt()) < 1e-15 * s.dt
    tr = s.run(precision=prec)
    ref = prob.run(dt=s.dt)
    assert _rel(tr, ref) < tol, _rel(tr, ref)
    xyz, first = dghex.dghex_nodes(s.ctx)
    idx = _node_map(prob, xyz, first)
    X = np.concatenate([m.coords for m in prob.meshes])
    p0 = W.seeded_field(11, X[:, 0], X[:, 1], X[:, 2])
    v0 = 2e6 * W.seeded_field(12, X[:, 0], X[:, 1], X[:, 2])
    g0 = np.zeros(s.ndof); g0[idx] = p0
    gv = np.zeros(s.ndof); gv[idx] = v0
    dghex.dghex_set_state(s.ctx, g0, gv)
    drive = np.zeros((1, w.pmuts.n_pmut, w.nsteps))
    for B in (1, 9 if prec == 1 else 5):
        tr = s.run(drive=np.zeros((B, w.pmuts.n_pmut, w.nsteps)), precision=prec, batch=B)
        ref = prob.run(dt=s.dt, drive=drive, p0=p0, v0=v0)
        for b in range(B):
            assert _rel(tr[b], ref[0]) < tol, (B, b, _rel(tr[b], ref[0]))
    s.close()


def test_pml_checkpoint_refused_and_removal(lib):
    from paper_2603_06267_gb300 import dghex, dgsem
    w = _pml_workload(nsteps=5)
    s = dghex.HexSolver(w)
    dt_layer = s.dt
    s.run(precision=0)
    with pytest.raises(dgsem.DgsemError) as e:
        dghex.dghex_state_save(s.ctx)
    assert e.value.code == dgsem.DGSEM_ESTATE
    for d in range(2):
        dghex.dghex_set_pml(s.ctx, d, np.zeros(6), 1e-3)
    dt, _ = dghex.dghex_get_dt(s.ctx)
    assert dt >= dt_layer
    s.run(precision=0)
    assert len(dghex.dghex_state_save(s.ctx)) > 0
    s.close()


def test_full_size_distorted_mesh_properties(lib):
    """The bench's general-hexahedron workload at full size (655,360 trilinear
    elements, 102.6M nodes, 1024 PMUTs, 64 patterns, FP32 vector path):
    linear in the drive, exactly time-shift invariant, each pattern equal bit
    for bit to the same drive run alone (scalar path), and within 1e-4 of the
    FP64 path (oracle-validated on small meshes) at receivers above the
    array."""
    from paper_2603_06267_gb300 import dghex
    S = 40
    w = H.hex_c3_like(nsteps=S, batch=64)
    # receivers 10 um above the membranes, where the first 40 steps already carry signal
    c = w.pmuts.centers[::16]
    w.receivers = np.column_stack([c, np.full(len(c), 10e-6)])
    s = dghex.HexSolver(w)
    rng = np.random.default_rng(13)
    d1 = rng.normal(size=(64, w.pmuts.n_pmut, S)) * 5.0
    d2 = rng.normal(size=(64, w.pmuts.n_pmut, S)) * 5.0
    t1 = s.run(drive=d1, precision=1)
    t2 = s.run(drive=d2, precision=1)
    t12 = s.run(drive=d1 + d2, precision=1)
    assert np.abs(t1).max() > 0 and np.all(np.isfinite(t12))
    assert _rel(t12, t1 + t2) < 1e-5
    k = 5
    ds = np.zeros_like(d1)
    ds[:, :, k:] = d1[:, :, :-k]
    ts = s.run(drive=ds, precision=1)
    assert np.array_equal(ts[:, :, k:], t1[:, :, :-k])
    for b in (0, 37):
        one = s.run(drive=np.ascontiguousarray(d1[b:b + 1]), precision=1, batch=1)
        assert np.array_equal(one[0], t1[b])
    t64 = s.run(drive=np.ascontiguousarray(d1[:1]), precision=0, batch=1)
    assert _rel(t1[0], t64[0]) < FP32_TOL
    s.close()


def test_diverging_run_is_reported(lib):
    from paper_2603_06267_gb300 import dghex, dgsem
    w = H.distorted_one_domain(nel=(3, 2, 2), order=4, nsteps=600)
    dt = HO.HexOracleProblem(w).stable_dt()
    bad = dghex.HexSolver(w, dt=4.0 * dt)
    for prec in (0, 1):
        with pytest.raises(dgsem.DgsemError) as e:
            bad.run(precision=prec)
        assert e.value.code == dgsem.DGSEM_EUNSTABLE
    bad.close()


def test_energy_diagnostic_matches_oracle_and_is_conserved(lib):
    """dghex_energy on the curved two-domain mesh equals the oracle's leapfrog
    energy and stays constant over a continued run (no forcing)."""
    from paper_2603_06267_gb300 import dghex, dgsem
    w = H.distorted_two_domain(nx_p=4, nz_p=2, nx_s=2, nz_s=2, n_pmut_side=2, nsteps=50, scramble=3)
    w.pmuts = None
    prob = HO.HexOracleProblem(w)
    s = dghex.HexSolver(w)
    xyz, first = dghex.dghex_nodes(s.ctx)
    idx = _node_map(prob, xyz, first)
    X = np.concatenate([m.coords for m in prob.meshes])
    p0 = W.seeded_field(3, X[:, 0], X[:, 1], X[:, 2])
    v0 = 1e6 * W.seeded_field(4, X[:, 0], X[:, 1], X[:, 2])
    g0 = np.zeros(s.ndof); g0[idx] = p0
    gv = np.zeros(s.ndof); gv[idx] = v0
    dghex.dghex_set_state(s.ctx, g0, gv)
    s.run(precision=0, batch=5)
    e1 = dghex.dghex_energy(s.ctx, 5)
    _, eo = prob.run(dt=s.dt, p0=p0, v0=v0, energy=True, batch=1)
    ref = eo[-1, 0, 0]
    assert abs(e1[0] - ref) < 1e-10 * abs(ref) and np.allclose(e1, e1[0], rtol=1e-14)
    s.run(precision=0, batch=5, nsteps=150, flags=dgsem.DGSEM_RUN_CONTINUE)
    e2 = dghex.dghex_energy(s.ctx, 5)
    assert abs(e2[0] - e1[0]) < 1e-12 * abs(e1[0])
    s.close()


@pytest.mark.parametrize("general", [False, True])
def test_unstructured_nonconforming_interface_parity(lib, general):
    """3:2 flat interface between independently distorted tilings (fine faces
    straddle coarse faces, so a fine face splits into several groups):
    Algorithm 3 on the GPU equals the oracle's, and FP64 / FP32 traces match
    with both interface kernels."""
    from paper_2603_06267_gb300 import dghex
    w = H.distorted_two_domain(nx_p=6, nz_p=1, nx_s=4, nz_s=2, bump=0.0, n_pmut_side=2, order_p=3, order_s=4,
                               nsteps=50, batch=9, steer=True)
    prob = HO.HexOracleProblem(w)
    s = dghex.HexSolver(w)
    dghex.dghex_set_interface_kernel(s.ctx, general)
    q, cf, ref = dghex.dghex_get_matches(s.ctx, len(w.fine_faces))
    split = 0
    for f, (F, refp, xq, per) in enumerate(prob.matches):
        assert [gi for gi, _ in per] == list(cf[f])
        assert np.max(np.abs(ref[f] - np.array([r for _, r in per]))) < 1e-12
        split += len({w.coarse_faces[g][0] for g in cf[f]}) > 1
    assert split > 0
    for prec, tol, B in ((0, FP64_TOL, 1), (1, FP32_TOL, 9)):
        drive = w.drive(s.dt, w.nsteps, B)
        tr = s.run(drive=drive, precision=prec, batch=B)
        ref_tr = prob.run(dt=s.dt, drive=drive, batch=B)
        assert _rel(tr, ref_tr) < tol, (prec, _rel(tr, ref_tr))
    s.close()


def test_c2_size_long_run_fp32_vs_fp64(lib):
    """The distorted config-2-class mesh (18.6M nodes, 256 PMUTs, 4000 steps,
    the length of the config-2 runs): FP32-mixed traces stay within 1e-4 of
    the FP64 path (oracle-validated on small meshes)."""
    from paper_2603_06267_gb300 import dghex
    w = H.hex_c2_like(nsteps=4000, batch=1, steer=False)
    s = dghex.HexSolver(w)
    t64 = s.run(precision=0)
    t32 = s.run(precision=1)
    assert np.abs(t64).max() > 0 and np.all(np.isfinite(t32))
    assert _rel(t32, t64) < FP32_TOL, _rel(t32, t64)
    s.close()
