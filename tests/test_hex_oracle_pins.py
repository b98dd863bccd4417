"""Pins of the general-hexahedron oracle against facts the mathematics fixes:
exact volumes and areas of trilinear elements under GLL quadrature, the
linear patch test across a bent 2:1 interface, invariance under rigid motions
and under re-listing elements in rotated local frames, the affine special case
(the pinned box oracle), spectral convergence of a rigid-box eigenvalue, and
the leapfrog energy invariant."""
import math

import numpy as np
import pytest

import workloads as W
from workloads import hex as H
from oracle import dgsem_oracle as O
from oracle import hex_oracle as HO


def _map_nodes(pa, pb, tol):
    """index into pb's node array of every node of pa (same positions, per
    domain: the two sides of the interface share positions but not nodes)."""
    from scipy.spatial import cKDTree
    out = []
    for ma, mb in zip(pa.meshes, pb.meshes):
        xa = np.column_stack(ma.all_coordinates()) if hasattr(ma, "all_coordinates") else ma.coords
        xb = np.column_stack(mb.all_coordinates()) if hasattr(mb, "all_coordinates") else mb.coords
        d, idx = cKDTree(xb).query(xa)
        assert np.max(d) < tol
        assert np.unique(idx).size == idx.size == xb.shape[0]
        out.append(idx + mb.offset)
    return np.concatenate(out)


def _coords(prob):
    return np.column_stack(prob.all_coordinates())


@pytest.fixture(scope="module")
def two_dom():
    w = H.distorted_two_domain(nx_p=4, nz_p=2, nx_s=2, nz_s=2, n_pmut_side=2, nsteps=40)
    return w, HO.HexOracleProblem(w)


def test_trilinear_map_of_corners_and_jacobian():
    rng = np.random.default_rng(0)
    V = rng.normal(size=(8, 3))
    X, J = HO.trilinear(V, HO.CORNERS)
    np.testing.assert_allclose(X, V, atol=1e-15)
    # finite differences of the map
    ref = rng.uniform(-1, 1, size=(4, 3))
    _, J = HO.trilinear(V, ref)
    for d in range(3):
        e = np.zeros(3); e[d] = 1e-6
        Xp, _ = HO.trilinear(V, ref + e)
        Xm, _ = HO.trilinear(V, ref - e)
        np.testing.assert_allclose((Xp - Xm) / 2e-6, J[:, :, d], rtol=1e-8, atol=1e-9)
    x = HO.trilinear(V * 0.1 + HO.CORNERS, np.array([[0.3, -0.2, 0.5]]))[0][0]
    ref = HO.newton_reference(V * 0.1 + HO.CORNERS, x)
    np.testing.assert_allclose(ref, [0.3, -0.2, 0.5], atol=1e-13)


@pytest.mark.parametrize("order", [2, 4, 6])
def test_mass_sums_to_box_volume(order):
    """sum_i M_ii = |Omega| exactly: |J| of a trilinear map has degree <= 2
    per direction, integrated exactly by N+1 GLL points for N >= 2."""
    w = H.distorted_one_domain(nel=(3, 2, 2), order=order)
    p = HO.HexOracleProblem(w)
    ext = w.box_extent
    assert abs(p.M.sum() - ext[0] * ext[1] * ext[2]) < 1e-12 * ext[0] * ext[1] * ext[2]
    assert np.min(p.meshes[0].detJ) > 0


def test_two_domain_mass_fills_the_box(two_dom):
    w, p = two_dom
    ext = w.box_extent
    vol = ext[0] * ext[1] * ext[2]
    assert abs(p.M.sum() - vol) < 1e-12 * vol


def test_pmut_face_weights_sum_to_plane_area(two_dom):
    """The z = 0 plane is flat and its elements' faces tile it, so the
    assembled face weights sum to its area exactly (planar bilinear faces
    have a polynomial surface Jacobian)."""
    w, p = two_dom
    _, xyz, Wf = p.pmut_face_nodes()
    assert np.all(np.abs(xyz[:, 2]) < 1e-18)
    area = w.box_extent[0] * w.box_extent[1]
    assert abs(Wf.sum() - area) < 1e-12 * area


def test_linear_patch_across_bent_interface(two_dom):
    """For u linear in x, (K u)_i = 0 at every node off the outer walls,
    including the curved non-conforming interface: the GLL volume rule is
    exact for the integrand (degree N+1 per direction), the GL face rule for
    the Nanson-weighted interface terms, and the jump of u vanishes."""
    w, p = two_dom
    X = _coords(p)
    rng = np.random.default_rng(1)
    a = rng.normal(size=3)
    u = X @ a + 0.7
    r = p.K @ u
    ext = np.array(w.box_extent)
    tol = 1e-9 * ext.max()
    inner = np.all((X > tol) & (X < ext[None, :] - tol), axis=1)
    scale = abs(p.K).sum(axis=1).max() * np.abs(u).max()
    assert inner.sum() > 100
    assert np.max(np.abs(r[inner])) < 1e-12 * scale
    # the wall rows carry the boundary flux c^2 int psi_i a.n: the test is not vacuous
    assert np.max(np.abs(r[~inner])) > 1e4 * np.max(np.abs(r[inner]))


def test_interface_nodes_are_inside_patch(two_dom):
    """The patch-test nodes include the interface nodes of both sides."""
    w, p = two_dom
    m0 = p.meshes[0]
    ids = m0.conn[w.fine_faces[:, 0]].ravel()
    X = _coords(p)[ids]
    assert np.any(np.abs(X[:, 2] - 2 * 25e-6) > 1e-7)   # the interface is bent


def test_matching_finds_the_parent_coarse_element(two_dom):
    """Algorithm 3 on the 2:1 lattice: every fine-face node lies in the coarse
    element above its parent position, and its reference position maps back
    to it."""
    w, p = two_dom
    nx_s = p.meshes[1].dom.lattice[0]
    nx_p = p.meshes[0].dom.lattice[0]
    for F, refp, xq, per in p.matches:
        e = F.elem
        i, j = e % nx_p, (e // nx_p) % nx_p
        parent = (j // 2) * nx_s + (i // 2)
        for q, (gi, refm) in enumerate(per):
            G = p.coarse_faces[gi]
            assert G.elem == parent
            x, _ = HO.trilinear(p.meshes[1].elem_verts(G.elem), refm[None, :])
            assert np.linalg.norm(x[0] - xq[q]) < 1e-12 * 50e-6
            assert abs(abs(refm[2]) - 1.0) < 1e-9          # on the coarse face


def test_rigid_motion_invariance():
    """K and M do not change when the whole mesh is rotated and moved (a
    transposed Jacobian or a normal in the wrong frame would change them)."""
    w = H.distorted_two_domain(nx_p=2, nz_p=1, nx_s=1, nz_s=1, n_pmut_side=1, order_p=3, order_s=4)
    p0 = HO.HexOracleProblem(w)
    rng = np.random.default_rng(5)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    for d in w.domains:
        d.vertices = d.vertices @ Q.T + np.array([1e-4, -2e-4, 3e-4])
    w.pmuts = None
    p1 = HO.HexOracleProblem(w)
    assert abs(p1.K - p0.K).max() < 1e-11 * abs(p0.K).max()
    np.testing.assert_allclose(p1.M, p0.M, rtol=1e-12)


def test_rotated_local_frames_give_the_same_operator():
    """Re-listing every element in a rotated local frame (and renumbering
    its faces) is the same physical mesh: same M, K up to node order."""
    wa = H.distorted_two_domain(nx_p=2, nz_p=1, nx_s=1, nz_s=1, n_pmut_side=1, order_p=3, order_s=4)
    wb = H.distorted_two_domain(nx_p=2, nz_p=1, nx_s=1, nz_s=1, n_pmut_side=1, order_p=3, order_s=4, scramble=7)
    assert not np.array_equal(wa.domains[0].elements, wb.domains[0].elements)
    pa, pb = HO.HexOracleProblem(wa), HO.HexOracleProblem(wb)
    idx = _map_nodes(pa, pb, 1e-12 * 50e-6)
    np.testing.assert_allclose(pb.M[idx], pa.M, rtol=1e-12)
    Kb = pb.K[idx][:, idx]
    assert abs(Kb - pa.K).max() < 1e-11 * abs(pa.K).max()
    Bb = pb.B[idx]
    assert abs(Bb - pa.B).max() < 1e-12 * abs(pa.B).max()


def test_affine_case_is_the_box_oracle():
    """On undistorted lattices the general oracle reproduces the (pinned)
    box oracle: mass, stiffness with the 2:1 interface, PMUT matrix, dt."""
    wb = W.small_two_domain(nx_p=2, nz_p=1, nx_s=1, nz_s=2, n_pmut_side=1, nsteps=10)
    wh = H.hex_workload_from_box(wb)
    pb, ph = O.OracleProblem(wb), HO.HexOracleProblem(wh)
    idx = _map_nodes(pb, ph, 1e-15)
    np.testing.assert_allclose(ph.M[idx], pb.M, rtol=1e-13)
    Kh = ph.K[idx][:, idx]
    assert abs(Kh - pb.K).max() < 1e-12 * abs(pb.K).max()
    assert abs(ph.B[idx] - pb.B).max() < 1e-13 * abs(pb.B).max()
    assert abs(ph.stable_dt() - pb.stable_dt()) < 1e-15 * pb.stable_dt()


def test_rigid_box_eigenvalue_converges_spectrally():
    """Rayleigh quotient of the interpolated rigid-box mode cos(pi x / L) on
    the distorted mesh tends to (c pi / L)^2, faster than algebraically."""
    errs = []
    for N in (2, 3, 4, 5, 6):
        w = H.distorted_one_domain(nel=(2, 2, 2), order=N, amp=0.12)
        p = HO.HexOracleProblem(w)
        X = _coords(p)
        L = w.box_extent[0]
        u = np.cos(math.pi * X[:, 0] / L)
        rq = (u @ (p.K @ u)) / (u @ (p.M * u))
        exact = (p.meshes[0].c * math.pi / L) ** 2
        errs.append(abs(rq / exact - 1.0))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-6 and errs[-1] < 1e-3 * errs[0], errs


def test_operator_symmetric_with_constant_kernel(two_dom):
    w, p = two_dom
    assert abs(p.K - p.K.T).max() < 1e-12 * abs(p.K).max()
    one = np.ones(p.nh)
    assert np.max(np.abs(p.K @ one)) < 1e-12 * abs(p.K).sum(axis=1).max()


def test_leapfrog_energy_is_conserved_on_curved_mesh(two_dom):
    """Acoustic part alone (no PMUT): Algorithm 1 keeps the leapfrog energy
    1/2 v.M v + 1/2 p.K p_next constant on the distorted two-domain mesh."""
    w, p = two_dom
    X = _coords(p)
    p0 = W.seeded_field(3, X[:, 0], X[:, 1], X[:, 2])
    pm = w.pmuts
    w.pmuts = None
    try:
        _, e = p.run(nsteps=30, p0=p0, energy=True, receivers=w.receivers[:2])
    finally:
        w.pmuts = pm
    lf = e[:, 0, 0]
    assert np.max(np.abs(lf - lf[0])) < 1e-11 * abs(lf[0])


def test_unmatched_interface_node_is_an_error():
    """A coarse face list missing a face leaves fine nodes without a
    neighbour: the matching raises instead of dropping them."""
    w = H.distorted_two_domain(nx_p=2, nz_p=1, nx_s=1, nz_s=1, n_pmut_side=1, order_p=2, order_s=2)
    w2 = H.distorted_two_domain(nx_p=4, nz_p=1, nx_s=2, nz_s=1, n_pmut_side=1, order_p=2, order_s=2)
    w2.coarse_faces = w2.coarse_faces[:3]
    with pytest.raises(ValueError):
        HO.HexOracleProblem(w2)
    HO.HexOracleProblem(w)


def test_absorbing_faces_on_the_affine_box_are_the_box_oracles():
    """Absorbing sides given as face lists of the affine lattice give the box
    oracle's C (and its damping-limited dt)."""
    wb = W.small_one_domain(nel=(3, 2, 2), order=4, nsteps=5)
    wb.domains[0].absorbing = (1, 0, 0, 1, 0, 1)
    wh = H.hex_workload_from_box(wb)
    lat = wh.domains[0].lattice
    wh.absorbing_faces = [np.concatenate([H.lattice_side_faces(lat, s) for s in (0, 3, 5)])]
    pb, ph = O.OracleProblem(wb), HO.HexOracleProblem(wh)
    idx = _map_nodes(pb, ph, 1e-15)
    np.testing.assert_allclose(ph.C[idx], pb.C, rtol=1e-13, atol=1e-30)
    assert abs(ph.stable_dt() - pb.stable_dt()) < 1e-15 * pb.stable_dt()


def test_absorbing_faces_dissipate_on_a_curved_mesh():
    """With absorbing faces (curved mesh) the leapfrog energy of the free
    acoustic field decreases monotonically and C sums to c times the
    absorbing area."""
    w = H.distorted_one_domain(nel=(3, 2, 2), order=4, nsteps=60)
    w.pmuts = None
    lat = w.domains[0].lattice
    w.absorbing_faces = [np.concatenate([H.lattice_side_faces(lat, s) for s in (1, 5)])]
    p = HO.HexOracleProblem(w)
    ext = w.box_extent
    area = ext[1] * ext[2] + ext[0] * ext[1]          # x+ and z+ walls (planar)
    assert abs(p.C.sum() - p.meshes[0].c * area) < 1e-12 * p.meshes[0].c * area
    X = _coords(p)
    p0 = W.seeded_field(4, X[:, 0], X[:, 1], X[:, 2])
    _, e = p.run(nsteps=80, p0=p0, energy=True, receivers=w.receivers[:1])
    lf = e[:, 0, 0]
    assert np.all(np.diff(lf) <= 1e-12 * lf[0]) and lf[-1] < 0.999 * lf[0]


def test_pml_on_the_affine_box_is_the_box_oracles():
    """Layers on an undistorted lattice give the box oracle's profiles, dt and
    traces (its PML is pinned by the plane-pulse reflection)."""
    wb = W.small_one_domain(nel=(4, 2, 2), order=3, nsteps=40)
    wb.domains[0].pml = (75e-6, 0.0, 0.0, 75e-6, 0.0, 75e-6)
    wh = H.hex_workload_from_box(wb)
    wh.pml, wh.pml_R = [wb.domains[0].pml], wb.domains[0].pml_R
    pb, ph = O.OracleProblem(wb), HO.HexOracleProblem(wh)
    idx = _map_nodes(pb, ph, 1e-15)
    np.testing.assert_allclose(ph.pml["zeta"][:, idx], pb.pml["zeta"], rtol=1e-12, atol=1e-6)
    assert abs(ph.stable_dt() - pb.stable_dt()) < 1e-15 * pb.stable_dt()
    dt = pb.stable_dt()
    tb = pb.run(dt=dt)
    th = ph.run(dt=dt)
    assert np.linalg.norm(th - tb) < 1e-11 * np.linalg.norm(tb)


def test_pml_on_a_curved_mesh_absorbs():
    """A smooth field in a distorted box with layers on every side loses
    most of its acoustic leapfrog energy, without late-time growth (the
    acoustic part alone is not an invariant of the layer system, so the first
    steps may exchange energy with Phi and psi)."""
    w = H.distorted_one_domain(nel=(4, 4, 3), order=3, nsteps=5, h=50e-6)
    w.pmuts = None
    w.pml, w.pml_R = [(50e-6,) * 6], 1e-3
    p = HO.HexOracleProblem(w)
    X = _coords(p)
    p0 = W.seeded_field(5, X[:, 0], X[:, 1], X[:, 2])
    _, e = p.run(nsteps=400, p0=p0, energy=True, receivers=w.receivers[:1])
    lf = e[:, 0, 0]
    assert np.all(np.isfinite(lf)) and lf[-1] < 1e-3 * lf[0]
    assert np.max(lf) < 1.1 * lf[0]
    # no late-time growth: every later window stays below the energy at step 200
    assert np.max(lf[240:]) < lf[200] and np.max(lf[320:]) < lf[280]


def test_unstructured_nonconforming_interface_matching():
    """A flat interface between a 6 x 6 fine tiling and an independently
    distorted 4 x 4 coarse tiling (3:2, faces straddling coarse faces):
    Algorithm 3 matches every fine Gauss node to the lowest-id coarse face
    whose element contains it (checked by brute force over all coarse
    elements), K is symmetric and annihilates constants."""
    w = H.distorted_two_domain(nx_p=6, nz_p=1, nx_s=4, nz_s=2, bump=0.0, n_pmut_side=1, order_p=3, order_s=4)
    p = HO.HexOracleProblem(w)
    m1 = p.meshes[1]
    straddled = 0
    for F, refp, xq, per in p.matches:
        elems = set()
        for q, (gi, refm) in enumerate(per):
            G = p.coarse_faces[gi]
            elems.add(G.elem)
            x, _ = HO.trilinear(m1.elem_verts(G.elem), refm[None, :])
            assert np.linalg.norm(x[0] - xq[q]) < 1e-12 * 1e-4
            # brute force: the lowest-id coarse face whose element contains the node
            first = None
            for gj, H2 in enumerate(p.coarse_faces):
                r = HO.newton_reference(m1.elem_verts(H2.elem), xq[q])
                if np.all(np.abs(r) <= 1.0 + 1e-10):
                    first = gj
                    break
            assert first == gi
        straddled += len(elems) > 1
    assert straddled > 0
    assert abs(p.K - p.K.T).max() < 1e-12 * abs(p.K).max()
    assert np.max(np.abs(p.K @ np.ones(p.nh))) < 1e-12 * abs(p.K).sum(axis=1).max()


def test_rayleigh_integral_on_a_distorted_mesh():
    """A 0.3 mm membrane moved with a prescribed acceleration (huge modal
    mass, no stiffness) in the flat z = 0 face of a distorted 0.6 mm cube:
    before the first wall echo the on-axis pressure is the Rayleigh integral
    of a baffled surface, p = rho / (2 pi) int a_n(y, t - R / c) / R dA.  Pins
    the Nanson-weighted PMUT matrix, kappa and the curved-element stiffness
    together; the error falls spectrally from N = 4 to N = 5."""
    a, z0, f = 0.3e-3, 0.15e-3, 8.0e6
    errs = []
    for N in (4, 5):
        w = H.distorted_one_domain(nel=(8, 8, 8), order=N, h=75e-6, amp=0.15, nsteps=10)
        w.pmuts = W.PmutArray(centers=np.array([[0.3e-3, 0.3e-3]]), side=a, freq_hz=np.array([[1.0]]),
                              damping=np.array([[0.0]]), eta=np.array([[1.0e6]]),
                              modal_mass=np.array([[1.0e6]]))
        w.receivers = np.array([[0.3e-3, 0.3e-3, z0]])
        w.drive_delay, w.drive_amp = np.zeros((1, 1)), np.ones((1, 1))
        w.burst_freq, w.burst_cycles = f, 1.0
        P = HO.HexOracleProblem(w)
        dt = P.stable_dt()
        S = int(0.31e-6 / dt)          # the x = 0 wall's first echo arrives at 0.316 us
        tr = P.run(nsteps=S, dt=dt)[0, 0]
        Tb = 1.0 / f

        def qdd(s):
            on = (s >= 0) & (s <= Tb)
            return np.where(on, np.sin(2 * math.pi * f * s) * 0.5 * (1 - np.cos(2 * math.pi * s / Tb)), 0.0)
        g, gw = np.polynomial.legendre.leggauss(80)
        X, Y = np.meshgrid(g, g, indexing="ij")
        wts = np.outer(gw, gw) * (a / 2) ** 2
        phi = (1 - X ** 2) ** 2 * (1 - Y ** 2) ** 2
        R = np.sqrt((X * a / 2) ** 2 + (Y * a / 2) ** 2 + z0 ** 2)
        rho, c = w.domains[0].rho, w.domains[0].c
        t = (np.arange(S) + 1) * dt
        ref = np.array([rho / (2 * math.pi) * np.sum(wts * qdd(tt - dt - R / c) * phi / R) for tt in t])
        assert np.abs(ref).max() > 0
        errs.append(np.linalg.norm(tr - ref) / np.linalg.norm(ref))
    assert errs[0] < 0.06 and errs[1] < 0.012, errs
    assert errs[0] / errs[1] > 3, errs
