"""Plain, slow FP64 CPU oracle for the DG-SEM step on general hexahedra.

TEST INFRASTRUCTURE ONLY.  Only tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code
with the CUDA path.

Paper passages followed (arXiv 2603.06267):
  * every element is K = X_K(K^) with a trilinear invertible map X_K of
    positive Jacobian (Sec. 3); V^DG is C0 Q_r inside each domain and
    discontinuous across Gamma_I;
  * bilinear forms of eq. (Wf_2) (volume term and the SIPG interface terms
    with gamma_F), lumped GLL mass (Sec. 3.1);
  * interface integrals on the quadrature nodes of the finer faces and the
    face matching of Algorithm 3 (normal filter |n+ + n-| < tol, one stored
    vertex per coarser face within r = max(diam) + eps of the node, Newton-
    Raphson for the reference position, containment in [-1, 1]^3), Sec. 5;
  * the time loop, PMUT model and receivers are those of ``dgsem_oracle``
    (Algorithm 1 with three vectors per field).

Readings where the paper is silent (the box oracle's readings apply; these
are the extra ones for curved elements):
  * the normal used by the matching filter is the face normal at the face
    centre (a bilinear face has no single normal);
  * h in gamma_F is |K| / |F| (element volume over face area), the element
    length normal to the face for a box; per interface quadrature node the
    minimum over the fine element and the matched coarse element; |K| and |F|
    are computed with the GLL rule of the element's order (exact for |K|);
  * the surface Jacobian at a face point is |J| |J^-T e_axis| (Nanson) and the
    outward normal J^-T e_axis / |J^-T e_axis| times the face's side sign;
  * the CFL length of an element is its shortest edge: dt = CFL * min_K
    (h_min,K / 2 * min GLL gap(N_K)) / c_max (the box reading for boxes);
  * the PMUT face weights W_j = sum_F w_a w_b |J_F| at the face's GLL nodes;
  * a receiver lies in the lowest-id element (primary first) whose Newton
    reference position is inside [-1, 1]^3 up to 1e-10;
  * absorbing faces: C_jj = sum_F c w_a w_b |J_F| at the face's GLL nodes
    (the box reading with the Nanson surface Jacobian), dt at most
    1 / max_j (C_jj / M_jj + alpha_j);
  * perfectly matched layers: the box reading (psi nodal, Phi element-local
    at the GLL nodes, Crank-Nicolson damping of Phi, half steps), the layers
    measured from the domain's bounding-box sides, gradients J^-T grad^.
Node numbering: nodes of one domain at the same physical position (within
1e-9 of the domain size) are one node, numbered in order of first appearance
over the elements (element order, then local index a + (N+1) b + (N+1)^2 c).
"""
from __future__ import annotations

import math
from typing import List, Optional

import numpy as np
import scipy.sparse as sp
from scipy.spatial import cKDTree

from .dgsem_oracle import (OracleProblem, gauss_legendre, gll_nodes_weights, reference_basis)

# reference corners, corner (i, j, k) at index i + 2 j + 4 k
CORNERS = np.array([[2 * (c & 1) - 1, 2 * ((c >> 1) & 1) - 1, 2 * ((c >> 2) & 1) - 1] for c in range(8)],
                   dtype=np.float64)


def trilinear(verts, ref):
    """X_K(ref) and J_K(ref) (J[n, i, d] = d X_i / d xi_d) of the trilinear
    map with corner vertices verts [8, 3] at reference points ref [n, 3]."""
    ref = np.atleast_2d(np.asarray(ref, dtype=np.float64))
    f = 0.5 * (1.0 + ref[:, None, :] * CORNERS[None, :, :])           # [n, 8, 3]
    shape = f.prod(axis=2)                                             # [n, 8]
    X = shape @ verts
    dshape = np.empty(f.shape)
    for d in range(3):
        others = [e for e in range(3) if e != d]
        dshape[:, :, d] = 0.5 * CORNERS[None, :, d] * f[:, :, others[0]] * f[:, :, others[1]]
    J = np.einsum("ncd,ci->nid", dshape, verts)
    return X, J


def newton_reference(verts, x, iters=50):
    """Reference position of x in the element with corners verts by
    Newton-Raphson on X_K(ref) = x, started at the centre."""
    ref = np.zeros(3)
    for _ in range(iters):
        X, J = trilinear(verts, ref[None, :])
        step = np.linalg.solve(J[0], X[0] - x)
        ref = ref - step
        if np.max(np.abs(step)) < 1e-15:
            break
    return ref


def face_points(f, st):
    """Reference points of local face f = 2 axis + side at face-local
    coordinates st [n, 2] (the two other axes in increasing order)."""
    ax, side = f // 2, f % 2
    t = [d for d in range(3) if d != ax]
    ref = np.zeros((len(st), 3))
    ref[:, ax] = 1.0 if side else -1.0
    ref[:, t[0]] = st[:, 0]
    ref[:, t[1]] = st[:, 1]
    return ref


def face_normal_and_jac(J, f):
    """Outward unit normal and surface Jacobian |J| |J^-T e_axis| at points
    of local face f, from the volume Jacobians J [n, 3, 3]."""
    ax, side = f // 2, f % 2
    Jinv = np.linalg.inv(J)
    g = Jinv[:, ax, :]                       # row ax of J^-1 = (J^-T e_ax)^T
    gn = np.linalg.norm(g, axis=1)
    det = np.linalg.det(J)
    sgn = 1.0 if side else -1.0
    return sgn * g / gn[:, None], det * gn


class HexMesh:
    """One domain of trilinear hexahedra with C0 GLL nodes of order N."""

    def __init__(self, dom, offset: int):
        self.dom = dom
        self.N = int(dom.order)
        self.c = float(dom.c)
        self.rho = float(dom.rho)
        self.verts = np.asarray(dom.vertices, dtype=np.float64)
        self.elems = np.asarray(dom.elements, dtype=np.int64)
        self.ne = self.elems.shape[0]
        self.xi, self.w = gll_nodes_weights(self.N)
        n = self.N + 1
        A, B, C = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
        # local index a + n b + n^2 c
        self.loc = np.stack([A.transpose(2, 1, 0).ravel(), B.transpose(2, 1, 0).ravel(),
                             C.transpose(2, 1, 0).ravel()], axis=1)
        self.ref_nodes = self.xi[self.loc]
        self.wq = self.w[self.loc].prod(axis=1)
        # physical positions of every element-local node
        X = np.empty((self.ne, n ** 3, 3))
        self.J = np.empty((self.ne, n ** 3, 3, 3))
        for e in range(self.ne):
            X[e], self.J[e] = trilinear(self.elem_verts(e), self.ref_nodes)
        self.detJ = np.linalg.det(self.J)
        if np.any(self.detJ <= 0.0):
            raise ValueError("element with a non-positive Jacobian")
        # C0 numbering: equal positions are one node (first appearance order)
        flat = X.reshape(-1, 3)
        size = float(np.max(np.ptp(self.verts, axis=0)))
        pairs = cKDTree(flat).query_pairs(1e-9 * size, output_type="ndarray")
        parent = np.arange(flat.shape[0])

        def root(i):
            while parent[i] != i:
                parent[i] = parent[parent[i]]
                i = parent[i]
            return i
        for a, b in pairs:
            ra, rb = root(a), root(b)
            if ra != rb:
                parent[max(ra, rb)] = min(ra, rb)
        roots = np.array([root(i) for i in range(flat.shape[0])])
        uniq, first = np.unique(roots, return_index=True)
        order = np.argsort(first)
        rank = np.empty(uniq.size, dtype=np.int64)
        rank[order] = np.arange(uniq.size)
        lookup = dict(zip(uniq.tolist(), rank.tolist()))
        self.conn = np.array([lookup[r] for r in roots], dtype=np.int64).reshape(self.ne, n ** 3) + offset
        self.nnode = uniq.size
        self.offset = offset
        self.coords = np.empty((self.nnode, 3))
        self.coords[self.conn.ravel() - offset] = flat

    def elem_verts(self, e):
        return self.verts[self.elems[e]]

    def volume(self, e):
        return float(np.sum(self.wq * self.detJ[e]))

    def face_area(self, e, f):
        """|F| with the GLL rule of the element's order (reading above)."""
        S, T = np.meshgrid(self.xi, self.xi, indexing="ij")
        st = np.column_stack([S.T.ravel(), T.T.ravel()])
        W = np.outer(self.w, self.w).T.ravel()
        _, J = trilinear(self.elem_verts(e), face_points(f, st))
        _, dS = face_normal_and_jac(J, f)
        return float(np.sum(W * dS))

    def face_local_nodes(self, f):
        """Local node indices on face f, ordered with the first tangential
        axis fastest, and their (a, b) GLL indices."""
        ax, side = f // 2, f % 2
        t = [d for d in range(3) if d != ax]
        fixed = self.N if side else 0
        sel = np.nonzero(self.loc[:, ax] == fixed)[0]
        key = self.loc[sel][:, t[1]] * (self.N + 1) + self.loc[sel][:, t[0]]
        sel = sel[np.argsort(key)]
        return sel, self.loc[sel][:, t[0]], self.loc[sel][:, t[1]]

    def h_min(self, e):
        V = self.elem_verts(e)
        edges = [(0, 1), (2, 3), (4, 5), (6, 7), (0, 2), (1, 3), (4, 6), (5, 7), (0, 4), (1, 5), (2, 6), (3, 7)]
        return min(float(np.linalg.norm(V[a] - V[b])) for a, b in edges)


def hex_element_stiffness(m: HexMesh, e: int, grad_ref):
    """K^e_ij = sum_q w_q |J_q| c^2 grad psi_i . grad psi_j, grad psi =
    J^-T grad^ psi, over the (N+1)^3 GLL points (eq. Wf_2, volume term)."""
    Jinv = np.linalg.inv(m.J[e])                                 # [q, d, x]
    grad = np.einsum("qdx,qjd->qjx", Jinv, grad_ref)
    return m.c ** 2 * np.einsum("q,qix,qjx->ij", m.wq * m.detJ[e], grad, grad, optimize=True)


class _HexFace:
    def __init__(self, mesh: HexMesh, elem: int, f: int):
        self.mesh, self.elem, self.f = mesh, int(elem), int(f)
        V = mesh.elem_verts(self.elem)
        ax, side = self.f // 2, self.f % 2
        cs = [c for c in range(8) if ((c >> ax) & 1) == side]
        self.verts = V[cs]
        self.vertex = self.verts[0]                   # the one stored vertex (Sec. 5)
        self.diam = float(np.max(np.linalg.norm(self.verts[:, None, :] - self.verts[None, :, :], axis=-1)))
        _, J = trilinear(V, face_points(self.f, np.zeros((1, 2))))
        n, _ = face_normal_and_jac(J, self.f)
        self.normal = n[0]                            # normal at the face centre
        self.area = mesh.face_area(self.elem, self.f)
        self.h = mesh.volume(self.elem) / self.area


def match_hex_interface(fine, coarse, quad_st, tol=0.5, eps=1e-12):
    """Algorithm 3 on trilinear elements: for each quadrature node of each
    finer face, the first coarser face (list order) with |n+ + n-| < tol whose
    stored vertex lies within max(diam) + eps of the node and whose element
    contains the node (Newton reference position in [-1, 1]^3)."""
    out = []
    for F in fine:
        V = F.mesh.elem_verts(F.elem)
        refp = face_points(F.f, quad_st)
        xq, _ = trilinear(V, refp)
        per = []
        for q in range(len(xq)):
            found = None
            for gi, G in enumerate(coarse):
                if np.linalg.norm(F.normal + G.normal) >= tol:
                    continue
                if np.linalg.norm(G.vertex - xq[q]) > max(F.diam, G.diam) + eps:
                    continue
                refm = newton_reference(G.mesh.elem_verts(G.elem), xq[q])
                if np.all(np.abs(refm) <= 1.0 + 1e-10):
                    found = (gi, refm)
                    break
            if found is None:
                raise ValueError("interface quadrature node without a coarse neighbour")
            per.append(found)
        out.append((F, refp, xq, per))
    return out


def hex_interface_matrix(prim: HexMesh, sec: HexMesh, fine_faces, coarse_faces, nh, alpha, nq, tol):
    """Sparse K_I of the three interface integrals of eq. (Wf_2) on the GL
    nodes of the finer faces, with per-node normals, Nanson weights and
    gamma_F = alpha cbar^2 max(N)^2 / min(h+, h-)."""
    g, gw = gauss_legendre(nq)
    S, T = np.meshgrid(g, g, indexing="ij")
    quad_st = np.column_stack([S.T.ravel(), T.T.ravel()])
    quad_w = np.outer(gw, gw).T.ravel()
    fine = [_HexFace(prim, e, f) for e, f in fine_faces]
    coarse = [_HexFace(sec, e, f) for e, f in coarse_faces]
    matches = match_hex_interface(fine, coarse, quad_st, tol)
    cp, cm = prim.c, sec.c
    cbar = 2.0 * cp * cm / (cp + cm)
    Nmax = max(prim.N, sec.N)
    rows, cols, vals = [], [], []
    for F, refp, xq, per in matches:
        Vp = prim.elem_verts(F.elem)
        _, Jp = trilinear(Vp, refp)
        nplus, dS = face_normal_and_jac(Jp, F.f)
        val_p, gref_p = reference_basis(prim.N, prim.xi, refp)
        grad_p = np.einsum("qdx,qjd->qjx", np.linalg.inv(Jp), gref_p)
        ids_p = prim.conn[F.elem]
        groups = {}
        for q, (gi, refm) in enumerate(per):
            groups.setdefault(coarse[gi].elem, (coarse[gi], []))[1].append((q, refm))
        for _, (G, items) in groups.items():
            qs = np.array([q for q, _ in items])
            refm = np.array([r for _, r in items])
            _, Jm = trilinear(sec.elem_verts(G.elem), refm)
            val_m, gref_m = reference_basis(sec.N, sec.xi, refm)
            grad_m = np.einsum("qdx,qjd->qjx", np.linalg.inv(Jm), gref_m)
            ids = np.concatenate([ids_p, sec.conn[G.elem]])
            n = nplus[qs]
            jump = np.concatenate([val_p[qs][:, :, None] * n[:, None, :],
                                   -val_m[:, :, None] * n[:, None, :]], axis=1)
            avg = np.concatenate([0.5 * cp ** 2 * grad_p[qs], 0.5 * cm ** 2 * grad_m], axis=1)
            W = quad_w[qs] * dS[qs]
            gam = alpha * cbar ** 2 * Nmax ** 2 / min(F.h, G.h)
            aj = np.einsum("q,qid,qjd->ij", W, jump, avg, optimize=True)
            blk = -aj - aj.T + gam * np.einsum("q,qid,qjd->ij", W, jump, jump, optimize=True)
            R, C = np.meshgrid(ids, ids, indexing="ij")
            nz = blk != 0.0
            rows.append(R[nz]); cols.append(C[nz]); vals.append(blk[nz])
    KI = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                       shape=(nh, nh)).tocsr()
    return KI, matches, coarse


class HexOracleProblem(OracleProblem):
    """Assembled M, K (volume + interface), PMUT matrix B and receivers for
    general hexahedral domains; the time loop is the box oracle's Algorithm 1."""

    def __init__(self, workload, penalty_alpha: Optional[float] = None, quad_pts: Optional[int] = None):
        self.w = workload
        self.meshes: List[HexMesh] = []
        off = 0
        for d in workload.domains:
            m = HexMesh(d, off)
            self.meshes.append(m)
            off += m.nnode
        self.nh = off
        alpha = workload.penalty_alpha if penalty_alpha is None else penalty_alpha
        nq = quad_pts if quad_pts is not None else (workload.quad_pts or 0)
        if nq == 0:
            nq = max(m.N for m in self.meshes) + 1
        self.alpha, self.nq = alpha, nq
        self._assemble_volume()
        self.gamma = None
        self.matches = None
        if len(self.meshes) == 2:
            KI, self.matches, self.coarse_faces = hex_interface_matrix(
                self.meshes[0], self.meshes[1], workload.fine_faces, workload.coarse_faces, self.nh,
                alpha, nq, workload.normal_tol)
            self.K = (self.K + KI).tocsr()
        self.Minv = 1.0 / self.M
        self._absorbing_matrix()
        self._hex_pml_setup()
        self._pmut_matrix()

    def _assemble_volume(self):
        rows, cols, vals = [], [], []
        M = np.zeros(self.nh)
        for m in self.meshes:
            _, grad_ref = reference_basis(m.N, m.xi, m.ref_nodes)
            for e in range(m.ne):
                Ke = hex_element_stiffness(m, e, grad_ref)
                ids = m.conn[e]
                R, C = np.meshgrid(ids, ids, indexing="ij")
                rows.append(R.ravel()); cols.append(C.ravel()); vals.append(Ke.ravel())
                np.add.at(M, ids, m.wq * m.detJ[e])
        self.K = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                               shape=(self.nh, self.nh)).tocsr()
        self.M = M

    def _absorbing_matrix(self):
        """Diagonal C of the damping form d of eq. (Wf_4) on the absorbing
        faces: C_jj = sum_F c w_a w_b |J_F| at the face's GLL nodes (the
        collocation of the box oracle, with the Nanson surface Jacobian)."""
        C = np.zeros(self.nh)
        faces = getattr(self.w, "absorbing_faces", None)
        if faces:
            for m, fl in zip(self.meshes, faces):
                if fl is None:
                    continue
                for e, f in np.asarray(fl).reshape(-1, 2):
                    sel, a, b = m.face_local_nodes(int(f))
                    _, J = trilinear(m.elem_verts(int(e)), m.ref_nodes[sel])
                    _, dS = face_normal_and_jac(J, int(f))
                    np.add.at(C, m.conn[int(e), sel], m.c * m.w[a] * m.w[b] * dS)
        self.C = C

    def _hex_pml_setup(self):
        """Perfectly matched layers (eq. full_problem rows 1-3, profile of
        Sec. 2) on curved elements: zeta_d at every node from its coordinate's
        depth into the layers of the domain's bounding box, and per layer
        element its node ids, the physical gradients J^-T grad^ psi at its GLL
        nodes, w |J| and c^2 -- the inputs of the box oracle's PML step."""
        self.pml = None
        layers = getattr(self.w, "pml", None)
        if not layers:
            return
        R = float(getattr(self.w, "pml_R", 1e-4))
        zeta = np.zeros((3, self.nh))
        elems = []
        for m, th in zip(self.meshes, layers):
            if th is None or not any(t > 0 for t in th):
                continue
            lo, hi = m.verts.min(axis=0), m.verts.max(axis=0)
            ids_all = np.arange(m.offset, m.offset + m.nnode)
            for d in range(3):
                for side, t in ((0, th[2 * d]), (1, th[2 * d + 1])):
                    if t <= 0:
                        continue
                    zt = m.c / t * math.log(1.0 / R)
                    x = m.coords[:, d]
                    s = (lo[d] + t - x) / t if side == 0 else (x - (hi[d] - t)) / t
                    s = np.clip(s, 0.0, 1.0)
                    zeta[d, ids_all] += zt * (s - np.sin(2 * math.pi * s) / (2 * math.pi))
            _, gref = reference_basis(m.N, m.xi, m.ref_nodes)
            for e in range(m.ne):
                ids = m.conn[e]
                if np.any(zeta[:, ids] != 0.0):
                    grad = np.einsum("qdx,qjd->qjx", np.linalg.inv(m.J[e]), gref)
                    elems.append((ids, grad, m.wq * m.detJ[e], m.c ** 2))
        if not elems:
            return
        z1, z2, z3 = zeta
        self.pml = dict(zeta=zeta, alpha=z1 + z2 + z3, beta=z1 * z2 + z2 * z3 + z3 * z1, gamma=z1 * z2 * z3,
                        elems=elems)

    def pmut_face_nodes(self):
        """Unique node ids on the PMUT faces, their positions and the
        assembled face weights W_j = sum_F w_a w_b |J_F|."""
        m = self.meshes[0]
        W = {}
        for e, f in self.w.pmut_faces:
            sel, a, b = m.face_local_nodes(int(f))
            _, J = trilinear(m.elem_verts(int(e)), m.ref_nodes[sel])
            _, dS = face_normal_and_jac(J, int(f))
            for s, wa, wb, ds in zip(sel, m.w[a], m.w[b], dS):
                j = int(m.conn[int(e), s])
                W[j] = W.get(j, 0.0) + wa * wb * ds
        ids = np.array(sorted(W), dtype=np.int64)
        return ids, m.coords[ids - m.offset], np.array([W[j] for j in ids])

    def _pmut_matrix(self):
        pm = self.w.pmuts
        if pm is None or self.w.pmut_faces is None:
            self.B = None
            return
        ids, xyz, Wf = self.pmut_face_nodes()
        K, Mm = pm.n_pmut, pm.n_modes
        rows, cols, vals = [], [], []
        for k in range(K):
            inside = pm.inside(k, xyz[:, 0], xyz[:, 1])
            for mm in range(Mm):
                un = pm.shape_un(k, mm, xyz[inside, 0], xyz[inside, 1])
                rows.append(ids[inside]); cols.append(np.full(inside.sum(), k * Mm + mm))
                vals.append(Wf[inside] * un)
        self.B = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                               shape=(self.nh, K * Mm)).tocsr()
        self.kappa = self.meshes[0].rho * self.meshes[0].c ** 2

    def receiver_matrix(self, points):
        points = np.asarray(points, dtype=np.float64).reshape(-1, 3)
        rows, cols, vals = [], [], []
        for r, x in enumerate(points):
            done = False
            for m in self.meshes:
                for e in range(m.ne):
                    V = m.elem_verts(e)
                    lo, hi = V.min(axis=0), V.max(axis=0)
                    pad = 1e-9 * float(np.max(hi - lo))
                    if np.any(x < lo - pad) or np.any(x > hi + pad):
                        continue
                    ref = newton_reference(V, x)
                    if np.all(np.abs(ref) <= 1.0 + 1e-10):
                        val, _ = reference_basis(m.N, m.xi, np.clip(ref, -1.0, 1.0)[None, :])
                        rows.append(np.full(m.conn[e].size, r)); cols.append(m.conn[e]); vals.append(val[0])
                        done = True
                        break
                if done:
                    break
            if not done:
                raise ValueError(f"receiver {r} outside the mesh")
        return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(len(points), self.nh)).tocsr()

    def stable_dt(self, cfl: Optional[float] = None):
        """CFL on the shortest element edge (reading R24), and with absorbing
        faces at most 1 / max_j (C_jj / M_jj) like the box oracle (the damping
        of Algorithm 1 is explicit)."""
        cfl = self.w.cfl if cfl is None else cfl
        cmax = max(m.c for m in self.meshes)
        hmin = min(min(m.h_min(e) for e in range(m.ne)) / 2.0 * float(np.min(np.diff(m.xi)))
                   for m in self.meshes)
        dt = cfl * hmin / cmax
        damp = self.C * self.Minv
        if self.pml is not None:
            damp = damp + self.pml["alpha"]
        sigma = float(np.max(damp))
        if sigma > 0.0:
            dt = min(dt, 1.0 / sigma)
        return dt

    def all_coordinates(self):
        X = np.concatenate([m.coords for m in self.meshes])
        return X[:, 0], X[:, 1], X[:, 2]
