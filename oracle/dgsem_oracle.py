"""Plain, slow FP64 CPU oracle for the DG-SEM + reduced-order PMUT explicit step.

TEST INFRASTRUCTURE ONLY.  Only tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code
with the CUDA path: it builds its own GLL/GL tables, its own element matrices
by quadrature, its own interface matrix by brute-force face matching, and
integrates with the paper's three-vector Newmark scheme literally.

Paper passages followed (arXiv 2603.06267):
  * problem: Sec. 2, eq. (full_problem) rows 1, 6-10 without PML;
    PMUT modal ODEs eq. (ode)/(pmut_problem).
  * TX -> RX switch (eq. ode row 2, eq. pmut_problem row 2): from step
    rx_switch on, phi_k^n = s / C_k sum_m eta_km q_km^n with the modal
    coordinates of step n (the q that Algorithm 1's PMUT solve pairs with
    p^n); s = +1 is the literal equation, s = -1 the stiffening reading.
  * perfectly matched layer, eq. (full_problem) rows 1-3 with the damping
    profile zeta_i of Sec. 2 (zeta~ = c / l log(1/R), the layer measured
    from its inner face).  Readings (the paper only says the scheme is
    similar to Algorithm 1): psi in the nodal space of p; Phi element-local
    at the GLL nodes; int (div Phi) v integrated by parts to -int Phi.grad v
    (the natural condition is on the total flux); psi and Phi at half steps
    like the velocity, the Phi damping by Crank-Nicolson, the alpha p' term on
    the predicted velocity like C p'_pred:
        psi^{n+1} = psi^{n+1/2} + dt/2 p^{n+1}
        Phi^{n+3/2} = [(1 - dt z/2) Phi^{n+1/2}
                       + dt c^2 ((alpha - 2 z) grad p^{n+1} + Z3 grad psi^{n+1})] / (1 + dt z/2)
        M p''^{n+1} = f - K p^{n+1} - C p'_pred - M (beta p^{n+1} + alpha p'_pred
                      + gamma psi^{n+1}) - G (Phi^{n+1/2} + Phi^{n+3/2}) / 2
        psi^{n+3/2} = psi^{n+1/2} + dt p^{n+1}
    with (G Phi)_j = sum_K sum_q w_q |J| Phi(x_q).grad psi_j(x_q); at rest
    (or at a set initial state) psi^{1/2} = 0, Phi^{1/2} = 0.
  * first-order absorbing boundary on Gamma_ABC: the damping form d of
    eq. (Wf_4), d(w, v) = sum_F int_F c w v, giving C of eq. (semi_SEM),
    applied to the predicted velocity as in Algorithm 1.
  * DG-SEM space V^DG (C0 Q_r inside each box, discontinuous across Gamma_I),
    bilinear forms m and a (SIPG), penalty gamma_F: Sec. 3, eqs. (Wf_1)-(Wf_2).
  * algebraic form M p'' + K p = f(q''), q'' + W q = g(p, phi), lumped GLL
    mass, f_i, g_m: Sec. 3.1, eqs. (semi_SEM), (semi_PMUT), (f_i), (g_m).
  * Newmark gamma = 1/2, beta = 0 predictor/corrector: Algorithm 1.
  * interface quadrature on the finer face and face matching (normal filter,
    one-vertex radius filter, Newton inverse map): Sec. 5, eq. (integral_DG),
    Algorithm 3.

Readings where the paper is silent:
  * modal ODE carries a modal mass and damping:
      mu (q'' + 2 zeta w q' + w^2 q) = int p U.n + eta phi,
    damping evaluated at the predicted velocity like C p'_pred in Alg. 1;
    mu = 1, zeta = 0 is the paper's literal equation.
  * the membrane integrals of f_i and g_m use GLL collocation on the face
    nodes, the same matrix B for both.
  * volume integrals use (N+1)^3-point GLL quadrature (spectral elements).
  * interface: q = max(N_in, N_out) + 1 Gauss-Legendre points per direction
    on each finer face; h in gamma_F is the element length normal to the
    face; c-bar is the harmonic mean.
  * time loop runs S steps (n = 0..S-1); trace sample n is p^{n+1}.
  * a non-zero initial state (p0, p'0) starts from p''0 = M^-1(-K p0 - C p'0).
  * the integral of d uses GLL collocation on the face nodes (like the
    lumped mass), so C is diagonal.  With absorbing sides dt is also held
    to 1 / max_j (C_jj / M_jj): the explicit damping of Algorithm 1 loses
    stability at a few times that (corner nodes of three absorbing sides).  The strong form's row 6 has the
    opposite sign convention to d; d is taken as written (it dissipates
    energy, which is what an absorbing condition does).
"""
from __future__ import annotations

import math
from typing import List, Optional

import numpy as np
import scipy.sparse as sp


# ----------------------------------------------------------------------------
# 1D polynomial tables (Sec. 3: GLL nodes of the SEM basis; Sec. 5: Gauss
# nodes of the interface quadrature)
# ----------------------------------------------------------------------------
def legendre_and_derivative(n: int, x):
    """P_n(x) and P_n'(x) by Bonnet's recurrence."""
    x = np.asarray(x, dtype=np.float64)
    p0 = np.ones_like(x)
    if n == 0:
        return p0, np.zeros_like(x)
    p1 = x.copy()
    d0 = np.zeros_like(x)
    d1 = np.ones_like(x)
    for k in range(1, n):
        p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
        d2 = d0 + (2 * k + 1) * p1
        p0, p1 = p1, p2
        d0, d1 = d1, d2
    return p1, d1


def gll_nodes_weights(N: int):
    """Gauss-Lobatto-Legendre nodes: -1, 1 and the roots of P_N'; weights
    2 / (N (N+1) P_N(x)^2)."""
    if N == 1:
        x = np.array([-1.0, 1.0])
    else:
        # Newton on P_N' from Chebyshev-Gauss-Lobatto guesses
        guess = -np.cos(np.pi * np.arange(1, N) / N)
        x_in = guess.copy()
        for _ in range(100):
            # second derivative from the Legendre ODE:
            # (1 - x^2) P'' = 2 x P' - N (N+1) P
            P, dP = legendre_and_derivative(N, x_in)
            d2P = (2 * x_in * dP - N * (N + 1) * P) / (1 - x_in ** 2)
            step = dP / d2P
            x_in = x_in - step
            if np.max(np.abs(step)) < 1e-16:
                break
        x = np.concatenate([[-1.0], x_in, [1.0]])
    P, _ = legendre_and_derivative(N, x)
    w = 2.0 / (N * (N + 1) * P ** 2)
    return x, w


def gauss_legendre(q: int):
    """Gauss-Legendre rule with q points (library routine)."""
    return np.polynomial.legendre.leggauss(q)


def lagrange_values(nodes, x):
    """l_a(x) for every node a, by the product formula. Shape [len(x), n]."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = nodes.size
    out = np.ones((x.size, n))
    for a in range(n):
        for m in range(n):
            if m != a:
                out[:, a] *= (x - nodes[m]) / (nodes[a] - nodes[m])
    return out


def lagrange_derivatives(nodes, x):
    """l_a'(x) for every node a: sum over the dropped factor of the product."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = nodes.size
    out = np.zeros((x.size, n))
    for a in range(n):
        for j in range(n):
            if j == a:
                continue
            term = np.full(x.size, 1.0 / (nodes[a] - nodes[j]))
            for m in range(n):
                if m != a and m != j:
                    term = term * (x - nodes[m]) / (nodes[a] - nodes[m])
            out[:, a] += term
    return out


# ----------------------------------------------------------------------------
# Mesh of one box domain (Sec. 3: hexahedra K = X_K(K^), affine special case
# of the trilinear maps; V_a^{r_a} is C0 inside the box)
# ----------------------------------------------------------------------------
class BoxMesh:
    def __init__(self, dom, offset: int):
        self.dom = dom
        self.N = int(dom.order)
        self.ne = tuple(int(v) for v in dom.nelem)
        self.h = tuple(float(dom.extent[i]) / self.ne[i] for i in range(3))
        self.origin = tuple(float(v) for v in dom.origin)
        self.c = float(dom.c)
        self.rho = float(dom.rho)
        self.xi, self.w = gll_nodes_weights(self.N)
        self.L = tuple(self.ne[i] * self.N + 1 for i in range(3))
        self.offset = offset
        self.nnode = self.L[0] * self.L[1] * self.L[2]
        # physical coordinate of lattice line i along axis d
        self.coord = []
        for d in range(3):
            e = np.arange(self.L[d]) // self.N
            a = np.arange(self.L[d]) % self.N
            e = np.minimum(e, self.ne[d] - 1)
            a = np.where(np.arange(self.L[d]) == self.L[d] - 1, self.N, a)
            self.coord.append(self.origin[d] + self.h[d] * (e + (self.xi[a] + 1.0) / 2.0))

    def node_id(self, i, j, k):
        return self.offset + (np.asarray(k) * self.L[1] + np.asarray(j)) * self.L[0] + np.asarray(i)

    def element_nodes(self, ex, ey, ez):
        """Global ids of the (N+1)^3 nodes of element (ex, ey, ez), a fastest."""
        N = self.N
        a = np.arange(N + 1)
        I, J, K = np.meshgrid(ex * N + a, ey * N + a, ez * N + a, indexing="ij")
        # order: index = (c * (N+1) + b) * (N+1) + a
        return self.node_id(I.transpose(2, 1, 0).ravel(), J.transpose(2, 1, 0).ravel(),
                            K.transpose(2, 1, 0).ravel())

    def element_map(self, ex, ey, ez, ref):
        """X_K(ref) for reference points ref [n, 3]."""
        ref = np.asarray(ref, dtype=np.float64)
        o = np.array([self.origin[d] + (ex, ey, ez)[d] * self.h[d] for d in range(3)])
        return o[None, :] + 0.5 * np.array(self.h)[None, :] * (ref + 1.0)

    def element_vertices(self, ex, ey, ez):
        corners = np.array([[sx, sy, sz] for sz in (-1, 1) for sy in (-1, 1) for sx in (-1, 1)], float)
        return self.element_map(ex, ey, ez, corners)

    def all_coordinates(self):
        X, Y, Z = np.meshgrid(self.coord[0], self.coord[1], self.coord[2], indexing="ij")
        # flatten in node-id order (i fastest)
        return (X.transpose(2, 1, 0).ravel(), Y.transpose(2, 1, 0).ravel(), Z.transpose(2, 1, 0).ravel())


def reference_basis(N, xi_nodes, pts):
    """Values and reference gradients of the (N+1)^3 tensor Lagrange basis at
    reference points pts [n, 3]; basis index (c*(N+1)+b)*(N+1)+a."""
    lx = lagrange_values(xi_nodes, pts[:, 0])
    ly = lagrange_values(xi_nodes, pts[:, 1])
    lz = lagrange_values(xi_nodes, pts[:, 2])
    dx = lagrange_derivatives(xi_nodes, pts[:, 0])
    dy = lagrange_derivatives(xi_nodes, pts[:, 1])
    dz = lagrange_derivatives(xi_nodes, pts[:, 2])
    n = N + 1
    val = np.einsum("pc,pb,pa->pcba", lz, ly, lx).reshape(len(pts), n ** 3)
    g0 = np.einsum("pc,pb,pa->pcba", lz, ly, dx).reshape(len(pts), n ** 3)
    g1 = np.einsum("pc,pb,pa->pcba", lz, dy, lx).reshape(len(pts), n ** 3)
    g2 = np.einsum("pc,pb,pa->pcba", dz, ly, lx).reshape(len(pts), n ** 3)
    return val, np.stack([g0, g1, g2], axis=-1)


def element_stiffness(mesh: BoxMesh):
    """K^e_ij = sum_q w_q |J| c^2 grad psi_i(x_q) . grad psi_j(x_q) over the
    (N+1)^3 GLL points (eq. Wf_2, volume term)."""
    N = mesh.N
    xi, w = mesh.xi, mesh.w
    P, Q, R = np.meshgrid(xi, xi, xi, indexing="ij")
    pts = np.stack([P.transpose(2, 1, 0).ravel(), Q.transpose(2, 1, 0).ravel(),
                    R.transpose(2, 1, 0).ravel()], axis=1)
    WP, WQ, WR = np.meshgrid(w, w, w, indexing="ij")
    wq = (WP * WQ * WR).transpose(2, 1, 0).ravel()
    _, grad_ref = reference_basis(N, xi, pts)
    Jinv = np.array([2.0 / mesh.h[d] for d in range(3)])
    detJ = mesh.h[0] * mesh.h[1] * mesh.h[2] / 8.0
    grad = grad_ref * Jinv[None, None, :]
    Ke = mesh.c ** 2 * detJ * np.einsum("q,qid,qjd->ij", wq, grad, grad, optimize=True)
    return Ke


def element_lumped_mass(mesh: BoxMesh):
    """M^e_ii = w_a w_b w_c |J| (GLL reduced integration, Sec. 3.1)."""
    w = mesh.w
    detJ = mesh.h[0] * mesh.h[1] * mesh.h[2] / 8.0
    return np.einsum("c,b,a->cba", w, w, w).ravel() * detJ


# ----------------------------------------------------------------------------
# Interface: Sec. 5 fine-face quadrature + Algorithm 3 matching, eq. (Wf_2)
# interface terms with gamma_F
# ----------------------------------------------------------------------------
class _Face:
    def __init__(self, mesh, elem, side):
        self.mesh, self.elem, self.side = mesh, elem, side   # side: 'top' (zeta=+1) or 'bottom'
        verts = mesh.element_vertices(*elem)
        if side == "top":
            self.verts = verts[4:]
            self.normal = np.array([0.0, 0.0, 1.0])
        else:
            self.verts = verts[:4]
            self.normal = np.array([0.0, 0.0, -1.0])
        self.vertex = self.verts[0]                 # the one stored vertex (Sec. 5)
        self.diam = float(np.max(np.linalg.norm(self.verts[:, None, :] - self.verts[None, :, :], axis=-1)))


def newton_inverse_map(mesh: BoxMesh, elem, x, iters=20):
    """Reference coordinates of x in element elem by Newton-Raphson on the
    trilinear map (for affine boxes it converges in one step)."""
    verts = mesh.element_vertices(*elem)
    ref = np.zeros(3)
    for _ in range(iters):
        s = [(1 - ref[0]) / 2, (1 + ref[0]) / 2]
        t = [(1 - ref[1]) / 2, (1 + ref[1]) / 2]
        u = [(1 - ref[2]) / 2, (1 + ref[2]) / 2]
        X = np.zeros(3)
        J = np.zeros((3, 3))
        idx = 0
        for kz in range(2):
            for ky in range(2):
                for kx in range(2):
                    v = verts[idx]
                    X += s[kx] * t[ky] * u[kz] * v
                    J[:, 0] += (-0.5 if kx == 0 else 0.5) * t[ky] * u[kz] * v
                    J[:, 1] += s[kx] * (-0.5 if ky == 0 else 0.5) * u[kz] * v
                    J[:, 2] += s[kx] * t[ky] * (-0.5 if kz == 0 else 0.5) * v
                    idx += 1
        step = np.linalg.solve(J, X - x)
        ref = ref - step
        if np.max(np.abs(step)) < 1e-15:
            break
    return ref


def match_interface(fine_faces, coarse_faces, quad_ref, tol=1e-9, eps=1e-12):
    """Algorithm 3: for each fine face and each of its quadrature nodes, find
    the coarse face with opposite normal whose stored vertex lies within
    r = max(diam) + eps of the node and whose element contains the node."""
    matches = []
    for F in fine_faces:
        ref_plus = np.column_stack([quad_ref, np.ones(len(quad_ref))])
        x_q = F.mesh.element_map(*F.elem, ref_plus)
        per_point = []
        for q in range(len(x_q)):
            found = None
            for G in coarse_faces:
                if np.linalg.norm(F.normal + G.normal) >= tol:
                    continue
                r = max(F.diam, G.diam) + eps
                if np.linalg.norm(G.vertex - x_q[q]) > r:
                    continue
                ref_minus = newton_inverse_map(G.mesh, G.elem, x_q[q])
                if np.all(np.abs(ref_minus) <= 1.0 + 1e-10):
                    found = (G, ref_minus)
                    break
            if found is None:
                raise ValueError("interface quadrature node without a coarse neighbour")
            per_point.append(found)
        matches.append((F, ref_plus, per_point))
    return matches


def interface_matrix(prim: BoxMesh, sec: BoxMesh, nh: int, alpha: float, nq: int):
    """Sparse K_I from the three interface integrals of eq. (Wf_2), on the
    quadrature nodes of the finer (primary) faces."""
    g, gw = gauss_legendre(nq)
    GX, GY = np.meshgrid(g, g, indexing="ij")
    quad_ref = np.column_stack([GX.T.ravel(), GY.T.ravel()])
    WX, WY = np.meshgrid(gw, gw, indexing="ij")
    quad_w = (WX * WY).T.ravel()
    fine = [_Face(prim, (ex, ey, prim.ne[2] - 1), "top")
            for ey in range(prim.ne[1]) for ex in range(prim.ne[0])]
    coarse = [_Face(sec, (ex, ey, 0), "bottom")
              for ey in range(sec.ne[1]) for ex in range(sec.ne[0])]
    matches = match_interface(fine, coarse, quad_ref)
    cp, cm = prim.c, sec.c
    cbar = 2.0 * cp * cm / (cp + cm)
    h_in, h_out = prim.h[2], sec.h[2]
    gamma = alpha * cbar ** 2 * max(prim.N, sec.N) ** 2 / min(h_in, h_out)
    rows, cols, vals = [], [], []
    n_plus = np.array([0.0, 0.0, 1.0])
    scale_p = np.array([2.0 / prim.h[d] for d in range(3)])
    scale_m = np.array([2.0 / sec.h[d] for d in range(3)])
    for F, ref_plus, per_point in matches:
        area_jac = prim.h[0] * prim.h[1] / 4.0            # |J_F+| of the fine face
        ids_p = prim.element_nodes(*F.elem)
        val_p, gref_p = reference_basis(prim.N, prim.xi, ref_plus)
        grad_p = gref_p * scale_p[None, None, :]
        # group the quadrature nodes of this fine face by their coarse element
        groups = {}
        for q, (G, ref_minus) in enumerate(per_point):
            groups.setdefault(G.elem, (G, []))[1].append((q, ref_minus))
        for _, (G, items) in groups.items():
            qs = np.array([q for q, _ in items])
            refm = np.array([r for _, r in items])
            ids_m = sec.element_nodes(*G.elem)
            val_m, gref_m = reference_basis(sec.N, sec.xi, refm)
            grad_m = gref_m * scale_m[None, None, :]
            ids = np.concatenate([ids_p, ids_m])
            # vector jump [v] = v+ n+ + v- n-, with n- = -n+  (Sec. 3)
            jump = np.concatenate([val_p[qs][:, :, None] * n_plus[None, None, :],
                                   val_m[:, :, None] * (-n_plus)[None, None, :]], axis=1)
            # average {c^2 grad v}: each basis function lives on one side only
            avg = np.concatenate([0.5 * cp ** 2 * grad_p[qs], 0.5 * cm ** 2 * grad_m], axis=1)
            W = quad_w[qs] * area_jac
            # blk[i, j] = sum_q W_q (-avg_j.jump_i - avg_i.jump_j + gamma jump_i.jump_j)
            aj = np.einsum("q,qid,qjd->ij", W, jump, avg, optimize=True)
            blk = -aj - aj.T + gamma * np.einsum("q,qid,qjd->ij", W, jump, jump, optimize=True)
            R, C = np.meshgrid(ids, ids, indexing="ij")
            nz = blk != 0.0
            rows.append(R[nz]); cols.append(C[nz]); vals.append(blk[nz])
    if not rows:
        return sp.csr_matrix((nh, nh)), gamma
    KI = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                       shape=(nh, nh)).tocsr()
    return KI, gamma


# ----------------------------------------------------------------------------
# Assembled operators
# ----------------------------------------------------------------------------
class OracleProblem:
    """Assembled M (diagonal), K (volume + interface), PMUT matrix B and the
    receiver interpolation for a list of box domains (primary first)."""

    def __init__(self, workload, penalty_alpha: Optional[float] = None, quad_pts: Optional[int] = None):
        self.w = workload
        self.meshes: List[BoxMesh] = []
        off = 0
        for d in workload.domains:
            m = BoxMesh(d, off)
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
        if len(self.meshes) == 2:
            KI, self.gamma = interface_matrix(self.meshes[0], self.meshes[1], self.nh, alpha, nq)
            self.K = (self.K + KI).tocsr()
        self.Minv = 1.0 / self.M
        self._absorbing_matrix()
        self._pml_setup()
        self._pmut_matrix()

    def _assemble_volume(self):
        rows, cols, vals = [], [], []
        M = np.zeros(self.nh)
        for m in self.meshes:
            Ke = element_stiffness(m)
            Me = element_lumped_mass(m)
            nzr, nzc = np.nonzero(Ke)
            kv = Ke[nzr, nzc]
            for ez in range(m.ne[2]):
                for ey in range(m.ne[1]):
                    for ex in range(m.ne[0]):
                        ids = m.element_nodes(ex, ey, ez)
                        rows.append(ids[nzr]); cols.append(ids[nzc]); vals.append(kv)
                        np.add.at(M, ids, Me)
        self.K = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                               shape=(self.nh, self.nh)).tocsr()
        self.M = M

    def _absorbing_matrix(self):
        """Diagonal C of the damping form d (eq. Wf_4): for every element face
        F on an absorbing box side, C_jj += c w_a w_b |J_F| at its GLL nodes."""
        C = np.zeros(self.nh)
        for dom, m in zip(self.w.domains, self.meshes):
            sides = getattr(dom, "absorbing", (0,) * 6)
            N = m.N
            for side in range(6):
                if not sides[side]:
                    continue
                d = side // 2                      # normal direction
                t1, t2 = [e for e in range(3) if e != d]
                jac = m.h[t1] * m.h[t2] / 4.0      # face Jacobian of the affine face
                fixed = 0 if side % 2 == 0 else m.L[d] - 1
                for e2 in range(m.ne[t2]):
                    for e1 in range(m.ne[t1]):
                        for b in range(N + 1):
                            for a in range(N + 1):
                                idx = [0, 0, 0]
                                idx[d] = fixed
                                idx[t1] = e1 * N + a
                                idx[t2] = e2 * N + b
                                C[m.node_id(*idx)] += dom.c * m.w[a] * m.w[b] * jac
        self.C = C

    def _pml_setup(self):
        """Damping profiles zeta_d at every node, the node coefficients
        alpha, beta, gamma, and per PML element its node ids, GLL gradient
        matrix, quadrature weights and zeta at its nodes."""
        self.pml = None
        zeta = np.zeros((3, self.nh))
        elems = []
        for dom, m in zip(self.w.domains, self.meshes):
            th = getattr(dom, "pml", (0.0,) * 6)
            if not any(t > 0 for t in th):
                continue
            R = float(getattr(dom, "pml_R", 1e-4))
            x = m.all_coordinates()
            ids_all = np.arange(m.offset, m.offset + m.nnode)
            for d in range(3):
                lo = m.origin[d]
                hi = lo + m.ne[d] * m.h[d]
                for side, t in ((0, th[2 * d]), (1, th[2 * d + 1])):
                    if t <= 0:
                        continue
                    zt = m.c / t * math.log(1.0 / R)
                    s = (lo + t - x[d]) / t if side == 0 else (x[d] - (hi - t)) / t
                    s = np.clip(s, 0.0, 1.0)
                    zeta[d, ids_all] += zt * (s - np.sin(2 * math.pi * s) / (2 * math.pi))
            # GLL gradient matrix of the reference element at its own nodes
            N = m.N
            xi, w = m.xi, m.w
            P, Q, Rr = np.meshgrid(xi, xi, xi, indexing="ij")
            pts = np.stack([P.transpose(2, 1, 0).ravel(), Q.transpose(2, 1, 0).ravel(),
                            Rr.transpose(2, 1, 0).ravel()], axis=1)
            WP, WQ, WR = np.meshgrid(w, w, w, indexing="ij")
            wq = (WP * WQ * WR).transpose(2, 1, 0).ravel() * (m.h[0] * m.h[1] * m.h[2] / 8.0)
            _, gref = reference_basis(N, xi, pts)
            grad = gref * np.array([2.0 / m.h[d] for d in range(3)])[None, None, :]
            for ez in range(m.ne[2]):
                for ey in range(m.ne[1]):
                    for ex in range(m.ne[0]):
                        ids = m.element_nodes(ex, ey, ez)
                        if np.any(zeta[:, ids] != 0.0):
                            elems.append((ids, grad, wq, m.c ** 2))
        if not elems:
            return
        z1, z2, z3 = zeta
        self.pml = dict(zeta=zeta, alpha=z1 + z2 + z3, beta=z1 * z2 + z2 * z3 + z3 * z1, gamma=z1 * z2 * z3,
                        elems=elems)

    def _pml_step(self, Phi, psi_half, p_new, dt):
        """Phi^{n+1/2} -> Phi^{n+3/2} on every PML element and the residual
        G (Phi^{n+1/2} + Phi^{n+3/2}) / 2; psi^{n+1} = psi^{n+1/2} + dt/2 p^{n+1}."""
        zeta = self.pml["zeta"]
        psi_int = psi_half + 0.5 * dt * p_new
        r = np.zeros_like(p_new)
        new = []
        for (ids, grad, wq, c2), F in zip(self.pml["elems"], Phi):
            z = zeta[:, ids]                                   # [3, nq]
            al = z.sum(axis=0)
            Z3 = np.stack([z[1] * z[2], z[2] * z[0], z[0] * z[1]])
            gp = np.einsum("qid,ib->dqb", grad, p_new[ids])
            gs = np.einsum("qid,ib->dqb", grad, psi_int[ids])
            Fn = ((1.0 - 0.5 * dt * z)[:, :, None] * F
                  + dt * c2 * ((al[None, :] - 2.0 * z)[:, :, None] * gp + Z3[:, :, None] * gs)) \
                / (1.0 + 0.5 * dt * z)[:, :, None]
            Fm = 0.5 * (F + Fn)
            np.add.at(r, ids, np.einsum("q,qid,dqb->ib", wq, grad, Fm))
            new.append(Fn)
        return new, psi_int, r

    def face_nodes(self):
        """Ids and (x, y) of the GLL nodes on the z = origin face of the
        primary box (Gamma_PMUT lies there)."""
        m = self.meshes[0]
        I, J = np.meshgrid(np.arange(m.L[0]), np.arange(m.L[1]), indexing="ij")
        I, J = I.T.ravel(), J.T.ravel()
        return m.node_id(I, J, 0), m.coord[0][I], m.coord[1][J], I, J

    def _face_weights(self):
        """Assembled 2D GLL face weights W_j = sum_F w_a w_b |J_F| of the
        primary z = origin face."""
        m = self.meshes[0]
        N = m.N
        Wf = np.zeros((m.L[1], m.L[0]))
        area = m.h[0] * m.h[1] / 4.0
        for ey in range(m.ne[1]):
            for ex in range(m.ne[0]):
                Wf[ey * N:ey * N + N + 1, ex * N:ex * N + N + 1] += np.outer(m.w, m.w) * area
        return Wf.ravel()

    def _pmut_matrix(self):
        """B_{j,(k,m)} = int_{gamma_k} psi_j U_{k,m}.n dsigma by GLL collocation
        on the face nodes (eqs. f_i and g_m)."""
        pm = self.w.pmuts
        if pm is None:
            self.B = None
            return
        ids, x, y, _, _ = self.face_nodes()
        Wf = self._face_weights()
        K, Mm = pm.n_pmut, pm.n_modes
        rows, cols, vals = [], [], []
        for k in range(K):
            inside = pm.inside(k, x, y)
            for mm in range(Mm):
                un = pm.shape_un(k, mm, x[inside], y[inside])
                rows.append(ids[inside]); cols.append(np.full(inside.sum(), k * Mm + mm))
                vals.append(Wf[inside] * un)
        self.B = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                               shape=(self.nh, K * Mm)).tocsr()
        self.kappa = self.meshes[0].rho * self.meshes[0].c ** 2

    # ---------------------------------------------------------------- receivers
    def receiver_matrix(self, points):
        """Row r: tensor Lagrange weights of the element containing point r
        (lowest element id on ties; primary box first)."""
        points = np.asarray(points, dtype=np.float64).reshape(-1, 3)
        rows, cols, vals = [], [], []
        for r, x in enumerate(points):
            done = False
            for m in self.meshes:
                lo = np.array(m.origin)
                hi = lo + np.array([m.ne[d] * m.h[d] for d in range(3)])
                tol = 1e-12 * np.max(hi - lo)
                if np.any(x < lo - tol) or np.any(x > hi + tol):
                    continue
                for ez in range(m.ne[2]):
                    for ey in range(m.ne[1]):
                        for ex in range(m.ne[0]):
                            elo = lo + np.array([ex, ey, ez]) * np.array(m.h)
                            ehi = elo + np.array(m.h)
                            if np.any(x < elo - tol) or np.any(x > ehi + tol):
                                continue
                            ref = np.clip(2.0 * (x - elo) / np.array(m.h) - 1.0, -1.0, 1.0)
                            val, _ = reference_basis(m.N, m.xi, ref[None, :])
                            ids = m.element_nodes(ex, ey, ez)
                            rows.append(np.full(ids.size, r)); cols.append(ids); vals.append(val[0])
                            done = True
                            break
                        if done:
                            break
                    if done:
                        break
                if done:
                    break
            if not done:
                raise ValueError(f"receiver {r} outside the mesh")
        return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(len(points), self.nh)).tocsr()

    # ---------------------------------------------------------------- time step
    def stable_dt(self, cfl: Optional[float] = None):
        """dt = CFL * min_K min_d (h_d / 2 * min GLL gap) / c_max  (reading of
        the CFL bound dt <~ h_min, Sec. 3.1).  With absorbing sides the
        damping term of Algorithm 1 is explicit (C acts on the predicted
        velocity), so dt is also held to 1 / max_j (C_jj / M_jj)."""
        cfl = self.w.cfl if cfl is None else cfl
        cmax = max(m.c for m in self.meshes)
        hmin = min(min(m.h) / 2.0 * float(np.min(np.diff(m.xi))) for m in self.meshes)
        dt = cfl * hmin / cmax
        damp = self.C * self.Minv
        if self.pml is not None:
            damp = damp + self.pml["alpha"]
        sigma = float(np.max(damp))
        if sigma > 0.0:
            dt = min(dt, 1.0 / sigma)
        return dt

    def all_coordinates(self):
        xs, ys, zs = [], [], []
        for m in self.meshes:
            x, y, z = m.all_coordinates()
            xs.append(x); ys.append(y); zs.append(z)
        return np.concatenate(xs), np.concatenate(ys), np.concatenate(zs)

    def run(self, nsteps=None, dt=None, drive=None, receivers=None, p0=None, v0=None,
            energy=False, batch=None, callback=None):
        """Algorithm 1 (Newmark gamma=1/2, beta=0) with three vectors per field.

        drive [B, K, S] volts at t^n; returns traces [B, R, S] with sample n =
        p^{n+1} at the receivers (and per-step energies if asked).
        """
        S = self.w.nsteps if nsteps is None else nsteps
        dt = self.stable_dt() if dt is None else dt
        B = self.w.batch if batch is None else batch
        rec = self.w.receivers if receivers is None else receivers
        Rm = self.receiver_matrix(rec)
        pm = self.w.pmuts
        if pm is not None:
            K, Mm = pm.n_pmut, pm.n_modes
            omega2 = ((2 * math.pi * pm.freq_hz) ** 2).reshape(-1)
            twozw = (2 * pm.damping * 2 * math.pi * pm.freq_hz).reshape(-1)
            mu = pm.modal_mass.reshape(-1)
            eta = pm.eta.reshape(-1)
            if drive is None:
                drive = self.w.drive(dt, S, B)
            drive = np.asarray(drive, dtype=np.float64)
            q = np.zeros((K * Mm, B)); qd = np.zeros_like(q); qdd = np.zeros_like(q)
            rx_on = self.w.rx_switch is not None
            if rx_on:
                cap = np.broadcast_to(np.asarray(self.w.rx_capacitance, dtype=np.float64), (K,))
            volts = np.zeros((B, K, S))
        p = np.zeros((self.nh, B)); pd = np.zeros_like(p); pdd = np.zeros_like(p)
        if p0 is not None:
            p = np.array(p0, dtype=np.float64).reshape(self.nh, -1) * np.ones((1, B))
            if v0 is not None:
                pd = np.array(v0, dtype=np.float64).reshape(self.nh, -1) * np.ones((1, B))
            pdd = self.Minv[:, None] * (-(self.K @ p) - self.C[:, None] * pd)
            if self.pml is not None:
                pdd = pdd - self.pml["beta"][:, None] * p - self.pml["alpha"][:, None] * pd
        if self.pml is not None:
            psi_half = np.zeros((self.nh, B))
            Phi = [np.zeros((3, len(e[0]), B)) for e in self.pml["elems"]]
        traces = np.zeros((B, len(rec), S))
        energies = [] if energy else None
        Minv = self.Minv[:, None]
        for n in range(S):
            if pm is not None:
                # PMUT predictor
                q_new = q + dt * qd + 0.5 * dt * dt * qdd
                qd_new = qd + 0.5 * dt * qdd
                # PMUT solve: q'' = -W q - 2 zeta w q'_pred + g(p^n, phi^n) / mu
                if rx_on and n >= self.w.rx_switch:
                    # open circuit: phi_k = s / C_k sum_m eta_km q_km^n
                    vk = (eta[:, None] * q).reshape(K, Mm, B).sum(axis=1)   # [K, B]
                    vk = (self.w.rx_sign / cap)[:, None] * vk
                else:
                    vk = drive[:, :, n].T                                   # [K, B]
                volts[:, :, n] = vk.T
                phi = np.repeat(vk, Mm, axis=0)                           # [(k,m), B]
                g = (self.B.T @ p) + eta[:, None] * phi
                qdd_new = -omega2[:, None] * q_new - twozw[:, None] * qd_new + g / mu[:, None]
                # PMUT corrector
                qd_new = qd_new + 0.5 * dt * qdd_new
            # acoustic predictor
            p_new = p + dt * pd + 0.5 * dt * dt * pdd
            pd_new = pd + 0.5 * dt * pdd
            # acoustic solve: p'' = M^-1 (f(q'') - K p - C p'_pred)
            rhs = -(self.K @ p_new) - self.C[:, None] * pd_new
            if pm is not None:
                rhs = rhs - self.kappa * (self.B @ qdd_new)
            if self.pml is not None:
                Phi, psi_int, r = self._pml_step(Phi, psi_half, p_new, dt)
                rhs = rhs - self.M[:, None] * (self.pml["beta"][:, None] * p_new + self.pml["alpha"][:, None] * pd_new
                                               + self.pml["gamma"][:, None] * psi_int) - r
                psi_half = psi_half + dt * p_new
            pdd_new = Minv * rhs
            # acoustic corrector
            pd_new = pd_new + 0.5 * dt * pdd_new
            if pm is not None:
                q, qd, qdd = q_new, qd_new, qdd_new
            p, pd, pdd = p_new, pd_new, pdd_new
            traces[:, :, n] = (Rm @ p).T
            if callback is not None:
                callback(n, p=p, pd=pd, pdd=pdd, q=q if pm is not None else None,
                         qd=qd if pm is not None else None, qdd=qdd if pm is not None else None)
            if energy:
                energies.append(self.energy(p, pd, pdd, dt,
                                            q if pm is not None else None,
                                            qd if pm is not None else None,
                                            qdd if pm is not None else None))
        self.final_state = dict(p=p, pd=pd, pdd=pdd)
        if pm is not None:
            self.final_state.update(q=q, qd=qd, qdd=qdd)
            self.voltages = volts
        if energy:
            return traces, np.array(energies)
        return traces

    def energy(self, p, pd, pdd, dt, q=None, qd=None, qdd=None):
        """Two energies after a step that produced (p, p', p'') = (p^{n+1}, ...).

        [0] leapfrog invariant of the acoustic part: with v = p' + dt/2 p''
            (the half-step velocity) and p_next = p + dt v,
            E = 1/2 v.M v + 1/2 p.K p_next, exactly conserved by Algorithm 1
            for symmetric K and no forcing;
        [1] semi-discrete coupled energy 1/2 p'.M p' + 1/2 p.K p
            + kappa/2 (q''.mu q'' + q'.mu W q'), conserved by eqs.
            (semi_SEM)-(semi_PMUT) without damping once phi is constant
            (Algorithm 1 conserves it up to O(dt^2)).
        """
        v = pd + 0.5 * dt * pdd
        p_next = p + dt * v
        e_lf = 0.5 * np.sum(v * (self.M[:, None] * v), axis=0) + 0.5 * np.sum(p * (self.K @ p_next), axis=0)
        e = 0.5 * np.sum(pd * (self.M[:, None] * pd), axis=0) + 0.5 * np.sum(p * (self.K @ p), axis=0)
        if q is not None and self.w.pmuts is not None:
            pm = self.w.pmuts
            mu = pm.modal_mass.reshape(-1)[:, None]
            om2 = ((2 * math.pi * pm.freq_hz) ** 2).reshape(-1)[:, None]
            e = e + 0.5 * self.kappa * np.sum(mu * qdd * qdd + mu * om2 * qd * qd, axis=0)
        return np.stack([e_lf, e])
