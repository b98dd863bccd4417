"""The pins catch plausible mistakes: each test plants one mistake in the
oracle (on the CPU, through monkeypatch, nothing persists) and runs the pin
that is meant to catch it, which must then fail.  A pin that still passed
with the mistake in place would not be pinning that part of the oracle."""
import numpy as np
import pytest

import test_hex_oracle_pins as hex_pins
import test_oracle_pins as box_pins
from oracle import dgsem_oracle as O
from oracle import hex_oracle as HO
from workloads import hex as H


def _two_dom():
    w = H.distorted_two_domain(nx_p=4, nz_p=2, nx_s=2, nz_s=2, n_pmut_side=2, nsteps=40)
    return w, HO.HexOracleProblem(w)


# ---------------------------------------------------------------- box oracle
def test_gll_weight_without_the_square_fails_exactness(monkeypatch):
    """w_i = 2 / (N (N+1) P_N(x_i)) instead of ... P_N(x_i)^2: the quadrature
    stops being exact to degree 2N-1."""
    orig = O.gll_nodes_weights

    def mutant(N):
        x, w = orig(N)
        P = np.polynomial.legendre.legval(x, [0] * N + [1])
        return x, 2.0 / (N * (N + 1) * np.abs(P))
    monkeypatch.setattr(O, "gll_nodes_weights", mutant)
    with pytest.raises(AssertionError):
        box_pins.test_gll_exactness(4)


def test_transposed_derivative_matrix_fails_the_lagrange_identities(monkeypatch):
    orig = O.lagrange_derivatives

    def mutant(nodes, x):
        D = orig(nodes, nodes)
        return O.lagrange_values(nodes, x) @ D.T        # l_a'(x) built from D^T
    monkeypatch.setattr(O, "lagrange_derivatives", mutant)
    with pytest.raises(AssertionError):
        box_pins.test_lagrange_identities(4)


def test_inverted_element_scaling_fails_the_anisotropic_pin(monkeypatch):
    """h_d / 2 in place of 2 / h_d in the affine gradient."""
    def mutant(mesh):
        N, xi, w = mesh.N, mesh.xi, mesh.w
        P, Q, R = np.meshgrid(xi, xi, xi, indexing="ij")
        pts = np.stack([P.transpose(2, 1, 0).ravel(), Q.transpose(2, 1, 0).ravel(),
                        R.transpose(2, 1, 0).ravel()], axis=1)
        WP, WQ, WR = np.meshgrid(w, w, w, indexing="ij")
        wq = (WP * WQ * WR).transpose(2, 1, 0).ravel()
        _, grad_ref = O.reference_basis(N, xi, pts)
        Jinv = np.array([mesh.h[d] / 2.0 for d in range(3)])
        detJ = mesh.h[0] * mesh.h[1] * mesh.h[2] / 8.0
        grad = grad_ref * Jinv[None, None, :]
        return mesh.c ** 2 * detJ * np.einsum("q,qid,qjd->ij", wq, grad, grad, optimize=True)
    monkeypatch.setattr(O, "element_stiffness", mutant)
    with pytest.raises(AssertionError):
        box_pins.test_element_stiffness_scaling_anisotropic()


class _SplitSignB:
    """B in the forcing f = -kappa B q'', -B^T in the projection g = B^T p."""

    def __init__(self, B):
        self.B = B

    @property
    def T(self):
        return -self.B.T

    def __matmul__(self, x):
        return self.B @ x


def test_sign_error_between_forcing_and_projection_fails_the_coupled_energy_pin(monkeypatch):
    """The membrane integral enters g with the opposite sign to the one it
    has in f: the coupling then feeds energy in instead of exchanging it.
    (Flipping kappa or B as a whole keeps the two consistent, conserves the
    correspondingly signed energy, and is a sign convention, not a mistake.)"""
    orig = O.OracleProblem._pmut_matrix

    def mutant(self):
        orig(self)
        if self.B is not None:
            self.B = _SplitSignB(self.B)
    monkeypatch.setattr(O.OracleProblem, "_pmut_matrix", mutant)
    with pytest.raises(AssertionError):
        box_pins.test_coupled_energy_first_order_drift()


@pytest.mark.parametrize("mistake", ["kappa_rho", "kappa_sign", "b_sign", "weights_doubled"])
def test_forcing_scale_and_sign_mistakes_fail_the_rayleigh_pin(monkeypatch, mistake):
    """kappa = rho instead of rho c^2, kappa or B with the wrong sign as a
    whole (consistent between f and g, so the energy pin cannot see it), or
    face weights doubled: the radiated pressure of a prescribed membrane
    motion is then wrong in scale or sign."""
    orig = O.OracleProblem._pmut_matrix

    def mutant(self):
        orig(self)
        if self.B is None:
            return
        if mistake == "kappa_rho":
            self.kappa = self.meshes[0].rho
        elif mistake == "kappa_sign":
            self.kappa = -self.kappa
        elif mistake == "b_sign":
            self.B = -self.B
        else:
            self.B = 2.0 * self.B
    monkeypatch.setattr(O.OracleProblem, "_pmut_matrix", mutant)
    with pytest.raises(AssertionError):
        box_pins.test_rayleigh_integral_of_a_baffled_membrane()


# ---------------------------------------------------------------- hex oracle
def test_gradient_with_j_inverse_untransposed_fails_the_linear_patch(monkeypatch):
    """grad psi = J^-1 grad^ psi instead of J^-T grad^ psi in the element
    stiffness: wrong on every distorted element."""
    def mutant(m, e, grad_ref):
        Jinv = np.linalg.inv(m.J[e])
        grad = np.einsum("qxd,qjd->qjx", Jinv, grad_ref)
        return m.c ** 2 * np.einsum("q,qix,qjx->ij", m.wq * m.detJ[e], grad, grad, optimize=True)
    monkeypatch.setattr(HO, "hex_element_stiffness", mutant)
    with pytest.raises(AssertionError):
        hex_pins.test_linear_patch_across_bent_interface(_two_dom())


def test_surface_jacobian_without_nanson_factor_fails_patch_and_face_weights(monkeypatch):
    """|J| in place of |J| |J^-T e_axis| as the surface Jacobian."""
    orig = HO.face_normal_and_jac

    def mutant(J, f):
        n, _ = orig(J, f)
        return n, np.linalg.det(J)
    monkeypatch.setattr(HO, "face_normal_and_jac", mutant)
    dom = _two_dom()
    with pytest.raises(AssertionError):
        hex_pins.test_linear_patch_across_bent_interface(dom)
    with pytest.raises(AssertionError):
        hex_pins.test_pmut_face_weights_sum_to_plane_area(dom)


def test_inward_interface_normal_fails_the_linear_patch(monkeypatch):
    """The consistency terms taken with n pointing into K+ on the interface
    (the normal of the volume terms' boundary stays outward)."""
    orig = HO.face_normal_and_jac
    calls = {"iface": False}

    def mutant(J, f):
        n, dS = orig(J, f)
        return (-n if calls["iface"] else n), dS
    orig_matrix = HO.hex_interface_matrix

    def matrix(*a, **k):
        calls["iface"] = True
        try:
            return orig_matrix(*a, **k)
        finally:
            calls["iface"] = False
    monkeypatch.setattr(HO, "face_normal_and_jac", mutant)
    monkeypatch.setattr(HO, "hex_interface_matrix", matrix)
    with pytest.raises(AssertionError):
        hex_pins.test_linear_patch_across_bent_interface(_two_dom())


@pytest.mark.parametrize("iters", [1, 3])
def test_truncated_newton_iteration_is_caught_by_the_containment_test(monkeypatch, iters):
    """Algorithm 3 with the Newton iteration for the coarse reference position
    stopped early: on trilinear (non-affine) elements the position is off by
    more than the containment slack (1e-10), so interface nodes near element
    edges find no coarse neighbour and building the operator fails.  (From
    four steps on the iteration has converged to rounding on these meshes.)"""
    orig = HO.newton_reference
    steps = iters
    monkeypatch.setattr(HO, "newton_reference", lambda verts, x, iters=50: orig(verts, x, iters=steps))
    with pytest.raises(ValueError, match="without a coarse neighbour"):
        hex_pins.test_linear_patch_across_bent_interface(_two_dom())


def test_penalty_length_from_the_wrong_ratio_fails_the_affine_pin(monkeypatch):
    """gamma_F with h = |F| / |K| in place of |K| / |F|: the affine case no
    longer reproduces the box oracle, whose penalty value is pinned."""
    orig_init = HO._HexFace.__init__

    def mutant(self, mesh, elem, f):
        orig_init(self, mesh, elem, f)
        self.h = self.area / mesh.volume(self.elem)
    monkeypatch.setattr(HO._HexFace, "__init__", mutant)
    with pytest.raises(AssertionError):
        hex_pins.test_affine_case_is_the_box_oracle()


def test_mass_with_the_mean_jacobian_fails_the_volume_pin(monkeypatch):
    """M_ii with the element's mean Jacobian determinant in place of its
    value at each GLL node of the trilinear map."""
    orig = HO.HexOracleProblem._assemble_volume

    def mutant(self):
        orig(self)
        self.M = np.zeros_like(self.M)
        for m in self.meshes:
            for e in range(m.ne):
                np.add.at(self.M, m.conn[e], m.wq * np.mean(m.detJ[e]))
    monkeypatch.setattr(HO.HexOracleProblem, "_assemble_volume", mutant)
    with pytest.raises(AssertionError):
        hex_pins.test_mass_sums_to_box_volume(4)
