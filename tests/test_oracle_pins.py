"""Pins of the CPU oracle against closed forms, invariants and brute force.

Each test fixes one part of the oracle with something other than the oracle
itself (a closed form, an exact identity of the discretisation, a limit),
chosen so that a plausible mistake in that part fails it.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import dgsem_oracle as O


# ----------------------------------------------------------------- 1D tables
def test_gll_n4_closed_form():
    """GLL N=4: {0, +-sqrt(3/7), +-1}, weights {32/45, 49/90, 1/10}."""
    x, w = O.gll_nodes_weights(4)
    np.testing.assert_allclose(x, [-1, -math.sqrt(3 / 7), 0, math.sqrt(3 / 7), 1], atol=1e-15)
    np.testing.assert_allclose(w, [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10], atol=1e-15)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7, 8])
def test_gll_exactness(N):
    """sum w x^k is exact for k <= 2N-1 and wrong at k = 2N."""
    x, w = O.gll_nodes_weights(N)
    for k in range(2 * N):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 1e-13
    assert abs(np.sum(w * x ** (2 * N)) - 2.0 / (2 * N + 1)) > 1e-6


def test_gll_n2_closed_form():
    x, w = O.gll_nodes_weights(2)
    np.testing.assert_allclose(x, [-1, 0, 1], atol=1e-15)
    np.testing.assert_allclose(w, [1 / 3, 4 / 3, 1 / 3], atol=1e-15)


@pytest.mark.parametrize("N", [2, 4, 6])
def test_lagrange_identities(N):
    """l_a(x_b) = delta_ab, sum_a l_a = 1, sum_a l_a' = 0, sum_a x_a l_a' = 1
    and sum_a x_a^N l_a'(x) = N x^(N-1) (derivatives exact on degree <= N)."""
    x, _ = O.gll_nodes_weights(N)
    np.testing.assert_allclose(O.lagrange_values(x, x), np.eye(N + 1), atol=1e-14)
    t = np.linspace(-1, 1, 17)
    L = O.lagrange_values(x, t)
    D = O.lagrange_derivatives(x, t)
    np.testing.assert_allclose(L.sum(axis=1), 1.0, atol=1e-13)
    np.testing.assert_allclose(D.sum(axis=1), 0.0, atol=1e-12)
    np.testing.assert_allclose(D @ x, 1.0, atol=1e-12)
    np.testing.assert_allclose(D @ x ** N, N * t ** (N - 1), atol=1e-11)


def test_gauss_legendre_matches_closed_form():
    g, w = O.gauss_legendre(3)
    np.testing.assert_allclose(g, [-math.sqrt(3 / 5), 0, math.sqrt(3 / 5)], atol=1e-15)
    np.testing.assert_allclose(w, [5 / 9, 8 / 9, 5 / 9], atol=1e-15)


# ------------------------------------------------------------ element level
def _kron3(A, Wm):
    """sum over directions of the Kronecker product with a fastest (basis index
    (c*(n)+b)*n+a): A acting on a, b or c."""
    return np.kron(np.kron(Wm, Wm), A) + np.kron(np.kron(Wm, A), Wm) + np.kron(np.kron(A, Wm), Wm)


def test_element_stiffness_n1_closed_form():
    """N=1 on the reference cube (h=2, c=1): A = 1/2 [[1,-1],[-1,1]], W = I."""
    dom = W.Domain((0, 0, 0), (2.0, 2.0, 2.0), (1, 1, 1), 1, c=1.0)
    Ke = O.element_stiffness(O.BoxMesh(dom, 0))
    A = 0.5 * np.array([[1.0, -1.0], [-1.0, 1.0]])
    np.testing.assert_allclose(Ke, _kron3(A, np.eye(2)), atol=1e-14)


def test_element_stiffness_n2_closed_form():
    """N=2 on the reference cube: hand-integrated 1D stiffness of the quadratic
    Lagrange basis on {-1,0,1} and GLL weights {1/3,4/3,1/3}."""
    dom = W.Domain((0, 0, 0), (2.0, 2.0, 2.0), (1, 1, 1), 2, c=1.0)
    Ke = O.element_stiffness(O.BoxMesh(dom, 0))
    A = np.array([[7 / 6, -4 / 3, 1 / 6], [-4 / 3, 8 / 3, -4 / 3], [1 / 6, -4 / 3, 7 / 6]])
    np.testing.assert_allclose(Ke, _kron3(A, np.diag([1 / 3, 4 / 3, 1 / 3])), atol=1e-13)


def test_element_stiffness_scaling_anisotropic():
    """Affine element with sizes (hx, hy, hz) and speed c: the x-part scales
    with c^2 hy hz / hx (checked on a linear field u = x: K u = c^2 * face flux)."""
    hx, hy, hz, c = 3.0, 0.5, 2.0, 1.7
    dom = W.Domain((0, 0, 0), (hx, hy, hz), (1, 1, 1), 3, c=c)
    m = O.BoxMesh(dom, 0)
    Ke = O.element_stiffness(m)
    x, y, z = m.all_coordinates()
    Ku = Ke @ x
    # K u = int c^2 grad x . grad psi = c^2 int d psi/dx = c^2 (face integrals of psi at x=hx minus x=0)
    _, w = O.gll_nodes_weights(3)
    expect = np.zeros_like(x)
    face_w = np.einsum("c,b->cb", w, w).ravel() * hy * hz / 4.0
    ids = np.arange(x.size).reshape(4, 4, 4)
    expect[ids[:, :, 3].ravel()] += c * c * face_w
    expect[ids[:, :, 0].ravel()] -= c * c * face_w
    np.testing.assert_allclose(Ku, expect, atol=1e-12 * np.abs(expect).max())


@pytest.mark.parametrize("N", [2, 4, 6])
def test_element_stiffness_kernel_and_symmetry(N):
    dom = W.Domain((0, 0, 0), (1e-4, 2e-4, 5e-5), (1, 1, 1), N)
    Ke = O.element_stiffness(O.BoxMesh(dom, 0))
    assert np.abs(Ke - Ke.T).max() <= 1e-12 * np.abs(Ke).max()
    assert np.abs(Ke.sum(axis=1)).max() <= 1e-11 * np.abs(Ke).max()


def test_lumped_mass_total_volume():
    dom = W.Domain((0, 0, 0), (3e-4, 2e-4, 1e-4), (3, 2, 2), 4)
    P = O.OracleProblem(W.Workload("m", [dom], 1, np.zeros((1, 3))))
    assert abs(P.M.sum() - 3e-4 * 2e-4 * 1e-4) < 1e-12 * 6e-12


# -------------------------------------------------------------- assembled K
def _interior_mask(P, x, y, z):
    lo = np.array([min(m.origin[d] for m in P.meshes) for d in range(3)])
    hi = np.array([max(m.origin[d] + m.ne[d] * m.h[d] for m in P.meshes) for d in range(3)])
    t = 1e-12
    return ((x > lo[0] + t) & (x < hi[0] - t) & (y > lo[1] + t) & (y < hi[1] - t)
            & (z > lo[2] + t) & (z < hi[2] - t))


@pytest.fixture(scope="module")
def two_domain():
    w = W.small_two_domain(nx_p=4, nz_p=2, nx_s=2, nz_s=2, n_pmut_side=2)
    return w, O.OracleProblem(w)


def test_patch_quadratic_across_nonconforming_interface(two_domain):
    """u = x^2, y^2, z^2: (M^-1 K u)_i = -2 c^2 at every node off the outer
    boundary, including nodes on both sides of the 2:1 interface (the SIPG
    terms vanish for a smooth u and the GL rule integrates them exactly)."""
    _, P = two_domain
    x, y, z = P.all_coordinates()
    inner = _interior_mask(P, x, y, z)
    c2 = P.meshes[0].c ** 2
    for u in (x * x, y * y, z * z):
        r = P.Minv * (P.K @ u) / c2
        np.testing.assert_allclose(r[inner], -2.0, atol=1e-9)


def test_patch_linear_and_constants(two_domain):
    _, P = two_domain
    x, y, z = P.all_coordinates()
    inner = _interior_mask(P, x, y, z)
    scale = np.abs(P.K).max()
    assert np.abs((P.K @ (x - 2 * y + 3 * z))[inner]).max() <= 1e-13 * scale
    assert np.abs(P.K @ np.ones(P.nh)).max() <= 1e-12 * scale


def test_stiffness_symmetric_psd(two_domain):
    """K symmetric (both SIPG consistency terms on the same quadrature) and
    positive semi-definite with the constants as its only kernel (alpha = 0.5)."""
    _, P = two_domain
    Kd = P.K.toarray()
    assert np.abs(Kd - Kd.T).max() <= 1e-13 * np.abs(Kd).max()
    ev = np.linalg.eigvalsh(Kd)
    assert ev[0] >= -1e-12 * ev[-1]
    assert ev[1] >= 1e-5 * ev[-1]


def test_penalty_value(two_domain):
    """gamma_F = alpha c-bar^2 max(N)^2 / min(h): 0.5 * 1500^2 * 36 / 25 um."""
    _, P = two_domain
    assert abs(P.gamma - 0.5 * 1500.0 ** 2 * 36 / 25e-6) <= 1e-6 * P.gamma


def test_default_dt_is_stable(two_domain):
    """dt * sqrt(lambda_max(M^-1 K)) < 2 for the default CFL 0.3 and alpha 0.5
    at the config-2 element sizes (primary 25 um N=4, secondary 50 um N=6)."""
    _, P = two_domain
    D = np.diag(1 / np.sqrt(P.M))
    lmax = np.linalg.eigvalsh(D @ P.K.toarray() @ D)[-1]
    dt = P.stable_dt()
    assert abs(dt - 8.4888e-10) < 1e-13
    assert dt * math.sqrt(lmax) < 1.6


def test_dt_config1():
    P = O.OracleProblem(W.config1_single_pmut(nsteps=1))
    assert abs(P.stable_dt() - 2.5901e-9) < 1e-13


# ------------------------------------------------------------- time stepping
def test_leapfrog_invariant_with_interface(two_domain):
    """Acoustic only: E = 1/2 v.M v + 1/2 p^n.K p^{n+1} is constant to rounding
    under Algorithm 1 (needs symmetric K incl. the interface)."""
    w, P = two_domain
    w2 = W.small_two_domain(nx_p=4, nz_p=2, nx_s=2, nz_s=2, n_pmut_side=2, nsteps=150)
    w2.pmuts = None
    P2 = O.OracleProblem(w2)
    x, y, z = P2.all_coordinates()
    p0 = W.seeded_field(3, x, y, z)
    _, E = P2.run(p0=p0, energy=True, receivers=np.array([[1e-5, 1e-5, 1e-5]]))
    e = E[:, 0, 0]
    assert (e.max() - e.min()) <= 1e-12 * e.mean()


def test_standing_wave_rigid_box():
    """p = cos(pi x/L) cos(pi y/L) cos(w t) in a rigid box: traces follow the
    closed form; the error drops by > 20x from N=4 to N=6 (spectral)."""
    errs = []
    for N in (4, 6):
        dom = W.Domain((0, 0, 0), (1e-4, 1e-4, 1e-4), (2, 2, 2), N)
        rec = np.array([[0.013e-3, 0.021e-3, 0.05e-3], [0.07e-3, 0.033e-3, 0.081e-3]])
        w = W.Workload("sw", [dom], 400, rec, cfl=0.05)
        P = O.OracleProblem(w)
        x, y, z = P.all_coordinates()
        p0, om = W.standing_wave_mode(dom, (1, 1, 0), x, y, z)
        dt = P.stable_dt()
        tr = P.run(p0=p0)
        mode_r, _ = W.standing_wave_mode(dom, (1, 1, 0), rec[:, 0], rec[:, 1], rec[:, 2])
        t = (np.arange(400) + 1) * dt
        exact = mode_r[:, None] * np.cos(om * t)[None, :]
        errs.append(np.abs(tr[0] - exact).max())
    assert errs[0] < 2e-3
    assert errs[1] < errs[0] / 20


def _isolated_pmut_workload(nsteps, zeta=0.0, freq=2.0e6):
    """A PMUT whose footprint holds no face node (side smaller than the node
    spacing away from nodes): g = eta phi / mu only, f = 0."""
    dom = W.Domain((0, 0, 0), (1e-4, 1e-4, 1e-4), (1, 1, 1), 2)
    pm = W.make_pmut_array([[0.27e-4, 0.27e-4]], 1e-6, [freq], zeta)
    return W.Workload("osc", [dom], nsteps, np.array([[5e-5, 5e-5, 5e-5]]), pm,
                      drive_delay=np.zeros((1, 1)), drive_amp=np.ones((1, 1)))


def test_modal_oscillator_exact_discrete_solution():
    """Undamped mode under a constant drive: Algorithm 1 from rest gives
    q_n = F/w^2 (1 - cos((n - 1/2) theta) / cos(theta / 2)),
    cos theta = 1 - (w dt)^2 / 2, F = eta phi / mu (exact to rounding)."""
    S = 300
    w = _isolated_pmut_workload(S)
    P = O.OracleProblem(w)
    assert P.B.nnz == 0
    dt = 2e-9
    drive = np.full((1, 1, S), 3.0)
    qs = []
    P.run(dt=dt, drive=drive, callback=lambda n, **st: qs.append(st["q"][0, 0]))
    pm = w.pmuts
    om = 2 * math.pi * pm.freq_hz[0, 0]
    F = pm.eta[0, 0] * 3.0 / pm.modal_mass[0, 0]
    th = math.acos(1 - (om * dt) ** 2 / 2)
    n = np.arange(1, S + 1)
    exact = F / om ** 2 * (1 - np.cos((n - 0.5) * th) / math.cos(th / 2))
    np.testing.assert_allclose(qs, exact, atol=1e-12 * np.abs(exact).max())


def test_modal_oscillator_damped_driven_converges():
    """Damped mode driven by phi = sin(w_d t): q converges to the analytic
    solution (Duhamel integral, closed form) as dt -> 0, at least first order."""
    zeta, f = 0.05, 2.0e6
    T = 2.0e-6
    wd = 2 * math.pi * 1.3e6
    errs = []
    for S in (400, 800, 1600):
        w = _isolated_pmut_workload(S, zeta=zeta, freq=f)
        P = O.OracleProblem(w)
        dt = T / S
        t = np.arange(S) * dt
        drive = np.sin(wd * t)[None, None, :]
        qs = []
        P.run(dt=dt, drive=drive, callback=lambda n, **st: qs.append(st["q"][0, 0]))
        pm = w.pmuts
        w0 = 2 * math.pi * f
        F = pm.eta[0, 0] / pm.modal_mass[0, 0]
        # steady state + transient of q'' + 2 z w0 q' + w0^2 q = F sin(wd t), q(0)=q'(0)=0
        H = F / complex(w0 ** 2 - wd ** 2, 2 * zeta * w0 * wd)
        A, ph = abs(H), np.angle(H)
        tt = (np.arange(S) + 1) * dt
        wdamp = w0 * math.sqrt(1 - zeta ** 2)
        # transient coefficients from q(0) = q'(0) = 0
        c1 = -A * math.sin(ph)
        c2 = (-A * wd * math.cos(ph) + zeta * w0 * c1) / wdamp
        qex = A * np.sin(wd * tt + ph) + np.exp(-zeta * w0 * tt) * (c1 * np.cos(wdamp * tt) + c2 * np.sin(wdamp * tt))
        errs.append(np.abs(np.array(qs) - qex).max() / np.abs(qex).max())
    assert errs[2] < 0.02
    assert errs[0] / errs[1] > 1.8 and errs[1] / errs[2] > 1.8


def test_coupled_energy_first_order_drift():
    """Coupled, zeta = 0, after the burst: the semi-discrete energy of
    eqs. (semi_SEM)-(semi_PMUT) is conserved up to the one-step lag of
    g(p^n) in Algorithm 1, so its drift halves when dt halves.  A sign error
    between f and g breaks this (kappa's value and the overall sign of the
    coupling are pinned by the Rayleigh-integral test)."""
    drifts = []
    for scale in (1.0, 0.5):
        w = W.config1_single_pmut(nsteps=int(700 / scale))
        w.domains[0] = W.Domain((0, 0, 0), (0.3e-3,) * 3, (4, 4, 4), 4)
        w.pmuts = W.make_pmut_array([[0.15e-3, 0.15e-3]], 60e-6, W.MODE_FREQS_5[:3], 0.0)
        w.receivers = np.array([[0.15e-3, 0.15e-3, 0.1e-3]])
        w.cfl = 0.3 * scale
        P = O.OracleProblem(w)
        dt = P.stable_dt()
        _, E = P.run(energy=True)
        e = E[int(1.5e-6 / dt) + 3:, 1, 0]
        drifts.append((e.max() - e.min()) / e.mean())
    assert drifts[0] < 0.2
    assert 1.7 < drifts[0] / drifts[1] < 2.3


def _rayleigh_case(N):
    """A 0.3 mm membrane (mode (1,1), unit peak) in the rigid z = 0 face of a
    0.6 mm water cube, moved with a prescribed acceleration: a huge modal mass
    makes the fluid's reaction negligible and no stiffness, so Algorithm 1
    gives q''^{n+1} = (eta / mu) phi^n exactly.  Returns the oracle's on-axis
    trace at z0 = 0.15 mm and the Rayleigh integral of the same motion."""
    L, a, z0, f = 0.6e-3, 0.3e-3, 0.15e-3, 8.0e6
    dom = W.Domain((0, 0, 0), (L, L, L), (8, 8, 8), N)
    pm = W.PmutArray(centers=np.array([[0.3e-3, 0.3e-3]]), side=a, freq_hz=np.array([[1.0]]),
                     damping=np.array([[0.0]]), eta=np.array([[1.0e6]]), modal_mass=np.array([[1.0e6]]))
    rec = np.array([[0.3e-3, 0.3e-3, z0]])
    w = W.Workload("rayleigh", [dom], 10, rec, pm, drive_delay=np.zeros((1, 1)), drive_amp=np.ones((1, 1)),
                   burst_freq=f, burst_cycles=1.0)
    P = O.OracleProblem(w)
    dt = P.stable_dt()
    # before the first echo: the membrane edge's image in the x = 0 wall is
    # 0.474 mm from the receiver (0.316 us)
    S = int(0.31e-6 / dt)
    tr = P.run(nsteps=S, dt=dt)[0, 0]                      # sample n = p^{n+1}
    Tb = 1.0 / f

    def qdd(s):                                             # eta / mu = 1 m/s^2 per volt
        on = (s >= 0) & (s <= Tb)
        return np.where(on, np.sin(2 * math.pi * f * s) * 0.5 * (1 - np.cos(2 * math.pi * s / Tb)), 0.0)
    g, gw = np.polynomial.legendre.leggauss(80)
    X, Y = np.meshgrid(g, g, indexing="ij")
    wts = np.outer(gw, gw) * (a / 2) ** 2
    phi = (1 - X ** 2) ** 2 * (1 - Y ** 2) ** 2
    R = np.sqrt((X * a / 2) ** 2 + (Y * a / 2) ** 2 + z0 ** 2)
    t = (np.arange(S) + 1) * dt
    # p(x, t) = rho / (2 pi) int a_n(y, t - R / c) / R dA for a baffled surface
    ref = np.array([dom.rho / (2 * math.pi) * np.sum(wts * qdd(tt - dt - R / dom.c) * phi / R) for tt in t])
    return tr, ref


def test_rayleigh_integral_of_a_baffled_membrane():
    """Prescribed membrane motion radiating into the half space before any
    wall echo: the pressure is the Rayleigh integral (rigid baffle), which
    fixes kappa = rho c^2, the sign and face weights of B and the forcing, and
    the wave speed; the error falls spectrally from N = 4 to N = 6."""
    errs = []
    for N in (4, 6):
        tr, ref = _rayleigh_case(N)
        assert np.abs(ref).max() > 0
        errs.append(np.linalg.norm(tr - ref) / np.linalg.norm(ref))
    assert errs[0] < 0.05 and errs[1] < 0.006, errs
    assert errs[0] / errs[1] > 5, errs


def test_symmetry_centred_pmut():
    """Centred PMUT on a symmetric mesh: the antisymmetric modes (eta = 0)
    stay at rounding level and mirror receivers record equal traces."""
    w = W.config1_single_pmut(nsteps=300)
    w.domains[0] = W.Domain((0, 0, 0), (0.3e-3,) * 3, (4, 4, 4), 4)
    w.pmuts = W.make_pmut_array([[0.15e-3, 0.15e-3]], 60e-6, W.MODE_FREQS_5[:3], 0.01)
    w.receivers = np.array([[0.05e-3, 0.11e-3, 0.1e-3], [0.25e-3, 0.11e-3, 0.1e-3],
                            [0.11e-3, 0.05e-3, 0.1e-3]])
    P = O.OracleProblem(w)
    tr = P.run()
    q = P.final_state["q"][:, 0]
    assert abs(q[1]) < 1e-12 * abs(q[0]) and abs(q[2]) < 1e-12 * abs(q[0])
    scale = np.abs(tr).max()
    assert np.abs(tr[0, 0] - tr[0, 1]).max() < 1e-11 * scale
    assert np.abs(tr[0, 0] - tr[0, 2]).max() < 1e-11 * scale


def test_linearity_and_time_shift():
    w = W.small_one_domain(nel=(3, 2, 2), nsteps=120, n_pmut_side=2)
    P = O.OracleProblem(w)
    dt = P.stable_dt()
    rng = np.random.default_rng(0)
    d1 = rng.normal(size=(1, 4, 120))
    d2 = rng.normal(size=(1, 4, 120))
    t1 = P.run(drive=d1)
    t2 = P.run(drive=d2)
    t12 = P.run(drive=d1 + d2)
    scale = np.abs(t12).max()
    assert np.abs(t12 - t1 - t2).max() < 1e-12 * scale
    k = 17
    ds = np.zeros_like(d1)
    ds[:, :, k:] = d1[:, :, :-k]
    ts = P.run(drive=ds)
    assert np.array_equal(ts[:, :, k:], t1[:, :, :-k])
    assert np.all(ts[:, :, :k] == 0.0)


def test_conforming_split_approaches_single_box():
    """Split a box into two stacked boxes with matching elements and order:
    the SIPG solution approaches the C0 single-box solution as alpha grows."""
    L, h = 1e-4, 2.5e-5
    rec = np.array([[0.031e-3, 0.047e-3, 0.022e-3], [0.061e-3, 0.012e-3, 0.081e-3]])
    one = W.Domain((0, 0, 0), (L, L, 2 * L), (2, 2, 4), 3)
    lo = W.Domain((0, 0, 0), (L, L, L), (2, 2, 2), 3)
    hi = W.Domain((0, 0, L), (L, L, L), (2, 2, 2), 3)
    ref = O.OracleProblem(W.Workload("cg", [one], 300, rec, cfl=0.02))
    dt = ref.stable_dt()
    x, y, z = ref.all_coordinates()
    p0, _ = W.standing_wave_mode(one, (1, 0, 1), x, y, z)
    t_ref = ref.run(p0=p0, dt=dt)
    errs = []
    for alpha in (1.0, 10.0, 100.0):
        P = O.OracleProblem(W.Workload("dg", [lo, hi], 300, rec, cfl=0.02, penalty_alpha=alpha))
        x2, y2, z2 = P.all_coordinates()
        q0, _ = W.standing_wave_mode(one, (1, 0, 1), x2, y2, z2)
        tr = P.run(p0=q0, dt=dt * 0.25 if alpha == 100.0 else dt, nsteps=1200 if alpha == 100.0 else 300)
        if alpha == 100.0:
            tr = tr[:, :, 3::4]
        errs.append(np.abs(tr - t_ref).max() / np.abs(t_ref).max())
    assert errs[0] < 0.05
    assert errs[1] < errs[0] and errs[2] < errs[1]


def test_face_matching_finds_coarse_quadrant(two_domain):
    """Algorithm 3 on the 2:1 interface: each fine face's quadrature nodes land
    in the coarse element above it, at reference coordinates of its quadrant."""
    _, P = two_domain
    prim, sec = P.meshes
    g, _ = O.gauss_legendre(3)
    ref = np.array([[a, b] for b in g for a in g])
    fine = [O._Face(prim, (ex, ey, prim.ne[2] - 1), "top") for ey in range(4) for ex in range(4)]
    coarse = [O._Face(sec, (ex, ey, 0), "bottom") for ey in range(2) for ex in range(2)]
    for F, _, pts in O.match_interface(fine, coarse, ref):
        ex, ey, _ = F.elem
        for q, (G, rm) in enumerate(pts):
            assert G.elem == (ex // 2, ey // 2, 0)
            assert abs(rm[2] + 1.0) < 1e-12
            expect_x = -1 + ((ex % 2) + (ref[q, 0] + 1) / 2)
            assert abs(rm[0] - expect_x) < 1e-12


# ---------------------------------------------------------------------------
# First-order absorbing boundary (damping form d of eq. Wf_4)
# ---------------------------------------------------------------------------
def _abc_box(absorbing, nel=(3, 2, 2), order=4, h=75e-6):
    dom = W.Domain((0, 0, 0), tuple(n * h for n in nel), nel, order, absorbing=absorbing)
    return W.Workload("abc_box", [dom], 10, np.array([[h, h, h]]))


def test_abc_matrix_is_face_quadrature_of_c():
    """C sums to c x (area of the absorbing sides); zero off those sides."""
    w = _abc_box((1, 0, 0, 1, 0, 1))
    P = O.OracleProblem(w)
    d = w.domains[0]
    Lx, Ly, Lz = d.extent
    assert abs(P.C.sum() - d.c * (Ly * Lz + Lx * Lz + Lx * Ly)) < 1e-12 * d.c * Lx * Ly
    x, y, z = P.all_coordinates()
    on = (np.isclose(x, 0) | np.isclose(y, Ly) | np.isclose(z, Lz))
    assert np.all(P.C[~on] == 0) and np.all(P.C[on] > 0)


def test_abc_discrete_energy_balance():
    """Algorithm 1 with C acting on the predicted velocity v^{n+1/2}:
    E^{n+1} - E^n = -(dt/2) v^{n+1/2}.C (v^{n+1/2} + v^{n+3/2}) exactly, with
    E the leapfrog energy 1/2 v.M v + 1/2 p^{n+1}.K p^{n+2}."""
    w = _abc_box((1, 1, 0, 1, 1, 0))
    P = O.OracleProblem(w)
    x, y, z = P.all_coordinates()
    p0 = W.seeded_field(4, x, y, z)
    v0 = 1e3 * W.seeded_field(5, x, y, z)
    dt = P.stable_dt()
    vs = []
    _, E = P.run(nsteps=40, dt=dt, p0=p0, v0=v0, energy=True, batch=1,
                 callback=lambda n, p, pd, pdd, **k: vs.append((pd + 0.5 * dt * pdd)[:, 0].copy()))
    e = E[:, 0, 0]
    for n in range(1, 40):
        pred = -0.5 * dt * np.dot(vs[n - 1] * P.C, vs[n - 1] + vs[n])
        assert abs((e[n] - e[n - 1]) - pred) <= 1e-9 * abs(e[n]), n
    assert e[-1] < e[0]


def test_abc_absorbs_a_normally_incident_plane_wave():
    """A plane pulse running along +x leaves through an absorbing x+ side
    (rigid walls normal to y and z keep it an exact plane wave): almost no
    energy remains, while a rigid x+ side reflects all of it."""
    h, N = 75e-6, 4
    nel = (24, 1, 1)
    out = {}
    for sides in [(0, 1, 0, 0, 0, 0), (0, 0, 0, 0, 0, 0)]:
        dom = W.Domain((0, 0, 0), tuple(n * h for n in nel), nel, N, absorbing=sides)
        w = W.Workload("pulse", [dom], 10, np.array([[h, h / 2, h / 2]]))
        P = O.OracleProblem(w)
        x, y, z = P.all_coordinates()
        Lx = dom.extent[0]
        p0, v0 = W.gaussian_pulse_x(dom, x, 0.6 * Lx, 2 * h, +1)
        dt = P.stable_dt()
        S = int((0.4 * Lx + 8 * h) / dom.c / dt)
        _, E = P.run(nsteps=S, dt=dt, p0=p0, v0=v0, energy=True, batch=1)
        out[sides[1]] = E[-1, 1, 0] / E[0, 1, 0]
    assert out[1] < 1e-3, out
    assert out[0] > 0.99, out


def test_abc_step_map_is_stable_at_the_chosen_dt():
    """Spectral radius of the damped leapfrog map (p^{n+1}, v^{n+1/2}) ->
    (p^{n+2}, v^{n+3/2}) with every side absorbing, at stable_dt(): <= 1."""
    for order, nel in [(2, (3, 2, 2)), (4, (2, 2, 2))]:
        w = _abc_box((1, 1, 1, 1, 1, 1), nel=nel, order=order)
        P = O.OracleProblem(w)
        dt = P.stable_dt()
        n = P.nh
        A = P.Minv[:, None] * P.K.toarray()
        s = P.Minv * P.C
        Vp, Vv = -dt * A, np.eye(n) - dt * np.diag(s)
        T = np.block([[np.eye(n) + dt * Vp, dt * Vv], [Vp, Vv]])
        assert np.max(np.abs(np.linalg.eigvals(T))) <= 1.0 + 1e-9
        # and the limit is the damping one here (three absorbing sides meet at the corners)
        assert abs(dt * np.max(s) - 1.0) < 1e-12


# ---------------------------------------------------------------------------
# TX -> RX switch of the PMUT voltage (eq. ode row 2, eq. pmut_problem row 2)
# ---------------------------------------------------------------------------
def _rx_workload(sign, rho=1.0e-12, nsteps=900, rx_switch=650):
    L = 0.3e-3
    dom = W.Domain((0.0, 0.0, 0.0), (L, L, L), (4, 4, 4), 4, rho=rho)
    pm = W.make_pmut_array([[0.15e-3, 0.15e-3]], 60e-6, W.MODE_FREQS_5[:3], 0.0)
    d, a = W._uniform_drive(1)
    w = W.Workload("rx", [dom], nsteps, np.array([[0.15e-3, 0.15e-3, 0.15e-3]]), pm, drive_delay=d, drive_amp=a)
    w.rx_switch, w.rx_capacitance, w.rx_sign = rx_switch, np.array([1.0e-12]), sign
    return w


@pytest.mark.parametrize("sign", [-1, +1])
def test_rx_open_circuit_modal_recurrence(sign):
    """With a negligible fluid density the membrane is decoupled, and after the
    switch Algorithm 1 (phi^n from q^n, stiffness on q^{n+1}) gives exactly
      q^{n+2} - 2 q^{n+1} + q^n = dt^2 (-W q^{n+1} + (s/C) mu^-1 eta eta^T q^n),
    and the recorded voltage is phi^n = (s/C) eta . q^n."""
    w = _rx_workload(sign)
    P = O.OracleProblem(w)
    dt = P.stable_dt()
    Q = []
    P.run(dt=dt, batch=1, callback=lambda n, q=None, **k: Q.append(q[:, 0].copy()))
    a = np.array([np.zeros(3)] + Q)                       # a[n] = q^n
    pm = w.pmuts
    eta, mu = pm.eta[0], pm.modal_mass[0]
    om2 = (2 * np.pi * pm.freq_hz[0]) ** 2
    Lam = (sign / 1.0e-12) * np.outer(eta / mu, eta)
    n0 = w.rx_switch
    scale = np.abs(a).max()
    assert scale > 0
    for n in range(n0, w.nsteps - 1):
        lhs = a[n + 2] - 2 * a[n + 1] + a[n]
        rhs = dt * dt * (-om2 * a[n + 1] + Lam @ a[n])
        assert np.abs(lhs - rhs).max() <= 1e-9 * scale, n
    volts = P.voltages[0, 0]
    for n in range(n0, w.nsteps):
        assert abs(volts[n] - (sign / 1.0e-12) * np.dot(eta, a[n])) <= 1e-12 * abs(volts).max()
    # before the switch the recorded voltage is the drive
    np.testing.assert_array_equal(volts[:n0], w.drive(dt, w.nsteps, 1)[0, 0, :n0])



# ---------------------------------------------------------------------------
# Perfectly matched layer (eq. full_problem rows 1-3, damping profile of Sec. 2)
# ---------------------------------------------------------------------------
def _pml_reflection(layer_el, R, rigid=False, h=75e-6):
    """Peak of the wave reflected back to an interior receiver by an x+ side
    carrying a PML of layer_el elements (rigid wall behind it) for a plane
    pulse that runs along +x."""
    nin = 16
    th = 0.0 if rigid else layer_el * h
    nel = (nin + (0 if rigid else layer_el), 1, 1)
    dom = W.Domain((0, 0, 0), tuple(n * h for n in nel), nel, 4, pml=(0, th, 0, 0, 0, 0), pml_R=R)
    Li = nin * h
    P = O.OracleProblem(W.Workload("pulse", [dom], 10, np.array([[0.3 * Li, h / 2, h / 2]])))
    x, y, z = P.all_coordinates()
    p0, v0 = W.gaussian_pulse_x(dom, x, 0.5 * Li, 1.5 * h, +1)
    dt = P.stable_dt()
    S = int((0.5 * Li + 2 * th + 0.7 * Li + 10 * h) / dom.c / dt)
    tr = P.run(nsteps=S, dt=dt, p0=p0, v0=v0, batch=1)[0, 0]
    n0 = int((0.2 * Li + 6 * h) / dom.c / dt)          # after the initial pulse has left the receiver
    return np.abs(tr[n0:]).max()


def test_pml_reflection_is_the_design_coefficient():
    """The profile zeta~ = c/l log(1/R) attenuates a normally incident wave by
    exactly R over the round trip through a rigid-backed layer (the profile
    integrates to l/2).  With the layer resolved (8 elements) the discrete
    reflection is within 10 % of R = 1e-2; a bare rigid wall reflects all."""
    assert abs(_pml_reflection(0, 1e-2, rigid=True) - 1.0) < 1e-3
    r = _pml_reflection(8, 1e-2)
    assert abs(r / 1e-2 - 1.0) < 0.1, r


def test_pml_small_design_reflection_absorbs_strongly():
    assert _pml_reflection(8, 1e-4) < 1e-3


def test_pml_long_run_decays_without_growth():
    """Seeded field in a box with PML on five sides: no growth over 1500
    steps, and almost everything is absorbed."""
    h = 75e-6
    dom = W.Domain((0, 0, 0), (5 * h, 3 * h, 3 * h), (5, 3, 3), 4,
                   pml=(h, h, h, h, 0, h), pml_R=1e-4)
    P = O.OracleProblem(W.Workload("s", [dom], 10, np.array([[2.5 * h, 1.5 * h, 1.5 * h]])))
    x, y, z = P.all_coordinates()
    p0 = W.seeded_field(3, x, y, z)
    tr = P.run(nsteps=1500, dt=P.stable_dt(), p0=p0, batch=1)
    assert np.abs(tr).max() <= 1.01 * np.abs(p0).max()
    assert np.abs(P.final_state["p"]).max() < 1e-2 * np.abs(p0).max()
