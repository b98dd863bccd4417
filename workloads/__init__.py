"""Seeded synthetic inputs for the DG-SEM + reduced-order PMUT time step.

This module is the only code shared by the CUDA path's tests/bench and the
CPU oracle.  It describes *inputs*: box geometry, material constants, PMUT
placement, mode-shape functions, modal parameters, drive voltages and
receiver positions.  It contains none of the method's arithmetic (no basis
functions, quadrature of the discretisation, assembly or time stepping).

The paper measures on its own meshes and on COMSOL comparisons that are not
available; the workloads below are synthetic stand-ins with the sizes of the
paper's problem class (water, c = 1500 m/s, rho = 1000 kg/m^3, square PMUT
membranes on the z = 0 face of a fine primary box, a coarser secondary box
stacked on top through a 2:1 non-conforming interface).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

WATER_C = 1500.0
WATER_RHO = 1000.0

# Mode table of a clamped square plate approximated by products of clamped
# beam polynomials (Sec. 2 reduced-order model, shapes U_{k,m}).  Entries:
# (shape-x, shape-y, frequency ratio to mode 1).  Ratios 1 : 2.04 : 3.01 : 3.66
# follow the clamped-square-plate eigenvalue ratios.
_MODE_TABLE = [
    ("p1", "p1", 1.0),
    ("p2", "p1", 2.05),
    ("p1", "p2", 2.05),
    ("p2", "p2", 3.0),
    ("p31", "p31", 3.65),   # symmetric combination phi3(x)phi1(y)+phi1(x)phi3(y)
]


def _p1(s):
    return (1.0 - s * s) ** 2


def _p2(s):
    return s * (1.0 - s * s) ** 2


def _p3(s):
    return (1.0 - s * s) ** 2 * (s * s - 1.0 / 11.0)


def _raw_shape(m: int, xi, eta):
    sx, sy, _ = _MODE_TABLE[m]
    if sx == "p31":
        return _p3(xi) * _p1(eta) + _p1(xi) * _p3(eta)
    f = {"p1": _p1, "p2": _p2}
    return f[sx](xi) * f[sy](eta)


def _shape_peak(m: int) -> float:
    s = np.linspace(-1.0, 1.0, 2001)
    X, Y = np.meshgrid(s, s, indexing="ij")
    return float(np.max(np.abs(_raw_shape(m, X, Y))))


_PEAKS = [_shape_peak(m) for m in range(len(_MODE_TABLE))]


def _shape_integrals(m: int):
    """(int phi_m dA / A, int phi_m^2 dA / A) over the reference square, exact
    for these polynomials (Gauss-Legendre with 12 points per direction)."""
    g, w = np.polynomial.legendre.leggauss(12)
    X, Y = np.meshgrid(g, g, indexing="ij")
    W = np.outer(w, w)
    phi = _raw_shape(m, X, Y) / _PEAKS[m]
    return float((W * phi).sum() / 4.0), float((W * phi * phi).sum() / 4.0)


@dataclass
class Domain:
    """Axis-aligned box meshed by nelem hexahedra of GLL order `order`.
    absorbing: per box side (x-, x+, y-, y+, z-, z+) 1 = first-order
    absorbing boundary (Gamma_ABC), 0 = rigid wall (Gamma_N).
    pml: per box side the thickness of a perfectly matched layer inside the
    box along that side (0 = none), pml_R its design reflection."""
    origin: tuple
    extent: tuple
    nelem: tuple
    order: int
    c: float = WATER_C
    rho: float = WATER_RHO
    absorbing: tuple = (0, 0, 0, 0, 0, 0)
    # perfectly matched layer: thickness (m) per box side, 0 = none, and the
    # design reflection coefficient R of the damping profile
    pml: tuple = (0.0, 0.0, 0.0, 0.0, 0.0, 0.0)
    pml_R: float = 1.0e-4


@dataclass
class PmutArray:
    """Square PMUT membranes on the z = origin_z face of the primary box.

    U_{k,m} = phi_m e_z points into the fluid; on that face the outward normal
    of the fluid domain is -e_z, so U_{k,m}.n = -phi_m (shape_un below).
    """
    centers: np.ndarray          # [K, 2] (x, y) in metres
    side: float                  # membrane side in metres
    freq_hz: np.ndarray          # [K, M]
    damping: np.ndarray          # [K, M] modal damping ratio zeta
    eta: np.ndarray              # [K, M] electromechanical coupling, N/V
    modal_mass: np.ndarray       # [K, M] kg

    @property
    def n_pmut(self) -> int:
        return int(self.centers.shape[0])

    @property
    def n_modes(self) -> int:
        return int(self.freq_hz.shape[1])

    def local_coords(self, k: int, x, y):
        xc, yc = self.centers[k]
        return 2.0 * (np.asarray(x) - xc) / self.side, 2.0 * (np.asarray(y) - yc) / self.side

    def inside(self, k: int, x, y):
        xi, eta = self.local_coords(k, x, y)
        return (np.abs(xi) < 1.0) & (np.abs(eta) < 1.0)

    def shape_un(self, k: int, m: int, x, y):
        """U_{k,m}.n at points (x, y) of the PMUT face (zero outside)."""
        xi, eta = self.local_coords(k, x, y)
        inside = (np.abs(xi) < 1.0) & (np.abs(eta) < 1.0)
        val = -_raw_shape(m, xi, eta) / _PEAKS[m]
        return np.where(inside, val, 0.0)


@dataclass
class Workload:
    name: str
    domains: List[Domain]
    nsteps: int
    receivers: np.ndarray                  # [R, 3]
    pmuts: Optional[PmutArray] = None
    cfl: float = 0.3
    penalty_alpha: float = 0.5
    quad_pts: int = 0                      # 0: max order + 1 Gauss points per direction
    batch: int = 1
    # drive description: per pattern b and PMUT k a delay (s) and an amplitude (V)
    drive_delay: Optional[np.ndarray] = None      # [B, K]
    drive_amp: Optional[np.ndarray] = None        # [B, K]
    burst_freq: float = 2.0e6
    burst_cycles: float = 3.0
    # TX -> RX switch: from step rx_switch on, membrane k's voltage is the
    # open-circuit value rx_sign / C_k sum_m eta_km q_km (None: transmit only)
    rx_switch: Optional[int] = None
    rx_capacitance: Optional[np.ndarray] = None   # [K] farads
    rx_sign: int = -1

    def drive(self, dt: float, nsteps: Optional[int] = None, batch: Optional[int] = None) -> np.ndarray:
        """phi_k(t^n) for t^n = n dt, n = 0..S-1, shape [B, K, S] (volts).

        Hann-windowed tone burst A sin(2 pi f t) (1 - cos(2 pi t / T_b)) / 2 on
        0 <= t <= T_b = cycles / f, delayed by the per-PMUT delay.
        """
        S = self.nsteps if nsteps is None else nsteps
        B = self.batch if batch is None else batch
        K = self.pmuts.n_pmut if self.pmuts is not None else 0
        out = np.zeros((B, K, S))
        if K == 0:
            return out
        t = np.arange(S) * dt
        Tb = self.burst_cycles / self.burst_freq
        for b in range(B):
            for k in range(K):
                tau = self.drive_delay[b, k]
                s = t - tau
                on = (s >= 0.0) & (s <= Tb)
                wave = np.sin(2 * math.pi * self.burst_freq * s) * 0.5 * (1.0 - np.cos(2 * math.pi * s / Tb))
                out[b, k] = np.where(on, self.drive_amp[b, k] * wave, 0.0)
        return out

    @property
    def ndof(self) -> int:
        n = 0
        for d in self.domains:
            n += int(np.prod([d.nelem[i] * d.order + 1 for i in range(3)]))
        return n


def make_pmut_array(centers, side, base_freqs, zeta, rho_s=1.0e-1, static_defl=1.0e-9,
                    freq_scale=None) -> PmutArray:
    """Modal parameters of a PMUT array.

    modal_mass mu_m = rho_s * int U_m^2 dA; coupling eta_m = e0 * (int phi_m dA / A)
    for a uniform electrode, with e0 chosen so that mode 1 deflects
    `static_defl` metres per volt statically (eta_1 = static_defl * mu_1 * w_1^2).
    """
    centers = np.asarray(centers, dtype=np.float64).reshape(-1, 2)
    K = centers.shape[0]
    M = len(base_freqs)
    scale = np.ones(K) if freq_scale is None else np.asarray(freq_scale, dtype=np.float64)
    freq = np.outer(scale, np.asarray(base_freqs, dtype=np.float64))
    area = side * side
    mean_phi = np.array([_shape_integrals(m)[0] for m in range(M)])
    mean_phi2 = np.array([_shape_integrals(m)[1] for m in range(M)])
    mu = np.tile(rho_s * area * mean_phi2, (K, 1))
    w1 = 2 * math.pi * freq[:, 0]
    e0 = static_defl * mu[:, 0] * w1 * w1 / mean_phi[0]
    eta = e0[:, None] * mean_phi[None, :]
    eta = np.where(np.abs(mean_phi)[None, :] < 1e-14, 0.0, eta)
    damping = np.full((K, M), float(zeta))
    return PmutArray(centers=centers, side=float(side), freq_hz=freq, damping=damping,
                     eta=eta, modal_mass=mu)


def _grid_centers(n, pitch, x0=0.0, y0=0.0):
    c = (np.arange(n) + 0.5) * pitch
    X, Y = np.meshgrid(c + x0, c + y0, indexing="ij")
    return np.stack([X.ravel(), Y.ravel()], axis=1)


def _uniform_drive(K, B=1, amp=10.0):
    return np.zeros((B, K)), np.full((B, K), amp)


MODE_FREQS_5 = [2.0e6 * r for (_, _, r) in _MODE_TABLE]


def config1_single_pmut(nsteps: int = 2000) -> Workload:
    """One 60 um PMUT (3 modes 2.0/4.1/4.1 MHz, zeta 0.01) centred on the z = 0
    face of a 0.6 mm water cube, 8^3 hexes at N = 4, rigid walls, 4 receivers."""
    L = 0.6e-3
    dom = Domain((0.0, 0.0, 0.0), (L, L, L), (8, 8, 8), 4)
    pm = make_pmut_array([[0.3e-3, 0.3e-3]], 60e-6, MODE_FREQS_5[:3], 0.01)
    rec = np.array([[0.3, 0.3, 0.15], [0.3, 0.3, 0.3], [0.3, 0.3, 0.45], [0.15, 0.45, 0.3]]) * 1e-3
    d, a = _uniform_drive(1)
    return Workload("config1_single_pmut", [dom], nsteps, rec, pm, drive_delay=d, drive_amp=a)


def _stacked(nx_p, nz_p, Lxy, Lz_p, nx_s, nz_s, Lz_s):
    prim = Domain((0.0, 0.0, 0.0), (Lxy, Lxy, Lz_p), (nx_p, nx_p, nz_p), 4)
    sec = Domain((0.0, 0.0, Lz_p), (Lxy, Lxy, Lz_s), (nx_s, nx_s, nz_s), 6)
    return [prim, sec]


def config2_array16(nsteps: int = 4000) -> Workload:
    """16x16 PMUTs (pitch 100 um, 5 modes, +-3 % frequency spread, seed 1) on a
    64x64x16 N=4 primary box below a 32x32x64 N=6 secondary box (2:1 interface);
    64 receivers on a plane 2 mm above the array."""
    rng = np.random.default_rng(1)
    doms = _stacked(64, 16, 1.6e-3, 0.4e-3, 32, 64, 3.2e-3)
    centers = _grid_centers(16, 100e-6)
    pm = make_pmut_array(centers, 60e-6, MODE_FREQS_5, 0.01,
                         freq_scale=rng.uniform(0.97, 1.03, size=centers.shape[0]))
    g = 100e-6 + 200e-6 * np.arange(8)
    X, Y = np.meshgrid(g, g, indexing="ij")
    rec = np.stack([X.ravel(), Y.ravel(), np.full(64, 2.0e-3)], axis=1)
    d, a = _uniform_drive(centers.shape[0])
    return Workload("config2_array16", doms, nsteps, rec, pm, drive_delay=d, drive_amp=a)


def config3_array32(nsteps: int = 8000, batch: int = 1, seed: int = 3) -> Workload:
    """32x32 = 1024 PMUTs (5 modes) on a 128x128x16 N=4 primary box
    (3.2 x 3.2 x 0.4 mm) below a 64x64x96 N=6 secondary box (3.2 x 3.2 x 4.8 mm);
    64 receivers at z = 2 mm."""
    rng = np.random.default_rng(seed)
    doms = _stacked(128, 16, 3.2e-3, 0.4e-3, 64, 96, 4.8e-3)
    centers = _grid_centers(32, 100e-6)
    pm = make_pmut_array(centers, 60e-6, MODE_FREQS_5, 0.01,
                         freq_scale=rng.uniform(0.97, 1.03, size=centers.shape[0]))
    g = 200e-6 + 400e-6 * np.arange(8)
    X, Y = np.meshgrid(g, g, indexing="ij")
    rec = np.stack([X.ravel(), Y.ravel(), np.full(64, 2.0e-3)], axis=1)
    d, a = _uniform_drive(centers.shape[0], batch)
    return Workload("config3_array32", doms, nsteps, rec, pm, batch=batch, drive_delay=d, drive_amp=a)


def config3_crop(nsteps: int = 8000, batch: int = 1) -> Workload:
    """The config-3 problem cropped to its first 8x8 block of PMUTs: a 32x32x16
    N=4 primary box (0.8 x 0.8 x 0.4 mm) below a 16x16x96 N=6 secondary box
    (0.8 x 0.8 x 4.8 mm), 6,510,658 nodes.  Element sizes, orders, heights,
    time step and horizon are config 3's; the 64 PMUTs are config 3's
    membranes (i, j) < 8 with their seeded frequency factors.  64 receivers on
    an 8x8 grid (pitch 100 um) at z = 2 mm.  The crop's x/y walls are rigid,
    so this is its own problem, small enough for the oracle."""
    full = config3_array32(nsteps=nsteps, batch=batch)
    doms = _stacked(32, 16, 0.8e-3, 0.4e-3, 16, 96, 4.8e-3)
    c = full.pmuts.centers
    keep = np.nonzero((c[:, 0] < 0.8e-3) & (c[:, 1] < 0.8e-3))[0]
    pm = PmutArray(centers=c[keep].copy(), side=full.pmuts.side, freq_hz=full.pmuts.freq_hz[keep].copy(),
                   damping=full.pmuts.damping[keep].copy(), eta=full.pmuts.eta[keep].copy(),
                   modal_mass=full.pmuts.modal_mass[keep].copy())
    g = 50e-6 + 100e-6 * np.arange(8)
    X, Y = np.meshgrid(g, g, indexing="ij")
    rec = np.stack([X.ravel(), Y.ravel(), np.full(64, 2.0e-3)], axis=1)
    d, a = _uniform_drive(keep.size, batch)
    return Workload("config3_crop", doms, nsteps, rec, pm, batch=batch, drive_delay=d, drive_amp=a)


def steering_patterns(centers: np.ndarray, batch: int, seed: int, c: float = WATER_C,
                      jitter: float = 5e-9, max_angle_deg: float = 30.0, amp=(0.8, 1.2),
                      base_amp: float = 10.0):
    """Beam-steering drive patterns: delay tau_k = x_k sin(theta)/c + N(0, jitter),
    shifted so that min tau = 0, theta ~ U[-max, max]; amplitude ~ U[amp] * base."""
    rng = np.random.default_rng(seed)
    K = centers.shape[0]
    theta = np.deg2rad(rng.uniform(-max_angle_deg, max_angle_deg, size=batch))
    x = centers[:, 0] - centers[:, 0].mean()
    delay = x[None, :] * np.sin(theta)[:, None] / c + rng.normal(0.0, jitter, size=(batch, K))
    delay -= delay.min(axis=1, keepdims=True)
    ampl = base_amp * rng.uniform(amp[0], amp[1], size=(batch, K))
    return delay, ampl, theta


def config4_batched(nsteps: int = 8000, batch: int = 64) -> Workload:
    """64 beam-steering drive patterns on the 1024-PMUT config-3 mesh (seed 4)."""
    w = config3_array32(nsteps=nsteps, batch=batch)
    w.name = "config4_batched"
    w.drive_delay, w.drive_amp, _ = steering_patterns(w.pmuts.centers, batch, seed=4)
    return w


def config4b_uneven(nsteps: int = 8000, batch: int = 64, sides=(8, 16, 24, 32)) -> List[Workload]:
    """Uneven arrays in one launch: for each side a in `sides`, an a x a PMUT
    array (pitch 100 um, 5 modes, +-3 % spread) on a 4a x 4a x 16 N=4 primary
    box (h = 25 um, 0.4 mm high) below a 2a x 2a x 96 N=6 secondary box
    (4.8 mm high), 64 receivers on an 8x8 grid at z = 2 mm, `batch`
    beam-steering drive patterns per array (seed 40 + a).  The 32 x 32 member
    is the config-3 mesh."""
    out = []
    for a in sides:
        rng = np.random.default_rng(1000 + a)
        L = a * 100e-6
        doms = _stacked(4 * a, 16, L, 0.4e-3, 2 * a, 96, 4.8e-3)
        centers = _grid_centers(a, 100e-6)
        pm = make_pmut_array(centers, 60e-6, MODE_FREQS_5, 0.01,
                             freq_scale=rng.uniform(0.97, 1.03, size=centers.shape[0]))
        g = (np.arange(8) + 0.5) * L / 8
        X, Y = np.meshgrid(g, g, indexing="ij")
        rec = np.stack([X.ravel(), Y.ravel(), np.full(64, 2.0e-3)], axis=1)
        d, amp, _ = steering_patterns(centers, batch, seed=40 + a)
        out.append(Workload(f"config4b_array{a}", doms, nsteps, rec, pm, batch=batch, drive_delay=d,
                            drive_amp=amp))
    return out


def small_two_domain(nx_p=4, nz_p=2, nx_s=2, nz_s=4, n_pmut_side=2, nsteps=200, batch=1,
                     order_p=4, order_s=6, seed=11, h_p=25e-6, n_modes=5,
                     penalty_alpha=0.5, steer=False) -> Workload:
    """A small primary/secondary pair with the config-2 element sizes (primary
    h = 25 um, secondary h = 2 h laterally) for parity runs the oracle finishes
    in seconds.  Receivers are scattered through both boxes."""
    rng = np.random.default_rng(seed)
    Lxy = nx_p * h_p
    Lz_p = nz_p * h_p
    hs = Lxy / nx_s
    Lz_s = nz_s * hs
    prim = Domain((0.0, 0.0, 0.0), (Lxy, Lxy, Lz_p), (nx_p, nx_p, nz_p), order_p)
    sec = Domain((0.0, 0.0, Lz_p), (Lxy, Lxy, Lz_s), (nx_s, nx_s, nz_s), order_s)
    pitch = Lxy / n_pmut_side
    centers = _grid_centers(n_pmut_side, pitch)
    side = min(60e-6, 0.6 * pitch)
    pm = make_pmut_array(centers, side, MODE_FREQS_5[:n_modes], 0.01,
                         freq_scale=rng.uniform(0.97, 1.03, size=centers.shape[0]))
    R = 12
    rec = np.column_stack([rng.uniform(0, Lxy, R), rng.uniform(0, Lxy, R),
                           rng.uniform(0.0, Lz_p + Lz_s, R)])
    if steer:
        d, a, _ = steering_patterns(centers, batch, seed + 1)
    else:
        d, a = _uniform_drive(centers.shape[0], batch)
        a = a * rng.uniform(0.5, 1.5, size=a.shape)
    return Workload("small_two_domain", [prim, sec], nsteps, rec, pm, batch=batch,
                    penalty_alpha=penalty_alpha, drive_delay=d, drive_amp=a)


def small_one_domain(nel=(3, 2, 2), order=4, nsteps=200, batch=1, seed=12, h=75e-6,
                     n_modes=3, n_pmut_side=1) -> Workload:
    """A single box with PMUTs on z = 0 (ragged element counts per axis)."""
    rng = np.random.default_rng(seed)
    L = tuple(n * h for n in nel)
    dom = Domain((0.0, 0.0, 0.0), L, tuple(nel), order)
    px = L[0] / n_pmut_side
    py = L[1] / n_pmut_side
    c = (np.arange(n_pmut_side) + 0.5)
    X, Y = np.meshgrid(c * px, c * py, indexing="ij")
    centers = np.stack([X.ravel(), Y.ravel()], axis=1)
    side = min(60e-6, 0.6 * min(px, py))
    pm = make_pmut_array(centers, side, MODE_FREQS_5[:n_modes], 0.01)
    R = 6
    rec = np.column_stack([rng.uniform(0, L[0], R), rng.uniform(0, L[1], R), rng.uniform(0, L[2], R)])
    d, a = _uniform_drive(centers.shape[0], batch)
    a = a * rng.uniform(0.5, 1.5, size=a.shape)
    return Workload("small_one_domain", [dom], nsteps, rec, pm, batch=batch, drive_delay=d, drive_amp=a)


def standing_wave_mode(domain: Domain, l: tuple, x, y, z):
    """Rigid-box eigenfunction prod_d cos(l_d pi (x_d - o_d) / L_d) and its
    angular frequency c |k| (closed form, used as an initial state)."""
    o, L = domain.origin, domain.extent
    val = (np.cos(l[0] * math.pi * (np.asarray(x) - o[0]) / L[0])
           * np.cos(l[1] * math.pi * (np.asarray(y) - o[1]) / L[1])
           * np.cos(l[2] * math.pi * (np.asarray(z) - o[2]) / L[2]))
    k2 = sum((l[i] * math.pi / L[i]) ** 2 for i in range(3))
    return val, domain.c * math.sqrt(k2)


def seeded_field(rng_seed: int, x, y, z, scale=1.0):
    """A smooth random field (sum of a few random cosines) for initial states."""
    rng = np.random.default_rng(rng_seed)
    out = np.zeros_like(np.asarray(x, dtype=np.float64))
    for _ in range(4):
        k = rng.uniform(500.0, 20000.0, size=3)
        ph = rng.uniform(0, 2 * math.pi, size=3)
        a = rng.normal()
        out = out + a * np.cos(k[0] * x + ph[0]) * np.cos(k[1] * y + ph[1]) * np.cos(k[2] * z + ph[2])
    return scale * out


def surrogate_array(batch: int = 64, seed: int = 5, nsteps: int = 2950) -> Workload:
    """Training/evaluation workload of the learned surrogate: an 8x8 PMUT array
    (pitch 100 um, 5 modes, +-3 % spread) on a 32x32x8 N=4 primary box
    (0.8 x 0.8 x 0.2 mm) under a 16x16x24 N=6 secondary box (0.8 x 0.8 x 1.2 mm),
    64 receivers on an 8x8 grid at z = 0.8 mm, beam-steering drive patterns.
    The config-4 mesh would cost ~0.8 TDoF-steps per pattern; this one ~5.6 G."""
    rng = np.random.default_rng(seed)
    doms = _stacked(32, 8, 0.8e-3, 0.2e-3, 16, 24, 1.2e-3)
    centers = _grid_centers(8, 100e-6)
    pm = make_pmut_array(centers, 60e-6, MODE_FREQS_5, 0.01,
                         freq_scale=rng.uniform(0.97, 1.03, size=centers.shape[0]))
    g = 50e-6 + 100e-6 * np.arange(8)
    X, Y = np.meshgrid(g, g, indexing="ij")
    rec = np.stack([X.ravel(), Y.ravel(), np.full(64, 0.8e-3)], axis=1)
    d, a, _ = steering_patterns(centers, batch, seed=seed + 1000)
    return Workload("surrogate_array", doms, nsteps, rec, pm, batch=batch, drive_delay=d, drive_amp=a)


def gaussian_pulse_x(domain: Domain, x, center: float, width: float, direction: int = 1):
    """Plane pulse g(x) = exp(-((x - center)/width)^2) travelling along
    direction * e_x at the domain's sound speed: p0 = g, p'0 = -direction c g'.
    With rigid walls normal to y and z this is an exact solution of the wave
    equation until it reaches an x side."""
    s = (np.asarray(x) - center) / width
    g = np.exp(-s * s)
    dg = -2.0 * s / width * g
    return g, -direction * domain.c * dg
