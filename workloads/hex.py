"""Seeded synthetic inputs for general hexahedral meshes (trilinear elements).

Like the rest of ``workloads`` this module only describes inputs: vertex
positions, element-to-vertex lists, the face lists of the interface and of the
PMUT plane, PMUT parameters, drive voltages and receiver positions.  It holds
none of the method's arithmetic.

Element convention (the one the C ABI documents): an element lists 8 vertex
ids; corner (i, j, k) in {0, 1}^3 sits at list position i + 2 j + 4 k and is
the image of the reference corner (2 i - 1, 2 j - 1, 2 k - 1).  Local face
f = 2 * axis + side is the face xi_axis = -1 (side 0) or +1 (side 1).

The meshes stand in for the body-fitted meshes of the paper's Sec. 6 (the
paper's own meshes are not available): a structured lattice of hexahedra whose
vertices are moved by a smooth displacement field.  The field keeps every outer
wall plane in place (vertices only slide inside their wall), so the union of
the elements stays the box; the interface between the fine primary and the
coarse secondary domain is bent into a bump.  Fine interface vertices are put
on the coarse faces' bilinear patches (at the images of the 2:1 sub-square
corners), so the two sides of the curved interface coincide geometrically.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import List, Optional

import numpy as np

from . import (WATER_C, WATER_RHO, MODE_FREQS_5, Workload, make_pmut_array, _grid_centers,
               _uniform_drive, steering_patterns)


@dataclass
class HexDomain:
    """One domain of trilinear hexahedra of GLL order `order`."""
    vertices: np.ndarray       # [nv, 3] metres
    elements: np.ndarray       # [ne, 8] vertex ids, corner (i, j, k) at i + 2 j + 4 k
    order: int
    c: float = WATER_C
    rho: float = WATER_RHO
    # lattice description kept for the generators' own bookkeeping (not an input of the method)
    lattice: Optional[tuple] = None   # (nx, ny, nz)


@dataclass
class HexWorkload(Workload):
    """Workload on general hexahedral domains (domain 0 = fine primary)."""
    fine_faces: Optional[np.ndarray] = None     # [nf, 2] (element, local face) of domain 0 on Gamma_I
    coarse_faces: Optional[np.ndarray] = None   # [nc, 2] of domain 1 on Gamma_I
    pmut_faces: Optional[np.ndarray] = None     # [np, 2] of domain 0 on Gamma_PMUT
    # first-order absorbing faces (Gamma_ABC) per domain: [n, 2] (element, local face) or None
    absorbing_faces: Optional[list] = None
    # perfectly matched layers per domain: thickness (m) along the sides x-, x+, y-, y+, z-, z+
    # of the domain's bounding box (None or zeros: none), design reflection pml_R
    pml: Optional[list] = None
    pml_R: float = 1.0e-4
    normal_tol: float = 0.5                     # Algorithm 3 |n+ + n-| < tol
    box_extent: Optional[tuple] = None          # the box the mesh fills (for receivers)

    @property
    def ndof(self) -> int:   # not known without the node numbering
        raise AttributeError("ndof of a general hexahedral workload comes from the mesh")


# The 24 proper rotations of the cube as maps of corner bit patterns.  A
# rotation R maps reference corner s in {-1, 1}^3 to R s; an element whose
# local frame is rotated lists at new position c the vertex of old corner
# R(c).  Generated from the axis permutations with sign flips of determinant +1.
def _cube_rotations():
    mats = []
    import itertools
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((-1, 1), repeat=3):
            R = np.zeros((3, 3))
            for r in range(3):
                R[r, perm[r]] = signs[r]
            if np.linalg.det(R) > 0:
                mats.append(R)
    return mats


_CORNERS = np.array([[2 * (c & 1) - 1, 2 * ((c >> 1) & 1) - 1, 2 * ((c >> 2) & 1) - 1] for c in range(8)])


def _corner_index(s):
    return int((s[0] > 0) + 2 * (s[1] > 0) + 4 * (s[2] > 0))


def _face_corners(f):
    ax, side = f // 2, f % 2
    return frozenset(c for c in range(8) if ((c >> ax) & 1) == side)


def scramble_orientation(elements: np.ndarray, faces_lists, seed: int):
    """Re-list every element in a randomly rotated local frame (same physical
    element, positive Jacobian kept) and renumber the local faces of the given
    (element, face) lists to match."""
    rng = np.random.default_rng(seed)
    rots = _cube_rotations()
    out = elements.copy()
    # per element: new position c -> old position perm[c]
    perms = []
    for e in range(elements.shape[0]):
        R = rots[rng.integers(len(rots))]
        perm = [_corner_index(R @ _CORNERS[c]) for c in range(8)]
        out[e] = elements[e, perm]
        perms.append(perm)
    new_lists = []
    for fl in faces_lists:
        fl = np.asarray(fl).copy()
        for r in range(fl.shape[0]):
            e, f = int(fl[r, 0]), int(fl[r, 1])
            old = _face_corners(f)
            perm = perms[e]
            for g in range(6):
                if frozenset(perm[c] for c in _face_corners(g)) == old:
                    fl[r, 1] = g
                    break
        new_lists.append(fl)
    return out, new_lists


def _lattice_elements(nx, ny, nz, offset=0):
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    el = np.zeros((i.size, 8), dtype=np.int64)
    for c in range(8):
        el[:, c] = offset + ((k + ((c >> 2) & 1)) * (ny + 1) + (j + ((c >> 1) & 1))) * (nx + 1) + (i + (c & 1))
    return el


def _eid(i, j, k, nx, ny):
    return (k * ny + j) * nx + i


def _lattice_points(origin, extent, n):
    xs = [origin[d] + extent[d] * np.arange(n[d] + 1) / n[d] for d in range(3)]
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def _displace(P, lo, hi, h, amp, phase, z_fixed_lo=True, z_fixed_hi=True):
    """Smooth displacement that is tangential on every wall of [lo, hi]:
    the d-component vanishes on the two walls normal to d."""
    P = P.copy()
    U = (P - lo) / (hi - lo)                       # unit cube coordinates
    d = np.zeros_like(P)
    d[:, 0] = amp * h[0] * np.sin(math.pi * U[:, 0]) * np.cos(2 * math.pi * U[:, 1] + phase[0]) \
        * np.cos(math.pi * U[:, 2] + phase[1])
    d[:, 1] = amp * h[1] * np.sin(math.pi * U[:, 1]) * np.cos(2 * math.pi * U[:, 2] + phase[2]) \
        * np.cos(math.pi * U[:, 0] + phase[3])
    d[:, 2] = amp * h[2] * np.sin(math.pi * U[:, 2]) * np.cos(2 * math.pi * U[:, 0] + phase[4]) \
        * np.cos(math.pi * U[:, 1] + phase[5])
    return P + d


def distorted_box(nel=(3, 3, 3), order=4, h=75e-6, amp=0.15, seed=21) -> HexDomain:
    """One box [0, nel h] of hexahedra with smoothly displaced vertices."""
    rng = np.random.default_rng(seed)
    ext = tuple(n * h for n in nel)
    P = _lattice_points((0.0, 0.0, 0.0), ext, nel)
    P = _displace(P, np.zeros(3), np.array(ext), np.full(3, h), amp, rng.uniform(0, 2 * math.pi, 6))
    return HexDomain(P, _lattice_elements(*nel), order, lattice=tuple(nel))


def distorted_two_domain(nx_p=4, nz_p=2, nx_s=2, nz_s=3, h_p=25e-6, order_p=4, order_s=6,
                         amp=0.12, bump=0.25, seed=31, n_pmut_side=2, n_modes=5, nsteps=200,
                         batch=1, n_recv=12, penalty_alpha=0.5, scramble: Optional[int] = None,
                         steer=False, ny_p=None, ny_s=None) -> HexWorkload:
    """Fine primary box (nx_p x ny_p x nz_p, order_p) under a coarse secondary
    box (nx_s x ny_s x nz_s, order_s), both distorted.  With twice the lateral
    element count on the fine side the interface is bent into a bump of height
    bump * h_p and the fine interface vertices lie on the coarse faces'
    bilinear patches (a nested 2:1 interface).  With any other ratio the
    interface is the flat plane z = nz_p h_p (bump must be 0) and each side
    keeps its own in-plane vertex displacement: the fine and coarse faces tile
    the plane independently (an unstructured non-conforming interface).  PMUT
    membranes sit on the flat z = 0 face.  `scramble` re-lists every element in
    a random rotated local frame (seeded)."""
    rng = np.random.default_rng(seed)
    ny_p = nx_p if ny_p is None else ny_p
    ny_s = nx_s if ny_s is None else ny_s
    nested = nx_p == 2 * nx_s and ny_p == 2 * ny_s
    assert nested or bump == 0.0, "a non-nested interface is kept flat (bump = 0)"
    Lx, Ly = nx_p * h_p, ny_p * h_p
    Lz_p = nz_p * h_p
    hs = Lx / nx_s
    assert abs(Ly / ny_s - hs) < 1e-12 * hs or not nested
    Lz_s = nz_s * hs
    zI = Lz_p
    ph = rng.uniform(0, 2 * math.pi, 12)

    def bump_z(x, y):
        return bump * h_p * np.sin(math.pi * x / Lx) * np.sin(math.pi * y / Ly)

    # secondary (coarse): lattice over [0, Lx] x [0, Ly] x [zI, zI + Lz_s]
    Ps = _lattice_points((0.0, 0.0, zI), (Lx, Ly, Lz_s), (nx_s, ny_s, nz_s))
    lo_s, hi_s = np.array([0.0, 0.0, zI]), np.array([Lx, Ly, zI + Lz_s])
    Ps = _displace(Ps, lo_s, hi_s, np.array([hs, hs, hs]), amp, ph[:6])
    # bend the bottom (interface) layer and blend the bend out towards the top
    base = _lattice_points((0.0, 0.0, zI), (Lx, Ly, Lz_s), (nx_s, ny_s, nz_s))
    wz = 1.0 - (base[:, 2] - zI) / Lz_s
    Ps[:, 2] += wz * bump_z(base[:, 0], base[:, 1])
    # primary (fine)
    Pp = _lattice_points((0.0, 0.0, 0.0), (Lx, Ly, Lz_p), (nx_p, ny_p, nz_p))
    basep = Pp.copy()
    Pp = _displace(Pp, np.zeros(3), np.array([Lx, Ly, Lz_p]), np.full(3, h_p), amp, ph[6:])
    Pp[:, 2] += basep[:, 2] / Lz_p * bump_z(basep[:, 0], basep[:, 1])
    # interface vertices of the primary: on the coarse bilinear patches (nested case)
    vs = lambda i, j, k: (k * (ny_s + 1) + j) * (nx_s + 1) + i
    for j in range(ny_p + 1 if nested else 0):
        for i in range(nx_p + 1):
            I, u = min(i // 2, nx_s - 1), (i - 2 * min(i // 2, nx_s - 1)) / 2.0
            J, v = min(j // 2, ny_s - 1), (j - 2 * min(j // 2, ny_s - 1)) / 2.0
            C00, C10 = Ps[vs(I, J, 0)], Ps[vs(I + 1, J, 0)]
            C01, C11 = Ps[vs(I, J + 1, 0)], Ps[vs(I + 1, J + 1, 0)]
            P = (1 - u) * (1 - v) * C00 + u * (1 - v) * C10 + (1 - u) * v * C01 + u * v * C11
            Pp[(nz_p * (ny_p + 1) + j) * (nx_p + 1) + i] = P
    Ep = _lattice_elements(nx_p, ny_p, nz_p)
    Es = _lattice_elements(nx_s, ny_s, nz_s)
    fine = np.array([[_eid(i, j, nz_p - 1, nx_p, ny_p), 5] for j in range(ny_p) for i in range(nx_p)])
    coarse = np.array([[_eid(i, j, 0, nx_s, ny_s), 4] for j in range(ny_s) for i in range(nx_s)])
    pmutf = np.array([[_eid(i, j, 0, nx_p, ny_p), 4] for j in range(ny_p) for i in range(nx_p)])
    if scramble is not None:
        Ep, (fine, pmutf) = scramble_orientation(Ep, [fine, pmutf], scramble)
        Es, (coarse,) = scramble_orientation(Es, [coarse], scramble + 1)
    prim = HexDomain(Pp, Ep, order_p, lattice=(nx_p, ny_p, nz_p))
    sec = HexDomain(Ps, Es, order_s, lattice=(nx_s, ny_s, nz_s))
    pitch = Lx / n_pmut_side
    centers = _grid_centers(n_pmut_side, pitch)
    side = min(60e-6, 0.6 * pitch)
    pm = make_pmut_array(centers, side, MODE_FREQS_5[:n_modes], 0.01,
                         freq_scale=rng.uniform(0.97, 1.03, size=centers.shape[0]))
    rec = np.column_stack([rng.uniform(0.05, 0.95, n_recv) * Lx, rng.uniform(0.05, 0.95, n_recv) * Ly,
                           rng.uniform(0.02, 0.98, n_recv) * (Lz_p + Lz_s)])
    if steer:
        d, a, _ = steering_patterns(centers, batch, seed + 1)
    else:
        d, a = _uniform_drive(centers.shape[0], batch)
        a = a * rng.uniform(0.5, 1.5, size=a.shape)
    return HexWorkload("distorted_two_domain", [prim, sec], nsteps, rec, pm, batch=batch,
                       penalty_alpha=penalty_alpha, drive_delay=d, drive_amp=a,
                       fine_faces=fine, coarse_faces=coarse, pmut_faces=pmutf,
                       box_extent=(Lx, Ly, Lz_p + Lz_s))


def distorted_one_domain(nel=(3, 3, 2), order=4, h=50e-6, amp=0.15, seed=41, nsteps=150, batch=1,
                         n_pmut_side=1, n_modes=3, n_recv=6, scramble: Optional[int] = None) -> HexWorkload:
    """One distorted box with PMUTs on its flat z = 0 face."""
    rng = np.random.default_rng(seed)
    dom = distorted_box(nel, order, h, amp, seed)
    ext = tuple(n * h for n in nel)
    pmutf = np.array([[_eid(i, j, 0, nel[0], nel[1]), 4] for j in range(nel[1]) for i in range(nel[0])])
    if scramble is not None:
        dom.elements, (pmutf,) = scramble_orientation(dom.elements, [pmutf], scramble)
    px, py = ext[0] / n_pmut_side, ext[1] / n_pmut_side
    c = np.arange(n_pmut_side) + 0.5
    X, Y = np.meshgrid(c * px, c * py, indexing="ij")
    centers = np.stack([X.ravel(), Y.ravel()], axis=1)
    side = min(60e-6, 0.6 * min(px, py))
    pm = make_pmut_array(centers, side, MODE_FREQS_5[:n_modes], 0.01)
    rec = np.column_stack([rng.uniform(0.05, 0.95, n_recv) * ext[0], rng.uniform(0.05, 0.95, n_recv) * ext[1],
                           rng.uniform(0.05, 0.95, n_recv) * ext[2]])
    d, a = _uniform_drive(centers.shape[0], batch)
    a = a * rng.uniform(0.5, 1.5, size=a.shape)
    return HexWorkload("distorted_one_domain", [dom], nsteps, rec, pm, batch=batch, drive_delay=d, drive_amp=a,
                       pmut_faces=pmutf, box_extent=ext)


def lattice_side_faces(lattice, side: int) -> np.ndarray:
    """(element, local face) of every element face on one side of a
    structured lattice (x-, x+, y-, y+, z-, z+ = 0..5), elements in lattice
    order, before any re-listing of element frames."""
    nx, ny, nz = lattice
    ax, hi = side // 2, side % 2
    out = []
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                ijk = (i, j, k)
                if ijk[ax] == (lattice[ax] - 1 if hi else 0):
                    out.append([_eid(i, j, k, nx, ny), side])
    return np.array(out, dtype=np.int64).reshape(-1, 2)


def hex_from_box(domain, offset_vertices=0) -> HexDomain:
    """The lattice hexahedra of an axis-aligned box domain as a general mesh
    (no displacement): the affine special case."""
    n = tuple(int(v) for v in domain.nelem)
    P = _lattice_points(domain.origin, domain.extent, n)
    return HexDomain(P, _lattice_elements(*n), int(domain.order), domain.c, domain.rho, lattice=n)


def hex_workload_from_box(w: Workload) -> HexWorkload:
    """A box workload (one box, or a primary/secondary pair stacked with a
    2:1 interface) restated as general hexahedra."""
    doms = [hex_from_box(d) for d in w.domains]
    p = w.domains[0]
    nx, ny, nz = (int(v) for v in p.nelem)
    pmutf = np.array([[_eid(i, j, 0, nx, ny), 4] for j in range(ny) for i in range(nx)])
    fine = coarse = None
    if len(doms) == 2:
        s = w.domains[1]
        sx, sy, _ = (int(v) for v in s.nelem)
        fine = np.array([[_eid(i, j, nz - 1, nx, ny), 5] for j in range(ny) for i in range(nx)])
        coarse = np.array([[_eid(i, j, 0, sx, sy), 4] for j in range(sy) for i in range(sx)])
    top = max(d.origin[2] + d.extent[2] for d in w.domains)
    return HexWorkload(w.name + "_hex", doms, w.nsteps, w.receivers, w.pmuts, cfl=w.cfl,
                       penalty_alpha=w.penalty_alpha, quad_pts=w.quad_pts, batch=w.batch,
                       drive_delay=w.drive_delay, drive_amp=w.drive_amp, burst_freq=w.burst_freq,
                       burst_cycles=w.burst_cycles, fine_faces=fine, coarse_faces=coarse, pmut_faces=pmutf,
                       box_extent=(p.extent[0], p.extent[1], top))


def hex_c2_like(nsteps=400, batch=1, amp=0.1, bump=0.3, seed=51, steer=True) -> HexWorkload:
    """A distorted version of the 16x16-PMUT mesh class: fine primary 64 x 64 x
    16 (h = 25 um, N = 4) under a coarse secondary 32 x 32 x 64 (N = 6) with a
    bent interface; 16 x 16 PMUTs at 100 um pitch; 64 receivers."""
    w = distorted_two_domain(nx_p=64, nz_p=16, nx_s=32, nz_s=64, h_p=25e-6, amp=amp, bump=bump, seed=seed,
                             n_pmut_side=16, n_modes=5, nsteps=nsteps, batch=batch, n_recv=64, steer=steer)
    w.name = "hex_c2_like"
    return w


def hex_c3_like(nsteps=400, batch=64, amp=0.1, bump=0.3, seed=61) -> HexWorkload:
    """The 1024-PMUT mesh class as distorted hexahedra: fine primary 128 x 128 x
    16 (h = 25 um, N = 4) under a coarse secondary 64 x 64 x 96 (N = 6) with a
    bent interface, 32 x 32 PMUTs at 100 um pitch, 64 receivers, beam-steering
    drive patterns."""
    w = distorted_two_domain(nx_p=128, nz_p=16, nx_s=64, nz_s=96, h_p=25e-6, amp=amp, bump=bump, seed=seed,
                             n_pmut_side=32, n_modes=5, nsteps=nsteps, batch=batch, n_recv=64, steer=True)
    w.name = "hex_c3_like"
    return w
