"""Parity at full size, in the benchmark's launch configuration, on sampled
outputs the oracle computes locally.

The batched config-4 mesh (128x128x16 N=4 primary under 64x64x96 N=6
secondary, 102,631,810 nodes) is run for S = 3 steps with 64 patterns in FP32
(the benchmark's configuration: automatic launch shape, so every CTA marches
through all 16 / 96 layers of its box; every tile variant) and with 8 patterns
in FP64.  An explicit step couples a node only to the nodes of its elements,
and a PMUT to the nodes of its footprint, so after S steps the value at a
point depends only on a neighbourhood a few elements wide.  The oracle runs
each of five sub-boxes (crops) of the mesh as its own problem -- rigid walls
where the crop cuts the mesh -- and its receivers at points more than S elements away from those cut walls
(and from PMUT footprints they cut) equal the full problem's.  The GPU run's receivers are those points.

Two linearly independent runs cover the path: (A) a smooth seeded initial
state p0, p'0 (set_state, the same for every pattern) with zero drive --
volume stencils in both boxes, the interface, the far walls, the ragged
last tile rows and the box's last x node; (B) rest with a seeded random drive
per pattern and PMUT -- the PMUT rows of Algorithm 1 near both ends of the
array, each pattern against its own oracle column.
"""
import numpy as np
import pytest

import workloads as W
from oracle import dgsem_oracle as O
from gpu_helpers import rel_l2

pytestmark = pytest.mark.gpu

S = 3
FP64_TOL = 1e-10
FP32_TOL = 1e-4
HP, HS = 25e-6, 50e-6          # element sizes of the primary and secondary boxes
ZP = 0.4e-3                    # interface height

# crops: element ranges [lo, hi) per axis of the primary and/or secondary box,
# and the box (in metres) in which sample points are drawn.  A cut wall changes
# the rows of its own nodes; after S steps the difference has spread S - 1
# elements inward (a PMUT footprint cut by it would carry it across the
# footprint one step later), so every sample box keeps more than S elements
# from every cut wall.
CROPS = {
    "pmut_corner": dict(prim=((0, 8), (0, 8), (0, 8)), sec=None,
                        valid=((0.0, 2 * HP), (0.0, 2 * HP), (0.0, 3 * HP))),
    "pmut_far": dict(prim=((120, 128), (120, 128), (0, 8)), sec=None,
                     valid=((126 * HP, 128 * HP), (126 * HP, 128 * HP), (0.0, 3 * HP))),
    "interface": dict(prim=((40, 56), (40, 56), (8, 16)), sec=((20, 28), (20, 28), (0, 6)),
                      valid=((46 * HP, 50 * HP), (46 * HP, 50 * HP), (13 * HP, ZP + 1.5 * HS))),
    "sec_far_top": dict(prim=None, sec=((56, 64), (56, 64), (88, 96)),
                        valid=((61 * HS, 64 * HS), (61 * HS, 64 * HS), (ZP + 93 * HS, ZP + 96 * HS))),
    "sec_mid": dict(prim=None, sec=((28, 36), (28, 36), (44, 52)),
                    valid=((31 * HS, 33 * HS), (31 * HS, 33 * HS), (ZP + 47 * HS, ZP + 49 * HS))),
}
PMUT_CROPS = ("pmut_corner", "pmut_far")
NPTS = 10


def _points():
    rng = np.random.default_rng(2024)
    pts = {}
    for name, c in CROPS.items():
        v = np.array(c["valid"])
        pts[name] = v[:, 0] + rng.uniform(0.0, 1.0, size=(NPTS, 3)) * (v[:, 1] - v[:, 0])
    return pts


def _field_terms(seed):
    """The terms of W.seeded_field (a sum of separable cosine products)."""
    rng = np.random.default_rng(seed)
    terms = []
    for _ in range(4):
        k = rng.uniform(500.0, 20000.0, size=3)
        ph = rng.uniform(0, 2 * np.pi, size=3)
        a = rng.normal()
        terms.append((k, ph, a))
    return terms


def _full_field(w, seed, scale):
    """W.seeded_field at every node of the full mesh, evaluated per box as
    outer products of the 1-D coordinate lines (node order of dgsem_set_state)."""
    out = []
    off = 0
    for dom in w.domains:
        m = O.BoxMesh(dom, off)
        off += m.nnode
        f = np.zeros((m.L[2], m.L[1], m.L[0]))
        for k, ph, a in _field_terms(seed):
            cx = np.cos(k[0] * m.coord[0] + ph[0])
            cy = np.cos(k[1] * m.coord[1] + ph[1])
            cz = np.cos(k[2] * m.coord[2] + ph[2])
            f += a * cz[:, None, None] * (cy[:, None] * cx[None, :])[None, :, :]
        out.append(scale * f.ravel())
    return np.concatenate(out)


def _crop_workload(full, name, pts):
    c = CROPS[name]
    doms = []
    for key, dom, h in (("prim", full.domains[0], HP), ("sec", full.domains[1], HS)):
        rng_ = c[key]
        if rng_ is None:
            continue
        o = tuple(dom.origin[d] + rng_[d][0] * h for d in range(3))
        e = tuple((rng_[d][1] - rng_[d][0]) * h for d in range(3))
        n = tuple(rng_[d][1] - rng_[d][0] for d in range(3))
        doms.append(W.Domain(o, e, n, dom.order))
    pm, keep = None, np.zeros(0, dtype=int)
    if name in PMUT_CROPS:
        lo = np.array(doms[0].origin[:2])
        hi = lo + np.array(doms[0].extent[:2])
        cen = full.pmuts.centers
        keep = np.nonzero(np.all((cen > lo) & (cen < hi), axis=1))[0]
        p = full.pmuts
        pm = W.PmutArray(centers=cen[keep].copy(), side=p.side, freq_hz=p.freq_hz[keep].copy(),
                         damping=p.damping[keep].copy(), eta=p.eta[keep].copy(),
                         modal_mass=p.modal_mass[keep].copy())
    wc = W.Workload(name, doms, S, pts, pm, penalty_alpha=full.penalty_alpha)
    return wc, keep


@pytest.fixture(scope="module")
def setup():
    full = W.config4_batched(nsteps=S, batch=64)
    pts = _points()
    allpts = np.concatenate([pts[n] for n in CROPS])
    p0 = _full_field(full, 31, 1.0)
    v0 = _full_field(full, 32, 1.0e6)
    rng = np.random.default_rng(33)
    drive = rng.normal(0.0, 10.0, size=(64, full.pmuts.n_pmut, S))
    return full, pts, allpts, p0, v0, drive


@pytest.fixture(scope="module")
def oracle_refs(setup):
    """Oracle traces per crop: run A (initial state, no drive; identical for
    every pattern, batch 1) and run B (rest, drive; 64 patterns).  The time
    step is the full mesh's (the two-box crop has both element kinds)."""
    full, pts, allpts, p0, v0, drive = setup
    crops = {name: _crop_workload(full, name, pts[name]) for name in CROPS}
    dt = O.OracleProblem(crops["interface"][0]).stable_dt()
    refA, refB = {}, {}
    for name, (wc, keep) in crops.items():
        P = O.OracleProblem(wc)
        X = P.all_coordinates()
        pa = W.seeded_field(31, *X)
        va = W.seeded_field(32, *X, scale=1.0e6)
        zero = np.zeros((1, len(keep), S)) if wc.pmuts is not None else None
        refA[name] = P.run(nsteps=S, dt=dt, drive=zero, p0=pa, v0=va, batch=1)[0]   # [R][S]
        if name in PMUT_CROPS:
            refB[name] = P.run(nsteps=S, dt=dt, drive=drive[:, keep, :], batch=64)    # [64][R][S]
    return dt, refA, refB


def _check(name, got, ref, tol):
    scale = np.abs(ref).max()
    assert scale > 0, name
    err = np.abs(got - ref).max() / scale
    assert err <= tol, (name, err)
    return err


def _gpu_runs(sol, setup, prec, batch):
    from paper_2603_06267_gb300 import dgsem
    full, pts, allpts, p0, v0, drive = setup
    zero = np.zeros((batch, full.pmuts.n_pmut, S))
    dgsem.dgsem_set_state(sol.ctx, p0, v0)
    trA = sol.run(drive=zero, precision=prec, batch=batch, nsteps=S, receivers=allpts)
    shapes = [dgsem.dgsem_vol_launch(sol.ctx, d) for d in range(2)]
    dgsem.dgsem_set_state(sol.ctx, None, None)
    trB = sol.run(drive=np.ascontiguousarray(drive[:batch]), precision=prec, batch=batch, nsteps=S,
                  receivers=allpts)
    return trA, trB, shapes


def _compare(setup, oracle_refs, prec, batch, trA, trB, tol):
    full, pts, allpts, p0, v0, drive = setup
    dt, refA, refB = oracle_refs
    errs = {}
    r0 = 0
    for name in CROPS:
        sl = slice(r0, r0 + NPTS)
        r0 += NPTS
        for b in range(batch):
            errs[("A", name)] = max(errs.get(("A", name), 0.0), _check(name, trA[b, sl], refA[name], tol))
        if name in PMUT_CROPS:
            for b in range(batch):
                errs[("B", name)] = max(errs.get(("B", name), 0.0), _check(name, trB[b, sl], refB[name][b], tol))
            # the patterns differ, so each is checked against its own column
            assert rel_l2(refB[name][0], refB[name][1]) > 1e-2
    return errs


def test_fullsize_fp32_64_patterns_every_tile_variant(setup, oracle_refs):
    from paper_2603_06267_gb300 import dgsem
    full = setup[0]
    sol = dgsem.Solver(full)
    assert abs(sol.dt - oracle_refs[0]) <= 1e-13 * sol.dt
    n = [dgsem.dgsem_num_tiles(sol.ctx, 1, d) for d in range(2)]
    for i in range(max(n)):
        tiles = (min(i, n[0] - 1), min(i, n[1] - 1))
        dgsem.dgsem_set_tiles(sol.ctx, 1, list(tiles))
        trA, trB, shapes = _gpu_runs(sol, setup, 1, 64)
        # the automatic shape at this size: every CTA takes every layer of its box
        for d in range(2):
            assert shapes[d]["layers_per_cta"] == full.domains[d].nelem[2] and shapes[d]["nchunks"] == 1
            assert shapes[d]["grid"][2] == 64
        errs = _compare(setup, oracle_refs, 1, 64, trA, trB, FP32_TOL)
        print(f"full size FP32, tiles {tiles}: max sampled error / scale per crop {errs}")
    sol.close()


def test_fullsize_fp64_8_patterns(setup, oracle_refs):
    from paper_2603_06267_gb300 import dgsem
    full = setup[0]
    sol = dgsem.Solver(full)
    trA, trB, shapes = _gpu_runs(sol, setup, 0, 8)
    for d in range(2):
        assert shapes[d]["layers_per_cta"] == full.domains[d].nelem[2]
    errs = _compare(setup, oracle_refs, 0, 8, trA, trB, FP64_TOL)
    print(f"full size FP64: max sampled error / scale per crop {errs}")
    sol.close()
