"""Thin ctypes binding of the general-hexahedron entry points of libdgsem.so
(include/dghex.h).

Argument marshalling only: every step runs in the CUDA kernels of the shared
library; importing raises if the library has not been built (no CPU
fallback).
"""
from __future__ import annotations

import ctypes
from ctypes import POINTER, byref, c_double, c_int, c_longlong, c_size_t, c_void_p

import numpy as np

from . import dgsem as _dg
from .dgsem import DGSEM_FP32_MIXED, DGSEM_FP64, DgsemError, _current_stream, _f64, _ptr  # noqa: F401

EXPORTED = [
    "dghex_mesh_create", "dghex_get_dt", "dghex_nodes", "dghex_pmut_nodes", "dghex_pmut_set", "dghex_get_matches",
    "dghex_set_absorbing_faces", "dghex_set_pml", "dghex_pmut_set_receive", "dghex_get_voltages", "dghex_state_save",
    "dghex_state_load",
    "dghex_run", "dghex_set_state", "dghex_get_pressure", "dghex_energy", "dghex_check_stability",
    "dghex_set_interface_kernel", "dghex_num_volume_variants", "dghex_set_volume_variant", "dghex_autotune",
    "dghex_profile",
    "dghex_kernel_stats", "dghex_destroy",
]
DGHEX_K_PMUT, DGHEX_K_VOL, DGHEX_K_IFACE, DGHEX_K_UPDATE, DGHEX_K_TAIL, DGHEX_K_PML = 0, 1, 2, 3, 4, 5


class HexDomainDesc(ctypes.Structure):
    _fields_ = [("order", c_int), ("c", c_double), ("rho", c_double), ("n_vert", c_int), ("vert", POINTER(c_double)),
                ("n_elem", c_int), ("elem", POINTER(c_int))]


class HexMeshDesc(ctypes.Structure):
    _fields_ = [("ndomains", c_int), ("domains", POINTER(HexDomainDesc)),
                ("n_fine_faces", c_int), ("fine_faces", POINTER(c_int)),
                ("n_coarse_faces", c_int), ("coarse_faces", POINTER(c_int)),
                ("n_pmut_faces", c_int), ("pmut_faces", POINTER(c_int)),
                ("cfl", c_double), ("dt", c_double), ("penalty_alpha", c_double),
                ("iface_quad_pts", c_int), ("normal_tol", c_double)]


_lib = None


def load_library():
    global _lib
    if _lib is not None:
        return _lib
    lib = _dg.load_library()
    vp = c_void_p
    lib.dghex_mesh_create.argtypes = [POINTER(HexMeshDesc), POINTER(vp)]
    lib.dghex_get_dt.argtypes = [vp, POINTER(c_double), POINTER(c_longlong)]
    lib.dghex_nodes.argtypes = [vp, POINTER(c_longlong), POINTER(c_longlong), POINTER(POINTER(c_double))]
    lib.dghex_pmut_nodes.argtypes = [vp, POINTER(c_int), POINTER(POINTER(c_double)), POINTER(POINTER(c_double))]
    lib.dghex_pmut_set.argtypes = [vp, c_int, c_int, vp, vp, vp, vp, vp, vp, vp]
    lib.dghex_get_matches.argtypes = [vp, POINTER(c_int), vp, vp, c_longlong]
    lib.dghex_run.argtypes = [vp, c_int, c_int, c_int, vp, c_int, vp, vp, c_int, vp]
    lib.dghex_set_state.argtypes = [vp, vp, vp]
    lib.dghex_get_pressure.argtypes = [vp, vp, c_size_t]
    lib.dghex_check_stability.argtypes = [vp, c_int, POINTER(c_double)]
    lib.dghex_energy.argtypes = [vp, vp, c_int]
    lib.dghex_set_absorbing_faces.argtypes = [vp, c_int, c_int, vp]
    lib.dghex_set_pml.argtypes = [vp, c_int, vp, c_double]
    lib.dghex_pmut_set_receive.argtypes = [vp, c_longlong, vp, c_int]
    lib.dghex_get_voltages.argtypes = [vp, vp, c_size_t]
    lib.dghex_state_save.argtypes = [vp, vp, POINTER(c_size_t)]
    lib.dghex_state_load.argtypes = [vp, vp, c_size_t]
    lib.dghex_set_interface_kernel.argtypes = [vp, c_int]
    lib.dghex_num_volume_variants.argtypes = [vp, POINTER(c_int)]
    lib.dghex_set_volume_variant.argtypes = [vp, c_int, vp]
    lib.dghex_autotune.argtypes = [vp, c_int, c_int, c_int, vp, vp]
    lib.dghex_profile.argtypes = [vp, c_int]
    lib.dghex_kernel_stats.argtypes = [vp, c_int, POINTER(c_double), POINTER(c_longlong)]
    lib.dghex_destroy.argtypes = [vp]
    lib.dghex_destroy.restype = None
    for name in EXPORTED:
        if name != "dghex_destroy":
            getattr(lib, name).restype = c_int
    _lib = lib
    return lib


def _check(code: int, where: str):
    if code != 0:
        raise DgsemError(code, where, _lib.dgsem_last_error().decode())


def _faces(desc, name, faces, keep):
    if faces is None:
        return
    f = np.ascontiguousarray(faces, dtype=np.int32).reshape(-1, 2)
    keep.append(f)
    setattr(desc, "n_" + name, f.shape[0])
    setattr(desc, name, f.ctypes.data_as(POINTER(c_int)))


def dghex_mesh_create(domains, fine_faces=None, coarse_faces=None, pmut_faces=None, cfl: float = 0.3,
                      dt: float = 0.0, penalty_alpha: float = 0.5, iface_quad_pts: int = 0,
                      normal_tol: float = 0.5) -> c_void_p:
    """domains: objects with vertices [nv, 3], elements [ne, 8], order, c, rho."""
    lib = load_library()
    keep = []
    arr = (HexDomainDesc * len(domains))()
    for i, d in enumerate(domains):
        v = np.ascontiguousarray(d.vertices, dtype=np.float64).reshape(-1, 3)
        e = np.ascontiguousarray(d.elements, dtype=np.int32).reshape(-1, 8)
        keep += [v, e]
        arr[i].order = int(d.order)
        arr[i].c = float(d.c)
        arr[i].rho = float(d.rho)
        arr[i].n_vert = v.shape[0]
        arr[i].vert = v.ctypes.data_as(POINTER(c_double))
        arr[i].n_elem = e.shape[0]
        arr[i].elem = e.ctypes.data_as(POINTER(c_int))
    desc = HexMeshDesc()
    desc.ndomains = len(domains)
    desc.domains = arr
    _faces(desc, "fine_faces", fine_faces, keep)
    _faces(desc, "coarse_faces", coarse_faces, keep)
    _faces(desc, "pmut_faces", pmut_faces, keep)
    desc.cfl, desc.dt, desc.penalty_alpha = cfl, dt, penalty_alpha
    desc.iface_quad_pts, desc.normal_tol = iface_quad_pts, normal_tol
    ctx = c_void_p()
    _check(lib.dghex_mesh_create(byref(desc), byref(ctx)), "dghex_mesh_create")
    return ctx


def dghex_get_dt(ctx):
    dt, nd = c_double(), c_longlong()
    _check(_lib.dghex_get_dt(ctx, byref(dt), byref(nd)), "dghex_get_dt")
    return dt.value, nd.value


def dghex_nodes(ctx):
    """(positions [ndof, 3], first node of domain 1)."""
    n, f = c_longlong(), c_longlong()
    p = POINTER(c_double)()
    _check(_lib.dghex_nodes(ctx, byref(n), byref(f), byref(p)), "dghex_nodes")
    return np.ctypeslib.as_array(p, shape=(n.value, 3)).copy(), f.value


def dghex_pmut_nodes(ctx):
    """(positions [n, 3], face weights [n]) of the Gamma_PMUT nodes."""
    n = c_int()
    x = POINTER(c_double)()
    w = POINTER(c_double)()
    _check(_lib.dghex_pmut_nodes(ctx, byref(n), byref(x), byref(w)), "dghex_pmut_nodes")
    if n.value == 0:
        return np.zeros((0, 3)), np.zeros(0)
    return np.ctypeslib.as_array(x, shape=(n.value, 3)).copy(), np.ctypeslib.as_array(w, shape=(n.value,)).copy()


def dghex_pmut_set(ctx, foot_ptr, foot_node, shape_un, freq_hz, damping, eta, modal_mass=None):
    foot_ptr = np.ascontiguousarray(foot_ptr, dtype=np.int32)
    foot_node = np.ascontiguousarray(foot_node, dtype=np.int32)
    freq_hz = np.ascontiguousarray(freq_hz, dtype=np.float64)
    K, M = freq_hz.shape
    shape_un = np.ascontiguousarray(shape_un, dtype=np.float64).reshape(-1, M)
    damping = np.ascontiguousarray(damping, dtype=np.float64)
    eta = np.ascontiguousarray(eta, dtype=np.float64)
    mm = None if modal_mass is None else np.ascontiguousarray(modal_mass, dtype=np.float64)
    _check(_lib.dghex_pmut_set(ctx, K, M, _ptr(foot_ptr), _ptr(foot_node), _ptr(shape_un), _ptr(freq_hz),
                               _ptr(damping), _ptr(eta), _ptr(mm)), "dghex_pmut_set")


def dghex_get_matches(ctx, n_fine_faces: int):
    """Algorithm 3 result: (q, coarse face per Gauss node [nff, q*q], reference
    position [nff, q*q, 3])."""
    q = c_int()
    _check(_lib.dghex_get_matches(ctx, byref(q), None, None, 0), "dghex_get_matches")
    n = n_fine_faces * q.value * q.value
    cf = np.zeros(n, dtype=np.int32)
    ref = np.zeros((n, 3))
    _check(_lib.dghex_get_matches(ctx, byref(q), _ptr(cf), _ptr(ref), n), "dghex_get_matches")
    return q.value, cf.reshape(n_fine_faces, -1), ref.reshape(n_fine_faces, -1, 3)


def dghex_run(ctx, precision: int, batch: int, nsteps: int, drive, recv_xyz, traces=None, flags: int = 0,
              stream=None):
    recv = np.ascontiguousarray(recv_xyz, dtype=np.float64).reshape(-1, 3)
    R = recv.shape[0]
    if traces is None:
        traces = np.zeros((batch, R, nsteps))
    drive = _f64(drive)
    if stream is None:
        stream = _current_stream()
    _check(_lib.dghex_run(ctx, precision, batch, nsteps, _ptr(drive), R, _ptr(recv), _ptr(traces), flags, stream),
           "dghex_run")
    return traces


def dghex_set_state(ctx, p0=None, v0=None):
    p0 = None if p0 is None else np.ascontiguousarray(p0, dtype=np.float64)
    v0 = None if v0 is None else np.ascontiguousarray(v0, dtype=np.float64)
    _check(_lib.dghex_set_state(ctx, _ptr(p0), _ptr(v0)), "dghex_set_state")


def dghex_get_pressure(ctx, batch: int, ndof: int) -> np.ndarray:
    out = np.zeros((batch, ndof))
    _check(_lib.dghex_get_pressure(ctx, _ptr(out), out.size), "dghex_get_pressure")
    return out


def dghex_set_absorbing_faces(ctx, domain: int, faces):
    """First-order absorbing faces ([n, 2] (element, local face)) of a domain."""
    f = np.ascontiguousarray(faces if faces is not None else np.zeros((0, 2)), dtype=np.int32).reshape(-1, 2)
    _check(_lib.dghex_set_absorbing_faces(ctx, domain, f.shape[0], _ptr(f) if f.size else None),
           "dghex_set_absorbing_faces")


def dghex_set_pml(ctx, domain: int, thickness, R: float = 1e-4):
    """Perfectly matched layers of the given thickness (m) along the sides
    x-, x+, y-, y+, z-, z+ of a domain's bounding box, design reflection R."""
    th = np.ascontiguousarray(thickness, dtype=np.float64)
    assert th.shape == (6,)
    _check(_lib.dghex_set_pml(ctx, domain, _ptr(th), float(R)), "dghex_set_pml")


def dghex_pmut_set_receive(ctx, n_switch: int, capacitance=None, sign: int = -1):
    cap = None if capacitance is None else np.ascontiguousarray(capacitance, dtype=np.float64)
    _check(_lib.dghex_pmut_set_receive(ctx, int(n_switch), _ptr(cap), int(sign)), "dghex_pmut_set_receive")


def dghex_get_voltages(ctx, batch: int, n_pmut: int, nsteps: int):
    out = np.zeros((batch, n_pmut, nsteps))
    _check(_lib.dghex_get_voltages(ctx, _ptr(out), out.size), "dghex_get_voltages")
    return out


def dghex_state_save(ctx) -> bytes:
    n = c_size_t(0)
    _check(_lib.dghex_state_save(ctx, None, byref(n)), "dghex_state_save")
    buf = ctypes.create_string_buffer(n.value)
    _check(_lib.dghex_state_save(ctx, buf, byref(n)), "dghex_state_save")
    return buf.raw[: n.value]


def dghex_state_load(ctx, blob: bytes):
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(_lib.dghex_state_load(ctx, buf, len(blob)), "dghex_state_load")


def dghex_energy(ctx, batch: int) -> np.ndarray:
    """Leapfrog energy 1/2 v.M v + 1/2 p^n.K p^{n+1} of each batch member (FP64 state)."""
    out = np.zeros(batch)
    _check(_lib.dghex_energy(ctx, _ptr(out), batch), "dghex_energy")
    return out


def dghex_check_stability(ctx, iters: int = 100):
    """(status, lambda_max of M^-1 K): status DGSEM_EUNSTABLE when dt is above
    0.95 * 2 / sqrt(lambda_max)."""
    lam = c_double()
    code = _lib.dghex_check_stability(ctx, iters, byref(lam))
    return code, lam.value


def dghex_set_interface_kernel(ctx, general: bool):
    """Force the full-evaluation interface kernel (True) or restore the
    automatic choice (False)."""
    _check(_lib.dghex_set_interface_kernel(ctx, 1 if general else 0), "dghex_set_interface_kernel")


def dghex_num_volume_variants(ctx) -> int:
    n = c_int()
    _check(_lib.dghex_num_volume_variants(ctx, byref(n)), "dghex_num_volume_variants")
    return n.value


def dghex_set_volume_variant(ctx, precision: int, variants):
    """Element-stiffness launch variant per domain for later runs at `precision`."""
    v = np.ascontiguousarray(variants, dtype=np.int32)
    _check(_lib.dghex_set_volume_variant(ctx, precision, _ptr(v)), "dghex_set_volume_variant")


def dghex_autotune(ctx, precision: int, batch: int, ndomains: int, reps: int = 3, stream=None):
    """Time every element-stiffness variant of each domain for `batch`
    patterns and keep the fastest; returns the chosen variant per domain."""
    out = np.zeros(ndomains, dtype=np.int32)
    if stream is None:
        stream = _current_stream()
    _check(_lib.dghex_autotune(ctx, precision, batch, reps, _ptr(out), stream), "dghex_autotune")
    return [int(x) for x in out]


def dghex_profile(ctx, enable: bool = True):
    _check(_lib.dghex_profile(ctx, 1 if enable else 0), "dghex_profile")


def dghex_kernel_stats(ctx, kind: int):
    ms, n = c_double(), c_longlong()
    _check(_lib.dghex_kernel_stats(ctx, kind, byref(ms), byref(n)), "dghex_kernel_stats")
    return ms.value, n.value


def dghex_destroy(ctx):
    if ctx is not None and _lib is not None:
        _lib.dghex_destroy(ctx)


class HexSolver:
    """Owns one general-hexahedron context built from a HexWorkload-like
    description (domains with vertices/elements/order/c/rho, fine_faces,
    coarse_faces, pmut_faces, cfl, penalty_alpha, quad_pts, normal_tol, pmuts)."""

    def __init__(self, workload, dt: float = 0.0):
        self.w = workload
        self.ctx = dghex_mesh_create(workload.domains, workload.fine_faces, workload.coarse_faces,
                                     workload.pmut_faces, cfl=workload.cfl, dt=dt,
                                     penalty_alpha=workload.penalty_alpha,
                                     iface_quad_pts=getattr(workload, "quad_pts", 0) or 0,
                                     normal_tol=getattr(workload, "normal_tol", 0.5))
        for d, faces in enumerate(getattr(workload, "absorbing_faces", None) or []):
            if faces is not None and len(faces):
                dghex_set_absorbing_faces(self.ctx, d, faces)
        for d, th in enumerate(getattr(workload, "pml", None) or []):
            if th is not None and any(t > 0 for t in th):
                dghex_set_pml(self.ctx, d, th, getattr(workload, "pml_R", 1e-4))
        self.dt, self.ndof = dghex_get_dt(self.ctx)
        self.K = 0
        if workload.pmuts is not None and workload.pmut_faces is not None:
            self.set_pmuts(workload.pmuts)
            if getattr(workload, "rx_switch", None) is not None:
                cap = np.broadcast_to(np.asarray(workload.rx_capacitance, dtype=np.float64), (self.K,))
                dghex_pmut_set_receive(self.ctx, workload.rx_switch, cap, workload.rx_sign)

    def set_pmuts(self, pm):
        xyz, _ = dghex_pmut_nodes(self.ctx)
        ptr = [0]
        nodes, vals = [], []
        for k in range(pm.n_pmut):
            idx = np.nonzero(pm.inside(k, xyz[:, 0], xyz[:, 1]))[0]
            nodes.append(idx)
            vals.append(np.stack([pm.shape_un(k, m, xyz[idx, 0], xyz[idx, 1]) for m in range(pm.n_modes)], axis=1))
            ptr.append(ptr[-1] + idx.size)
        dghex_pmut_set(self.ctx, np.array(ptr), np.concatenate(nodes),
                       np.concatenate(vals) if vals else np.zeros((0, pm.n_modes)),
                       pm.freq_hz, pm.damping, pm.eta, pm.modal_mass)
        self.K = pm.n_pmut

    def run(self, drive=None, precision=DGSEM_FP64, batch=None, nsteps=None, receivers=None, traces=None,
            flags=0, stream=None):
        B = self.w.batch if batch is None else batch
        S = self.w.nsteps if nsteps is None else nsteps
        rec = self.w.receivers if receivers is None else receivers
        if drive is None and self.K > 0:
            drive = self.w.drive(self.dt, S, B)
        return dghex_run(self.ctx, precision, B, S, drive, rec, traces=traces, flags=flags, stream=stream)

    def close(self):
        dghex_destroy(self.ctx)
        self.ctx = None

    def __del__(self):
        try:
            if self.ctx is not None:
                self.close()
        except Exception:
            pass
