"""Thin ctypes binding of libdgsem.so (include/dgsem.h).

Argument marshalling only: every step of the time loop runs in the CUDA
kernels of the shared library.  Arrays may be numpy arrays (host) or torch
CUDA tensors (device pointers are passed through).  If the library has not
been built, importing the binding raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, byref, c_double, c_int, c_longlong, c_size_t, c_void_p
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdgsem.so")

DGSEM_OK = 0
DGSEM_EINVAL = -1
DGSEM_ENOMEM = -2
DGSEM_ECUDA = -3
DGSEM_EUNSTABLE = -4
DGSEM_ETIMEOUT = -5
DGSEM_ENOMATCH = -6
DGSEM_ESTATE = -7
DGSEM_FP64 = 0
DGSEM_FP32_MIXED = 1
DGSEM_RUN_CONTINUE = 1

EXPORTED = [
    "dgsem_mesh_create", "dgsem_set_absorbing", "dgsem_set_pml", "dgsem_selftest_wait", "dgsem_get_dt", "dgsem_check_stability", "dgsem_pmut_nodes", "pmut_array_set",
    "pmut_set_receive", "dgsem_get_voltages",
    "dgsem_run", "dgsem_run_multi", "dgsem_set_state", "dgsem_get_pressure", "dgsem_get_pmut_state", "dgsem_energy", "dgsem_state_save",
    "dgsem_state_load",
    "dgsem_num_tiles", "dgsem_set_tiles", "dgsem_autotune",
    "dgsem_set_layers", "dgsem_vol_launch", "dgsem_profile", "dgsem_kernel_stats", "dgsem_sample_noalloc", "dgsem_measure_peak", "dgsem_last_error",
    "dgsem_destroy",
]
DGSEM_K_PMUT_RECV, DGSEM_K_IFACE, DGSEM_K_VOL0, DGSEM_K_VOL1, DGSEM_K_PML = 0, 1, 2, 3, 4


class DgsemError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where} failed with status {code}: {msg}")
        self.code = code


class DomainDesc(ctypes.Structure):
    _fields_ = [("origin", c_double * 3), ("extent", c_double * 3), ("nelem", c_int * 3),
                ("order", c_int), ("c", c_double), ("rho", c_double)]


class MeshDesc(ctypes.Structure):
    _fields_ = [("ndomains", c_int), ("domains", POINTER(DomainDesc)),
                ("n_fine_faces", c_int), ("fine_faces", POINTER(c_int)),
                ("n_coarse_faces", c_int), ("coarse_faces", POINTER(c_int)),
                ("cfl", c_double), ("dt", c_double), ("penalty_alpha", c_double),
                ("iface_quad_pts", c_int)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libdgsem.so and declare the prototypes (raises if not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -m paper_2603_06267_gb300.build` "
                           "(the CUDA path has no CPU fallback)")
    lib = ctypes.CDLL(path)
    vp = c_void_p
    lib.dgsem_mesh_create.argtypes = [POINTER(MeshDesc), POINTER(vp)]
    lib.dgsem_get_dt.argtypes = [vp, POINTER(c_double), POINTER(c_double), POINTER(c_longlong)]
    lib.dgsem_set_absorbing.argtypes = [vp, c_int, vp]
    lib.dgsem_set_pml.argtypes = [vp, c_int, vp, c_double]
    lib.dgsem_selftest_wait.argtypes = [vp, vp]
    lib.pmut_set_receive.argtypes = [vp, c_longlong, vp, c_int]
    lib.dgsem_get_voltages.argtypes = [vp, vp, c_size_t]
    lib.dgsem_check_stability.argtypes = [vp, c_int, POINTER(c_double)]
    lib.dgsem_pmut_nodes.argtypes = [vp, POINTER(c_int), POINTER(POINTER(c_double))]
    lib.pmut_array_set.argtypes = [vp, c_int, c_int, vp, vp, vp, vp, vp, vp, vp]
    lib.dgsem_run.argtypes = [vp, c_int, c_int, c_int, vp, c_int, vp, vp, c_int, vp]
    lib.dgsem_run_multi.argtypes = [c_int, vp, c_int, vp, c_int, vp, vp, vp, vp, c_int, vp]
    lib.dgsem_set_state.argtypes = [vp, vp, vp]
    lib.dgsem_get_pressure.argtypes = [vp, vp, c_size_t]
    lib.dgsem_get_pmut_state.argtypes = [vp, vp, vp, vp, c_size_t]
    lib.dgsem_energy.argtypes = [vp, vp, c_int]
    lib.dgsem_state_save.argtypes = [vp, vp, POINTER(c_size_t)]
    lib.dgsem_state_load.argtypes = [vp, vp, c_size_t]
    lib.dgsem_num_tiles.argtypes = [vp, c_int, c_int, POINTER(c_int)]
    lib.dgsem_set_tiles.argtypes = [vp, c_int, vp]
    lib.dgsem_autotune.argtypes = [vp, c_int, c_int, c_int, vp, vp]
    lib.dgsem_set_layers.argtypes = [vp, vp]
    lib.dgsem_measure_peak.argtypes = [c_int, POINTER(c_double), vp]
    lib.dgsem_vol_launch.argtypes = [vp, c_int, vp]
    lib.dgsem_sample_noalloc.argtypes = [vp, c_int, vp, vp, c_size_t, vp]
    lib.dgsem_profile.argtypes = [vp, c_int]
    lib.dgsem_kernel_stats.argtypes = [vp, c_int, POINTER(c_double), POINTER(c_longlong)]
    lib.dgsem_last_error.restype = ctypes.c_char_p
    lib.dgsem_last_error.argtypes = []
    lib.dgsem_destroy.argtypes = [vp]
    lib.dgsem_destroy.restype = None
    for name in EXPORTED:
        if name not in ("dgsem_last_error", "dgsem_destroy"):
            getattr(lib, name).restype = c_int
    _lib = lib
    return lib


def _check(code: int, where: str):
    if code != DGSEM_OK:
        raise DgsemError(code, where, _lib.dgsem_last_error().decode())


def _ptr(a) -> Optional[int]:
    """Address of a contiguous numpy array or torch tensor (None passes NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"], "arrays must be C-contiguous"
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous(), "tensors must be contiguous"
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _f64(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        import torch
        assert a.dtype == torch.float64
        return a.contiguous()
    return np.ascontiguousarray(a, dtype=np.float64)


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:  # pragma: no cover
        pass
    return None


# ------------------------------------------------------------------ C names
def dgsem_mesh_create(domains: Sequence, cfl: float = 0.3, dt: float = 0.0, penalty_alpha: float = 0.5,
                      iface_quad_pts: int = 0, fine_faces=None, coarse_faces=None) -> c_void_p:
    """domains: objects with origin, extent, nelem, order, c, rho (primary first)."""
    lib = load_library()
    arr = (DomainDesc * len(domains))()
    for i, d in enumerate(domains):
        arr[i].origin = (c_double * 3)(*[float(v) for v in d.origin])
        arr[i].extent = (c_double * 3)(*[float(v) for v in d.extent])
        arr[i].nelem = (c_int * 3)(*[int(v) for v in d.nelem])
        arr[i].order = int(d.order)
        arr[i].c = float(d.c)
        arr[i].rho = float(d.rho)
    desc = MeshDesc()
    desc.ndomains = len(domains)
    desc.domains = arr
    keep = []
    if fine_faces is not None:
        ff = np.ascontiguousarray(fine_faces, dtype=np.int32)
        keep.append(ff)
        desc.n_fine_faces = ff.size
        desc.fine_faces = ff.ctypes.data_as(POINTER(c_int))
    if coarse_faces is not None:
        cf = np.ascontiguousarray(coarse_faces, dtype=np.int32)
        keep.append(cf)
        desc.n_coarse_faces = cf.size
        desc.coarse_faces = cf.ctypes.data_as(POINTER(c_int))
    desc.cfl = cfl
    desc.dt = dt
    desc.penalty_alpha = penalty_alpha
    desc.iface_quad_pts = iface_quad_pts
    ctx = c_void_p()
    _check(lib.dgsem_mesh_create(byref(desc), byref(ctx)), "dgsem_mesh_create")
    return ctx


def dgsem_set_absorbing(ctx, box: int, sides):
    """First-order absorbing box sides (x-, x+, y-, y+, z-, z+), eq. Wf_4."""
    arr = np.ascontiguousarray([1 if v else 0 for v in sides], dtype=np.int32)
    assert arr.shape == (6,)
    _check(_lib.dgsem_set_absorbing(ctx, box, _ptr(arr)), "dgsem_set_absorbing")


def dgsem_selftest_wait(ctx, stream=None):
    """Run the failure-path self test (a bounded device wait that must give up)."""
    if stream is None:
        stream = _current_stream()
    _check(_lib.dgsem_selftest_wait(ctx, stream), "dgsem_selftest_wait")


def dgsem_set_pml(ctx, box: int, thickness, R: float = 1e-4):
    """Perfectly matched layer of the given thickness (m) along the sides
    x-, x+, y-, y+, z-, z+ of a box (0 = none), design reflection R."""
    arr = np.ascontiguousarray(thickness, dtype=np.float64)
    assert arr.shape == (6,)
    _check(_lib.dgsem_set_pml(ctx, box, _ptr(arr), float(R)), "dgsem_set_pml")


def pmut_set_receive(ctx, n_switch: int, capacitance=None, sign: int = -1):
    """TX -> RX switch: from step n_switch on, phi_k = sign / C_k sum_m eta_km q_km
    (n_switch < 0: transmit only)."""
    cap = None if capacitance is None else np.ascontiguousarray(capacitance, dtype=np.float64)
    _check(_lib.pmut_set_receive(ctx, int(n_switch), _ptr(cap), int(sign)), "pmut_set_receive")


def dgsem_get_voltages(ctx, batch: int, n_pmut: int, nsteps: int):
    """[batch, n_pmut, nsteps] voltages used by the last dgsem_run."""
    out = np.zeros((batch, n_pmut, nsteps))
    _check(_lib.dgsem_get_voltages(ctx, _ptr(out), out.size), "dgsem_get_voltages")
    return out


def dgsem_get_dt(ctx):
    dt, dts, nd = c_double(), c_double(), c_longlong()
    _check(_lib.dgsem_get_dt(ctx, byref(dt), byref(dts), byref(nd)), "dgsem_get_dt")
    return dt.value, dts.value, nd.value


def dgsem_check_stability(ctx, iters: int = 50):
    lam = c_double()
    code = _lib.dgsem_check_stability(ctx, iters, byref(lam))
    return code, lam.value


def dgsem_pmut_nodes(ctx) -> np.ndarray:
    n = c_int()
    p = POINTER(c_double)()
    _check(_lib.dgsem_pmut_nodes(ctx, byref(n), byref(p)), "dgsem_pmut_nodes")
    return np.ctypeslib.as_array(p, shape=(n.value, 2)).copy()


def pmut_array_set(ctx, foot_ptr, foot_node, shape_un, freq_hz, damping, eta, modal_mass=None):
    foot_ptr = np.ascontiguousarray(foot_ptr, dtype=np.int32)
    foot_node = np.ascontiguousarray(foot_node, dtype=np.int32)
    freq_hz = np.ascontiguousarray(freq_hz, dtype=np.float64)
    K, M = freq_hz.shape
    shape_un = np.ascontiguousarray(shape_un, dtype=np.float64).reshape(-1, M)
    damping = np.ascontiguousarray(damping, dtype=np.float64)
    eta = np.ascontiguousarray(eta, dtype=np.float64)
    mm = None if modal_mass is None else np.ascontiguousarray(modal_mass, dtype=np.float64)
    _check(_lib.pmut_array_set(ctx, K, M, _ptr(foot_ptr), _ptr(foot_node), _ptr(shape_un), _ptr(freq_hz),
                               _ptr(damping), _ptr(eta), _ptr(mm)), "pmut_array_set")


def dgsem_run(ctx, precision: int, batch: int, nsteps: int, drive, recv_xyz, traces=None, flags: int = 0,
              stream=None):
    """Returns the traces array [batch][n_recv][nsteps] (numpy unless a torch
    tensor was passed in `traces`)."""
    recv = np.ascontiguousarray(recv_xyz, dtype=np.float64).reshape(-1, 3)
    R = recv.shape[0]
    if traces is None:
        traces = np.zeros((batch, R, nsteps))
    drive = _f64(drive)
    if stream is None:
        stream = _current_stream()
    _check(_lib.dgsem_run(ctx, precision, batch, nsteps, _ptr(drive), R, _ptr(recv), _ptr(traces), flags,
                          stream), "dgsem_run")
    return traces


def dgsem_run_multi(ctxs, precision: int, batch, nsteps: int, drives, recv_xyz, traces=None, flags: int = 0,
                    stream=None):
    """dgsem_run on several contexts in one launch (parallel graph branches).
    drives / recv_xyz: per-context arrays; returns the per-context traces."""
    n = len(ctxs)
    carr = (c_void_p * n)(*[c.value if isinstance(c, c_void_p) else c for c in ctxs])
    barr = np.ascontiguousarray(batch, dtype=np.int32)
    recvs = [np.ascontiguousarray(r, dtype=np.float64).reshape(-1, 3) for r in recv_xyz]
    nr = np.array([r.shape[0] for r in recvs], dtype=np.int32)
    if traces is None:
        traces = [np.zeros((int(barr[i]), int(nr[i]), nsteps)) for i in range(n)]
    drives = [_f64(d) for d in drives]
    darr = (c_void_p * n)(*[_ptr(d) for d in drives])
    rarr = (c_void_p * n)(*[_ptr(r) for r in recvs])
    tarr = (c_void_p * n)(*[_ptr(t) for t in traces])
    if stream is None:
        stream = _current_stream()
    _check(_lib.dgsem_run_multi(n, carr, precision, _ptr(barr), nsteps, darr, _ptr(nr), rarr, tarr, flags, stream),
           "dgsem_run_multi")
    return traces


def dgsem_set_state(ctx, p0=None, v0=None):
    p0 = None if p0 is None else np.ascontiguousarray(p0, dtype=np.float64)
    v0 = None if v0 is None else np.ascontiguousarray(v0, dtype=np.float64)
    _check(_lib.dgsem_set_state(ctx, _ptr(p0), _ptr(v0)), "dgsem_set_state")


def dgsem_get_pressure(ctx, batch: int, ndof: int) -> np.ndarray:
    out = np.zeros((batch, ndof))
    _check(_lib.dgsem_get_pressure(ctx, _ptr(out), out.size), "dgsem_get_pressure")
    return out


def dgsem_get_pmut_state(ctx, batch: int, n_pmut: int, n_modes: int):
    """(q, q', q'') of the PMUT array after the last run, each [batch][n_pmut][n_modes]."""
    out = [np.zeros((batch, n_pmut, n_modes)) for _ in range(3)]
    _check(_lib.dgsem_get_pmut_state(ctx, _ptr(out[0]), _ptr(out[1]), _ptr(out[2]), out[0].size),
           "dgsem_get_pmut_state")
    return tuple(out)


def dgsem_energy(ctx, batch: int) -> np.ndarray:
    """Leapfrog energy 1/2 v.M v + 1/2 p^n.K p^{n+1} of each batch member, in FP64 (either state precision)."""
    out = np.zeros(batch)
    _check(_lib.dgsem_energy(ctx, _ptr(out), batch), "dgsem_energy")
    return out


def dgsem_state_save(ctx) -> bytes:
    n = c_size_t(0)
    _check(_lib.dgsem_state_save(ctx, None, byref(n)), "dgsem_state_save")
    buf = ctypes.create_string_buffer(n.value)
    _check(_lib.dgsem_state_save(ctx, buf, byref(n)), "dgsem_state_save")
    return buf.raw[: n.value]


def dgsem_state_load(ctx, blob: bytes):
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(_lib.dgsem_state_load(ctx, buf, len(blob)), "dgsem_state_load")


def dgsem_num_tiles(ctx, precision: int, box: int) -> int:
    n = c_int()
    _check(_lib.dgsem_num_tiles(ctx, precision, box, byref(n)), "dgsem_num_tiles")
    return n.value


def _num_boxes(ctx) -> int:
    """Boxes of the context (the C calls that take one value per box read
    exactly this many from their array)."""
    n = c_int()
    nb = 0
    while nb < 64 and _lib.dgsem_num_tiles(ctx, 0, nb, byref(n)) == DGSEM_OK:
        nb += 1
    return nb


def _per_box(ctx, values, where):
    arr = np.ascontiguousarray(values, dtype=np.int32).ravel()
    nb = _num_boxes(ctx)
    if arr.size != nb:
        raise ValueError(f"{where}: one value per box ({nb}), got {arr.size}")
    return arr


def dgsem_set_tiles(ctx, precision: int, tiles):
    t = _per_box(ctx, tiles, "dgsem_set_tiles")
    _check(_lib.dgsem_set_tiles(ctx, precision, _ptr(t)), "dgsem_set_tiles")


def dgsem_autotune(ctx, precision: int, batch: int, ndomains: int, reps: int = 3, stream=None):
    """Times every tile variant of each box's volume kernel and keeps the
    fastest; returns the chosen variant per box."""
    out = np.zeros(ndomains, dtype=np.int32)
    if stream is None:
        stream = _current_stream()
    _check(_lib.dgsem_autotune(ctx, precision, batch, reps, _ptr(out), stream), "dgsem_autotune")
    return out


def dgsem_set_layers(ctx, layers_per_cta: Sequence[int]):
    """Element layers per CTA of each box's volume kernel (0 = automatic)."""
    arr = _per_box(ctx, layers_per_cta, "dgsem_set_layers")
    _check(_lib.dgsem_set_layers(ctx, _ptr(arr)), "dgsem_set_layers")


def dgsem_vol_launch(ctx, box: int) -> dict:
    """Shape of box `box`'s volume launch in the last run."""
    out = np.zeros(8, dtype=np.int32)
    _check(_lib.dgsem_vol_launch(ctx, box, _ptr(out)), "dgsem_vol_launch")
    return dict(grid=tuple(int(v) for v in out[:3]), block=tuple(int(v) for v in out[3:6]),
                layers_per_cta=int(out[6]), nchunks=int(out[7]))


def dgsem_sample_noalloc(ctx, recv_xyz, out, stream=None):
    """Sample the current pressure field at recv_xyz ([R][3], R <= 64) into the
    device tensor `out` ([batch][R] float64, contiguous) without any device
    allocation, for callers whose device memory belongs to another allocator
    or to a fixed budget.  Returns after the stream has finished."""
    import torch
    if not isinstance(out, torch.Tensor) or not out.is_cuda or out.dtype != torch.float64 \
            or not out.is_contiguous():
        raise TypeError("out must be a contiguous float64 CUDA tensor of [batch][R] values")
    recv = np.ascontiguousarray(recv_xyz, dtype=np.float64).reshape(-1, 3)
    if stream is None:
        stream = _current_stream()
    _check(_lib.dgsem_sample_noalloc(ctx, recv.shape[0], _ptr(recv), _ptr(out), out.numel(), stream),
           "dgsem_sample_noalloc")
    return out


def dgsem_measure_peak(precision: int, stream=None) -> float:
    """FMA rate of the current device in TFLOP/s (FP64 DFMA or packed FP32)."""
    load_library()
    v = c_double()
    if stream is None:
        stream = _current_stream()
    _check(_lib.dgsem_measure_peak(precision, byref(v), stream), "dgsem_measure_peak")
    return v.value


def dgsem_profile(ctx, enable: bool = True):
    _check(_lib.dgsem_profile(ctx, 1 if enable else 0), "dgsem_profile")


def dgsem_kernel_stats(ctx, kind: int):
    """(total milliseconds, launches) of one kernel kind since dgsem_profile."""
    ms, n = c_double(), c_longlong()
    _check(_lib.dgsem_kernel_stats(ctx, kind, byref(ms), byref(n)), "dgsem_kernel_stats")
    return ms.value, n.value


def dgsem_destroy(ctx):
    if ctx is not None and _lib is not None:
        _lib.dgsem_destroy(ctx)


# ------------------------------------------------------------------ helper
class Solver:
    """Owns one context built from a workload-like description (objects with
    the attributes of include/dgsem.h: domains, cfl, penalty_alpha, quad_pts,
    pmuts with centers/inside/shape_un/freq_hz/damping/eta/modal_mass)."""

    def __init__(self, workload, dt: float = 0.0):
        self.w = workload
        self.ctx = dgsem_mesh_create(workload.domains, cfl=workload.cfl, dt=dt,
                                     penalty_alpha=workload.penalty_alpha,
                                     iface_quad_pts=getattr(workload, "quad_pts", 0) or 0)
        for d, dom in enumerate(workload.domains):
            sides = getattr(dom, "absorbing", None)
            if sides is not None and any(sides):
                dgsem_set_absorbing(self.ctx, d, sides)
            th = getattr(dom, "pml", None)
            if th is not None and any(t > 0 for t in th):
                dgsem_set_pml(self.ctx, d, th, getattr(dom, "pml_R", 1e-4))
        self.dt, _, self.ndof = dgsem_get_dt(self.ctx)
        self.K = 0
        if workload.pmuts is not None:
            self.set_pmuts(workload.pmuts)
            if getattr(workload, "rx_switch", None) is not None:
                cap = np.broadcast_to(np.asarray(workload.rx_capacitance, dtype=np.float64), (self.K,))
                pmut_set_receive(self.ctx, workload.rx_switch, cap, workload.rx_sign)

    def set_pmuts(self, pm):
        xy = dgsem_pmut_nodes(self.ctx)
        ptr = [0]
        nodes, vals = [], []
        for k in range(pm.n_pmut):
            idx = np.nonzero(pm.inside(k, xy[:, 0], xy[:, 1]))[0]
            nodes.append(idx)
            vals.append(np.stack([pm.shape_un(k, m, xy[idx, 0], xy[idx, 1]) for m in range(pm.n_modes)], axis=1))
            ptr.append(ptr[-1] + idx.size)
        pmut_array_set(self.ctx, np.array(ptr), np.concatenate(nodes),
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
        return dgsem_run(self.ctx, precision, B, S, drive, rec, traces=traces, flags=flags, stream=stream)

    def close(self):
        dgsem_destroy(self.ctx)
        self.ctx = None

    def __del__(self):
        try:
            if self.ctx is not None:
                self.close()
        except Exception:
            pass
