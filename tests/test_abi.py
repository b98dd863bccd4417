"""C ABI checks that need no GPU: the library loads, exports every function
declared in include/dgsem.h, and rejects bad arguments before touching CUDA."""
import os
import re

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _built():
    from paper_2603_06267_gb300 import dgsem
    return os.path.exists(dgsem.LIB_PATH)


@pytest.fixture(scope="module")
def lib():
    if not _built():
        import __graft_entry__ as g
        g.build()
    from paper_2603_06267_gb300 import dgsem
    return dgsem.load_library()


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "dgsem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:int|void|const char\*)\s+(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_core_entry_points():
    names = _declared_functions()
    for n in ("dgsem_mesh_create", "pmut_array_set", "dgsem_run", "dgsem_destroy", "dgsem_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_binding_lists_every_declared_symbol():
    from paper_2603_06267_gb300 import dgsem
    assert sorted(dgsem.EXPORTED) == _declared_functions()


def test_invalid_mesh_rejected_without_gpu(lib):
    from paper_2603_06267_gb300 import dgsem
    d = W.Domain((0, 0, 0), (1e-4, 1e-4, 1e-4), (2, 2, 2), 4)
    with pytest.raises(dgsem.DgsemError) as e:
        dgsem.dgsem_mesh_create([d, d, d])
    assert e.value.code == dgsem.DGSEM_EINVAL
    bad = W.Domain((0, 0, 0), (1e-4, 1e-4, 1e-4), (2, 2, 2), 9)
    with pytest.raises(dgsem.DgsemError) as e:
        dgsem.dgsem_mesh_create([bad])
    assert e.value.code == dgsem.DGSEM_EINVAL and "order" in str(e.value)
    neg = W.Domain((0, 0, 0), (1e-4, -1e-4, 1e-4), (2, 2, 2), 4)
    with pytest.raises(dgsem.DgsemError) as e:
        dgsem.dgsem_mesh_create([neg])
    assert e.value.code == dgsem.DGSEM_EINVAL
    with pytest.raises(dgsem.DgsemError):
        dgsem.dgsem_mesh_create([d], cfl=0.0, dt=0.0)


def test_null_context_calls_fail_cleanly(lib):
    from ctypes import c_void_p
    from paper_2603_06267_gb300 import dgsem
    assert lib.dgsem_run(None, 0, 1, 1, None, 0, None, None, 0, None) == dgsem.DGSEM_EINVAL
    assert lib.dgsem_get_dt(None, None, None, None) == dgsem.DGSEM_EINVAL
    lib.dgsem_destroy(None)
    assert b"NULL" in lib.dgsem_last_error()


def test_new_entry_points_reject_bad_arguments_before_cuda(lib):
    """The rate probes, the layer setter, the launch-shape getter and the PMUT
    state getter check their arguments before any CUDA call."""
    from ctypes import byref, c_double
    from paper_2603_06267_gb300 import dgsem
    from paper_2603_06267_gb300 import surrogate as S
    S.load()
    v = c_double(-1.0)
    assert lib.dgsem_measure_peak(7, byref(v), None) == dgsem.DGSEM_EINVAL
    assert lib.dgsem_measure_peak(0, None, None) == dgsem.DGSEM_EINVAL
    assert lib.srg_gemm_bench(512, 32, 2048, 1, byref(v), None) == dgsem.DGSEM_EINVAL
    assert lib.srg_gemm_bench(512, 2048, 2048, 0, byref(v), None) == dgsem.DGSEM_EINVAL
    assert lib.srg_gemm_bench(512, 2048, 2048, 1, None, None) == dgsem.DGSEM_EINVAL
    layers = np.zeros(2, dtype=np.int32)
    shape = np.zeros(8, dtype=np.int32)
    assert lib.dgsem_set_layers(None, layers.ctypes.data) == dgsem.DGSEM_EINVAL
    assert lib.dgsem_vol_launch(None, 0, shape.ctypes.data) == dgsem.DGSEM_EINVAL
    assert lib.dgsem_get_pmut_state(None, None, None, None, 0) == dgsem.DGSEM_EINVAL
    assert lib.dgsem_sample_noalloc(None, 1, None, None, 0, None) == dgsem.DGSEM_EINVAL


def test_surrogate_symbols_exported(lib):
    src = open(os.path.join(ROOT, "include", "surrogate.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = sorted(set(re.findall(r"^\s*(?:int|void|size_t|const char\*)\s+(\w+)\s*\(", src, flags=re.M)))
    from paper_2603_06267_gb300 import surrogate
    assert sorted(surrogate.SRG_EXPORTED) == names
    for n in names:
        assert hasattr(lib, n), n


def _declared_hex_functions():
    src = open(os.path.join(ROOT, "include", "dghex.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(\w+)\s*\(", src, flags=re.M)))


def test_library_exports_every_general_hexahedron_symbol(lib):
    names = _declared_hex_functions()
    assert "dghex_mesh_create" in names and "dghex_run" in names
    for name in names:
        assert hasattr(lib, name), name


def test_hex_binding_lists_every_declared_symbol():
    from paper_2603_06267_gb300 import dghex
    assert sorted(dghex.EXPORTED) == _declared_hex_functions()


def test_invalid_hex_mesh_rejected_without_gpu(lib):
    """Bad orders, vertex ids and face lists are refused on the host."""
    from paper_2603_06267_gb300 import dghex, dgsem
    from workloads import hex as H
    w = H.distorted_two_domain(nx_p=2, nz_p=1, nx_s=1, nz_s=1, n_pmut_side=1, order_p=2, order_s=2)
    prim, sec = w.domains
    bad = H.HexDomain(prim.vertices, prim.elements, 9)
    with pytest.raises(dgsem.DgsemError) as e:
        dghex.dghex_mesh_create([bad])
    assert e.value.code == dgsem.DGSEM_EINVAL and "order" in str(e.value)
    els = prim.elements.copy()
    els[0, 3] = prim.vertices.shape[0]
    with pytest.raises(dgsem.DgsemError) as e:
        dghex.dghex_mesh_create([H.HexDomain(prim.vertices, els, 2)])
    assert e.value.code == dgsem.DGSEM_EINVAL and "vertex" in str(e.value)
    with pytest.raises(dgsem.DgsemError) as e:
        dghex.dghex_mesh_create([prim, sec])          # two domains without the interface lists
    assert e.value.code == dgsem.DGSEM_EINVAL
    inner = np.array([[0, 1]])                        # the face shared by elements 0 and 1
    with pytest.raises(dgsem.DgsemError) as e:
        dghex.dghex_mesh_create([prim], pmut_faces=inner)
    assert e.value.code == dgsem.DGSEM_EINVAL and "boundary" in str(e.value)


def test_volume_variant_calls_refuse_a_null_context_without_gpu(lib):
    """The element-stiffness variant calls check their arguments on the host
    before any device work: a NULL context is DGSEM_EINVAL."""
    import ctypes
    from paper_2603_06267_gb300 import dgsem
    n = ctypes.c_int(-1)
    assert lib.dghex_num_volume_variants(None, ctypes.byref(n)) == dgsem.DGSEM_EINVAL
    v = (ctypes.c_int * 2)(0, 0)
    assert lib.dghex_set_volume_variant(None, dgsem.DGSEM_FP32_MIXED, v) == dgsem.DGSEM_EINVAL
    out = (ctypes.c_int * 2)()
    assert lib.dghex_autotune(None, dgsem.DGSEM_FP32_MIXED, 8, 1, out, None) == dgsem.DGSEM_EINVAL
