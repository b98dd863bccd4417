"""Roofline block of the general-hexahedron bench line: the dominant kernel,
its algorithmic bytes and flops, and the bound chosen by the ridge point."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

ORDERS, NELEM, NDOF, B = [4, 6], [262144, 393216], 102631810, 64


def _kstats(vol_ms, upd_ms):
    # per kind (total ms, launches): pmut, vol (two domains), iface, update, tail, pml
    return [(1.0, 5), (vol_ms, 10), (24.8, 5), (upd_ms, 5), (0.8, 10), (0.0, 0)]


def test_fp32_stiffness_dominant_is_reported_against_the_fp32_pipe():
    import bench
    roof = bench.hex_roofline(_kstats(213.2, 112.2), ORDERS, NELEM, NDOF, B, True, 6685.5)
    # 12 n^4 + 18 n^3 flops per element and member (n = 5 and 7), averaged over the two launches
    flops = (262144 * 64 * (12 * 625 + 18 * 125) + 393216 * 64 * (12 * 2401 + 18 * 343)) / 2
    assert roof["bound"] == "alu" and roof["kernel"] == "vol" and roof["unit"] == "TFLOP/s"
    assert roof["alg_flops_per_launch"] == pytest.approx(flops)
    assert roof["achieved"] == pytest.approx(flops / 21.32e-3 / 1e12)
    assert roof["peak"] == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)
    assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"])
    # bytes: p once per node, residual slots written, geometry (6 words) and node ids once
    ploc = 262144 * 125 + 393216 * 343
    vbytes = (NDOF * B * 4 + ploc * B * 4 + ploc * (6 * 4 + 4)) / 2
    assert roof["alg_bytes_per_launch"] == pytest.approx(vbytes)
    assert flops / vbytes > roof["peak"] * 1e12 / (6685.5e9)          # above the ridge
    assert roof["hbm_frac"] == pytest.approx(vbytes / 21.32e-3 / 6685.5e9)


def test_update_dominant_is_reported_against_hbm():
    import bench
    roof = bench.hex_roofline(_kstats(50.0, 112.2), ORDERS, NELEM, NDOF, B, True, 6685.5)
    ploc = 262144 * 125 + 393216 * 343
    ubytes = NDOF * B * 4 * 4 + ploc * B * 4 + NDOF * 8 + ploc * 4
    assert roof["bound"] == "hbm" and roof["kernel"] == "update" and roof["unit"] == "GB/s"
    assert roof["achieved"] == pytest.approx(ubytes / 22.44e-3 / 1e9)
    assert roof["peak_source"] == "measured"


def test_fp64_stiffness_is_reported_against_the_fp64_rate_and_fallback_peak():
    import bench
    roof = bench.hex_roofline(_kstats(200.0, 112.2), ORDERS, NELEM, NDOF, 8, False, None)
    assert roof["bound"] == "alu" and roof["peak"] == 1.25
    roof_hbm = bench.hex_roofline(_kstats(10.0, 112.2), ORDERS, NELEM, NDOF, 8, False, None)
    assert roof_hbm["peak"] == 6800.0 and roof_hbm["peak_source"] == "fallback"


class _Dom:
    def __init__(self, nelem, order):
        self.nelem, self.order = nelem, order


BOX = [_Dom((128, 128, 16), 4), _Dom((64, 64, 96), 6)]


def test_box_fp32_secondary_volume_against_hbm():
    """config-4 shape: the secondary box (N = 6) dominates; 16 B per node and
    pattern (p and v read, v and p_next written) over its 385 x 385 x 577
    lattice, against the measured copy bandwidth, with the ncu traffic."""
    import bench
    kstats = [(9.36, 40), (19.77, 60), (60.77, 20), (343.53, 20), (0.0, 0)]
    roof = bench.box_roofline(kstats, BOX, 64, True, 6685.5, lambda k: 86.2336e9 if k == "vol_secondary" else None)
    nodes = 385 * 385 * 577
    assert roof["kernel"] == "vol_secondary" and roof["bound"] == "hbm"
    assert roof["alg_bytes_per_launch"] == nodes * 64 * 16
    assert roof["achieved"] == pytest.approx(nodes * 64 * 16 / 17.1765e-3 / 1e9)
    assert roof["frac"] == pytest.approx(roof["achieved"] / 6685.5)
    assert roof["traffic"] == 86.2336e9
    # traffic is only quoted for the batch sizes the capture was scaled to
    assert bench.box_roofline(kstats, BOX, 8, True, 6685.5, lambda k: 1.0)["traffic"] is None


def test_box_fp64_against_the_fp64_rate():
    import bench
    kstats = [(1.0, 10), (2.0, 30), (12.0, 10), (57.0, 10), (0.0, 0)]
    roof = bench.box_roofline(kstats, BOX, 1, False, 6685.5, lambda k: None)
    nodes = 385 * 385 * 577
    assert roof["bound"] == "alu" and roof["peak"] == 1.25
    assert roof["achieved"] == pytest.approx(nodes * 2 * (3 * 8 + 4) / 5.7e-3 / 1e12)
    assert roof["hbm_achieved_gbs"] == pytest.approx(nodes * 32 / 5.7e-3 / 1e9)
    # a kernel other than a volume kernel dominating: no roofline block
    assert bench.box_roofline([(9.0, 1), (1.0, 1), (1.0, 1), (1.0, 1), (0.0, 0)], BOX, 1, False, None,
                              lambda k: None) is None


def test_box_roofline_takes_the_workload_domains():
    import bench
    import workloads as W
    w = W.config4_batched(nsteps=2)
    kstats = [(9.36, 40), (19.77, 60), (60.77, 20), (343.53, 20), (0.0, 0)]
    roof = bench.box_roofline(kstats, w.domains, w.batch, True, None, lambda k: None)
    assert roof["alg_bytes_per_launch"] == 385 * 385 * 577 * 64 * 16 and roof["peak_source"] == "fallback"
