"""The bench line's roofline arithmetic (CPU only): the measured DRAM bytes
per SDSN launch and how they scale, the batched kernel's ALU roofline, and
the job rate."""
from types import SimpleNamespace

import pytest

import bench


def test_sdsn_traffic_measured_and_scaled():
    # n = 1000: the ncu figure, independent of the sweep count (on chip).
    assert bench.sdsn_traffic(1000, 4, 196.0) == 4.18e6
    assert bench.sdsn_traffic(1000, 4, 10.0) == 4.18e6
    # n >= 6144: bytes per element and pass times n^2 (sweeps + 1); at the
    # captured size and sweep count it gives back the capture (59.16 GB).
    t = bench.sdsn_traffic(6144, 4, 200.0)
    assert t == pytest.approx(59.16e9, rel=2e-3)
    assert bench.sdsn_traffic(8192, 4, 200.0) == pytest.approx(t * (8192 / 6144) ** 2)
    # no capture covers these: reported as null
    assert bench.sdsn_traffic(4039, 4, 200.0) is None
    assert bench.sdsn_traffic(1000, 8, 200.0) is None


def test_batch_roofline_counts_algorithmic_flops():
    ns = [10, 64]
    infos = [SimpleNamespace(outer_iters=2, total_sweeps=30),
             SimpleNamespace(outer_iters=1, total_sweeps=5)]
    flops = (2 * (4 * 10 ** 3 + 6 * 10 ** 2) + 30 * 7 * 10 ** 2
             + 1 * (4 * 64 ** 3 + 6 * 64 ** 2) + 5 * 7 * 64 ** 2)
    r = bench.batch_roofline(ns, infos, 1e-3)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(flops / 1e-3 / 1e12)
    assert r["peak"] == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])


def test_job_rate_is_units_of_all_ranks_over_the_slowest():
    assert bench.job_rate(10, 1, 2.0) == pytest.approx(5.0)
    assert bench.job_rate(10, 4, 2.0) == pytest.approx(20.0)


def test_cluster_sdsn_roofline_is_alu_on_the_cluster_sms():
    # n = 1000 FP32: the whole iterate stays in one 16-CTA cluster, so the
    # roofline counts 5 n^2 FP32 operations per sweep against 16 SMs x 128
    # lanes x 2.07 GHz, with the whole-GPU fraction beside it.
    info = SimpleNamespace(ms_sdsn=6.7, ms_gemm=0.35, ms_polish=1.06, ms_update=0.33,
                           ms_rounding=0.18, ms_total=8.9, total_sweeps=2040, polish_sweeps=40,
                           outer_iters=10)
    r = bench.roofline([info], 1000, "tf32", {"hbm_gbs": 6800.0}, "measured")
    assert r["bound"] == "alu" and r["kernel"] == "sdsn_cluster_kernel<2, 8>"
    assert r["peak"] == pytest.approx(16 * 128 * 2.07 / 1e3)
    assert r["achieved"] == pytest.approx(5e6 * 2000 / 6.7e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["gpu_frac"] == pytest.approx(r["achieved"] / (152 * 128 * 2.07 / 1e3))
    assert r["traffic"] == 4.18e6
    # n = 50: the two-warp form, against its 64 lanes
    small = SimpleNamespace(**{**vars(info), "ms_sdsn": 0.8, "total_sweeps": 1393,
                               "polish_sweeps": 24, "outer_iters": 8})
    rs = bench.roofline([small], 50, "tf32", {"hbm_gbs": 6800.0}, "measured")
    assert rs["bound"] == "alu" and rs["kernel"] == "sdsn_warp_kernel<2>"
    assert rs["peak"] == pytest.approx(64 * 2.07 / 1e3)
    assert rs["achieved"] == pytest.approx(5 * 2500 * 1369 / 0.8e-3 / 1e12)
    assert bench.roofline([small], 20, "tf32", {"hbm_gbs": 6800.0},
                          "measured")["kernel"] == "sdsn_warp_kernel<1>"
    # above the cluster range the FP32 SDSN streams through HBM
    big = SimpleNamespace(**{**vars(info), "ms_sdsn": 490.0})
    assert bench.roofline([big], 8192, "tf32", {"hbm_gbs": 6800.0}, "measured")["bound"] == "hbm"


def test_packed_batch_addresses_and_views():
    # The batch bench's packed buffers: entry k's address is the buffer base
    # plus the byte offset of the entries before it, its view holds exactly
    # that entry, and the address array has one 8-byte entry per pair (the
    # form the binding passes to the library as it is).
    torch = pytest.importorskip("torch")
    import numpy as np
    rng = np.random.default_rng(3)
    shapes = [(int(n), int(n)) for n in rng.integers(2, 40, size=17)]
    src = [rng.random(sh) for sh in shapes]
    pk = bench.Packed(torch, shapes, torch.float64, "cpu", src=src)
    assert pk.addr.dtype == np.uint64 and pk.addr.shape == (17,)
    off = 0
    for k, (sh, a) in enumerate(zip(shapes, src)):
        assert int(pk.addr[k]) == pk.buf.data_ptr() + 8 * off
        assert pk.views[k].data_ptr() == int(pk.addr[k])
        assert np.array_equal(pk.views[k].numpy(), a)
        off += sh[0] * sh[1]
    pv = bench.Packed(torch, [(n,) for n, _ in shapes], torch.int32, "cpu")
    assert int(pv.addr[1]) - int(pv.addr[0]) == 4 * shapes[0][0]


def test_batch_roofline_counts_the_algorithmic_flops():
    # Per pair: 4 n^3 + 6 n^2 flops per outer iteration (the two products and
    # the update with its delta) and 7 n^2 per SDSN sweep, over the call's
    # time, against the FP32 CUDA-core peak.
    infos = [SimpleNamespace(outer_iters=3, total_sweeps=50),
             SimpleNamespace(outer_iters=2, total_sweeps=20)]
    r = bench.batch_roofline([10, 64], infos, 1e-3)
    flops = 3 * (4 * 10 ** 3 + 6 * 100) + 50 * 7 * 100 + 2 * (4 * 64 ** 3 + 6 * 64 ** 2) + \
        20 * 7 * 64 ** 2
    assert r["bound"] == "alu" and r["achieved"] == pytest.approx(flops / 1e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / bench.FP32_ALU_TFLOPS)
    assert bench.FP32_ALU_TFLOPS == pytest.approx(152 * 128 * 2 * 2.07 / 1e3)
