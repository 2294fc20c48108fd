"""The bench's roofline arithmetic (host logic, no GPU): the dominant tensor-core launch's
achieved rate is its algorithmic flops per launch over its average launch time; the first
layer counts the method's K = N + 2, not the device's three-term K; the fused output layers
count both products; DRAM traffic scales from the captured 262,144-cell chunk."""
import pytest

import bench

WIDTHS = [32, 1600, 800, 400, 29]        # the 30-species network: N + 2 inputs, N - 1 outputs


def _dom(name, launches, ms):
    return name, (launches, ms, 0.0, 0.0)


def test_dominant_layer_two():
    # 4 launches of 2,097,152 cells (two steps of 4,194,304) at 3.8 ms each
    d = bench.dominant_gemm(_dom("gemm_tn_kernel<208> 800x1600", 4, 15.2), 4194304, 2097152, WIDTHS, 1940.2, 2)
    per_cell = 2.0 * 1600 * 800
    assert d["cells_per_launch"] == 2097152
    assert d["avg_ms"] == pytest.approx(3.8)
    assert d["achieved"] == pytest.approx(2097152 * per_cell / 3.8e-3 / 1e12)
    assert d["frac"] == pytest.approx(d["achieved"] / 1940.2)


def test_first_layer_counts_the_method_k():
    # the launch's K is 96 (three BF16 terms of 32 padded inputs); the method's work is 2 * 32 * 1600
    d = bench.dominant_gemm(_dom("gemm_tn_kernel<256> 1600x96", 2, 4.0), 4194304, 2097152, WIDTHS, 1940.2, 1)
    assert d["mflop_per_cell"] == pytest.approx(2.0 * 32 * 1600 / 1e6)


def test_fused_output_layers_count_both_products():
    d = bench.dominant_gemm(_dom("gemm_fused34_kernel 400x800+29x400", 2, 2.5), 4194304, 2097152, WIDTHS,
                            1940.2, 1)
    assert d["mflop_per_cell"] == pytest.approx(2.0 * (800 * 400 + 400 * 29) / 1e6)


def test_traffic_scales_from_the_captured_chunk():
    old = bench.MECH
    try:
        bench.MECH = "c2"
        chunk = bench.GEMM_CHUNK_TRAFFIC["c2"]["gemm_tn_kernel<208> 800x1600"]
        assert bench.gemm_traffic(2097152, "gemm_tn_kernel<208> 800x1600") == pytest.approx(8 * chunk)
        assert bench.gemm_traffic(262144) == pytest.approx(sum(bench.GEMM_CHUNK_TRAFFIC["c2"].values()))
        assert bench.gemm_traffic(262144, "not captured") is None
        bench.MECH = "c5"
        assert bench.gemm_traffic(262144) is None              # no capture for the 53-species network
    finally:
        bench.MECH = old


def test_network_flops_per_cell():
    # 2 sum fan_in fan_out over 32-1600-800-400-29: the 3.3256 MFLOP per cell of the aggregate
    mflop = 2.0 * sum(a * b for a, b in zip(WIDTHS[:-1], WIDTHS[1:])) / 1e6
    assert mflop == pytest.approx(3.3256, abs=1e-4)


def test_props_full_line():
    # 10 timed steps, 31.5 ms of props launches: 3.15 ms per step on 16 N^2 + 30 N flops per cell
    prof = {"props_kernel<f32>": (10, 31.5, 0.0, 0.0), "gemm_tn_kernel<208> 800x1600": (20, 76.0, 0.0, 0.0)}
    line = bench.props_full_line(prof, 4194304, 10, 30)
    assert line["ms_per_step"] == pytest.approx(3.15)
    assert line["roofline"]["flops_per_cell"] == 15300
    assert line["roofline"]["achieved"] == pytest.approx(4194304 * 15300 / 3.15e-3 / 1e12)
    assert bench.props_full_line({}, 4194304, 10, 30) is None


def test_guarded_keeps_the_error():
    out = bench.guarded(lambda: 1 / 0)
    assert out == {"error": "ZeroDivisionError: division by zero"}
