"""Host-side arithmetic of bench.py's roofline: the algorithmic bytes per
fused step of each layout, the layout-keyed DRAM traffic from the committed
ncu summary, and the float64 peak derived from unit counts and clocks."""
import bench


def test_step_byte_models():
    n, nnz = 2_097_152, 14_581_760            # the 128^3 diffusion system
    # CSR / SELL-32: values and int32 columns once, row pointers, 4 vector passes
    assert bench.csr_step_bytes(n, nnz) == nnz * 12 + 4 * (n + 1) + 32 * n == 250_478_596
    assert bench.csr_step_bytes(n, nnz, 4, 4) == nnz * 8 + 4 * (n + 1) + 16 * n
    # offset-pattern layout: no column indices, 8 bytes of slice data per 32 rows
    assert bench.psell_step_bytes(n, nnz) == nnz * 8 + 8 * (n // 32) + 32 * n == 184_287_232
    assert bench.step_bytes_for("psell", n, nnz, 8, 8) == bench.psell_step_bytes(n, nnz)
    assert bench.step_bytes_for("sell", n, nnz, 8, 8) == bench.csr_step_bytes(n, nnz)
    # 3x3 blocks: 9 values and one block column per block
    assert bench.bsr3_step_bytes(30, 10) == 10 * (9 * 8 + 4) + 4 * 11 + 32 * 30


def test_traffic_is_keyed_by_layout_and_precision():
    assert bench.read_traffic("c2:2097152:psell", "f64") == 171_503_104
    assert bench.read_traffic("c2:2097152:sell", "f64") == 229_708_800
    # no capture of this kernel in its current form: no number
    assert bench.read_traffic("c2:2097152:psell", "f32") is None
    assert bench.read_traffic("c2:2097152", "f64") is None
    # traffic at or below the algorithmic bytes: no re-reads
    assert bench.read_traffic("c2:2097152:psell", "f64") <= bench.psell_step_bytes(2_097_152, 14_581_760)


def test_float64_peak_from_unit_counts():
    # 2 float64 FMA per clock per SM x 2 flops x 152 SMs x 2.07 GHz
    assert bench.FP64_PEAK_TFLOPS == round(2 * 2 * 152 * 2.070e9 / 1e12, 4) == 1.2586
    assert "2 float64 FMA/clk/SM" in bench.FP64_PEAK_SOURCE


def test_host_info_names_the_cpu_and_its_cores():
    info = bench.host_info()
    assert isinstance(info["host_cpu"], str) and info["host_cpu"]
    assert isinstance(info["host_nproc"], int) and info["host_nproc"] >= 1
