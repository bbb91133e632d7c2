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
    assert bench.step_bytes_for({"spmv_format": "psell"}, n, nnz, 8, 8) == bench.psell_step_bytes(n, nnz)
    assert bench.step_bytes_for({"spmv_format": "sell"}, n, nnz, 8, 8) == bench.csr_step_bytes(n, nnz)
    # a constant diagonal folded into the step coefficients is not stored: n values fewer
    folded = {"spmv_format": "psell", "diag_folded": 1}
    assert bench.step_bytes_for(folded, n, nnz, 8, 8) == bench.psell_step_bytes(n, nnz - n) == 184_287_232 - 8 * n
    assert bench.stored_nnz(folded, n, nnz) == nnz - n
    assert bench.stored_nnz({"spmv_format": "psell", "diag_folded": 0}, n, nnz) == nnz
    # 3x3 blocks: 9 values and one block column per block
    assert bench.bsr3_step_bytes(30, 10) == 10 * (9 * 8 + 4) + 4 * 11 + 32 * 30


def test_traffic_is_keyed_by_layout_and_precision():
    assert bench.read_traffic("c2:2097152:psell", "f64") == 171_503_104
    assert bench.read_traffic("c2:2097152:sell", "f64") == 229_708_800
    assert bench.read_traffic("c2:2097152:psell", "f32") == 87_088_640
    assert bench.read_traffic("c2:2097152:psell", "bf16") == 55_056_128
    # the layout with its constant diagonal folded out: its own captures
    assert bench.read_traffic("c2:2097152:psell-fold", "f64") == 155_038_976
    assert bench.read_traffic("c2:2097152:psell-fold", "f64") <= bench.psell_step_bytes(2_097_152, 14_581_760 - 2_097_152)
    # no capture of this kernel in this form: no number
    assert bench.read_traffic("c2:2097152:psell", "f16") is None
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


def test_oracle_errors_of_the_cpu_leg(tmp_path):
    """The CPU leg's error of a GPU solution against the oracle: 0 for the
    oracle's own solution, and the relative size of a planted perturbation
    otherwise (checked on two small stencil systems, in the scaled-back
    original variables)."""
    import math
    import pickle
    import types
    import numpy as np
    import oracle as O
    import workloads as W
    samples = []
    for (nx, ny, nz, w) in ((6, 5, 4, (1.0, 0.3, 0.1)), (9, 7, 3, (0.2, 1.0, 0.5))):
        st = W.stencil7_aniso(nx, ny, nz, *w)
        sc = W.Stencil7(nx, ny, nz, 1.0, st.cx / st.c0, st.cy / st.c0, st.cz / st.c0)
        lo, hi = W.stencil7_bounds(sc)
        b = W.uniform_vector(st.n, seed=nx)
        mv = O.stencil7_matvec(nx, ny, nz, 1.0, sc.cx, sc.cy, sc.cz)
        prm = O.cheb_params(lo, hi, bench.S_THETA)
        dis = 1.0 / math.sqrt(st.c0)
        ro = O.pcg(mv, dis * b, lambda r: O.cheb_apply(mv, r, prm, 8), m=8, tol=bench.TOL, maxit=1000)
        samples.append({"dims": [nx, ny, nz], "c": [st.c0, st.cx, st.cy, st.cz], "lo": lo, "hi": hi, "k": 8,
                        "b": b, "x": dis * ro.x, "iters": ro.iters})
    bumped = dict(samples[1])
    bumped["x"] = samples[1]["x"] * (1.0 + 1e-3)
    path = tmp_path / "e.pkl"
    with open(path, "wb") as f:
        pickle.dump({"c4": samples, "c5": [bumped]}, f)
    out = bench.oracle_errors(str(path), types.SimpleNamespace(grid=None))
    assert [d["rel_err"] for d in out["c4"]["samples"]] == [0.0, 0.0]
    assert out["c4"]["samples"][0]["oracle_iters"] == samples[0]["iters"]
    assert abs(out["c5"]["max_rel_err"] - 1e-3) < 1e-12
