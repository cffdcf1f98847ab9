"""The product arm of bench.py prints one short JSON line with the measurement
contract's keys, whatever its sections hold (they go to the detail file in
full); and the CPU run of the paper's own test produces its table.  No GPU."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

CONTRACT = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
            "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "cpu_baseline", "clocks", "gpu_launches")


def stub_core():
    return {
        "metric": bench.METRIC, "value": 49.9, "unit": "TFLOP/s", "n_gpus": 1, "steps": 20, "warmup": 5,
        "ms_per_step": 22.0, "step_ms": {"median": 22.0, "min": 21.9, "max": 22.1}, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic", "precision": "8 BF16 slices",
        "config": {"workload": bench.WORKLOAD, "N": 8192, "P": 8192, "M": 8192, "slices": 8, "beta": 7,
                   "parallelism": "single", "l2": "inputs (1 GiB) larger than L2"},
        "roofline": {"bound": "tensor", "achieved": 1867.0, "peak": 1899.5, "unit": "TFLOP/s", "frac": 0.98,
                     "traffic": 2.0e10, "kernel": "emu_slice_gemm_tcgen05", "peak_source": "measured bf16_tflops",
                     "frac_of_bf16_tflops_sustained": 1.1, "algorithmic_unit": "36 slice pairs x 2NPM"},
        "kernel_ms_per_launch": {"emu_slice_gemm_tcgen05": 21.2, "emu_split_rows": 0.33, "emu_col_max": 0.11,
                                 "emu_split_cols": 0.33},
        "gpu_launches": 80, "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 200},
    }


def stub_sections():
    big = {str(n): {m: {"ms": 1.0, "tflops": 1.0, "fp64_pipe_frac": 0.9} for m in
                    ("naive", "kahan", "winograd", "winograd_scaled", "strassen", "strassen_winograd",
                     "emulated_8_slices", "naive_ordered", "naive_unrolled_4")} for n in bench.FP64_SWEEP}
    arm = {"saturated_requests_per_s": 700.0, "saturated_tflops": 0.8,
           "paced": {"arrival_rate_rps": 490.0, "requests": 10000, "p50_ms": 3.0, "p99_ms": 20.0, "mean_ms": 4.0,
                     "max_ms": 40.0, "requests_per_s": 490.0, "status": 0}}
    return {
        "e2e": {"value": 42.3, "unit": "TFLOP/s", "ms_per_step": 26.0, "steps": 20, "statistic": "median",
                "ms_mean": 26.5, "ms_min": 25.9, "ms_max": 27.0, "ms_each": [26.0] * 20, "clocks": {},
                "h2d_bytes_per_step": 1073741824, "d2h_bytes_per_step": 536870912, "call": "mm_emulated_host"},
        "plain_fp64": {"value": 1.1, "unit": "TFLOP/s", "ms": 999.0, "rel_inf_err_sampled": 2e-16,
                       "fp64_pipe_frac": 0.9, "kernel": "gemm_f64_dmma"},
        "accuracy": {"rel_inf_err_sampled": 3.7e-17, "rows_sampled": [0, 2048, 4096, 6144], "target": 1e-14,
                     "reference": "oracle Dot2"},
        "fp64_peak": {"dfma_tflops": 1.2, "dmma_tflops": 1.25, "clocks": {"sm_mhz": 2070.0}, "how": "probe"},
        "serving": {"requests": 10000, "saturated": {"requests_per_s": 14000.0}, "paced": {"p50_ms": 1.2,
                                                                                           "p99_ms": 5.5},
                    "like_for_like_1e-14": {"fp64_one_at_a_time": arm, "emulated": arm,
                                            "emulated_at_fp64_rate": {"p50_ms": 0.5, "p99_ms": 3.0}},
                    "load_sweep": {str(f): {"p50_ms": 1.0, "p99_ms": 2.0} for f in (0.3, 0.5, 1.0)}},
        "fp64_methods": {"by_size": big},
        "paper_table": {"n": {"800": {m: {"time_s": 1.0} for m in range(12)}}},
        "slice_sweep": {"bf16": {str(s): {"ms": 1.0} for s in range(3, 9)}},
        "grouped_vs_single": {"grouped": {"ms": 14.0, "tflops": 24.0}, "one_call_each": {"tflops": 9.0}},
        "shape_4096x16384x4096": {"tflops": 46.3},
        "strassen_over_emulated": {"8192": {"strassen_winograd_1": {"tflops": 52.8}}},
        "cpu_baseline": {"value": 0.0045, "unit": "TFLOP/s", "cores": 16, "kind": "oracle", "sample": "192 rows",
                         "single_thread": {"value": 0.0003}},
    }


def test_compact_line_has_the_contract_keys_and_stays_short():
    sections = stub_sections()
    assert len(json.dumps(sections)) > 6000  # the sections alone would make a long line
    line = bench.compact_line(stub_core(), sections)
    text = json.dumps(line)
    assert len(text) < 4096, len(text)
    for key in CONTRACT:
        assert key in line, key
    assert line["value"] > 0 and line["higher_is_better"] is True
    for key in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert key in line["roofline"], key
    for key in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert key in line["e2e"], key
    assert line["e2e"]["h2d_bytes_per_step"] > 0 and "ms_each" not in line["e2e"]
    for key in ("value", "unit", "cores", "kind", "sample"):
        assert key in line["cpu_baseline"], key
    assert line["summary"]["serving"]["1e-14_fp64_one_at_a_time"]["p99_ms"] == 20.0
    assert json.loads(text) == line  # strict JSON round trip


def test_compact_line_without_optional_sections():
    line = bench.compact_line(stub_core(), {})
    assert "summary" not in line and line["value"] == 49.9


def test_paper_table_cpu_small(orc):
    t = bench.paper_table_cpu(sizes=(8, 17), repeats=1)
    for n in ("8", "17"):
        rows = t["n"][n]
        assert len(rows) == 10
        assert rows["NaivKahan (N)"]["norm_inf_N_minus_C"] == 0.0
        for r in rows.values():
            assert r["time_s"] > 0 and r["norm_inf_N_minus_C"] < 1e-10
