"""Host-side helpers of bench.py, on the CPU: the FP64 table-build timing, the oracle's
single-thread and transform rates, and the guard that keeps a failing optional leg from
ending the run before its JSON line."""
import bench


def test_bench_times_the_host_table_build():
    """The bench's `tables` entry: the FP64 host build of the basis and the LSC geometry on
    host-only handles (no device needed), once per gradient table."""
    from dataclasses import replace
    cfg = replace(bench.workload_config(256), dirs_per_shell=(30, 30), bvals=(1000.0, 2000.0), rings=2, sectors=6)
    dirs, bvals = bench.table(cfg)
    rec = bench.time_tables(cfg, dirs, bvals, repeats=1)
    assert rec["sh_basis_ms"] > 0 and rec["lsc_geometry_ms"] > 0 and rec["precision"] == "f64"


def test_bench_times_the_oracle_on_one_thread():
    """The bench's single-thread oracle leg: a child interpreter with the BLAS pools held to
    one thread runs the reference arm and its rate is reported."""
    rec = bench.time_oracle_single_thread(steps=1, warm=0, timeout_s=120)
    assert "unavailable" not in rec, rec
    assert rec["value"] > 0 and rec["cores"] == 1


def test_bench_times_the_oracle_transforms():
    from dataclasses import replace
    cfg = replace(bench.workload_config(256), dirs_per_shell=(30, 30), bvals=(1000.0, 2000.0))
    dirs, bvals = bench.table(cfg)
    rec = bench.time_oracle_transforms(cfg, dirs, bvals, n_vox=512, reps=1)
    assert rec["signal2sh_voxels_per_s"] > 0 and rec["sh2signal_voxels_per_s"] > 0 and rec["kind"] == "oracle"


def test_bench_optional_legs_report_failures_instead_of_raising():
    assert bench.guarded("leg", lambda a, b=0: a + b, 1, b=2) == 3
    rec = bench.guarded("leg", lambda: 1 / 0)
    assert rec == {"unavailable": "leg: ZeroDivisionError: division by zero"}


def test_bench_tail_summary_is_short_and_complete():
    """The summary closing the JSON line carries the headline of every leg and stays short
    enough to survive a truncated tail of the line."""
    import json
    leg = {"ms": 0.3, "frac_hbm": 0.612345678, "err_vs_oracle": 1.23456e-7}
    line = {"value": 13003702.74, "err_vs_oracle_bf16": {"s_out": 4.4e-3, "ds_in": 4.2e-3},
            "roofline": {"frac": 0.8312345, "step_frac_of_tensor_peak": 0.61},
            "fp32": {"value": 2.1e6, "err_vs_oracle": {"s_out": 1.3e-6, "ds_in": 1.1e-6}},
            "transforms": {k: dict(leg) for k in ("signal2sh_f32", "sh2signal_f32", "signal2sh_bf16_in",
                                                   "sh2signal_bf16_in")},
            "learned": {"heldout": {"rel_l2_net": 0.0912345, "rel_l2_fallback": 0.4987654},
                        "volume": {"voxels_per_s": 5.0812345e6, "rel_l2_net": 0.0956789, "rel_l2_fallback": 0.51234}}}
    s = bench.tail_summary(line)
    assert s["bf16_vps"] == 13000000.0 and s["gemm_frac"] == 0.8312 and s["fp32_err"] == [1.3e-6, 1.1e-6]
    assert s["signal2sh_f32"] == [0.6123, 1.235e-7]
    assert s["net_vs_fallback"] == [0.09123, 0.4988] and s["volume"] == [5081000.0, 0.09568, 0.5123]
    assert len(json.dumps(s)) < 600
    assert bench.tail_summary({"value": 1.0})["fp32_vps"] is None  # a missing leg reads as null
