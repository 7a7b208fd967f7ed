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
