"""Host logic of bench.py that needs no GPU: the parsing of the nvidia-smi clock samples taken
during a timed region (the median SM clock, the maximum, and the throttle reasons that reject a
run), and the peak lookup."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _clocks(tmp_path, lines):
    sys.path.insert(0, ROOT)
    import bench
    c = bench.Clocks(None)
    c.path = str(tmp_path / "clocks.csv")
    with open(c.path, "w") as f:
        f.write("\n".join(lines) + "\n")
    c.f = open(os.devnull, "w")
    c.proc = _Done()
    return c.stop()


def test_median_clock_and_no_reasons(tmp_path):
    rows = [f"0, {mhz}, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active"
            for mhz in (2070, 2055, 2070, 1980, 2070)]
    got = _clocks(tmp_path, rows)
    assert got["sm_mhz"] == 2070 and got["sm_max_mhz"] == 2070 and got["reasons"] == [] and got["samples"] == 5


def test_throttle_reasons_are_collected(tmp_path):
    rows = ["0, 1700, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 1650, 2070, 1400.0, 0x28, Active, Not Active, Active, Not Active",
            "malformed line",
            "0, [N/A], 2070, 1400.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    got = _clocks(tmp_path, rows)
    assert got["samples"] == 2 and got["sm_mhz"] == 1675
    assert got["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]


def test_no_samples_and_no_tool(tmp_path):
    assert _clocks(tmp_path, ["garbage"])["reasons"] == ["no samples"]
    sys.path.insert(0, ROOT)
    import bench
    assert bench.Clocks(None).stop()["reasons"] == ["nvidia-smi unavailable"]


def test_peaks_fall_back_without_the_measured_file(monkeypatch, tmp_path):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.load_peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6794.8}')
    assert bench.load_peaks() == (6794.8, "measured")


def test_cli_and_config_of_the_single_solve_workloads(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    for argv, want in ((["bench.py"], "large single solve"),
                       (["bench.py", "--workload", "interferometry", "--bits", "4", "--bits-y", "8"],
                        "interferometry-shaped"),
                       (["bench.py", "--workload", "mri"], "MRI-shaped")):
        monkeypatch.setattr(sys, "argv", argv)
        args = bench.parse()
        assert args.steps >= 1 and args.warmup >= 3
        cfg = bench.config(args, 1)
        assert cfg["workload"].startswith(want) and cfg["parallelism"] == "single GPU"
        assert cfg["bits_y"] == (args.bits_y or args.bits) and "model" not in cfg
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    args = bench.parse()
    assert args.impl == "reference" and args.gpus == 2


def test_cpu_sample_is_one_definition_and_records_the_host():
    # the reference arm and the cpu_baseline of the line time the same bounded oracle sample,
    # on every host core, and say how many threads ran and on which CPU
    sys.path.insert(0, ROOT)
    import inspect

    import bench
    import oracle
    import synth
    sig = inspect.signature(bench.oracle_sample)
    assert sig.parameters["rows"].default == bench.SAMPLE_ROWS
    assert sig.parameters["iters"].default == bench.SAMPLE_ITERS
    p = synth.gaussian(128, 512, 8, seed=1, snr_db=30.0)
    n0 = oracle.get_threads()
    try:
        out = bench.oracle_sample(p, 8, 300, rows=64, iters=5)
    finally:
        oracle.set_threads(n0)
    assert out["kind"] == "oracle" and out["extrapolated"] is True
    assert out["cores"] == (os.cpu_count() or 1) and out["nproc"] == os.cpu_count()
    assert isinstance(out["cpu_model"], str) and out["cpu_model"]
    assert out["value"] > 0 and "first 64 of 128 rows" in out["sample"]
