"""Host-side logic of the benchmark (CPU): the kernel fingerprint that keys the committed
DRAM-traffic summaries, the reading of those summaries, the clock-record parsing that
decides whether a run is kept, and the reference arm's output line."""
import os
import shutil

import pytest

import bench


def test_kernel_fingerprint_ignores_comments_and_layout_but_not_code(tmp_path, monkeypatch):
    csrc = os.path.join(bench.ROOT, "paper_2609_32920_gb300", "csrc")
    root = tmp_path / "repo"
    shutil.copytree(csrc, root / "paper_2609_32920_gb300" / "csrc")
    monkeypatch.setattr(bench, "ROOT", str(root))
    fp0 = bench.kernel_fingerprint()
    assert len(fp0) == 16 and int(fp0, 16) >= 0
    k = root / "paper_2609_32920_gb300" / "csrc" / "lt_kernels.cu"
    src = k.read_text()
    k.write_text("// a new comment\n" + src.replace("\n", "\n\n", 3) + "\n/* and another */\n")
    assert bench.kernel_fingerprint() == fp0
    k.write_text(src.replace("constexpr int kDraws = 4;", "constexpr int kDraws = 5;"))
    assert bench.kernel_fingerprint() != fp0


def test_committed_traffic_summaries_match_the_current_kernels():
    """bench.py reports roofline.traffic only while the kernels match the capture: the
    committed summaries must carry the current fingerprint and both per-launch figures."""
    for wl in bench.WORKLOADS:
        for key in ("primal", "lrb3_backward"):
            tb = bench.profiled_traffic(wl, key)
            assert isinstance(tb, int) and tb > 0, (wl, key)


def test_traffic_is_dropped_when_the_kernels_change(monkeypatch):
    monkeypatch.setattr(bench, "kernel_fingerprint", lambda: "0" * 16)
    assert bench.profiled_traffic("slab512_hm128", "lrb3_backward") is None
    assert bench.profiled_traffic("no_such_workload", "primal") is None


def test_clock_record_reasons_and_median(tmp_path):
    c = bench.Clocks(0)
    c.path = str(tmp_path / "clk.csv")
    rows = ["2070, 2070, 400.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "2055, 2070, 600.3, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            "2070, 2070, 500.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "garbage line"]
    (tmp_path / "clk.csv").write_text("\n".join(rows) + "\n")

    class Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    c.proc, c.f = Done(), open(c.path, "a")
    r = c.stop()
    assert r["samples"] == 3 and r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0
    assert r["power_w_max"] == pytest.approx(600.3)
    assert r["reasons"] == ["sw_power_cap"]


def test_workload_config_names_the_workload():
    for wl in bench.WORKLOADS:
        cfg = bench.workload_config(1 << bench.WORKLOADS[wl]["paths_log2"], wl)
        assert cfg["workload"] == wl and cfg["paths_per_gpu"] == 1 << bench.WORKLOADS[wl]["paths_log2"]
        assert "model" not in cfg


def _ref_args(**kw):
    import argparse
    a = dict(gpus=1, steps=2, warmup=3, impl="reference", workload="box256_hm32", paths_log2=0)
    a.update(kw)
    return argparse.Namespace(**a)


def test_reference_arm_prints_one_contract_line(oracle, monkeypatch, capsys):
    """`bench.py --impl reference` (the FP64 oracle on the host cores): one JSON line with the
    contract's keys, the GPU arm's metric and workload, and zero host<->device bytes.  The
    oracle's sample is forced small here; the arm itself sizes it by time."""
    import json
    monkeypatch.setattr(bench, "oracle_sample", lambda sc, dI, s, n_norm, depth: (64, 0.01, 2))
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.delenv("RANK", raising=False)
    assert bench.run_reference(_ref_args()) == 0
    out = [l for l in capsys.readouterr().out.splitlines() if l.strip()]
    assert len(out) == 1
    line = json.loads(out[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["value"] > 0
    assert (line["steps"], line["warmup"], line["n_gpus"]) == (2, 3, 1)
    assert line["config"] == bench.workload_config(1 << 22, "box256_hm32")
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["cores"] == 2 and "64 of the workload's" in line["cpu_baseline"]["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": "paths/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(bench, "oracle_sample", lambda *a: (_ for _ in ()).throw(AssertionError("rank 1 ran")))
    assert bench.run_reference(_ref_args()) == 0
    assert capsys.readouterr().out == ""
