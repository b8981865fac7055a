"""The benchmark's reference arm runs on the host alone (the oracle, timed on
the host cores) and prints one JSON line with the contract's keys; checked here
on the smallest workload so that it needs no GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--config", "c0", "--steps", "1", "--warmup", "1"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference"
    assert d["warmup"] >= 3  # at least three warm-up steps, whatever was asked
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["name"] == "c0" and "N=100" in d["config"]["workload"]


def test_bench_options_are_documented():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--help"],
                       capture_output=True, text=True, timeout=120, cwd=ROOT)
    assert r.returncode == 0
    for opt in ("--gpus", "--steps", "--warmup", "--impl", "--config", "--row", "--shape"):
        assert opt in r.stdout, opt


def test_traffic_figures_come_from_committed_profiles():
    """Every DRAM-traffic figure the bench reports is one that an ncu summary
    under profiles/ states, for a workload the bench knows and a launch shape
    the library accepts."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    prof = os.path.join(ROOT, "profiles")
    text = "".join(open(os.path.join(prof, f)).read() for f in sorted(os.listdir(prof)))
    assert bench.STEP_DRAM_BYTES
    for key, nbytes in bench.STEP_DRAM_BYTES.items():
        (cfg, warps, tile, chunk, tpl, rpl), sym = key[:6], key[6:7] == ("sym",)
        assert len(key) == 6 or (sym and key[7:] in ((), ("block",))), key
        assert cfg == "c1" or cfg in bench.CONFIGS, cfg
        assert tile & (tile - 1) == 0 and chunk % 64 == 0
        if sym:
            assert tile == 32 and rpl == 1 and (warps, tpl) in ((4, 2), (4, 4), (8, 2), (2, 4))
        else:
            assert tpl in (1, 2, 3)
            assert (warps in (4, 8, 16) and rpl == 1) or (rpl in (2, 4) and warps == rpl)
        assert "%.4g MB" % (nbytes / 1e6) in text, (cfg, nbytes)
