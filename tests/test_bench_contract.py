"""Host-side checks of bench.py's JSON contract (no GPU): every workload the
command line accepts has its metric and workload description, the descriptions
that take the matrix size format, and a traffic record is reported only for the
source it was measured on."""
import hashlib
import importlib.util
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


WORKLOADS = ("dense4096", "batch", "small", "large", "learned", "compare4096", "complex2048", "integrator")


@pytest.mark.parametrize("workload", WORKLOADS)
def test_every_workload_has_metric_and_description(bench, workload, monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", workload])
    args = bench.parse()
    assert args.workload == workload
    assert bench.METRICS[workload]
    assert bench.WORKLOAD_DESC[workload]


def test_defaults_are_the_headline_run(bench, monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    args = bench.parse()
    assert (args.gpus, args.workload, args.impl) == (1, "dense4096", "ours")
    assert args.warmup >= 3 and args.steps >= 1


@pytest.mark.parametrize("workload", ["dense4096", "large", "complex2048"])
def test_sized_descriptions_format(bench, workload):
    assert "4096" in bench.WORKLOAD_DESC[workload].format(n=4096)


def test_traffic_record_follows_the_source(bench, monkeypatch):
    import hashlib
    srcs = ("gemm_f64.cu", "internal.h")
    h = hashlib.sha256()
    for src in srcs:
        h.update(open(os.path.join(ROOT, "paper_1710_10989_gb300", "csrc", src), "rb").read())
    monkeypatch.setitem(bench.NCU_TRAFFIC, "k_gemm_f64", (srcs, h.hexdigest(), 4096, 1.0e9))
    assert bench.ncu_traffic("k_gemm_f64", 4096) == 1.0e9
    assert bench.ncu_traffic("k_gemm_f64", 2048) is None          # another size: no record
    monkeypatch.setitem(bench.NCU_TRAFFIC, "k_gemm_f64", (srcs, "0" * 64, 4096, 1.0e9))
    assert bench.ncu_traffic("k_gemm_f64", 4096) is None          # a source changed since the capture
    assert bench.ncu_traffic("no_such_kernel", 4096) is None


def test_pair_kernel_traffic_record_is_current(bench):
    """The split product's DRAM traffic in the bench line was captured from the
    sources as they are now (a change to the kernel or its headers drops it)."""
    assert bench.ncu_traffic("k_ozaki_pair", 4096) is not None


def test_reference_arm_runs_the_oracle_alone_on_the_same_config(bench, monkeypatch):
    """--impl reference times the oracle without loading the CUDA library, and
    prints the same `config` the main arm prints for that workload (here the dense
    workload's twelve matrices at N = 96, so that it runs in seconds)."""
    import json
    import subprocess
    code = ("import runpy, sys\n"
            "sys.argv = ['bench.py', '--impl', 'reference', '--n', '96', '--steps', '4']\n"
            "runpy.run_path('bench.py', run_name='__main__')\n"
            "maps = open('/proc/self/maps').read()\n"
            "print('LOADED', 'libbbcexpm' in maps, 'paper_1710_10989_gb300.api' in sys.modules)\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = r.stdout.strip().splitlines()
    line = json.loads(lines[0])
    assert lines[-1] == "LOADED False False"
    assert line["impl"] == "reference" and line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["cpu_baseline"]["cpu_model"] == bench.host_cpu() != ""
    monkeypatch.setattr(sys, "argv", ["bench.py", "--n", "96"])
    args = bench.parse()
    mats = bench.dense_workload(96)
    prods = bench.products_of(mats)            # the main arm's selection: the library's own
    assert line["config"] == bench.dense_config(args, 96, mats, prods, 1)
    assert line["config"]["products_per_step"] == 84


def test_reference_cycle_samples_the_mix(bench):
    """Every four consecutive reference steps hold the workload's mean product count."""
    mats = bench.dense_workload(96)
    from oracle import oracle as O
    prods = bench.products_of(mats, select=lambda v, u: O.select(v, "new", u))
    assert sorted(bench.DENSE_CYCLE) == list(range(12))
    for k in range(0, 12, 4):
        assert sum(prods[i] for i in bench.DENSE_CYCLE[k:k + 4]) == 4 * sum(prods) / len(prods)


def test_reference_arm_under_two_ranks_prints_once():
    """Under torchrun with two ranks the reference arm runs on rank 0 alone: rank 1
    exits 0 without output, rank 0 prints the one line with n_gpus = 2."""
    import json
    import subprocess
    out = {}
    for rank in (1, 0):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank))
        r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--n", "96", "--steps", "2",
                            "--gpus", "2"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stderr
        out[rank] = r.stdout.strip()
    assert out[1] == ""
    line = json.loads(out[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
