"""bench.py's host logic on CPU: the multi-rank path (two gloo ranks, each with its own
timing, agree on the slowest rank's time; the replicas exchange nothing else), and the
DRAM traffic taken from the committed ncu summaries, and the reference arm (the FP64
oracle on the host cores) alone and under two torchrun ranks."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        out[rank] = bench.max_over_ranks(10.0 + 5.0 * rank, "cpu", world)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn")
        assert dict(out) == {0: 15.0, 1: 15.0}


def test_max_over_ranks_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.25, "cpu", 1) == 3.25


def test_profile_traffic_only_while_the_digest_matches(tmp_path, monkeypatch):
    """roofline.traffic comes from a committed ncu summary only while its source digest
    is the current kernel sources' (a changed kernel reports null)."""
    import bench
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "x.md").write_text(
        "- source_sha256: `abc`\n- traffic_bytes_per_launch_f32: 123\n"
        "- traffic_bytes_per_step_f32: 45\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setitem(bench.PROFILE, "march", "x.md")
    monkeypatch.setattr(bench, "step_kernel_digest", lambda kernel="march": "abc")
    assert bench.profile_traffic("march", "f32") == 123
    assert bench.profile_traffic("march", "traffic_bytes_per_step_f32") == 45
    assert bench.profile_traffic("march", "f64") is None
    monkeypatch.setattr(bench, "step_kernel_digest", lambda kernel="march": "def")
    assert bench.profile_traffic("march", "f32") is None


def test_committed_profiles_describe_the_current_kernels():
    """The step kernel's and the batched kernel's ncu summaries were taken on the current
    sources: after a change to them, capture their DRAM bytes again (profiles/*.md give
    the commands) before the bench can report traffic."""
    import bench
    assert bench.profile_traffic("march", "f32") is not None, "profiles/march_kernel_reactive2d.md"
    assert bench.profile_traffic("batch", "traffic_bytes_per_step_f32") is not None, \
        "profiles/batch_kernel_batched.md"


REPO = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CONTRACT = ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
            "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
            "cpu_baseline", "e2e")


def _json_lines(stdout):
    import json
    return [json.loads(l) for l in stdout.splitlines() if l.strip().startswith("{")]


def _run(cmd, timeout=600):
    import subprocess
    import sys
    env = dict(os.environ, OMP_NUM_THREADS="2")
    return subprocess.run([sys.executable] + cmd, cwd=REPO, env=env, capture_output=True,
                          text=True, timeout=timeout)


def test_reference_arm_prints_one_contract_line():
    """bench.py --impl reference times the FP64 oracle on the host cores and prints one
    JSON line with the keys of the bench contract; its e2e moves no bytes."""
    r = _run(["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"])
    assert r.returncode == 0, r.stderr[-2000:]
    (d,) = _json_lines(r.stdout)
    assert all(k in d for k in CONTRACT), [k for k in CONTRACT if k not in d]
    assert d["impl"] == "reference" and d["value"] > 0 and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 2
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["e2e"]["d2h_bytes_per_step"] == 0 and d["e2e"]["unit"] == d["unit"]


def test_reference_arm_under_two_ranks_prints_once():
    """Launched as the driver launches N > 1 (torchrun, one process per rank), rank 0 alone
    runs the oracle and prints; the other rank exits 0 without work."""
    r = _run(["-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
              "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
              "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"])
    assert r.returncode == 0, r.stderr[-2000:]
    (d,) = _json_lines(r.stdout)
    assert d["impl"] == "reference" and d["n_gpus"] == 2
