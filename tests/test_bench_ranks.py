"""bench.py's host logic on CPU: the multi-rank path (two gloo ranks, each with its own
timing, agree on the slowest rank's time; the replicas exchange nothing else), and the
DRAM traffic taken from the committed ncu summaries."""
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
