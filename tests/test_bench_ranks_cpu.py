"""The multi-rank path of bench.py on the CPU: two gloo ranks run the replica aggregation
(barrier, maximum of the timed region over ranks, whole-job rate) and the reference arm,
which works on rank 0 only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        dist.barrier()
        ms_local = 10.0 * (rank + 1)           # rank 1 is the slowest
        rate, ms = bench.replica_rate(64 * 5, ms_local, world, dist, device="cpu")
        total = bench.reduce_over_ranks(rank + 1.0, dist, "sum", device="cpu")
        out[rank] = (rate, ms, total)
    finally:
        dist.destroy_process_group()


def test_replica_rate_takes_the_slowest_rank():
    world, port = 2, _free_port()
    out = tmp.Manager().dict()
    tmp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for rank in range(world):
        rate, ms, total = out[rank]
        assert ms == 20.0
        assert rate == pytest.approx(world * 64 * 5 / 0.020)
        assert total == 3.0


def test_single_rank_needs_no_process_group():
    import bench
    rate, ms = bench.replica_rate(100, 50.0, 1, None)
    assert (rate, ms) == (2000.0, 50.0)
    assert bench.reduce_over_ranks(7.0, None) == 7.0


def test_reference_arm_works_on_rank_0_only(capsys):
    import sys

    import bench
    argv = sys.argv
    sys.argv = ["bench.py", "--impl", "reference", "--gpus", "2"]
    try:
        args = bench.parse()
    finally:
        sys.argv = argv
    assert bench.run_reference(args, rank=1, world=2) is None
    assert capsys.readouterr().out == ""


def test_oracle_sample_keeps_the_batch_mix():
    """The reference arm and the CPU baseline time complete sets, four of every degree M per
    step, taken in turn, so the sample keeps the batch's even mix of M and every set is
    reached."""
    import bench
    import inputs
    sets = inputs.batch_sets(64, 0)
    seen = set()
    for step in range(8):
        pick = bench.oracle_sample(sets, step, 4)
        Ms = [sets[i][0] for i in pick]
        assert sorted(set(Ms)) == sorted({M for M, _ in sets})
        assert all(Ms.count(M) == 4 for M in set(Ms))
        seen.update(pick)
    assert seen == set(range(len(sets)))


def test_profiled_figures_only_for_the_captured_kernel(tmp_path, monkeypatch):
    """The bench cites the committed ncu summary of the spread (DRAM traffic, shared-memory pipe)
    only while the kernel sources hash as at the capture and the summary names the instantiation
    the bench runs; otherwise it reports nothing rather than stale counters."""
    import hashlib
    import bench
    h = hashlib.sha256()
    for f in ("spread2d.cuh", "common.cuh", "jobset.cuh"):
        with open(os.path.join(bench.ROOT, "paper_2302_00414_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    good = h.hexdigest()[:16]
    prof_dir = tmp_path / "profiles"
    prof_dir.mkdir()
    def write(sha, kernel):
        (prof_dir / "s.md").write_text(f"kernel: {kernel}\nsource_sha256: {sha}\n"
                                       "dram_bytes_per_launch: 1000\nsmem_pipe_frac: 0.5\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # the sources are read from the real tree: point ROOT's csrc at it through a link
    os.symlink(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2302_00414_gb300"),
               tmp_path / "paper_2302_00414_gb300")
    write(good, "k_spread2d<float, 4, 0, 0>")
    assert bench.profiled("s.md", kernel="k_spread2d<float, 4, 0, 0>") == {"dram_bytes_per_launch": 1000.0,
                                                                            "smem_pipe_frac": 0.5}
    assert bench.profiled("s.md", kernel="k_spread2d<float, 4, 0, 1>") == {}
    write("0" * 16, "k_spread2d<float, 4, 0, 0>")
    assert bench.profiled("s.md", kernel="k_spread2d<float, 4, 0, 0>") == {}

