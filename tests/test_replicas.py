"""The multi-GPU path of bench.py is replicas only: every rank solves its own copy of the
workload and only the step time is reduced (maximum over ranks).  Checked here with two gloo
ranks on the CPU, and the reference arm's rule that ranks other than 0 do no work."""

import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t, v = bench.job_rate(2.0 + 3.0 * rank, 256, world, dist, "cpu")  # ranks take 2 ms and 5 ms
        q.put((rank, t, v))
    finally:
        dist.destroy_process_group()


def test_job_rate_takes_the_slowest_rank_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, v in res:
        assert t == 5.0
        assert v == pytest.approx(2 * 256 / 5e-3)


def test_ranks_solve_distinct_energies_covering_the_grid():
    sys.path.insert(0, ROOT)
    import numpy as np

    import bench
    import workloads as w

    np.testing.assert_array_equal(bench.rank_energies(3.0, 256, 0, 1), w.WORKLOADS["ci2d_batched"]["eps"])
    for world in (2, 4, 8):
        parts = [bench.rank_energies(3.0, 256, r, world) for r in range(world)]
        assert all(p.size == 256 for p in parts)
        allp = np.sort(np.concatenate(parts))
        np.testing.assert_allclose(allp, w.eps_grid(3.0, 256 * world), rtol=0, atol=0)
        assert all(p.min() < 0.1 and p.max() > 2.9 for p in parts)  # each rank spans the range


def test_job_rate_single_rank():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.job_rate(4.0, 100, 1) == (4.0, 100 / 4e-3)


def test_reference_arm_ranks_other_than_zero_do_no_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True, env=env, timeout=300)
    assert out.returncode == 0
    assert out.stdout.strip() == ""


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` (the CPU oracle on a bounded sample of the benchmark workload)
    prints one JSON line with the contract's keys, its own metric/unit and zero copy bytes."""
    import json
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, check=True, cwd=root, timeout=600).stdout
    lines = [l for l in out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] == os.cpu_count()  # the oracle runs over every host core
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in d["config"]


def test_bench_level_helpers_match_the_oracle():
    """The bench's main leg forms total energies and open final levels without the oracle; its
    host helpers agree with the oracle's definitions (Eq. Econserv, open channels E_vf < E)."""
    sys.path.insert(0, ROOT)
    import bench
    import workloads
    from oracle import vibronic as o

    for desc, vi in ((workloads.ci2d_model(12), [1, 2]), (workloads.co2_like_model(basis=(4, 3, 3, 2)), [1, 0, 2, 1])):
        for eps in (0.05, 0.7, 2.9):
            E = eps + bench.level_energy(desc, vi)
            assert abs(E - o.total_energy(desc, eps, vi)) < 1e-12
            assert bench.open_final_levels(desc, E) == [list(map(int, v)) for v in o.open_levels(desc, E)]


def test_bench_stencil_point_count_matches_the_oracle_operator():
    """The FP64 roofline of the bench counts 4 flops per stencil point; its point count equals the
    off-diagonal nonzeros of an interior row of the oracle's A (CI2D terms have distinct offsets)."""
    sys.path.insert(0, ROOT)
    import numpy as np

    import bench
    import workloads
    from oracle import vibronic as o

    desc = workloads.ci2d_model(12)
    A = o.a_matrix(desc, 3.0).tocsr()
    n_g, n_u = (m["n"] for m in desc["modes"])
    counts = []
    for d in range(desc["n_states"]):
        row = d * n_g * n_u + (n_g // 2) * n_u + n_u // 2  # an interior element of state d
        counts.append(A.indptr[row + 1] - A.indptr[row] - 1)
    assert max(counts) == bench.stencil_points(desc) == 8
