"""The multi-rank benchmark path on CPU: two gloo ranks, as torch.distributed.run
would start them.  The path runs independent replicas (one image stream per
GPU); the only collective is the max over ranks of the timed region."""
import ctypes
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        env = bench.dist_env()
        slowest = bench.max_over_ranks(10.0 + 5.0 * rank)
        q.put((rank, env, bench.rank_seeds(rank), slowest))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [(0, 2, 0), (1, 2, 1)]
    assert all(r[3] == 15.0 for r in res)  # max over ranks, on every rank
    seeds0, seeds1 = res[0][2], res[1][2]
    assert len(set(seeds0) | set(seeds1)) == 6  # each replica has its own images


def test_single_rank_helpers():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert abs(bench.job_mpix(2, 10, 1000.0) - 2 * 1024 * 1024 * 10 / 1e6) < 1e-9
    assert bench.candidate_pairs(64, 64, R=3) == sum(
        (min(56, i + 3) - max(0, i - 3) + 1) * (min(56, j + 3) - max(0, j - 3) + 1) - 1
        for i in sorted(set(min(p * 3, 56) for p in range(20))) for j in sorted(set(min(q * 3, 56) for q in range(20))))


def test_tc_executed_flop_closed_form():
    # 1024^2, s = 3, R = 19: 340 grid rows in tiles of 16; the union of a tile's
    # windows spans 65 rows for the first tile, 84 inside, 76 for tile 20 and
    # 28 for the 4-row last tile -> 33 + 19 x 42 + 38 + 14 = 883 two-row
    # chunks per tile column, 43 tile columns, 3 x 2 x 128 x 128 x 64 FLOP each
    import bench
    assert bench.tc_executed_flop(1024, 1024) == 883 * 43 * 3 * 2 * 128 * 128 * 64


def test_launch_count_matches_launch_list():
    # one 1024^2 grayscale denoise launched 35 kernels in the ncu launch list
    # (profiles/launches_denoise_1024.md: 142 launches over 4 denoises, 2 of
    # them the bench's L2-flush fill)
    import bench
    from types import SimpleNamespace
    p = SimpleNamespace(cycle_spins=2, levels=3, stages=2, translations=1)
    assert bench.launches_per_denoise(p, 1) == 35 == (142 - 2) // 4
    assert bench.launches_per_denoise(p, 3) == 71
    # Sec. 5 preset: direct matching in both stages, 2 translations with their shifts
    q = SimpleNamespace(cycle_spins=2, levels=3, stages=2, translations=2)
    assert bench.launches_per_denoise(q, 1, (False, False)) == 2 * (1 + 7 + 15 + 2) + 2 * (1 + 7 + 2 + 3)


def test_engine_choice_mirrors_library():
    import torch
    if torch.cuda.is_available():
        pytest.skip("passes fake device pointers: runs where no GPU is visible")
    import bench
    from paper_2103_10765_gb300 import build, gbm3d
    build.build_library()
    lib = gbm3d.load()
    for preset in (0, 1):
        p = gbm3d.params_default(preset)
        for stage in (1, 2):
            g = gbm3d.params_stage(p, stage)
            K = p.k1 if stage == 1 else p.k2
            expect = bench.tc_supported(1024, 1024, g.patch, g.step, p.search_radius, K)
            q = g.replace(match_engine=2)
            if not expect:
                # engine 2 on an unsupported geometry is refused on the host, before any
                # launch (the pointers are never dereferenced)
                fake = ctypes.c_void_p(0x1000)
                st = lib.gbm3d_match(fake, 1024, 1024, 1024, ctypes.byref(q), K, fake, None, None, None)
                assert st == gbm3d.EUNSUPPORTED, (preset, stage)
    assert bench.tc_supported(1024, 1024, 8, 3, 19, 16) and bench.tc_supported(1024, 1024, 8, 3, 19, 32)
    assert not bench.tc_supported(1024, 1024, 8, 8, 16, 16) and not bench.tc_supported(1024, 1024, 16, 16, 16, 16)


def test_clock_sampler_keeps_only_timed_window(tmp_path, monkeypatch):
    """The bench's clock record holds the samples taken while the timed region ran:
    a fake nvidia-smi reports 1000 MHz before the region and 2070 MHz with
    sw_power_cap during it."""
    import time

    import bench
    flag = tmp_path / "in_region"
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\n"
                    f"while true; do if [ -e {flag} ]; then "
                    "echo '0, 2070, 2070, 900.0, Not Active, Not Active, Not Active, Active'; "
                    "else echo '0, 1000, 2070, 100.0, Not Active, Not Active, Not Active, Not Active'; fi; "
                    "sleep 0.05; done\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}:{os.environ['PATH']}")
    with bench.ClockSampler(0) as clk:
        assert clk.stamped, "sampler did not start"
        flag.touch()
        time.sleep(0.12)
        clk.mark_start()
        time.sleep(0.4)
        clk.mark_end()
        flag.unlink()
        time.sleep(0.15)
    s = clk.summary()
    assert s["samples"] >= 4
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
