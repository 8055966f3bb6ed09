"""Host-side checks of bench.py that need no GPU.

The roofline's `traffic` comes from an ncu capture recorded with the source
key of the captured kernel; the key must change with any edit of the
kernel's code (the file or a header it includes) and must not change with
an edit of its comments or blank lines.
"""
import os
import shutil

import bench


def _copy_sources(tmp_path):
    src = os.path.join(bench.ROOT, "paper_2609_28519_gb300", "csrc")
    dst = tmp_path / "paper_2609_28519_gb300" / "csrc"
    dst.mkdir(parents=True)
    for names in bench.KERNEL_SOURCES.values():
        for name in names:
            shutil.copy(os.path.join(src, name), dst / name)
    return dst


def test_source_key_tracks_code_not_comments(tmp_path, monkeypatch):
    dst = _copy_sources(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    key = bench.source_key("k_fused<16,16,FWD,tiled>")
    assert key == bench.source_key("k_fused<16,16,INV,tiled>")  # one key per kernel family

    kernel = dst / "fp32_fused.cu"
    text = kernel.read_text()
    kernel.write_text("// a new comment line\n\n" + text.replace("{\n", "{  // trailing comment\n", 1))
    assert bench.source_key("k_fused<16,16,FWD,tiled>") == key

    kernel.write_text(text.replace("{\n", "{ (void)0;\n", 1))
    assert bench.source_key("k_fused<16,16,FWD,tiled>") != key

    kernel.write_text(text)
    header = dst / "dct_cores.cuh"
    header.write_text(header.read_text() + "\nstatic const int kProbe = 1;\n")
    assert bench.source_key("k_fused<16,16,FWD,tiled>") != key
    # the tensor-core kernel does not include the 1D cores
    tc = bench.source_key("k_tc_split<16,tiled>")
    header.write_text(header.read_text().replace("\nstatic const int kProbe = 1;\n", "\nstatic const int kProbe = 2;\n"))
    assert bench.source_key("k_tc_split<16,tiled>") == tc


def test_dominant_kernel_names_the_route_the_image_takes(tmp_path, monkeypatch):
    """The 2048^2 image of 16 x 16 blocks is 1024 chunks of 16 tiles: with
    at least 1024 / 7 SMs they fit one wave of the one-wave kernel's 7 CTAs
    per SM, so the FP32 route runs that kernel; with fewer it is the
    persistent kernel."""
    assert bench.dominant_kernel(1, "FWD", 152) == "k_strip16_wave<FWD>"
    assert bench.dominant_kernel(1, "INV", 147) == "k_strip16_wave<INV>"
    assert bench.dominant_kernel(1, "FWD", 400) == "k_strip16_wave<FWD>"
    assert bench.dominant_kernel(1, "FWD", 146) == "k_fused<16,16,FWD,tiled>"   # 1022 < 1024 chunks
    assert bench.dominant_kernel(3, "INV", 152) == "k_tc_split<16,16,INV,tiled>"
    assert bench.dominant_kernel(2, "FWD", 152) == "dense<16,16,FWD,tiled>"
    # one source key for the whole file; no record for a kernel without sources
    assert bench.source_key("k_strip16_wave<FWD>") == bench.source_key("k_fused<16,16,FWD,tiled>")
    assert bench.traffic_from_profiles("dense<16,16,FWD,tiled>") is None
    # a record whose key is stale is not used
    prof = tmp_path / "profiles"
    prof.mkdir()
    key = bench.source_key("k_strip16_wave<FWD>")
    (prof / "traffic_per_launch.txt").write_text(
        f"# header\nk_strip16_wave<FWD> 123 {key} 456\nk_strip16_wave<INV> 789 0000000000000000 1\n")
    _copy_sources(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_from_profiles("k_strip16_wave<FWD>") == 123.0
    assert bench.traffic_from_profiles("k_strip16_wave<FWD>", 3) == 456.0
    assert bench.traffic_from_profiles("k_strip16_wave<INV>") is None



def _rank_main(rank, world, port, ms_local, out_q):
    import os
    import sys
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    import bench as b
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = b._dist_env()
        dist.barrier()
        ms = b.job_time_ms(ms_local, w)
        out_q.put((r, w, local, ms, b.job_value_gbs(ms, 100, 1 << 26, w)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_max_time_and_whole_job_value():
    """world_size 2 over gloo on CPU: every rank takes the slower rank's time,
    and the value counts both ranks' steps over that time."""
    import multiprocessing as mp
    import socket
    with socket.socket() as sck:
        sck.bind(("127.0.0.1", 0))
        port = sck.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = {0: 12.5, 1: 20.0}
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, times[r], q)) for r in (0, 1)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, world, local, ms, value) in enumerate(got):
        assert (rank, world, local) == (r, 2, r)
        assert ms == 20.0
        assert abs(value - 2 * 100 * (1 << 26) / 20e-3 / 1e9) < 1e-6


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    """Under torchrun the reference arm runs on rank 0 only; the other ranks
    return 0 at once (no oracle, no output)."""
    import argparse
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.run_reference(argparse.Namespace(steps=1, warmup=1)) == 0
