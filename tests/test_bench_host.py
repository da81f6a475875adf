"""Host logic of bench.py: replica aggregation over ranks (gloo, 2 processes
on the CPU), the clock-sample parser and the reference arm's JSON contract."""

import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, fl = 10.0 + rank, 100.0 * (rank + 1)
    res = bench.reduce_max_sum([t, fl], ["max", "sum"], None)
    out[rank] = res
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_gloo():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        assert out[r] == [11.0, 300.0]


def test_reduce_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max_sum([1.5, 2.0], ["max", "sum"]) == [1.5, 2.0]


def test_clock_parser():
    sys.path.insert(0, ROOT)
    import bench

    class FakeProc:
        def terminate(self):
            pass

        def communicate(self, timeout=None):
            lines = ["0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active",
                     "0, 1900, 2070, 1300.0, 0x4, Not Active, Not Active, Not Active, Active",
                     "0, 2070, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
            return "\n".join(lines), ""

    cs = bench.ClockSampler(0)
    cs.proc = FakeProc()
    r = cs.stop()
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]


@pytest.mark.slow
def test_reference_arm_json_line():
    env = dict(os.environ, OMP_NUM_THREADS="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0", "--workload", "fp64_gmres30_16cube"],
                       capture_output=True, text=True, env=env, timeout=600)
    assert p.returncode == 0, p.stderr
    line = json.loads(p.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "GFLOP/s"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["value"] > 0


def test_gs_traffic_only_for_unchanged_kernel_sources(monkeypatch):
    import bench
    monkeypatch.setitem(bench.GS_TRAFFIC, "bytes_per_launch", 1.0e6)
    monkeypatch.setitem(bench.GS_TRAFFIC, "sources_sha256", "0" * 64)
    assert bench.gs_traffic() is None
    monkeypatch.setitem(bench.GS_TRAFFIC, "sources_sha256", bench.gs_sources_sha256())
    assert bench.gs_traffic() == 1.0e6
    assert bench.gs_traffic("mxp_gmres50_320cube") is None
    monkeypatch.setitem(bench.GS_TRAFFIC, "bytes_per_launch", None)
    assert bench.gs_traffic() is None


def test_gs_kernel_text_blocks_found(tmp_path, monkeypatch):
    # the hash covers the kernel and the helpers it inlines; each block must be
    # found, and an edit inside one changes the hash while one outside does not
    import bench
    sha = bench.gs_sources_sha256()
    assert sha is not None and len(sha) == 64
    for rel, start, end in bench.GS_KERNEL_TEXT:
        text = open(os.path.join(ROOT, rel)).read()
        i = text.find(start)
        assert i >= 0 and text.find(end, i + len(start)) > i
    rel, start, _ = bench.GS_KERNEL_TEXT[0]
    text = open(os.path.join(ROOT, rel)).read()
    (tmp_path / "paper_2507_11512_gb300" / "csrc").mkdir(parents=True)
    for r, _, _ in bench.GS_KERNEL_TEXT:
        dst = tmp_path / r
        if not dst.exists():
            dst.write_text(open(os.path.join(ROOT, r)).read())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / rel).write_text("// an edit outside the kernel\n" + text)
    assert bench.gs_sources_sha256() == sha
    i = text.find(start) + len(start)
    (tmp_path / rel).write_text(text[:i] + "\n// an edit inside the kernel" + text[i:])
    assert bench.gs_sources_sha256() != sha
