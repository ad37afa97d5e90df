"""CPU checks of bench.py: the multi-rank aggregation over gloo (world size 2) and the reference
arm's JSON contract (the FP64 oracle on the host cores)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [120.0, 150.0][rank]            # rank 1 is the slower one
    atoms = [4_000_000, 4_000_000][rank]
    res = bench.combine_ranks(ms, atoms, steps=100)
    out.put((rank, res))
    dist.destroy_process_group()


def test_combine_ranks_gloo_world2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        ms, total, value = got[r]
        assert ms == 150.0                       # the slowest rank sets the time
        assert total == 8_000_000                # atoms of all ranks
        assert value == pytest.approx(8_000_000 * 100 / 0.150)


def test_reference_arm_json_contract():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "3",
                          "--warmup", "3", "--ref-seconds", "2"], capture_output=True, text=True, timeout=300,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "particle-timesteps/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["steps"] == 3 and d["warmup"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_do_nothing():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "3",
                          "--warmup", "3"], capture_output=True, text=True, timeout=120, cwd=ROOT, env=env)
    assert out.returncode == 0 and out.stdout.strip() == ""


def test_code_hash_ignores_comments_only(tmp_path):
    import bench
    a = tmp_path / "a.cu"
    b = tmp_path / "b.cu"
    c = tmp_path / "c.cu"
    a.write_text("// header\n__global__ void k(int* p) { p[0] = 1; /* note */ }\n")
    b.write_text("// another header\n\n__global__ void k(int* p)\n{\n    p[0] = 1;  // same code\n}\n")
    c.write_text("__global__ void k(int* p) { p[0] = 2; }\n")
    assert bench.code_hash(str(a)) == bench.code_hash(str(b))
    assert bench.code_hash(str(a)) != bench.code_hash(str(c))


class _FakeClocks:
    """Stand-in for the NVML source: a clock that drops and a power-cap reason on some samples."""

    def __init__(self):
        self.k = 0

    def sample(self):
        self.k += 1
        return (2070.0 if self.k % 3 else 1900.0), 2070.0, (0x4 if self.k % 5 == 0 else 0)


def test_clock_sampler_has_samples_for_a_short_region():
    import time
    import bench
    with bench.ClockSampler(0, period=0.001, source=_FakeClocks()) as clk:
        time.sleep(0.02)
    s = clk.summary()
    assert s["samples"] >= 3 and s["source"] == "nvml"
    assert s["sm_max_mhz"] == 2070.0 and s["sm_mhz"] in (1900.0, 2070.0)
    assert s["reasons"] in ([], ["sw_power_cap"])
    with bench.ClockSampler(0, period=0.001, source=_FakeClocks()) as clk:
        pass                                    # an empty region still has the entry and exit samples
    assert clk.summary()["samples"] >= 2
