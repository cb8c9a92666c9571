"""Host-side logic of bench.py: multi-rank aggregation over gloo (world size 2,
CPU), the reference arm's JSON line, and the roofline bookkeeping."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    bench.dist_setup("gloo")
    # rank r "took" 1 + r seconds for 1000 units
    thr, tmax = bench.aggregate(1000, 1.0 + rank)
    bench.barrier()
    with open(os.path.join(out, f"r{rank}.json"), "w") as f:
        json.dump({"thr": thr, "tmax": tmax, "max": bench.reduce_max(float(rank * 10))}, f)
    dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = 29500 + os.getpid() % 1000
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        d = json.load(open(tmp_path / f"r{r}.json"))
        # whole-job throughput: units of all ranks over the slowest rank's time
        assert d["tmax"] == 2.0
        assert d["thr"] == pytest.approx(2000 / 2.0)
        assert d["max"] == 10.0


def _shard_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import numpy as np
    import torch.distributed as dist
    bench.dist_setup("gloo")
    w, _ = bench.workload_for_rank(2, rank, world, "elements")
    np.savez(os.path.join(out, f"s{rank}.npz"), q=w.q, g=w.mesh.g, Jinv=w.mesh.Jinv,
             rho_ref=w.rho_ref, rhotheta_ref=w.rhotheta_ref)
    bench.barrier()
    dist.destroy_process_group()


def test_element_sharding_partitions_one_mesh(tmp_path):
    """Two gloo ranks take contiguous element ranges that cover the mesh once,
    and their workloads are, point for point, the whole mesh's."""
    import numpy as np
    import torch.multiprocessing as mp
    from paper_1604_08501_gb300 import workload as wl
    ranges = bench.shard_ranges(2, 2)
    assert ranges == [(0, 2), (2, 4)]
    for world in (1, 3, 4):
        r = bench.shard_ranges(5, world)
        assert r[0][0] == 0 and r[-1][1] == 5 * world
        assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
        assert len({b - a for a, b in r}) == 1
    port = 29600 + os.getpid() % 1000
    mp.spawn(_shard_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    whole = wl.make_workload(7, (2, 2, 4), seed=1)
    parts = [np.load(tmp_path / f"s{r}.npz") for r in range(2)]
    assert sum(p["q"].shape[1] for p in parts) == whole.M
    for name, ref in (("q", whole.q), ("g", whole.mesh.g), ("Jinv", whole.mesh.Jinv),
                      ("rho_ref", whole.rho_ref), ("rhotheta_ref", whole.rhotheta_ref)):
        assert np.array_equal(np.concatenate([p[name] for p in parts], axis=-1), ref), name


def test_single_process_aggregate_is_identity():
    thr, tmax = bench.aggregate(500, 2.0)
    assert (thr, tmax) == (250.0, 2.0)


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--n", "3", "--steps", "2", "--warmup", "3"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "GDOF/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["higher_is_better"] is True


def test_roofline_entries_pick_the_binding_bound():
    from paper_1604_08501_gb300 import workload as wl
    w = wl.make_workload(7, 1, seed=0)
    roof, other = bench.roofline_entries("vol_rhs_fp64_kernel<8>", 1.0, w)
    assert roof["bound"] == "alu" and other["bound"] == "hbm"
    roof, other = bench.roofline_entries("vol_rhs_df64_kernel<8>", 1.0, w)
    assert roof["bound"] == "hbm"
    assert roof["achieved"] == pytest.approx(176 * w.M / 1e-3 / 1e9)


def test_cpu_baseline_records_all_cores_and_one_core():
    from paper_1604_08501_gb300 import workload as wl
    w = wl.make_workload(2, 4, seed=1)
    d = bench.cpu_baseline(w, parity_w=wl.make_workload(1, 2, seed=0))
    assert d["kind"] == "oracle" and d["value"] > 0 and d["cores"] >= 1
    assert d["single_core"]["cores"] == 1 and d["single_core"]["value"] > 0
    assert d["parity_workload"]["points"] == 8 * 8 and d["parity_workload"]["value"] > 0
    assert isinstance(d["cpu_model"], str) and d["cpu_model"]


def test_traffic_record_is_dropped_once_a_source_changes(tmp_path, monkeypatch):
    # A DRAM-traffic record counts only while the kernel's sources hash as they
    # did when the counters were taken; comment edits do not count as changes.
    src = tmp_path / "k.cu"
    src.write_text("__global__ void k(float *x) { x[0] = 1.f; }  // first\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "profiles").mkdir()
    rec = {"k": {"dram_bytes_per_launch": 123.0, "sources": ["k.cu"],
                 "sources_sha": bench.sources_sha(["k.cu"])}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    assert bench.load_traffic("k") == 123.0
    src.write_text("/* a note */ __global__ void k(float *x) {\n x[0] = 1.f; }  // edited\n")
    assert bench.load_traffic("k") == 123.0
    assert bench.load_traffic("other") is None
    src.write_text("__global__ void k(float *x) { x[0] = 2.f; }\n")
    assert bench.load_traffic("k") is None
