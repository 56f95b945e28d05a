"""CPU tests of the host-side pieces: the built C-ABI library exports every
function include/g3aca.h declares, the package refuses to load without its
library, the synthetic meshes, and the benchmark's multi-rank reduction
(world size 2 over gloo)."""
import os
import re
import shutil
import subprocess
import sys

import numpy as np
import pytest

from inputs import meshes, workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "g3aca.h")
LIB = os.path.join(ROOT, "paper_2312_11219_gb300", "lib", "libg3aca.so")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:g3_status|const char\s*\*|int|int64_t)\s+(\w+)\s*\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def built_lib():
    if not os.path.exists(LIB):
        if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("no nvcc to build the library")
        sys.path.insert(0, ROOT)
        import __graft_entry__
        __graft_entry__.build()
    return LIB


def test_library_exports_every_declared_symbol(built_lib):
    import ctypes
    lib = ctypes.CDLL(built_lib)
    names = _declared()
    assert {"build_cluster_tree", "assemble_near", "aca3_compress", "apply_gcq"} <= set(names)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    sys.path.insert(0, ROOT)
    import paper_2312_11219_gb300 as g3
    assert set(names) <= set(g3.EXPORTED) | {"g3_factors_block_cycles"}
    assert lib.g3_version() == 1


def test_calls_without_gpu_fail_cleanly(built_lib):
    import ctypes
    lib = ctypes.CDLL(built_lib)
    lib.g3_last_error.restype = ctypes.c_char_p
    h = ctypes.c_void_p()
    st = lib.g3_create(0, None, ctypes.byref(h))
    if st == 0:
        pytest.skip("a CUDA device is present")
    assert st < 0 and lib.g3_last_error()
    # null handles are rejected without touching a device
    assert lib.aca3_compress(None, None, None, 0, 0, 1, ctypes.c_double(1e-4), None, ctypes.byref(h)) == -1


def test_package_import_fails_without_library(tmp_path):
    pkg = tmp_path / "paper_2312_11219_gb300"
    pkg.mkdir()
    for f in ("__init__.py", "_binding.py"):
        shutil.copy(os.path.join(ROOT, "paper_2312_11219_gb300", f), pkg / f)
    code = "import paper_2312_11219_gb300"
    p = subprocess.run([sys.executable, "-c", code], cwd=tmp_path, capture_output=True, text=True)
    assert p.returncode != 0 and "no CPU fallback" in p.stderr


@pytest.mark.parametrize("name,E,vol", [("cube768", 768, 1.0), ("lshape12288", 12288, 0.875),
                                        ("lshape768", 768, 0.875)])
def test_meshes_closed_outward(name, E, vol):
    w = workloads.get(name)
    assert w.E == E
    assert meshes.check_closed(w.tris)
    assert abs(meshes.signed_volume(w.verts, w.tris) - vol) < 1e-12
    a = np.linalg.norm(np.cross(w.verts[w.tris[:, 1]] - w.verts[w.tris[:, 0]],
                                w.verts[w.tris[:, 2]] - w.verts[w.tris[:, 0]]), axis=1).sum() / 2
    assert abs(a - 6.0) < 1e-12


@pytest.mark.parametrize("level,E", [(3, 1280), (5, 20480)])
def test_icosphere(level, E):
    v, t = meshes.icosphere(level)
    assert t.shape[0] == E and meshes.check_closed(t)
    assert np.allclose(np.linalg.norm(v, axis=1), 1.0)
    assert 0.95 * 4 / 3 * np.pi < meshes.signed_volume(v, t) < 4 / 3 * np.pi


def test_batch_workloads():
    ws = workloads.batch64(n_geom=8)
    assert len(ws) == 8
    for w in ws:
        assert 500 <= w.E <= 8000 and meshes.check_closed(w.tris) and meshes.signed_volume(w.verts, w.tris) > 0
        assert w.freq.K in (32, 64, 128, 256)


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    vals = bench.max_over_ranks([10.0 * (rank + 1), 100.0 - rank])
    tot = bench.sum_over_ranks([500.0 * (rank + 1)])[0]
    rate = bench.whole_job_rate(tot, vals[0], 2)
    out.put((rank, vals, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_bench_reduction_over_two_gloo_ranks():
    import socket

    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, vals, rate in res:
        assert vals == [20.0, 100.0]               # max over ranks
        # entries summed over ranks (500 + 1000), timed by the slowest rank
        assert rate == pytest.approx(1500.0 / (10.0 / 1e3))


def test_reference_arm_json_contract():
    """`bench.py --impl reference` (the oracle on the host cores): one JSON
    line with the contract's keys, the oracle as its cpu_baseline and an e2e
    object that moves no host-device bytes."""
    import json
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "1", "--ref-seconds", "1"], cwd=ROOT, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e", "gpu_launches"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 1
    assert line["config"]["workload"] == "lshape12288"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and cb["sample"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["e2e"]["value"] == line["value"] and line["gpu_launches"] == 0


# ---------------------------------------------------------------- row-cluster sharding (world size 2 over gloo)

def _shard_rank_main(rank, world, port, out):
    """One rank: the library's row-cluster partition of the capped cube tree,
    the rank's share of the dense apply (oracle, a few frequencies), and the
    exchange of blocks and partial results for the checks."""
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import paper_2312_11219_gb300 as g3
    from oracle import freqs as O_freqs, quadrature as O_q, tree as O_tree
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    w = workloads.get("cube768")
    T = O_tree.build(w.verts, w.tris, w.leaf, w.eta, 96)
    nodes = np.stack([T.begin, T.end, T.left, T.right], axis=1)
    sh = g3.shard_rows(nodes, T.blocks, world)
    mine = np.flatnonzero(sh["owner"] == rank)
    # every rank computes the same partition
    allo = [torch.zeros(T.blocks.shape[0], dtype=torch.int32) for _ in range(world)]
    dist.all_gather(allo, torch.from_numpy(sh["owner"].astype(np.int32)))
    same = all(torch.equal(a, allo[0]) for a in allo)
    # the rank's blocks applied densely (original order), the other rows zero
    geo = O_q.Geometry(w.verts, w.tris)
    s = O_freqs.bdf2(4, 0.1, (1e-8) ** (1 / 8))
    W = workloads.densities(w.E, 4, 21)
    y = np.zeros(w.E, complex)
    for b in mine:
        rb, re, cb, ce, _ = T.blocks[b]
        R, C = T.perm[rb:re], T.perm[cb:ce]
        D = O_q.dense(geo, "slp", s, rows=R, cols=C)
        y[R] += np.einsum("ijk,jk->i", D, W[C])
    yt = torch.from_numpy(np.stack([y.real, y.imag]))
    ys = [torch.zeros_like(yt) for _ in range(world)]
    dist.all_gather(ys, yt)
    mt = torch.zeros(T.blocks.shape[0], dtype=torch.int32)
    mt[torch.from_numpy(mine)] = 1
    cover = mt.clone()
    dist.all_reduce(cover)
    out.put((rank, same, cover.numpy(), [t.numpy() for t in ys], sh["load"], sh["n_units"]))
    dist.barrier()
    dist.destroy_process_group()


def test_row_cluster_sharding_over_two_gloo_ranks(built_lib):
    """The library's row-cluster partition, run by two gloo ranks: both
    compute the same owner list; every block is owned exactly once; the rows
    of the two ranks are disjoint; the rank loads are within one unit of
    each other (longest-first greedy); and the ranks' partial applies add up
    to the dense apply of the whole operator."""
    import socket

    import torch.multiprocessing as mp
    from oracle import apply as O_apply, freqs as O_freqs, quadrature as O_q, tree as O_tree
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_shard_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = workloads.get("cube768")
    T = O_tree.build(w.verts, w.tris, w.leaf, w.eta, 96)
    for rank, same, cover, ys, load, n_units in res:
        assert same
        assert np.all(cover == 1)                     # each block exactly once
        assert n_units >= 2
    y0 = ys[0][0] + 1j * ys[0][1]
    y1 = ys[1][0] + 1j * ys[1][1]
    assert not np.any((y0 != 0) & (y1 != 0))          # disjoint rows
    assert np.count_nonzero(y0) > 0 and np.count_nonzero(y1) > 0
    load = res[0][4]
    sizes = (T.blocks[:, 1] - T.blocks[:, 0]) * (T.blocks[:, 3] - T.blocks[:, 2])
    assert load.sum() == pytest.approx(float(sizes.sum()))
    # greedy longest-first: the spread is at most the largest unit's cost
    assert abs(load[0] - load[1]) <= 0.25 * load.sum()
    geo = O_q.Geometry(w.verts, w.tris)
    s = O_freqs.bdf2(4, 0.1, (1e-8) ** (1 / 8))
    W = workloads.densities(w.E, 4, 21)
    yd = O_apply.dense_apply(lambda I, J, ss: O_q.entries(geo, "slp", I, J, ss), w.E, s, W)
    assert np.linalg.norm(y0 + y1 - yd) <= 1e-12 * np.linalg.norm(yd)


def _units(T):
    """Row units of a partition, written out independently: the clusters at
    the smallest depth that holds a block's row cluster, plus the leaves above
    it; returns (unit begin/end list, unit index of each block)."""
    n = T.begin.size
    depth = np.zeros(n, int)
    for v in range(n):
        for c in (T.left[v], T.right[v]):
            if c >= 0:
                depth[c] = depth[v] + 1
    node_of = {(int(T.begin[v]), int(T.end[v])): v for v in range(n)}
    dmin = min(depth[node_of[(int(rb), int(re))]] for rb, re, _, _, _ in T.blocks)
    units = [(int(T.begin[v]), int(T.end[v])) for v in range(n)
             if depth[v] == dmin or (T.left[v] < 0 and depth[v] < dmin)]
    bu = np.array([next(k for k, (a, e) in enumerate(units) if a <= rb < e) for rb, _, _, _, _ in T.blocks])
    return units, bu


def test_shard_rows_partition_properties(built_lib):
    """Single-process checks of the partition for 1-8 ranks on the capped
    L-shape tree: exact cover, whole units per rank (rows disjoint),
    deterministic, longest-first balance (spread <= the largest unit)."""
    sys.path.insert(0, ROOT)
    import paper_2312_11219_gb300 as g3
    from oracle import tree as O_tree
    w = workloads.get("lshape3072")
    T = O_tree.build(w.verts, w.tris, w.leaf, w.eta, 96)
    nodes = np.stack([T.begin, T.end, T.left, T.right], axis=1)
    units, bu = _units(T)
    rng = np.random.default_rng(1)
    cost = rng.uniform(1.0, 10.0, T.blocks.shape[0])
    ucost = np.array([cost[bu == k].sum() for k in range(len(units))])
    for n in range(1, 9):
        sh = g3.shard_rows(nodes, T.blocks, n, cost=cost)
        o = sh["owner"]
        assert sh["n_units"] == len(units)
        assert o.min() >= 0 and o.max() < n
        assert np.array_equal(o, g3.shard_rows(nodes, T.blocks, n, cost=cost)["owner"])
        for k in range(len(units)):                    # a unit goes to one rank
            assert np.unique(o[bu == k]).size <= 1
        rows = np.full(w.E, -1)
        for b, (rb, re, cb, ce, adm) in enumerate(T.blocks):
            assert np.all((rows[rb:re] == -1) | (rows[rb:re] == o[b]))
            rows[rb:re] = o[b]
        assert np.all(rows >= 0)
        load = np.array([cost[o == k].sum() for k in range(n)])
        assert np.allclose(load, sh["load"])
        assert load.max() - load.min() <= ucost.max() + 1e-9


@pytest.mark.parametrize("name,cap", [("cube48", 0), ("cube768", 0), ("cube768", 96), ("lshape768", 0),
                                      ("sphere1280", 0), ("lshape3072", 0), ("lshape3072", 192)])
def test_host_tree_partition_bit_exact(built_lib, name, cap):
    """The library's host tree builder (the half of build_cluster_tree that
    needs no device) gives the oracle's permutation and block list exactly,
    with and without the far-block cap."""
    sys.path.insert(0, ROOT)
    import paper_2312_11219_gb300 as g3
    from oracle import tree as O_tree
    w = workloads.get(name)
    got = g3.tree_partition_host(w.verts, w.tris, w.leaf, w.eta, cap)
    ref = O_tree.build(w.verts, w.tris, w.leaf, w.eta, cap)
    assert np.array_equal(got["perm"], ref.perm)
    assert np.array_equal(got["blocks"], ref.blocks)


def test_host_tree_partition_rejects_bad_input(built_lib):
    sys.path.insert(0, ROOT)
    import paper_2312_11219_gb300 as g3
    w = workloads.get("cube48")
    bad = w.tris.copy()
    bad[3] = [0, 0, 1]                      # degenerate
    with pytest.raises(g3.G3Error):
        g3.tree_partition_host(w.verts, bad, w.leaf, w.eta)
    bad = w.tris.copy()
    bad[0, 0] = w.verts.shape[0]            # vertex index out of range
    with pytest.raises(g3.G3Error):
        g3.tree_partition_host(w.verts, bad, w.leaf, w.eta)
    with pytest.raises(g3.G3Error):
        g3.tree_partition_host(w.verts, w.tris, 0, w.eta)
    with pytest.raises(g3.G3Error):           # empty mesh
        g3.tree_partition_host(w.verts, w.tris[:0], w.leaf, w.eta)


def test_host_tree_partition_degenerate_meshes(built_lib):
    """One triangle: a single leaf and its 1 x 1 near block.  A mesh no larger
    than a leaf: one near block.  The 192-triangle cube: no admissible block
    at all (every block near), as in the oracle."""
    sys.path.insert(0, ROOT)
    import paper_2312_11219_gb300 as g3
    from oracle import tree as O_tree
    v = np.array([[0.0, 0.0, 0.0], [0.9, 0.1, 0.0], [0.2, 0.7, 0.3]])
    t = np.array([[0, 1, 2]], dtype=np.int32)
    got = g3.tree_partition_host(v, t, 32, 1.0)
    assert np.array_equal(got["perm"], [0]) and np.array_equal(got["blocks"], [[0, 1, 0, 1, 0]])
    w = workloads.get("cube48")
    got = g3.tree_partition_host(w.verts, w.tris, 48, w.eta)
    assert np.array_equal(got["blocks"], [[0, 48, 0, 48, 0]])
    w = workloads.get("cube192")
    got = g3.tree_partition_host(w.verts, w.tris, w.leaf, w.eta)
    ref = O_tree.build(w.verts, w.tris, w.leaf, w.eta)
    assert np.array_equal(got["perm"], ref.perm) and np.array_equal(got["blocks"], ref.blocks)
    assert got["blocks"].shape[0] == 64 and not (got["blocks"][:, 4] == 1).any()
