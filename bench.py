"""Benchmark of the three-way ACA hot path on one or more GB300s.

One step = one pass of the whole path on the workload's synthetic input:
cluster tree + cluster-order geometry, the frequency set, and for each
operator (single and double layer) the near-field assembly, the three-way
ACA of every admissible block (one persistent launch) and the apply to the
seeded densities at all frequencies.

Metric: ENTRY evaluations per second (rows, columns and fibers of the
three-way ACA plus the near field), with the apply's GB/s alongside.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
    python bench.py --impl reference ...   (the CPU oracle on the host cores)

Multi-GPU: one problem divided by row clusters (g3_shard_rows /
g3_tree_subset): each rank assembles, compresses and applies the blocks of
its row clusters, with disjoint output rows and no collective on the data
path (strong scaling); the timed region is bracketed by barriers, the step
time is the maximum over ranks and the entries are summed over ranks.

Workloads: lshape12288 (default), lshape12288_nocap, sphere20480 (Galerkin),
sphere81920, batch64 (64 meshes in one compression launch per operator).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "3-way ACA entries/s & apply GB/s (1 GB300); learned+batched vs plain at 1e-4"

# special-function-unit operations per collocation entry: 7 quadrature points,
# each one rsqrt, one ex2, one sin and one cos (Galerkin: 16 points)
# DRAM bytes (read + write) per low-rank k_aca3 launch of the 12,288-triangle
# L-shape, mean of the single and double layer, from one ncu capture of each
# operator's launch (dram__bytes_read.sum + dram__bytes_write.sum: 36.8 GB and
# 41.8 GB) of the current kernel; other workloads have no capture (null)
ACA_TRAFFIC_BYTES = {"lshape12288": 0.5 * (19234748160 + 17581539072 + 23269448960 + 18566676224)}
# DRAM bytes (read + write) of one apply of each operator of the same workload
# (every kernel of apply_gcq, from one ncu capture per operator: 7,131.4 MB
# single layer, 6,899.9 MB double layer); the bench's steady-state apply bytes
# are the same sum over both operators
APPLY_TRAFFIC_BYTES = {"lshape12288": 7131350656 + 6899897472}
MUFU_PER_ENTRY = 28
MUFU_PER_ENTRY_GALERKIN = 64
# special-function-unit results per clock per SM for rsqrt / sin / cos
SFU_PER_CLK_SM = 16


def _peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        d["source"] = "measured"
        return d
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0,
            "source": "fallback"}


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        # raw samples: G3_CLOCKS_DIR if set, else the temporary directory (the
        # JSON line carries their summary)
        import tempfile
        self.path = os.path.join(os.environ.get("G3_CLOCKS_DIR") or tempfile.gettempdir(),
                                 f"clocks_rank{index}_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self) -> dict:
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle legs: timing (cpu_baseline and the reference arm) and the error
# of the timed GPU results against the float64 oracle
# ---------------------------------------------------------------------------

_ORACLE_CACHE: dict = {}


def mesh_list(name: str):
    """The workload's meshes: one, or the 64 of the batched workload."""
    from inputs import workloads
    if name == "batch64":
        return workloads.batch64()
    return [workloads.get(name)]


def _oracle_setup(name: str):
    """(workload, geometry, tree, frequency set) of a mesh; `name` is a
    workload name or "batch64[g]" for mesh g of the batch."""
    if name not in _ORACLE_CACHE:
        from oracle import freqs as O_freqs, quadrature as O_q, tree as O_tree
        if name.startswith("batch64["):
            w = mesh_list("batch64")[int(name[8:-1])]
        else:
            w = mesh_list(name)[0]
        geo = O_q.Geometry(w.verts, w.tris)
        T = O_tree.build(w.verts, w.tris, w.leaf, w.eta, w.max_block)
        fs = O_freqs.frequency_set(w.freq)
        _ORACLE_CACHE[name] = (w, geo, T, fs)
    return _ORACLE_CACHE[name]


def _entry_fn(w, geo, ker):
    """The oracle's ENTRY(I, J, s) of the workload's scheme."""
    if w.scheme == "colloc7":
        from oracle import quadrature as O_q
        return lambda I, J, s: O_q.entries(geo, ker, I, J, s)
    from oracle import galerkin as O_g
    return lambda I, J, s: O_g.entries(w.verts, w.tris, I, J, s)


def _oracle_job(job):
    """One unit of oracle work: compress far block b of operator `ker` (or
    evaluate near block b at every unique frequency).  Returns entries."""
    import numpy as np
    from oracle import aca3 as O_aca
    name, ker, b = job
    w, geo, T, fs = _oracle_setup(name)
    su = fs["s"][fs["uniq"]]
    rb, re, cb, ce, adm = T.blocks[b]
    ef = _entry_fn(w, geo, ker)
    if adm:
        op = O_aca.BemBlock(ef, T.perm[rb:re], T.perm[cb:ce], su)
        O_aca.aca3(op, w.eps3, s_abs=np.abs(su))
        return int(op.generated)
    R, C = T.perm[rb:re], T.perm[cb:ce]
    I = np.repeat(R, C.size)
    J = np.tile(C, R.size)
    ef(I, J, su)
    return int(I.size * su.size)


def _oracle_warm(names):
    for n in names:
        _oracle_setup(n)
    return os.getpid()


def _mesh_names(name: str, n_mesh: int) -> list[str]:
    return [f"batch64[{g}]" for g in range(n_mesh)] if name == "batch64" else [name]


def oracle_sample(name: str, seconds: float, seed: int, cores: int) -> dict:
    """Oracle entries/s on a seeded random sample of the workload's blocks
    (far blocks through the oracle's three-way ACA, near blocks through its
    dense quadrature, in the workload's far/near proportion; for the batch,
    blocks of eight seeded meshes), run on a spawn pool of `cores` processes
    for about `seconds` of wall time."""
    import multiprocessing as mp

    import numpy as np
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    rng = np.random.default_rng(seed)
    names = _mesh_names(name, 64)
    if len(names) > 1:
        names = [names[int(g)] for g in np.sort(rng.choice(len(names), 8, replace=False))]
    setups = {n: _oracle_setup(n) for n in names}
    jobs = []
    for i in range(100000):
        n = names[i % len(names)]
        w, geo, T, fs = setups[n]
        ker = w.kernels[(i // len(names)) % len(w.kernels)]
        far = np.nonzero(T.blocks[:, 4] == 1)[0]
        near = np.nonzero(T.blocks[:, 4] == 0)[0]
        pick_far = rng.random() < far.size / (far.size + near.size)
        b = int(rng.choice(far if pick_far else near))
        jobs.append((n, ker, b))
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_warm, [names] * cores)
        t0 = time.perf_counter()
        entries = 0
        done = 0
        it = pool.imap_unordered(_oracle_job, jobs, chunksize=1)
        for e in it:
            entries += e
            done += 1
            if time.perf_counter() - t0 > seconds:
                break
        wall = time.perf_counter() - t0
        pool.terminate()
    kers = "/".join(setups[names[0]][0].kernels)
    return {"value": entries / wall, "unit": "entries/s", "cores": cores, "kind": "oracle",
            "sample": f"{done} seeded random blocks of {name} ({kers}; far blocks through the "
                      f"oracle's three-way ACA, near blocks densely), {wall:.1f} s wall",
            "entries": entries, "seconds": wall}


def _dense_row_job(job):
    """y_ref[i] = sum_l sum_j A(s_l)[i, j] W[j, l] of one row (original order),
    optionally restricted to the column ranges of a block list."""
    import numpy as np
    from oracle import apply as O_apply
    from inputs import workloads
    name, ker, i, seed, cols = job
    w, geo, T, fs = _oracle_setup(name)
    key = ("W", name, seed)
    if key not in _ORACLE_CACHE:   # the seeded densities, regenerated in the worker
        _ORACLE_CACHE[key] = workloads.densities(w.E, w.freq.K, seed)
    W = _ORACLE_CACHE[key]
    ef = _entry_fn(w, geo, ker)
    if cols is None:
        return O_apply.dense_apply(ef, w.E, fs["s"], W, rows=[i])[0]
    A = ef(np.full(cols.size, i), cols, fs["s"])
    return np.sum(A * W[cols, :])


def oracle_rows(jobs, cores: int) -> list:
    import multiprocessing as mp
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        return pool.map(_dense_row_job, jobs, chunksize=1)


def apply_errors(name: str, kernels, ys: dict, seeds: list, n_rows: int, seed: int, cores: int) -> dict:
    """Relative error ||y - y_ref|| / ||y_ref|| of the timed run's applies on
    seeded sampled rows against the float64 oracle's dense apply (every entry
    at all K frequencies), per operator (and per mesh of a batch: three
    seeded meshes)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    names = _mesh_names(name, len(seeds))
    picks = list(range(len(names))) if len(names) == 1 else sorted(rng.choice(len(names), 3, replace=False).tolist())
    out = {}
    for ker in kernels:
        for g in picks:
            w = _oracle_setup(names[g])[0]
            rows = np.sort(rng.choice(w.E, min(n_rows, w.E), replace=False))
            ref = np.array(oracle_rows([(names[g], ker, int(i), seeds[g], None) for i in rows], cores))
            got = ys[(ker, g)][rows]
            key = ker if len(names) == 1 else f"{ker}[{g}]"
            out[key] = {"rel_err": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)), "rows": int(rows.size)}
    return out


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def max_over_ranks(values: list[float], device=None) -> list[float]:
    """Element-wise maximum of `values` over all ranks (identity for one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return list(values)
    t = torch.tensor(values, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def sum_over_ranks(values: list[float], device=None) -> list[float]:
    """Element-wise sum of `values` over all ranks (identity for one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return list(values)
    t = torch.tensor(values, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return [float(x) for x in t.cpu()]


def whole_job_rate(units_all_ranks: float, ms_max: float, steps: int) -> float:
    """Units processed by all ranks per second, timed by the slowest rank."""
    return units_all_ranks / ((ms_max / steps) / 1e3)


def train_predictor(g3, ctx, kernels, prec):
    """Block predictor trained on the compressions of configurations 1-3
    (the 768-triangle cube, the 12,288-triangle L-shape with both operators,
    the 20,480-triangle Galerkin icosphere): features and labels from the
    library, training on the GPU."""
    import time

    import numpy as np

    from inputs import workloads
    X, Y = [], []
    for name in ("cube768", "lshape12288", "sphere20480"):
        w = workloads.get(name)
        T = g3.build_cluster_tree(ctx, w.verts, w.tris, w.leaf, w.eta, max_block=w.max_block)
        F = g3.freqs_from_spec(ctx, w.freq)
        for ker in w.kernels:
            fa = g3.aca3_compress(ctx, T, F, ker, scheme=w.scheme, prec=prec, eps3=w.eps3)
            X.append(g3.block_features(ctx, T, F, ker, w.eps3))
            Y.append(fa.labels())
    X, Y = np.concatenate(X), np.concatenate(Y)
    t0 = time.perf_counter()
    net = g3.mlp_train(ctx, X, Y, epochs=150, batch=256, seed=1)
    secs = time.perf_counter() - t0
    p = net.predict(X)
    return net, {"samples": int(X.shape[0]), "epochs": 150, "seconds": secs,
                 "mae_log2_r3": float(np.abs(p[:, 0] - Y[:, 0]).mean()),
                 "data": "cube768 + lshape12288 (slp, dlp) + sphere20480 (Galerkin) compressions"}


def plain_vs_batched(g3, ctx, w, T, F, ker, n_blocks: int, seed: int, prec: str, eps_plain: float,
                     eps_ours: float, mlp=None, mlp_use=0, shape=None) -> dict:
    """The same seeded sample of far blocks (stratified by block size),
    compressed by the plain arm (float64, one block per launch) and by ours
    (the timed configuration: mixed precision, one persistent launch,
    predictor); device times and the subset trees for the error leg."""
    import numpy as np
    tg = T.get()
    far = tg["far_index"]
    sizes = (tg["blocks"][far, 1] - tg["blocks"][far, 0]) * (tg["blocks"][far, 3] - tg["blocks"][far, 2])
    rng = np.random.default_rng(seed)
    order = np.argsort(sizes, kind="stable")
    strata = np.array_split(order, 8)
    per = max(1, n_blocks // len(strata))
    pick = np.sort(np.concatenate([rng.choice(s, min(per, s.size), replace=False) for s in strata if s.size]))
    owner = np.ones(tg["blocks"].shape[0], dtype=np.int32)
    owner[far[pick]] = 0
    S = g3.tree_subset(ctx, T, owner, 0)
    plain = g3.aca3_compress(ctx, S, F, ker, scheme=w.scheme, prec="fp64", eps3=eps_plain, unbatched=1)
    ours = g3.aca3_compress(ctx, S, F, ker, scheme=w.scheme, prec=prec, eps3=eps_ours, mlp=mlp, mlp_use=mlp_use,
                            **(shape or {}))
    ps, os_ = plain.stats(), ours.stats()
    return {"tree": S, "plain": plain, "ours": ours, "blocks": int(pick.size),
            "plain_ms": ps["ms"], "ours_ms": os_["ms"], "plain_entries": ps["entries"], "ours_entries": os_["entries"],
            "plain_crosses": ps["crosses"], "ours_crosses": os_["crosses"]}


def run_ours(args, rank: int, world: int, local_rank: int) -> dict | None:
    import numpy as np
    import torch

    import paper_2312_11219_gb300 as g3
    from inputs import workloads

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    ws = mesh_list(args.workload)
    batch = len(ws) > 1
    kernels = list(ws[0].kernels)
    scheme = ws[0].scheme
    Ws = [workloads.densities(w.E, w.freq.K, w.density_seed) for w in ws]
    Wds = [torch.from_numpy(W).to(dev) for W in Ws]
    stream = torch.cuda.current_stream(dev)
    ctx = g3.Context(local_rank, stream.cuda_stream)
    prec = args.precision
    keep = {}

    # the learned part: a predictor trained (untimed, like any model) on the
    # compressions of the smaller configurations, used by every timed compression
    net, train_info = None, None
    if args.mlp_use:
        net, train_info = train_predictor(g3, ctx, kernels, prec)

    def make_tree(w):
        """The mesh's tree; with several ranks, this rank's row-cluster shard."""
        T = g3.build_cluster_tree(ctx, w.verts, w.tris, w.leaf, w.eta, max_block=w.max_block)
        if world == 1:
            return T
        tg = T.get()
        sh = g3.shard_rows(tg["nodes"], tg["blocks"], world)
        return g3.tree_subset(ctx, T, sh["owner"], rank)

    # launch shape per operator from the autotuner (untimed; cached in the context)
    tune = {}
    if not args.no_autotune and not batch:
        T0 = make_tree(ws[0])
        F0 = g3.freqs_from_spec(ctx, ws[0].freq)
        for ker in kernels:
            tune[ker] = g3.autotune(ctx, T0, F0, ker, scheme=scheme, prec=prec, eps3=ws[0].eps3)
        del T0, F0

    def step(host: bool, mlp=None, mlp_use=0):
        trees = [make_tree(w) for w in ws]
        freqs = [g3.freqs_from_spec(ctx, w.freq) for w in ws]
        rec = {"entries_aca": 0, "entries_face_dense": 0, "entries_near": 0, "aca_ms": 0.0, "near_ms": 0.0, "apply_ms": 0.0,
               "apply_near_ms": 0.0, "apply_bytes": 0, "apply_near_bytes": 0, "factor_bytes": 0,
               "dense_bytes": 0, "crosses": 0, "stats": {}}
        for ker in kernels:
            keep.pop(ker, None)   # the previous step's operator first: two at once do not fit the largest workloads
            nfs = [g3.assemble_near(ctx, T, F, ker, scheme=scheme, prec=prec) for T, F in zip(trees, freqs)]
            shape = {k: tune[ker][k] for k in ("threads", "dense_face_max", "residual_face_max")} if ker in tune else {}
            if batch:
                fas = g3.aca3_compress_batch(ctx, trees, freqs, ker, scheme=scheme, prec=prec, eps3=ws[0].eps3,
                                             mlp=mlp, mlp_use=mlp_use)
            else:
                fas = [g3.aca3_compress(ctx, trees[0], freqs[0], ker, scheme=scheme, prec=prec, eps3=ws[0].eps3,
                                        mlp=mlp, mlp_use=mlp_use, **shape)]
            ys = []
            for g, (T, nf, fa) in enumerate(zip(trees, nfs, fas)):
                ys.append(g3.apply_gcq(ctx, T, nf, fa, Ws[g] if host else Wds[g]))
                la = ctx.last_apply()
                rec["apply_ms"] += la["ms"]
                rec["apply_near_ms"] += la["near_ms"]
                rec["apply_bytes"] += la["bytes"]
                rec["apply_near_bytes"] += la["near_bytes"]
            st = fas[0].stats()           # a batch's times and entries are the whole launch's
            rec["entries_aca"] += st["entries"]
            rec["entries_face_dense"] += st["entries_face_dense"]
            rec["aca_ms"] += st["ms"]
            for nf in nfs:
                ni = nf.info()
                rec["entries_near"] += ni["entries"]
                rec["near_ms"] += ni["ms"]
            for fa in fas:
                sf = fa.stats()
                rec["factor_bytes"] += sf["factor_bytes"]
                rec["dense_bytes"] += sf["dense_bytes"]
                rec["crosses"] += sf["crosses"]
            rec["stats"][ker] = st
            keep[ker] = (trees, freqs, nfs, fas, ys)
        return rec

    def timed(n: int, host: bool):
        recs = []
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n):
            recs.append(step(host, net, args.mlp_use))
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        return recs, e0.elapsed_time(e1)

    for _ in range(args.warmup):
        step(False, net, args.mlp_use)
    launches0 = ctx.launch_count()
    with Clocks(local_rank) as clk:
        recs, ms = timed(args.steps, host=False)
    launches = ctx.launch_count() - launches0
    # the timed run's results (device path), kept for the error leg
    ys_timed = {(ker, g): y.cpu().numpy() for ker in kernels for g, y in enumerate(keep[ker][4])}
    # end to end through the C ABI with host buffers (mesh in, densities in, y out)
    e_steps = max(1, args.steps // 2)
    erecs, ems = timed(e_steps, host=True)
    r0 = recs[-1]
    t_max, e_max = max_over_ranks([ms, ems], device=dev)
    entries_all, launches_all, aca_entries_all = sum_over_ranks(
        [r0["entries_aca"] + r0["entries_near"], launches, r0["entries_aca"]], device=dev)
    peaks = _peaks()
    props = torch.cuda.get_device_properties(dev)
    n_sm = props.multi_processor_count
    # dominant kernel: the persistent three-way ACA launch (mean over timed steps and operators)
    aca_ms = sum(r["aca_ms"] for r in recs) / (len(recs) * len(kernels))
    aca_entries = r0["entries_aca"] / len(kernels)
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    sfu_peak = SFU_PER_CLK_SM * n_sm * sm_mhz * 1e6              # SFU results/s (unit counts x clock)
    mufu = MUFU_PER_ENTRY_GALERKIN if scheme != "colloc7" else MUFU_PER_ENTRY
    achieved_sfu = aca_entries * mufu / (aca_ms / 1e3)
    # entries the kernel evaluates in all: Algorithm 1's plus the dense residual
    # working faces (an evaluation order: they replace the sums over earlier crosses)
    evaluated_sfu = (r0["entries_aca"] + r0["entries_face_dense"]) / len(kernels) * mufu / (aca_ms / 1e3)
    measured = {k: ctx.peak(k) for k in ("rsqrt", "ex2", "sin", "ffma", "dfma")}
    apply_ms = sum(r["apply_ms"] for r in recs) / len(recs)
    near_ms = sum(r["apply_near_ms"] for r in recs) / len(recs)
    apply_gbs = r0["apply_bytes"] / (apply_ms / 1e3) / 1e9
    near_gbs = r0["apply_near_bytes"] / (near_ms / 1e3) / 1e9 if near_ms > 0 else None
    # each part of the apply alone (the near field, the far field) and both
    # together as in the timed apply (the two overlap on two streams), each
    # best of three on the operators of the last timed step
    def measure_parts():
        """Best of three for each part; a function so that no operator
        outlives it (the A/B steps below need the memory)."""
        parts = {"near_ms": 0.0, "near_bytes": 0, "far_ms": 0.0, "far_bytes": 0, "both_ms": 0.0, "both_bytes": 0}
        for ker in kernels:
            trees, freqs, nfs, fas, _ = keep[ker]
            for g, (T, nf, fa) in enumerate(zip(trees, nfs, fas)):
                for part, a, b in (("near", nf, None), ("far", None, fa), ("both", nf, fa)):
                    best = None
                    for _ in range(3):
                        g3.apply_gcq(ctx, T, a, b, Wds[g])
                        la = ctx.last_apply()
                        best = la if best is None or la["ms"] < best["ms"] else best
                    parts[part + "_ms"] += best["ms"]
                    parts[part + "_bytes"] += best["bytes"]
        return parts

    parts = measure_parts()
    apply_parts = {k: {"ms": parts[k + "_ms"], "bytes": parts[k + "_bytes"],
                       "gbs": parts[k + "_bytes"] / (parts[k + "_ms"] / 1e3) / 1e9 if parts[k + "_ms"] > 0 else None}
                   for k in ("near", "far", "both")}
    # the far field with its x formation on the CUDA cores instead of the tensor cores
    ctx.set_apply_tensor_cores(False)
    parts_cc = measure_parts()
    ctx.set_apply_tensor_cores(True)
    apply_parts["far_cuda_cores"] = {"ms": parts_cc["far_ms"], "bytes": parts_cc["far_bytes"],
                                     "gbs": parts_cc["far_bytes"] / (parts_cc["far_ms"] / 1e3) / 1e9
                                     if parts_cc["far_ms"] > 0 else None}
    # steady-state apply (the operator is applied once per time step, many times
    # per compression): both operators, 10 applies each after one untimed apply,
    # mean CUDA-event time per apply
    def steady_apply(n=10):
        ms_tot, bytes_tot = 0.0, 0
        for ker in kernels:
            trees, freqs, nfs, fas, _ = keep[ker]
            for g, (T, nf, fa) in enumerate(zip(trees, nfs, fas)):
                g3.apply_gcq(ctx, T, nf, fa, Wds[g])
                for _ in range(n):
                    g3.apply_gcq(ctx, T, nf, fa, Wds[g])
                    la = ctx.last_apply()
                    ms_tot += la["ms"] / n
                    bytes_tot += la["bytes"] / n
        return ms_tot, bytes_tot
    steady_ms, steady_bytes = steady_apply()
    # learned + batched vs plain at equal accuracy: one seeded block sample,
    # both arms (single meshes only; the plain arm is one block per launch)
    vs_plain = None
    pv = None
    if not batch and world == 1 and args.plain_blocks > 0:
        trees, freqs, _, _, _ = keep[kernels[0]]
        shape = {k: tune[kernels[0]][k] for k in ("threads", "dense_face_max")} if kernels[0] in tune else {}
        pv = plain_vs_batched(g3, ctx, ws[0], trees[0], freqs[0], kernels[0], args.plain_blocks, 17, prec,
                              ws[0].eps3, ws[0].eps3, net, args.mlp_use, shape)
        vs_plain = {"value": pv["plain_ms"] / pv["ours_ms"], "same_blocks": True, "blocks": pv["blocks"],
                    "operator": kernels[0], "plain_ms": pv["plain_ms"], "ours_ms": pv["ours_ms"],
                    "plain_eps3": ws[0].eps3, "ours_eps3": ws[0].eps3,
                    "plain_entries_per_s": pv["plain_entries"] / (pv["plain_ms"] / 1e3),
                    "ours_entries_per_s": pv["ours_entries"] / (pv["ours_ms"] / 1e3),
                    "plain_crosses": pv["plain_crosses"], "ours_crosses": pv["ours_crosses"],
                    "sample": f"{pv['blocks']} far blocks of {kernels[0]} drawn by seed 17, stratified by block "
                              "size (8 strata); plain = float64, one block per launch; ours = the timed "
                              "configuration (mixed precision, one persistent launch, predictor)"}
    # what the predictor gains: the same compression without it, and with
    # queue order + pool size only (one step each, after the timed region);
    # and the first compression on a fresh context (no pool size learned from
    # earlier compressions yet), with the plain estimate and the predictor's
    learned = None
    if net is not None and world == 1:
        ab = {}
        for label, (m, u) in {"none": (None, 0), "order_pool": (net, 3), "all": (net, 7)}.items():
            r = step(False, m, u)
            ab[label] = {"aca_ms": r["aca_ms"], "crosses": r["crosses"], "factor_bytes": r["factor_bytes"],
                         "spilled_blocks": sum(st["spilled_blocks"] for st in r["stats"].values()),
                         "pool_regrows": sum(st["pool_regrows"] for st in r["stats"].values())}
        # the operators are not needed any more (their trees are): free them
        # before the fresh contexts allocate theirs
        for k in list(keep):
            keep[k] = keep[k][:2] + (None, None, None)
        fresh = {}
        for label, (m, u) in {"plain_estimate": (None, 0), "predicted_pool": (net, 2)}.items():
            c2 = g3.Context(local_rank, stream.cuda_stream)
            T2 = g3.build_cluster_tree(c2, ws[0].verts, ws[0].tris, ws[0].leaf, ws[0].eta, max_block=ws[0].max_block)
            F2 = g3.freqs_from_spec(c2, ws[0].freq)
            tot = {"aca_ms": 0.0, "wall_ms": 0.0, "spilled_blocks": 0, "pool_regrows": 0}
            for ker in kernels:
                torch.cuda.synchronize(dev)
                t_w = time.perf_counter()
                st2 = g3.aca3_compress(c2, T2, F2, ker, scheme=scheme, prec=prec, eps3=ws[0].eps3, mlp=m,
                                       mlp_use=u).stats()
                # wall time of the call: the device time plus the host work around it
                # (pool allocation and, for an over-reserved pool, its trim copy)
                tot["wall_ms"] += 1e3 * (time.perf_counter() - t_w)
                tot["aca_ms"] += st2["ms"]
                tot["spilled_blocks"] += st2["spilled_blocks"]
                tot["pool_regrows"] += st2["pool_regrows"]
            fresh[label] = tot
            del T2, F2, c2
        learned = {"mlp_use": args.mlp_use, "training": train_info, "ab": ab, "fresh_context": fresh}
    # the time-stepping consumer (g3_gcq_history) with the gCQ set of the graded
    # steps (N_Q = 256) on at least 131,072 elements: an HBM stream of X (read
    # and written) and W (written), 24 bytes per element and frequency (complex64)
    gcq_hist = None
    if world == 1 and not batch:
        st_ = workloads.graded_steps(64)
        Fg = g3.g3_freqs_gcq(ctx, 256, float(st_.min()), float(st_.max()))
        E0 = max(ws[0].E, 131072)   # X and W of 268 MB each: larger than L2
        Xg = torch.zeros((256, E0), dtype=torch.complex64, device=dev).t()
        Wg = torch.empty((256, E0), dtype=torch.complex64, device=dev).t()
        thg = torch.ones(E0, dtype=torch.complex64, device=dev)
        for _ in range(3):
            g3.gcq_history(ctx, Fg, Xg, thg, float(st_[0]), float(st_[1]), Wg)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        reps = 20
        e0.record(stream)
        for r in range(reps):
            g3.gcq_history(ctx, Fg, Xg, thg, float(st_[r % 64]), float(st_[(r + 1) % 64]), Wg)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms_h = e0.elapsed_time(e1) / reps
        byt = E0 * 256 * 24
        gcq_hist = {"ms": ms_h, "bytes": byt, "gbs": byt / (ms_h / 1e3) / 1e9,
                    "frac_hbm": byt / (ms_h / 1e3) / 1e9 / _peaks()["hbm_gbs"],
                    "note": f"{E0} elements x 256 gCQ frequencies, complex64 (X and W larger than L2), "
                            f"mean of {reps} launches"}
    # the pivot estimate of eq. (index) against the dense expansion (single
    # layer, collocation; the double layer keeps the dense expansion)
    pivot_ab = None
    if world == 1 and not batch and "slp" in kernels and scheme == "colloc7":
        trees, freqs, _, _, _ = keep["slp"]
        shape = {k: tune["slp"][k] for k in ("threads", "dense_face_max")} if "slp" in tune else {}
        pivot_ab = {}
        for label, pi in (("dense_expansion", 0), ("eq_index", 1)):
            stp = g3.aca3_compress(ctx, trees[0], freqs[0], "slp", scheme=scheme, prec=prec, eps3=ws[0].eps3, mlp=net,
                                   mlp_use=args.mlp_use, pivot_index=pi, **shape).stats()
            pivot_ab[label] = {"aca_ms": stp["ms"], "crosses": stp["crosses"], "entries": stp["entries"],
                               "factor_bytes": stp["factor_bytes"]}
    # where a step's wall time goes: the same calls as one step, each followed
    # by a synchronize (untimed by the bench line; host work shows up here)
    breakdown = None
    if world == 1 and not batch:
        keep.clear()
        wall = {"tree": 0.0, "freqs": 0.0, "assemble_near": 0.0, "aca3_compress": 0.0, "apply_gcq": 0.0}
        host = {}

        def lap(key, fn):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            r = fn()
            torch.cuda.synchronize(dev)
            wall[key] += (time.perf_counter() - t0) * 1e3
            return r

        Tb = lap("tree", lambda: make_tree(ws[0]))
        Fb = lap("freqs", lambda: g3.freqs_from_spec(ctx, ws[0].freq))
        for ker in kernels:
            shape = {k: tune[ker][k] for k in ("threads", "dense_face_max", "residual_face_max")} if ker in tune else {}
            nfb = lap("assemble_near", lambda: g3.assemble_near(ctx, Tb, Fb, ker, scheme=scheme, prec=prec))
            fab = lap("aca3_compress", lambda: g3.aca3_compress(ctx, Tb, Fb, ker, scheme=scheme, prec=prec,
                                                                eps3=ws[0].eps3, mlp=net, mlp_use=args.mlp_use,
                                                                **shape))
            lap("apply_gcq", lambda: g3.apply_gcq(ctx, Tb, nfb, fab, Wds[0]))
            sb = fab.stats()
            for k, v in sb["ms_host"].items():
                host[k] = host.get(k, 0.0) + v
            host["device_ms"] = host.get("device_ms", 0.0) + sb["ms"]
            del nfb, fab
        breakdown = {k: round(v, 3) for k, v in wall.items()}
        breakdown["aca3_compress_parts"] = {k: round(v, 3) for k, v in host.items()}
        breakdown["note"] = ("wall ms of one step's calls, each followed by a synchronize; the compression's "
                             "own host timers (set-up, launch rounds, read-back, apply plan) and device time")
    if rank != 0:
        return None
    ms_step = t_max / args.steps
    value = whole_job_rate(entries_all, t_max, args.steps)
    aca_eps = sum(r["entries_aca"] for r in recs) / (sum(r["aca_ms"] for r in recs) / 1e3)
    h2d = sum(int(w.verts.nbytes + w.tris.nbytes) for w in ws) + len(kernels) * sum(int(W.nbytes) for W in Ws)
    d2h = len(kernels) * sum(int(w.E * 16) for w in ws)
    out = {
        "metric": METRIC,
        "value": value,
        "unit": "entries/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "strong",
        "vs_baseline": None,
        "dtype": "f32" if prec == "mixed" else "f64",
        "data": "synthetic",
        "config": {**(workloads.describe(ws[0]) if not batch else
                      {"workload": "batch64", "meshes": len(ws), "triangles": int(sum(w.E for w in ws)),
                       "K": sorted({w.freq.K for w in ws}), "kernels": kernels, "scheme": scheme,
                       "eps3": ws[0].eps3, "max_block": ws[0].max_block}),
                   "precision": prec,
                   "l2": "inputs larger than L2: near field %.1f GB and factors %.1f GB per operator, "
                         "no flush" % (r0["apply_near_bytes"] / len(kernels) / 1e9,
                                       r0["factor_bytes"] / len(kernels) / 1e9),
                   "parallelism": ("single GPU" if world == 1 else
                                   f"row-cluster shards x{world} (one problem divided, no data-path collective)")},
        "apply_gbs": steady_bytes / (steady_ms / 1e3) / 1e9,
        "apply_ms_steady": steady_ms,
        "apply_gbs_first_after_compression": apply_gbs,
        "near_apply_gbs": near_gbs,
        "apply_parts": apply_parts,
        "entries_per_step": entries_all,
        "entries_aca": aca_entries_all,
        "entries_face_dense": r0["entries_face_dense"],
        "entries_near": entries_all - aca_entries_all,
        "phase_ms": {"aca3_compress": r0["aca_ms"], "assemble_near": r0["near_ms"], "apply_gcq": r0["apply_ms"]},
        "storage_ratio": r0["factor_bytes"] / r0["dense_bytes"] if r0["dense_bytes"] else None,
        "crosses": r0["crosses"],
        "gpu_launches": int(launches_all),
        "e2e": {"value": whole_job_rate(entries_all, e_max, e_steps), "unit": "entries/s",
                "h2d_bytes_per_step": int(h2d * world), "d2h_bytes_per_step": int(d2h * world)},
        "roofline": {"bound": "alu", "achieved": achieved_sfu / 1e12, "peak": sfu_peak / 1e12,
                     "unit": "Tops/s (special-function unit)", "frac": achieved_sfu / sfu_peak,
                     "traffic": ACA_TRAFFIC_BYTES.get(args.workload) if world == 1 else None,
                     "traffic_unit": "bytes per launch",
                     "kernel": "k_aca3",
                     "frac_evaluated": evaluated_sfu / sfu_peak,
                     "note": f"{mufu} SFU ops per entry x {aca_entries:.4g} entries per launch (Algorithm 1's "
                             f"rows, columns, samples and fibers) / {aca_ms:.1f} ms; peak = {SFU_PER_CLK_SM}/clk/SM x "
                             f"{n_sm} SMs x {sm_mhz:.0f} MHz (unit counts and clock, matching the measured rsqrt / sin "
                             "rates); frac_evaluated adds the entries of the dense residual working faces"},
        "roofline_apply": {"bound": "hbm", "achieved": steady_bytes / (steady_ms / 1e3) / 1e9,
                           "peak": peaks["hbm_gbs"], "unit": "GB/s",
                           "frac": steady_bytes / (steady_ms / 1e3) / 1e9 / peaks["hbm_gbs"],
                           "traffic": APPLY_TRAFFIC_BYTES.get(args.workload) if world == 1 else None,
                           "traffic_unit": "bytes per apply of every operator", "bytes": steady_bytes,
                           "kernel": "apply_gcq (all kernels)", "peak_source": peaks["source"],
                           "note": "algorithmic bytes (near field, factors, W, y) / CUDA-event time of the whole "
                                   "apply, mean of 10 applies per operator after one untimed apply (steady state: "
                                   "the operator is applied once per time step); far-field x formation on the "
                                   "tensor cores"},
        "measured_pipes_ops_per_s": measured,
        "vs_plain": vs_plain,
        "clocks": clk.summary(),
        "peaks_source": peaks["source"],
        "learned": learned,
        "pivot_index_ab": pivot_ab,
        "step_breakdown_ms": breakdown,
        "gcq_history": gcq_hist,
        "autotune": tune or None,
        "compression_entries_per_s": aca_eps,
    }
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = oracle_sample(args.workload, args.cpu_seconds, 7, os.cpu_count() or 1)
        # error of the timed results against the float64 oracle on sampled rows
        out["apply_error_vs_oracle"] = apply_errors(args.workload, kernels, ys_timed,
                                                    [w.density_seed for w in ws], args.error_rows, 5,
                                                    os.cpu_count() or 1)
        if pv is not None:
            out["vs_plain"]["errors"] = plain_arm_errors(g3, ctx, ws[0], kernels[0], pv, ws[0].density_seed, Wds[0],
                                                         args.error_rows, os.cpu_count() or 1)
    return out


def plain_arm_errors(g3, ctx, w, ker, pv, seed: int, Wd, n_rows: int, cores: int) -> dict:
    """Far-field apply of the sampled blocks by both arms against the float64
    oracle's dense apply of the same blocks, on seeded sampled rows."""
    import numpy as np
    S = pv["tree"]
    sg = S.get()
    perm, blocks = sg["perm"], sg["blocks"]
    rng = np.random.default_rng(11)
    cand = np.unique(np.concatenate([perm[rb:re] for rb, re, _, _, _ in blocks]))
    rows = np.sort(rng.choice(cand, min(n_rows, cand.size), replace=False))
    jobs = []
    for i in rows:
        cols = []
        for rb, re, cb, ce, _ in blocks:
            if i in set(perm[rb:re].tolist()):
                cols.append(perm[cb:ce])
        jobs.append((w.name, ker, int(i), seed, np.concatenate(cols)))
    ref = np.array(oracle_rows(jobs, cores))
    out = {}
    for arm in ("plain", "ours"):
        y = g3.apply_gcq(ctx, S, None, pv[arm], Wd).cpu().numpy()
        out[arm] = float(np.linalg.norm(y[rows] - ref) / np.linalg.norm(ref))
    out["rows"] = int(rows.size)
    return out


def run_reference(args) -> dict:
    """The CPU oracle as it stands, on the host cores, same workload and metric."""
    from inputs import workloads as _wl
    p1 = args.workload != "batch64" and _wl.get(args.workload).extra.get("p1")
    res = []
    for i in range(args.warmup + args.steps):
        if p1:
            w1 = _wl.get(args.workload)
            r = p1_oracle_sample(w1, list(w1.kernels), args.ref_seconds, 100 + i)
        else:
            r = oracle_sample(args.workload, args.ref_seconds, 100 + i, os.cpu_count() or 1)
        if i >= args.warmup:
            res.append(r)
    ent = sum(r["entries"] for r in res)
    sec = sum(r["seconds"] for r in res)
    value = ent / sec
    from inputs import workloads
    ws = mesh_list(args.workload)
    w = ws[0]
    cfg = workloads.describe(w) if len(ws) == 1 else {"workload": "batch64", "meshes": len(ws)}
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "entries/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / len(res),
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {**cfg, "precision": "fp64 (oracle)"},
            "cpu_baseline": {"value": value, "unit": "entries/s", "cores": res[0]["cores"], "kind": "oracle",
                             "sample": res[0]["sample"]},
            "e2e": {"value": value, "unit": "entries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}


def run_profile_case(args) -> dict:
    """One small invocation for a profiler (no timing loop, no baselines): the
    workload's tree and frequencies, one compression of `--profile-case`'s
    operator (256 threads, dense faces up to 48^2), then the near field and two
    applies.  Launch order: the compression's low-rank launch, its dense-face
    launch, the near-field assembly, then per apply k_apply_prep,
    k_apply_near (side stream), k_apply_far_dense, k_far_lr_tc (narrow and
    wide blocks), k_apply_finish."""
    import torch
    import paper_2312_11219_gb300 as g3
    from inputs import workloads
    w = workloads.get(args.workload)
    ker = args.profile_case
    ctx = g3.Context(0)
    T = g3.build_cluster_tree(ctx, w.verts, w.tris, w.leaf, w.eta, max_block=w.max_block)
    F = g3.freqs_from_spec(ctx, w.freq)
    fa = g3.aca3_compress(ctx, T, F, ker, scheme=w.scheme, prec=args.precision, eps3=w.eps3, threads=256,
                          dense_face_max=48 * 48)
    nf = g3.assemble_near(ctx, T, F, ker, scheme=w.scheme, prec=args.precision)
    dt = torch.complex64 if args.precision == "mixed" else torch.complex128
    Wd = torch.from_numpy(workloads.densities(w.E, w.freq.K, w.density_seed)).to("cuda", dt)
    for _ in range(2):
        g3.apply_gcq(ctx, T, nf, fa, Wd)
    torch.cuda.synchronize()
    st, la = fa.stats(), ctx.last_apply()
    return {"profile_case": ker, "workload": args.workload, "aca_ms": st["ms"], "aca_lowrank_ms": st["ms_lowrank"],
            "crosses": st["crosses"], "entries": st["entries"], "n_far": st["n_far"], "apply_ms": la["ms"],
            "apply_bytes": la["bytes"], "near_ms": la["near_ms"], "near_bytes": la["near_bytes"]}


# ---------------------------------------------------------------------------
# the Neumann problem: Galerkin operators of linear continuous elements
# ---------------------------------------------------------------------------

def _p1_entry_fn(w, op):
    """The oracle's ENTRY of element-local shape functions (original indices
    3 e + a), through its local 3 x 3 blocks."""
    import numpy as np
    from oracle import galerkin_p1 as P1

    def f(I, J, s):
        out = np.zeros((len(I), np.atleast_1d(s).size), complex)
        cache = {}
        for t, (i, j) in enumerate(zip(I, J)):
            key = (int(i) // 3, int(j) // 3)
            if key not in cache:
                cache[key] = P1.local_block(w.verts, w.tris, key[0], key[1], s, op)
            out[t] = cache[key][int(i) % 3, int(j) % 3]
        return out
    return f


def p1_oracle_sample(w, kernels, seconds: float, seed: int) -> dict:
    """Oracle entries/s (one host thread) on seeded random blocks of the
    linear-element operators: far blocks through the oracle's three-way ACA,
    near blocks through its local blocks, in the far/near proportion."""
    import time as _t

    import numpy as np
    from oracle import aca3 as O_aca, freqs as O_freqs, tree as O_tree
    T = O_tree.build(w.verts, w.tris, w.leaf, w.eta, w.max_block)
    fs = O_freqs.frequency_set(w.freq)
    su = fs["s"][fs["uniq"]]
    rng = np.random.default_rng(seed)
    ops = {"hyp": "d", "adj": "kp"}
    ent, nb, t0 = 0, 0, _t.perf_counter()
    while _t.perf_counter() - t0 < seconds:
        ker = kernels[nb % len(kernels)]
        ef = _p1_entry_fn(w, ops[ker])
        b = int(rng.integers(0, T.blocks.shape[0]))
        rb, re, cb, ce, adm = T.blocks[b]
        rows = (3 * T.perm[rb:re][:, None] + np.arange(3)[None, :]).ravel()
        cols = (3 * T.perm[cb:ce][:, None] + np.arange(3)[None, :]).ravel()
        if adm:
            op = O_aca.BemBlock(ef, rows, cols, su)
            O_aca.aca3(op, w.eps3, s_abs=np.abs(su))
            ent += int(op.generated)
        else:
            ef(np.repeat(rows, cols.size), np.tile(cols, rows.size), su)
            ent += rows.size * cols.size * su.size
        nb += 1
    sec = _t.perf_counter() - t0
    return {"value": ent / sec, "unit": "entries/s", "cores": 1, "kind": "oracle",
            "sample": f"{nb} seeded random blocks of {w.name} ({', '.join(kernels)}; far blocks through the "
                      f"oracle's three-way ACA, near blocks densely), {sec:.1f} s wall, one host thread",
            "entries": ent, "seconds": sec}


def run_neumann(args, rank: int, world: int, local_rank: int) -> dict | None:
    """The timed step on a linear-element workload: per operator (hypersingular,
    adjoint double layer) the tree of element-local shape functions, the near
    field, the three-way ACA and one nodal apply; one GPU."""
    import numpy as np
    import torch
    import paper_2312_11219_gb300 as g3
    from inputs import workloads
    from oracle import freqs as O_freqs, galerkin_p1 as P1
    if world > 1:
        raise SystemExit(f"{args.workload}: one GPU only")
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = workloads.get(args.workload)
    nv = w.verts.shape[0]
    W = workloads.densities(nv, w.freq.K, w.density_seed)
    Wd = torch.from_numpy(W).to(dev, torch.complex64)
    stream = torch.cuda.current_stream(dev)
    ctx = g3.Context(local_rank, stream.cuda_stream)
    keep = {}

    def step(host: bool):
        T = g3.build_cluster_tree(ctx, w.verts, w.tris, w.leaf, w.eta, max_block=w.max_block)
        T1 = g3.build_p1_tree(ctx, T)
        F = g3.freqs_from_spec(ctx, w.freq)
        rec = {"entries_aca": 0, "entries_face_dense": 0, "entries_near": 0, "aca_ms": 0.0, "near_ms": 0.0,
               "apply_ms": 0.0, "apply_bytes": 0, "crosses": 0, "factor_bytes": 0, "dense_bytes": 0}
        for ker in w.kernels:
            keep.pop(ker, None)
            nf = g3.assemble_near(ctx, T1, F, ker, scheme="galerkin4x4", prec="mixed")
            fa = g3.aca3_compress(ctx, T1, F, ker, scheme="galerkin4x4", prec="mixed", eps3=w.eps3)
            y = g3.apply_gcq(ctx, T1, nf, fa, W if host else Wd)
            la, st, ni = ctx.last_apply(), fa.stats(), nf.info()
            rec["entries_aca"] += st["entries"]
            rec["entries_face_dense"] += st["entries_face_dense"]
            rec["entries_near"] += ni["entries"]
            rec["aca_ms"] += st["ms"]
            rec["near_ms"] += ni["ms"]
            rec["apply_ms"] += la["ms"]
            rec["apply_bytes"] += la["bytes"]
            rec["crosses"] += st["crosses"]
            rec["factor_bytes"] += st["factor_bytes"]
            rec["dense_bytes"] += st["dense_bytes"]
            keep[ker] = (T1, nf, fa, y)
        return rec

    def timed(n: int, host: bool):
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        recs = [step(host) for _ in range(n)]
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return recs, e0.elapsed_time(e1)

    for _ in range(args.warmup):
        step(False)
    launches0 = ctx.launch_count()
    with Clocks(local_rank) as clk:
        recs, ms = timed(args.steps, False)
    launches = ctx.launch_count() - launches0
    ys = {ker: keep[ker][3].cpu().numpy() for ker in w.kernels}
    e_steps = max(1, args.steps // 2)
    _, ems = timed(e_steps, True)
    r0 = recs[-1]
    entries = r0["entries_aca"] + r0["entries_near"]
    peaks = _peaks()
    props = torch.cuda.get_device_properties(dev)
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    sfu_peak = SFU_PER_CLK_SM * props.multi_processor_count * sm_mhz * 1e6
    aca_ms = sum(r["aca_ms"] for r in recs) / (len(recs) * len(w.kernels))
    aca_entries = r0["entries_aca"] / len(w.kernels)
    achieved = aca_entries * MUFU_PER_ENTRY_GALERKIN / (aca_ms / 1e3)
    evaluated = (r0["entries_aca"] + r0["entries_face_dense"]) / len(w.kernels) * MUFU_PER_ENTRY_GALERKIN / (aca_ms / 1e3)
    # steady-state apply, both operators, 10 applies each after one untimed apply
    st_ms, st_bytes = 0.0, 0
    for ker in w.kernels:
        T1, nf, fa, _ = keep[ker]
        g3.apply_gcq(ctx, T1, nf, fa, Wd)
        for _ in range(10):
            g3.apply_gcq(ctx, T1, nf, fa, Wd)
            la = ctx.last_apply()
            st_ms += la["ms"] / 10
            st_bytes += la["bytes"] / 10
    apply_gbs = st_bytes / (st_ms / 1e3) / 1e9
    out = {
        "metric": "3-way ACA entries/s & apply GB/s (1 GB300); learned+batched vs plain at 1e-4",
        "value": whole_job_rate(entries, ms, args.steps), "unit": "entries/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "triangles": w.E, "vertices": nv, "K": w.freq.K, "freqs": w.freq.kind,
                   "kernels": list(w.kernels), "scheme": "galerkin4x4, linear continuous elements (element-local "
                   "shape functions, nodal densities)", "leaf": w.leaf, "eta": w.eta, "eps3": w.eps3,
                   "precision": "mixed", "l2": "near field %.2f GB per operator (not larger than L2 on every "
                   "operator: no flush; the timed step builds every operator anew)" % (
                       r0["entries_near"] / len(w.kernels) * 8 / 1e9), "parallelism": "single GPU"},
        "gpu_launches": int(launches),
        "entries_per_step": entries, "entries_aca": r0["entries_aca"], "entries_near": r0["entries_near"],
        "entries_face_dense": r0["entries_face_dense"],
        "phase_ms": {"aca3_compress": r0["aca_ms"], "assemble_near": r0["near_ms"], "apply_gcq": r0["apply_ms"]},
        "storage_ratio": r0["factor_bytes"] / r0["dense_bytes"] if r0["dense_bytes"] else None,
        "crosses": r0["crosses"], "apply_gbs": apply_gbs, "apply_ms_steady": st_ms,
        "e2e": {"value": whole_job_rate(entries, ems, e_steps), "unit": "entries/s",
                "h2d_bytes_per_step": int(W.nbytes * len(w.kernels)),
                "d2h_bytes_per_step": int(nv * 16 * len(w.kernels))},
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": sfu_peak / 1e12,
                     "unit": "Tops/s (special-function unit)", "frac": achieved / sfu_peak, "traffic": None,
                     "kernel": "k_aca3 (linear elements)", "frac_evaluated": evaluated / sfu_peak,
                     "note": f"{MUFU_PER_ENTRY_GALERKIN} SFU ops per entry (16 kernel evaluations) x "
                             f"{aca_entries:.4g} entries per launch / {aca_ms:.1f} ms"},
        "roofline_apply": {"bound": "hbm", "achieved": apply_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                           "frac": apply_gbs / peaks["hbm_gbs"], "traffic": None, "kernel": "apply_gcq (all kernels)",
                           "peak_source": peaks["source"]},
        "clocks": clk.summary(), "peaks_source": peaks["source"],
    }
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = p1_oracle_sample(w, list(w.kernels), args.cpu_seconds, 7)
        fs = O_freqs.frequency_set(w.freq)
        rows = np.sort(np.random.default_rng(3).choice(nv, 2, replace=False))
        errs = {}
        for ker, op in (("hyp", "d"), ("adj", "kp")):
            R = P1.nodal_rows(w.verts, w.tris, rows, fs["s"], op)
            ref = np.einsum("rjk,jk->r", R, W)
            errs[ker] = {"rel_err": float(np.linalg.norm(ys[ker][rows] - ref) / np.linalg.norm(ref)),
                         "rows": int(rows.size)}
        out["apply_error_vs_oracle"] = errs
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="lshape12288")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--plain-blocks", type=int, default=400,
                    help="far blocks in the same-sample plain float64 vs batched comparison (0 = skip)")
    ap.add_argument("--error-rows", type=int, default=24,
                    help="sampled rows of the apply error against the float64 oracle (cpu_baseline leg)")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--ref-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--mlp-use", type=int, default=3,
                    help="predictor uses in the timed compressions (1 order, 2 pool, 4 k1; 0 = no predictor)")
    ap.add_argument("--profile-case", default=None, choices=["slp", "dlp"],
                    help="run one compression and two applies of --workload for a profiler, then exit")
    args = ap.parse_args()
    if args.profile_case:
        print(json.dumps(run_profile_case(args)), flush=True)
        return
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    from inputs import workloads as _wl
    if args.workload not in ("batch64",) and _wl.get(args.workload).extra.get("p1"):
        out = run_neumann(args, rank, world, local_rank)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    out = run_ours(args, rank, world, local_rank)
    if out is not None:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
