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

Multi-GPU: each rank runs its own copy of the workload (independent
problems, no collective on the data path; weak scaling); the timed region
is bracketed by barriers and the step time is the maximum over ranks.
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
# each one rsqrt, one ex2, one sin and one cos
MUFU_PER_ENTRY = 28
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
# CPU oracle timing (cpu_baseline leg and the reference arm)
# ---------------------------------------------------------------------------

_ORACLE_CACHE: dict = {}


def _oracle_setup(name: str):
    if name not in _ORACLE_CACHE:
        from inputs import workloads
        from oracle import freqs as O_freqs, quadrature as O_q, tree as O_tree
        w = workloads.get(name)
        geo = O_q.Geometry(w.verts, w.tris)
        T = O_tree.build(w.verts, w.tris, w.leaf, w.eta, w.max_block)
        fs = O_freqs.frequency_set(w.freq)
        _ORACLE_CACHE[name] = (w, geo, T, fs)
    return _ORACLE_CACHE[name]


def _oracle_job(job):
    """One unit of oracle work: compress far block b of operator `ker` (or
    evaluate near block b at every unique frequency).  Returns entries."""
    import numpy as np
    from oracle import aca3 as O_aca, quadrature as O_q
    name, ker, b = job
    w, geo, T, fs = _oracle_setup(name)
    su = fs["s"][fs["uniq"]]
    rb, re, cb, ce, adm = T.blocks[b]
    ef = lambda I, J, s: O_q.entries(geo, ker, I, J, s)
    if adm:
        op = O_aca.BemBlock(ef, T.perm[rb:re], T.perm[cb:ce], su)
        O_aca.aca3(op, w.eps3, s_abs=np.abs(su))
        return int(op.generated)
    R, C = T.perm[rb:re], T.perm[cb:ce]
    I = np.repeat(R, C.size)
    J = np.tile(C, R.size)
    ef(I, J, su)
    return int(I.size * su.size)


def _oracle_warm(name):
    _oracle_setup(name)
    return os.getpid()


def oracle_sample(name: str, seconds: float, seed: int, cores: int) -> dict:
    """Oracle entries/s on a seeded random sample of the workload's blocks
    (far blocks through the oracle's three-way ACA, near blocks through its
    dense quadrature, in the workload's far/near proportion), run on a spawn
    pool of `cores` processes for about `seconds` of wall time."""
    import multiprocessing as mp

    import numpy as np
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    w, geo, T, fs = _oracle_setup(name)
    rng = np.random.default_rng(seed)
    far = np.nonzero(T.blocks[:, 4] == 1)[0]
    near = np.nonzero(T.blocks[:, 4] == 0)[0]
    jobs = []
    for i in range(100000):
        ker = w.kernels[i % len(w.kernels)]
        pick_far = rng.random() < far.size / (far.size + near.size)
        b = int(rng.choice(far if pick_far else near))
        jobs.append((name, ker, b))
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_warm, [name] * cores)
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
    return {"value": entries / wall, "unit": "entries/s", "cores": cores, "kind": "oracle",
            "sample": f"{done} seeded random blocks of {name} ({'/'.join(w.kernels)}; far blocks through the "
                      f"oracle's three-way ACA, near blocks densely), {wall:.1f} s wall",
            "entries": entries, "seconds": wall}


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


def whole_job_rate(units_per_rank: float, world: int, ms_max: float, steps: int) -> float:
    """Units processed by all ranks per second, timed by the slowest rank."""
    return units_per_rank * world / ((ms_max / steps) / 1e3)


def train_predictor(g3, ctx, kernels, prec):
    """Block predictor trained on the compressions of cube768 and lshape3072
    (features and labels from the library, training on the GPU)."""
    import time

    import numpy as np

    from inputs import workloads
    X, Y = [], []
    for name in ("cube768", "lshape3072"):
        w = workloads.get(name)
        T = g3.build_cluster_tree(ctx, w.verts, w.tris, w.leaf, w.eta, max_block=w.max_block)
        F = g3.freqs_from_spec(ctx, w.freq)
        for ker in kernels:
            fa = g3.aca3_compress(ctx, T, F, ker, prec=prec, eps3=w.eps3)
            X.append(g3.block_features(ctx, T, F, ker, w.eps3))
            Y.append(fa.labels())
    X, Y = np.concatenate(X), np.concatenate(Y)
    t0 = time.perf_counter()
    net = g3.mlp_train(ctx, X, Y, epochs=150, batch=256, seed=1)
    secs = time.perf_counter() - t0
    p = net.predict(X)
    return net, {"samples": int(X.shape[0]), "epochs": 150, "seconds": secs,
                 "mae_log2_r3": float(np.abs(p[:, 0] - Y[:, 0]).mean()),
                 "data": "cube768 + lshape3072 compressions"}


def run_ours(args, rank: int, world: int, local_rank: int) -> dict | None:
    import numpy as np
    import torch

    import paper_2312_11219_gb300 as g3
    from inputs import workloads

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = workloads.get(args.workload)
    kernels = list(w.kernels)
    W = workloads.densities(w.E, w.freq.K, w.density_seed)
    Wd = torch.from_numpy(W).to(dev)
    stream = torch.cuda.current_stream(dev)
    ctx = g3.Context(local_rank, stream.cuda_stream)
    prec = args.precision
    keep = {}

    # the learned part: a predictor trained (untimed, like any model) on the
    # compressions of two smaller meshes, used by every timed compression
    net, train_info = None, None
    if args.mlp_use:
        net, train_info = train_predictor(g3, ctx, kernels, prec)

    # launch shape per operator from the autotuner (untimed; cached in the context)
    tune = {}
    if not args.no_autotune:
        T0 = g3.build_cluster_tree(ctx, w.verts, w.tris, w.leaf, w.eta, max_block=w.max_block)
        F0 = g3.freqs_from_spec(ctx, w.freq)
        for ker in kernels:
            tune[ker] = g3.autotune(ctx, T0, F0, ker, scheme=w.scheme, prec=prec, eps3=w.eps3)
        del T0, F0

    def step(host: bool, mlp=None, mlp_use=0):
        T = g3.build_cluster_tree(ctx, w.verts, w.tris, w.leaf, w.eta, max_block=w.max_block)
        F = g3.freqs_from_spec(ctx, w.freq)
        rec = {"entries_aca": 0, "entries_near": 0, "aca_ms": 0.0, "near_ms": 0.0, "apply_ms": 0.0,
               "apply_near_ms": 0.0, "apply_bytes": 0, "apply_near_bytes": 0, "factor_bytes": 0,
               "dense_bytes": 0, "crosses": 0, "stats": {}}
        for ker in kernels:
            nf = g3.assemble_near(ctx, T, F, ker, scheme=w.scheme, prec=prec)
            shape = {k: tune[ker][k] for k in ("threads", "dense_face_max")} if ker in tune else {}
            fa = g3.aca3_compress(ctx, T, F, ker, scheme=w.scheme, prec=prec, eps3=w.eps3, mlp=mlp, mlp_use=mlp_use,
                                  **shape)
            y = g3.apply_gcq(ctx, T, nf, fa, W if host else Wd)
            st = fa.stats()
            ni = nf.info()
            la = ctx.last_apply()
            rec["entries_aca"] += st["entries"]
            rec["entries_near"] += ni["entries"]
            rec["aca_ms"] += st["ms"]
            rec["near_ms"] += ni["ms"]
            rec["apply_ms"] += la["ms"]
            rec["apply_near_ms"] += la["near_ms"]
            rec["apply_bytes"] += la["bytes"]
            rec["apply_near_bytes"] += la["near_bytes"]
            rec["factor_bytes"] += st["factor_bytes"]
            rec["dense_bytes"] += st["dense_bytes"]
            rec["crosses"] += st["crosses"]
            rec["stats"][ker] = st
            keep[ker] = (T, F, nf, fa, y)
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
    # end to end through the C ABI with host buffers (mesh in, densities in, y out)
    e_steps = max(1, args.steps // 2)
    erecs, ems = timed(e_steps, host=True)
    t_max, e_max = max_over_ranks([ms, ems], device=dev)
    if rank != 0:
        return None
    r0 = recs[-1]
    entries = r0["entries_aca"] + r0["entries_near"]
    ms_step = t_max / args.steps
    value = whole_job_rate(entries, world, t_max, args.steps)
    peaks = _peaks()
    props = torch.cuda.get_device_properties(dev)
    n_sm = props.multi_processor_count
    # dominant kernel: the persistent three-way ACA launch (mean over timed steps and operators)
    aca_ms = sum(r["aca_ms"] for r in recs) / (len(recs) * len(kernels))
    aca_entries = r0["entries_aca"] / len(kernels)
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    sfu_peak = SFU_PER_CLK_SM * n_sm * sm_mhz * 1e6              # SFU results/s (unit counts x clock)
    achieved_sfu = aca_entries * MUFU_PER_ENTRY / (aca_ms / 1e3)
    measured = {k: ctx.peak(k) for k in ("rsqrt", "ex2", "sin", "ffma", "dfma")}
    apply_ms = sum(r["apply_ms"] for r in recs) / len(recs)
    near_ms = sum(r["apply_near_ms"] for r in recs) / len(recs)
    apply_gbs = r0["apply_bytes"] / (apply_ms / 1e3) / 1e9
    near_gbs = r0["apply_near_bytes"] / (near_ms / 1e3) / 1e9
    # far part of the apply (everything but the near-field stream: factors,
    # W read once, y written once); the near field runs on a second stream
    # next to the far-field kernels, so this is the far part's share of the
    # apply's wall time
    far_gbs = (r0["apply_bytes"] - r0["apply_near_bytes"]) / ((apply_ms - near_ms) / 1e3) / 1e9
    # plain baseline: float64, one block per launch (host loop), on a bounded
    # sample of the first admissible blocks of the single layer
    T, F, nf, fa, y = keep[kernels[0]]
    plain = g3.aca3_compress(ctx, T, F, kernels[0], prec="fp64", eps3=w.eps3, unbatched=1,
                             max_blocks=args.plain_blocks).stats()
    ours_sample = g3.aca3_compress(ctx, T, F, kernels[0], prec=prec, eps3=w.eps3,
                                   max_blocks=args.plain_blocks).stats()
    plain_eps = plain["entries"] / (plain["ms"] / 1e3)
    # what the predictor gains: the same compression without it, and with
    # queue order + pool size only (one step each, after the timed region)
    learned = None
    if net is not None:
        ab = {}
        for label, (m, u) in {"none": (None, 0), "order_pool": (net, 3), "all": (net, 7)}.items():
            r = step(False, m, u)
            ab[label] = {"aca_ms": r["aca_ms"], "crosses": r["crosses"], "factor_bytes": r["factor_bytes"],
                         "spilled_blocks": sum(st["spilled_blocks"] for st in r["stats"].values()),
                         "pool_regrows": sum(st["pool_regrows"] for st in r["stats"].values())}
        learned = {"mlp_use": args.mlp_use, "training": train_info, "ab": ab}
    aca_eps = sum(r["entries_aca"] for r in recs) / (sum(r["aca_ms"] for r in recs) / 1e3)
    out = {
        "metric": METRIC,
        "value": value,
        "unit": "entries/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if prec == "mixed" else "f64",
        "data": "synthetic",
        "config": {**workloads.describe(w), "precision": prec,
                   "l2": "inputs larger than L2: near field %.1f GB and factors %.1f GB per operator, "
                         "no flush" % (r0["apply_near_bytes"] / len(kernels) / 1e9,
                                       r0["factor_bytes"] / len(kernels) / 1e9),
                   "parallelism": f"independent replicas x{world}"},
        "apply_gbs": apply_gbs,
        "near_apply_gbs": near_gbs,
        "far_apply_gbs": far_gbs,
        "entries_per_step": entries,
        "entries_aca": r0["entries_aca"],
        "entries_near": r0["entries_near"],
        "phase_ms": {"aca3_compress": r0["aca_ms"], "assemble_near": r0["near_ms"], "apply_gcq": r0["apply_ms"]},
        "storage_ratio": r0["factor_bytes"] / r0["dense_bytes"] if r0["dense_bytes"] else None,
        "crosses": r0["crosses"],
        "gpu_launches": int(launches),
        "e2e": {"value": whole_job_rate(entries, world, e_max, e_steps), "unit": "entries/s",
                "h2d_bytes_per_step": int(w.verts.nbytes + w.tris.nbytes + len(kernels) * W.nbytes),
                "d2h_bytes_per_step": int(len(kernels) * w.E * 16)},
        "roofline": {"bound": "alu", "achieved": achieved_sfu / 1e12, "peak": sfu_peak / 1e12,
                     "unit": "Tops/s (special-function unit)", "frac": achieved_sfu / sfu_peak, "traffic": None,
                     "kernel": "k_aca3",
                     "note": f"{MUFU_PER_ENTRY} SFU ops per entry x {aca_entries:.4g} entries per launch / "
                             f"{aca_ms:.1f} ms; peak = {SFU_PER_CLK_SM}/clk/SM x {n_sm} SMs x {sm_mhz:.0f} MHz"},
        "roofline_apply": {"bound": "hbm", "achieved": near_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                           "frac": near_gbs / peaks["hbm_gbs"], "traffic": None, "kernel": "k_apply_near",
                           "peak_source": peaks["source"]},
        "measured_pipes_ops_per_s": measured,
        "vs_plain": {"value": aca_eps / plain_eps, "plain_entries_per_s": plain_eps,
                     "ours_same_sample_entries_per_s": ours_sample["entries"] / (ours_sample["ms"] / 1e3),
                     "ours_full_entries_per_s": aca_eps,
                     "sample": f"first {plain['blocks_run']} admissible blocks of {kernels[0]}, float64, one "
                               f"block per launch vs the mixed-precision persistent launch over all blocks"},
        "clocks": clk.summary(),
        "peaks_source": peaks["source"],
        "learned": learned,
        "autotune": tune or None,
    }
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = oracle_sample(args.workload, args.cpu_seconds, 7, os.cpu_count() or 1)
    return out


def run_reference(args) -> dict:
    """The CPU oracle as it stands, on the host cores, same workload and metric."""
    res = []
    for i in range(args.warmup + args.steps):
        r = oracle_sample(args.workload, args.ref_seconds, 100 + i, os.cpu_count() or 1)
        if i >= args.warmup:
            res.append(r)
    ent = sum(r["entries"] for r in res)
    sec = sum(r["seconds"] for r in res)
    value = ent / sec
    from inputs import workloads
    w = workloads.get(args.workload)
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "entries/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / len(res),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {**workloads.describe(w), "precision": "fp64 (oracle)"},
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
    k_apply_near, k_apply_far_dense, k_far_vx, k_far_uy, k_apply_finish."""
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="lshape12288")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--plain-blocks", type=int, default=400)
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
