"""ctypes binding of the C ABI in include/g3aca.h.

Argument marshalling only: every step of the hot path runs in the CUDA
library.  The functions keep the C names (build_cluster_tree,
assemble_near, aca3_compress, apply_gcq); handles are wrapped in small
classes that free themselves.  PyTorch is used only for device buffers and
the current CUDA stream.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libg3aca.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build the CUDA library first "
        "(python -c 'import __graft_entry__ as g; g.build()'); there is no CPU fallback")

_lib = C.CDLL(LIB_PATH)

# "hyp": hypersingular operator D, "adj": adjoint double layer K' (Galerkin,
# linear continuous elements, on a tree of build_p1_tree)
KERNELS = {"slp": 0, "dlp": 1, "hyp": 4, "adj": 5}
SCHEMES = {"colloc7": 0, "galerkin4x4": 1}
PRECISIONS = {"fp64": 0, "mixed": 1}
STATUS = {0: "G3_OK", -1: "G3_EINVAL", -2: "G3_ENOMEM", -3: "G3_ECUDA", -4: "G3_ETIMEOUT",
          -5: "G3_ENOCONV", -6: "G3_EOVERFLOW", -7: "G3_EUNSUPPORTED"}

_p = C.c_void_p
_pp = C.POINTER(C.c_void_p)
_i32p = C.POINTER(C.c_int32)
_dp = C.POINTER(C.c_double)
_i64p = C.POINTER(C.c_int64)


class Opts(C.Structure):
    _fields_ = [("face_rank_max", C.c_int), ("unbatched", C.c_int), ("ctas_per_sm", C.c_int),
                ("threads", C.c_int), ("no_recompress", C.c_int), ("order_by_cost", C.c_int),
                ("k1", _i32p), ("cost", C.POINTER(C.c_float)), ("pool_factor", C.c_double),
                ("eps_face", C.c_double), ("max_blocks", C.c_int), ("dense_face_max", C.c_int),
                ("literal_stop", C.c_int), ("mlp", C.c_void_p), ("mlp_use", C.c_int),
                ("face_floor_scale", C.c_double), ("trunc_floor_scale", C.c_double), ("pivot_index", C.c_int),
                ("graph", C.c_int), ("whole_matrix", C.c_int), ("residual_face_max", C.c_int)]


class TrainOpts(C.Structure):
    _fields_ = [("epochs", C.c_int), ("batch", C.c_int), ("lr", C.c_double), ("beta1", C.c_double),
                ("beta2", C.c_double), ("adam_eps", C.c_double), ("seed", C.c_uint64), ("no_graph", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("n_far", C.c_int64), ("entries", C.c_int64), ("crosses", C.c_int64),
                ("crosses_computed", C.c_int64), ("face_rank_sum", C.c_int64), ("factor_bytes", C.c_int64),
                ("dense_bytes", C.c_int64), ("r3_max", C.c_int32), ("face_rank_max", C.c_int32),
                ("zero_blocks", C.c_int32), ("capped_faces", C.c_int32), ("pool_regrows", C.c_int32),
                ("status_bits", C.c_int32), ("ms", C.c_double), ("phase_cycles", C.c_int64 * 7),
                ("ctas", C.c_int32), ("recompress_fallbacks", C.c_int32), ("blocks_run", C.c_int32),
                ("dense_crosses", C.c_int64), ("ms_lowrank", C.c_double), ("ms_dense", C.c_double),
                ("spilled_blocks", C.c_int32), ("mlp_used", C.c_int32), ("ms_mlp", C.c_double),
                ("face_check_restarts", C.c_int64), ("stop_check_overrides", C.c_int64),
                ("sub_cycles", C.c_int64 * 12), ("ms_host", C.c_double * 4), ("entries_face_dense", C.c_int64)]


def _sig(name, res, *args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = list(args)
    return f


_ci = C.c_int
_sig("g3_create", _ci, _ci, _p, _pp)
_sig("g3_set_stream", _ci, _p, _p)
_sig("g3_set_apply_tensor_cores", _ci, _p, _ci)
_sig("g3_destroy", _ci, _p)
_sig("g3_last_error", C.c_char_p)
_sig("g3_version", _ci)
_sig("g3_launch_count", C.c_int64, _p)
_sig("g3_kernel_name", C.c_char_p, _p, _ci, _i64p)
_sig("g3_freqs_bdf2", _ci, _p, _ci, C.c_double, C.c_double, _pp)
_sig("g3_freqs_gcq", _ci, _p, _ci, C.c_double, C.c_double, _pp)
_sig("g3_freqs_from_array", _ci, _p, _dp, _ci, _pp)
_sig("g3_freqs_info", _ci, _p, C.POINTER(_ci), C.POINTER(_ci))
_sig("g3_freqs_get", _ci, _p, _dp, _dp, _i32p, _i32p)
_sig("g3_freqs_free", _ci, _p)
_sig("build_cluster_tree", _ci, _p, _dp, _ci, _i32p, _ci, _ci, C.c_double, _pp)
_sig("build_cluster_tree_capped", _ci, _p, _dp, _ci, _i32p, _ci, _ci, C.c_double, _ci, _pp)
_sig("build_p1_tree", _ci, _p, _p, _pp)
_sig("g3_tree_info", _ci, _p, *(C.POINTER(_ci),) * 5)
_sig("g3_shard_rows", _ci, _i32p, _ci, _i32p, _ci, _dp, _ci, _i32p, _dp, C.POINTER(_ci))
_sig("g3_tree_partition_host", _ci, _dp, _ci, _i32p, _ci, _ci, C.c_double, _ci, _i32p, _i32p, C.c_int64,
     C.POINTER(C.c_int64))
_sig("g3_tree_subset", _ci, _p, _p, _i32p, _ci, _pp)
_sig("g3_tree_get", _ci, _p, _i32p, _i32p, _dp, _i32p, _i32p)
_sig("g3_tree_free", _ci, _p)
_sig("g3_entries", _ci, _p, _p, _p, _ci, _ci, _ci, _i32p, _i32p, _ci, _i32p, _ci, _dp)
_sig("assemble_near", _ci, _p, _p, _p, _ci, _ci, _ci, _pp)
_sig("g3_near_info", _ci, _p, _i64p, _i64p, _dp)
_sig("g3_near_get_block", _ci, _p, _ci, _dp)
_sig("g3_near_free", _ci, _p)
_sig("aca3_compress", _ci, _p, _p, _p, _ci, _ci, _ci, C.c_double, C.POINTER(Opts), _pp)
_sig("g3_autotune", _ci, _p, _p, _p, _ci, _ci, _ci, C.c_double, C.POINTER(Opts), _dp)
_sig("aca3_compress_batch", _ci, _p, _p, _p, _ci, _ci, _ci, _ci, C.c_double, C.POINTER(Opts), _p)
_sig("aca3_compress_separable", _ci, _p, _dp, _dp, _dp, _ci, _ci, _ci, _ci, _ci, C.c_double, C.POINTER(Opts), _pp)
_sig("g3_factors_stats", _ci, _p, C.POINTER(Stats))
_sig("g3_factors_ranks", _ci, _p, _i32p)
_sig("g3_factors_get_block", _ci, _p, _ci, _i32p, _i32p, _dp, _dp, _dp, _i32p)
_sig("g3_factors_block_cycles", _ci, _p, _i64p)
_sig("g3_factors_block_phases", _ci, _p, _i64p)
_sig("g3_factors_free", _ci, _p)
_sig("apply_gcq", _ci, _p, _p, _p, _p, _p, _p, _ci, _ci, _ci)
_sig("g3_apply_last", _ci, _p, _dp, _i64p, _dp, _i64p)
_sig("g3_peak", _ci, _p, _ci, _dp, _dp)
_sig("apply_gcq_noalloc", _ci, _p, _p, _p, _p, _p, _p, _ci)
_sig("g3_gcq_history", _ci, _p, _p, _ci, _p, _p, C.c_double, C.c_double, _p, _ci)
_fp = C.POINTER(C.c_float)
_sig("g3_mlp_create", _ci, _p, _fp, _fp, _fp, C.c_uint64, _pp)
_sig("g3_mlp_train", _ci, _p, _fp, _fp, _ci, C.POINTER(TrainOpts), _pp)
_sig("g3_mlp_fit", _ci, _p, _p, _fp, _fp, _ci, C.POINTER(TrainOpts), _fp)
_sig("g3_mlp_grad", _ci, _p, _p, _fp, _fp, _ci, _fp, _fp)
_sig("g3_mlp_predict", _ci, _p, _p, _fp, _ci, _fp)
_sig("g3_mlp_get", _ci, _p, _fp, _fp, _fp, _i64p, _fp, _fp)
_sig("g3_mlp_free", _ci, _p)
_sig("g3_block_features", _ci, _p, _p, _p, _ci, C.c_double, _fp)
_sig("g3_factors_labels", _ci, _p, _p, _fp)

EXPORTED = ["g3_create", "g3_set_stream", "g3_set_apply_tensor_cores", "g3_destroy", "g3_last_error", "g3_version", "g3_launch_count",
            "g3_kernel_name", "g3_freqs_bdf2", "g3_freqs_gcq", "g3_freqs_from_array", "g3_freqs_info", "g3_freqs_get", "g3_freqs_free",
            "build_cluster_tree", "build_cluster_tree_capped", "build_p1_tree", "g3_shard_rows", "g3_tree_partition_host", "g3_tree_subset", "g3_tree_info", "g3_tree_get", "g3_tree_free", "g3_entries", "assemble_near",
            "g3_near_info", "g3_near_get_block", "g3_near_free", "aca3_compress", "aca3_compress_batch", "g3_autotune", "aca3_compress_separable",
            "g3_factors_stats", "g3_factors_ranks", "g3_factors_block_cycles", "g3_factors_block_phases", "g3_factors_get_block", "g3_factors_free", "apply_gcq",
            "g3_apply_last", "g3_peak", "apply_gcq_noalloc", "g3_gcq_history", "g3_mlp_create", "g3_mlp_train", "g3_mlp_fit",
            "g3_mlp_grad", "g3_mlp_predict", "g3_mlp_get", "g3_mlp_free", "g3_block_features", "g3_factors_labels"]

MLP_NF = 12
MLP_NP = 5122


class G3Error(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib.g3_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")


def _check(st: int, where: str) -> None:
    if st != 0:
        raise G3Error(st, where)


def _arr(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(C.POINTER(ct))


class _Handle:
    _free = None

    def __init__(self, h, keep=()):
        self.h = h
        self._keep = keep   # objects this handle depends on (kept alive)

    def close(self):
        if self.h and self._free is not None:
            type(self)._free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context(_Handle):
    _free = _lib.g3_destroy

    def __init__(self, device: int = 0, stream=None):
        if stream is None:
            import torch
            stream = torch.cuda.current_stream(device).cuda_stream
        h = C.c_void_p()
        _check(_lib.g3_create(device, C.c_void_p(stream), C.byref(h)), "g3_create")
        super().__init__(h)
        self.device = device

    def set_stream(self, stream) -> None:
        _check(_lib.g3_set_stream(self.h, C.c_void_p(stream)), "g3_set_stream")

    def set_apply_tensor_cores(self, on: bool) -> None:
        """Far-field x formation of float32 applies on the tensor cores (default) or the CUDA cores."""
        _check(_lib.g3_set_apply_tensor_cores(self.h, 1 if on else 0), "g3_set_apply_tensor_cores")

    def launch_count(self) -> int:
        return int(_lib.g3_launch_count(self.h))

    def kernel_launches(self) -> dict:
        out, i = {}, 0
        n = C.c_int64()
        while True:
            name = _lib.g3_kernel_name(self.h, i, C.byref(n))
            if name is None:
                return out
            out[name.decode()] = int(n.value)
            i += 1

    def peak(self, kind: str) -> float:
        """Measured operations/s of one pipe: ffma, rsqrt, ex2, sin, cos, dfma."""
        k = ["ffma", "rsqrt", "ex2", "sin", "cos", "dfma"].index(kind)
        ops, ms = C.c_double(), C.c_double()
        _check(_lib.g3_peak(self.h, k, C.byref(ops), C.byref(ms)), "g3_peak")
        return ops.value

    def last_apply(self) -> dict:
        ms, nms = C.c_double(), C.c_double()
        b, nb = C.c_int64(), C.c_int64()
        _check(_lib.g3_apply_last(self.h, C.byref(ms), C.byref(b), C.byref(nms), C.byref(nb)), "g3_apply_last")
        return {"ms": ms.value, "bytes": b.value, "near_ms": nms.value, "near_bytes": nb.value}


class Freqs(_Handle):
    _free = _lib.g3_freqs_free

    def info(self) -> tuple[int, int]:
        K, Ku = C.c_int(), C.c_int()
        _check(_lib.g3_freqs_info(self.h, C.byref(K), C.byref(Ku)), "g3_freqs_info")
        return K.value, Ku.value

    def get(self) -> dict:
        K, Ku = self.info()
        s = np.zeros(2 * K)
        w = np.zeros(2 * K)
        u = np.zeros(Ku, dtype=np.int32)
        p = np.zeros(K, dtype=np.int32)
        _check(_lib.g3_freqs_get(self.h, _ptr(s, C.c_double), _ptr(w, C.c_double), _ptr(u, C.c_int32),
                                 _ptr(p, C.c_int32)), "g3_freqs_get")
        return {"s": s.view(np.complex128), "omega": w.view(np.complex128), "uniq": u, "partner": p}


def g3_freqs_bdf2(ctx: Context, K: int, lam: float, dt: float) -> Freqs:
    h = C.c_void_p()
    _check(_lib.g3_freqs_bdf2(ctx.h, K, lam, dt, C.byref(h)), "g3_freqs_bdf2")
    return Freqs(h, (ctx,))


def g3_freqs_gcq(ctx: Context, NQ: int, dt_min: float, dt_max: float) -> Freqs:
    h = C.c_void_p()
    _check(_lib.g3_freqs_gcq(ctx.h, NQ, dt_min, dt_max, C.byref(h)), "g3_freqs_gcq")
    return Freqs(h, (ctx,))


def g3_freqs_from_array(ctx: Context, s) -> Freqs:
    """Frequency set from a complex array (conjugate pairs detected)."""
    a = np.ascontiguousarray(np.asarray(s, dtype=np.complex128))
    h = C.c_void_p()
    _check(_lib.g3_freqs_from_array(ctx.h, _ptr(a.view(np.float64), C.c_double), a.size, C.byref(h)),
           "g3_freqs_from_array")
    return Freqs(h, (ctx,))


def freqs_from_spec(ctx: Context, spec) -> Freqs:
    if spec.kind == "bdf2":
        return g3_freqs_bdf2(ctx, spec.K, spec.lam, spec.dt)
    return g3_freqs_gcq(ctx, spec.K, spec.dt_min, spec.dt_max)


class Tree(_Handle):
    _free = _lib.g3_tree_free

    def info(self) -> dict:
        v = [C.c_int() for _ in range(5)]
        _check(_lib.g3_tree_info(self.h, *[C.byref(x) for x in v]), "g3_tree_info")
        return dict(zip(["ne", "n_nodes", "n_blocks", "n_far", "n_near"], [x.value for x in v]))

    def get(self) -> dict:
        i = self.info()
        perm = np.zeros(i["ne"], dtype=np.int32)
        nodes = np.zeros((i["n_nodes"], 4), dtype=np.int32)
        boxes = np.zeros((i["n_nodes"], 6))
        blocks = np.zeros((i["n_blocks"], 5), dtype=np.int32)
        far = np.zeros(i["n_far"], dtype=np.int32)
        _check(_lib.g3_tree_get(self.h, _ptr(perm, C.c_int32), _ptr(nodes, C.c_int32), _ptr(boxes, C.c_double),
                                _ptr(blocks, C.c_int32), _ptr(far, C.c_int32)), "g3_tree_get")
        return {"perm": perm, "nodes": nodes, "boxes": boxes, "blocks": blocks, "far_index": far}


def build_cluster_tree(ctx: Context, verts, tris, leaf: int = 32, eta: float = 1.0, max_block: int = 0) -> Tree:
    """Cluster tree and block partition; max_block > 0 caps the larger side of
    a far block (build_cluster_tree_capped)."""
    v = _arr(verts, np.float64)
    t = _arr(tris, np.int32)
    h = C.c_void_p()
    _check(_lib.build_cluster_tree_capped(ctx.h, _ptr(v, C.c_double), v.shape[0], _ptr(t, C.c_int32), t.shape[0],
                                          leaf, eta, max_block, C.byref(h)), "build_cluster_tree")
    return Tree(h, (ctx,))


def build_p1_tree(ctx: Context, tree: Tree) -> Tree:
    """Tree of element-local linear shape functions over an element tree:
    row 3 e + a is local vertex a of element e (cluster position 3 p + a);
    the operators "hyp" and "adj" with scheme "galerkin4x4" run on it, and
    apply_gcq on it takes nodal densities (nv rows) and returns nodal y."""
    h = C.c_void_p()
    _check(_lib.build_p1_tree(ctx.h, tree.h, C.byref(h)), "build_p1_tree")
    return Tree(h, (ctx,))


def tree_partition_host(verts, tris, leaf: int, eta: float, max_block: int = 0) -> dict:
    """The cluster tree's permutation and block list from the host builder
    alone (no context or device): the same arrays as `Tree.get()`."""
    v = np.ascontiguousarray(verts, dtype=np.float64)
    t = np.ascontiguousarray(tris, dtype=np.int32)
    nb = C.c_int64(0)
    _check(_lib.g3_tree_partition_host(_ptr(v, C.c_double), v.shape[0], _ptr(t, C.c_int32), t.shape[0], leaf, eta,
                                       max_block, None, None, 0, C.byref(nb)), "g3_tree_partition_host")
    perm = np.empty(t.shape[0], dtype=np.int32)
    blocks = np.empty((nb.value, 5), dtype=np.int32)
    _check(_lib.g3_tree_partition_host(_ptr(v, C.c_double), v.shape[0], _ptr(t, C.c_int32), t.shape[0], leaf, eta,
                                       max_block, _ptr(perm, C.c_int32), _ptr(blocks, C.c_int32), nb.value,
                                       C.byref(nb)), "g3_tree_partition_host")
    return {"perm": perm, "blocks": blocks}


def shard_rows(nodes, blocks, n_ranks: int, cost=None) -> dict:
    """Row-cluster partition of a block list over n_ranks (host only, no GPU):
    {"owner": [n_blocks], "load": [n_ranks], "n_units": int}."""
    nd = _arr(nodes, np.int32)
    bl = _arr(blocks, np.int32)
    nb = bl.shape[0]
    owner = np.zeros(max(nb, 1), dtype=np.int32)
    load = np.zeros(n_ranks)
    nu = C.c_int()
    c = None if cost is None else _arr(cost, np.float64)
    _check(_lib.g3_shard_rows(_ptr(nd, C.c_int32), nd.shape[0], _ptr(bl, C.c_int32), nb,
                              None if c is None else _ptr(c, C.c_double), n_ranks, _ptr(owner, C.c_int32),
                              _ptr(load, C.c_double), C.byref(nu)), "g3_shard_rows")
    return {"owner": owner[:nb], "load": load, "n_units": nu.value}


def tree_subset(ctx: Context, tree: Tree, owner, rank: int) -> Tree:
    """The blocks of `tree` owned by `rank` (g3_tree_subset)."""
    o = _arr(owner, np.int32)
    if o.size != tree.info()["n_blocks"]:
        raise ValueError("owner must have one entry per block")
    h = C.c_void_p()
    _check(_lib.g3_tree_subset(ctx.h, tree.h, _ptr(o, C.c_int32), rank, C.byref(h)), "g3_tree_subset")
    return Tree(h, (ctx,))


def g3_entries(ctx: Context, tree: Tree, freqs: Freqs, kernel: str, rows, cols, kidx, prec: str = "fp64",
               scheme: str = "colloc7") -> np.ndarray:
    r = _arr(rows, np.int32)
    c = _arr(cols, np.int32)
    k = _arr(kidx, np.int32)
    out = np.zeros(2 * r.size * k.size)
    _check(_lib.g3_entries(ctx.h, tree.h, freqs.h, KERNELS[kernel], SCHEMES[scheme], PRECISIONS[prec],
                           _ptr(r, C.c_int32), _ptr(c, C.c_int32), r.size, _ptr(k, C.c_int32), k.size,
                           _ptr(out, C.c_double)), "g3_entries")
    return out.view(np.complex128).reshape(r.size, k.size)


class Near(_Handle):
    _free = _lib.g3_near_free

    def info(self) -> dict:
        n, b, ms = C.c_int64(), C.c_int64(), C.c_double()
        _check(_lib.g3_near_info(self.h, C.byref(n), C.byref(b), C.byref(ms)), "g3_near_info")
        return {"entries": n.value, "bytes": b.value, "ms": ms.value}

    def block(self, b: int, M: int, N: int, Ku: int) -> np.ndarray:
        out = np.zeros(2 * M * N * Ku)
        _check(_lib.g3_near_get_block(self.h, b, _ptr(out, C.c_double)), "g3_near_get_block")
        return out.view(np.complex128).reshape(Ku, M, N)


def assemble_near(ctx: Context, tree: Tree, freqs: Freqs, kernel: str = "slp", scheme: str = "colloc7",
                  prec: str = "mixed") -> Near:
    h = C.c_void_p()
    _check(_lib.assemble_near(ctx.h, tree.h, freqs.h, KERNELS[kernel], SCHEMES[scheme], PRECISIONS[prec],
                              C.byref(h)), "assemble_near")
    return Near(h, (ctx, tree, freqs))


class Factors(_Handle):
    _free = _lib.g3_factors_free

    def stats(self) -> dict:
        s = Stats()
        _check(_lib.g3_factors_stats(self.h, C.byref(s)), "g3_factors_stats")
        out = {f: getattr(s, f) for f, _ in Stats._fields_}
        out["phase_cycles"] = dict(zip(["face", "recompress", "formation", "pivot", "fiber", "norm", "next_k"],
                                       list(s.phase_cycles)))
        out["sub_cycles"] = dict(zip(["rc_gram", "rc_cholesky", "rc_core", "rc_jacobi", "rc_rest", "face_table",
                                      "face_rows", "face_columns", "face_norm", "face_samples", "line_entries", "dense_residual_faces"],
                                     list(s.sub_cycles)))
        out["ms_host"] = dict(zip(["setup", "rounds", "readback", "apply_plan"], list(s.ms_host)))
        return out

    def ranks(self) -> np.ndarray:
        n = self.stats()["n_far"]
        r = np.zeros(n, dtype=np.int32)
        _check(_lib.g3_factors_ranks(self.h, _ptr(r, C.c_int32)), "g3_factors_ranks")
        return r

    def block_cycles(self) -> np.ndarray:
        n = self.stats()["n_far"]
        c = np.zeros(n, dtype=np.int64)
        _check(_lib.g3_factors_block_cycles(self.h, _ptr(c, C.c_int64)), "g3_factors_block_cycles")
        return c

    def block_phases(self) -> np.ndarray:
        """[n_far, 10]: SM cycles per phase (face, recompress, formation, pivot,
        fiber, norm, next_k), the block's face ACA steps, and its start and end
        times (GPU global timer, ns)."""
        n = self.stats()["n_far"]
        c = np.zeros((max(n, 1), 10), dtype=np.int64)
        _check(_lib.g3_factors_block_phases(self.h, _ptr(c, C.c_int64)), "g3_factors_block_phases")
        return c[:n]

    def block(self, i: int, M: int, N: int, Ku: int) -> dict:
        r3 = C.c_int32()
        _check(_lib.g3_factors_get_block(self.h, i, C.byref(r3), None, None, None, None, None), "g3_factors_get_block")
        n = r3.value
        fr = np.zeros(max(n, 1), dtype=np.int32)
        _check(_lib.g3_factors_get_block(self.h, i, C.byref(r3), _ptr(fr, C.c_int32), None, None, None, None),
               "g3_factors_get_block")
        fr = fr[:n]
        U = np.zeros(2 * int(fr.sum()) * M + 2)
        V = np.zeros(2 * int(fr.sum()) * N + 2)
        F = np.zeros(2 * n * Ku + 2)
        P = np.zeros(3 * n + 1, dtype=np.int32)
        _check(_lib.g3_factors_get_block(self.h, i, C.byref(r3), _ptr(fr, C.c_int32), _ptr(U, C.c_double),
                                         _ptr(V, C.c_double), _ptr(F, C.c_double), _ptr(P, C.c_int32)),
               "g3_factors_get_block")
        Uc = U[:-2].view(np.complex128)
        Vc = V[:-2].view(np.complex128)
        us, vs, ou, ov = [], [], 0, 0
        for r in fr:
            us.append(Uc[ou:ou + r * M].reshape(r, M).T)
            vs.append(Vc[ov:ov + r * N].reshape(r, N).T)
            ou += r * M
            ov += r * N
        return {"U": us, "V": vs, "f": F[:-2].view(np.complex128).reshape(n, Ku),
                "piv": P[:-1].reshape(n, 3), "face_ranks": fr}

    def labels(self) -> np.ndarray:
        """Predictor training labels [n_far, 2]: log2(1 + r3), k* / Ku."""
        n = self.stats()["n_far"]
        out = np.zeros((max(n, 1), 2), dtype=np.float32)
        _check(_lib.g3_factors_labels(self._keep[0].h, self.h, _ptr(out, C.c_float)), "g3_factors_labels")
        return out[:n]


def _train_opts(**kw) -> TrainOpts:
    o = TrainOpts()
    for k, v in kw.items():
        if v is not None:
            setattr(o, k, v)
    return o


def _f32(a, shape_tail):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    if a.ndim != 2 or a.shape[1] != shape_tail:
        raise ValueError(f"expected an [n, {shape_tail}] array, got {a.shape}")
    return a


class Mlp(_Handle):
    """Block rank / first-frequency predictor (12 -> 64 -> 64 -> 2)."""
    _free = _lib.g3_mlp_free

    def predict(self, feats) -> np.ndarray:
        X = _f32(feats, MLP_NF)
        out = np.zeros((max(X.shape[0], 1), 2), dtype=np.float32)
        _check(_lib.g3_mlp_predict(self._keep[0].h, self.h, _ptr(X, C.c_float), X.shape[0], _ptr(out, C.c_float)),
               "g3_mlp_predict")
        return out[:X.shape[0]]

    def grad(self, feats, labels):
        X, Y = _f32(feats, MLP_NF), _f32(labels, 2)
        g = np.zeros(MLP_NP, dtype=np.float32)
        loss = np.zeros(1, dtype=np.float32)
        _check(_lib.g3_mlp_grad(self._keep[0].h, self.h, _ptr(X, C.c_float), _ptr(Y, C.c_float), X.shape[0],
                                _ptr(g, C.c_float), _ptr(loss, C.c_float)), "g3_mlp_grad")
        return g, float(loss[0])

    def fit(self, feats, labels, **opts) -> np.ndarray:
        X, Y = _f32(feats, MLP_NF), _f32(labels, 2)
        o = _train_opts(**opts)
        epochs = o.epochs or 200
        batch = o.batch or 256
        losses = np.zeros(epochs * (-(-X.shape[0] // batch)), dtype=np.float32)
        _check(_lib.g3_mlp_fit(self._keep[0].h, self.h, _ptr(X, C.c_float), _ptr(Y, C.c_float), X.shape[0],
                               C.byref(o), _ptr(losses, C.c_float)), "g3_mlp_fit")
        return losses

    def get(self) -> dict:
        P, m, v = (np.zeros(MLP_NP, dtype=np.float32) for _ in range(3))
        mean, inv = np.zeros(MLP_NF, dtype=np.float32), np.zeros(MLP_NF, dtype=np.float32)
        t = C.c_int64()
        _check(_lib.g3_mlp_get(self.h, _ptr(P, C.c_float), _ptr(m, C.c_float), _ptr(v, C.c_float), C.byref(t),
                               _ptr(mean, C.c_float), _ptr(inv, C.c_float)), "g3_mlp_get")
        return {"params": P, "m": m, "v": v, "t": t.value, "mean": mean, "inv_std": inv}


def mlp_create(ctx: Context, params=None, mean=None, inv_std=None, seed: int = 0) -> Mlp:
    keep = [None if a is None else np.ascontiguousarray(np.asarray(a, dtype=np.float32)) for a in (params, mean, inv_std)]
    if keep[0] is not None and keep[0].size != MLP_NP:
        raise ValueError(f"params must have {MLP_NP} values")
    for a in keep[1:]:
        if a is not None and a.size != MLP_NF:
            raise ValueError(f"mean / inv_std must have {MLP_NF} values")
    ptrs = [None if a is None else _ptr(a, C.c_float) for a in keep]
    h = C.c_void_p()
    _check(_lib.g3_mlp_create(ctx.h, *ptrs, seed, C.byref(h)), "g3_mlp_create")
    return Mlp(h, (ctx,))


def mlp_train(ctx: Context, feats, labels, **opts) -> Mlp:
    X, Y = _f32(feats, MLP_NF), _f32(labels, 2)
    o = _train_opts(**opts)
    h = C.c_void_p()
    _check(_lib.g3_mlp_train(ctx.h, _ptr(X, C.c_float), _ptr(Y, C.c_float), X.shape[0], C.byref(o), C.byref(h)),
           "g3_mlp_train")
    return Mlp(h, (ctx,))


def block_features(ctx: Context, tree: Tree, freqs: Freqs, kernel: str = "slp", eps3: float = 1e-4) -> np.ndarray:
    n = tree.info()["n_far"]
    out = np.zeros((max(n, 1), MLP_NF), dtype=np.float32)
    _check(_lib.g3_block_features(ctx.h, tree.h, freqs.h, KERNELS[kernel], eps3, _ptr(out, C.c_float)),
           "g3_block_features")
    return out[:n]


def _opts(**kw) -> Opts:
    o = Opts()
    keep = []
    for k, v in kw.items():
        if v is None:
            continue
        if k == "k1":
            a = _arr(v, np.int32)
            keep.append(a)
            o.k1 = _ptr(a, C.c_int32)
        elif k == "cost":
            a = _arr(v, np.float32)
            keep.append(a)
            o.cost = _ptr(a, C.c_float)
        elif k == "mlp":
            keep.append(v)
            o.mlp = v.h
        else:
            setattr(o, k, v)
    o._keep = keep
    return o


def aca3_compress(ctx: Context, tree: Tree, freqs: Freqs, kernel: str = "slp", scheme: str = "colloc7",
                  prec: str = "mixed", eps3: float = 1e-4, **opts) -> Factors:
    o = _opts(**opts)
    h = C.c_void_p()
    _check(_lib.aca3_compress(ctx.h, tree.h, freqs.h, KERNELS[kernel], SCHEMES[scheme], PRECISIONS[prec], eps3,
                              C.byref(o), C.byref(h)), "aca3_compress")
    return Factors(h, (ctx, tree, freqs))


def autotune(ctx: Context, tree: Tree, freqs: Freqs, kernel: str = "slp", scheme: str = "colloc7",
             prec: str = "mixed", eps3: float = 1e-4, **opts) -> dict:
    """Fastest launch shape of aca3_compress on this problem (cached per
    problem class in the context): {"threads", "dense_face_max",
    "residual_face_max", "ms"}."""
    o = _opts(**opts)
    ms = C.c_double()
    _check(_lib.g3_autotune(ctx.h, tree.h, freqs.h, KERNELS[kernel], SCHEMES[scheme], PRECISIONS[prec], eps3,
                            C.byref(o), C.byref(ms)), "g3_autotune")
    return {"threads": o.threads, "dense_face_max": o.dense_face_max, "residual_face_max": o.residual_face_max,
            "ms": ms.value}


def aca3_compress_batch(ctx: Context, trees, freqs, kernel: str = "slp", scheme: str = "colloc7",
                        prec: str = "mixed", eps3: float = 1e-4, **opts) -> list:
    """All admissible blocks of several meshes in one persistent launch;
    returns one Factors per mesh."""
    n = len(trees)
    if len(freqs) != n or n == 0:
        raise ValueError("need one frequency set per tree")
    th = (C.c_void_p * n)(*[t.h for t in trees])
    fh = (C.c_void_p * n)(*[f.h for f in freqs])
    out = (C.c_void_p * n)()
    o = _opts(**opts)
    _check(_lib.aca3_compress_batch(ctx.h, th, fh, n, KERNELS[kernel], SCHEMES[scheme], PRECISIONS[prec], eps3,
                                    C.byref(o), out), "aca3_compress_batch")
    return [Factors(C.c_void_p(out[j]), (ctx, trees[j], freqs[j])) for j in range(n)]


def aca3_compress_separable(ctx: Context, a, b, c, prec: str = "fp64", eps3: float = 1e-6, **opts) -> Factors:
    a = _arr(a, np.complex128)
    b = _arr(b, np.complex128)
    c = _arr(c, np.complex128)
    R, M = a.shape
    N = b.shape[1]
    Ku = c.shape[1]
    o = _opts(**opts)
    h = C.c_void_p()
    _check(_lib.aca3_compress_separable(ctx.h, _ptr(a.view(np.float64), C.c_double), _ptr(b.view(np.float64), C.c_double),
                                        _ptr(c.view(np.float64), C.c_double), R, M, N, Ku, PRECISIONS[prec], eps3,
                                        C.byref(o), C.byref(h)), "aca3_compress_separable")
    return Factors(h, (ctx,))


def apply_gcq(ctx: Context, tree: Tree, near: Near | None, factors: Factors | None, W, Y=None, mode: str = "sum"):
    """y = sum_l A(s_l) w_l.  W: torch CUDA tensor (device path) or numpy array
    (host path: copies inside the call), complex64 or complex128, shape [M, K]
    with column l = w_l (the call reads W in column-major order)."""
    mode_i = {"sum": 0, "perfreq": 1}[mode]
    nh = near.h if near is not None else None
    fh = factors.h if factors is not None else None
    if isinstance(W, np.ndarray):
        dt = 1 if W.dtype == np.complex128 else 0
        Wc = np.asfortranarray(W)
        M = W.shape[0]
        out = np.zeros(M if mode_i == 0 else W.shape, dtype=W.dtype, order="F")
        _check(_lib.apply_gcq(ctx.h, tree.h, nh, fh, Wc.ctypes.data_as(C.c_void_p), out.ctypes.data_as(C.c_void_p),
                              dt, mode_i, 1), "apply_gcq")
        return out
    import torch
    if not (W.is_cuda and W.dtype in (torch.complex64, torch.complex128)):
        raise TypeError("W must be a complex CUDA tensor or a numpy array")
    dt = 1 if W.dtype == torch.complex128 else 0
    Wt = W.t().contiguous()          # [K, M]: column l of W contiguous
    M = W.shape[0]
    if Y is None:
        Y = torch.empty(M if mode_i == 0 else (W.shape[1], M), dtype=W.dtype, device=W.device)
    _check(_lib.apply_gcq(ctx.h, tree.h, nh, fh, C.c_void_p(Wt.data_ptr()), C.c_void_p(Y.data_ptr()), dt, mode_i, 0),
           "apply_gcq")
    return Y if mode_i == 0 else Y.t()


def apply_gcq_noalloc(ctx: Context, tree: Tree, near: Near | None, factors: Factors | None, W, Y):
    """Allocation-free apply (same result as apply_gcq on device buffers).

    W: complex CUDA tensor [M, K] whose columns are contiguous in memory (the
    transpose of a contiguous [K, M] tensor, e.g. ``Wt.t()``); Y: preallocated
    complex CUDA tensor [M] of W's dtype.  Neither this wrapper nor the
    library allocates device memory; both read and write in order on the
    context's stream."""
    import torch
    if not (W.is_cuda and W.dtype in (torch.complex64, torch.complex128)):
        raise TypeError("W must be a complex CUDA tensor")
    if W.dim() != 2 or not W.t().is_contiguous():
        raise ValueError("W must be [M, K] with contiguous columns (pass Wt.t() of a contiguous [K, M] tensor)")
    if Y is None or not (Y.is_cuda and Y.dtype == W.dtype and Y.is_contiguous() and Y.numel() == W.shape[0]):
        raise ValueError("Y must be a preallocated contiguous CUDA tensor [M] of W's dtype")
    dt = 1 if W.dtype == torch.complex128 else 0
    _check(_lib.apply_gcq_noalloc(ctx.h, tree.h, near.h if near is not None else None,
                                  factors.h if factors is not None else None, C.c_void_p(W.data_ptr()),
                                  C.c_void_p(Y.data_ptr()), dt), "apply_gcq_noalloc")
    return Y


def gcq_history(ctx: Context, freqs: Freqs, X, theta, dt_prev: float, dt_next: float, W=None):
    """One gCQ history step (g3_gcq_history): X [M, K] complex CUDA tensor with
    contiguous columns (updated in place), theta [M] (or None), returns
    W [M, K] (the weights for apply_gcq) in X's layout."""
    import torch
    if not (X.is_cuda and X.dtype in (torch.complex64, torch.complex128)) or not X.t().is_contiguous():
        raise ValueError("X must be a complex CUDA tensor [M, K] with contiguous columns")
    M = X.shape[0]
    if W is None:
        W = torch.empty((X.shape[1], M), dtype=X.dtype, device=X.device).t()
    th = None
    if theta is not None:
        if not (theta.is_cuda and theta.dtype == X.dtype and theta.is_contiguous() and theta.numel() == M):
            raise ValueError("theta must be a contiguous CUDA tensor [M] of X's dtype")
        th = C.c_void_p(theta.data_ptr())
    dt = 1 if X.dtype == torch.complex128 else 0
    _check(_lib.g3_gcq_history(ctx.h, freqs.h, M, C.c_void_p(X.data_ptr()), th, dt_prev, dt_next,
                               C.c_void_p(W.data_ptr()), dt), "g3_gcq_history")
    return W
