"""Python binding of libskm (C ABI in include/skm.h): argument marshalling only.

Every step of the clustering runs in the CUDA library; this module builds the
argument structs, hands over pointers (numpy arrays for host memory, torch tensors
for device memory) and turns status codes into exceptions. There is no CPU fallback:
if the library cannot be built or loaded, every call raises.

The functions ``skm_create``, ``skm_fit``, ``skm_assign``, ``skm_update``,
``skm_set_centroids``, ``skm_get_centroids``, ``skm_get_stats`` and ``skm_destroy``
mirror the C entry points of the same names. ``SphericalKMeans`` is a thin owner of
one context on top of them.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

SKM_OK, SKM_ERR_INVALID, SKM_ERR_OOM, SKM_ERR_BUDGET, SKM_ERR_CUDA, SKM_ERR_STATE, SKM_ERR_TIMEOUT = range(7)
STATUS_NAMES = {0: "SKM_OK", 1: "SKM_ERR_INVALID", 2: "SKM_ERR_OOM", 3: "SKM_ERR_BUDGET",
                4: "SKM_ERR_CUDA", 5: "SKM_ERR_STATE", 6: "SKM_ERR_TIMEOUT"}
SKM_FP32, SKM_BF16 = 0, 1
SKM_PRUNE_NONE, SKM_PRUNE_NCC, SKM_PRUNE_NCC_INDEX = 0, 1, 2
PRUNE_MODES = {"none": SKM_PRUNE_NONE, "ncc": SKM_PRUNE_NCC, "ncc_index": SKM_PRUNE_NCC_INDEX}

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class skm_config(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("precision", ctypes.c_int32), ("prune", ctypes.c_int32),
                ("max_iter", ctypes.c_int32), ("shift_tol", ctypes.c_double),
                ("rescore", ctypes.c_int32), ("rescore_tau", ctypes.c_double),
                ("mem_budget", ctypes.c_size_t), ("device", ctypes.c_int32),
                ("stream", ctypes.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("alloc_user", ctypes.c_void_p), ("timing", ctypes.c_int32),
                ("sparse_div", ctypes.c_int32), ("index_levels", ctypes.c_int32),
                ("index_lambda", ctypes.c_double * 4), ("index_min_changed", ctypes.c_int32),
                ("index_max_cands", ctypes.c_int32), ("head_terms", ctypes.c_int32)]


class skm_csr(ctypes.Structure):
    _fields_ = [("n_docs", ctypes.c_int64), ("n_terms", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p),
                ("values", ctypes.c_void_p), ("on_device", ctypes.c_int32)]


class skm_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("sims", ctypes.c_int64), ("fmas", ctypes.c_int64),
                ("bytes", ctypes.c_int64), ("docs_pruned", ctypes.c_int64),
                ("docs_full", ctypes.c_int64), ("docs_rescored", ctypes.c_int64),
                ("docs_rescored_full", ctypes.c_int64), ("moved_total", ctypes.c_int64),
                ("ms_score", ctypes.c_double), ("ms_decide", ctypes.c_double),
                ("ms_update", ctypes.c_double), ("launches_score", ctypes.c_int64),
                ("launches_total", ctypes.c_int64), ("fmas_exec", ctypes.c_int64),
                ("ms_index", ctypes.c_double), ("sparse_rows", ctypes.c_int64),
                ("sparse_entries", ctypes.c_int64), ("index_docs", ctypes.c_int64),
                ("index_sims", ctypes.c_int64), ("index_entries", ctypes.c_int64),
                ("index_products", ctypes.c_int64), ("ms_query", ctypes.c_double),
                ("head_terms", ctypes.c_int32), ("nnz_head", ctypes.c_int64), ("ms_head", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class skm_batch_item(ctypes.Structure):
    _fields_ = [("docs", skm_csr), ("k", ctypes.c_int32), ("init_doc_ids", ctypes.c_void_p),
                ("assign_out", ctypes.c_void_p), ("objective_out", ctypes.c_void_p)]


class skm_batch_config(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int32), ("rescore", ctypes.c_int32), ("rescore_tau", ctypes.c_double),
                ("device", ctypes.c_int32), ("stream", ctypes.c_void_p), ("alloc", ALLOC_FN),
                ("free", FREE_FN), ("alloc_user", ctypes.c_void_p), ("tune_cache", ctypes.c_char_p),
                ("use_graph", ctypes.c_int32)]


class skm_batch_stats(ctypes.Structure):
    _fields_ = [("ms_total", ctypes.c_double), ("ms_setup", ctypes.c_double), ("ms_loop", ctypes.c_double),
                ("fmas", ctypes.c_int64), ("tiles", ctypes.c_int64), ("graph_nodes", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("tuned", ctypes.c_int32),
                ("shape_instances", ctypes.c_int32 * 5), ("message", ctypes.c_char * 256)]

    def as_dict(self) -> dict:
        d = {name: getattr(self, name) for name, _ in self._fields_ if name not in ("shape_instances", "message")}
        d["shape_instances"] = dict(zip(("lane16", "lane32", "w128", "w256", "w512"), list(self.shape_instances)))
        d["message"] = self.message.decode(errors="replace")
        return d


class skm_server_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("mem_budget", ctypes.c_size_t), ("n_job_slots", ctypes.c_int32),
                ("max_batch_docs", ctypes.c_int64), ("max_batch_nnz", ctypes.c_int64),
                ("job_precision", ctypes.c_int32), ("job_prune", ctypes.c_int32), ("rescore_tau", ctypes.c_double)]


class skm_server_result(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("status", ctypes.c_int), ("n_docs", ctypes.c_int64),
                ("assign", ctypes.POINTER(ctypes.c_int32)), ("score", ctypes.POINTER(ctypes.c_float)),
                ("objective", ctypes.POINTER(ctypes.c_double)), ("iters", ctypes.c_int32),
                ("latency_ms", ctypes.c_double), ("queue_ms", ctypes.c_double), ("batch_docs", ctypes.c_int32),
                ("message", ctypes.c_char * 256)]


class skm_server_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("assign_submitted", "assign_done", "fit_submitted", "fit_done",
                                              "rejected", "failed", "assign_batches", "max_batch_docs_seen",
                                              "docs_assigned", "docs_clustered", "assign_queued", "fit_queued")] + \
               [("jobs_running", ctypes.c_int32), ("peak_jobs_running", ctypes.c_int32),
                ("jobs_mem", ctypes.c_size_t), ("resident_mem", ctypes.c_size_t)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


REQ_STATES = {0: "queued", 1: "running", 2: "done", 3: "rejected", 4: "failed", 5: "cancelled"}

EXPORTS = ("skm_config_default", "skm_create", "skm_destroy", "skm_last_error", "skm_fit",
           "skm_assign", "skm_update", "skm_set_centroids", "skm_get_centroids", "skm_n_terms",
           "skm_get_stats", "skm_mem_used", "skm_fit_batched", "skm_server_create", "skm_server_submit_assign",
           "skm_server_submit_fit", "skm_server_wait", "skm_server_release", "skm_server_get_stats",
           "skm_server_destroy", "skm_assign_fixed_scratch", "skm_init_kmeanspp",
           "skm_index_candidates", "skm_device_code_version")

# skm_assign_fixed_scratch: capacity of its fixed scratch, in (document x 256-column slice) units
FIXED_SCRATCH_SLICE = 256
FIXED_SCRATCH_UNITS = 1_048_568


def load(build_if_missing: bool = True):
    """Load libskm.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB_PATH
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libskm.so not found at {path}; run paper_2108_00895_gb300.build")
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        st = ctypes.c_int
        sig = {
            "skm_config_default": (None, [ctypes.POINTER(skm_config), ctypes.c_int32]),
            "skm_create": (st, [ctypes.POINTER(skm_config), ctypes.POINTER(P)]),
            "skm_destroy": (st, [P]),
            "skm_last_error": (ctypes.c_char_p, [P]),
            "skm_fit": (st, [P, ctypes.POINTER(skm_csr), P, P, P, P]),
            "skm_assign": (st, [P, ctypes.POINTER(skm_csr), P, P]),
            "skm_update": (st, [P, ctypes.POINTER(skm_csr), P, P]),
            "skm_init_kmeanspp": (st, [P, ctypes.POINTER(skm_csr), P, P]),
            "skm_index_candidates": (st, [P, ctypes.POINTER(skm_csr), ctypes.c_int32, P]),
            "skm_set_centroids": (st, [P, ctypes.c_int32, P, ctypes.c_int32]),
            "skm_get_centroids": (st, [P, P, ctypes.c_int32]),
            "skm_n_terms": (ctypes.c_int32, [P]),
            "skm_get_stats": (st, [P, ctypes.POINTER(skm_stats)]),
            "skm_mem_used": (ctypes.c_size_t, [P]),
            "skm_device_code_version": (st, [ctypes.POINTER(ctypes.c_int32)]),
            "skm_assign_fixed_scratch": (st, [ctypes.POINTER(skm_csr), ctypes.c_int32, P, ctypes.c_int64,
                                              P, P, P]),
            "skm_fit_batched": (st, [ctypes.POINTER(skm_batch_config), ctypes.POINTER(skm_batch_item),
                                     ctypes.c_int32, ctypes.POINTER(skm_batch_stats)]),
            "skm_server_create": (st, [ctypes.POINTER(skm_server_config), P, ctypes.POINTER(P)]),
            "skm_server_submit_assign": (st, [P, ctypes.POINTER(skm_csr), ctypes.POINTER(ctypes.c_uint64)]),
            "skm_server_submit_fit": (st, [P, ctypes.POINTER(skm_csr), ctypes.c_int32, P, ctypes.c_int32,
                                           ctypes.POINTER(ctypes.c_uint64)]),
            "skm_server_wait": (st, [P, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(skm_server_result)]),
            "skm_server_release": (st, [P, ctypes.c_uint64]),
            "skm_server_get_stats": (st, [P, ctypes.POINTER(skm_server_stats)]),
            "skm_server_destroy": (st, [P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


class SkmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(ctx, status: int):
    if status != SKM_OK:
        msg = load().skm_last_error(ctx) if ctx else b""
        raise SkmError(status, (msg or b"").decode(errors="replace"))


# ------------------------------------------------------------------ marshalling
def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x):
    if x is None:
        return None
    if _is_torch(x):
        return x.data_ptr()
    return x.ctypes.data


def make_csr(docs, n_terms: int | None = None):
    """skm_csr from a ``synth.Csr`` (host numpy) or a tuple of torch CUDA tensors
    (row_ptr int64, col_idx int32, values float32) with ``n_terms``. Returns (struct,
    keep-alive tuple, on_device)."""
    if isinstance(docs, tuple):
        rp, ci, va = docs
        on_dev = int(rp.is_cuda)
        d = int(n_terms)
        n = int(rp.shape[0] - 1)
        e = int(ci.shape[0])
        keep = (rp, ci, va)
    else:
        rp = np.ascontiguousarray(docs.row_ptr, dtype=np.int64)
        ci = np.ascontiguousarray(docs.col_idx, dtype=np.int32)
        va = np.ascontiguousarray(docs.values, dtype=np.float32)
        on_dev = 0
        d = int(docs.n_terms if n_terms is None else n_terms)
        n = int(rp.shape[0] - 1)
        e = int(ci.shape[0])
        keep = (rp, ci, va)
    c = skm_csr(n, d, e, _ptr(keep[0]), _ptr(keep[1]), _ptr(keep[2]), on_dev)
    return c, keep, on_dev


# ------------------------------------------------------------------ C entry points
def skm_config_default(k: int) -> skm_config:
    cfg = skm_config()
    load().skm_config_default(ctypes.byref(cfg), int(k))
    return cfg


def skm_create(cfg: skm_config):
    ctx = ctypes.c_void_p()
    st = load().skm_create(ctypes.byref(cfg), ctypes.byref(ctx))
    if st != SKM_OK:
        raise SkmError(st, "skm_create failed (invalid config, no device, or out of memory)")
    return ctx


def skm_destroy(ctx) -> None:
    if ctx:
        load().skm_destroy(ctx)


def skm_last_error(ctx) -> str:
    return (load().skm_last_error(ctx) or b"").decode(errors="replace")


def skm_fit(ctx, csr: skm_csr, init_ids, assign_out, objective_out=None, iters_out=None) -> int:
    it = ctypes.c_int32(0)
    _check(ctx, load().skm_fit(ctx, ctypes.byref(csr), _ptr(init_ids), _ptr(assign_out),
                               _ptr(objective_out), ctypes.byref(it)))
    if iters_out is not None:
        iters_out[0] = it.value
    return it.value


def skm_init_kmeanspp(ctx, csr: skm_csr, uniforms, ids_out) -> None:
    _check(ctx, load().skm_init_kmeanspp(ctx, ctypes.byref(csr), _ptr(uniforms), _ptr(ids_out)))


def skm_index_candidates(ctx, csr: skm_csr, level: int, bits) -> None:
    _check(ctx, load().skm_index_candidates(ctx, ctypes.byref(csr), int(level), _ptr(bits)))


def skm_assign(ctx, csr: skm_csr, assign_out, score_out=None) -> None:
    _check(ctx, load().skm_assign(ctx, ctypes.byref(csr), _ptr(assign_out), _ptr(score_out)))


def skm_update(ctx, csr: skm_csr, assign) -> int:
    n = ctypes.c_int32(0)
    _check(ctx, load().skm_update(ctx, ctypes.byref(csr), _ptr(assign), ctypes.byref(n)))
    return n.value


def skm_set_centroids(ctx, n_terms: int, centroids, on_device: int) -> None:
    _check(ctx, load().skm_set_centroids(ctx, int(n_terms), _ptr(centroids), int(on_device)))


def skm_get_centroids(ctx, out, on_device: int) -> None:
    _check(ctx, load().skm_get_centroids(ctx, _ptr(out), int(on_device)))


def skm_assign_fixed_scratch(csr: skm_csr, k: int, centroids, ld: int, assign_out, score_out=None,
                             stream: int | None = None) -> None:
    """FP32 assignment without any device allocation (see include/skm.h): every buffer is the
    caller's, the scratch is a fixed array inside the library. Device tensors only."""
    st = load().skm_assign_fixed_scratch(ctypes.byref(csr), int(k), _ptr(centroids), int(ld),
                                         _ptr(assign_out), _ptr(score_out), stream or None)
    if st != SKM_OK:
        raise SkmError(st, "skm_assign_fixed_scratch failed")


def skm_fit_batched(cfg: skm_batch_config, items, stats: skm_batch_stats) -> None:
    arr = (skm_batch_item * len(items))(*items)
    st = load().skm_fit_batched(ctypes.byref(cfg), arr, len(items), ctypes.byref(stats))
    if st != SKM_OK:
        raise SkmError(st, stats.message.decode(errors="replace"))


def fit_batched(instances, max_iter: int, rescore: bool = True, tau: float = 0.0, use_graph: bool = True,
                tune_cache: str | None = None, device: int = 0, stream: int | None = None,
                allocator: str = "torch"):
    """Batched form: instances = [(docs, k, init_ids), ...] with docs a ``synth.Csr`` (host) or a
    (row_ptr, col_idx, values, n_terms) tuple of device tensors. Returns
    ([(assign, objective[max_iter]), ...], stats dict)."""
    cfg = skm_batch_config()
    cfg.max_iter = int(max_iter)
    cfg.rescore = int(bool(rescore))
    cfg.rescore_tau = float(tau)
    cfg.device = int(device)
    cfg.use_graph = int(bool(use_graph))
    cfg.tune_cache = tune_cache.encode() if tune_cache else None
    alloc = None
    if allocator == "torch":
        import torch
        if stream is None:
            stream = torch.cuda.current_stream(device).cuda_stream
        alloc = _TorchAllocator(int(device), int(stream or 0))
        cfg.alloc = alloc.alloc_cb
        cfg.free = alloc.free_cb
    cfg.stream = stream or None
    keep, items, outs = [], [], []
    for docs, k, ids in instances:
        if isinstance(docs, tuple) and len(docs) == 4:
            csr, kp, on_dev = make_csr(docs[:3], docs[3])
        else:
            csr, kp, on_dev = make_csr(docs)
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        if on_dev:
            import torch
            a = torch.empty(csr.n_docs, dtype=torch.int32, device=kp[0].device)
        else:
            a = np.empty(csr.n_docs, np.int32)
        obj = np.zeros(max_iter, np.float64)
        keep.append((kp, ids, a, obj))
        items.append(skm_batch_item(csr, int(k), _ptr(ids), _ptr(a), _ptr(obj)))
        outs.append((a, obj))
    stats = skm_batch_stats()
    skm_fit_batched(cfg, items, stats)
    return outs, stats.as_dict()


def skm_get_stats(ctx) -> skm_stats:
    s = skm_stats()
    _check(ctx, load().skm_get_stats(ctx, ctypes.byref(s)))
    return s


# ------------------------------------------------------------------ owner class
class _TorchAllocator:
    """Device memory from PyTorch's caching allocator, handed to the library."""

    def __init__(self, device: int, stream_ptr: int):
        import torch
        self.torch = torch
        self.device = device
        self.stream = stream_ptr
        self.alloc_cb = ALLOC_FN(self._alloc)
        self.free_cb = FREE_FN(self._free)

    def _alloc(self, nbytes, user):
        try:
            return self.torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream or None)
        except Exception:      # out of memory: the library reports SKM_ERR_OOM
            return None

    def _free(self, ptr, nbytes, user):
        self.torch.cuda.caching_allocator_delete(int(ptr))


@dataclass
class FitResult:
    assign: np.ndarray
    objective: np.ndarray
    iters: int
    stats: dict


class SphericalKMeans:
    """One libskm context: exact spherical k-means on one GPU.

    precision: "fp32" or "bf16" (scored centroid copy); prune: "none", "ncc" (Sec. 3.1
    skip) or "ncc_index" (plus the threshold index of Sec. 3.2, with the minimum dot
    products index_lambdas, used in steps after more than index_min_changed centroids
    changed; -1 = every step; fits use the index only with index_max_cands > 0, and
    documents with more candidates than that are scored densely); rescore: FP64 rescoring of near ties; tau: margin threshold;
    sparse_div: centroid rows with at most k / sparse_div nonzeros are scored from their
    nonzero lists (0 = off; results are identical either way). head_terms: BF16 scoring of
    the collection's most frequent terms on the tensor cores (0 = automatic, -1 = off, > 0 =
    that many; assignments are exact either way).
    """

    def __init__(self, k: int, precision: str = "fp32", prune: str = "none", max_iter: int = 20,
                 shift_tol: float = -1.0, rescore: bool = True, tau: float = 0.0, device: int = 0,
                 stream: int | None = None, mem_budget: int = 0, timing: bool = False,
                 allocator: str = "torch", sparse_div: int = 0, index_lambdas=None,
                 index_min_changed: int | None = None, index_max_cands: int = 0, head_terms: int = 0):
        self.lib = load()
        cfg = skm_config_default(k)
        cfg.precision = {"fp32": SKM_FP32, "bf16": SKM_BF16}[precision]
        cfg.prune = PRUNE_MODES[prune]
        if index_lambdas is not None:
            lam = [float(x) for x in index_lambdas]
            if not 1 <= len(lam) <= 4:
                raise ValueError("1 to 4 index thresholds")
            cfg.index_levels = len(lam)
            for q, v in enumerate(lam):
                cfg.index_lambda[q] = v
        if index_min_changed is not None:
            cfg.index_min_changed = int(index_min_changed)
        cfg.index_max_cands = int(index_max_cands)
        cfg.max_iter = int(max_iter)
        cfg.shift_tol = float(shift_tol)
        cfg.rescore = int(bool(rescore))
        cfg.rescore_tau = float(tau)
        cfg.mem_budget = int(mem_budget)
        cfg.device = int(device)
        cfg.timing = int(bool(timing))
        cfg.sparse_div = int(sparse_div)
        cfg.head_terms = int(head_terms)
        if stream is None and allocator == "torch":
            import torch
            stream = torch.cuda.current_stream(device).cuda_stream
        cfg.stream = stream or None
        self._alloc = None
        if allocator == "torch":
            self._alloc = _TorchAllocator(int(device), int(stream or 0))
            cfg.alloc = self._alloc.alloc_cb
            cfg.free = self._alloc.free_cb
        self.cfg = cfg
        self.k = int(k)
        self.max_iter = int(max_iter)
        self.ctx = skm_create(cfg)

    def close(self):
        if getattr(self, "ctx", None):
            skm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # --------------------------------------------------------------- calls
    def fit(self, docs, init_ids, n_terms: int | None = None, assign_out=None) -> FitResult:
        csr, keep, on_dev = make_csr(docs, n_terms)
        ids = np.ascontiguousarray(init_ids, dtype=np.int32)
        if assign_out is None:
            if on_dev:
                import torch
                assign_out = torch.empty(csr.n_docs, dtype=torch.int32, device=keep[0].device)
            else:
                assign_out = np.empty(csr.n_docs, np.int32)
        obj = np.zeros(self.max_iter, np.float64)
        it = skm_fit(self.ctx, csr, ids, assign_out, obj)
        return FitResult(assign_out, obj[:it].copy(), it, skm_get_stats(self.ctx).as_dict())

    def init_kmeanspp(self, docs, uniforms, n_terms: int | None = None) -> np.ndarray:
        """k-means++ seeds (k document ids) drawn with the given k uniforms in [0, 1)."""
        csr, keep, on_dev = make_csr(docs, n_terms)
        u = np.ascontiguousarray(uniforms, dtype=np.float64)
        if u.shape[0] < self.k:
            raise ValueError("need k uniforms")
        if on_dev:
            import torch
            ids = torch.empty(self.k, dtype=torch.int32, device=keep[0].device)
            skm_init_kmeanspp(self.ctx, csr, u, ids)
            return ids.cpu().numpy()
        ids = np.empty(self.k, np.int32)
        skm_init_kmeanspp(self.ctx, csr, u, ids)
        return ids

    def assign(self, docs, n_terms: int | None = None, assign_out=None, score_out=None,
               want_scores: bool = True):
        csr, keep, on_dev = make_csr(docs, n_terms)
        if assign_out is None:
            if on_dev:
                import torch
                assign_out = torch.empty(csr.n_docs, dtype=torch.int32, device=keep[0].device)
                if want_scores and score_out is None:
                    score_out = torch.empty(csr.n_docs, dtype=torch.float32, device=keep[0].device)
            else:
                assign_out = np.empty(csr.n_docs, np.int32)
                if want_scores and score_out is None:
                    score_out = np.empty(csr.n_docs, np.float32)
        skm_assign(self.ctx, csr, assign_out, score_out)
        return assign_out, score_out

    def index_candidates(self, docs, level: int, n_terms: int | None = None) -> np.ndarray:
        """Candidate sets of the threshold index at index_lambdas[level] for the resident
        centroids: a bool matrix [n_docs, k] (Sec. 3.2 query, no baseline)."""
        csr, keep, on_dev = make_csr(docs, n_terms)
        W = (self.k + 31) // 32
        bits = np.zeros((csr.n_docs, W), np.uint32)
        skm_index_candidates(self.ctx, csr, level, bits)
        return np.unpackbits(bits.view(np.uint8), axis=1, bitorder="little")[:, :self.k].astype(bool)

    def update(self, docs, assign, n_terms: int | None = None) -> int:
        csr, keep, on_dev = make_csr(docs, n_terms)
        a = assign if on_dev else np.ascontiguousarray(assign, dtype=np.int32)
        return skm_update(self.ctx, csr, a)

    def set_centroids(self, C) -> None:
        if _is_torch(C):
            C = C.contiguous()
            skm_set_centroids(self.ctx, C.shape[0], C, int(C.is_cuda))
        else:
            C = np.ascontiguousarray(C, dtype=np.float32)
            skm_set_centroids(self.ctx, C.shape[0], C, 0)

    def centroids(self) -> np.ndarray:
        d = self.lib.skm_n_terms(self.ctx)
        out = np.empty((d, self.k), np.float32)
        skm_get_centroids(self.ctx, out, 0)
        return out

    def stats(self) -> dict:
        return skm_get_stats(self.ctx).as_dict()

    def mem_used(self) -> int:
        return int(self.lib.skm_mem_used(self.ctx))


class Server:
    """Serving form (see include/skm.h): continuous batching of assignment requests on a
    resident context, clustering jobs beside it under a device-memory budget."""

    def __init__(self, resident: "SphericalKMeans", mem_budget: int, n_job_slots: int = 2,
                 max_batch_docs: int = 65536, max_batch_nnz: int = 65536 * 200, job_precision: str = "bf16",
                 job_prune: str = "ncc", tau: float = 1e-4, device: int = 0):
        self.lib = load()
        cfg = skm_server_config()
        cfg.device = int(device)
        cfg.mem_budget = int(mem_budget)
        cfg.n_job_slots = int(n_job_slots)
        cfg.max_batch_docs = int(max_batch_docs)
        cfg.max_batch_nnz = int(max_batch_nnz)
        cfg.job_precision = {"fp32": SKM_FP32, "bf16": SKM_BF16}[job_precision]
        cfg.job_prune = PRUNE_MODES[job_prune]
        cfg.rescore_tau = float(tau)
        self.resident = resident
        h = ctypes.c_void_p()
        st = self.lib.skm_server_create(ctypes.byref(cfg), resident.ctx, ctypes.byref(h))
        if st != SKM_OK:
            raise SkmError(st, "skm_server_create failed")
        self.h = h
        self._keep = {}

    def submit_assign(self, docs) -> int:
        csr, keep, on_dev = make_csr(docs)
        t = ctypes.c_uint64(0)
        st = self.lib.skm_server_submit_assign(self.h, ctypes.byref(csr), ctypes.byref(t))
        if st != SKM_OK:
            raise SkmError(st, "submit_assign rejected the request")
        self._keep[t.value] = keep
        return t.value

    def submit_fit(self, docs, k: int, init_ids, max_iter: int) -> int:
        csr, keep, on_dev = make_csr(docs)
        ids = np.ascontiguousarray(init_ids, dtype=np.int32)
        t = ctypes.c_uint64(0)
        st = self.lib.skm_server_submit_fit(self.h, ctypes.byref(csr), int(k), _ptr(ids), int(max_iter),
                                            ctypes.byref(t))
        if st != SKM_OK:
            raise SkmError(st, "submit_fit rejected the request")
        self._keep[t.value] = keep
        return t.value

    def wait(self, ticket: int, timeout_ms: float = -1.0, release: bool = True) -> dict | None:
        r = skm_server_result()
        st = self.lib.skm_server_wait(self.h, ctypes.c_uint64(ticket), float(timeout_ms), ctypes.byref(r))
        if st == SKM_ERR_TIMEOUT:
            return None
        if st != SKM_OK:
            raise SkmError(st, "skm_server_wait failed")
        n = int(r.n_docs)
        out = {"state": REQ_STATES.get(r.state, r.state), "status": int(r.status), "n_docs": n,
               "latency_ms": r.latency_ms, "queue_ms": r.queue_ms, "batch_docs": r.batch_docs,
               "iters": r.iters, "message": r.message.decode(errors="replace")}
        out["assign"] = np.ctypeslib.as_array(r.assign, shape=(n,)).copy() if r.assign else None
        out["score"] = np.ctypeslib.as_array(r.score, shape=(n,)).copy() if r.score else None
        out["objective"] = np.ctypeslib.as_array(r.objective, shape=(r.iters,)).copy() \
            if r.objective and r.iters > 0 else None
        if release:
            self.lib.skm_server_release(self.h, ctypes.c_uint64(ticket))
            self._keep.pop(ticket, None)
        return out

    def stats(self) -> dict:
        s = skm_server_stats()
        self.lib.skm_server_get_stats(self.h, ctypes.byref(s))
        return s.as_dict()

    def close(self):
        if getattr(self, "h", None):
            self.lib.skm_server_destroy(self.h)
            self.h = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
