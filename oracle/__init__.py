"""FP64 CPU oracle for exact sparse spherical k-means (test infrastructure only).

This package checks the CUDA path and is never part of it. Only the test suite,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import it.
It shares no code with the CUDA library; the two meet only in the seeded inputs from
``paper_2108_00895_gb300.synth``.

Every function follows a passage of Knittel, Koch and Ertl, "Efficient Sparse
Spherical k-Means for Document Clustering" (DocEng 2021):

* ``assign``: the assignment step, Sec. 2 (argmax of the dot product of unit vectors).
* ``update``: the centroid update, Sec. 2 (normalised sum of the members).
* ``objective``: the spherical k-means objective sum_i x_i . c_{a_i}.
* ``fit``: the Lloyd loop of Sec. 2, with the non-changing-clusters skip (Sec. 3.1)
  and the dot product indexing structure (Sec. 3.2) as modes, and the stop rule of
  Sec. 4.1.
* ``min_overlaps``, ``index_candidates``: the threshold index of Sec. 3.2 (Lemma 3.1).
* ``kmeanspp``: k-means++ seeding, the initial assignment Sec. 2 names.

The arithmetic lives in ``skm_oracle.c`` (plain C, IEEE double, no FMA contraction).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "skm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MODE_PLAIN, MODE_NCC, MODE_NCC_INDEX, MODE_INDEX = 0, 1, 2, 3
MODES = {"plain": MODE_PLAIN, "ncc": MODE_NCC, "ncc_index": MODE_NCC_INDEX, "index": MODE_INDEX}
PAPER_LAMBDAS = (0.1, 0.25, 0.4, 0.6)   # Sec. 4.1: the set of minimum dot products


def build(force: bool = False) -> str:
    """Compile the oracle into ``liboracle.so`` (gcc, OpenMP, FP contraction off)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
                    "-shared", "-fPIC", "-Wall", "-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_P = ctypes.c_void_p
_I64, _I32, _D, _INT = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_int


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            sig = {
                "oracle_num_threads": (_INT, []),
                "oracle_set_threads": (None, [_INT]),
                "oracle_assign": (None, [_I64, _P, _P, _P, _I32, _I32, _P, _INT, _P, _P, _P]),
                "oracle_scores": (None, [_I64, _P, _P, _P, _I32, _P, _INT, _P]),
                "oracle_objective": (_D, [_I64, _P, _P, _P, _I32, _P, _INT, _P]),
                "oracle_update": (_I32, [_I64, _P, _P, _P, _I32, _I32, _P, _P, _P, _P, _P, _P]),
                "oracle_init_centroids": (None, [_P, _P, _P, _I32, _I32, _P, _P]),
                "oracle_centroids_subset": (None, [_I64, _P, _P, _P, _I32, _P, _I32, _P, _P]),
                "oracle_index_min_overlaps": (_INT, [_I32, _P, _D, _P, _P]),
                "oracle_index_candidates": (_I64, [_I64, _P, _P, _I32, _I32, _P, _D, _P, _P, _I64]),
                "oracle_fit": (_I32, [_I64, _P, _P, _P, _I32, _I32, _P, _I32, _D, _INT, _INT, _P,
                                      _I32, _P, _P, _P, _P, _P]),
                "oracle_kmeanspp": (_INT, [_I64, _P, _P, _P, _I32, _I32, _P, _P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data


def _csr_args(docs):
    rp = np.ascontiguousarray(docs.row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(docs.col_idx, dtype=np.int32)
    va = np.ascontiguousarray(docs.values, dtype=np.float32)
    return rp, ci, va


def _cent(C: np.ndarray):
    if C.dtype == np.float32:
        return np.ascontiguousarray(C), 1
    return np.ascontiguousarray(C, dtype=np.float64), 0


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def assign(docs, C: np.ndarray):
    """Sec. 2 assignment: (a, s1, s2) with a_i = argmax_j x_i . c_j (ties: lowest j),
    s1 the best and s2 the runner-up similarity. C is term-major d x k (float64 or
    float32; float32 entries are widened exactly to double)."""
    rp, ci, va = _csr_args(docs)
    Cc, f32 = _cent(C)
    n = docs.n_docs
    a = np.empty(n, np.int32)
    s1 = np.empty(n, np.float64)
    s2 = np.empty(n, np.float64)
    _load().oracle_assign(n, _ptr(rp), _ptr(ci), _ptr(va), Cc.shape[0], Cc.shape[1], _ptr(Cc), f32,
                          _ptr(a), _ptr(s1), _ptr(s2))
    return a, s1, s2


def scores(docs, C: np.ndarray) -> np.ndarray:
    """All similarities s_ij (N x k); small inputs only."""
    rp, ci, va = _csr_args(docs)
    Cc, f32 = _cent(C)
    out = np.empty((docs.n_docs, Cc.shape[1]), np.float64)
    _load().oracle_scores(docs.n_docs, _ptr(rp), _ptr(ci), _ptr(va), Cc.shape[1], _ptr(Cc), f32,
                          _ptr(out))
    return out


def objective(docs, C: np.ndarray, a: np.ndarray) -> float:
    """sum_i x_i . c_{a_i} in FP64, i ascending."""
    rp, ci, va = _csr_args(docs)
    Cc, f32 = _cent(C)
    aa = np.ascontiguousarray(a, dtype=np.int32)
    return float(_load().oracle_objective(docs.n_docs, _ptr(rp), _ptr(ci), _ptr(va), Cc.shape[1],
                                          _ptr(Cc), f32, _ptr(aa)))


@dataclass
class UpdateResult:
    C: np.ndarray          # d x k float64, new centroids
    changed: np.ndarray    # uint8[k], membership changed
    n_changed: int
    shift: float           # max_j ||c_j(new) - c_j(old)||^2
    sizes: np.ndarray      # int64[k]


def update(docs, a: np.ndarray, C_prev: np.ndarray, a_prev: np.ndarray | None = None) -> UpdateResult:
    """Sec. 2 centroid update: c_j = S_j / ||S_j|| (empty clusters keep C_prev)."""
    rp, ci, va = _csr_args(docs)
    C = np.array(C_prev, dtype=np.float64, order="C", copy=True)
    d, k = C.shape
    aa = np.ascontiguousarray(a, dtype=np.int32)
    ap = None if a_prev is None else np.ascontiguousarray(a_prev, dtype=np.int32)
    changed = np.empty(k, np.uint8)
    shift = np.zeros(1, np.float64)
    sizes = np.empty(k, np.int64)
    n = _load().oracle_update(docs.n_docs, _ptr(rp), _ptr(ci), _ptr(va), d, k, _ptr(aa),
                              None if ap is None else _ptr(ap), _ptr(C), _ptr(changed), _ptr(shift),
                              _ptr(sizes))
    if n < 0:
        raise MemoryError("oracle_update: allocation failed")
    return UpdateResult(C, changed, int(n), float(shift[0]), sizes)


def centroids_subset(docs, a: np.ndarray, clusters) -> np.ndarray:
    """Sec. 2 centroids of the listed clusters only: d x len(clusters) float64 (zero
    column for a cluster without members)."""
    rp, ci, va = _csr_args(docs)
    aa = np.ascontiguousarray(a, dtype=np.int32)
    sel = np.ascontiguousarray(clusters, dtype=np.int32)
    out = np.empty((docs.n_terms, len(sel)), np.float64)
    _load().oracle_centroids_subset(docs.n_docs, _ptr(rp), _ptr(ci), _ptr(va), docs.n_terms, _ptr(aa),
                                    len(sel), _ptr(sel), _ptr(out))
    return out


def init_centroids(docs, k: int, init_ids: np.ndarray) -> np.ndarray:
    """c_j = x_{init_j}, term-major d x k float64."""
    rp, ci, va = _csr_args(docs)
    ids = np.ascontiguousarray(init_ids, dtype=np.int32)
    C = np.empty((docs.n_terms, k), np.float64)
    _load().oracle_init_centroids(_ptr(rp), _ptr(ci), _ptr(va), docs.n_terms, k, _ptr(ids), _ptr(C))
    return C


def min_overlaps(values_desc: np.ndarray, lam: float):
    """Minimum overlap counts (Sec. 3.2 build step 3) by the linear two-pointer method
    of the footnote and by the direct method; returns (linear, naive, differ)."""
    v = np.ascontiguousarray(values_desc, dtype=np.float64)
    m = v.shape[0]
    lin = np.empty(m, np.int32)
    nai = np.empty(m, np.int32)
    bad = _load().oracle_index_min_overlaps(m, _ptr(v), float(lam), _ptr(lin), _ptr(nai))
    return lin, nai, bool(bad)


def index_candidates(docs, C: np.ndarray, lam: float):
    """Candidate centroids of every doc from the threshold index for one lambda
    (Sec. 3.2 query); returns a list of int32 arrays (ascending)."""
    rp, ci, _ = _csr_args(docs)
    Cc = np.ascontiguousarray(C, dtype=np.float64)
    d, k = Cc.shape
    cap = docs.n_docs * k
    ptr = np.empty(docs.n_docs + 1, np.int64)
    out = np.empty(max(cap, 1), np.int32)
    n = _load().oracle_index_candidates(docs.n_docs, _ptr(rp), _ptr(ci), d, k, _ptr(Cc), float(lam),
                                        _ptr(ptr), _ptr(out), cap)
    assert n <= cap
    return [out[ptr[i]:ptr[i + 1]].copy() for i in range(docs.n_docs)]


@dataclass
class FitResult:
    C: np.ndarray             # d x k float64
    a: np.ndarray             # int32[N]
    iters: int
    objective: np.ndarray     # per assignment step
    n_changed: np.ndarray     # docs whose assignment changed, per step
    sims: np.ndarray          # similarities computed, per step


def fit(docs, k: int, init_ids: np.ndarray, max_iter: int, shift_tol: float = -1.0,
        mode: str = "plain", lambdas=PAPER_LAMBDAS, index_min_changed: int = -1) -> FitResult:
    """Sec. 2 Lloyd loop from the centroids x_{init_j}; modes 'plain', 'ncc' (Sec. 3.1),
    'index' and 'ncc_index' (Sec. 3.2). Stops on unchanged assignments, on the shift
    test (Sec. 4.1; shift_tol < 0 disables it) or after max_iter assignment steps."""
    rp, ci, va = _csr_args(docs)
    d = docs.n_terms
    ids = np.ascontiguousarray(init_ids, dtype=np.int32)
    lam = np.ascontiguousarray(lambdas, dtype=np.float64)
    C = np.empty((d, k), np.float64)
    a = np.empty(docs.n_docs, np.int32)
    obj = np.zeros(max_iter, np.float64)
    nch = np.zeros(max_iter, np.int64)
    sims = np.zeros(max_iter, np.int64)
    it = _load().oracle_fit(docs.n_docs, _ptr(rp), _ptr(ci), _ptr(va), d, k, _ptr(ids), max_iter,
                            float(shift_tol), MODES[mode], len(lam), _ptr(lam), int(index_min_changed),
                            _ptr(C), _ptr(a), _ptr(obj), _ptr(nch), _ptr(sims))
    if it < 0:
        raise MemoryError("oracle_fit: allocation failed")
    return FitResult(C, a, int(it), obj[:it].copy(), nch[:it].copy(), sims[:it].copy())


def kmeanspp(docs, k: int, uniforms: np.ndarray) -> np.ndarray:
    """k-means++ seeds (Sec. 2's named initialisation; readings K1-K2 in skm_oracle.c):
    document ids drawn with probability proportional to 1 - max over seeds of x . seed,
    using the given uniforms in [0, 1)."""
    rp, ci, va = _csr_args(docs)
    u = np.ascontiguousarray(uniforms, dtype=np.float64)
    if u.shape[0] < k:
        raise ValueError("need k uniforms")
    ids = np.empty(k, np.int32)
    if _load().oracle_kmeanspp(docs.n_docs, _ptr(rp), _ptr(ci), _ptr(va), docs.n_terms, int(k), _ptr(u), _ptr(ids)) != 0:
        raise MemoryError("oracle_kmeanspp: allocation failed")
    return ids
