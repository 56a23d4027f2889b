"""Seeded synthetic tf-idf corpora (input generation only).

The paper clusters tf-idf bag-of-words vectors of tweets and arXiv abstracts
(Section 4.1): each present term gets term frequency times the log of the inverse
document frequency, stop words are dropped and every vector is scaled to unit
length. Those collections are not available here, so this module draws seeded
stand-ins with lognormal document lengths and Zipf-distributed term ids. The exact
definition is in ``synth.c``.

This module holds no clustering arithmetic. Both the FP64 oracle and the CUDA path
take its output as input, and it is the only code they share.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB_PATH = os.path.join(_HERE, "libskmsynth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``synth.c`` into ``libskmsynth.so`` next to it (gcc, OpenMP)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-Wall",
                    "-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.synth_corpus_draw.restype = ctypes.c_void_p
            lib.synth_corpus_draw.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_double,
                                              ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                              ctypes.c_uint64]
            lib.synth_corpus_nnz.restype = ctypes.c_int64
            lib.synth_corpus_nnz.argtypes = [ctypes.c_void_p]
            lib.synth_corpus_fill.restype = ctypes.c_int
            lib.synth_corpus_fill.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_void_p]
            lib.synth_corpus_free.restype = None
            lib.synth_corpus_free.argtypes = [ctypes.c_void_p]
            lib.synth_init_ids.restype = ctypes.c_int
            lib.synth_init_ids.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64,
                                           ctypes.c_void_p]
            lib.synth_uniform.restype = None
            lib.synth_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64,
                                          ctypes.c_void_p]
            _lib = lib
    return _lib


@dataclass(frozen=True)
class Csr:
    """A document collection in CSR form: unit-length rows, ascending column ids."""
    row_ptr: np.ndarray   # int64 [N+1]
    col_idx: np.ndarray   # int32 [E]
    values: np.ndarray    # float32 [E]
    n_terms: int

    @property
    def n_docs(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.col_idx.shape[0])

    def rows(self, ids) -> "Csr":
        """The sub-collection of the given document ids, in the given order."""
        ids = np.asarray(ids, dtype=np.int64)
        lens = self.row_ptr[ids + 1] - self.row_ptr[ids]
        rp = np.zeros(len(ids) + 1, dtype=np.int64)
        np.cumsum(lens, out=rp[1:])
        take = np.concatenate([np.arange(self.row_ptr[i], self.row_ptr[i + 1]) for i in ids]) \
            if len(ids) else np.zeros(0, dtype=np.int64)
        return Csr(rp, self.col_idx[take].copy(), self.values[take].copy(), self.n_terms)

    def dense(self, dtype=np.float64) -> np.ndarray:
        """Dense N x d copy (small corpora only)."""
        out = np.zeros((self.n_docs, self.n_terms), dtype=dtype)
        for i in range(self.n_docs):
            a, b = self.row_ptr[i], self.row_ptr[i + 1]
            out[i, self.col_idx[a:b]] = self.values[a:b]
        return out


def make_corpus(n_docs: int, n_terms: int, nnz_mean: float, nnz_lo: int, nnz_hi: int,
                zipf_s: float, seed: int) -> Csr:
    """Draw a seeded tf-idf corpus (definition in ``synth.c``)."""
    lib = _load()
    h = lib.synth_corpus_draw(int(n_docs), int(n_terms), float(nnz_mean), int(nnz_lo),
                              int(nnz_hi), float(zipf_s), int(seed))
    if not h:
        raise ValueError("synth_corpus_draw: invalid arguments or out of memory")
    e = lib.synth_corpus_nnz(h)
    row_ptr = np.empty(n_docs + 1, dtype=np.int64)
    col = np.empty(e, dtype=np.int32)
    val = np.empty(e, dtype=np.float32)
    rc = lib.synth_corpus_fill(h, row_ptr.ctypes.data, col.ctypes.data, val.ctypes.data)
    if rc != 0:
        raise RuntimeError("synth_corpus_fill failed")
    return Csr(row_ptr, col, val, int(n_terms))


def init_ids(n_docs: int, k: int, seed: int) -> np.ndarray:
    """k distinct document ids from a seeded partial Fisher-Yates shuffle."""
    out = np.empty(k, dtype=np.int32)
    if _load().synth_init_ids(int(n_docs), int(k), int(seed), out.ctypes.data) != 0:
        raise ValueError("init_ids: need 1 <= k <= n_docs")
    return out


def uniform(seed: int, stream: int, n: int) -> np.ndarray:
    """n uniform doubles in (0,1) from the same counter-based generator."""
    out = np.empty(n, dtype=np.float64)
    _load().synth_uniform(int(seed), int(stream), int(n), out.ctypes.data)
    return out


def sample_ids(n_docs: int, n_sample: int, seed: int) -> np.ndarray:
    """A seeded sorted sample of distinct document ids (for bounded checks)."""
    n_sample = min(int(n_sample), int(n_docs))
    return np.sort(init_ids(n_docs, n_sample, seed)).astype(np.int64)
