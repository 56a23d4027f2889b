"""Sparse rows of the centroid matrix (inverted-index form of Sec. 3.2).

Rows with few nonzeros are scored from their nonzero lists in CSR order instead of being
gathered densely. Every product the lists skip is an exact zero, so scores, assignments,
objectives and centroids must be bit-identical to the dense pass, whatever the threshold:
sparse_div 1 makes every row sparse, 0 none. Sizes cover several slices with a ragged last
slice, both precisions and the pruned (moved-centroid) matrix of Sec. 3.1.
"""
import numpy as np
import pytest

import oracle
from paper_2108_00895_gb300 import synth, workloads

pytestmark = pytest.mark.gpu

MARGIN = 1e-5


@pytest.fixture(scope="module")
def skm():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2108_00895_gb300 import skm as mod
    mod.load()
    return mod


def _trained(docs, k, seed, iters=2):
    ids = synth.init_ids(docs.n_docs, k, seed)
    return oracle.fit(docs, k, ids, iters).C.astype(np.float32)


def _assign(skm, C, docs, precision, div, rescore=True):
    # sparse rows replace the dense rows of the plain scoring pass, which is what they are
    # compared with: the tensor-core head path (another rounding of the frequent terms) is off
    with skm.SphericalKMeans(C.shape[1], precision=precision, sparse_div=div, rescore=rescore,
                             head_terms=-1) as km:
        km.set_centroids(C)
        a, s = km.assign(docs)
        st = km.stats()
    return a, s, st


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("k", [300, 1500])
def test_assign_sparse_rows_bit_identical_to_dense(skm, precision, k):
    docs = synth.make_corpus(2500, 20000, 80, 5, 600, 1.05, 7100 + k)
    C = _trained(docs, k, 7200 + k)
    for rescore in (False, True):
        a0, s0, st0 = _assign(skm, C, docs, precision, 0, rescore)
        assert st0["sparse_rows"] == 0 and st0["fmas_exec"] == st0["fmas"]
        for div in (8, 2, 1):
            a, s, st = _assign(skm, C, docs, precision, div, rescore)
            np.testing.assert_array_equal(a, a0)
            np.testing.assert_array_equal(s.view(np.uint32), s0.view(np.uint32))
            assert st["sparse_rows"] > 0 and st["sparse_entries"] > 0
            assert 0 < st["fmas_exec"] < st["fmas"] == st0["fmas"]
    # and the sparse pass is still the exact argmax of the FP64 oracle
    a_or, s1, s2 = oracle.assign(docs, C)
    clear = (s1 - s2) >= MARGIN
    assert not np.any((a0 != a_or) & clear)


def test_sparse_row_counts_match_the_matrix(skm):
    """Rows stored sparsely are exactly those with at most k / sparse_div nonzeros; each
    row's list per 256-column FP32 slice is padded to whole 16-byte vectors (2 entries)."""
    k = 640
    docs = synth.make_corpus(3000, 12000, 60, 5, 400, 1.1, 7301)
    C = _trained(docs, k, 7302)
    per_slice = np.stack([(C[:, s:s + 256] != 0).sum(axis=1) for s in range(0, k, 256)], axis=1)
    stored = ((per_slice + 1) // 2 * 2).sum(axis=1)
    nz = per_slice.sum(axis=1)
    for div in (1, 4, 16):
        _, _, st = _assign(skm, C, docs, "fp32", div)
        rare = nz <= k // div
        assert st["sparse_rows"] == int(np.count_nonzero(rare & (nz > 0)))
        assert st["sparse_entries"] == int(stored[rare].sum())


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_fit_with_sparse_rows_bit_identical(skm, precision):
    """Whole NCC fits (full, pruned and refull passes, rebuilt index after every update)."""
    w = workloads.SMALL.scaled(n_docs=8000, n_terms=15000, k=700, nnz_mean=70.0)
    docs = w.corpus()
    ids = w.init_ids()
    runs = {}
    for div in (0, 8, 1):
        with skm.SphericalKMeans(w.k, precision=precision, prune="ncc", max_iter=12, sparse_div=div,
                                 head_terms=-1) as km:
            r = km.fit(docs, ids)
            runs[div] = (r, km.centroids())
    r0, C0 = runs[0]
    for div in (8, 1):
        r, C = runs[div]
        assert r.iters == r0.iters
        np.testing.assert_array_equal(r.assign, r0.assign)
        np.testing.assert_array_equal(r.objective, r0.objective)
        np.testing.assert_array_equal(C, C0)
        assert r.stats["sparse_rows"] > 0
        assert r.stats["fmas_exec"] < r.stats["fmas"] == r0.stats["fmas"]
    assert r0.stats["docs_pruned"] > 0


def test_documents_made_only_of_sparse_rows(skm):
    """Documents whose terms all have sparse rows: a planted block vocabulary where each
    block's terms appear in one cluster only, so every row holds a single nonzero."""
    rng = np.random.default_rng(7400)
    k, per, n_blocks, n = 96, 40, 96, 6000
    rows, cols, vals = [], [], []
    for i in range(n):
        b = i % n_blocks
        t = np.sort(rng.choice(per, size=6, replace=False)) + b * per
        v = rng.random(6) + 0.1
        rows.append(np.full(6, i)); cols.append(t); vals.append(v / np.linalg.norm(v))
    r = np.concatenate(rows); c = np.concatenate(cols).astype(np.int32); v = np.concatenate(vals).astype(np.float32)
    rp = np.zeros(n + 1, np.int64); np.cumsum(np.bincount(r, minlength=n), out=rp[1:])
    docs = synth.Csr(rp, c, v, per * n_blocks)
    ids = np.arange(k, dtype=np.int32)           # one seed document per block
    out = {}
    for div in (0, 8):
        with skm.SphericalKMeans(k, precision="bf16", prune="ncc", max_iter=5, sparse_div=div) as km:
            out[div] = km.fit(docs, ids)
    np.testing.assert_array_equal(out[8].assign, out[0].assign)
    np.testing.assert_array_equal(out[8].assign, np.arange(n) % n_blocks)
    assert out[8].stats["sparse_rows"] == np.unique(c).size     # every present term: one cluster
