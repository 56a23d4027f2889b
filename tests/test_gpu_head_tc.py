"""The BF16 scoring pass with the collection's most frequent terms on the tensor cores.

The head terms' products run as a dense FP16 matrix product (tcgen05, TMEM accumulators) and
the other nonzeros on the gather path; the decision is exact either way. Checks, through the
C ABI, against the FP64 oracle and against the same context with the head path off:
  assignments   equal to the plain BF16 pass everywhere (both are the exact argmax after FP64
                rescoring), and to the oracle wherever its top-2 margin is at least 1e-5;
  scores        within the scoring pass's bound beta s + alpha of the oracle's;
  fits          the pruned fit equals the full fit bit for bit with the head path on, and the
                fit equals the oracle's;
on ragged sizes: document counts that are not a multiple of the 128-document tile, column
counts that are not a multiple of the 512-column slice, head sizes from 64 to 2048, and
documents whose nonzeros are all in the head or none are.
"""
import numpy as np
import pytest

import oracle
from paper_2108_00895_gb300 import synth

pytestmark = pytest.mark.gpu

MARGIN = 1e-5
OBJ_RTOL = 1e-6
CENT_ATOL = 1e-5


@pytest.fixture(scope="module")
def skm():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2108_00895_gb300 import skm as mod
    mod.load()
    return mod


def _beta_bf16(docs):
    """The BF16 scoring pass's relative bound per document: 2^-8 + gamma_n (1 + 2^-8), and the
    head path's absolute term 2^-33 sqrt(n) + 2^-24."""
    n = np.diff(docs.row_ptr).astype(np.float64)
    nu = n * 2.0 ** -24
    uc = 2.0 ** -8
    return uc + nu / (1 - nu) * (1 + uc), np.sqrt(n) * 2.0 ** -33 + 2.0 ** -24


def _assign(skm, docs, C, k, head, **kw):
    with skm.SphericalKMeans(k, precision="bf16", head_terms=head, **kw) as km:
        km.set_centroids(C)
        a, s = km.assign(docs)
        st = km.stats()
    return a, s, st


@pytest.mark.parametrize("n,d,k,head", [(1003, 3000, 300, 64), (2051, 6000, 777, 0), (1500, 5000, 1100, 256),
                                        (1640, 9000, 1537, 2048), (600, 2500, 513, 128)])
def test_assign_with_head_matches_oracle_and_plain_pass(skm, n, d, k, head):
    docs = synth.make_corpus(n, d, 60, 5, 400, 1.1, 700 + k)
    k = min(k, n)
    C = oracle.fit(docs, k, synth.init_ids(n, k, 800 + k), 2).C.astype(np.float32)
    a_p, s_p, st_p = _assign(skm, docs, C, k, -1)
    a_t, s_t, st_t = _assign(skm, docs, C, k, head)
    assert st_p["head_terms"] == 0
    assert st_t["head_terms"] >= 64 and st_t["head_terms"] % 64 == 0
    if head > 0:
        assert st_t["head_terms"] == min(head, d // 64 * 64)
    assert 0 < st_t["nnz_head"] < docs.nnz
    np.testing.assert_array_equal(a_t, a_p)
    a_or, s1, s2 = oracle.assign(docs, C)
    clear = (s1 - s2) >= MARGIN
    assert clear.mean() > 0.9
    np.testing.assert_array_equal(a_t[clear], a_or[clear])
    beta, alpha = _beta_bf16(docs)
    err = np.abs(s_t.astype(np.float64) - s1)
    # the reported score is the scoring pass's (or, after rescoring, the FP64 one's)
    assert np.all(err <= beta * s1 + alpha + 1e-30)


def test_documents_all_head_or_no_head(skm):
    """Rows made only of head terms (empty tail) and rows with no head term (zero head sum)."""
    base = synth.make_corpus(1200, 4000, 60, 5, 400, 1.1, 901)
    k = 520
    C = oracle.fit(base, k, synth.init_ids(base.n_docs, k, 902), 2).C.astype(np.float32)
    rng = np.random.default_rng(903)
    rows = []
    for i in range(300):      # frequent terms only (ids below 40: all in the head)
        t = np.sort(rng.choice(40, size=int(rng.integers(1, 20)), replace=False))
        v = rng.random(len(t)) + 0.1
        rows.append((t, v / np.linalg.norm(v)))
    for i in range(300):      # rare terms only (ids above 3000)
        t = np.sort(rng.choice(np.arange(3000, 4000), size=int(rng.integers(1, 30)), replace=False))
        v = rng.random(len(t)) + 0.1
        rows.append((t, v / np.linalg.norm(v)))
    rp = np.zeros(len(rows) + 1, np.int64)
    rp[1:] = np.cumsum([len(t) for t, _ in rows])
    docs = synth.Csr(rp, np.concatenate([t for t, _ in rows]).astype(np.int32),
                     np.concatenate([v for _, v in rows]).astype(np.float32), 4000)
    with skm.SphericalKMeans(k, precision="bf16", head_terms=64) as km:
        km.set_centroids(C)
        km.assign(base)                     # chooses the head set from the base collection
        a, s = km.assign(docs)
        assert km.stats()["head_terms"] == 64
    a_p, s_p, _ = _assign(skm, docs, C, k, -1)
    np.testing.assert_array_equal(a, a_p)
    a_or, s1, s2 = oracle.assign(docs, C)
    clear = (s1 - s2) >= MARGIN
    np.testing.assert_array_equal(a[clear], a_or[clear])
    beta, alpha = _beta_bf16(docs)
    assert np.all(np.abs(s.astype(np.float64) - s1) <= beta * s1 + alpha + 1e-30)


@pytest.mark.parametrize("copies", [9, 70])
def test_near_ties_collect_and_full_fp64_with_head(skm, copies):
    """More tied candidates than the top list holds, scored with the head path: the collect
    pass recomputes the head-path scores, and the FP64 passes decide exactly."""
    docs = synth.make_corpus(600, 900, 20, 3, 60, 1.1, 904)
    rng = np.random.default_rng(905)
    k = 300 + copies
    C = (rng.random((900, k)) * (rng.random((900, k)) < 0.05)).astype(np.float32)
    # the copies point along the collection's mean, the best centroid of most documents
    strong = docs.dense().sum(axis=0).astype(np.float32)
    for q in range(copies):
        C[:, 10 + q] = strong
    C /= np.maximum(np.linalg.norm(C, axis=0, keepdims=True), 1e-30)
    a, _, st = _assign(skm, docs, C, k, 64)
    assert st["head_terms"] == 64
    a_or, _, _ = oracle.assign(docs, C)
    np.testing.assert_array_equal(a, a_or)
    assert st["docs_rescored"] + st["docs_rescored_full"] > 0
    if copies > 64:
        assert st["docs_rescored_full"] > 0


@pytest.mark.parametrize("head", [64, 0])
def test_fit_pruned_equals_full_with_head_and_matches_oracle(skm, head):
    """Sec. 3.1 stays exact with the head path: the pruned fit (compacted head matrix of the
    moved centroids) equals the full fit bit for bit, and both equal the oracle's fit."""
    docs = synth.make_corpus(5000, 9000, 60, 5, 400, 1.1, 906)
    k = 600
    ids = synth.init_ids(docs.n_docs, k, 907)
    out = {}
    for prune in ("none", "ncc"):
        with skm.SphericalKMeans(k, precision="bf16", prune=prune, max_iter=15, head_terms=head) as km:
            r = km.fit(docs, ids)
            out[prune] = (r, km.centroids())
    (rf, Cf), (rp, Cp) = out["none"], out["ncc"]
    assert rf.stats["head_terms"] > 0 and rp.stats["head_terms"] == rf.stats["head_terms"]
    assert rp.iters == rf.iters
    np.testing.assert_array_equal(rp.assign, rf.assign)
    np.testing.assert_array_equal(rp.objective, rf.objective)
    np.testing.assert_array_equal(Cp, Cf)
    assert rp.stats["docs_pruned"] > 0
    ref = oracle.fit(docs, k, ids, 15)
    assert rp.iters == ref.iters
    np.testing.assert_array_equal(rp.assign, ref.a)
    np.testing.assert_allclose(rp.objective, ref.objective, rtol=OBJ_RTOL, atol=0)
    assert np.abs(Cp - ref.C).max() < CENT_ATOL


def test_head_path_off_below_its_shapes(skm):
    """FP32 scoring, BF16 with k <= 256 (256-column slices) and a vocabulary under 64 terms
    keep the plain pass."""
    docs = synth.make_corpus(500, 3000, 40, 5, 200, 1.1, 908)
    small_vocab = synth.make_corpus(500, 60, 10, 3, 30, 1.1, 909)
    for prec, dd, k in (("fp32", docs, 300), ("bf16", docs, 200), ("bf16", small_vocab, 300)):
        k = min(k, dd.n_docs)
        C = oracle.fit(dd, k, synth.init_ids(dd.n_docs, k, 910), 1).C.astype(np.float32)
        with skm.SphericalKMeans(k, precision=prec) as km:
            km.set_centroids(C)
            km.assign(dd)
            assert km.stats()["head_terms"] == 0


@pytest.mark.parametrize("div", [8, 1])
def test_sparse_rows_on_the_tail_bit_identical(skm, div):
    """Sparse centroid rows (lists of a row's nonzeros) over the tail nonzeros: only products
    with exact zeros are skipped, so the scores equal those of the dense rows bit for bit, on
    the assignment step and over a whole NCC fit."""
    docs = synth.make_corpus(3000, 20000, 80, 5, 600, 1.05, 911)
    k = 700
    C = oracle.fit(docs, k, synth.init_ids(docs.n_docs, k, 912), 2).C.astype(np.float32)
    a0, s0, st0 = _assign(skm, docs, C, k, 128)
    a1, s1, st1 = _assign(skm, docs, C, k, 128, sparse_div=div)
    assert st1["head_terms"] == 128 and st1["sparse_rows"] > 0
    np.testing.assert_array_equal(a1, a0)
    np.testing.assert_array_equal(s1.view(np.uint32), s0.view(np.uint32))
    ids = synth.init_ids(docs.n_docs, k, 913)
    out = {}
    for sd in (0, div):
        with skm.SphericalKMeans(k, precision="bf16", prune="ncc", max_iter=8, head_terms=128, sparse_div=sd) as km:
            r = km.fit(docs, ids)
            out[sd] = (r, km.centroids())
    (r0, C0), (r1, C1) = out[0], out[div]
    assert r1.iters == r0.iters
    np.testing.assert_array_equal(r1.assign, r0.assign)
    np.testing.assert_array_equal(r1.objective, r0.objective)
    np.testing.assert_array_equal(C1, C0)
    assert r1.stats["fmas_exec"] < r1.stats["fmas"] == r0.stats["fmas"]
