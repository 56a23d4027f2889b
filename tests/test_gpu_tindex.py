"""Threshold index of Sec. 3.2 on the GPU (prune = "ncc_index") against the oracle.

The GPU index bounds each entry's minimum overlap count from below (value bins instead of
a sort) and clamps counts at 255, so its candidate sets must contain the oracle's exact ones
(the paper's construction), and with them every centroid with x . c >= lambda ||x||
(Lemma 3.1). The candidates are scored in FP64 and the rest cannot win, so a fit with the
index equals the fit without it bit for bit, and the oracle's NCC+INDEX fit.
"""
import numpy as np
import pytest

import oracle
from paper_2108_00895_gb300 import synth, workloads

pytestmark = pytest.mark.gpu

LAMBDAS = oracle.PAPER_LAMBDAS
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


SHAPES = {
    # short documents over a large vocabulary (tweets of Sec. 4.1)
    "tweets": workloads.TWEETS.scaled(n_docs=5000, n_terms=50000, k=150, max_iter=25, shift_tol=-1.0),
    # longer documents (abstracts of Sec. 4.1); k = 97 leaves a ragged bitmap word
    "abstracts": workloads.ABSTRACTS.scaled(n_docs=3000, n_terms=30000, k=97, max_iter=20, shift_tol=-1.0),
    # up to 400 nonzeros: overlap counts of documents over 255 nonzeros saturate
    "small": workloads.SMALL.scaled(n_docs=3000, n_terms=6000, k=70, max_iter=20),
}


def _trained(docs, k, ids, iters=3):
    return oracle.fit(docs, k, ids, iters).C.astype(np.float32)


def _as_matrix(lists, k):
    m = np.zeros((len(lists), k), bool)
    for i, c in enumerate(lists):
        m[i, c] = True
    return m


@pytest.mark.parametrize("shape", list(SHAPES))
def test_candidates_contain_oracle_candidates_and_every_high_similarity(skm, shape):
    w = SHAPES[shape]
    docs = w.corpus()
    C = _trained(docs, w.k, w.init_ids())
    _check_candidates(skm, w, docs, C)


def test_candidates_with_rows_on_both_fill_paths(skm):
    """k = 600: the frequent terms' rows hold more than 256 nonzeros (lists filled from the
    bitmap in two passes), the rare terms' rows fewer (staged fill); both give the oracle's
    candidates."""
    w = workloads.TWEETS.scaled(n_docs=6000, n_terms=20000, k=600, max_iter=15, shift_tol=-1.0)
    docs = w.corpus()
    C = _trained(docs, w.k, w.init_ids(), iters=2)
    row_nz = (C != 0).sum(axis=1)
    assert (row_nz > 256).sum() >= 10 and ((row_nz > 0) & (row_nz <= 256)).sum() >= 1000
    _check_candidates(skm, w, docs, C)


def _check_candidates(skm, w, docs, C):
    S = oracle.scores(docs, C)
    xn = np.sqrt(np.add.reduceat(docs.values.astype(np.float64) ** 2, docs.row_ptr[:-1]))
    overlap = oracle.scores(docs, (C != 0).astype(np.float32)) > 0   # shares a nonzero term
    short = np.diff(docs.row_ptr) <= 40     # longer documents are not indexed
    with skm.SphericalKMeans(w.k, prune="ncc_index") as km:
        km.set_centroids(C)
        for level, lam in enumerate(LAMBDAS):
            gpu = km.index_candidates(docs, level)
            ref = _as_matrix(oracle.index_candidates(docs, C.astype(np.float64), lam), w.k)
            assert not (ref & ~gpu).any(), f"lambda {lam}: oracle candidate missing"
            assert not ((S >= lam * xn[:, None]) & ~gpu).any(), f"lambda {lam}: high similarity missing"
            assert gpu[~short].all(), "documents over 40 nonzeros report every centroid"
            gpu, ref = gpu[short], ref[short]
            assert not (gpu & ~overlap[short]).any(), f"lambda {lam}: candidate without a shared term"
            # the value-bin bound stays close to the exact counts
            assert gpu.sum() <= 1.3 * ref.sum() + short.sum(), (lam, gpu.sum(), ref.sum())
            assert short.sum() > 0.3 * docs.n_docs


@pytest.mark.parametrize("precision,cap", [("fp32", 256), ("bf16", 256), ("fp32", 16)])
@pytest.mark.parametrize("shape", list(SHAPES))
def test_fit_with_index_equals_full_fit_bit_for_bit(skm, shape, precision, cap):
    """cap 256 indexes every short document whose baseline reaches a threshold (up to 256
    candidates); cap 16 sends those with more candidates to the dense passes."""
    w = SHAPES[shape]
    docs = w.corpus()
    ids = w.init_ids()
    runs = {}
    for prune in ("none", "ncc_index"):
        with skm.SphericalKMeans(w.k, precision=precision, prune=prune, max_iter=w.max_iter,
                                 index_min_changed=-1, index_max_cands=cap) as km:
            r = km.fit(docs, ids)
            runs[prune] = (r, km.centroids())
    (full, Cf), (ix, Ci) = runs["none"], runs["ncc_index"]
    assert ix.iters == full.iters
    np.testing.assert_array_equal(ix.assign, full.assign)
    np.testing.assert_array_equal(ix.objective, full.objective)
    np.testing.assert_array_equal(Ci, Cf)
    if cap == 256:
        assert ix.stats["index_docs"] > 0
        assert ix.stats["sims"] < full.stats["sims"]


@pytest.mark.parametrize("shape", ["tweets", "abstracts"])
def test_fit_with_index_matches_oracle_ncc_index(skm, shape):
    w = SHAPES[shape]
    docs = w.corpus()
    ids = w.init_ids()
    ref = oracle.fit(docs, w.k, ids, w.max_iter, mode="ncc_index", index_min_changed=-1)
    with skm.SphericalKMeans(w.k, prune="ncc_index", max_iter=w.max_iter, index_min_changed=-1,
                             index_max_cands=256) as km:
        r = km.fit(docs, ids)
        C = km.centroids()
    assert r.iters == ref.iters
    np.testing.assert_array_equal(r.assign, ref.a)
    np.testing.assert_allclose(r.objective, ref.objective, rtol=OBJ_RTOL, atol=0)
    assert np.abs(C - ref.C).max() < CENT_ATOL


def test_index_min_changed_gates_the_index(skm):
    """Sec. 4.3: the index serves a step only when more than index_min_changed centroids
    changed; a gate no step passes leaves the plain NCC loop."""
    w = SHAPES["tweets"]
    docs = w.corpus()
    ids = w.init_ids()
    out = {}
    for gate in (-1, 40, 10 ** 9):
        with skm.SphericalKMeans(w.k, prune="ncc_index", max_iter=w.max_iter, index_min_changed=gate,
                                 index_max_cands=256) as km:
            out[gate] = km.fit(docs, ids)
    assert out[10 ** 9].stats["index_docs"] == 0
    assert out[-1].stats["index_docs"] > out[40].stats["index_docs"] > 0
    for gate in (40, 10 ** 9):
        np.testing.assert_array_equal(out[gate].assign, out[-1].assign)
        np.testing.assert_array_equal(out[gate].objective, out[-1].objective)


def test_fits_without_a_cap_run_ncc_alone(skm):
    """Without a candidate cap a fit does not use the index (the dense NCC passes are the
    faster path on this GPU); its result is the NCC fit's, bit for bit."""
    w = SHAPES["tweets"]
    docs = w.corpus()
    ids = w.init_ids()
    out = {}
    for prune in ("ncc", "ncc_index"):
        with skm.SphericalKMeans(w.k, prune=prune, max_iter=w.max_iter, index_min_changed=-1) as km:
            out[prune] = km.fit(docs, ids)
    assert out["ncc_index"].stats["index_docs"] == 0
    np.testing.assert_array_equal(out["ncc_index"].assign, out["ncc"].assign)
    np.testing.assert_array_equal(out["ncc_index"].objective, out["ncc"].objective)


def test_custom_thresholds_and_documents_below_every_threshold(skm):
    """One high threshold: most baselines stay below it and those documents go to the
    dense passes; the result is still the full fit's."""
    w = SHAPES["abstracts"]
    docs = w.corpus()
    ids = w.init_ids()
    with skm.SphericalKMeans(w.k, prune="none", max_iter=w.max_iter) as km:
        full = km.fit(docs, ids)
    with skm.SphericalKMeans(w.k, prune="ncc_index", max_iter=w.max_iter, index_min_changed=-1,
                             index_lambdas=[0.95], index_max_cands=256) as km:
        r = km.fit(docs, ids)
    np.testing.assert_array_equal(r.assign, full.assign)
    np.testing.assert_array_equal(r.objective, full.objective)
    assert r.stats["docs_full"] + r.stats["docs_pruned"] > 0


def test_invalid_index_arguments(skm):
    docs = synth.make_corpus(200, 500, 12, 3, 30, 1.1, 41)
    with skm.SphericalKMeans(8, prune="ncc_index") as km:
        km.fit(docs, np.arange(8))
        with pytest.raises(skm.SkmError):
            km.index_candidates(docs, 4)
        with pytest.raises(skm.SkmError):
            km.index_candidates(docs, -1)
    for bad in ([0.5, 0.25], [0.0], [1.5], [0.1] * 5):
        with pytest.raises((skm.SkmError, ValueError)):
            skm.SphericalKMeans(8, prune="ncc_index", index_lambdas=bad)
    with pytest.raises(skm.SkmError):
        skm.SphericalKMeans(8, prune="ncc_index", index_max_cands=-1)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_index_kept_by_the_update_equals_a_fresh_build(skm, precision):
    """After a fit with the index, the bitmap and value bins that the update kept current give
    the same candidate sets as an index built from scratch on the final centroids."""
    w = SHAPES["tweets"]
    docs = w.corpus()
    ids = w.init_ids()
    with skm.SphericalKMeans(w.k, precision=precision, prune="ncc_index", max_iter=8, index_min_changed=-1,
                             index_max_cands=256) as km:
        r = km.fit(docs, ids)
        assert r.stats["index_docs"] > 0
        C = km.centroids()
        kept = [km.index_candidates(docs, level) for level in range(len(LAMBDAS))]
    with skm.SphericalKMeans(w.k, precision=precision, prune="ncc_index") as km:
        km.set_centroids(C)
        fresh = [km.index_candidates(docs, level) for level in range(len(LAMBDAS))]
    for level in range(len(LAMBDAS)):
        np.testing.assert_array_equal(kept[level], fresh[level])
