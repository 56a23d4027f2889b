"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (the contract of the method):
  assignments   bit-exact, except documents whose oracle top-2 margin is below 1e-5;
  objective     1e-6 relative;
  centroids     1e-5 max-abs (the FP32 master copy).
Sizes span several scoring slices with ragged tails (k not a multiple of the slice
width), document batches not a multiple of the block size, and rows longer than one
32-entry staging chunk.
"""
import numpy as np
import pytest

import oracle
from paper_2108_00895_gb300 import synth, workloads

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


def _check_assign(docs, C32, a_gpu, label=""):
    a_or, s1, s2 = oracle.assign(docs, C32)
    clear = (s1 - s2) >= MARGIN
    bad = np.nonzero((a_gpu != a_or) & clear)[0]
    assert len(bad) == 0, f"{label}: {len(bad)} clear-margin mismatches, first {bad[:5]}"
    return clear


def _corpus(n, d, mean, lo, hi, s, seed):
    return synth.make_corpus(n, d, mean, lo, hi, s, seed)


def _trained_centroids(docs, k, seed, iters=3):
    """Realistic centroids: a few oracle Lloyd steps from seeded documents, as float32."""
    ids = synth.init_ids(docs.n_docs, k, seed)
    r = oracle.fit(docs, k, ids, iters)
    return r.C.astype(np.float32)


# ---------------------------------------------------------------- assignment step
@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("k", [1, 7, 300, 777])
def test_assign_matches_oracle(skm, precision, k):
    docs = _corpus(1203, 4000, 60, 5, 400, 1.1, 500 + k)
    C = _trained_centroids(docs, k, 900 + k)
    with skm.SphericalKMeans(k, precision=precision) as km:
        km.set_centroids(C)
        a, s = km.assign(docs)
        np.testing.assert_array_equal(km.centroids(), C)
    clear = _check_assign(docs, C, a, f"{precision} k={k}")
    assert clear.mean() > 0.5
    # reported score = similarity of the chosen centroid (FP64 where rescored)
    exact = np.array([oracle.scores(docs.rows([i]), C[:, [a[i]]])[0, 0] for i in range(0, docs.n_docs, 97)])
    tol = 1e-5 if precision == "fp32" else 3e-3
    np.testing.assert_allclose(s[::97], exact, rtol=0, atol=tol)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_bf16_worst_case_rounding_is_rescored(skm, precision):
    """BF16 keeps an 8-bit significand, so its unit roundoff is 2^-8: a value just above a
    midpoint above 0.5 rounds up by almost 2^-9, i.e. by 2^-8 of itself. Here centroid 0 has
    its first coordinate rounded up that far and centroid 1 its first coordinate rounded
    down that far; centroid 1 is exactly better by 1.6e-5, yet its BF16 score is lower by
    0.003125, which exceeds 2 * 2^-9 * s1 but not 2 * 2^-8 * s1. Only a bound with the
    correct unit roundoff sends the document to FP64 rescoring."""
    h = 2.0 ** -9
    C = np.array([[0.5 + h + 1e-6, 0.5 + h - 1e-6],
                  [0.5, 0.5 + 3e-5]], dtype=np.float32)          # d x k: terms x centroids
    docs = synth.Csr(np.array([0, 2], np.int64), np.array([0, 1], np.int32),
                     np.array([0.8, 0.6], np.float32), 2)
    a_or, s1, s2 = oracle.assign(docs, C)
    assert a_or[0] == 1 and s1[0] - s2[0] > 1e-5
    with skm.SphericalKMeans(2, precision=precision) as km:
        km.set_centroids(C)
        a, s = km.assign(docs)
    assert a[0] == 1
    assert abs(s[0] - s1[0]) < 1e-6       # the rescored (FP64) similarity of centroid 1


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_assign_without_rescoring_is_plain_argmax_within_error_bound(skm, precision):
    docs = _corpus(800, 3000, 40, 5, 300, 1.1, 77)
    C = _trained_centroids(docs, 64, 78)
    with skm.SphericalKMeans(64, precision=precision, rescore=False) as km:
        km.set_centroids(C)
        a, _ = km.assign(docs)
    a_or, s1, s2 = oracle.assign(docs, C)
    bound = 2.0 * (2.0 ** -8 if precision == "bf16" else 2e-4) * s1
    clear = (s1 - s2) > bound
    np.testing.assert_array_equal(a[clear], a_or[clear])


def test_assign_ties_go_to_lowest_index(skm):
    # duplicate centroids: every document ties between columns 2 and 5
    docs = _corpus(300, 500, 20, 3, 60, 1.1, 11)
    rng = np.random.default_rng(3)
    C = rng.random((500, 8)).astype(np.float32)
    C /= np.linalg.norm(C, axis=0, keepdims=True)
    C[:, 5] = C[:, 2]
    C[:, [0, 1, 3, 4, 6, 7]] *= 0.01
    for prec in ("fp32", "bf16"):
        with skm.SphericalKMeans(8, precision=prec) as km:
            km.set_centroids(C)
            a, _ = km.assign(docs)
        a_or, _, _ = oracle.assign(docs, C)
        np.testing.assert_array_equal(a, a_or)
        assert (a != 5).all()


@pytest.mark.parametrize("copies", [9, 70])
def test_assign_many_near_ties_collect_and_full_fp64(skm, copies):
    """More tied candidates than the top list holds: 9 copies go through the collect pass,
    70 copies exceed its capacity and go to FP64 scoring against all k."""
    docs = _corpus(400, 600, 20, 3, 60, 1.1, 14)
    rng = np.random.default_rng(15)
    k = copies + 20
    C = (rng.random((600, k)) * 0.05).astype(np.float32)
    strong = rng.random(600).astype(np.float32)
    for q in range(copies):
        C[:, 10 + q] = strong
    C /= np.linalg.norm(C, axis=0, keepdims=True)
    for prec in ("fp32", "bf16"):
        with skm.SphericalKMeans(k, precision=prec) as km:
            km.set_centroids(C)
            a, _ = km.assign(docs)
            st = km.stats()
        a_or, _, _ = oracle.assign(docs, C)
        np.testing.assert_array_equal(a, a_or)
        assert st["docs_rescored"] + st["docs_rescored_full"] > 0
        if copies > 64:
            assert st["docs_rescored_full"] > 0


def test_assign_documents_sharing_no_term_with_any_centroid(skm):
    """All scores zero: every exact score is zero and centroid 0 (lowest index) wins."""
    docs = _corpus(300, 800, 15, 3, 40, 1.1, 16)
    rng = np.random.default_rng(17)
    C = rng.random((800, 12)).astype(np.float32)
    used = np.unique(docs.col_idx[docs.row_ptr[5]:docs.row_ptr[6]])
    C[used, :] = 0.0                        # document 5 overlaps no centroid
    C /= np.linalg.norm(C, axis=0, keepdims=True)
    with skm.SphericalKMeans(12, precision="bf16") as km:
        km.set_centroids(C)
        a, s = km.assign(docs)
    a_or, s1, _ = oracle.assign(docs, C)
    assert s1[5] == 0.0 and a[5] == 0 and s[5] == 0.0
    _check_assign(docs, C, a)


def test_assign_device_buffers(skm):
    import torch
    docs = _corpus(500, 2000, 30, 5, 200, 1.1, 12)
    C = _trained_centroids(docs, 40, 13)
    dev = (torch.from_numpy(docs.row_ptr).cuda(), torch.from_numpy(docs.col_idx).cuda(),
           torch.from_numpy(docs.values).cuda())
    with skm.SphericalKMeans(40, precision="bf16") as km:
        km.set_centroids(torch.from_numpy(C).cuda())
        a, s = km.assign(dev, n_terms=docs.n_terms)
        a_host, _ = km.assign(docs)
    np.testing.assert_array_equal(a.cpu().numpy(), a_host)
    _check_assign(docs, C, a_host)


# ---------------------------------------------------------------- update step
@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_update_matches_oracle(skm, precision):
    docs = _corpus(1500, 3000, 50, 5, 300, 1.1, 21)
    k = 300
    rng = np.random.default_rng(21)
    a = rng.integers(0, k, docs.n_docs).astype(np.int32)
    a[a == 17] = 18                                   # empty cluster keeps its centroid
    C0 = rng.random((docs.n_terms, k)).astype(np.float32)
    with skm.SphericalKMeans(k, precision=precision) as km:
        km.set_centroids(C0)
        n_re = km.update(docs, a)
        C = km.centroids()
    ref = oracle.update(docs, a, C0.astype(np.float64))
    assert n_re == (ref.sizes > 0).sum()
    np.testing.assert_array_equal(C[:, 17], C0[:, 17])
    assert np.abs(C - ref.C).max() < CENT_ATOL
    assert np.abs(C - ref.C).max() < 1e-6         # FP64 sums, one FP32 rounding


# ---------------------------------------------------------------- Lloyd loop
def _fit_both(skm, w, docs, ids, precision, prune, max_iter, shift_tol=-1.0):
    with skm.SphericalKMeans(w.k, precision=precision, prune=prune, max_iter=max_iter,
                             shift_tol=shift_tol) as km:
        r = km.fit(docs, ids)
        C = km.centroids()
    return r, C


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_fit_small_workload_matches_oracle(skm, precision, small_corpus):
    w, docs, ids = small_corpus
    ref = oracle.fit(docs, w.k, ids, w.max_iter)
    r, C = _fit_both(skm, w, docs, ids, precision, "none", w.max_iter)
    assert r.iters == ref.iters
    np.testing.assert_array_equal(r.assign, ref.a)
    np.testing.assert_allclose(r.objective, ref.objective, rtol=OBJ_RTOL, atol=0)
    assert np.abs(C - ref.C).max() < CENT_ATOL


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_fit_pruned_equals_full_bit_for_bit(skm, precision):
    """Sec. 3.1 is exact: the non-changing-clusters skip gives the same trajectory."""
    w = workloads.SMALL.scaled(n_docs=6000, n_terms=8000, k=150)
    docs = w.corpus()
    ids = w.init_ids()
    full, Cf = _fit_both(skm, w, docs, ids, precision, "none", 25)
    pr, Cp = _fit_both(skm, w, docs, ids, precision, "ncc", 25)
    assert pr.iters == full.iters
    np.testing.assert_array_equal(pr.assign, full.assign)
    np.testing.assert_array_equal(pr.objective, full.objective)
    np.testing.assert_array_equal(Cp, Cf)
    assert pr.stats["docs_pruned"] > 0
    assert pr.stats["sims"] < full.stats["sims"]


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_fit_large_vocabulary_short_documents(skm, precision):
    """Short documents over a large vocabulary (the tweets shape of Sec. 4.1): the update
    clears only the nonzeros of recomputed columns (their members' or seed document's
    terms), and steps with more than half of the clusters moved are scored in full. The
    pruned fit must equal the full one and the oracle."""
    w = workloads.TWEETS.scaled(n_docs=4000, n_terms=60000, k=160, max_iter=25, shift_tol=-1.0)
    docs = w.corpus()
    ids = w.init_ids()
    ref = oracle.fit(docs, w.k, ids, w.max_iter)
    full, Cf = _fit_both(skm, w, docs, ids, precision, "none", w.max_iter)
    pr, Cp = _fit_both(skm, w, docs, ids, precision, "ncc", w.max_iter)
    assert pr.iters == full.iters == ref.iters
    np.testing.assert_array_equal(pr.assign, full.assign)
    np.testing.assert_array_equal(Cp, Cf)
    np.testing.assert_array_equal(pr.assign, ref.a)
    np.testing.assert_allclose(pr.objective, ref.objective, rtol=OBJ_RTOL, atol=0)
    assert np.abs(Cp - ref.C).max() < CENT_ATOL
    assert pr.stats["docs_pruned"] > 0


def test_fit_step_locked_against_oracle(skm):
    """Each step checked on its own: the oracle's update of the GPU assignment gives the GPU
    centroids, and the oracle's assignment with the GPU centroids gives the GPU assignment."""
    w = workloads.SMALL.scaled(n_docs=3000, n_terms=6000, k=60)
    docs = w.corpus()
    ids = w.init_ids()
    prev_C = oracle.init_centroids(docs, w.k, ids).astype(np.float32)
    prev_a = None
    for t in range(1, 7):
        r, C = _fit_both(skm, w, docs, ids, "bf16", "ncc", t)
        if r.iters < t:
            break
        _check_assign(docs, prev_C, r.assign, f"step {t}")
        ref = oracle.update(docs, r.assign, prev_C.astype(np.float64), prev_a)
        assert np.abs(C - ref.C).max() < CENT_ATOL
        obj = oracle.objective(docs, prev_C, r.assign)
        assert abs(r.objective[-1] - obj) <= OBJ_RTOL * abs(obj)
        prev_C, prev_a = C, r.assign


def test_fit_objective_never_decreases(skm):
    w = workloads.SMALL.scaled(n_docs=4000, n_terms=6000, k=80)
    r, _ = _fit_both(skm, w, w.corpus(), w.init_ids(), "bf16", "ncc", 30)
    d = np.diff(r.objective)
    assert (d >= -1e-9 * np.abs(r.objective[1:])).all()


def test_fit_shift_stop_rule_matches_oracle(skm):
    docs, ids = _corpus(2500, 4000, 40, 5, 300, 1.1, 31), None
    ids = synth.init_ids(docs.n_docs, 50, 32)
    ref = oracle.fit(docs, 50, ids, 40, shift_tol=1e-4)
    with skm.SphericalKMeans(50, precision="fp32", prune="ncc", max_iter=40, shift_tol=1e-4) as km:
        r = km.fit(docs, ids)
    assert r.iters == ref.iters
    np.testing.assert_array_equal(r.assign, ref.a)


# ---------------------------------------------------------------- special cases
def test_k1_and_k_equals_n(skm):
    docs = _corpus(64, 2000, 20, 3, 60, 1.1, 41)
    with skm.SphericalKMeans(1, max_iter=3) as km:
        r = km.fit(docs, np.array([5]))
        assert (r.assign == 0).all()
        m = docs.dense().sum(axis=0)
        np.testing.assert_allclose(km.centroids()[:, 0], m / np.linalg.norm(m), atol=1e-6)
    with skm.SphericalKMeans(64, max_iter=3) as km:
        r = km.fit(docs, np.arange(64))
        np.testing.assert_array_equal(r.assign, np.arange(64))
        assert r.iters == 2


def test_single_term_documents_and_planted_blocks(skm):
    rng = np.random.default_rng(51)
    k, per, width = 6, 40, 10
    rp, cols, vals = [0], [], []
    for b in range(k):
        for q in range(per):
            n = 1 if q % 5 == 0 else 7
            c = np.sort(rng.choice(width, n, replace=False)) + b * width
            v = rng.random(n).astype(np.float64) + 0.1
            v /= np.linalg.norm(v)
            cols += c.tolist()
            vals += v.tolist()
            rp.append(len(cols))
    docs = synth.Csr(np.array(rp, np.int64), np.array(cols, np.int32), np.array(vals, np.float32), k * width)
    init = np.array([b * per + 1 for b in range(k)])
    ref = oracle.fit(docs, k, init, 10)
    with skm.SphericalKMeans(k, prune="ncc", max_iter=10) as km:
        r = km.fit(docs, init)
    np.testing.assert_array_equal(r.assign, ref.a)
    np.testing.assert_array_equal(r.assign, np.repeat(np.arange(k), per))


# ---------------------------------------------------------------- errors
def test_invalid_inputs_are_rejected(skm):
    docs = _corpus(100, 500, 10, 3, 30, 1.1, 61)
    with skm.SphericalKMeans(5) as km:
        with pytest.raises(skm.SkmError) as e:
            km.assign(docs)                                    # no centroids yet
        assert e.value.status == skm.SKM_ERR_STATE
        with pytest.raises(skm.SkmError) as e:
            km.fit(docs, np.array([1, 1, 2, 3, 4]))            # duplicate initial ids
        assert e.value.status == skm.SKM_ERR_INVALID
        bad = synth.Csr(docs.row_ptr, docs.col_idx.copy(), docs.values.copy(), docs.n_terms)
        bad.values[3] = -bad.values[3]
        with pytest.raises(skm.SkmError) as e:
            km.fit(bad, np.arange(5))
        assert e.value.status == skm.SKM_ERR_INVALID and "negative" in str(e.value)
        bad = synth.Csr(docs.row_ptr, docs.col_idx.copy(), docs.values.copy(), docs.n_terms)
        bad.col_idx[0], bad.col_idx[1] = bad.col_idx[1], bad.col_idx[0]
        with pytest.raises(skm.SkmError) as e:
            km.fit(bad, np.arange(5))
        assert "increasing" in str(e.value)
        bad = synth.Csr(docs.row_ptr, docs.col_idx.copy(), docs.values * 1.01, docs.n_terms)
        with pytest.raises(skm.SkmError) as e:
            km.fit(bad, np.arange(5))
        assert "norm" in str(e.value)
        bad = synth.Csr(docs.row_ptr.copy(), docs.col_idx, docs.values, docs.n_terms)
        bad.row_ptr[5] = docs.nnz + 100          # offsets past the arrays are flagged, not read
        with pytest.raises(skm.SkmError) as e:
            km.fit(bad, np.arange(5))
        assert e.value.status == skm.SKM_ERR_INVALID and "offsets" in str(e.value)
        # the context is still usable after rejected calls
        r = km.fit(docs, np.arange(5))
        assert r.iters >= 1


def test_memory_budget_is_enforced(skm):
    docs = _corpus(2000, 5000, 60, 5, 400, 1.1, 71)
    with skm.SphericalKMeans(20, mem_budget=1 << 20) as km:
        with pytest.raises(skm.SkmError) as e:
            km.fit(docs, np.arange(20))
        assert e.value.status == skm.SKM_ERR_BUDGET


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_fit_with_very_frequent_terms_matches_oracle(skm, precision):
    """Terms with more than 32,768 postings are summed in chunks by many blocks (the update's
    split path); two terms here exceed that, 22 more take the one-block heavy path. The fit
    must equal the oracle's."""
    docs = synth.make_corpus(90000, 20000, 10, 2, 60, 1.05, 4242)
    df = np.bincount(docs.col_idx, minlength=docs.n_terms)
    assert (df > 32768).sum() >= 2
    k = 60
    ids = synth.init_ids(docs.n_docs, k, 4243)
    ref = oracle.fit(docs, k, ids, 12)
    with skm.SphericalKMeans(k, precision=precision, prune="ncc", max_iter=12) as km:
        r = km.fit(docs, ids)
        C = km.centroids()
    assert r.iters == ref.iters
    np.testing.assert_array_equal(r.assign, ref.a)
    np.testing.assert_allclose(r.objective, ref.objective, rtol=OBJ_RTOL, atol=0)
    assert np.abs(C - ref.C).max() < CENT_ATOL
