"""Pins for the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: numpy brute force
on dense copies, closed forms, hand-derived fixtures under tests/golden/, invariants
the paper states (exactness of the accelerations, Lemma 3.1) and special cases.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2108_00895_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _csr_from_lists(rows, d):
    rp = [0]
    cols, vals = [], []
    for c, v in rows:
        cols += c
        vals += v
        rp.append(len(cols))
    return synth.Csr(np.array(rp, np.int64), np.array(cols, np.int32), np.array(vals, np.float32), d)


def _tiny(seed, n=150, d=300, k=12, mean=20, lo=3, hi=80, s=1.1):
    docs = synth.make_corpus(n, d, mean, lo, hi, s, seed)
    return docs, synth.init_ids(n, k, seed + 7), k


# ---------------------------------------------------------------- Sec. 2 assignment
@pytest.mark.parametrize("seed", [11, 12, 13])
def test_assign_matches_dense_bruteforce(seed):
    docs, ids, k = _tiny(seed)
    rng = np.random.default_rng(seed)
    C = rng.random((docs.n_terms, k)) * (rng.random((docs.n_terms, k)) < 0.3)
    C /= np.linalg.norm(C, axis=0, keepdims=True)
    X = docs.dense()
    S = X @ C                                 # all similarities, independent summation
    a, s1, s2 = oracle.assign(docs, C)
    np.testing.assert_allclose(s1, S.max(axis=1), rtol=0, atol=1e-13)
    srt = np.sort(S, axis=1)
    np.testing.assert_allclose(s2, srt[:, -2], rtol=0, atol=1e-13)
    clear = (srt[:, -1] - srt[:, -2]) > 1e-12
    assert clear.sum() > 0.9 * len(clear)
    np.testing.assert_array_equal(a[clear], S.argmax(axis=1)[clear])
    # every similarity, one by one
    np.testing.assert_allclose(oracle.scores(docs, C), S, rtol=0, atol=1e-13)


def test_assign_ties_go_to_lowest_index():
    # two identical centroids and a zero-overlap document: ties everywhere
    docs = _csr_from_lists([([0], [1.0]), ([2], [1.0]), ([1], [1.0])], 3)
    C = np.zeros((3, 3))
    C[0, 1] = C[0, 2] = 1.0       # centroids 1 and 2 identical
    C[1, 0] = 1.0
    a, s1, s2 = oracle.assign(docs, C)
    assert list(a) == [1, 0, 0]   # doc 1 overlaps nothing: all zero -> index 0
    assert s1[0] == 1.0 and s2[0] == 1.0


def test_assign_float32_centroids_widen_exactly():
    docs, ids, k = _tiny(5)
    rng = np.random.default_rng(5)
    C32 = rng.random((docs.n_terms, k)).astype(np.float32)
    a1, s1, _ = oracle.assign(docs, C32)
    a2, s2, _ = oracle.assign(docs, C32.astype(np.float64))
    np.testing.assert_array_equal(a1, a2)
    np.testing.assert_array_equal(s1, s2)


# ---------------------------------------------------------------- Sec. 2 update
@pytest.mark.parametrize("seed", [21, 22])
def test_update_matches_closed_form(seed):
    docs, ids, k = _tiny(seed)
    rng = np.random.default_rng(seed)
    a = rng.integers(0, k, docs.n_docs).astype(np.int32)
    a[a == 3] = 4                              # make cluster 3 empty
    C_prev = rng.random((docs.n_terms, k))
    r = oracle.update(docs, a, C_prev)
    X = docs.dense()
    onehot = np.zeros((docs.n_docs, k))
    onehot[np.arange(docs.n_docs), a] = 1
    S = X.T @ onehot
    nrm = np.linalg.norm(S, axis=0)
    for j in range(k):
        if nrm[j] == 0:
            np.testing.assert_array_equal(r.C[:, j], C_prev[:, j])   # empty keeps previous
        else:
            np.testing.assert_allclose(r.C[:, j], S[:, j] / nrm[j], rtol=0, atol=1e-15)
            assert abs(np.linalg.norm(r.C[:, j]) - 1.0) < 1e-14
    assert r.sizes[3] == 0 and r.sizes.sum() == docs.n_docs
    shifts = ((r.C - C_prev) ** 2).sum(axis=0)
    assert abs(r.shift - shifts.max()) < 1e-12
    # no previous assignment: every cluster that received members changed
    np.testing.assert_array_equal(r.changed, (r.sizes > 0).astype(np.uint8))


def test_update_changed_flags_follow_membership():
    docs, ids, k = _tiny(31)
    rng = np.random.default_rng(31)
    a_prev = rng.integers(0, k, docs.n_docs).astype(np.int32)
    a = a_prev.copy()
    a[5] = (a_prev[5] + 1) % k                  # one document moves
    C0 = oracle.update(docs, a_prev, np.zeros((docs.n_terms, k))).C
    r = oracle.update(docs, a, C0, a_prev)
    expect = np.zeros(k, np.uint8)
    expect[[a_prev[5], a[5]]] = 1
    np.testing.assert_array_equal(r.changed, expect)
    # unchanged membership gives bit-identical centroids (the reading behind Sec. 3.1)
    same = expect == 0
    np.testing.assert_array_equal(r.C[:, same], C0[:, same])


# ---------------------------------------------------------------- hand fixtures
def test_hand_lloyd_example():
    g = json.load(open(os.path.join(GOLD, "hand_lloyd.json")))
    docs = _csr_from_lists(g["docs"], g["n_terms"])
    for mode in ("plain", "ncc", "index", "ncc_index"):
        r = oracle.fit(docs, g["k"], np.array(g["init_ids"]), 10, mode=mode)
        assert list(r.a) == g["assign"]
        assert r.iters == g["iters"]
        np.testing.assert_allclose(r.objective, g["objective"], rtol=0, atol=1e-7)
    C0 = oracle.init_centroids(docs, g["k"], np.array(g["init_ids"]))
    u = oracle.update(docs, np.array(g["assign"], np.int32), C0)
    np.testing.assert_allclose(u.C, g["centroids_after_update_1"], rtol=0, atol=1e-7)


def test_hand_min_overlap():
    g = json.load(open(os.path.join(GOLD, "hand_min_overlap.json")))
    for case in g["cases"]:
        lin, nai, differ = oracle.min_overlaps(np.array(case["values"]), g["lambda"])
        assert list(lin) == case["min_overlap"]
        assert list(nai) == case["min_overlap"]
        assert not differ


# ---------------------------------------------------------------- Sec. 3.2 index
@pytest.mark.parametrize("seed", [41, 42, 43])
def test_min_overlap_linear_equals_naive(seed):
    rng = np.random.default_rng(seed)
    for _ in range(200):
        m = int(rng.integers(1, 60))
        v = np.sort(rng.random(m) ** 3)[::-1]
        v /= np.linalg.norm(v) * rng.uniform(0.8, 1.2)
        for lam in (0.1, 0.25, 0.4, 0.6, 0.9):
            lin, nai, differ = oracle.min_overlaps(v, lam)
            assert not differ
            np.testing.assert_array_equal(lin, nai)


@pytest.mark.parametrize("lam", [0.1, 0.25, 0.4, 0.6])
def test_index_candidates_superset_of_bruteforce(lam):
    """Lemma 3.1 and the build guarantee: every centroid with x.c >= lambda is a candidate."""
    docs, ids, k = _tiny(51, n=200, d=250, k=16, mean=12)
    r = oracle.fit(docs, k, ids, 3)           # realistic, sparse-ish centroids
    S = docs.dense() @ r.C
    cands = oracle.index_candidates(docs, r.C, lam)
    total = 0
    for i in range(docs.n_docs):
        need = np.nonzero(S[i] >= lam)[0]
        assert set(need.tolist()) <= set(cands[i].tolist())
        total += len(cands[i])
    assert total < docs.n_docs * k             # the filter removes something


def test_lemma_3_1_property():
    """Lemma 3.1 on random sparse unit vectors: c.x >= lam implies sum_{t in nnz(x)} c_t^2 >= lam^2."""
    rng = np.random.default_rng(61)
    n = 40
    hits = 0
    for _ in range(4000):
        x = rng.random(n) * (rng.random(n) < 0.2)
        c = rng.random(n) * (rng.random(n) < 0.5)
        if not x.any() or not c.any():
            continue
        x /= np.linalg.norm(x)
        c /= np.linalg.norm(c)
        dot = float(c @ x)
        lam = rng.uniform(0.0, 1.0)
        if dot >= lam:
            hits += 1
            assert (c[x != 0] ** 2).sum() >= lam * lam - 1e-12
    assert hits > 100


# ---------------------------------------------------------------- loop invariants
@pytest.mark.parametrize("seed", [71, 72])
def test_objective_never_decreases(seed):
    docs, ids, k = _tiny(seed, n=400, d=600, k=15)
    r = oracle.fit(docs, k, ids, 30)
    assert r.iters >= 3
    diffs = np.diff(r.objective)
    assert (diffs >= -1e-12 * np.abs(r.objective[1:])).all()


@pytest.mark.parametrize("mode", ["ncc", "index", "ncc_index"])
def test_accelerated_modes_equal_plain(mode, small_corpus):
    """Sec. 3: both strategies are exact; assignments and objectives equal plain mode."""
    w, docs, ids = small_corpus
    ref = oracle.fit(docs, w.k, ids, w.max_iter, mode="plain")
    r = oracle.fit(docs, w.k, ids, w.max_iter, mode=mode, index_min_changed=-1)
    np.testing.assert_array_equal(r.a, ref.a)
    np.testing.assert_array_equal(r.objective, ref.objective)
    np.testing.assert_array_equal(r.n_changed, ref.n_changed)
    np.testing.assert_array_equal(r.C, ref.C)
    # Table 1 ordering: the non-changing-clusters skip never computes more similarities
    assert (r.sims <= ref.sims).all() or mode == "index"
    if mode != "index":
        assert r.sims.sum() < ref.sims.sum()


def test_accelerated_modes_equal_plain_with_stop_rule():
    docs, ids, k = _tiny(81, n=600, d=800, k=30, mean=25)
    ref = oracle.fit(docs, k, ids, 25, shift_tol=1e-4, mode="plain")
    for mode in ("ncc", "ncc_index"):
        r = oracle.fit(docs, k, ids, 25, shift_tol=1e-4, mode=mode, index_min_changed=-1)
        assert r.iters == ref.iters
        np.testing.assert_array_equal(r.a, ref.a)


# ---------------------------------------------------------------- special cases
def test_k1_gives_normalised_mean():
    docs, _, _ = _tiny(91)
    r = oracle.fit(docs, 1, np.array([3]), 5)
    assert (r.a == 0).all()
    m = docs.dense().sum(axis=0)
    np.testing.assert_allclose(r.C[:, 0], m / np.linalg.norm(m), rtol=0, atol=1e-15)


def test_planted_disjoint_clusters_recovered():
    """Documents on disjoint vocabulary blocks, each sharing a term with its block's initial
    document (6 of 8 terms drawn): step 1 separates the blocks and step 2 confirms."""
    rng = np.random.default_rng(101)
    k, per, width = 5, 20, 8
    rows, truth = [], []
    for b in range(k):
        for _ in range(per):
            cols = np.sort(rng.choice(width, 6, replace=False)) + b * width
            v = rng.random(6) + 0.1
            v /= np.linalg.norm(v)
            rows.append((cols.tolist(), v.tolist()))
            truth.append(b)
    docs = _csr_from_lists(rows, k * width)
    init = np.array([b * per for b in range(k)])
    r = oracle.fit(docs, k, init, 10)
    np.testing.assert_array_equal(r.a, np.array(truth))
    assert r.iters == 2


def test_k_equals_n_every_doc_its_own_cluster():
    docs, _, _ = _tiny(111, n=40, d=400, k=40, mean=15)
    ids = np.arange(40)
    a, s1, _ = oracle.assign(docs, oracle.init_centroids(docs, 40, ids))
    np.testing.assert_array_equal(a, np.arange(40))
    np.testing.assert_allclose(s1, 1.0, atol=1e-6)    # unit up to float32 storage of x


def test_fixed_point_keeps_centroids():
    docs, ids, k = _tiny(121)
    r = oracle.fit(docs, k, ids, 50)
    assert r.n_changed[-1] == 0                          # converged
    u = oracle.update(docs, r.a, r.C, r.a)
    assert u.n_changed == 0
    np.testing.assert_array_equal(u.C, r.C)


def test_objective_matches_sum_of_best():
    docs, ids, k = _tiny(131)
    r = oracle.fit(docs, k, ids, 4)
    a, s1, _ = oracle.assign(docs, r.C)
    assert abs(oracle.objective(docs, r.C, a) - s1.sum()) < 1e-12


def test_centroids_subset_matches_full_update():
    docs, ids, k = _tiny(141)
    rng = np.random.default_rng(141)
    a = rng.integers(0, k, docs.n_docs).astype(np.int32)
    full = oracle.update(docs, a, np.zeros((docs.n_terms, k))).C
    sel = np.array([3, 0, 7])
    np.testing.assert_array_equal(oracle.centroids_subset(docs, a, sel), full[:, sel])


# ---------------------------------------------------------------- k-means++ seeding (Sec. 2)
def _docs_from_golden(g):
    d = g["docs"]
    return synth.Csr(np.array(d["row_ptr"], np.int64), np.array(d["col_idx"], np.int32),
                     np.array(d["values"], np.float32), d["n_terms"])


def test_hand_kmeanspp():
    g = json.load(open(os.path.join(GOLD, "hand_kmeanspp.json")))
    docs = _docs_from_golden(g)
    for case in g["cases"]:
        ids = oracle.kmeanspp(docs, len(case["ids"]), np.array(case["uniforms"]))
        assert list(ids) == case["ids"]


def test_kmeanspp_first_seed_and_only_weighted_document():
    """Seed 0 is floor(u0 N). With 30 copies of one document and one orthogonal document,
    after a copy is drawn the orthogonal document is the only one with positive weight, so
    it is drawn whatever u1 is; then every weight is zero and the smallest undrawn
    document follows."""
    rows = [([0, 1], [0.6, 0.8])] * 30 + [([2], [1.0])]
    docs = _csr_from_lists(rows, 3)
    for u1 in (0.0, 0.37, 0.999):
        ids = oracle.kmeanspp(docs, 3, np.array([0.5, u1, 0.5]))
        assert ids[0] == 15 and ids[1] == 30 and ids[2] == 0


def test_kmeanspp_draws_in_proportion_to_distance():
    """Over evenly spaced u1, seed 1 lands on each document in proportion to
    1 - x . seed0 (D^2 sampling for unit vectors), computed here from a dense copy."""
    docs, _, _ = _tiny(41, n=60, d=120, k=2)
    X = np.zeros((docs.n_docs, docs.n_terms))
    for i in range(docs.n_docs):
        a, b = docs.row_ptr[i], docs.row_ptr[i + 1]
        X[i, docs.col_idx[a:b]] = docs.values[a:b]
    u0 = 0.25
    s0 = int(np.floor(u0 * docs.n_docs))
    dist = np.maximum(1.0 - X @ X[s0], 0.0)
    dist[s0] = 0.0
    w = np.floor(dist * 2.0 ** 32)
    Q = 20000
    counts = np.zeros(docs.n_docs)
    for q in range(Q):
        ids = oracle.kmeanspp(docs, 2, np.array([u0, (q + 0.5) / Q]))
        assert ids[0] == s0
        counts[ids[1]] += 1
    expect = Q * w / w.sum()
    assert np.all(np.abs(counts - expect) <= 1.0 + 1e-9)


def test_kmeanspp_seeds_are_distinct():
    docs, _, _ = _tiny(43, n=200, d=300, k=50)
    u = synth.uniform(17, 1, 50)
    ids = oracle.kmeanspp(docs, 50, u)
    assert len(set(ids.tolist())) == 50
    assert ids.min() >= 0 and ids.max() < docs.n_docs


def test_kmeanspp_picks_equal_exact_rational_arithmetic_at_every_boundary():
    """Brute force in exact rational arithmetic (Python fractions; every float32 value and
    every product is an exact rational): the weights w_i = floor((1 - x_i . x_s) 2^32) and the
    second seed for uniforms placed on both sides of every prefix-sum boundary. A pick there
    changes with a single unit of weight, so a distance computed in float (errors of hundreds
    of units) fails; double is off by far less than a unit. Boundaries whose exact weight lies
    within 1e-4 of an integer are skipped, because no finite precision decides them."""
    from fractions import Fraction
    docs = synth.make_corpus(24, 40, 8, 3, 16, 1.05, 4711)
    n = docs.n_docs
    X = [dict() for _ in range(n)]
    for i in range(n):
        for p in range(docs.row_ptr[i], docs.row_ptr[i + 1]):
            X[i][int(docs.col_idx[p])] = Fraction(float(docs.values[p]))
    u0 = 0.3
    s0 = int(np.floor(u0 * n))
    w, fracs = [], []
    for i in range(n):
        dist = 1 - sum(v * X[s0].get(t, 0) for t, v in X[i].items())
        scaled = dist * 2 ** 32
        wi = int(scaled // 1) if (i != s0 and dist > 0) else 0
        w.append(wi)
        fracs.append(float(scaled - int(scaled // 1)) if wi else 0.5)
    W = sum(w)
    cum = np.cumsum(np.array(w, dtype=object))
    checked = 0
    for m in range(n):
        if w[m] == 0 or not (1e-4 < fracs[m] < 1 - 1e-4):
            continue
        if any(w[i] and not (1e-4 < fracs[i] < 1 - 1e-4) for i in range(m)):
            break
        for T in (int(cum[m]) - 1, int(cum[m])):
            if T >= W:
                continue
            u1 = (T + 0.5) / W
            assert int(np.floor(u1 * W)) == T
            exact = next(i for i in range(n) if w[i] and cum[i] > T)
            ids = oracle.kmeanspp(docs, 2, np.array([u0, u1]))
            assert ids[0] == s0 and ids[1] == exact
            checked += 1
    assert checked >= 10
