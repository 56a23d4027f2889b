"""k-means++ seeding on the GPU (skm_init_kmeanspp) against the oracle.

The seeds are a deterministic function of the documents and the uniforms (integer weights,
exact prefix sums, dot products summed in double in CSR order), so the GPU must return the
oracle's ids exactly: on the hand-worked fixture, on corpora spanning several weight chunks
(8192 documents each) with a ragged last chunk, with host and device inputs, for k = 1 and
k = N (the last draws find every weight zero).
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2108_00895_gb300 import synth, workloads

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def skm():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2108_00895_gb300 import skm as mod
    mod.load()
    return mod


def _seeds(skm, docs, k, u, device=False):
    with skm.SphericalKMeans(k) as km:
        if device:
            import torch
            dev = (torch.from_numpy(docs.row_ptr).cuda(), torch.from_numpy(docs.col_idx).cuda(),
                   torch.from_numpy(docs.values).cuda())
            return km.init_kmeanspp(dev, u, n_terms=docs.n_terms)
        return km.init_kmeanspp(docs, u)


def test_hand_fixture(skm):
    g = json.load(open(os.path.join(GOLD, "hand_kmeanspp.json")))
    d = g["docs"]
    docs = synth.Csr(np.array(d["row_ptr"], np.int64), np.array(d["col_idx"], np.int32),
                     np.array(d["values"], np.float32), d["n_terms"])
    for case in g["cases"]:
        assert list(_seeds(skm, docs, len(case["ids"]), np.array(case["uniforms"]))) == case["ids"]


@pytest.mark.parametrize("shape", ["small", "tweets", "abstracts"])
def test_seeds_equal_oracle(skm, shape):
    w = {"small": workloads.SMALL.scaled(n_docs=21000, n_terms=9000, k=120),
         "tweets": workloads.TWEETS.scaled(n_docs=30001, n_terms=50000, k=200),
         "abstracts": workloads.ABSTRACTS.scaled(n_docs=17003, n_terms=30000, k=150)}[shape]
    docs = w.corpus()
    for seed in (1, 2):
        u = synth.uniform(900 + seed, 3, w.k)
        ref = oracle.kmeanspp(docs, w.k, u)
        got = _seeds(skm, docs, w.k, u, device=(seed == 2))
        np.testing.assert_array_equal(got, ref)
        assert len(set(got.tolist())) == w.k


def test_k1_and_k_equals_n(skm):
    docs = synth.make_corpus(40, 200, 12, 3, 40, 1.1, 77)
    u = synth.uniform(78, 1, 40)
    assert _seeds(skm, docs, 1, u[:1])[0] == int(np.floor(u[0] * 40))
    got = _seeds(skm, docs, 40, u)
    np.testing.assert_array_equal(got, oracle.kmeanspp(docs, 40, u))
    assert sorted(got.tolist()) == list(range(40))


def test_uniforms_outside_unit_interval_are_rejected(skm):
    docs = synth.make_corpus(50, 100, 10, 3, 30, 1.1, 79)
    for bad in (1.0, -0.25, float("nan")):
        u = np.full(5, 0.5)
        u[2] = bad
        with pytest.raises(skm.SkmError):
            _seeds(skm, docs, 5, u)


def test_fit_from_kmeanspp_seeds_matches_oracle(skm):
    w = workloads.SMALL.scaled(n_docs=3000, n_terms=6000, k=40)
    docs = w.corpus()
    u = synth.uniform(55, 2, w.k)
    ids = _seeds(skm, docs, w.k, u)
    ref = oracle.fit(docs, w.k, ids, 15)
    with skm.SphericalKMeans(w.k, precision="fp32", prune="ncc", max_iter=15) as km:
        r = km.fit(docs, ids)
    assert r.iters == ref.iters
    np.testing.assert_array_equal(r.assign, ref.a)
