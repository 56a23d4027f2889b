"""Serving form: continuous batching of assignment requests on a resident model while
clustering jobs run beside it. Every result must equal the same request run alone, and the
FP64 oracle's result within the method's contract: assignments exact wherever the oracle's
top-2 margin is at least 1e-5, objectives to 1e-6 relative."""
import numpy as np
import pytest

import oracle
from paper_2108_00895_gb300 import synth

MARGIN = 1e-5
OBJ_RTOL = 1e-6

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2108_00895_gb300 import skm
    skm.load()
    return torch, skm


def _slice(docs, a, b):
    rp = docs.row_ptr[a:b + 1] - docs.row_ptr[a]
    return synth.Csr(rp.copy(), docs.col_idx[docs.row_ptr[a]:docs.row_ptr[b]].copy(),
                     docs.values[docs.row_ptr[a]:docs.row_ptr[b]].copy(), docs.n_terms)


def _resident(torch, skm, pool, k):
    stream = torch.cuda.Stream()
    km = skm.SphericalKMeans(k, precision="bf16", prune="ncc", max_iter=4, allocator="cuda",
                             stream=stream.cuda_stream)
    km.fit(pool, synth.init_ids(pool.n_docs, k, 7))
    km._stream = stream
    return km


def test_results_alone_equal_results_in_the_mix(env):
    torch, skm = env
    pool = synth.make_corpus(12000, 3000, 40, 5, 300, 1.1, 5150)
    km = _resident(torch, skm, pool, 60)
    rng = np.random.default_rng(9)
    reqs = []
    for _ in range(40):
        n = int(np.exp(rng.uniform(0, np.log(400))))
        a = int(rng.integers(0, pool.n_docs - n))
        reqs.append(_slice(pool, a, a + n))
    alone = [km.assign(r) for r in reqs]                     # before the server owns the context
    C_res = km.centroids()                                   # the resident FP32 master
    jobs = [(_slice(pool, 0, 3000), 17), (_slice(pool, 1000, 5000), 40), (_slice(pool, 2000, 4500), 9)]
    job_ids = [synth.init_ids(d.n_docs, k, 100 + q) for q, (d, k) in enumerate(jobs)]
    alone_jobs = []
    for (d, k), ids in zip(jobs, job_ids):
        with skm.SphericalKMeans(k, precision="bf16", prune="ncc", max_iter=6, tau=1e-4) as j:
            r = j.fit(d, ids)
            alone_jobs.append((r.assign.copy(), r.objective.copy()))
    budget = km.mem_used() + (4 << 30)
    with skm.Server(km, budget, n_job_slots=2, max_batch_docs=2048, max_batch_nnz=2048 * 300, tau=1e-4) as srv:
        tickets = []
        for q, r in enumerate(reqs):                          # interleave jobs with the stream of requests
            tickets.append(("a", q, srv.submit_assign(r)))
            if q % 13 == 0 and q // 13 < len(jobs):
                jq = q // 13
                tickets.append(("f", jq, srv.submit_fit(jobs[jq][0], jobs[jq][1], job_ids[jq], 6)))
        batched = 0
        served, served_jobs = [], []
        for kind, q, t in tickets:
            res = srv.wait(t)
            assert res["state"] == "done", res["message"]
            if kind == "a":
                np.testing.assert_array_equal(res["assign"], alone[q][0])
                np.testing.assert_array_equal(res["score"], alone[q][1])
                batched += res["batch_docs"] > reqs[q].n_docs
                served.append((q, res["assign"].copy(), res["score"].copy()))
            else:
                np.testing.assert_array_equal(res["assign"], alone_jobs[q][0])
                np.testing.assert_array_equal(res["objective"], alone_jobs[q][1])
                served_jobs.append((q, res["assign"].copy(), res["objective"].copy()))
        st = srv.stats()
    assert st["assign_done"] == len(reqs) and st["fit_done"] == len(jobs)
    assert st["assign_batches"] < len(reqs) and batched > 0   # requests were merged into batches
    # against the FP64 oracle: every served assignment on the resident centroids, and every
    # clustering job run as a plain Lloyd fit from the same initial documents
    checked = 0
    for q, a_srv, s_srv in served:
        a_or, s1, s2 = oracle.assign(reqs[q], C_res)
        clear = (s1 - s2) >= MARGIN
        bad = np.nonzero((a_srv != a_or) & clear)[0]
        assert len(bad) == 0, f"request {q}: {len(bad)} clear-margin mismatches"
        # the reported score is the BF16-pass (or FP64-rescored) similarity of the winner:
        # within the BF16 error bound 2^-8 s + FP32 accumulation of the oracle's
        np.testing.assert_allclose(s_srv, s1, rtol=2.0 ** -7, atol=1e-6)
        checked += int(clear.sum())
    assert checked > 0.9 * sum(r.n_docs for r in reqs)
    for q, a_job, obj_job in served_jobs:
        d, k = jobs[q]
        ref = oracle.fit(d, k, job_ids[q], 6)
        # free-running trajectories agree when no document sits on a near tie
        assert len(obj_job) == ref.iters
        np.testing.assert_array_equal(a_job, ref.a)
        np.testing.assert_allclose(obj_job, ref.objective, rtol=OBJ_RTOL, atol=0)


def test_budget_admission_rejects_and_serialises(env):
    torch, skm = env
    pool = synth.make_corpus(6000, 20000, 30, 5, 200, 1.1, 5151)
    km = _resident(torch, skm, pool, 20)
    small = _slice(pool, 0, 2000)
    with skm.Server(km, km.mem_used() + (1 << 30), n_job_slots=2, max_batch_docs=512, max_batch_nnz=512 * 200) as srv:
        reserve = srv.stats()["resident_mem"]
    # a budget that holds small jobs but never a k = 3000 job on d = 20000
    with skm.Server(km, reserve + (300 << 20), n_job_slots=2, max_batch_docs=512, max_batch_nnz=512 * 200) as srv:
        big = srv.submit_fit(pool, 3000, synth.init_ids(pool.n_docs, 3000, 3), 3)
        t1 = srv.submit_fit(small, 8, synth.init_ids(small.n_docs, 8, 4), 3)
        t2 = srv.submit_fit(small, 9, synth.init_ids(small.n_docs, 9, 5), 3)
        assert srv.wait(big)["state"] == "rejected"
        assert srv.wait(t1)["state"] == "done" and srv.wait(t2)["state"] == "done"
        st = srv.stats()
    assert st["rejected"] == 1 and st["fit_done"] == 2
