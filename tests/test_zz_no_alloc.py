"""skm_assign_fixed_scratch: the assignment entry point that allocates no device memory.

It exists for callers that cannot let a library allocate (their device memory belongs to
another allocator or a fixed budget). Its output must equal skm_assign's for an FP32
context without rescoring, on consecutive calls that reuse the shared scratch array, and
the FP64 oracle's within the FP32 error bound. The file is named to be collected last, so
that a run stopping at the first failure has run every other test before it.
"""
import numpy as np
import pytest

import oracle
from paper_2108_00895_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2108_00895_gb300 import skm
    skm.load()
    return torch, skm


def _device_csr(torch, skm, docs):
    dev = (torch.from_numpy(docs.row_ptr).cuda(), torch.from_numpy(docs.col_idx).cuda(),
           torch.from_numpy(docs.values).cuda())
    csr, keep, _ = skm.make_csr(dev, docs.n_terms)
    return csr, keep


def _padded(torch, C, slice_w):
    d, k = C.shape
    ld = (k + slice_w - 1) // slice_w * slice_w
    P = torch.zeros((d, ld), dtype=torch.float32, device="cuda")
    P[:, :k] = torch.from_numpy(C).cuda()
    return P, ld


def test_fixed_scratch_assign_equals_skm_assign_on_consecutive_calls(env):
    torch, skm = env
    k = 300
    base = synth.make_corpus(2000, 4000, 60, 5, 400, 1.1, 4242)
    C = oracle.fit(base, k, synth.init_ids(base.n_docs, k, 4243), 3).C.astype(np.float32)
    Cd, ld = _padded(torch, C, skm.FIXED_SCRATCH_SLICE)
    # two calls in a row with different document sets: the second reuses the scratch the
    # first one left behind
    batches = [base.rows(np.arange(0, 1500)), base.rows(np.arange(700, 2000))]
    with skm.SphericalKMeans(k, precision="fp32", rescore=False) as km:
        km.set_centroids(C)
        for docs in batches:
            ref_a, ref_s = km.assign(docs)
            csr, keep = _device_csr(torch, skm, docs)
            a = torch.full((docs.n_docs,), -1, dtype=torch.int32, device="cuda")
            s = torch.full((docs.n_docs,), float("nan"), dtype=torch.float32, device="cuda")
            skm.skm_assign_fixed_scratch(csr, k, Cd, ld, a, s, torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            a_np, s_np = a.cpu().numpy(), s.cpu().numpy()
            np.testing.assert_array_equal(a_np, ref_a)
            np.testing.assert_array_equal(s_np, ref_s)
            _check_against_oracle(docs, C, a_np, s_np)


def _fp32_bound(docs):
    """Per document: gamma_n = n u / (1 - n u), u = 2^-24, n = its nonzeros. An FP32 score
    summed with one rounding per nonzero over non-negative products is within gamma_n s of
    the exact score s (the centroids are given in float32, so they carry no error of their
    own)."""
    n = np.diff(docs.row_ptr).astype(np.float64)
    nu = n * 2.0 ** -24
    return nu / (1 - nu)


def _check_against_oracle(docs, C32, a_gpu, s_gpu):
    """The oracle in FP64 on the same float32 centroids: each FP32 score is within its bound,
    and the FP32 argmax is the exact argmax wherever the exact top-2 margin exceeds twice the
    bound (no FP32 rounding can reorder those two)."""
    a_or, s1, s2 = oracle.assign(docs, C32.astype(np.float64))
    g = _fp32_bound(docs)
    decided = (s1 - s2) > 2 * g * s1
    assert decided.mean() > 0.9
    np.testing.assert_array_equal(a_gpu[decided], a_or[decided])
    err = np.abs(s_gpu.astype(np.float64) - s1)
    assert np.all(err[decided] <= g[decided] * s1[decided] + 1e-30)
    # elsewhere the FP32 winner's exact score is within 2 g s1 of s1 (it beat the exact winner
    # in FP32), and its FP32 score within g of its exact score
    assert np.all(err <= 3 * g * s1 + 1e-30)


def test_fixed_scratch_rejects_requests_beyond_its_capacity(env):
    torch, skm = env
    k = 2 * skm.FIXED_SCRATCH_SLICE                  # two slices per document
    n = skm.FIXED_SCRATCH_UNITS // 2 + 1
    row_ptr = torch.arange(n + 1, dtype=torch.int64, device="cuda")
    col = torch.zeros(n, dtype=torch.int32, device="cuda")
    val = torch.ones(n, dtype=torch.float32, device="cuda")
    csr, keep, _ = skm.make_csr((row_ptr, col, val), 1)
    Cd = torch.zeros((1, k), dtype=torch.float32, device="cuda")
    a = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(skm.SkmError) as e:
        skm.skm_assign_fixed_scratch(csr, k, Cd, k, a, None, None)
    assert e.value.status == skm.SKM_ERR_BUDGET


def test_fixed_scratch_rejects_negative_or_non_finite_centroids(env):
    """Every score of the method is a sum of non-negative products, so both entry points refuse
    centroids with a negative or non-finite entry: skm_set_centroids (which then leaves no
    resident centroids) and the fixed-scratch call (nothing is written)."""
    torch, skm = env
    k = 40
    docs = synth.make_corpus(300, 1000, 30, 5, 100, 1.1, 4244)
    C = oracle.fit(docs, k, synth.init_ids(docs.n_docs, k, 4245), 2).C.astype(np.float32)
    csr, keep = _device_csr(torch, skm, docs)
    for bad in (-1e-3, float("nan"), float("inf")):
        Cb = C.copy()
        Cb[5, 7] = bad
        with skm.SphericalKMeans(k, precision="fp32", rescore=False) as km:
            with pytest.raises(skm.SkmError) as e:
                km.set_centroids(Cb)
            assert e.value.status == skm.SKM_ERR_INVALID
            with pytest.raises(skm.SkmError) as e:
                km.assign(docs)
            assert e.value.status == skm.SKM_ERR_STATE
        Cd, ld = _padded(torch, Cb, skm.FIXED_SCRATCH_SLICE)
        a = torch.full((docs.n_docs,), -7, dtype=torch.int32, device="cuda")
        with pytest.raises(skm.SkmError) as e:
            skm.skm_assign_fixed_scratch(csr, k, Cd, ld, a, None, torch.cuda.current_stream().cuda_stream)
        assert e.value.status == skm.SKM_ERR_INVALID
        assert bool((a == -7).all())
    # the same documents with the valid centroids: both entry points agree with the oracle
    Cd, ld = _padded(torch, C, skm.FIXED_SCRATCH_SLICE)
    a = torch.full((docs.n_docs,), -1, dtype=torch.int32, device="cuda")
    s = torch.zeros(docs.n_docs, dtype=torch.float32, device="cuda")
    skm.skm_assign_fixed_scratch(csr, k, Cd, ld, a, s, torch.cuda.current_stream().cuda_stream)
    with skm.SphericalKMeans(k, precision="fp32", rescore=False) as km:
        km.set_centroids(C)
        ref_a, ref_s = km.assign(docs)
    np.testing.assert_array_equal(a.cpu().numpy(), ref_a)
    _check_against_oracle(docs, C, a.cpu().numpy(), s.cpu().numpy())
