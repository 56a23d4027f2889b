"""skm_assign_fixed_scratch: the assignment entry point that allocates no device memory.

It exists for callers that cannot let a library allocate (their device memory belongs to
another allocator or a fixed budget). Its output must equal skm_assign's for an FP32
context without rescoring, on consecutive calls that reuse the shared scratch array. The
file is named to be collected last, so that a run stopping at the first failure has run
every other test before it.
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
            np.testing.assert_array_equal(a.cpu().numpy(), ref_a)
            np.testing.assert_array_equal(s.cpu().numpy(), ref_s)


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
