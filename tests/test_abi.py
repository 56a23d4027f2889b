"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports every entry
point that include/skm.h declares, and the ctypes structs match the C layout."""
import os
import re
import subprocess

import pytest

from paper_2108_00895_gb300 import build, skm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "skm.h")


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"SKM_API[^;(]*?\b(skm_\w+)\s*\(", text)))


def test_header_declares_the_abi():
    names = _declared()
    assert set(names) == set(skm.EXPORTS)
    for must in ("skm_create", "skm_assign", "skm_update", "skm_fit", "skm_destroy"):
        assert must in names


def test_library_builds_and_exports_every_symbol():
    path = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (skm_\w+)", out))
    missing = set(_declared()) - exported
    assert not missing, f"not exported: {missing}"
    lib = skm.load()
    for name in _declared():
        assert hasattr(lib, name)


def test_build_compiles_for_sm_103a_only():
    """The nvcc command line targets exactly sm_103a (one -gencode, arch-specific)."""
    assert build.ARCH == "-gencode=arch=compute_103a,code=sm_103a"


@pytest.mark.gpu
def test_loaded_kernels_are_sm_103_code():
    """The CUDA runtime reports the loaded scoring kernel as compiled for sm_103."""
    import ctypes
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    torch.cuda.init()
    v = ctypes.c_int32(0)
    assert skm.load().skm_device_code_version(ctypes.byref(v)) == skm.SKM_OK
    assert v.value == 103


def _c_layout():
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "skm.h"
#define F(T, f) printf(#T "." #f " %zu\n", offsetof(T, f));
int main(void) {
  printf("skm_config %zu\n", sizeof(skm_config));
  printf("skm_csr %zu\n", sizeof(skm_csr));
  printf("skm_stats %zu\n", sizeof(skm_stats));
  F(skm_config, shift_tol) F(skm_config, rescore_tau) F(skm_config, mem_budget)
  F(skm_config, stream) F(skm_config, alloc) F(skm_config, alloc_user) F(skm_config, timing)
  F(skm_csr, nnz) F(skm_csr, row_ptr) F(skm_csr, on_device)
  F(skm_stats, sims) F(skm_stats, ms_score) F(skm_stats, launches_total)
  return 0;
}
'''
    tmp = os.path.join(os.environ.get("TMPDIR", "/tmp"), f"skm_layout_{os.getpid()}")
    with open(tmp + ".c", "w") as f:
        f.write(src)
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), "-o", tmp, tmp + ".c"], check=True)
    lines = subprocess.run([tmp], capture_output=True, text=True, check=True).stdout.split("\n")
    os.remove(tmp)
    os.remove(tmp + ".c")
    return dict(line.split() for line in lines if line)


def test_ctypes_structs_match_c_layout():
    c = _c_layout()
    assert int(c["skm_config"]) == skm.ctypes.sizeof(skm.skm_config)
    assert int(c["skm_csr"]) == skm.ctypes.sizeof(skm.skm_csr)
    assert int(c["skm_stats"]) == skm.ctypes.sizeof(skm.skm_stats)
    for key, val in c.items():
        if "." in key:
            struct, field = key.split(".")
            assert getattr(getattr(skm, struct), field).offset == int(val), key


def test_create_rejects_invalid_config_without_touching_a_gpu():
    cfg = skm.skm_config_default(0)        # k = 0 is invalid: rejected before any CUDA call
    with pytest.raises(skm.SkmError) as e:
        skm.skm_create(cfg)
    assert e.value.status == skm.SKM_ERR_INVALID
