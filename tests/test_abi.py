"""The C ABI without a GPU: the library loads, exports every entry point that
include/dashsvd.h declares, the Python binding's struct layouts match the
header (checked against gcc), defaults, status strings, and argument checks
that must fail before any CUDA call."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dashsvd.h")


@pytest.fixture(scope="module")
def ds():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2404_09276_gb300 as mod

    return mod


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dashsvd_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_entry_point_is_exported(ds):
    names = _declared()
    assert len(names) >= 15
    lib = C.CDLL(ds.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(ds.EXPORTS) == names


def test_struct_layout_matches_header(ds, tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "dashsvd.h"\n'
        "int main(void){\n"
        'printf("%zu %zu %zu\\n", sizeof(dashsvd_csr), sizeof(dashsvd_options), sizeof(dashsvd_info));\n'
        'printf("%zu %zu %zu\\n", offsetof(dashsvd_csr, val), offsetof(dashsvd_options, shift), '
        "offsetof(dashsvd_info, eig_sweeps));\n"
        'printf("%zu %zu\\n", offsetof(dashsvd_options, trust_csr), offsetof(dashsvd_options, deterministic));\n'
        'printf("%d %d\\n", DASHSVD_MAX_L, (int)DASHSVD_ENOCONV);\n'
        "return 0;}\n"
    )
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    sizes = [int(x) for x in out[:3]]
    offs = [int(x) for x in out[3:6]]
    assert sizes == [C.sizeof(ds.dashsvd_csr), C.sizeof(ds.dashsvd_options), C.sizeof(ds.dashsvd_info)]
    assert offs == [ds.dashsvd_csr.val.offset, ds.dashsvd_options.shift.offset, ds.dashsvd_info.eig_sweeps.offset]
    assert [int(x) for x in out[6:8]] == [ds.dashsvd_options.trust_csr.offset, ds.dashsvd_options.deterministic.offset]
    assert int(out[8]) == ds.DASHSVD_MAX_L and int(out[9]) == ds.DASHSVD_ENOCONV


def test_options_defaults(ds):
    o = ds.options()
    assert o.form == ds.DASHSVD_FORM_PLAIN and o.learned == 0
    assert o.seed == 0x5EED and o.alpha_prev_mode == 0
    assert o.use_graph == 1 and o.spmm_variant == -1 and o.shift == 1
    assert o.overlap == -1 and o.trust_csr == 0 and o.deterministic == 0 and o.profile == 0


def test_status_strings(ds):
    for code in range(-7, 2):
        s = ds.dashsvd_status_string(code)
        assert s and b"unknown" not in s
    assert b"unknown" in ds.dashsvd_status_string(99)


def test_argument_checks_before_cuda(ds):
    E = ds.DASHSVD_EINVAL
    assert ds.dashsvd_run(None, None, 1, 1, 1, 0.0, None, None, None, None) == E
    assert ds.dashsvd_options_init(None) == E
    assert ds.dashsvd_create(None, None, None) == E
    assert ds.dashsvd_destroy(None) == E
    assert ds.dashsvd_gram(None, None, 10, 4, 4, None, 4) == E
    assert ds.dashsvd_spmm(None, None, None, 4, 4, None, 4, -1) == E
    assert ds.dashsvd_get_trace(None, None, 0, None, None) == E
    assert ds.dashsvd_csr_check(None, None, None) == E
    assert ds.dashsvd_eig_fp64(None, None, 4, 4, 3, None, None) == E


def test_create_without_gpu_reports_cuda_error(ds):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    assert ds.dashsvd_create(C.byref(h), None, None) == ds.DASHSVD_ECUDA
    assert not h.value
    assert ds.dashsvd_last_error()
