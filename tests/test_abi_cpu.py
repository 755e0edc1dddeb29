"""The C ABI library builds for sm_103a, loads, and exports every symbol include/lsp.h declares.

No compute call is made here (no GPU on this host); only argument checks that fail before any
CUDA call are exercised.
"""

import ctypes
import os

import pytest

from paper_1607_02560_gb300 import build as B
from paper_1607_02560_gb300 import lsp


@pytest.fixture(scope="module")
def L():
    B.build()
    return lsp.lib()


def test_every_declared_symbol_is_exported(L):
    names = lsp.declared_symbols()
    assert "lsp_build_stencils" in names and "lsp_set_potential" in names
    assert len(names) >= 14
    for name in names:
        assert hasattr(L, name), name


def test_default_opts(L):
    o = lsp.default_opts()
    assert (o.t, o.policy, o.mode, o.eig_method, o.use_graph, o.nd_leaf) == (1, 1, 0, 0, 0, 0)


@pytest.mark.parametrize("d,n", [(0, 16), (4, 16), (2, 12), (2, 4), (2, 8192), (3, 512),
                                 (1, 4), (1, 8192)])
def test_create_rejects_bad_sizes_before_touching_the_device(L, d, n):
    h = ctypes.c_void_p()
    st = L.lsp_create(d, n, None, ctypes.byref(h))
    assert st == 1 and not h.value  # LSP_ERR_ARG


def test_null_context_is_rejected(L):
    assert L.lsp_destroy(None) == 0
    assert L.lsp_set_potential(None, None, 0) == 1
    assert L.lsp_build_stencils(None, None) == 1
    assert L.lsp_synchronize(None) == 1
    assert L.lsp_get_rows_async(None, b"Q", None) == 1
    assert L.lsp_wait_rows(None) == 1
    assert L.lsp_last_error(None) == b"null context"


def test_status_codes_match_header():
    text = open(lsp.HEADER).read()
    for code, name in lsp.STATUS.items():
        assert f"{name} = {code}" in text


def test_product_path_does_not_import_the_oracle():
    import os
    pkg = os.path.dirname(lsp.__file__)
    for root, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h")):
                src = open(os.path.join(root, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f


def test_bounds_checked_kernels_compile():
    """The -DLSP_CHECKS build (index checks that report through the error word) compiles."""
    import shutil
    import subprocess
    import tempfile
    from paper_1607_02560_gb300 import build as B
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no nvcc")
    with tempfile.TemporaryDirectory() as tmp:
        for name in ("k_rows.cu", "k_stage.cu"):
            src = os.path.join(B.CSRC, name)
            cmd = [B.nvcc(), *B.ARCH, *B.FLAGS, "-DLSP_CHECKS", "-c", src, "-o",
                   os.path.join(tmp, name + ".o")]
            r = subprocess.run(cmd, capture_output=True, text=True)
            assert r.returncode == 0, r.stderr[-2000:]
