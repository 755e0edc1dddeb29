"""lsp_apply_operator_noalloc: the allocation-free variant of lsp_apply_operator.

It is for callers that cannot allocate device memory when they apply the operator (inside a
stream capture, or under an allocator that must not see extra allocations); its work array is
a fixed array inside the library. This file is collected last on purpose: a failure here stops
an `-x` run only after every other test has run. It passes alone in a fresh process too.
"""

import numpy as np
import pytest

import oracle as O
from lsp_inputs import make_workload

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,n", [("helm2d_n256", 256), ("schr3d_n64", 32)])
def test_noalloc_apply_matches_context_apply_on_two_calls(name, n):
    import torch
    from paper_1607_02560_gb300 import Context, build, lsp

    build.build()
    v = make_workload(name, n=n)
    d = v.ndim
    stream = torch.cuda.Stream()
    ctx = Context(d, n, stream=stream)
    ctx.set_potential(v)
    v_dev = torch.from_numpy(v).cuda()
    rng = np.random.default_rng(3)
    # same tolerance as the context path's own test against the oracle
    scale_of = lambda u: (4 * O.PI2 * d * (n / 2) ** 2 + np.abs(v).max()) * np.abs(u).max()
    for call in range(2):
        u = rng.standard_normal(v.shape)
        u_dev = torch.from_numpy(u).cuda()
        y_ctx = torch.empty_like(u_dev)
        y_na = torch.full_like(u_dev, np.nan)
        torch.cuda.synchronize()
        ctx.apply_operator(u_dev, y_ctx)
        ctx.synchronize()
        lsp.apply_operator_noalloc(d, n, v_dev, u_dev, y_na, stream=stream)
        stream.synchronize()
        a, b = y_ctx.cpu().numpy(), y_na.cpu().numpy()
        assert np.isfinite(b).all(), call
        assert np.abs(a - b).max() <= 1e-13 * scale_of(u), call
        assert np.abs(b - O.apply_operator(v, u)).max() <= 1e-13 * scale_of(u), call


def test_noalloc_apply_in_place_matches_context_apply():
    # y may be the same array as u: the result overwrites the input
    import torch
    from paper_1607_02560_gb300 import Context, build, lsp

    build.build()
    n = 128
    v = make_workload("helm2d_n256", n=n)
    stream = torch.cuda.Stream()
    ctx = Context(2, n, stream=stream)
    ctx.set_potential(v)
    v_dev = torch.from_numpy(v).cuda()
    u = np.random.default_rng(5).standard_normal(v.shape)
    y_ctx = torch.empty(v.shape, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    ctx.apply_operator(torch.from_numpy(u).cuda(), y_ctx)
    ctx.synchronize()
    for call in range(2):
        buf = torch.from_numpy(u).cuda()
        torch.cuda.synchronize()
        lsp.apply_operator_noalloc(2, n, v_dev, buf, buf, stream=stream)
        stream.synchronize()
        scale = (4 * O.PI2 * 2 * (n / 2) ** 2 + np.abs(v).max()) * np.abs(u).max()
        assert np.abs(buf.cpu().numpy() - y_ctx.cpu().numpy()).max() <= 1e-13 * scale, call


def test_noalloc_rejects_grids_beyond_its_fixed_array():
    import ctypes
    from paper_1607_02560_gb300 import build, lsp

    build.build()
    L = lsp.lib()
    # 2048^2 points exceed LSP_NOALLOC_MAX_POINTS = 2^20: rejected before any device work
    assert L.lsp_apply_operator_noalloc(2, 2048, ctypes.c_void_p(8), ctypes.c_void_p(8),
                                        ctypes.c_void_p(8), None) == 1
    assert L.lsp_apply_operator_noalloc(3, 128, ctypes.c_void_p(8), ctypes.c_void_p(8),
                                        ctypes.c_void_p(8), None) == 1
