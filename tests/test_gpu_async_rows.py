"""Asynchronous host copies of the rows (lsp_get_rows_async, lsp_wait_rows).

Copies started after one build and still in flight while the next builds run must deliver the
rows of their own build: bit for bit the rows a synchronous lsp_get_rows returns right after
that build (the rows themselves are checked against the oracle in the parity tests).
"""

import numpy as np
import pytest

from lsp_inputs import make_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1607_02560_gb300 import build as B
    B.build()


def _pinned(torch, shape):
    return torch.empty(shape, dtype=torch.float64, pin_memory=True)


def test_async_rows_of_consecutive_builds_match_their_own_build():
    import torch
    from paper_1607_02560_gb300 import Context

    n = 512
    vs = [make_workload("helm2d_n1024", seed=s, n=n) for s in (11, 12, 13, 14)]
    stream = torch.cuda.Stream()
    ctx = Context(2, n, stream=stream)
    ref = []
    for v in vs:
        ctx.set_potential(v)
        ctx.build_stencils(policy="local", use_graph=True)
        ref.append([ctx.get_rows(w) for w in "QCP"])
    assert not np.array_equal(ref[0][2], ref[1][2])  # a stale copy would be seen
    outs = [[_pinned(torch, (ctx.N, ctx.mu)) for _ in "QCP"] for _ in vs]
    for v, o in zip(vs, outs):  # no wait between the steps
        ctx.set_potential(v)
        ctx.build_stencils(policy="local", use_graph=True)
        for w, t in zip("QCP", o):
            ctx.get_rows_async(w, t)
    ctx.wait_rows()
    for r, o in zip(ref, outs):
        for a, b in zip(r, o):
            assert np.array_equal(a, b.numpy())

    # wider rows (t = 2, 25 per point) regrow the staging copies; the earlier copies still land
    first = [_pinned(torch, (ctx.N, ctx.mu)) for _ in "QCP"]
    for w, t in zip("QCP", first):
        ctx.get_rows_async(w, t)
    ctx.build_stencils(policy="paper", t=2, nd_leaf=8)
    wide = _pinned(torch, (ctx.N, ctx.mu))
    ctx.get_rows_async("P", wide)
    ctx.wait_rows()
    assert ctx.mu == 25
    assert np.array_equal(wide.numpy(), ctx.get_rows("P"))
    for a, b in zip(ref[-1], first):
        assert np.array_equal(a, b.numpy())
    ctx.close()


def test_async_rows_refusals():
    import torch
    from paper_1607_02560_gb300 import Context
    from paper_1607_02560_gb300.lsp import LspError

    v = make_workload("helm2d_n32")
    ctx = Context(2, 32, stream=torch.cuda.Stream())
    host = np.empty((ctx.N, ctx.mu))
    with pytest.raises(LspError):
        ctx.get_rows_async("Q", host)  # no build yet
    ctx.set_potential(v)
    ctx.build_stencils(policy="local")
    with pytest.raises(ValueError):
        ctx.get_rows_async("Q", torch.empty((ctx.N, ctx.mu), dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        ctx.get_rows_async("Q", np.empty((ctx.N, ctx.mu - 1)))
    with pytest.raises(LspError):
        ctx.get_rows_async("X", host)
    ctx.get_rows_async("C", host)  # pageable memory works too (the copy is not overlapped)
    ctx.wait_rows()
    assert np.array_equal(host, ctx.get_rows("C"))
    ctx.close()


def test_pinned_potential_is_read_by_the_statistics_kernel():
    """Page-locked host v is read by the statistics kernel over the host link (no copy engine):
    same stored potential, statistics and rows as pageable host v; a NaN is still refused."""
    import torch
    from paper_1607_02560_gb300 import Context
    from paper_1607_02560_gb300.lsp import LspError

    n = 256
    v = make_workload("helm2d_n1024", seed=21, n=n)
    ctx = Context(2, n, stream=torch.cuda.Stream())
    ctx.set_potential(v)  # pageable: copied first
    ctx.build_stencils(policy="local")
    rows = [ctx.get_rows(w) for w in "QCP"]
    u = torch.from_numpy(np.random.default_rng(3).standard_normal(n * n)).cuda()
    y0 = torch.empty_like(u)
    ctx.apply_operator(u, y0)
    ctx.synchronize()
    pin = torch.empty(v.shape, dtype=torch.float64, pin_memory=True)
    pin.copy_(torch.from_numpy(v))
    ctx.set_potential(pin.numpy())
    ctx.build_stencils(policy="local")
    for w, r in zip("QCP", rows):
        assert np.array_equal(ctx.get_rows(w), r)
    y1 = torch.empty_like(u)
    ctx.apply_operator(u, y1)  # reads the stored v
    ctx.synchronize()
    assert torch.equal(y0, y1)
    pin[3, 5] = float("nan")
    with pytest.raises(LspError, match="NaN"):
        ctx.set_potential(pin.numpy())
    ctx.close()
