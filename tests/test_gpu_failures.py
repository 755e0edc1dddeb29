"""Failure detection without a GPU fault: the bounded waits of the tensor-core kernel run out
on purpose (a wait limit of one nanosecond, so every wait whose operand is not already there
gives up), allocation failures are injected on the host, and a bounds-checked build of the
library runs the parity workloads with no index leaving its array.

A wait that runs out makes the kernel drain its own copies and tensor-core work in flight
(those waits keep their 1 s limit), free its tensor memory and return; the host sees
LSP_ERR_TIMEOUT and the context stays usable. Nothing here faults, traps or hangs a GPU."""

import json
import os
import subprocess
import sys

import numpy as np
import pytest

from lsp_inputs import helmholtz_random_bumps, make_workload

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def stream():
    import torch
    from paper_1607_02560_gb300 import build
    build.build()
    return torch.cuda.Stream()


def test_a_wait_that_runs_out_reports_timeout_and_the_context_recovers(stream):
    import torch
    from paper_1607_02560_gb300 import Context, LspError, Mlp
    from paper_1607_02560_gb300.learned import make_pool
    n = 64
    mlp = Mlp(2, seed=2, stream=stream)
    pots = [helmholtz_random_bumps(n, 2 * np.pi * n / 4, 16, s) for s in (100, 101)]
    X, T = make_pool(mlp, pots, 4096, stream)
    torch.cuda.synchronize()
    mlp.fit_normalization(X, T, X.shape[0])
    ctx = Context(2, n, stream=stream)
    ctx.set_mlp(mlp)
    ctx.set_potential(pots[0])
    ctx.build_stencils(mode="learned")
    ctx.synchronize()
    assert ctx.mode_used() == "learned"
    good = [ctx.get_rows(k).copy() for k in "QCP"]
    mlp.set_wait_limit(1)
    ctx.build_stencils(mode="learned")
    with pytest.raises(LspError) as e:
        ctx.synchronize()
    assert e.value.status == 6  # LSP_ERR_TIMEOUT
    mlp.set_wait_limit(0)  # back to 1 s: the same context builds the same rows again
    ctx.build_stencils(mode="learned")
    ctx.synchronize()
    for k, r in zip("QCP", good):
        assert np.array_equal(ctx.get_rows(k), r)
    # the eigen path of the same context is unaffected
    ctx.build_stencils(mode="fp64")
    ctx.synchronize()


def test_an_injected_allocation_failure_returns_oom(stream):
    from paper_1607_02560_gb300 import Context, LspError, lsp
    v = make_workload("helm2d_n256", n=64)
    ref = Context(2, 64, stream=stream)
    ref.set_potential(v)
    ref.build_stencils(policy="local")
    want = [ref.get_rows(k).copy() for k in "QCP"]
    ctx = Context(2, 64, stream=stream)
    ctx.set_potential(v)
    try:
        for after in (0, 3):
            lsp.inject_alloc_failure(after)
            with pytest.raises(LspError) as e:
                ctx.build_stencils(policy="local")
            assert e.value.status == 5  # LSP_ERR_OOM
    finally:
        lsp.inject_alloc_failure(-1)
    ctx.build_stencils(policy="local")
    ctx.synchronize()
    for k, r in zip("QCP", want):
        assert np.array_equal(ctx.get_rows(k), r)


_CHECKED = r'''
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from lsp_inputs import make_workload
from paper_1607_02560_gb300 import Context, lsp
assert lsp.LIB_PATH.endswith("liblsp_checks.so"), lsp.LIB_PATH
out = {}
for name, n, kw in json.loads(sys.argv[2]):
    v = make_workload(name, n=n)
    ctx = Context(v.ndim, n)
    ctx.set_potential(v)
    ctx.build_stencils(**kw)
    ctx.synchronize()  # raises LSP_ERR_STATE if a checked index left its array
    out[f"{name}/{n}/{sorted(kw.items())}"] = [float(ctx.get_rows(k).sum()) for k in "QCP"]
    ctx.close()
print(json.dumps(out))
'''

CASES = [("helm2d_n256", 64, {"policy": "local"}), ("helm2d_n256", 64, {"policy": "paper"}),
         ("helm2d_n256", 64, {"policy": "local", "mode": "mixed"}),
         ("schr3d_n64", 16, {"policy": "local"}), ("schr3d_n64", 16, {"policy": "paper"}),
         ("helm2d_n32", 32, {"policy": "local", "t": 2, "nd_leaf": 8}),
         ("helm2d_n1024", 1024, {"policy": "local"})]


def test_bounds_checked_build_runs_the_workloads_cleanly(stream):
    from paper_1607_02560_gb300 import Context, build
    lib = build.build(checks=True)
    env = dict(os.environ, LSP_LIBRARY=lib)
    p = subprocess.run([sys.executable, "-c", _CHECKED, ROOT, json.dumps(CASES)], env=env,
                       capture_output=True, text=True, timeout=900)
    assert p.returncode == 0, p.stderr[-3000:]
    got = json.loads(p.stdout.strip().splitlines()[-1])
    for name, n, kw in CASES:  # the checked build computes the same rows
        v = make_workload(name, n=n)
        ctx = Context(v.ndim, n, stream=stream)
        ctx.set_potential(v)
        ctx.build_stencils(**kw)
        want = [float(ctx.get_rows(k).sum()) for k in "QCP"]
        assert got[f"{name}/{n}/{sorted(kw.items())}"] == want, (name, n, kw)
