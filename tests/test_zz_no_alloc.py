"""The allocation-free entry point, casimir_run_noalloc, against casimir_run and the oracle.

casimir_run_noalloc serves callers that cannot let a library allocate device memory
(a host whose GPU memory is already reserved by its own pool, a memory manager that
must not be re-entered from its own callbacks, a loop that cannot absorb cudaFree's
device-wide synchronisation): its scratch lives in a static device array.  This file
is collected last so that a run stopping at the first failure has run every other test.
The test itself allocates the output buffer; the entry point allocates nothing.  Two
calls in a row must both match casimir_run (the existing entry point) and the FP64
oracle simulation by simulation, because the array keeps the previous call's contents.
"""
import ctypes

import numpy as np
import pytest

import oracle
import workloads as W
from parity_bounds import assert_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pk():
    from paper_0906_5170_gb300 import build
    build.build()
    import paper_0906_5170_gb300 as pkg
    return pkg


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_noalloc_matches_run_on_two_calls(pk, prec):
    import torch
    ctx = pk.Context(0)
    p = W.piston_small(n_steps=500, precision=prec)
    _, ref, _ = ctx.plan(p).run(per_sim=True)
    Fo, parts, sims = oracle.force(p, return_parts=True)
    kw = np.array([p["k_points"][s["k"]]["weight"] for s in sims])
    plan = pk.Plan(p)                                   # host-only plan: no context, no device memory
    n = plan.info()["n_sims"]
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()
    for _ in range(2):
        out.fill_(float("nan"))
        torch.cuda.synchronize()
        pk.capi.check(pk.lib().casimir_run_noalloc(plan.h, ctypes.c_void_p(out.data_ptr()),
                                                   ctypes.c_void_p(stream.cuda_stream)))
        stream.synchronize()
        got = out.cpu().numpy() * kw          # the entry point leaves out the k-point weight
        if prec == "fp64":
            assert np.all(np.abs(got - ref) <= 1e-10 * np.abs(ref))
        else:
            assert np.max(np.abs(got - ref)) <= 2e-5 * np.max(np.abs(ref))
        assert_parity(got, float(np.sum(got)), parts, Fo, p["n_steps"], prec == "fp64", "noalloc " + prec)
    ctx.close()


def test_noalloc_rejects_plans_beyond_the_static_array(pk):
    import torch
    plan = pk.Plan(W.config2_piston(W.config2_heights()[7], n_steps=10))
    out = torch.empty(plan.info()["n_sims"], dtype=torch.float64, device="cuda")
    rc = pk.lib().casimir_run_noalloc(plan.h, ctypes.c_void_p(out.data_ptr()), None)
    assert rc == -2
    assert b"static array" in pk.lib().casimir_last_error()
