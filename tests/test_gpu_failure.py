"""Failure detection on the device without a GPU fault.

Every wait in the library's kernels is bounded (2 s on %globaltimer); when it
runs out the kernel sets the handle's error flag and returns, and the host
reads SK_ERR_TIMEOUT.  sketch_selftest_wait makes such a wait run out (a
barrier that nothing completes) and the context must stay usable: a sketch
run afterwards still matches the oracle.  No trap, assert, bad address or
endless loop is involved.
"""
import time

import numpy as np
import pytest

from oracle import operators as ops
from oracle import sketch as osk
from paper_2302_01977_gb300 import inputs
from tests.util import TOL, dev_padded, ensure_built, host, rel_fro

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


def test_bounded_wait_runs_out_and_the_context_stays_usable():
    from paper_2302_01977_gb300 import jlsketch as jl
    t0 = time.monotonic()
    rc = jl.sketch_selftest_wait()
    dt = time.monotonic() - t0
    assert rc == jl.SK_ERR_TIMEOUT
    assert 1.5 <= dt < 60
    # the context works: an SJLT sketch against the oracle
    n, d = 512, 64
    A = inputs.dense_matrix(n, n, seed=3).astype(np.float32)
    h = jl.sketch_create("sjlt_block", n, d, 4, 9, d)
    try:
        S = torch.empty((n, d), dtype=torch.float32, device="cuda")
        St = torch.empty_like(S)
        jl.sketch_apply(h, dev_padded(A, torch.float32), S=S, St=St)
        jl.sketch_device_status(h)
    finally:
        jl.sketch_destroy(h)
    S0, St0 = osk.apply(A.astype(np.float64), ops.Operator("sjlt_block", n, d, 4, 9).dense())
    assert rel_fro(host(S), S0) <= TOL["f32"] and rel_fro(host(St), St0) <= TOL["f32"]
