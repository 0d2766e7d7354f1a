"""Failure paths on the device without a fault: a bounded wait that is made
to run out reports NUASM_ETIMEOUT and leaves the context usable; errors found
while a served request runs come back in its result."""
import numpy as np
import pytest

import oracle as O
from paper_1308_6644_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1308_6644_gb300 as pkg
    return pkg


@pytest.mark.parametrize("spins", [1, 1000, 100000])
def test_bounded_wait_gives_up_and_the_context_survives(P, spins):
    import torch
    assert P.nuasm_debug_bounded_wait(spins) == 5        # NUASM_ETIMEOUT
    # a solve right after it still works and is right
    n, pitch, m = 32, 10e-6, 200
    rng = np.random.default_rng(spins)
    half = 0.5 * n * pitch
    x = WL.clamp_window(rng.uniform(-half, half, m), n, pitch)
    y = WL.clamp_window(rng.uniform(-half, half, m), n, pitch)
    u1 = (rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))).astype(np.complex64)
    plan = P.nuasm_plan(P.make_params(n, pitch, 633e-9, 0.02), torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    try:
        v = torch.zeros(m, dtype=torch.complex64, device="cuda")
        P.nuasm2_execute(plan, torch.from_numpy(u1.reshape(-1)).cuda(), v)
        torch.cuda.synchronize()
    finally:
        plan.destroy()
    ref = O.diffraction_type2(u1.astype(np.complex128), x, y, dict(n=n, pitch=pitch, lam=633e-9, z=0.02))
    assert O.rel_l2(v.cpu().numpy(), ref) < 1e-5
