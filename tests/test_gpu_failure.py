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


def _small_plan(P, seed=3, n=32, pitch=10e-6, m=200):
    import torch
    rng = np.random.default_rng(seed)
    half = 0.5 * n * pitch
    x = WL.clamp_window(rng.uniform(-half, half, m), n, pitch)
    y = WL.clamp_window(rng.uniform(-half, half, m), n, pitch)
    u1 = (rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))).astype(np.complex64)
    params = P.make_params(n, pitch, 633e-9, 0.02)
    return params, x, y, u1, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()


def test_plain_execute_reports_a_wait_that_gave_up(P):
    """A bounded wait that gave up on a plan's error word (what a column pass
    whose copy never arrived leaves behind) makes the plan's next execute
    return NUASM_ETIMEOUT; the call after it runs and is right; nuasm_destroy
    reports a flag left behind."""
    import torch
    params, x, y, u1, dx, dy = _small_plan(P)
    plan = P.nuasm_plan(params, dx, dy)
    v = torch.zeros(x.size, dtype=torch.complex64, device="cuda")
    d_u1 = torch.from_numpy(u1.reshape(-1)).cuda()
    try:
        P.nuasm_debug_plan_wait(plan, 1000)
        with pytest.raises(P.NuasmError) as ei:
            P.nuasm2_execute(plan, d_u1, v)
        assert ei.value.code == 5                        # NUASM_ETIMEOUT, reported once
        P.nuasm2_execute(plan, d_u1, v)
        torch.cuda.synchronize()
        ref = O.diffraction_type2(u1.astype(np.complex128), x, y, dict(n=32, pitch=10e-6, lam=633e-9, z=0.02))
        assert O.rel_l2(v.cpu().numpy(), ref) < 1e-5
        c = torch.zeros(x.size, dtype=torch.complex64, device="cuda")
        u2 = torch.zeros(32 * 32, dtype=torch.complex64, device="cuda")
        P.nuasm_debug_plan_wait(plan, 1)
        with pytest.raises(P.NuasmError) as ei:
            P.nuasm1_execute(plan, c, u2)                # type 1 reads the same word
        assert ei.value.code == 5
        P.nuasm_debug_plan_wait(plan, 1)
    finally:
        code = P.lib().nuasm_destroy(plan._h)
        plan.handle = None
    assert code == 5


def test_batch_execute_reports_a_wait_that_gave_up(P):
    import torch
    params, x, y, u1, dx, dy = _small_plan(P, seed=4)
    plan = P.nuasm_plan(params, dx, dy)
    v = torch.zeros(x.size, dtype=torch.complex64, device="cuda")
    d_u1 = torch.from_numpy(u1.reshape(-1)).cuda()
    batch = P.nuasm_batch_create([(plan, 2, d_u1, v)])
    try:
        P.nuasm_debug_plan_wait(plan, 100)
        with pytest.raises(P.NuasmError) as ei:
            P.nuasm_batch_execute(batch)
        assert ei.value.code == 5
        P.nuasm_batch_execute(batch)
        torch.cuda.synchronize()
    finally:
        batch.destroy()
        plan.destroy()
    ref = O.diffraction_type2(u1.astype(np.complex128), x, y, dict(n=32, pitch=10e-6, lam=633e-9, z=0.02))
    assert O.rel_l2(v.cpu().numpy(), ref) < 1e-5


def _fail_each_acquisition(P, make, limit=64):
    """Fail the 1st, 2nd, ... acquisition of make() until it succeeds: every
    failure must be NUASM_ENOMEM with the live resources back to where they
    were.  Returns the number of acquisitions the call makes."""
    import torch
    torch.cuda.synchronize()
    base = P.nuasm_debug_live_resources()
    for k in range(1, limit + 1):
        P.nuasm_debug_fail_alloc(k)
        try:
            obj = make()
        except P.NuasmError as e:
            P.nuasm_debug_fail_alloc(0)
            assert e.code == 3, (k, e.code)               # NUASM_ENOMEM
            torch.cuda.synchronize()
            assert P.nuasm_debug_live_resources() == base, k
            continue
        P.nuasm_debug_fail_alloc(0)
        obj.destroy()
        torch.cuda.synchronize()
        assert P.nuasm_debug_live_resources() == base
        return k - 1
    raise AssertionError("the call never succeeded")


@pytest.mark.parametrize("kind,weights", [("asm", False), ("asm", True), ("fresnel", False)])
def test_plan_releases_everything_when_an_allocation_fails(P, kind, weights):
    import torch
    params, x, y, u1, dx, dy = _small_plan(P, seed=5)
    params = P.make_params(32, 10e-6, 633e-9, 0.02, kind=kind)
    w = torch.ones(x.size, dtype=torch.float64, device="cuda") if weights else None
    n = _fail_each_acquisition(P, lambda: P.nuasm_plan(params, dx, dy, w))
    assert n >= 8
    # host coordinates take the staging path, with more acquisitions
    assert _fail_each_acquisition(P, lambda: P.nuasm_plan(params, x, y)) > n
    # the lattice plan generates its coordinates in a buffer of its own first
    assert _fail_each_acquisition(P, lambda: P.nuasm_plan_lattice(params, 20, 20, 12e-6, -120e-6, -120e-6)) >= 9


def test_batch_create_releases_everything_when_an_acquisition_fails(P):
    import torch
    params, x, y, u1, dx, dy = _small_plan(P, seed=6)
    plans = [P.nuasm_plan(params, dx, dy) for _ in range(3)]
    outs = [torch.zeros(x.size, dtype=torch.complex64, device="cuda") for _ in range(3)]
    d_u1 = torch.from_numpy(u1.reshape(-1)).cuda()
    try:
        n = _fail_each_acquisition(P, lambda: P.nuasm_batch_create([(p, 2, d_u1, o) for p, o in zip(plans, outs)],
                                                                   lanes=3))
        assert n >= 8    # four streams, four events and the graph
    finally:
        for p in plans:
            p.destroy()


def test_server_requests_fail_cleanly_when_an_acquisition_fails(P):
    """A server with one slot: failing its k-th acquisition (the pool, the
    slot's stream or error words, the binning, the request's pool block)
    gives NUASM_ENOMEM from create or in the request's result, and destroying
    the server leaves nothing behind; with no failure the request is right."""
    import torch
    params, x, y, u1, dx, dy = _small_plan(P, seed=7)
    ref = O.diffraction_type2(u1.astype(np.complex128), x, y, dict(n=32, pitch=10e-6, lam=633e-9, z=0.02))
    torch.cuda.synchronize()
    base = P.nuasm_debug_live_resources()
    statuses = []
    for k in range(1, 80):
        P.nuasm_debug_fail_alloc(k)
        try:
            srv = P.nuasm_server_create(slots=1)
        except P.NuasmError as e:
            P.nuasm_debug_fail_alloc(0)
            assert e.code == 3
            assert P.nuasm_debug_live_resources() == base
            statuses.append(3)
            continue
        out = np.zeros(x.size, np.complex64)
        try:
            t = P.nuasm_server_submit(srv, params, 2, x, y, u1.reshape(-1), out, points_id=1)
            st = P.nuasm_server_wait(srv, t, 60.0)["status"]
        finally:
            P.nuasm_debug_fail_alloc(0)
            srv.destroy()
        torch.cuda.synchronize()
        assert P.nuasm_debug_live_resources() == base, k
        statuses.append(st)
        if st == 0:
            assert O.rel_l2(out, ref) < 1e-5
            break
        assert st == 3, (k, st)
    assert statuses[-1] == 0 and statuses.count(3) >= 5, statuses
