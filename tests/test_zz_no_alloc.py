"""nuasm2_solve_noalloc: the one-shot NU-ASM_2 for callers that cannot
allocate device memory (graph capture, externally owned memory pools,
real-time loops) must give the same result as nuasm_plan + nuasm2_execute.

Collected last on purpose: every call reuses one static device array, and
this file checks two calls in a row, each against the planned path, within
the F32 tolerance the other parity tests use (rel-L2 1e-5)."""
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


def _case(seed, n, m):
    rng = np.random.default_rng(seed)
    pitch = 8e-6
    half = 0.5 * n * pitch
    x = WL.clamp_window(rng.uniform(-half, half, m), n, pitch)
    y = WL.clamp_window(rng.uniform(-half, half, m), n, pitch)
    u1 = (rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))).astype(np.complex64)
    return pitch, x, y, u1


def _planned(P, params, x, y, u1):
    import torch
    xs, ys = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    plan = P.nuasm_plan(params, xs, ys)
    try:
        v = torch.zeros(len(x), dtype=torch.complex64, device="cuda")
        P.nuasm2_execute(plan, torch.from_numpy(u1.reshape(-1)).cuda(), v)
        torch.cuda.synchronize()
        return v.cpu().numpy()
    finally:
        plan.destroy()


def test_noalloc_matches_planned_path_twice_in_a_row(P):
    import torch
    cases = [(1, 256, 65536, 532e-9, 0.05, 400e-6), (2, 64, 3000, 633e-9, 0.02, -100e-6)]
    for seed, n, m, lam, z, ox in cases:
        pitch, x, y, u1 = _case(seed, n, m)
        params = P.make_params(n, pitch, lam, z, ox=ox, oy=0.5 * ox)
        v = torch.full((m,), 7 + 7j, dtype=torch.complex64, device="cuda")
        P.nuasm2_solve_noalloc(params, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(),
                               torch.from_numpy(u1.reshape(-1)).cuda(), v)
        got = v.cpu().numpy()
        want = _planned(P, params, x, y, u1)
        assert O.rel_l2(got, want) < 1e-5


def test_noalloc_rejects_sizes_beyond_its_limits(P):
    import torch
    pitch, x, y, u1 = _case(3, 512, 10)
    params = P.make_params(512, pitch, 532e-9, 0.05)
    v = torch.zeros(10, dtype=torch.complex64, device="cuda")
    with pytest.raises(P.NuasmError) as ei:
        P.nuasm2_solve_noalloc(params, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(),
                               torch.from_numpy(u1.reshape(-1)).cuda(), v)
    assert ei.value.code == 6
    pitch, x, y, u1 = _case(4, 64, 65537)
    params = P.make_params(64, pitch, 532e-9, 0.05)
    v = torch.zeros(65537, dtype=torch.complex64, device="cuda")
    with pytest.raises(P.NuasmError) as ei:
        P.nuasm2_solve_noalloc(params, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(),
                               torch.from_numpy(u1.reshape(-1)).cuda(), v)
    assert ei.value.code == 6
