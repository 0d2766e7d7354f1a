"""Batched planes (one CUDA graph over many plans) and the serving loop
(continuous batching with resident point sets), through the C ABI.

A batch item is checked against the same solve run alone through the plain
entry points (nuasm_plan + nuasm*_execute), a served request against the same
request served alone, and both, for a sample, against the FP64 oracle.  Type 2
runs are deterministic and must agree bit for bit; type 1 spreading
accumulates with shared-memory atomics whose order varies, so type 1 results
agree to rounding (rel-L2 1e-6 in FP32, 1e-13 in FP64).  A served request and
the plain path agree within the parity tolerance (1e-5 FP32, 1e-10 FP64): a
plan tabulates the non-separable ASM phase factor, a request evaluates it per
mode."""
import numpy as np
import pytest

import oracle as O
from paper_1308_6644_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-5, "f64": 1e-10}
SAME = {"f32": 1e-6, "f64": 1e-13}
CDT = {"f32": np.complex64, "f64": np.complex128}


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1308_6644_gb300 as pkg
    return pkg


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _points(seed, n, m, pitch):
    rng = np.random.default_rng(seed)
    half = 0.5 * n * pitch
    return (WL.clamp_window(rng.uniform(-half, half, m), n, pitch),
            WL.clamp_window(rng.uniform(-half, half, m), n, pitch))


def _values(seed, count, prec):
    rng = np.random.default_rng(seed)
    return (rng.normal(size=count) + 1j * rng.normal(size=count)).astype(CDT[prec])


def _execute(P, plan, kind, type_, inp, out):
    if kind == "asm":
        (P.nuasm1_execute if type_ == 1 else P.nuasm2_execute)(plan, inp, out)
    else:
        P.nufresnel_execute(plan, type_, inp, out)


def _same(a, b, prec, type_):
    if type_ == 2:
        return np.array_equal(a, b)
    return O.rel_l2(a, b) < SAME[prec]


# ---------------------------------------------------------------- batches
PLANES = [  # kind, type, prec, n, m, z, lambda
    ("asm", 1, "f32", 32, 300, 0.02, 633e-9),
    ("asm", 2, "f32", 64, 900, 0.05, 532e-9),
    ("fresnel", 1, "f32", 64, 500, 0.10, 450e-9),
    ("fresnel", 2, "f64", 32, 200, 0.03, 633e-9),
    ("asm", 2, "f32", 128, 5000, 0.20, 532e-9),
    ("asm", 1, "f64", 64, 700, 0.04, 633e-9),
    ("asm", 2, "f32", 256, 20000, 0.35, 450e-9),
    ("fresnel", 1, "f64", 256, 3000, 0.06, 532e-9),   # FP64 at N' = 512: double-float passes
]


def _make_planes(P):
    import torch
    planes = []
    for i, (kind, type_, prec, n, m, z, lam) in enumerate(PLANES):
        pitch = 8e-6
        x, y = _points(700 + i, n, m, pitch)
        params = P.make_params(n, pitch, lam, z, ox=10e-6 * i, kind=kind, prec=prec)
        plan = P.nuasm_plan(params, _t(x), _t(y))
        count_in = m if type_ == 1 else n * n
        count_out = n * n if type_ == 1 else m
        inp = _t(_values(800 + i, count_in, prec))
        tdt = torch.complex64 if prec == "f32" else torch.complex128
        planes.append(dict(kind=kind, type=type_, prec=prec, n=n, x=x, y=y, z=z, lam=lam, ox=10e-6 * i,
                           plan=plan, inp=inp, out=torch.zeros(count_out, dtype=tdt, device="cuda"),
                           ref=torch.zeros(count_out, dtype=tdt, device="cuda")))
    return planes


def _destroy(planes):
    for p in planes:
        p["plan"].destroy()


def test_batch_matches_single_calls_and_the_oracle(P):
    import torch
    planes = _make_planes(P)
    try:
        batch = P.nuasm_batch_create([(p["plan"], p["type"], p["inp"], p["out"]) for p in planes], lanes=3)
        lanes, kernels = batch.info()
        assert lanes == 3 and kernels == 4 * len(planes)
        batch.execute()
        for p in planes:
            _execute(P, p["plan"], p["kind"], p["type"], p["inp"], p["ref"])
        torch.cuda.synchronize()
        for p in planes:
            got, ref = p["out"].cpu().numpy(), p["ref"].cpu().numpy()
            assert _same(got, ref, p["prec"], p["type"]), (p["kind"], p["type"], p["n"])
        for p in planes[:4] + planes[-1:]:   # the last: FP64 at N' = 512
            prm = dict(n=p["n"], pitch=8e-6, lam=p["lam"], z=p["z"], ox=p["ox"], kind=p["kind"])
            vals = p["inp"].cpu().numpy().astype(np.complex128)
            if p["type"] == 1:
                want = O.diffraction_type1(p["x"], p["y"], vals, prm).reshape(-1)
            else:
                want = O.diffraction_type2(vals.reshape(p["n"], p["n"]), p["x"], p["y"], prm)
            assert O.rel_l2(p["out"].cpu().numpy(), want) < TOL[p["prec"]]
        batch.destroy()
    finally:
        _destroy(planes)


def test_batch_replay_reads_new_inputs(P):
    import torch
    planes = _make_planes(P)[:4]
    try:
        batch = P.nuasm_batch_create([(p["plan"], p["type"], p["inp"], p["out"]) for p in planes], lanes=2)
        batch.execute()
        for i, p in enumerate(planes):
            p["inp"].copy_(_t(_values(900 + i, p["inp"].numel(), p["prec"])))
        batch.execute()
        for p in planes:
            _execute(P, p["plan"], p["kind"], p["type"], p["inp"], p["ref"])
        torch.cuda.synchronize()
        for p in planes:
            assert _same(p["out"].cpu().numpy(), p["ref"].cpu().numpy(), p["prec"], p["type"])
        batch.destroy()
    finally:
        _destroy(planes)


def test_batch_items_sharing_a_plan_and_type3(P):
    """Two inputs through one plan (they share its workspace, so one lane runs
    them in order) and a type-3 item."""
    import torch
    n, pitch, m = 64, 8e-6, 1500
    x, y = _points(41, n, m, pitch)
    x2, y2 = _points(42, n, 800, pitch)
    params = P.make_params(n, pitch, 532e-9, 0.05, ox=20e-6)
    pa = P.nuasm_plan(params, _t(x), _t(y))
    pd = P.nuasm_plan(params, _t(x2), _t(y2))
    try:
        u_a, u_b = _t(_values(1, n * n, "f32")), _t(_values(2, n * n, "f32"))
        c = _t(_values(3, m, "f32"))
        outs = [torch.zeros(m, dtype=torch.complex64, device="cuda") for _ in range(2)]
        v3 = torch.zeros(800, dtype=torch.complex64, device="cuda")
        batch = P.nuasm_batch_create([(pa, 2, u_a, outs[0]), (pa, 2, u_b, outs[1]), (pa, 3, c, v3, pd)], lanes=4)
        assert batch.info()[0] == 1          # every item writes pa's workspace
        batch.execute()
        torch.cuda.synchronize()
        for u, o in ((u_a, outs[0]), (u_b, outs[1])):
            ref = torch.zeros_like(o)
            P.nuasm2_execute(pa, u, ref)
            torch.cuda.synchronize()
            assert np.array_equal(o.cpu().numpy(), ref.cpu().numpy())
        ref3 = torch.zeros_like(v3)
        P.nuasm3_execute(pa, pd, c, ref3)
        torch.cuda.synchronize()
        assert O.rel_l2(v3.cpu().numpy(), ref3.cpu().numpy()) < SAME["f32"]
        batch.destroy()
    finally:
        pa.destroy()
        pd.destroy()


def test_batch_rejects_host_arrays(P):
    n, pitch = 32, 8e-6
    x, y = _points(5, n, 100, pitch)
    plan = P.nuasm_plan(P.make_params(n, pitch, 633e-9, 0.02), _t(x), _t(y))
    try:
        with pytest.raises(P.NuasmError) as ei:
            P.nuasm_batch_create([(plan, 2, np.zeros(n * n, np.complex64), np.zeros(100, np.complex64))])
        assert ei.value.code == 1
    finally:
        plan.destroy()


# ---------------------------------------------------------------- serving
def _requests(P):
    """Requests over three resident point sets (ids 11, 12, 13) and one FP64
    set (id 14), with wavelength, distance, offset, kind and type varying
    between requests on the same set, plus two unkept sets (id 0)."""
    sets = {11: (64, 800), 12: (32, 300), 13: (128, 3000), 14: (256, 500), 0: (32, 150)}
    pts = {k: _points(1000 + k, n, m, 8e-6) for k, (n, m) in sets.items()}
    reqs = []
    rng = np.random.default_rng(77)
    ids = [11, 12, 13, 11, 13, 12, 14, 11, 0, 13, 14, 12, 11, 13, 0, 11]
    for i, sid in enumerate(ids):
        n, m = sets[sid]
        prec = "f64" if sid == 14 else "f32"
        kind = "fresnel" if i % 3 == 2 else "asm"
        type_ = 1 + (i % 2)
        z = float(rng.uniform(0.01, 0.5))
        lam = float(rng.choice([450e-9, 532e-9, 633e-9]))
        params = P.make_params(n, 8e-6, lam, z, ox=float(rng.uniform(-50e-6, 50e-6)), kind=kind, prec=prec)
        inp = _values(2000 + i, m if type_ == 1 else n * n, prec)
        out = np.zeros(n * n if type_ == 1 else m, CDT[prec])
        reqs.append(dict(id=sid, params=params, type=type_, kind=kind, prec=prec, n=n, x=pts[sid][0],
                         y=pts[sid][1], inp=inp, out=out, z=z, lam=lam))
    return reqs


def _served_alone(P, reqs):
    """Each request through a one-slot server with nothing else in flight."""
    outs = []
    srv = P.nuasm_server_create(slots=1)
    try:
        for r in reqs:
            out = np.zeros_like(r["out"])
            t = P.nuasm_server_submit(srv, r["params"], r["type"], r["x"], r["y"], r["inp"], out,
                                      points_id=r["id"])
            assert P.nuasm_server_wait(srv, t, 120.0)["status"] == 0
            outs.append(out)
    finally:
        srv.destroy()
    return outs


def _alone(P, r):
    """The request on the plain path: its own plan and one execute.  A plan
    tabulates the non-separable ASM phase factor once, a served request
    evaluates it per mode, so the two agree within the parity tolerance."""
    plan = P.nuasm_plan(r["params"], r["x"], r["y"])
    try:
        out = np.zeros_like(r["out"])
        _execute(P, plan, r["kind"], r["type"], r["inp"], out)
        import torch
        torch.cuda.synchronize()
        return out
    finally:
        plan.destroy()


def test_server_results_alone_and_in_the_mix(P):
    """Every served result equals the same request served alone (bit for bit
    for type 2; type 1 sums in floating point atomically) and the plain path
    within the parity tolerance."""
    reqs = _requests(P)
    plain = [_alone(P, r) for r in reqs]
    alone = _served_alone(P, reqs)
    srv = P.nuasm_server_create(slots=4)
    try:
        tickets = [P.nuasm_server_submit(srv, r["params"], r["type"], r["x"], r["y"], r["inp"], r["out"],
                                         points_id=r["id"]) for r in reqs]
        results = [P.nuasm_server_wait(srv, t, 120.0) for t in tickets]
        st = P.nuasm_server_stats(srv)
    finally:
        srv.destroy()
    for r, res, a, q in zip(reqs, results, alone, plain):
        assert res["status"] == 0
        assert _same(r["out"], a, r["prec"], r["type"]), (r["id"], r["kind"], r["type"])
        assert O.rel_l2(r["out"], q) < TOL[r["prec"]], (r["id"], r["kind"], r["type"])
    assert st["completed"] == len(reqs) and st["failed"] == 0
    kept = {r["id"] for r in reqs if r["id"]}
    unkept = sum(1 for r in reqs if not r["id"])
    assert st["bins_built"] == len(kept) + unkept
    assert st["bins_reused"] == len(reqs) - st["bins_built"]
    assert st["resident_sets"] == len(kept)
    assert 0 < st["p50_ms"] <= st["p99_ms"]
    # one request per set against the oracle
    seen = set()
    for r in reqs:
        if r["id"] in seen:
            continue
        seen.add(r["id"])
        prm = dict(n=r["n"], pitch=8e-6, lam=r["lam"], z=r["z"], ox=r["params"].ox, kind=r["kind"])
        vals = r["inp"].astype(np.complex128)
        if r["type"] == 1:
            want = O.diffraction_type1(r["x"], r["y"], vals, prm).reshape(-1)
        else:
            want = O.diffraction_type2(vals.reshape(r["n"], r["n"]), r["x"], r["y"], prm)
        assert O.rel_l2(r["out"], want) < TOL[r["prec"]]


def test_server_evicts_under_a_small_budget(P):
    """Six point sets of 100k points, a 16 MB budget: resident sets are evicted
    least recently used and rebuilt, results unchanged."""
    n, pitch, m = 128, 8e-6, 100_000
    pts = [_points(3000 + k, n, m, pitch) for k in range(6)]
    reqs = []
    for i in range(12):
        k = i % 6
        params = P.make_params(n, pitch, 532e-9, 0.05 + 0.01 * i)
        reqs.append(dict(id=k + 1, params=params, type=2, kind="asm", prec="f32", n=n, x=pts[k][0], y=pts[k][1],
                         inp=_values(4000 + i, n * n, "f32"), out=np.zeros(m, np.complex64)))
    srv = P.nuasm_server_create(slots=2, hbm_budget=16 << 20)
    try:
        tickets = [P.nuasm_server_submit(srv, r["params"], 2, r["x"], r["y"], r["inp"], r["out"], points_id=r["id"])
                   for r in reqs]
        results = [P.nuasm_server_wait(srv, t, 120.0) for t in tickets]
        st = P.nuasm_server_stats(srv)
    finally:
        srv.destroy()
    assert all(res["status"] == 0 for res in results)
    assert st["evictions"] > 0 and st["bins_built"] > 6
    again = _served_alone(P, reqs[:3] + reqs[-3:])
    for r, a in zip(reqs[:3] + reqs[-3:], again):
        assert np.array_equal(r["out"], a)
        assert O.rel_l2(r["out"], _alone(P, r)) < TOL["f32"]


def test_server_device_arrays_and_out_of_window_points(P):
    import torch
    n, pitch, m = 64, 8e-6, 600
    x, y = _points(51, n, m, pitch)
    params = P.make_params(n, pitch, 633e-9, 0.03)
    u1 = _values(52, n * n, "f32")
    out_d = torch.zeros(m, dtype=torch.complex64, device="cuda")
    bad_x = x.copy()
    bad_x[7] = 0.5 * n * pitch          # on the excluded edge of the window
    srv = P.nuasm_server_create(slots=2)
    try:
        t_bad = P.nuasm_server_submit(srv, params, 2, bad_x, y, u1, np.zeros(m, np.complex64), points_id=5)
        t_ok = P.nuasm_server_submit(srv, params, 2, _t(x), _t(y), _t(u1), out_d, points_id=6)
        bad = P.nuasm_server_wait(srv, t_bad, 60.0)
        ok = P.nuasm_server_wait(srv, t_ok, 60.0)
        with pytest.raises(P.NuasmError):
            P.nuasm_server_wait(srv, t_ok, 1.0)      # a ticket is forgotten once waited for
        st = P.nuasm_server_stats(srv)
    finally:
        srv.destroy()
    assert bad["status"] == 2 and ok["status"] == 0
    assert st["failed"] == 1 and st["resident_sets"] == 1
    ref = torch.zeros_like(out_d)
    plan = P.nuasm_plan(params, _t(x), _t(y))
    try:
        P.nuasm2_execute(plan, _t(u1), ref)
        torch.cuda.synchronize()
    finally:
        plan.destroy()
    assert O.rel_l2(out_d.cpu().numpy(), ref.cpu().numpy()) < TOL["f32"]


def test_server_accepts_requests_from_several_threads(P):
    """Four client threads submit and wait at once; every result equals the
    request solved alone."""
    import threading
    reqs = _requests(P)[:12]
    alone = _served_alone(P, reqs)
    srv = P.nuasm_server_create(slots=3)
    errors = []

    def client(idx):
        try:
            for k in idx:
                r = reqs[k]
                t = P.nuasm_server_submit(srv, r["params"], r["type"], r["x"], r["y"], r["inp"], r["out"],
                                          points_id=r["id"])
                res = P.nuasm_server_wait(srv, t, 120.0)
                if res["status"] != 0:
                    errors.append((k, res["status"]))
        except Exception as e:   # pragma: no cover - reported below
            errors.append((idx, repr(e)))

    threads = [threading.Thread(target=client, args=(list(range(i, len(reqs), 4)),)) for i in range(4)]
    try:
        for t in threads:
            t.start()
        for t in threads:
            t.join()
    finally:
        srv.destroy()
    assert not errors
    for r, a in zip(reqs, alone):
        assert _same(r["out"], a, r["prec"], r["type"])
