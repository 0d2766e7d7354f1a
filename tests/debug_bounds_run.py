"""Runs every kernel family of the library once through the C ABI and prints,
as one JSON list, the bounds records (skipped out-of-range accesses) that
the library reports after each case.  Meant for the bounds-checking debug
library: `NUASM_LIBRARY=.../libnuasm_debug.so python tests/debug_bounds_run.py`
(tests/test_gpu_debug_bounds.py runs it so).  Needs a GPU."""
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import torch  # noqa: E402

import paper_1308_6644_gb300 as P  # noqa: E402
from paper_1308_6644_gb300 import workloads as WL  # noqa: E402

DEV = torch.device("cuda")
CDT = {"f32": (np.complex64, torch.complex64), "f64": (np.complex128, torch.complex128)}


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def values(rng, m, prec):
    return dev(WL.random_phasor(rng, (m,)).astype(CDT[prec][0]))


def solve(params, x, y, type_, prec, rng, w=None):
    """One plan and one execute of `type_` (1, 2) on device points."""
    plan = P.nuasm_plan(params, dev(x), dev(y), None if w is None else dev(w))
    n, m = params.n, len(x)
    try:
        src = values(rng, m if type_ == 1 else n * n, prec)
        out = torch.zeros(n * n if type_ == 1 else m, dtype=CDT[prec][1], device=DEV)
        if params.kind == P.KIND_FRESNEL:
            P.nufresnel_execute(plan, type_, src, out)
        else:
            (P.nuasm1_execute if type_ == 1 else P.nuasm2_execute)(plan, src, out)
        torch.cuda.synchronize()
    finally:
        plan.destroy()


def random_points(rng, m, n, pitch):
    h = 0.5 * n * pitch * (1 - 1e-9)
    return rng.uniform(-h, h, m), rng.uniform(-h, h, m)


def cases():
    rng = np.random.default_rng(7)
    lam, z = 633e-9, 0.02
    for prec in ("f32", "f64"):
        for kind in ("asm", "fresnel"):
            for type_ in (1, 2):
                x, y = random_points(rng, 3000, 64, 10e-6)
                p = P.make_params(64, 10e-6, lam, z, kind=kind, prec=prec)
                yield f"{kind} type {type_} {prec} N 64", lambda p=p, x=x, y=y, t=type_, q=prec: solve(p, x, y, t, q, rng)
    for tile in (16, 32, 64):
        x, y = random_points(rng, 20000, 128, 8e-6)
        p = P.make_params(128, 8e-6, lam, z, tile=tile)
        yield f"type 1 f32 tile {tile}", lambda p=p, x=x, y=y: solve(p, x, y, 1, "f32", rng, w=np.ones(len(x)))
    x, y = random_points(rng, 5000, 64, 10e-6)
    for prec, tol in (("f32", 1e-6), ("f64", 1e-12)):
        p = P.make_params(64, 10e-6, lam, z, prec=prec, tol=tol, kernel="gaussian")
        for type_ in (1, 2):
            yield f"gaussian {prec} tol {tol} type {type_}", lambda p=p, t=type_, q=prec: solve(p, x, y, t, q, rng)

    def type3():
        p = P.make_params(64, 10e-6, lam, z)
        xs, ys = random_points(rng, 2000, 64, 10e-6)
        xd, yd = random_points(rng, 2500, 64, 10e-6)
        a, b = P.nuasm_plan(p, dev(xs), dev(ys)), P.nuasm_plan(p, dev(xd), dev(yd))
        try:
            out = torch.zeros(2500, dtype=torch.complex64, device=DEV)
            P.nuasm3_execute(a, b, values(rng, 2000, "f32"), out)
            torch.cuda.synchronize()
        finally:
            a.destroy()
            b.destroy()
    yield "type 3 f32 N 64", type3

    def lattice():
        p = P.make_params(128, 8e-6, lam, z)
        plan = P.nuasm_plan_lattice(p, 100, 90, 9e-6, -450e-6, -405e-6)
        try:
            out = torch.zeros(9000, dtype=torch.complex64, device=DEV)
            P.nuasm2_execute(plan, values(rng, 128 * 128, "f32"), out)
            torch.cuda.synchronize()
        finally:
            plan.destroy()
    yield "lattice type 2", lattice

    def batch():
        plans, items = [], []
        for k, (n, t) in enumerate(((256, 1), (512, 2), (128, 2))):
            x, y = random_points(rng, 40000, n, 8e-6)
            pl = P.nuasm_plan(P.make_params(n, 8e-6, lam, 0.01 * (k + 1)), dev(x), dev(y))
            plans.append(pl)
            inp = values(rng, len(x) if t == 1 else n * n, "f32")
            out = torch.zeros(n * n if t == 1 else len(x), dtype=torch.complex64, device=DEV)
            items.append((pl, t, inp, out))
        b = P.nuasm_batch_create(items)
        try:
            b.execute()
            torch.cuda.synchronize()
        finally:
            b.destroy()
            for pl in plans:
                pl.destroy()
    yield "batch of three planes", batch

    def noalloc():
        p = P.make_params(128, 8e-6, lam, z)
        x, y = random_points(rng, 30000, 128, 8e-6)
        out = torch.zeros(len(x), dtype=torch.complex64, device=DEV)
        P.nuasm2_solve_noalloc(p, dev(x), dev(y), values(rng, 128 * 128, "f32"), out)
        torch.cuda.synchronize()
    yield "no-allocation type 2", noalloc

    c2 = WL.nuasm2_graded(seed=1002, n=1024, pitch=8e-6)
    p2 = P.make_params(c2.n, c2.pitch, c2.lam, c2.z, ox=c2.ox, oy=c2.oy)
    for type_ in (2, 1):
        yield f"graded N 1024, 1M points, type {type_}", lambda t=type_: solve(p2, c2.x, c2.y, t, "f32", rng)
    c3 = WL.fresnel_clustered(1003, type_=2)
    for prec in ("f32", "f64"):
        p3 = P.make_params(c3.n, c3.pitch, c3.lam, c3.z, ox=c3.ox, oy=c3.oy, kind=c3.kind, prec=prec)
        for type_ in (1, 2):
            yield (f"clustered N 2048, 4M points, type {type_} {prec}",
                   lambda p=p3, t=type_, q=prec: solve(p, c3.x, c3.y, t, q, rng))


def main():
    if P.nuasm_debug_bounds() is None:
        raise SystemExit(f"{P.LIB_PATH} has no bounds checks (set NUASM_LIBRARY to the debug library)")
    out = []
    for name, run in cases():
        run()
        hits, site, index, limit = P.nuasm_debug_bounds(reset=True)
        out.append({"case": name, "hits": hits, "site": site, "index": index, "limit": limit})
    print(json.dumps(out))


if __name__ == "__main__":
    main()
