"""Serving: requests of different sizes and RHS counts run concurrently
through the scheduler; each result must be the same as the one of the same
request solved alone (bitwise: the scheduler runs exactly the same kernels),
resident plans are reused under their key, and device-side inputs work.
Requests shaped like the large ones of the serving stream (b = 96 with 64 RHS,
a 32x32 b64 array with 40 RHS, perimeter edge layout through the side spectra)
are checked against the oracle: residual components on sampled rows from its
direct product (|r_k| <= tol ||v|| follows from ||r|| <= tol ||v||), and a
small request solved to 1e-11 against its LU solution."""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_04710_gb300 import synth, ztoep

pytestmark = pytest.mark.gpu

MIX = [(6, 16, 24, 3, 1), (8, 32, 32, 20, 2), (5, 8, 0, 1, 3), (10, 16, 40, 7, 4), (7, 24, 28, 16, 5),
       (4, 8, 16, 2, 6), (9, 12, 36, 5, 7), (6, 16, 24, 17, 8)]


def opts():
    o = ztoep.ztoep_default_opts()
    o.tol = 1e-8
    return o


def alone(prob):
    plan = ztoep.Plan.from_problem(prob)
    X, info, st = plan.solve(torch.from_numpy(prob.V.copy()).cuda(), opts=opts())
    plan.close()
    return X.cpu(), info


def test_mix_equals_alone_and_runs_concurrently():
    probs = [synth.make_problem(nx, nx, b, e, seed=sd, rhs="planewave", nrhs=r) for nx, b, e, r, sd in MIX]
    s = ztoep.Scheduler(hbm_budget=16 << 30, workers=3)
    outs, ids = [], []
    for p in probs:
        X = torch.zeros((p.nrhs, p.n), dtype=torch.complex128).pin_memory()
        Vh = torch.from_numpy(p.V.copy()).pin_memory()
        ids.append(s.submit((p.nx, p.ny, p.b, p.n_edge), p.T, p.B if p.n_edge else None,
                            p.C if p.n_edge else None, Vh, X, opts=opts(), on_device=False))
        outs.append(X)
    for rid, p, X in zip(ids, probs, outs):
        rc, st, info = s.wait(rid, 120000)
        assert rc == 0 and st.status == 0
        assert max(i["rel_residual"] for i in info) <= 1e-8
        Xa, _ = alone(p)
        assert torch.equal(X, Xa)
    assert s.stats().max_in_flight >= 2
    s.close()


def test_resident_plan_reused_under_key():
    p = synth.make_problem(8, 8, 16, 32, seed=12, rhs="planewave", nrhs=4)
    s = ztoep.Scheduler(hbm_budget=8 << 30, workers=2)
    res = []
    for k in range(3):
        V = torch.from_numpy(p.V[k:k + 2].copy()).pin_memory() if k < 2 else torch.from_numpy(p.V.copy()).pin_memory()
        X = torch.zeros_like(V).pin_memory()
        rid = s.submit((8, 8, 16, 32), p.T, p.B, p.C, V, X, opts=opts(), plan_key=777, on_device=False)
        rc, st, info = s.wait(rid, 120000)
        assert rc == 0 and st.status == 0
        res.append((st.plan_reused, X))
    assert [r[0] for r in res] == [0, 1, 1]
    Xa, _ = alone(p)
    assert torch.equal(res[2][1], Xa)
    st = s.stats()
    assert st.plans_built == 1 and st.plans_reused == 2 and st.resident_plan_bytes > 0
    s.close()


def test_device_side_inputs():
    d = synth.make_problem_device(8, 8, 32, 128, seed=5, nrhs=18)
    X = torch.zeros_like(d["V"])
    s = ztoep.Scheduler(hbm_budget=8 << 30, workers=1)
    rid = s.submit((8, 8, 32, 128), d["T"], d["B"], d["C"], d["V"], X, opts=opts(), on_device=True)
    rc, st, info = s.wait(rid, 120000)
    assert rc == 0 and st.status == 0 and max(i["rel_residual"] for i in info) <= 1e-8
    # the device generator follows the host recipe to rounding
    ph = synth.make_problem(8, 8, 32, 128, seed=5, rhs="planewave", nrhs=18)
    assert np.max(np.abs(d["T"].cpu().numpy() - ph.T)) <= 1e-12 * np.max(np.abs(ph.T))
    assert np.max(np.abs(d["B"].cpu().numpy() - ph.B)) <= 1e-12 * np.max(np.abs(ph.B))
    assert np.max(np.abs(d["V"].cpu().numpy() - ph.V)) <= 1e-12
    s.close()


def sample_rows(prob, count, seed=9):
    rng = np.random.default_rng(seed)
    rows = rng.choice(prob.n, size=min(count, prob.n), replace=False)
    edge = np.arange(prob.n_toep, prob.n)[:: max(1, prob.n_edge // 16)]
    return np.unique(np.concatenate([rows, edge, [0, prob.n_toep - 1, prob.n - 1]]))


def test_stream_shaped_requests_against_oracle():
    # (nx, b, nrhs, design seed, tol): E = 16 nx, 4 edge unknowns per cell side
    shapes = [(24, 96, 64, 1001, 1e-8), (32, 64, 40, 1002, 1e-8), (6, 32, 5, 1003, 1e-11)]
    probs = [synth.make_problem(nx, nx, b, 16 * nx, seed=sd, rhs="planewave", nrhs=r) for nx, b, r, sd, _ in shapes]
    assert all(p.edge_per_cell == 4 for p in probs)
    s = ztoep.Scheduler(hbm_budget=48 << 30, workers=3)
    subs = []
    for p, (nx, b, r, sd, tol) in zip(probs, shapes):
        o = opts()
        o.tol = tol
        T, B, C, V = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (p.T, p.B, p.C, p.V))
        X = torch.zeros_like(V)
        rid = s.submit((nx, nx, b, p.n_edge, None, 0, 0, 4), T, B, C, V, X, opts=o, on_device=True)
        subs.append((rid, p, o, X))
    for rid, p, o, X in subs:
        rc, st, info = s.wait(rid, 300000)
        assert rc == 0 and st.status == 0
        Xh = X.cpu().numpy()
        assert max(i["rel_residual"] for i in info) <= o.tol
        rows = sample_rows(p, 160)
        r = p.V[:, rows] - oracle.matvec_rows(p, Xh, rows)
        vn = np.linalg.norm(p.V, axis=1)
        assert np.all(np.abs(r) <= o.tol * vn[:, None])
        # the same request alone on the same layout: bitwise the same result
        plan = ztoep.Plan.from_problem(p, structured=True)
        Xa, _, sta = plan.solve(torch.from_numpy(p.V.copy()).cuda(), opts=o)
        plan.close()
        assert sta == 0 and torch.equal(X.cpu(), Xa.cpu())
        if p.n <= 4096:  # small request: the solution against the oracle's LU
            Z = oracle.assemble(p)
            xref = oracle.LU(Z).solve(p.V)
            err = np.linalg.norm(Xh - xref, axis=1) / np.linalg.norm(xref, axis=1)
            assert err.max() <= 1e-7
            assert oracle.relres(Z, Xh, p.V).max() <= o.tol
    assert s.stats().max_in_flight >= 2
    s.close()


def test_grouped_solves_equal_alone():
    """group_max = 4, one worker: consecutive compatible requests (device
    inputs, sizes within a factor 4) run as grouped solves; each result is
    bitwise the one of the request solved alone."""
    shapes = [(6, 16, 24, 3, 31), (7, 16, 28, 2, 32), (6, 24, 24, 4, 33), (5, 16, 20, 3, 34), (8, 12, 32, 2, 35)]
    probs = [synth.make_problem(nx, nx, b, e, seed=sd, rhs="planewave", nrhs=r) for nx, b, e, r, sd in shapes]
    s = ztoep.Scheduler(hbm_budget=16 << 30, workers=1, group_max=4)
    subs = []
    for p in probs:
        T, B, C, V = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (p.T, p.B, p.C, p.V))
        X = torch.zeros_like(V)
        subs.append((s.submit((p.nx, p.ny, p.b, p.n_edge), T, B, C, V, X, opts=opts(), on_device=True), p, X))
    for rid, p, X in subs:
        rc, st, info = s.wait(rid, 120000)
        assert rc == 0 and st.status == 0
        assert max(i["rel_residual"] for i in info) <= 1e-8
        Xa, _ = alone(p)
        assert torch.equal(X.cpu(), Xa)
    assert s.stats().groups >= 1
    s.close()
