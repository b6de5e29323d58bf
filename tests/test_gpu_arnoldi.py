"""Arnoldi steps that take the second Gram-Schmidt pass: a system close to the
identity makes every new vector nearly dependent on the basis.  A RHS alone
and in a batch must get bitwise the same solution (the same chunk rows,
reduction tree and second-pass decision), the count of second passes is
reported per RHS, and the solution matches the oracle's LU; the host-driven
loop matches the graph."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
from paper_2506_04710_gb300 import synth, ztoep

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def opts(prec, tol):
    o = ztoep.ztoep_default_opts()
    o.prec, o.tol = prec, tol
    return o


def near_identity(nx, ny, b, n_edge, eps, seed, nrhs):
    """Z = I + eps (couplings of a synthetic array): a new Arnoldi vector is
    w = v + O(eps), almost in the span, so every step takes the second pass."""
    p = synth.make_problem(nx, ny, b, n_edge, seed=seed, rhs="planewave", nrhs=nrhs)
    T = p.T * eps
    T[ny - 1, nx - 1] += np.eye(b)
    C = p.C * eps + np.eye(n_edge)
    return dataclasses.replace(p, T=T, B=p.B * eps, C=C)


@pytest.mark.parametrize("prec", [ztoep.ZTOEP_MIXED, ztoep.ZTOEP_FP64])
def test_second_pass_alone_equals_batch(prec):
    prob = near_identity(6, 5, 8, 20, 1e-3, seed=41, nrhs=12)
    plan = ztoep.Plan.from_problem(prob)
    V = dev(prob.V)
    Xb, infob, st = plan.solve(V, opts=opts(prec, 1e-11))
    assert st == 0
    for r in (0, 5, 11):
        Xa, infoa, sta = plan.solve(V[r:r + 1].contiguous(), opts=opts(prec, 1e-11))
        assert sta == 0
        assert infoa[0]["second_passes"] > 0
        assert infoa[0]["second_passes"] == infob[r]["second_passes"]
        assert torch.equal(Xa[0], Xb[r]), r
    Z = oracle.assemble(prob)
    xref = oracle.LU(Z).solve(prob.V)
    Xh = Xb.cpu().numpy()
    assert oracle.relres(Z, Xh, prob.V).max() <= 1e-11
    err = np.linalg.norm(Xh - xref, axis=1) / np.linalg.norm(xref, axis=1)
    assert err.max() <= 1e-10
    plan.close()


def test_host_loop_matches_graph():
    prob = synth.make_problem(8, 6, 16, 28, seed=43, rhs="planewave", nrhs=2)
    plan = ztoep.Plan.from_problem(prob)
    V = dev(prob.V)
    o = opts(ztoep.ZTOEP_MIXED, 1e-10)
    Xg, ig, st = plan.solve(V, opts=o)
    o2 = opts(ztoep.ZTOEP_MIXED, 1e-10)
    o2.flags = ztoep.ZTOEP_FLAG_HOST_LOOP
    Xh, ih, st2 = plan.solve(V, opts=o2)
    assert st == 0 and st2 == 0
    assert torch.equal(Xg, Xh)
    assert [(i["inner_iters"], i["outer"]) for i in ig] == [(i["inner_iters"], i["outer"]) for i in ih]
    plan.close()
