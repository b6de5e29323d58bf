"""One solve over several systems of different sizes (ztoep_solve_group):
every Arnoldi, residual and update step is one launch over all members' RHS,
the members' products run concurrently, and each member must get exactly the
result it gets alone (bitwise: the per-RHS arithmetic is the same), in both
precisions, through the graph and the host-driven loop; the results are also
checked against the oracle (true residual from its dense product, solution
against its LU at 1e-11)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_04710_gb300 import synth, ztoep

pytestmark = pytest.mark.gpu

MEMBERS = [
    dict(nx=6, ny=5, b=16, n_edge=22, rhs="planewave", nrhs=3, seed=21),
    dict(nx=9, ny=4, b=40, n_edge=24, rhs="planewave", nrhs=1, seed=22),
    dict(nx=4, ny=4, b=8, n_edge=16, rhs="ones", nrhs=2, seed=23),
    dict(nx=5, ny=3, b=3, n_edge=10, gap_column=2, edge_layout="split", rhs="ports", seed=24),
    dict(nx=7, ny=7, b=24, n_edge=0, rhs="planewave", nrhs=5, seed=25),
]


def opts(prec, tol=1e-8, flags=0):
    o = ztoep.ztoep_default_opts()
    o.prec, o.tol = prec, tol
    o.flags = ztoep.ZTOEP_FLAG_ZERO_GUESS | flags
    return o


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def members():
    probs = [synth.make_problem(**kw) for kw in MEMBERS]
    plans = [ztoep.Plan.from_problem(p) for p in probs]
    yield probs, plans
    for pl in plans:
        pl.close()


def solve_alone(plan, prob, o):
    V = dev(prob.V)
    X = torch.zeros_like(V)
    info = ztoep.info_array(prob.nrhs)
    st = ztoep.ztoep_solve(plan.handle, o, prob.nrhs, V, X, info)
    torch.cuda.synchronize()
    return st, X.cpu(), [(i.inner_iters, i.outer, i.rel_residual) for i in info]


def solve_group(plans, probs, o):
    V = [dev(p.V) for p in probs]
    X = [torch.zeros_like(v) for v in V]
    infos = [ztoep.info_array(p.nrhs) for p in probs]
    st = ztoep.ztoep_solve_group([pl.handle for pl in plans], o, V, X, infos)
    torch.cuda.synchronize()
    return st, [x.cpu() for x in X], [[(i.inner_iters, i.outer, i.rel_residual) for i in inf] for inf in infos]


@pytest.mark.parametrize("prec", [ztoep.ZTOEP_MIXED, ztoep.ZTOEP_FP64])
def test_group_equals_alone_bitwise(members, prec):
    probs, plans = members
    o = opts(prec)
    st, Xg, infog = solve_group(plans, probs, o)
    assert st == ztoep.ZTOEP_OK
    for pl, p, Xi, ii in zip(plans, probs, Xg, infog):
        sta, Xa, infoa = solve_alone(pl, p, opts(prec))
        assert sta == ztoep.ZTOEP_OK
        assert torch.equal(Xi, Xa)
        assert ii == infoa


def test_group_host_loop_matches_graph(members):
    probs, plans = members
    st, Xg, infog = solve_group(plans, probs, opts(ztoep.ZTOEP_MIXED))
    sth, Xh, infoh = solve_group(plans, probs, opts(ztoep.ZTOEP_MIXED, flags=ztoep.ZTOEP_FLAG_HOST_LOOP))
    assert st == sth == ztoep.ZTOEP_OK
    for a, b in zip(Xg, Xh):
        assert torch.equal(a, b)
    assert infog == infoh


def test_group_against_oracle(members):
    probs, plans = members
    st, Xg, _ = solve_group(plans, probs, opts(ztoep.ZTOEP_MIXED, tol=1e-11))
    assert st == ztoep.ZTOEP_OK
    for p, X in zip(probs, Xg):
        Z = oracle.assemble(p)
        Xh = X.numpy()
        assert oracle.relres(Z, Xh, p.V).max() <= 1e-11
        xref = oracle.LU(Z).solve(p.V)
        err = np.linalg.norm(Xh - xref, axis=1) / np.linalg.norm(xref, axis=1)
        assert err.max() <= 1e-7
        mask = oracle.unknown_mask(p)
        assert np.all(Xh[:, mask == 0] == 0)


def test_group_with_tensor_core_member(members):
    """A member with 24 RHS (tensor-core products) beside small ones."""
    probs, plans = members
    big = synth.make_problem(8, 6, 32, 28, seed=26, rhs="planewave", nrhs=24)
    pb = ztoep.Plan.from_problem(big)
    try:
        st, Xg, infog = solve_group([pb, plans[0], plans[2]], [big, probs[0], probs[2]], opts(ztoep.ZTOEP_MIXED))
        assert st == ztoep.ZTOEP_OK
        sta, Xa, infoa = solve_alone(pb, big, opts(ztoep.ZTOEP_MIXED))
        assert torch.equal(Xg[0], Xa) and infog[0] == infoa
    finally:
        pb.close()


def test_group_rejects_bad_arguments(members):
    probs, plans = members
    o = opts(ztoep.ZTOEP_MIXED)
    V = [dev(p.V) for p in probs[:2]]
    X = [torch.zeros_like(v) for v in V]
    h = [pl.handle for pl in plans[:2]]
    assert ztoep.ztoep_solve_group([h[0], h[0]], o, V, X) == ztoep.ZTOEP_ERR_ARG  # one plan twice
    assert ztoep.ztoep_solve_group([h[0], h[1]], o, [V[0], V[1]], [V[0], X[1]]) == ztoep.ZTOEP_ERR_ARG  # V == X
    many = [h[0]] * 9
    assert ztoep.ztoep_solve_group(many, o, [V[0]] * 9, [X[0]] * 9) == ztoep.ZTOEP_ERR_ARG
    assert ztoep.ztoep_solve_group([], o, [], []) == ztoep.ZTOEP_ERR_ARG
