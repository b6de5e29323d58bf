"""Level-1 solve by the Schur complement (Sec. II-D, Eqs. solveEqSystem1/2)
through the C-ABI: the batched GMRES with a plan of A alone, the FP64
contractions and the Gauss-Jordan solve of S give the solution of the whole
system (against the oracle's LU and its own Schur solve), in both precisions
of the A-solves, with a gap grid and with nonzero edge rows in V."""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_04710_gb300 import synth, ztoep

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def plan_of_A(prob):
    act = prob.active if not prob.active.all() else None
    return ztoep.Plan(prob.nx, prob.ny, prob.b, 0, dev(prob.T), None, None, act)


@pytest.mark.parametrize("shape", ["6x5_b8_e20", "7x5_gap_b6_e24", "10x8_b4_e280"])
@pytest.mark.parametrize("prec", [ztoep.ZTOEP_FP64, ztoep.ZTOEP_MIXED])
def test_schur_solve_matches_lu(shape, prec):
    if shape == "6x5_b8_e20":
        prob = synth.make_problem(6, 5, 8, 20, seed=3, rhs="planewave", nrhs=3)
    elif shape == "7x5_gap_b6_e24":
        prob = synth.make_problem(7, 5, 6, 24, seed=4, rhs="planewave", nrhs=2, gap_column=3, edge_layout="split")
    else:  # more edge unknowns than one 256-RHS chunk of A-solves
        prob = synth.make_problem(10, 8, 4, 280, seed=8, rhs="planewave", nrhs=2)
    pa = plan_of_A(prob)
    o = ztoep.ztoep_default_opts()
    o.prec = prec
    o.tol = 1e-12 if prec == ztoep.ZTOEP_FP64 else 1e-10
    X = torch.empty((prob.V.shape[0], prob.n), dtype=torch.complex128, device="cuda")
    info = ztoep.info_array(prob.V.shape[0])
    st = ztoep.ztoep_solve_schur(pa.handle, prob.n_edge, dev(prob.B), dev(prob.C), o, prob.V.shape[0],
                                 dev(prob.V), X, info)
    assert st == 0
    Xg = X.cpu().numpy()
    Z = oracle.assemble(prob)
    xref = oracle.LU(Z).solve(prob.V)
    res = oracle.relres(Z, Xg, prob.V)
    assert res.max() <= (1e-10 if prec == ztoep.ZTOEP_FP64 else 1e-8), res
    err = np.linalg.norm(Xg - xref, axis=1) / np.linalg.norm(xref, axis=1)
    assert err.max() <= (1e-9 if prec == ztoep.ZTOEP_FP64 else 1e-7), err
    mask = oracle.unknown_mask(prob)  # absent elements: identity rows, x = v there
    tol_id = 1e-12 if prec == ztoep.ZTOEP_FP64 else 1e-8
    assert np.max(np.abs(Xg[:, mask == 0] - prob.V[:, mask == 0]), initial=0.0) <= tol_id * np.max(np.abs(prob.V))
    pa.close()


def test_schur_solve_against_oracle_schur_with_edge_rhs():
    """V with nonzero edge rows (the paper's outer step has V_E = 0; the
    general form adds V_E - B U): against the oracle's Schur solve."""
    prob = synth.make_problem(4, 4, 6, 16, seed=2, rhs="planewave", nrhs=2)
    nt = prob.n_toep
    Z = oracle.assemble(prob)
    A = Z[:nt, :nt]
    xs = oracle.schur_solve(A, prob.B, prob.C, prob.V)
    pa = plan_of_A(prob)
    o = ztoep.ztoep_default_opts()
    o.prec = ztoep.ZTOEP_FP64
    o.tol = 1e-13
    X = torch.empty((2, prob.n), dtype=torch.complex128, device="cuda")
    assert ztoep.ztoep_solve_schur(pa.handle, prob.n_edge, dev(prob.B), dev(prob.C), o, 2, dev(prob.V), X) == 0
    Xg = X.cpu().numpy()
    assert np.max(np.abs(Xg - xs)) <= 1e-9 * np.max(np.abs(xs))
    pa.close()


def test_schur_solve_bad_arguments():
    prob = synth.make_problem(3, 3, 4, 8, seed=1)
    full = ztoep.Plan.from_problem(prob)
    pa = plan_of_A(prob)
    o = ztoep.ztoep_default_opts()
    V = dev(prob.V)
    X = torch.empty_like(V)
    B, C = dev(prob.B), dev(prob.C)
    assert ztoep.ztoep_solve_schur(full.handle, 8, B, C, o, 1, V, X) == ztoep.ZTOEP_ERR_ARG  # plan has edges
    assert ztoep.ztoep_solve_schur(pa.handle, 0, B, C, o, 1, V, X) == ztoep.ZTOEP_ERR_ARG
    assert ztoep.ztoep_solve_schur(pa.handle, 8, B, C, o, 1, V, V) == ztoep.ZTOEP_ERR_ARG
    full.close()
    pa.close()
