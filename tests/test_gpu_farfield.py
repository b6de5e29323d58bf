"""Far field on the array-factor grid (Eqs. farfieldBasis / tensorProd) on
the GPU through the C-ABI, against the oracle's direct summation over the
parts at the same directions (FP64), including masked elements, edge
unknowns present in the vector (not part of the element component) and an
explicit embedding size."""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_04710_gb300 import synth, ztoep

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("nx,ny,b,E,gap,lx,nrhs,npol", [
    (4, 3, 5, 12, None, 0, 1, 2),
    (7, 5, 12, 20, 3, 0, 3, 2),
    (6, 6, 8, 24, None, 16, 2, 3),
    (1, 1, 4, 4, None, 0, 1, 1),
])
def test_far_field_grid_matches_direct_sum(nx, ny, b, E, gap, lx, nrhs, npol):
    prob = synth.make_problem(nx, ny, b, E, seed=nx * 7 + ny, rhs="planewave", nrhs=nrhs, gap_column=gap,
                              edge_layout="split" if gap is not None else "one")
    plan = ztoep.Plan.from_problem(prob, lx=lx)
    Lx, Ly = plan.info.lx, plan.info.ly
    rng = np.random.default_rng(nx)
    I = rng.standard_normal((nrhs, prob.n)) + 1j * rng.standard_normal((nrhs, prob.n))
    uv = synth.grid_directions(Lx, Ly)
    Fh = synth.far_field_basis(prob, uv, npol)
    F = plan.far_field(dev(I), dev(Fh), synth.K0, 376.73).cpu().numpy()
    ref = oracle.far_field(prob, I[:, :prob.n_toep], uv, Fh, synth.K0, 376.73)
    assert F.shape == ref.shape
    assert np.max(np.abs(F - ref)) <= 1e-12 * np.max(np.abs(ref))
    plan.close()


def test_far_field_of_a_solution():
    """The far field of a mixed-precision solution equals the oracle's far field
    of the same solution vector (the contraction adds no error of its own)."""
    prob = synth.make_problem(8, 8, 16, 32, seed=2, rhs="planewave", nrhs=2)
    plan = ztoep.Plan.from_problem(prob)
    o = ztoep.ztoep_default_opts()
    o.tol = 1e-8
    X, _, st = plan.solve(dev(prob.V), opts=o)
    assert st == 0
    uv = synth.grid_directions(plan.info.lx, plan.info.ly)
    Fh = synth.far_field_basis(prob, uv)
    F = plan.far_field(X, dev(Fh), synth.K0, 376.73).cpu().numpy()
    ref = oracle.far_field(prob, X.cpu().numpy()[:, :prob.n_toep], uv, Fh, synth.K0, 376.73)
    assert np.max(np.abs(F - ref)) <= 1e-12 * np.max(np.abs(ref))
    plan.close()


def test_far_field_bad_arguments():
    prob = synth.make_problem(3, 3, 4, 0, seed=1)
    plan = ztoep.Plan.from_problem(prob)
    I = dev(prob.V)
    Fh = torch.zeros((plan.info.lx * plan.info.ly, 2, 4), dtype=torch.complex128, device="cuda")
    F = torch.empty((1, plan.info.lx * plan.info.ly, 2), dtype=torch.complex128, device="cuda")
    assert ztoep.ztoep_far_field_grid(plan.handle, 1, I, 0, Fh, 1.0, 1.0, F) == ztoep.ZTOEP_ERR_ARG
    assert ztoep.ztoep_far_field_grid(plan.handle, 0, I, 2, Fh, 1.0, 1.0, F) == ztoep.ZTOEP_ERR_ARG
    assert ztoep.ztoep_far_field_grid(plan.handle, 1, I, 2, Fh, float("nan"), 1.0, F) == ztoep.ZTOEP_ERR_ARG
    assert ztoep.ztoep_far_field_grid(plan.handle, 1, I, 2, Fh, 1.0, 1.0, F) == 0
    plan.close()
