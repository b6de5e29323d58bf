"""Port matrices (Sec. IV-B) on the GPU through the C-ABI: the admittance
Y = L I^ L and the power-wave scattering matrix against the oracle, from
random currents (exact gather, FP64 elimination vs the oracle's inverse) and
from delta-port solves of small arrays (error bounded by the solve
tolerance), plus the error statuses."""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_04710_gb300 import synth, ztoep

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("p,n", [(1, 7), (5, 40), (33, 500), (160, 2000)])
def test_port_matrices_match_oracle_on_random_currents(p, n):
    rng = np.random.default_rng(p)
    I = rng.standard_normal((p, n)) + 1j * rng.standard_normal((p, n))
    ports = rng.choice(n, size=p, replace=False)
    lens = rng.uniform(0.2, 2.0, p)
    z0 = rng.uniform(20.0, 100.0, p)
    Y, S = ztoep.port_matrices(dev(I), ports, lens, z0)
    Yr = oracle.port_admittance(I, ports, lens)
    assert rel(Y.cpu().numpy(), Yr) <= 1e-15
    Sr = oracle.scattering(Yr, z0)
    assert rel(S.cpu().numpy(), Sr) <= 1e-10


def delta_ports(prob):
    """Unknown index of each active element's basis function 0 (the port of
    the ports excitation), in element order."""
    act = np.flatnonzero(prob.active.reshape(-1))
    return act * prob.b


@pytest.mark.parametrize("gap", [False, True])
def test_port_matrices_after_delta_port_solve(gap):
    prob = synth.make_problem(7 if gap else 6, 5, 8, 20, seed=9, rhs="ports",
                              gap_column=3 if gap else None, edge_layout="split" if gap else "one")
    ports = delta_ports(prob)
    assert prob.V.shape[0] == len(ports)
    assert np.all(prob.V[np.arange(len(ports)), ports] == 1.0)
    plan = ztoep.Plan.from_problem(prob)
    o = ztoep.ztoep_default_opts()
    o.prec = ztoep.ZTOEP_FP64
    o.tol = 1e-13
    Xs, info, st = plan.solve(dev(prob.V), opts=o)
    assert st == 0
    lens = np.linspace(0.4, 0.6, len(ports))
    z0 = np.full(len(ports), 50.0)
    Y, S = ztoep.port_matrices(Xs, ports, lens, z0)
    Z = oracle.assemble(prob)
    Iref = np.linalg.solve(Z, prob.V.T).T
    Yr = oracle.port_admittance(Iref, ports, lens)
    Sr = oracle.scattering(Yr, z0)
    Yg, Sg = Y.cpu().numpy(), S.cpu().numpy()
    assert rel(Yg, Yr) <= 1e-9
    assert rel(Sg, Sr) <= 1e-8
    assert rel(Yg, Yg.T) <= 1e-9  # reciprocity (Z^T = Z)
    plan.close()


def test_port_matrices_statuses():
    I = dev(np.ones((3, 10), complex))
    Y = torch.empty((3, 3), dtype=torch.complex128, device="cuda")
    S = torch.empty_like(Y)
    ok = dict(ports=np.array([0, 4, 9]), edge_len=np.ones(3), z0=np.full(3, 50.0))
    bad = [dict(ok, ports=np.array([0, 4, 10])), dict(ok, edge_len=np.array([1.0, 0.0, 1.0])),
           dict(ok, z0=np.array([50.0, -1.0, 50.0]))]
    for kw in bad:
        assert ztoep.ztoep_port_matrices(3, 10, I, kw["ports"], kw["edge_len"], kw["z0"], Y, S) == ztoep.ZTOEP_ERR_ARG
    assert ztoep.ztoep_port_matrices(3, 10, I, ok["ports"], ok["edge_len"], ok["z0"], Y, Y) == ztoep.ZTOEP_ERR_ARG
    # I + G Y exactly singular: one port with y = -1/z0 (z0 = 0.5, y = -2)
    Ising = dev(np.full((1, 4), -2.0 + 0j))
    Y1 = torch.empty((1, 1), dtype=torch.complex128, device="cuda")
    S1 = torch.empty_like(Y1)
    st = ztoep.ztoep_port_matrices(1, 4, Ising, np.array([2]), np.ones(1), np.full(1, 0.5), Y1, S1)
    assert st == ztoep.ZTOEP_ERR_NONFINITE
