"""Autotuner: a tuned plan computes the same product (to the parity bounds)
and solves to the tolerance; the choice is reused from the cache; a plan
built from an explicit choice gives bitwise the tuned plan's results; and a
RHS is summed identically alone and in a batch on a tuned plan."""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_04710_gb300 import synth, ztoep

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def check_products(prob, plan, X):
    ref = oracle.matvec_blocks(prob, X)
    Xd = dev(X)
    y64 = plan.matvec(Xd, ztoep.ZTOEP_FP64).cpu().numpy()
    assert np.max(np.abs(y64 - ref)) <= 1e-12 * np.max(np.abs(ref))
    y32 = plan.matvec(Xd, ztoep.ZTOEP_MIXED).cpu().numpy()
    err = np.linalg.norm(y32 - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= 2e-6


@pytest.mark.parametrize("nrhs", [3, 20])
def test_autotuned_plan_parity_and_cache(nrhs):
    prob = synth.make_problem(10, 6, 24, 40, seed=8, rhs="planewave", nrhs=nrhs)
    plan = ztoep.Plan.from_problem(prob, autotune=nrhs)
    t = plan.tune
    assert t.candidates > 1 and t.nrhs == nrhs
    assert 0 < t.product_us <= t.default_us
    assert t.lx >= 19 and t.ly >= 11 and plan.info.lx == t.lx and plan.info.ly == t.ly
    X = np.concatenate([prob.V, synth.manufactured_solution(prob, 2, seed=4)])
    check_products(prob, plan, X)
    o = ztoep.ztoep_default_opts()
    o.tol = 1e-10
    Xs, info, st = plan.solve(dev(prob.V), opts=o)
    assert st == 0
    assert oracle.relres(prob, Xs.cpu().numpy(), prob.V).max() <= 1e-10
    # second call: from the cache, same choice
    plan2 = ztoep.Plan.from_problem(prob, autotune=nrhs)
    t2 = plan2.tune
    assert t2.candidates == 0
    for k in ("lx", "ly", "rad_order_x", "rad_order_y", "fft_channels_x", "fft_threads_x", "fft_channels_y",
              "fft_threads_y", "fft_kernel_x", "fft_kernel_y", "bp_split", "bp_ctas_per_sm", "tc_kchunk"):
        assert getattr(t2, k) == getattr(t, k), k
    # explicit choice: bitwise the same products and solution
    plan3 = ztoep.Plan.from_problem(prob, tune=t)
    Xd = dev(X)
    for prec in (ztoep.ZTOEP_FP64, ztoep.ZTOEP_MIXED):
        assert torch.equal(plan.matvec(Xd, prec), plan3.matvec(Xd, prec))
    Xs3, _, st3 = plan3.solve(dev(prob.V), opts=o)
    assert st3 == 0 and torch.equal(Xs, Xs3)
    got = ztoep.ztoep_plan_get_tune(plan3.handle)
    assert got.lx == t.lx and got.bp_split == t.bp_split
    for p in (plan, plan2, plan3):
        p.close()


def test_tuned_plan_batch_invariance():
    prob = synth.make_problem(7, 5, 16, 24, seed=21, rhs="planewave", nrhs=3)
    plan = ztoep.Plan.from_problem(prob, autotune=1)
    o = ztoep.ztoep_default_opts()
    o.tol = 1e-9
    Xb, _, st = plan.solve(dev(prob.V), opts=o)
    Xa, _, st1 = plan.solve(dev(prob.V[1:2]), opts=o)
    assert st == 0 and st1 == 0
    assert torch.equal(Xb[1:2], Xa)
    plan.close()


def test_bad_tune_rejected():
    prob = synth.make_problem(4, 4, 8, 8, seed=1)
    t = ztoep.TuneInfo()
    t.fft_threads_x = 100  # not a supported block size
    with pytest.raises(ztoep.ZtoepError):
        ztoep.Plan.from_problem(prob, tune=t)
    t = ztoep.TuneInfo()
    t.fft_kernel_y = 3  # no such kernel
    with pytest.raises(ztoep.ZtoepError):
        ztoep.Plan.from_problem(prob, tune=t)
    t = ztoep.TuneInfo()
    t.lx = 6  # below 2 nx - 1
    with pytest.raises(ztoep.ZtoepError):
        ztoep.Plan.from_problem(prob, tune=t)


# Embedding sizes with a register pass (every split P1 x P2 of the table's
# shapes: powers of two, 3, 5 and mixed factors, gcd 1..16 threads per line)
# and sizes without one (150, 160, 240: the shared-memory kernel serves both
# settings there).
REG_SIZES = [(4, 3, 8, 9), (5, 6, 10, 12), (8, 8, 15, 16), (9, 10, 18, 20), (12, 13, 24, 25), (14, 15, 27, 30),
             (16, 18, 32, 36), (20, 23, 40, 45), (24, 25, 48, 50), (27, 30, 54, 60), (32, 36, 64, 72),
             (38, 40, 75, 80), (41, 45, 81, 90), (48, 50, 96, 100), (60, 64, 120, 128), (68, 72, 135, 144),
             (75, 80, 150, 160), (120, 128, 240, 256)]


@pytest.mark.parametrize("nx,ny,lx,ly", REG_SIZES)
def test_register_passes_match_shared_memory_passes(nx, ny, lx, ly):
    """The register FFT passes (tune fft_kernel 2) and the shared-memory
    Stockham passes (fft_kernel 1) compute the same FP32 product to FP32
    rounding, and both match the FP64 oracle on sampled rows within the
    mixed-product bound; channel batches 2..64 of the register kernel agree."""
    b = 6 if lx * ly > 20000 else 10
    prob = synth.make_problem(nx, ny, b, 0, seed=nx + ny, rhs="planewave", nrhs=2)
    X = prob.V
    rows = np.unique(np.concatenate([np.arange(0, prob.n, max(1, prob.n // 64)), [prob.n - 1]]))
    ref = oracle.matvec_rows(prob, X, rows)
    outs = []
    for fk, ch in ((1, 0), (2, 0), (2, 2), (2, 8), (2, 64)):
        t = ztoep.TuneInfo()
        t.lx, t.ly = lx, ly
        t.fft_kernel_x = t.fft_kernel_y = fk
        t.fft_channels_x = t.fft_channels_y = ch
        plan = ztoep.Plan.from_problem(prob, tune=t)
        assert plan.info.lx == lx and plan.info.ly == ly
        y = plan.matvec(dev(X), ztoep.ZTOEP_MIXED).cpu().numpy()
        plan.close()
        err = np.linalg.norm(y[:, rows] - ref, axis=1) / np.linalg.norm(ref, axis=1)
        assert err.max() <= 2e-6, (fk, ch, err)
        outs.append(y)
    scale = np.max(np.abs(outs[0]))
    for y in outs[1:]:
        assert np.max(np.abs(y - outs[0])) <= 1e-5 * scale


def test_register_pass_masked_grid_and_edges():
    """Register passes on the gap grid (absent elements pass x through) with
    edge unknowns: parity with the oracle for both pass kernels."""
    prob = synth.make_problem(9, 5, 12, 20, seed=3, rhs="planewave", nrhs=3, gap_column=4)
    ref = oracle.matvec_blocks(prob, prob.V)
    for fk in (1, 2):
        t = ztoep.TuneInfo()
        t.fft_kernel_x = t.fft_kernel_y = fk
        plan = ztoep.Plan.from_problem(prob, tune=t)
        y = plan.matvec(dev(prob.V), ztoep.ZTOEP_MIXED).cpu().numpy()
        plan.close()
        err = np.linalg.norm(y - ref, axis=1) / np.linalg.norm(ref, axis=1)
        assert err.max() <= 2e-6, (fk, err)
