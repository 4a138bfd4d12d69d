"""GPU adjoint (md_adjoint, md_pair_hist, torch.autograd bridge) against the
FP64 oracle's adjoint and FP64 central finite differences.

The GPU path evaluates forces and Hessian-vector products in FP32 with an
FP64 adjoint state, so its gradients agree with the FP64 oracle to the FP32
level of the trajectory: tolerances here are relative to the vector norm
(||g_gpu - g_ref|| / ||g_ref||): 2e-4 against the oracle's adjoint of the
same loss gradient, 2e-3 against finite differences of the FP64 oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2406_04210_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ljmd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_04210_gb300 import build, ljmd as m
    build.build()
    m.load()
    return m


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def test_pair_hist_matches_oracle(ljmd):
    s = inputs.lj4000()
    b = ljmd.from_system(s, "mixed_ds")
    h, _ = b.pair_hist(64, 2.5, 2.5 / 64, 2.8)
    ho = oracle.hist(s.box, s.pos)
    assert np.abs(h[0] - ho).max() <= 1e-5 * ho.max()
    rng = np.random.default_rng(1)
    coef = rng.normal(size=64)
    _, g = b.pair_hist(64, 2.5, 2.5 / 64, 2.8, coef=coef)
    go = oracle.hist_grad(s.box, s.pos, coef)
    assert rel(g, go) <= 1e-4


@pytest.mark.parametrize("prec", ["mixed_ds", "fp64"])
@pytest.mark.parametrize("nsteps,ckpt", [(1, 1), (12, 4), (20, 20)])
def test_adjoint_matches_oracle_adjoint(ljmd, prec, nsteps, ckpt):
    s = inputs.fcc_system(6, seed=13)            # 864 particles, L = 10.1
    lj = oracle.LJ(s.eps, s.sigma, s.rcut)
    r = oracle.run(s.box, s.pos, s.vel, lj, s.skin, s.dt, nsteps, traj=True)
    rng = np.random.default_rng(nsteps)
    lx_T = rng.normal(size=s.pos.shape)
    lv_T = rng.normal(size=s.pos.shape)
    lx0, lv0, ge, gs = oracle.adjoint(s.box, r["traj"], lj, s.dt, lx_T, lv_T)
    b = ljmd.from_system(s, prec)
    b.integrate(s.dt, nsteps, thermo=False, ckpt_every=ckpt)
    gx0, gv0, gge, ggs = b.adjoint(lx_T, lv_T)
    assert rel(gx0, lx0) <= 2e-4
    assert rel(gv0, lv0) <= 2e-4
    assert abs(gge[0, 0] - ge[0, 0]) <= 2e-4 * abs(ge[0, 0])
    assert abs(ggs[0, 0] - gs[0, 0]) <= 2e-4 * abs(gs[0, 0])
    # the box is back at the end-of-run state
    p, v, _ = b.get_state()
    d = p - r["pos"]
    d -= s.box * np.rint(d / s.box)
    assert np.abs(d).max() < 1e-4


def test_adjoint_binary_mixture(ljmd):
    s = inputs.binary_random_system(n=1500, seed=23)
    lj = oracle.LJ(s.eps, s.sigma, s.rcut)
    s.pos, _, _ = oracle.fire(s.box, s.pos, lj, s.type, maxit=300, ftol=1e-2)
    r = oracle.run(s.box, s.pos, s.vel, lj, s.skin, s.dt, 8, type_=s.type, traj=True)
    rng = np.random.default_rng(3)
    lx_T = rng.normal(size=s.pos.shape)
    lv_T = rng.normal(size=s.pos.shape)
    lx0, lv0, ge, gs = oracle.adjoint(s.box, r["traj"], lj, s.dt, lx_T, lv_T, type_=s.type)
    b = ljmd.from_system(s, "mixed_ds")
    b.integrate(s.dt, 8, thermo=False, ckpt_every=4)
    gx0, gv0, gge, ggs = b.adjoint(lx_T, lv_T)
    assert rel(gx0, lx0) <= 5e-4
    assert rel(gv0, lv0) <= 5e-4
    assert rel(gge, ge) <= 5e-4 and rel(ggs, gs) <= 5e-4


def _oracle_loss(s, eps, sigma, x0, v0, nsteps, target, wv):
    lj = oracle.LJ([[eps]], [[sigma]], s.rcut)
    r = oracle.run(s.box, x0, v0, lj, s.skin, s.dt, nsteps)
    loss, _, _ = oracle.hist_loss(s.box, r["pos"], target)
    return loss + float(np.sum(wv * r["vel"]))


def test_gradients_match_fp64_finite_differences(ljmd):
    # the differentiable workload's loss on a small box: histogram of the
    # final frame against a target, plus a linear velocity term
    s = inputs.fcc_system(4, seed=21)            # 256 particles
    nsteps = 10
    rng = np.random.default_rng(6)
    target = oracle.hist(s.box, s.pos) * 0.9
    wv = 0.01 * rng.normal(size=s.pos.shape)
    b = ljmd.from_system(s, "mixed_ds")
    b.integrate(s.dt, nsteps, thermo=False, ckpt_every=5)
    h, _ = b.pair_hist(64, 2.5, 2.5 / 64, 2.8)
    coef = 2.0 * (h[0] - target) / 64
    _, lx_T = b.pair_hist(64, 2.5, 2.5 / 64, 2.8, coef=coef)
    gx0, gv0, ge, gs = b.adjoint(lx_T, wv)
    hstep = 1e-6
    u = rng.normal(size=s.pos.shape)
    fd = (_oracle_loss(s, 1.0, 1.0, s.pos + hstep * u, s.vel, nsteps, target, wv)
          - _oracle_loss(s, 1.0, 1.0, s.pos - hstep * u, s.vel, nsteps, target, wv)) / (2 * hstep)
    assert np.sum(gx0 * u) == pytest.approx(fd, rel=2e-3)
    fd = (_oracle_loss(s, 1.0 + hstep, 1.0, s.pos, s.vel, nsteps, target, wv)
          - _oracle_loss(s, 1.0 - hstep, 1.0, s.pos, s.vel, nsteps, target, wv)) / (2 * hstep)
    assert ge[0, 0] == pytest.approx(fd, rel=2e-3)
    fd = (_oracle_loss(s, 1.0, 1.0 + hstep, s.pos, s.vel, nsteps, target, wv)
          - _oracle_loss(s, 1.0, 1.0 - hstep, s.pos, s.vel, nsteps, target, wv)) / (2 * hstep)
    assert gs[0, 0] == pytest.approx(fd, rel=2e-3)


def test_autograd_bridge(ljmd):
    import torch
    s = inputs.fcc_system(4, seed=21)
    nsteps = 10
    target = torch.tensor(oracle.hist(s.box, s.pos) * 0.9)
    x0 = torch.tensor(s.pos, device="cuda", requires_grad=True)
    v0 = torch.tensor(s.vel, device="cuda", requires_grad=True)
    eps = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    sigma = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    b = ljmd.from_system(s, "mixed_ds")
    xT, vT = ljmd.TrajectoryFn.apply(x0, v0, eps, sigma, b, s.dt, nsteps, 5)
    loss = ljmd.PairHistLossFn.apply(xT, b, target, 64, 2.5, 2.5 / 64, 2.8)
    loss.backward()
    # same gradients through the C ABI directly
    c = ljmd.from_system(s, "mixed_ds")
    c.integrate(s.dt, nsteps, thermo=False, ckpt_every=5)
    h, _ = c.pair_hist(64, 2.5, 2.5 / 64, 2.8)
    coef = 2.0 * (h[0] - target.numpy()) / 64
    _, lx_T = c.pair_hist(64, 2.5, 2.5 / 64, 2.8, coef=coef)
    gx0, gv0, ge, gs = c.adjoint(lx_T, np.zeros_like(lx_T))
    assert rel(x0.grad.cpu().numpy(), gx0) <= 1e-6
    assert rel(v0.grad.cpu().numpy(), gv0) <= 1e-6
    assert float(eps.grad) == pytest.approx(ge[0, 0], rel=1e-6)
    assert float(sigma.grad) == pytest.approx(gs[0, 0], rel=1e-6)


def test_adjoint_requires_record(ljmd):
    s = inputs.fcc_system(4, seed=2)
    b = ljmd.from_system(s, "mixed_ds")
    b.integrate(s.dt, 5, thermo=False)
    with pytest.raises(ljmd.MDError) as ei:
        b.adjoint(np.zeros((s.n, 3)), np.zeros((s.n, 3)))
    assert ei.value.status == 8


def test_autograd_backward_refuses_a_replaced_record(ljmd):
    # two forwards on one box, then the first one's backward: the box holds
    # only the second record, so the backward must fail rather than return
    # the second run's gradients; the loss also refuses positions that are
    # not the box's current state
    import torch
    s = inputs.fcc_system(4, seed=21)
    b = ljmd.from_system(s, "mixed_ds")
    target = torch.tensor(oracle.hist(s.box, s.pos) * 0.9)
    x0 = torch.tensor(s.pos, device="cuda", requires_grad=True)
    v0 = torch.tensor(s.vel, device="cuda", requires_grad=True)
    eps = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    sigma = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    xa, va = ljmd.TrajectoryFn.apply(x0, v0, eps, sigma, b, s.dt, 10, 5)
    rec_a = b.info().record_id
    assert rec_a > 0
    xb, vb = ljmd.TrajectoryFn.apply(x0, v0, eps, sigma, b, s.dt, 20, 5)
    assert b.info().record_id > rec_a
    with pytest.raises(ValueError):
        ljmd.PairHistLossFn.apply(xa, b, target, 64, 2.5, 2.5 / 64, 2.8)
    with pytest.raises(ljmd.MDError) as ei:
        (xa * xa).sum().backward()
    assert ei.value.status == 8
    loss = ljmd.PairHistLossFn.apply(xb, b, target, 64, 2.5, 2.5 / 64, 2.8)
    loss.backward()
    assert torch.isfinite(x0.grad).all()
    b.set_state(s.pos, s.vel)
    assert b.info().record_id == 0
