"""GPU parity at the full sizes of the five workloads, in the launch
configuration bench.py times (autotuned).  Where the FP64 oracle cannot
finish in seconds, sampled outputs are computed one by one (each sampled
particle's neighbourhood as a small system in the same periodic box), or a
property that holds at any size is checked.
"""
import numpy as np
import pytest

import oracle
from forcecheck import figures, pair_scale, report
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


def neighbourhood(box, pos, i, radius, tree):
    """Indices of every particle within `radius` of particle i (i first)."""
    idx = np.array(tree.query_ball_point(np.mod(pos[i], box), radius), dtype=np.int64)
    idx = idx[idx != i]
    return np.concatenate([[i], idx])


def sampled_checks(b, s, lj, rl, nsample, rng, check_lists=True, tol=1e-5, name="sample"):
    from scipy.spatial import cKDTree
    f, _, _ = b.force()
    tree = cKDTree(np.mod(s.pos, s.box), boxsize=s.box)
    sample = rng.choice(s.n, size=nsample, replace=False)
    if check_lists:
        count, nbr, pos_used = b.nlist()
        np.testing.assert_array_equal(pos_used, np.mod(s.pos, s.box))
    types = s.type
    got_f, ref_f, scale = [], [], []
    for i in sample:
        idx = neighbourhood(s.box, s.pos, i, rl + 0.5, tree)
        sub = s.pos[idx]
        st = types[idx]
        fo, _, _ = oracle.forces_brute(s.box, sub, lj, st)
        # pair-magnitude scale of particle i (the force tolerance's S_i)
        d = sub[1:] - sub[0]
        d -= s.box * np.rint(d / s.box)
        r2 = np.sum(d * d, axis=1)
        S = 0.0
        for k in range(len(r2)):
            a, c = st[0], st[k + 1]
            S += abs(oracle.pair(lj.eps[a, c], lj.sigma[a, c], lj.rcut[a, c], 1, r2[k])[0]) * np.sqrt(r2[k])
        got_f.append(f[i])
        ref_f.append(fo[0])
        scale.append(S)
        assert np.linalg.norm(f[i] - fo[0]) <= tol * S, i
        if check_lists:
            nl = oracle.nlist(s.box, sub, rl, use_cells=False)
            ref = np.sort(idx[nl.list[0, : nl.count[0]]])
            got = np.sort(nbr[i, : count[i]])
            assert np.array_equal(got, ref), i
    report(name, figures(np.array(got_f), np.array(ref_f), np.array(scale)))
    return f


def test_lj4m_sampled_forces_lists_and_invariants(ljmd):
    s = inputs.lj4m()
    lj = oracle.LJ(s.eps, s.sigma, s.rcut)
    b = ljmd.from_system(s, "mixed_ds")
    b.autotune(reps=2, cache=False)
    rng = np.random.default_rng(0)
    f = sampled_checks(b, s, lj, 2.8, 200, rng, name="lj4m sample of 200")
    # Newton III over 4M particles (FP32 pair sums)
    assert np.abs(f.sum(axis=0)).max() <= 1e-7 * np.abs(f).sum()
    p0 = s.vel.sum(axis=0)
    th = b.integrate(s.dt, 100)
    _, v, _ = b.get_state()
    assert np.abs(v.sum(axis=0) - p0).max() <= 1e-5 * s.n ** 0.5
    E = th[:, 0, 0] + th[:, 0, 1]
    assert np.abs(E - E[0]).max() / s.n < 1e-3
    assert b.info().rebuilds >= 5


def test_binary256k_sampled_forces_and_lists(ljmd):
    s = inputs.binary_random_system(seed=inputs.SEEDS["binary256k"])
    lj = oracle.LJ(s.eps, s.sigma, s.rcut)
    for prec, tol in (("mixed_ds", 1e-5), ("fp64", 1e-12)):
        b = ljmd.from_system(s, prec)
        b.autotune(reps=2, cache=False)
        sampled_checks(b, s, lj, float(s.rcut.max()) + s.skin, 100, np.random.default_rng(1), tol=tol,
                       name=f"binary256k {prec} sample of 100")
        b.close()


def test_replicas512_sampled_replicas(ljmd):
    systems = inputs.replica_systems(512, seed=inputs.SEEDS["replicas512"])
    n = [x.n for x in systems]
    pos = np.concatenate([x.pos for x in systems])
    vel = np.concatenate([x.vel for x in systems])
    box = np.stack([x.box for x in systems])
    b = ljmd.Box(pos, box, vel, n=n, precision="mixed_ds")
    b.set_lj(1.0, 1.0, 2.5, 0.3)
    b.autotune(reps=2, cache=False)
    f, e, w = b.force()
    th = b.integrate(0.005, 10)
    p2, v2, _ = b.get_state()
    off = np.concatenate([[0], np.cumsum(n)])
    rng = np.random.default_rng(2)
    for r in rng.choice(512, size=6, replace=False):
        x = systems[r]
        lj = oracle.LJ(x.eps, x.sigma, x.rcut)
        fo, eo, _ = oracle.forces(x.box, x.pos, lj)
        S = pair_scale(x.box, x.pos, lj)
        fr = f[off[r]:off[r + 1]]
        report(f"replicas512 replica {r} (N = {x.n})", figures(fr, fo, S))
        assert (np.linalg.norm(fr - fo, axis=1) / S).max() <= 1e-5
        assert abs(e[r] - eo) <= 1e-5 * abs(eo)
        rr = oracle.run(x.box, x.pos, x.vel, lj, 0.3, 0.005, 10)
        d = p2[off[r]:off[r + 1]] - rr["pos"]
        d -= x.box * np.rint(d / x.box)
        assert np.abs(d).max() <= 1e-4
        np.testing.assert_allclose(th[:, r, 1], rr["thermo"][:, 1], rtol=1e-5)


def test_lj32000_adjoint_vs_oracle(ljmd):
    s = inputs.lj32000()
    lj = oracle.LJ(s.eps, s.sigma, s.rcut)
    nsteps, k = 20, 10
    r = oracle.run(s.box, s.pos, s.vel, lj, s.skin, s.dt, nsteps, traj=True)
    target = oracle.hist(s.box, s.pos) * 0.9
    _, lx_T, _ = oracle.hist_loss(s.box, r["pos"], target)
    lv_T = np.zeros_like(lx_T)
    lx0, lv0, ge, gs = oracle.adjoint(s.box, r["traj"], lj, s.dt, lx_T, lv_T)
    b = ljmd.from_system(s, "mixed_ds")
    b.autotune(reps=2, cache=False)
    b.integrate(s.dt, nsteps, thermo=False, ckpt_every=k)
    gx0, gv0, gge, ggs = b.adjoint(lx_T, lv_T)
    rel = lambda a, c: np.linalg.norm(a - c) / np.linalg.norm(c)
    assert rel(gx0, lx0) <= 2e-4 and rel(gv0, lv0) <= 2e-4
    assert abs(gge[0, 0] - ge[0, 0]) <= 2e-4 * abs(ge[0, 0])
    assert abs(ggs[0, 0] - gs[0, 0]) <= 2e-4 * abs(gs[0, 0])


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("mixed_ds", 1e-4)])
def test_lj4000_hundred_steps(ljmd, prec, tol):
    s = inputs.lj4000()
    lj = oracle.LJ(s.eps, s.sigma, s.rcut)
    b = ljmd.from_system(s, prec)
    th = b.integrate(s.dt, 100)
    p, v, img = b.get_state()
    r = oracle.run(s.box, s.pos, s.vel, lj, s.skin, s.dt, 100)
    d = p - r["pos"]
    d -= s.box * np.rint(d / s.box)
    assert np.abs(d).max() <= tol
    np.testing.assert_allclose(th[:, 0, 0], r["thermo"][:, 0], rtol=10 * tol)
