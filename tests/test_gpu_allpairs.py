"""The all-to-all workload (Sec. 4: untruncated LJ forces between all pairs,
velocity-Verlet, and the stochastic Andersen-like "Boltzmann" thermostat) and
the thermostat on the truncated path, against the FP64 oracle.

Force tolerances as in test_gpu_md.py: max_i |dF_i| / S_i with
S_i = sum_j |F_ij|, 1e-5 for FP32 forces and 1e-12 for FP64.  The thermostat's
collision decisions are integer comparisons of the same Philox words on both
sides, so the same particles collide; the redrawn velocities agree to the
last bits of the FP64 log/cos/sin, and 10-step trajectories to 1e-4.
"""
import numpy as np
import pytest

import oracle
from paper_2406_04210_gb300 import inputs

pytestmark = pytest.mark.gpu

INF = np.full((1, 1), np.inf)


@pytest.fixture(scope="module")
def ljmd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_04210_gb300 import build, ljmd as m
    build.build()
    m.load()
    return m


def _all_pairs_box(ljmd, s, prec):
    b = ljmd.Box(s.pos, s.box, s.vel, s.type, precision=prec)
    b.set_lj(s.eps, s.sigma, INF, s.skin, True)
    return b


def _pair_scale(box, pos):
    """S_i = sum_j |F_ij| over all pairs (minimum image, no cutoff), and
    W_abs = sum_{i<j} |f_ij| r_ij^2, the scale of the virial's sum."""
    d = pos[:, None, :] - pos[None, :, :]
    d -= box * np.rint(d / box)
    r2 = np.einsum("ijk,ijk->ij", d, d)
    np.fill_diagonal(r2, 1.0)
    s6 = r2 ** -3
    f = 48.0 / r2 * (s6 * s6 - 0.5 * s6)
    np.fill_diagonal(f, 0.0)                         # no self pair
    return (np.abs(f) * np.sqrt(r2)).sum(axis=1), 0.5 * float((np.abs(f) * r2).sum())


def _close_traj(p, v, r, box, tol):
    d = p - r["pos"]
    d -= box * np.rint(d / box)
    assert np.abs(d).max() <= tol
    vrms = np.sqrt(np.mean(r["vel"] ** 2))
    assert np.abs(v - r["vel"]).max() <= tol * vrms


@pytest.mark.parametrize("prec,tol", [("mixed_ds", 1e-5), ("mixed_fp64", 1e-5), ("fp64", 1e-12)])
def test_all_pairs_forces_match_oracle(ljmd, prec, tol):
    s = inputs.fcc_subset_system(2000, 0.8442, 0.722, 41)
    b = _all_pairs_box(ljmd, s, prec)
    f, e, w = b.force()
    lj = oracle.LJ(s.eps, s.sigma, INF)
    fo, eo, wo = oracle.forces_brute(s.box, s.pos, lj)
    S, wabs = _pair_scale(s.box, s.pos)
    assert np.max(np.linalg.norm(f - fo, axis=1) / S) <= tol
    assert abs(e[0] - eo) <= tol * abs(eo)
    assert abs(w[0] - wo) <= tol * wabs


@pytest.mark.parametrize("prec,tol", [("mixed_ds", 1e-4), ("fp64", 1e-9)])
def test_all_pairs_trajectory_with_thermostat(ljmd, prec, tol):
    s = inputs.fcc_subset_system(2000, 0.8442, 0.722, 43)
    b = _all_pairs_box(ljmd, s, prec)
    b.set_thermostat(1.5, 20.0, 11)                # rate dt = 0.1: ~200 collisions a step
    th = b.integrate(s.dt, 10)
    p, v, _ = b.get_state()
    r = oracle.run(s.box, s.pos, s.vel, oracle.LJ(s.eps, s.sigma, INF), s.skin, s.dt, 10,
                   thermostat=(1.5, 20.0, 11))
    _close_traj(p, v, r, s.box, tol)
    np.testing.assert_allclose(th[:, 0, 3], r["thermo"][:, 3], rtol=10 * tol)


def test_thermostat_on_the_truncated_path(ljmd):
    s = inputs.lj4000()
    b = ljmd.from_system(s, "mixed_ds")
    b.set_thermostat(1.2, 10.0, 5)
    b.integrate(s.dt, 10)
    p, v, _ = b.get_state()
    r = oracle.run(s.box, s.pos, s.vel, oracle.LJ(s.eps, s.sigma, s.rcut), s.skin, s.dt, 10,
                   thermostat=(1.2, 10.0, 5))
    _close_traj(p, v, r, s.box, 1e-4)


def test_thermostat_step_index_continues_across_calls(ljmd):
    # 4 + 6 steps through two md_integrate calls (and graphs) = 10 steps at once
    s = inputs.lj4000()
    b = ljmd.from_system(s, "mixed_ds")
    b.set_thermostat(1.2, 10.0, 8)
    b.integrate(s.dt, 4)
    b.integrate(s.dt, 6)
    p, v, _ = b.get_state()
    r = oracle.run(s.box, s.pos, s.vel, oracle.LJ(s.eps, s.sigma, s.rcut), s.skin, s.dt, 10,
                   thermostat=(1.2, 10.0, 8))
    _close_traj(p, v, r, s.box, 1e-4)


def test_thermostat_replicas_have_their_own_streams(ljmd):
    systems = [inputs.fcc_subset_system(n, 0.8, 1.0, 50 + i) for i, n in enumerate((700, 900, 1100))]
    n = [x.n for x in systems]
    pos = np.concatenate([x.pos for x in systems])
    vel = np.concatenate([x.vel for x in systems])
    box = np.stack([x.box for x in systems])
    b = ljmd.Box(pos, box, vel, n=n)
    b.set_lj(1.0, 1.0, 2.5, 0.3)
    T = np.array([0.8, 1.4, 2.0])
    b.set_thermostat(T, 10.0, 21)
    b.integrate(0.005, 10)
    p, v, _ = b.get_state()
    off = np.concatenate([[0], np.cumsum(n)])
    for r_ in range(3):
        x = systems[r_]
        rr = oracle.run(x.box, x.pos, x.vel, oracle.LJ(x.eps, x.sigma, x.rcut), 0.3, 0.005, 10,
                        thermostat=(T[r_], 10.0, 21 + r_))   # key = seed + replica
        _close_traj(p[off[r_]:off[r_ + 1]], v[off[r_]:off[r_ + 1]], rr, x.box, 1e-4)


def test_thermostat_reaches_the_bath_temperature(ljmd):
    s = inputs.lj4000()
    b = ljmd.from_system(s, "mixed_ds")
    b.set_thermostat(1.5, 10.0, 2)
    th = b.integrate(s.dt, 2000)
    T = th[1000:, 0, 3].mean()
    assert abs(T - 1.5 * s.n / (s.n - 1)) < 0.02


def test_guards(ljmd):
    s = inputs.fcc_subset_system(500, 0.8442, 0.722, 3)
    b = _all_pairs_box(ljmd, s, "mixed_ds")
    b.integrate(s.dt, 5, thermo=False, ckpt_every=5)
    with pytest.raises(ljmd.MDError) as ei:
        b.adjoint(np.zeros((s.n, 3)), np.zeros((s.n, 3)))
    assert ei.value.status == 1
    with pytest.raises(ljmd.MDError):
        b.nlist()
    c = ljmd.from_system(inputs.lj4000(), "mixed_ds")
    c.set_thermostat(1.0, 1.0, 0)
    with pytest.raises(ljmd.MDError) as ei:
        c.integrate(0.005, 10, thermo=False, ckpt_every=5)
    assert ei.value.status == 1
    c.set_thermostat(None, 0.0)                     # off again: records work
    c.integrate(0.005, 10, thermo=False, ckpt_every=5)
