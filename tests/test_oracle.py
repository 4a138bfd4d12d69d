"""Pins of the FP64 oracle against facts that do not come from its own code.

Every function of oracle/ljmd_oracle.c is checked here against a closed form,
an invariant of Hamiltonian dynamics, a finite difference, an independent
library routine (scipy's periodic k-d tree) or brute force (see the header of
ljmd_oracle.c for the map).  CPU only.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2406_04210_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden", "lj_pair_closed_forms.txt")


def _golden():
    out = {}
    for line in open(GOLD):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


# --- pair function -----------------------------------------------------------

def test_pair_closed_forms():
    g = _golden()
    rmin = g["r_min"]
    assert abs(rmin - 2.0 ** (1.0 / 6.0)) < 1e-15
    f, u, _, _ = oracle.pair(1.0, 1.0, 2.5, 1, rmin * rmin)
    assert abs(f) < 1e-13                      # force vanishes at the minimum
    assert abs(u - g["u_min_shifted"]) < 1e-13
    f, u, _, _ = oracle.pair(1.0, 1.0, 2.5, 1, 1.0)
    assert abs(u - g["u_sigma_shifted"]) < 1e-13
    assert abs(f * 1.0 - g["f_sigma"]) < 1e-12  # |F| = f * r at r = sigma
    f, u, _, _ = oracle.pair(1.0, 1.0, 2.5, 0, 1.0)
    assert abs(u) < 1e-15                      # unshifted U(sigma) = 0
    # shifted potential is continuous at the cutoff, zero beyond
    _, u_in, _, _ = oracle.pair(1.0, 1.0, 2.5, 1, (2.5 - 1e-9) ** 2)
    assert abs(u_in) < 1e-9
    assert tuple(oracle.pair(1.0, 1.0, 2.5, 1, 2.5 ** 2)) == (0.0, 0.0, 0.0, 0.0)
    _, u_rc_unshifted, _, _ = oracle.pair(1.0, 1.0, 2.5, 0, (2.5 - 1e-12) ** 2)
    assert abs(u_rc_unshifted - g["u_rc"]) < 1e-10


def test_pair_scaling_laws():
    # U is linear in eps and depends on r only through r/sigma (rc scaled too)
    for r in (0.93, 1.2, 1.7, 2.3):
        a = oracle.pair(1.0, 1.0, 2.5, 1, r * r)
        b = oracle.pair(1.7, 1.0, 2.5, 1, r * r)
        c = oracle.pair(1.0, 0.8, 2.0, 1, (0.8 * r) ** 2)
        assert abs(b[1] - 1.7 * a[1]) < 1e-12 * max(1, abs(a[1]))
        assert abs(c[1] - a[1]) < 1e-12 * max(1, abs(a[1]))
        # f = -U'/r has dimension 1/length^2: f(0.8 r; 0.8) = f(r; 1) / 0.8^2
        assert abs(c[0] * 0.64 - a[0]) < 1e-11 * max(1, abs(a[0]))


@pytest.mark.parametrize("r", [0.95, 1.05, 1.3, 1.9, 2.4])
def test_pair_derivatives_fd(r):
    h = 1e-5
    U = lambda x: oracle.pair(1.3, 0.9, 2.25, 1, x * x)[1]
    f, _, pp, p_over_r = oracle.pair(1.3, 0.9, 2.25, 1, r * r)
    dU = (U(r + h) - U(r - h)) / (2 * h)
    assert abs(-dU / r - f) < 1e-7 * max(1.0, abs(f))
    assert abs(p_over_r * r - dU) < 1e-7 * max(1.0, abs(dU))
    dP = lambda x: oracle.pair(1.3, 0.9, 2.25, 1, x * x)[3] * x
    d2 = (dP(r + h) - dP(r - h)) / (2 * h)
    assert abs(pp - d2) < 1e-6 * max(1.0, abs(pp))


def test_min_image():
    assert oracle.min_image(9.0, 10.0) == pytest.approx(-1.0)
    assert oracle.min_image(-9.0, 10.0) == pytest.approx(1.0)
    assert oracle.min_image(4.0, 10.0) == pytest.approx(4.0)


# --- forces ------------------------------------------------------------------

def test_two_particles_across_boundary():
    L = 10.0
    box = np.array([L, L, L])
    pos = np.array([[0.2, 5.0, 5.0], [L - 0.8, 5.0, 5.0]])
    lj = oracle.LJ.single()
    f, e, w = oracle.forces_brute(box, pos, lj)
    g = _golden()
    assert f[0, 0] == pytest.approx(24.0, abs=1e-11)     # pushed towards +x
    assert f[1, 0] == pytest.approx(-24.0, abs=1e-11)
    assert np.abs(f[:, 1:]).max() == 0.0
    assert e == pytest.approx(g["u_sigma_shifted"], abs=1e-13)
    assert w == pytest.approx(24.0, abs=1e-11)           # d.F = f r^2 = 24
    fl, el, wl = oracle.forces(box, pos, lj, use_cells=True)
    np.testing.assert_allclose(fl, f, atol=1e-12)
    assert el == pytest.approx(e) and wl == pytest.approx(w)


@pytest.fixture(scope="module")
def small_fluid():
    return inputs.fcc_subset_system(500, 0.8442, 0.722, seed=11)


def test_newton_third_law(small_fluid):
    s = small_fluid
    lj = oracle.LJ(s.eps, s.sigma, s.rcut)
    f, _, _ = oracle.forces_brute(s.box, s.pos, lj)
    assert np.abs(f.sum(axis=0)).max() < 1e-12 * np.abs(f).sum()


def test_list_forces_equal_brute(small_fluid):
    s = small_fluid
    lj = oracle.LJ(s.eps, s.sigma, s.rcut)
    fb, eb, wb = oracle.forces_brute(s.box, s.pos, lj)
    nl = oracle.nlist(s.box, s.pos, 2.8, use_cells=True)
    fl, el, wl = oracle.forces_list(s.box, s.pos, lj, nl)
    np.testing.assert_allclose(fl, fb, rtol=0, atol=1e-11 * np.abs(fb).max())
    assert el == pytest.approx(eb, rel=1e-12)
    assert wl == pytest.approx(wb, rel=1e-12)


def test_binary_forces_list_equal_brute():
    rng = np.random.default_rng(3)
    eps, sig, rc = inputs.binary_params()
    n = 400
    L = (n / 1.2) ** (1 / 3)
    box = np.array([L, L, L])
    pos = inputs.random_insertion(n, box, 0.7, rng)
    t = (rng.uniform(size=n) < 0.2).astype(np.int32)
    lj = oracle.LJ(eps, sig, rc)
    fb, eb, wb = oracle.forces_brute(box, pos, lj, t)
    fl, el, wl = oracle.forces(box, pos, lj, t)
    np.testing.assert_allclose(fl, fb, rtol=0, atol=1e-11 * np.abs(fb).max())
    assert el == pytest.approx(eb, rel=1e-12) and wl == pytest.approx(wb, rel=1e-12)


def test_energy_gradient_is_minus_force(small_fluid):
    s = small_fluid
    lj = oracle.LJ(s.eps, s.sigma, s.rcut)
    rng = np.random.default_rng(5)
    u = rng.normal(size=s.pos.shape)
    u /= np.linalg.norm(u)
    # h balances the O(h^2) truncation against the rounding noise of a
    # ~3000-valued E_pot sum (~3e-11 / 2h)
    h = 1e-5
    f, _, _ = oracle.forces_brute(s.box, s.pos, lj)
    _, ep, _ = oracle.forces_brute(s.box, s.pos + h * u, lj)
    _, em, _ = oracle.forces_brute(s.box, s.pos - h * u, lj)
    fd = (ep - em) / (2 * h)
    assert fd == pytest.approx(-np.sum(f * u), rel=1e-4)


def test_virial_is_volume_derivative(small_fluid):
    # scaling all coordinates and the box by lam: dU/dlam|_1 = -W
    s = small_fluid
    lj = oracle.LJ(s.eps, s.sigma, s.rcut)
    _, _, w = oracle.forces_brute(s.box, s.pos, lj)
    h = 1e-7
    _, ep, _ = oracle.forces_brute(s.box * (1 + h), s.pos * (1 + h), lj)
    _, em, _ = oracle.forces_brute(s.box * (1 - h), s.pos * (1 - h), lj)
    assert (ep - em) / (2 * h) == pytest.approx(-w, rel=1e-6)


# --- neighbour lists ---------------------------------------------------------

def _kdtree_sets(box, pos, rl):
    from scipy.spatial import cKDTree
    t = cKDTree(pos, boxsize=box)
    pairs = t.query_pairs(rl, output_type="ndarray")
    sets = [[] for _ in range(pos.shape[0])]
    for i, j in pairs:
        sets[i].append(j)
        sets[j].append(i)
    return [np.array(sorted(x), dtype=np.int64) for x in sets]


@pytest.mark.parametrize("case", ["lj4000", "faces", "nc3"])
def test_nlist_cells_equal_brute_and_kdtree(case):
    if case == "lj4000":
        s = inputs.lj4000()
        box, pos = s.box, s.pos
    elif case == "faces":
        # particles exactly on cell faces and at x = 0
        L = 8.4 * 1.0001
        box = np.array([L, L, L])
        g = np.linspace(0, L, 13, endpoint=False)
        pos = np.stack(np.meshgrid(g[::2], g[::3], g[::2], indexing="ij"), -1).reshape(-1, 3)
        pos[::7, 0] = 0.0
    else:
        L = 3 * 2.8 + 1e-3      # exactly 3 cells per dimension
        rng = np.random.default_rng(9)
        box = np.array([L, L, L])
        pos = rng.uniform(0, L, size=(300, 3))
    rl = 2.8
    a = oracle.nlist(box, pos, rl, use_cells=True)
    b = oracle.nlist(box, pos, rl, use_cells=False)
    sa, sb = a.sets(), b.sets()
    sk = _kdtree_sets(box, pos, rl)
    for i in range(len(sa)):
        assert np.array_equal(sa[i], sb[i])
        assert np.array_equal(sa[i], sk[i])


# --- dynamics ----------------------------------------------------------------

@pytest.fixture(scope="module")
def run500(small_fluid):
    s = small_fluid
    lj = oracle.LJ(s.eps, s.sigma, s.rcut)
    return oracle.run(s.box, s.pos, s.vel, lj, s.skin, 0.005, 400)


def test_momentum_conserved(small_fluid, run500):
    p0 = small_fluid.vel.sum(axis=0)
    p1 = run500["vel"].sum(axis=0)
    assert np.abs(p1 - p0).max() < 1e-12 * small_fluid.n


def test_energy_conserved_and_dt2_scaling(small_fluid):
    s = small_fluid
    lj = oracle.LJ(s.eps, s.sigma, s.rcut)
    fl = []
    for dt, n in ((0.004, 250), (0.002, 500)):
        r = oracle.run(s.box, s.pos, s.vel, lj, s.skin, dt, n)
        E = r["thermo"][:, 0] + r["thermo"][:, 1]
        fl.append(E.max() - E.min())
        assert fl[-1] / s.n < 2e-3
        assert r["builds"] > 2          # the skin rule triggered rebuilds
    ratio = fl[0] / fl[1]
    assert 2.5 < ratio < 6.0            # velocity-Verlet: energy error ~ dt^2


def test_time_reversibility(small_fluid):
    s = small_fluid
    lj = oracle.LJ(s.eps, s.sigma, s.rcut)
    a = oracle.run(s.box, s.pos, s.vel, lj, s.skin, 0.005, 100)
    b = oracle.run(s.box, a["pos"], -a["vel"], lj, s.skin, 0.005, 100)
    d = b["pos"] - s.pos
    d -= s.box * np.rint(d / s.box)
    assert np.abs(d).max() < 1e-8
    assert np.abs(b["vel"] + s.vel).max() < 1e-8


def test_temperature_definition(small_fluid, run500):
    # T = 2 E_kin / (3N - 3) with E_kin = 1/2 sum v^2 at the final step
    r = run500
    ek = 0.5 * float(np.sum(r["vel"] ** 2))
    assert r["thermo"][-1, 1] == pytest.approx(ek, rel=1e-12)
    assert r["thermo"][-1, 3] == pytest.approx(2 * ek / (3 * small_fluid.n - 3), rel=1e-12)


# --- second derivatives ------------------------------------------------------

def test_hvp_matches_force_differences(small_fluid):
    s = small_fluid
    lj = oracle.LJ(s.eps, s.sigma, s.rcut)
    rng = np.random.default_rng(8)
    u = rng.normal(size=s.pos.shape)
    h = 1e-6
    fp, _, _ = oracle.forces_brute(s.box, s.pos + h * u, lj)
    fm, _, _ = oracle.forces_brute(s.box, s.pos - h * u, lj)
    fd = -(fp - fm) / (2 * h)
    hu = oracle.hvp(s.box, s.pos, lj, u)
    np.testing.assert_allclose(hu, fd, rtol=0, atol=1e-5 * np.abs(fd).max())


def test_param_derivatives_match_force_differences():
    rng = np.random.default_rng(4)
    eps, sig, rc = inputs.binary_params()
    n = 300
    L = (n / 1.2) ** (1 / 3)
    box = np.array([L, L, L])
    pos = inputs.random_insertion(n, box, 0.75, rng)
    t = (rng.uniform(size=n) < 0.3).astype(np.int32)
    lam = rng.normal(size=(n, 3))
    lj = oracle.LJ(eps, sig, rc)
    ge, gs = oracle.dforce_dparam(box, pos, lj, lam, t)
    assert np.allclose(ge, ge.T) and np.allclose(gs, gs.T)
    for a, b in ((0, 0), (0, 1), (1, 1)):
        for which, g in (("eps", ge), ("sigma", gs)):
            h = 1e-6
            vals = []
            for sgn in (1, -1):
                e2, s2 = eps.copy(), sig.copy()
                tgt = e2 if which == "eps" else s2
                tgt[a, b] += sgn * h
                if a != b:
                    tgt[b, a] += sgn * h
                f, _, _ = oracle.forces_brute(box, pos, oracle.LJ(e2, s2, rc), t)
                vals.append(np.sum(lam * f))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert g[a, b] == pytest.approx(fd, rel=1e-5, abs=1e-6), (which, a, b)


# --- histogram loss ----------------------------------------------------------

def test_hist_normalisation_poisson_sum():
    # For a pair well inside (0, 2.5) and w = bin width D, the Gaussian sampled
    # at the bin centres (k + 1/2) D sums to
    # sqrt(2 pi) (1 + 2 sum_m exp(-2 pi^2 m^2) cos(2 pi m (r/D - 1/2)))
    # (Poisson summation; terms m >= 2 are below 1e-34).
    box = np.array([10.0, 10.0, 10.0])
    for r in (0.9, 1.234, 1.77):
        pos = np.array([[1.0, 1.0, 1.0], [1.0 + r, 1.0, 1.0]])
        h = oracle.hist(box, pos)
        ph = 2 * math.pi * (r / (2.5 / 64) - 0.5)
        expect = math.sqrt(2 * math.pi) * (1 + 2 * math.exp(-2 * math.pi ** 2) * math.cos(ph)) / 2.0
        assert h.sum() == pytest.approx(expect, rel=1e-10)
        k = int(r / (2.5 / 64))
        assert np.argmax(h) in (k, k + 1)


def test_hist_grad_fd(small_fluid):
    s = small_fluid
    rng = np.random.default_rng(2)
    target = oracle.hist(s.box, s.pos) * (1 + 0.1 * rng.normal(size=64))
    loss, g, _ = oracle.hist_loss(s.box, s.pos, target)
    u = rng.normal(size=s.pos.shape)
    h = 1e-6
    lp, _, _ = oracle.hist_loss(s.box, s.pos + h * u, target)
    lm, _, _ = oracle.hist_loss(s.box, s.pos - h * u, target)
    assert (lp - lm) / (2 * h) == pytest.approx(np.sum(g * u), rel=1e-5)


# --- adjoint -----------------------------------------------------------------

def _traj_loss(s, lj, pos0, vel0, nsteps, target, wv):
    r = oracle.run(s.box, pos0, vel0, lj, s.skin, s.dt, nsteps, traj=True)
    loss, g, _ = oracle.hist_loss(s.box, r["pos"], target)
    loss += float(np.sum(wv * r["vel"]))
    return loss, g, r


def test_adjoint_matches_finite_differences():
    s = inputs.fcc_system(4, seed=21)          # 256 particles, L = 6.72
    lj = oracle.LJ(s.eps, s.sigma, s.rcut)
    rng = np.random.default_rng(6)
    nsteps = 10
    target = oracle.hist(s.box, s.pos) * 0.9
    wv = 0.01 * rng.normal(size=s.pos.shape)
    loss, g, r = _traj_loss(s, lj, s.pos, s.vel, nsteps, target, wv)
    lx0, lv0, ge, gs = oracle.adjoint(s.box, r["traj"], lj, s.dt, g, wv)
    u = rng.normal(size=s.pos.shape)
    h = 1e-6
    lp = _traj_loss(s, lj, s.pos + h * u, s.vel, nsteps, target, wv)[0]
    lm = _traj_loss(s, lj, s.pos - h * u, s.vel, nsteps, target, wv)[0]
    assert (lp - lm) / (2 * h) == pytest.approx(np.sum(lx0 * u), rel=1e-5)
    lp = _traj_loss(s, lj, s.pos, s.vel + h * u, nsteps, target, wv)[0]
    lm = _traj_loss(s, lj, s.pos, s.vel - h * u, nsteps, target, wv)[0]
    assert (lp - lm) / (2 * h) == pytest.approx(np.sum(lv0 * u), rel=1e-5)
    for which, g_ in (("eps", ge), ("sigma", gs)):
        vals = []
        for sgn in (1, -1):
            e2, s2 = s.eps.copy(), s.sigma.copy()
            (e2 if which == "eps" else s2)[0, 0] += sgn * h
            vals.append(_traj_loss(s, oracle.LJ(e2, s2, s.rcut), s.pos, s.vel, nsteps,
                                   target, wv)[0])
        assert (vals[0] - vals[1]) / (2 * h) == pytest.approx(g_[0, 0], rel=1e-5)


# --- input relaxation --------------------------------------------------------

def test_fire_relaxes():
    s = inputs.binary_random_system(n=500, seed=5)
    lj = oracle.LJ(s.eps, s.sigma, s.rcut)
    _, e0, _ = oracle.forces(s.box, s.pos, lj, s.type)
    pos, it, fmax = oracle.fire(s.box, s.pos, lj, s.type, maxit=5000, ftol=1e-3)
    _, e1, _ = oracle.forces(s.box, pos, lj, s.type)
    assert fmax < 1e-3 and e1 < e0


# ---------------------------------------------------------------------------
# Counter-based random numbers and the Andersen-like thermostat (Sec. 4: the
# "Boltzmann" thermostat of the all-to-all workload), and the all-pairs form.
# ---------------------------------------------------------------------------
KAT = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def test_philox_known_answer_vectors():
    # Published known-answer vectors of Philox4x32-10 (Salmon et al., SC'11;
    # Random123 distribution): they fix the multipliers, the Weyl key
    # increments, the round count and the order of the output words
    rows = [[int(x, 16) for x in ln.split()] for ln in open(KAT)
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for w in rows:
        out = oracle.philox4x32(w[:4], w[4:6])
        assert [int(x) for x in out] == w[6:], [hex(int(x)) for x in out]


def test_philox_uniform_independent_and_mixing():
    key = (1234, 5678)
    words = np.concatenate([oracle.philox4x32((i, 0, 0, 0), key) for i in range(16384)]).astype(np.int64)
    # uniform top bytes: chi-square with 255 degrees of freedom (mean 255, sd 22.6)
    counts = np.bincount(words >> 24, minlength=256)
    chi2 = float(((counts - len(words) / 256) ** 2 / (len(words) / 256)).sum())
    assert 185 < chi2 < 330
    # every bit set half the time (sd 0.002)
    bits = (words[:, None] >> np.arange(32)) & 1
    assert np.all(np.abs(bits.mean(axis=0) - 0.5) < 0.012)
    # avalanche: one flipped counter bit changes about half of the 128 output bits
    rng = np.random.default_rng(0)
    dist = []
    for _ in range(256):
        c = rng.integers(0, 2 ** 32, size=4, dtype=np.uint64).astype(np.uint32)
        c2 = c.copy()
        c2[rng.integers(0, 4)] ^= np.uint32(1 << int(rng.integers(0, 32)))
        a, b = oracle.philox4x32(c, key), oracle.philox4x32(c2, key)
        dist.append(sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(a, b)))
    assert 61 < np.mean(dist) < 67
    # another key gives an unrelated stream
    other = np.concatenate([oracle.philox4x32((i, 0, 0, 0), (1235, 5678)) for i in range(4096)])
    assert np.mean(other == words[: 4 * 4096].astype(np.uint32)) < 1e-3


def test_thermostat_collision_rate_and_maxwell_boltzmann():
    from scipy import stats
    n = 20000
    zero = np.zeros((n, 3))
    # rate dt = 0.1: collisions ~ Binomial(n, 0.1)
    v, hits = oracle.thermostat(zero, 2.0, 20.0, 0.005, 99, 7)
    assert abs(hits - 0.1 * n) < 5 * np.sqrt(n * 0.1 * 0.9)
    moved = np.any(v != 0.0, axis=1)
    assert moved.sum() == hits
    # a different step draws different particles
    v2, hits2 = oracle.thermostat(zero, 2.0, 20.0, 0.005, 99, 8)
    assert np.any(np.any(v2 != 0.0, axis=1) != moved)
    # rate dt >= 1: every particle is redrawn from N(0, T) per component
    v, hits = oracle.thermostat(zero, 2.0, 1000.0, 0.005, 5, 0)
    assert hits == n
    g = v.ravel() / np.sqrt(2.0)
    assert abs(g.mean()) < 5 * np.sqrt(1.0 / g.size)
    assert abs(g.var() - 1.0) < 5 * np.sqrt(2.0 / g.size)
    assert abs(stats.kurtosis(g, fisher=False) - 3.0) < 5 * np.sqrt(24.0 / g.size)
    assert stats.kstest(g, "norm").pvalue > 1e-4


def test_thermostat_reaches_the_bath_temperature():
    # canonical ensemble: <E_kin> = 3/2 N T_bath, reported as 2 E_kin/(3N - 3)
    s = inputs.fcc_system(5, seed=31)               # 500 particles, T 0.722
    lj = oracle.LJ(s.eps, s.sigma, s.rcut)
    r = oracle.run(s.box, s.pos, s.vel, lj, s.skin, s.dt, 1500, thermostat=(1.5, 10.0, 3))
    T = r["thermo"][500:, 3].mean()
    assert abs(T - 1.5 * s.n / (s.n - 1)) < 0.04


def test_all_pairs_forces_and_run():
    s = inputs.fcc_system(4, seed=17)               # 256 particles, L = 6.72
    inf = np.full((1, 1), np.inf)
    lj = oracle.LJ(s.eps, s.sigma, inf)
    f, e, _ = oracle.forces_brute(s.box, s.pos, lj)
    assert np.abs(f.sum(axis=0)).max() < 1e-10 * np.abs(f).sum()          # Newton III
    rng = np.random.default_rng(4)
    u = rng.normal(size=s.pos.shape)
    h = 1e-6
    ep = oracle.forces_brute(s.box, s.pos + h * u, lj)[1]
    em = oracle.forces_brute(s.box, s.pos - h * u, lj)[1]
    assert (ep - em) / (2 * h) == pytest.approx(-np.sum(f * u), rel=1e-6)  # F = -grad U
    r = oracle.run(s.box, s.pos, s.vel, lj, s.skin, s.dt, 200)
    assert r["builds"] == 0                                                # no lists
    E = r["thermo"][:, 0] + r["thermo"][:, 1]
    # NVE: the minimum-image force flips at a separation of L/2 (the energy is
    # continuous there), so the integration error is first order in dt:
    # bounded by 5e-4 per particle over 200 steps (1.8e-4 observed)
    assert np.abs(E - E[0]).max() / s.n < 5e-4
    assert np.abs(r["vel"].sum(axis=0) - s.vel.sum(axis=0)).max() < 1e-10
