"""Both FP32 list-form force kernels against the FP64 oracle (Sec. 4/5: LJ
pair forces, energy and virial over the Verlet lists).

md_set_force_kernel selects the chunk kernel (128 consecutive particles per
work item, neighbour offsets gathered from global memory) or the tiled kernel
(bricks of up to 2 x 2 x 2 cells, the brick's neighbourhood staged in shared
memory in the frame of the brick's centre; neighbourhoods beyond the
2048-particle tile evaluated from global memory).  Every case runs both, with the tolerances of
tests/test_gpu_md.py: max_i |dF_i| / S_i <= 1e-5, E_pot relative 1e-5, W
against W_abs, 10-step trajectories within 1e-4.
"""
import numpy as np
import pytest

import oracle
from forcecheck import figures, pair_scale, report
from paper_2406_04210_gb300 import inputs

pytestmark = pytest.mark.gpu

KINDS = ["chunks", "tiles"]


@pytest.fixture(scope="module")
def ljmd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_04210_gb300 import build, ljmd as m
    build.build()
    m.load()
    return m


def _lj(s):
    return oracle.LJ(s.eps, s.sigma, s.rcut, True)


def _check_forces(f, e, w, fo, eo, wo, S, tag):
    report(tag, figures(f, fo, S))
    err = np.linalg.norm(f - fo, axis=1) / S
    assert err.max() <= 1e-5, err.max()
    assert abs(e - eo) <= 1e-5 * abs(eo)
    assert abs(w - wo) <= 1e-5 * 0.5 * 2.5 * S.sum()


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("prec", ["mixed_ds", "mixed_fp64"])
def test_lj4000_forces_energy_virial(ljmd, kind, prec):
    s = inputs.lj4000()
    b = ljmd.from_system(s, prec)
    b.force_kernel = kind
    assert b.force_kernel == kind
    f, e, w = b.force()
    lj = _lj(s)
    fo, eo, wo = oracle.forces(s.box, s.pos, lj)
    _check_forces(f, e[0], w[0], fo, eo, wo, pair_scale(s.box, s.pos, lj), f"lj4000 {prec} {kind}")


@pytest.mark.parametrize("kind", KINDS)
def test_lj4000_ten_steps(ljmd, kind):
    s = inputs.lj4000()
    b = ljmd.from_system(s, "mixed_ds")
    b.force_kernel = kind
    th = b.integrate(s.dt, 10)
    pos, vel, img = b.get_state()
    r = oracle.run(s.box, s.pos, s.vel, _lj(s), s.skin, s.dt, 10)
    d = pos - r["pos"]
    d -= s.box * np.rint(d / s.box)
    assert np.abs(d).max() <= 1e-4
    assert np.abs(vel - r["vel"]).max() <= 1e-4 * np.sqrt(np.mean(s.vel ** 2))
    np.testing.assert_array_equal(img, r["img"])
    wabs = 0.5 * 2.5 * pair_scale(s.box, s.pos, _lj(s)).sum()
    np.testing.assert_allclose(th[:, 0, [0, 1, 3]], r["thermo"][:, [0, 1, 3]], rtol=1e-5, atol=1e-8)
    assert np.abs(th[:, 0, 2] - r["thermo"][:, 2]).max() <= 1e-5 * wabs


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("n", [4000, 3472])
def test_ten_steps_without_energies(ljmd, kind, n):
    # steps without per-step energies run the kernels' force-only variants;
    # the monatomic fluid and the binary mixture, against the oracle's run
    if n == 4000:
        s = inputs.lj4000()
    else:
        s = inputs.binary_random_system(n=n, seed=17)
        lj = _lj(s)
        s.pos, _, _ = oracle.fire(s.box, s.pos, lj, s.type, maxit=300, ftol=1e-2)
        s.vel = np.random.default_rng(3).normal(0.0, np.sqrt(0.7), size=s.pos.shape)
        s.vel -= s.vel.mean(axis=0)
    b = ljmd.from_system(s, "mixed_ds")
    b.force_kernel = kind
    b.integrate(s.dt, 10, thermo=False)
    pos, vel, img = b.get_state()
    types = None if n == 4000 else s.type
    r = oracle.run(s.box, s.pos, s.vel, _lj(s), s.skin, s.dt, 10, types)
    d = pos - r["pos"]
    d -= s.box * np.rint(d / s.box)
    assert np.abs(d).max() <= 1e-4
    assert np.abs(vel - r["vel"]).max() <= 1e-4 * np.sqrt(np.mean(s.vel ** 2))


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("n", [3000, 3472])
def test_binary_mixture(ljmd, kind, n):
    # density 1.2: n = 3000 gives 4 cells of 3.39 per edge, so a brick's
    # 4 x 4 x 4-cell neighbourhood is the whole box, beyond the tile, and the
    # tiled kernel takes its global-memory path; n = 3472 (L = 14.25, 5 cells
    # of 2.85 per edge, bricks of 2 and 1 cells) gives neighbourhoods of up
    # to ~1780, inside the tile, with the species read from the tile
    s = inputs.binary_random_system(n=n, seed=17)
    lj = _lj(s)
    pos, _, _ = oracle.fire(s.box, s.pos, lj, s.type, maxit=300, ftol=1e-2)
    s.pos = pos
    b = ljmd.from_system(s, "mixed_ds")
    b.force_kernel = kind
    f, e, w = b.force()
    fo, eo, wo = oracle.forces(s.box, s.pos, lj, s.type)
    _check_forces(f, e[0], w[0], fo, eo, wo, pair_scale(s.box, s.pos, lj, s.type), f"binary{n} {kind}")


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("n,L,scale", [(700, 8.41, 1.0), (250, 7.6, 1.0), (700, 8.41, 1.5), (700, 8.41, 2.0)])
def test_three_two_and_one_cells_per_edge(ljmd, kind, n, L, scale):
    # 3 cells per edge (bricks of 2 and 1 cells); 2 cells of 3.8 (one brick
    # of 2 x 2 x 2 whose neighbourhood repeats each cell 8 times with
    # different image shifts, 2000 particles, inside the tile); 2 cells of
    # 4.2 (bricks of one cell: 27 copies of 87, beyond the tile); 1 cell (27
    # copies of the box, beyond the tile)
    rng = np.random.default_rng(n)
    box = np.array([L, L, L])
    pos = rng.uniform(0, L, size=(n, 3))
    pos, _, _ = oracle.fire(box, pos, oracle.LJ.single(), maxit=200, ftol=1.0)
    b = ljmd.Box(pos, box, None, precision="mixed_ds")
    b.set_lj(1.0, 1.0, 2.5, 0.3)
    b.force_kernel = kind
    b.set_layout(cell_scale=scale)
    f, e, w = b.force()
    fo, eo, wo = oracle.forces_brute(box, pos, oracle.LJ.single())
    S = pair_scale(box, pos, oracle.LJ.single())
    _check_forces(f, e[0], w[0], fo, eo, wo, S, f"{n} in {L} scale {scale} {kind}")


@pytest.mark.parametrize("kind", KINDS)
def test_batched_replicas(ljmd, kind):
    systems = inputs.replica_systems(nrep=6, nmin=500, nmax=3000, seed=5)
    n = [x.n for x in systems]
    b = ljmd.Box(np.concatenate([x.pos for x in systems]), np.stack([x.box for x in systems]),
                 np.concatenate([x.vel for x in systems]), n=n, precision="mixed_ds")
    b.set_lj(1.0, 1.0, 2.5, 0.3)
    b.force_kernel = kind
    f, e, w = b.force()
    th = b.integrate(0.005, 10)
    p2 = b.get_state()[0]
    o = 0
    for r, x in enumerate(systems):
        lj = _lj(x)
        fo, eo, wo = oracle.forces(x.box, x.pos, lj)
        S = pair_scale(x.box, x.pos, lj)
        _check_forces(f[o:o + x.n], e[r], w[r], fo, eo, wo, S, f"replica {r} (N = {x.n}) {kind}")
        rr = oracle.run(x.box, x.pos, x.vel, lj, 0.3, 0.005, 10)
        d = p2[o:o + x.n] - rr["pos"]
        d -= x.box * np.rint(d / x.box)
        assert np.abs(d).max() <= 1e-4
        np.testing.assert_allclose(th[:, r, [0, 1, 3]], rr["thermo"][:, [0, 1, 3]], rtol=1e-5, atol=1e-8)
        o += x.n


def test_kernels_agree_and_switch_freely(ljmd):
    # the two kernels on the same lists: the same forces up to FP32
    # rounding order; switching back reproduces the first result bit for bit
    s = inputs.fcc_system(12, seed=4)   # 6912 particles
    b = ljmd.from_system(s, "mixed_ds")
    out = {}
    for kind in ("tiles", "chunks", "tiles"):
        b.force_kernel = kind
        f, e, w = b.force()
        if kind in out:
            np.testing.assert_array_equal(f, out[kind][0])
            assert e[0] == out[kind][1] and w[0] == out[kind][2]
        out[kind] = (f, e[0], w[0])
    S = pair_scale(s.box, s.pos, _lj(s))
    assert (np.linalg.norm(out["tiles"][0] - out["chunks"][0], axis=1) / S).max() <= 2e-6
    assert abs(out["tiles"][1] - out["chunks"][1]) <= 2e-6 * abs(out["chunks"][1])


def test_force_kernel_option_is_checked(ljmd):
    s = inputs.lj4000()
    b = ljmd.from_system(s, "mixed_ds")
    assert b.force_kernel == "auto"
    lib, h = b._lib, b._h
    assert lib.md_set_force_kernel(h, 3) == 1
    assert lib.md_set_force_kernel(h, -1) == 1
    assert b.force_kernel == "auto"


def test_autotune_keeps_a_chosen_force_kernel(ljmd):
    s = inputs.lj4000()
    b = ljmd.from_system(s, "mixed_ds")
    b.force_kernel = "tiles"
    t = b.autotune(reps=1, cache=False)
    assert t["force_kernel"] == "tiles" and b.force_kernel == "tiles"
    f, e, w = b.force()
    lj = _lj(s)
    fo, eo, wo = oracle.forces(s.box, s.pos, lj)
    _check_forces(f, e[0], w[0], fo, eo, wo, pair_scale(s.box, s.pos, lj), "lj4000 tiles after autotune")
