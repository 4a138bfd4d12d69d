"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (the readings behind them are in tests/forcecheck.py):
  * neighbour sets: identical to the oracle's FP64 definition (bit-exact
    membership, compared after sorting by user index) in every precision;
  * forces: max_i |F_i - F_i^oracle| / S_i <= 1e-5 (FP32 pair forces) and
    <= 1e-12 (FP64), S_i = sum_j |F_ij| the per-particle sum of pair-force
    magnitudes (the scale of the sum F_i = sum_j F_ij);
  * E_pot: relative 1e-5 (FP32) / 1e-12 (FP64); W (a sum of terms of both
    signs that crosses zero as a fluid equilibrates): |dW| <= tol * W_abs
    with W_abs = sum_{i<j} |f_ij| r_ij^2 <= rc/2 sum_i S_i;
  * 10-step trajectories: max min-image |dx| <= 1e-4 sigma and
    max |dv| <= 1e-4 v_rms.
"""
import numpy as np
import pytest

import oracle
from forcecheck import figures, pair_scale, report
from paper_2406_04210_gb300 import inputs

pytestmark = pytest.mark.gpu

PRECS = ["mixed_ds", "mixed_fp64", "fp64"]
FTOL = {"mixed_ds": 1e-5, "mixed_fp64": 1e-5, "fp64": 1e-12}
ETOL = {"mixed_ds": 1e-5, "mixed_fp64": 1e-5, "fp64": 1e-12}


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


def thermo_close(th, ref, wabs, tol=1e-5):
    """Per-step (E_pot, E_kin, W, T) against the oracle's."""
    np.testing.assert_allclose(th[:, [0, 1, 3]], ref[:, [0, 1, 3]], rtol=tol, atol=1e-8)
    assert np.abs(th[:, 2] - ref[:, 2]).max() <= tol * wabs


def check_lists(b, s, rl):
    count, nbr, pos_used = b.nlist()
    np.testing.assert_array_equal(pos_used, np.mod(s.pos, s.box))   # built from the inputs
    ref = oracle.nlist(s.box, pos_used, rl, use_cells=True)
    assert np.array_equal(count, ref.count)
    for i in range(s.n):
        got = np.sort(nbr[i, : count[i]])
        assert np.array_equal(got, ref.list[i, : ref.count[i]]), i


@pytest.mark.parametrize("prec", PRECS)
def test_lj4000_lists_forces_energy(ljmd, prec):
    s = inputs.lj4000()
    b = ljmd.from_system(s, prec)
    check_lists(b, s, 2.5 + 0.3)
    f, e, w = b.force()
    lj = _lj(s)
    fo, eo, wo = oracle.forces(s.box, s.pos, lj)
    S = pair_scale(s.box, s.pos, lj)
    err = np.linalg.norm(f - fo, axis=1) / S
    report(f"lj4000 {prec}", figures(f, fo, S))
    assert err.max() <= FTOL[prec], err.max()
    assert abs(e[0] - eo) <= ETOL[prec] * abs(eo)
    assert abs(w[0] - wo) <= ETOL[prec] * 0.5 * 2.5 * S.sum()


@pytest.mark.parametrize("prec", PRECS)
def test_lj4000_ten_steps(ljmd, prec):
    s = inputs.lj4000()
    b = ljmd.from_system(s, prec)
    th = b.integrate(s.dt, 10)
    pos, vel, img = b.get_state()
    r = oracle.run(s.box, s.pos, s.vel, _lj(s), s.skin, s.dt, 10)
    d = pos - r["pos"]
    d -= s.box * np.rint(d / s.box)
    vrms = np.sqrt(np.mean(s.vel ** 2))
    assert np.abs(d).max() <= 1e-4
    assert np.abs(vel - r["vel"]).max() <= 1e-4 * vrms
    np.testing.assert_array_equal(img, r["img"])
    # thermo after every step: E_pot, E_kin, W, T
    wabs = 0.5 * 2.5 * pair_scale(s.box, s.pos, _lj(s)).sum()
    thermo_close(th[:, 0, :], r["thermo"], wabs)


@pytest.mark.parametrize("prec", PRECS)
def test_lj4000_rebuild_parity_after_motion(ljmd, prec):
    # lists rebuilt during a run still equal the FP64 definition at the
    # positions they were built from
    s = inputs.lj4000()
    b = ljmd.from_system(s, prec)
    b.integrate(s.dt, 60, thermo=False)
    assert b.info().rebuilds >= 2
    b.neighbour_update(force=True)
    count, nbr, pos_used = b.nlist()
    ref = oracle.nlist(s.box, pos_used, 2.8)
    assert np.array_equal(count, ref.count)
    for i in range(s.n):
        assert np.array_equal(np.sort(nbr[i, : count[i]]), ref.list[i, : ref.count[i]])


def test_binary_mixture_parity(ljmd):
    s = inputs.binary_random_system(n=3000, seed=17)
    lj = _lj(s)
    pos, it, fmax = oracle.fire(s.box, s.pos, lj, s.type, maxit=300, ftol=1e-2)
    s.pos = pos
    for prec in PRECS:
        b = ljmd.from_system(s, prec)
        rl = float(s.rcut.max()) + s.skin
        check_lists(b, s, rl)
        f, e, w = b.force()
        fo, eo, wo = oracle.forces(s.box, s.pos, lj, s.type)
        S = pair_scale(s.box, s.pos, lj, s.type)
        report(f"binary3000 {prec}", figures(f, fo, S))
        assert (np.linalg.norm(f - fo, axis=1) / S).max() <= FTOL[prec]
        assert abs(e[0] - eo) <= ETOL[prec] * abs(eo)
        th = b.integrate(s.dt, 10)
        r = oracle.run(s.box, s.pos, s.vel, lj, s.skin, s.dt, 10, type_=s.type)
        p2, v2, _ = b.get_state()
        d = p2 - r["pos"]
        d -= s.box * np.rint(d / s.box)
        assert np.abs(d).max() <= 1e-4


@pytest.mark.parametrize("n,L", [(1, 9.0), (2, 9.0), (60, 5.7), (200, 8.5), (700, 8.41)])
def test_small_and_degenerate_boxes(ljmd, n, L):
    # 1-2 particles, 2 cells per dimension (L < 3 rl) and exactly 3 cells
    rng = np.random.default_rng(n)
    box = np.array([L, L, L])
    pos = rng.uniform(0, L, size=(n, 3)) if n > 2 else np.array([[0.1, 1, 1], [L - 0.9, 1, 1]])[:n]
    if n > 2:
        pos, _, _ = oracle.fire(box, pos, oracle.LJ.single(), maxit=200, ftol=1.0)
    vel = rng.normal(0, 0.5, size=(n, 3))
    b = ljmd.Box(pos, box, vel, precision="fp64")
    b.set_lj(1.0, 1.0, 2.5, 0.3)
    s = inputs.System(box, pos, vel, np.zeros(n, np.int32), np.ones((1, 1)), np.ones((1, 1)),
                      np.full((1, 1), 2.5))
    check_lists(b, s, 2.8)
    f, e, w = b.force()
    fo, eo, wo = oracle.forces_brute(box, pos, oracle.LJ.single())
    np.testing.assert_allclose(f, fo, rtol=0, atol=1e-11 * max(1.0, np.abs(fo).max()))


@pytest.mark.parametrize("scale", [1.5, 2.0])
def test_one_and_two_cells_per_edge(ljmd, scale):
    # cells larger than a third of the box: 2 (scale 1.5) or 1 (scale 2.0)
    # cell per edge, so neighbour cells repeat with different image shifts
    n, L = 700, 8.41
    rng = np.random.default_rng(n)
    box = np.array([L, L, L])
    pos = rng.uniform(0, L, size=(n, 3))
    pos, _, _ = oracle.fire(box, pos, oracle.LJ.single(), maxit=200, ftol=1.0)
    b = ljmd.Box(pos, box, None, precision="mixed_ds")
    b.set_lj(1.0, 1.0, 2.5, 0.3)
    b.set_layout(cell_scale=scale)
    s = inputs.System(box, pos, np.zeros((n, 3)), np.zeros(n, np.int32), np.ones((1, 1)), np.ones((1, 1)),
                      np.full((1, 1), 2.5))
    check_lists(b, s, 2.8)
    f, e, w = b.force()
    fo, eo, wo = oracle.forces_brute(box, pos, oracle.LJ.single())
    S = pair_scale(box, pos, oracle.LJ.single())
    assert (np.linalg.norm(f - fo, axis=1) / S).max() <= 1e-5


def test_cell_faces_and_boundaries(ljmd):
    # particles exactly on cell faces, at x = 0 and just below L
    rl = 2.8
    L = 3 * rl
    box = np.array([L, L, L])
    g = np.arange(0, L, rl / 2)
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    pos[::5, 1] = np.nextafter(L, 0)
    n = pos.shape[0]
    b = ljmd.Box(pos, box, None, precision="mixed_ds")
    b.set_lj(1.0, 1.0, 2.5, 0.3)
    s = inputs.System(box, pos, np.zeros((n, 3)), np.zeros(n, np.int32), np.ones((1, 1)),
                      np.ones((1, 1)), np.full((1, 1), 2.5))
    check_lists(b, s, rl)


def test_batched_replicas_match_single_boxes(ljmd):
    systems = inputs.replica_systems(nrep=6, nmin=500, nmax=3000, seed=5)
    n = [x.n for x in systems]
    pos = np.concatenate([x.pos for x in systems])
    vel = np.concatenate([x.vel for x in systems])
    box = np.stack([x.box for x in systems])
    b = ljmd.Box(pos, box, vel, n=n, precision="mixed_ds")
    b.set_lj(1.0, 1.0, 2.5, 0.3)
    f, e, w = b.force()
    th = b.integrate(0.005, 10)
    p2, v2, _ = b.get_state()
    o = 0
    for r, x in enumerate(systems):
        lj = _lj(x)
        fo, eo, wo = oracle.forces(x.box, x.pos, lj)
        S = pair_scale(x.box, x.pos, lj)
        assert (np.linalg.norm(f[o:o + x.n] - fo, axis=1) / S).max() <= 1e-5
        assert abs(e[r] - eo) <= 1e-5 * abs(eo)
        rr = oracle.run(x.box, x.pos, x.vel, lj, 0.3, 0.005, 10)
        d = p2[o:o + x.n] - rr["pos"]
        d -= x.box * np.rint(d / x.box)
        assert np.abs(d).max() <= 1e-4
        thermo_close(th[:, r, :], rr["thermo"], 0.5 * 2.5 * S.sum())
        o += x.n


def test_replicas_rebuilding_at_different_steps_keep_exact_lists(ljmd):
    # replicas at different temperatures rebuild at different steps: each
    # rebuild visits only the rebuilding replicas' cells and chunks; every
    # replica's lists still equal the FP64 definition at the positions they
    # were built from
    systems = inputs.replica_systems(nrep=6, nmin=500, nmax=3000, seed=11, T_range=(0.5, 2.5))
    n = [x.n for x in systems]
    pos = np.concatenate([x.pos for x in systems])
    vel = np.concatenate([x.vel for x in systems])
    box = np.stack([x.box for x in systems])
    b = ljmd.Box(pos, box, vel, n=n, precision="mixed_ds")
    b.set_lj(1.0, 1.0, 2.5, 0.3)
    b.integrate(0.005, 60, thermo=False)
    assert b.info().rebuilds >= 3
    count, nbr, pos_used = b.nlist()
    o = 0
    for x in systems:
        ref = oracle.nlist(x.box, pos_used[o:o + x.n], 2.8)
        assert np.array_equal(count[o:o + x.n], ref.count)
        for i in range(x.n):
            got = np.sort(nbr[o + i, : count[o + i]]) - o
            assert np.array_equal(got, ref.list[i, : ref.count[i]]), i
        o += x.n


def test_capacity_overflow_recovers(ljmd):
    s = inputs.lj4000()
    ref = ljmd.from_system(s, "mixed_ds")
    th_ref = ref.integrate(s.dt, 200)
    b = ljmd.from_system(s, "mixed_ds")
    count, _, _ = b.nlist()
    # full rows (capacities are whole blocks of 16 entries; the longest list
    # here grows from 79 to 83 entries within 40 steps): a later build overflows
    b.set_tuning(capacity=int((count.max() + 15) // 16 * 16))
    k0 = b.info().capacity
    th = b.integrate(s.dt, 200)
    assert b.info().capacity > k0
    # same trajectory up to FP32 summation order
    np.testing.assert_allclose(th[:, 0, 0], th_ref[:, 0, 0], rtol=1e-4)
    # a capacity below the largest list forces an immediate regrow
    b.set_tuning(capacity=8)
    assert b.info().capacity > 8
    check_lists(b, inputs.System(s.box, b.nlist()[2], s.vel, s.type, s.eps, s.sigma, s.rcut),
                2.8)


@pytest.mark.parametrize("prec", PRECS)
def test_energy_conservation(ljmd, prec):
    s = inputs.fcc_system(8, seed=3)    # 2048 particles
    b = ljmd.from_system(s, prec)
    th = b.integrate(s.dt, 2000)
    E = th[:, 0, 0] + th[:, 0, 1]
    assert np.abs(E - E[0]).max() / s.n < 5e-4
    # no systematic drift beyond the fluctuation level
    slope = np.polyfit(np.arange(E.size) * s.dt, E / s.n, 1)[0]
    assert abs(slope) < 1e-4


def test_deterministic(ljmd):
    s = inputs.lj4000()
    out = []
    for _ in range(2):
        b = ljmd.from_system(s, "mixed_ds")
        th = b.integrate(s.dt, 50)
        out.append((b.get_state()[0], th))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])


def test_conditional_and_plain_step_graphs_agree(ljmd):
    # the list update as a conditional graph node (default) or as kernels that
    # exit early: the same trajectory bit for bit, fewer launches with the node
    s = inputs.lj4000()
    out = []
    for cond in (True, False):
        b = ljmd.from_system(s, "mixed_ds")
        b.graph_conditional = cond
        assert b.graph_conditional == cond
        l0 = b.info().launches
        th = b.integrate(s.dt, 50)
        out.append((b.get_state()[0], th, b.info().launches - l0, b.info().rebuilds))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
    assert out[0][3] == out[1][3] >= 1
    assert out[0][2] < out[1][2]


def test_set_state_roundtrip(ljmd):
    s = inputs.lj4000()
    b = ljmd.from_system(s, "mixed_fp64")
    b.integrate(s.dt, 20, thermo=False)
    p, v, _ = b.get_state()
    c = ljmd.from_system(s, "mixed_fp64")
    c.set_state(p, v)
    np.testing.assert_allclose(c.get_state()[0], np.mod(p, s.box), rtol=0, atol=1e-12)
    fa, ea, _ = b.force()
    fb, eb, _ = c.force()
    assert abs(ea[0] - eb[0]) < 1e-5 * abs(ea[0])


def test_box_too_small_rejected(ljmd):
    b = ljmd.Box(np.zeros((4, 3)) + 1.0, [5.0, 5.0, 5.0])
    with pytest.raises(ljmd.MDError) as ei:
        b.set_lj(1.0, 1.0, 2.5, 0.3)
    assert ei.value.status == 5


def test_layout_kernel_and_graph_options_are_checked(ljmd):
    # out-of-range options are refused with MD_ERR_ARG and change nothing
    s = inputs.lj4000()
    b = ljmd.from_system(s, "mixed_ds")
    lib, h = b._lib, b._h
    assert lib.md_set_layout(h, 0.9, 0) == 1          # cell edge below the list radius
    assert lib.md_set_layout(h, float("nan"), 0) == 1
    assert lib.md_set_layout(h, 1.0, 2) == 1          # no such order
    assert lib.md_set_list_kernel(h, 3) == 1
    assert lib.md_set_list_kernel(h, -1) == 1
    assert lib.md_set_graph_conditional(h, 2) == 1
    assert b.layout() == {"cell_scale": 1.0, "order": "zrun"}
    assert b.list_kernel == "auto" and not b.graph_conditional
    check_lists(b, s, 2.8)


def test_torch_device_arrays(ljmd):
    import torch
    s = inputs.lj4000()
    pos = torch.tensor(s.pos, device="cuda")
    vel = torch.tensor(s.vel, device="cuda")
    b = ljmd.Box(pos, s.box, vel, precision="mixed_ds")
    b.set_lj(1.0, 1.0, 2.5, 0.3)
    out = torch.zeros((s.n, 3), dtype=torch.float64, device="cuda")
    b.force(out=out)
    fh, _, _ = b.force()
    np.testing.assert_array_equal(out.cpu().numpy(), fh)


def test_autotune_keeps_results(ljmd):
    s = inputs.lj4000()
    b = ljmd.from_system(s, "mixed_ds")
    f0, e0, _ = b.force()
    t = b.autotune(reps=2, cache=False)
    assert 1 <= t["force_blocks_per_sm"] <= 32 and 1 <= t["list_blocks_per_sm"] <= 32
    assert 1 <= t["segment_cells"] <= 16
    assert t["list_kernel"] in ("lanes", "quads") and b.list_kernel == t["list_kernel"]
    assert t["force_kernel"] in ("chunks", "tiles") and b.force_kernel == t["force_kernel"]
    f1, e1, _ = b.force()
    S = pair_scale(s.box, s.pos, _lj(s))
    assert (np.linalg.norm(f1 - f0, axis=1) / S).max() <= 1e-5
    check_lists(b, s, 2.8)
    b.set_tuning(segment_cells=1, force_blocks_per_sm=2)
    th = b.integrate(s.dt, 10)
    r = oracle.run(s.box, s.pos, s.vel, _lj(s), s.skin, s.dt, 10)
    d = b.get_state()[0] - r["pos"]
    d -= s.box * np.rint(d / s.box)
    assert np.abs(d).max() <= 1e-4


def test_autotune_keeps_a_chosen_list_kernel(ljmd):
    s = inputs.lj4000()
    b = ljmd.from_system(s, "mixed_ds")
    b.list_kernel = "quads"
    t = b.autotune(reps=1, cache=False)
    assert t["list_kernel"] == "quads" and b.list_kernel == "quads"
    check_lists(b, s, 2.8)


@pytest.mark.parametrize("scale,order", [(1.0, "morton"), (1.3, "zrun"), (1.3, "morton")])
def test_cell_layouts_keep_lists_forces_and_trajectories(ljmd, scale, order):
    # the binning's layout options (cell edge over the list radius, order
    # inside cells) change neither the lists (the FP64 definition) nor, beyond
    # FP32 summation order, the forces and trajectories
    s = inputs.lj4000()
    b = ljmd.from_system(s, "mixed_ds")
    b.set_layout(cell_scale=scale, order=order)
    assert b.layout() == {"cell_scale": scale, "order": order}
    check_lists(b, s, 2.8)
    f, e, w = b.force()
    lj = _lj(s)
    fo, eo, wo = oracle.forces(s.box, s.pos, lj)
    S = pair_scale(s.box, s.pos, lj)
    assert (np.linalg.norm(f - fo, axis=1) / S).max() <= 1e-5
    assert abs(e[0] - eo) <= 1e-5 * abs(eo)
    b.integrate(s.dt, 10)
    pos, vel, img = b.get_state()
    r = oracle.run(s.box, s.pos, s.vel, lj, s.skin, s.dt, 10)
    d = pos - r["pos"]
    d -= s.box * np.rint(d / s.box)
    assert np.abs(d).max() <= 1e-4
    np.testing.assert_array_equal(img, r["img"])
    b.neighbour_update(force=True)
    count, nbr, pos_used = b.nlist()
    ref = oracle.nlist(s.box, pos_used, 2.8)
    assert np.array_equal(count, ref.count)


def test_a_layout_whose_tiles_overflow_is_refused_and_the_old_one_kept(ljmd):
    # lj4000 at 1.7 list radii per cell edge: 3 cells a side, ~148 particles a
    # cell, so the 27 cells around any cell hold all 4000 particles, more than
    # the quad kernel's tile addresses.  The box keeps its layout and correct
    # lists.  (The lane kernel has no tile: there the layout is accepted.)
    s = inputs.lj4000()
    b = ljmd.from_system(s, "mixed_ds")
    b.list_kernel = "quads"
    b.set_layout(cell_scale=1.3, order="morton")
    with pytest.raises(ljmd.MDError) as ei:
        b.set_layout(cell_scale=1.7, order="zrun")
    assert "2048" in str(ei.value)
    assert b.layout() == {"cell_scale": 1.3, "order": "morton"}
    check_lists(b, s, 2.8)
    f, e, w = b.force()
    lj = _lj(s)
    fo, eo, wo = oracle.forces(s.box, s.pos, lj)
    S = pair_scale(s.box, s.pos, lj)
    assert (np.linalg.norm(f - fo, axis=1) / S).max() <= 1e-5


@pytest.mark.parametrize("kind", ["quads", "lanes"])
@pytest.mark.parametrize("case", ["lj4000", "binary3000", "lj4000_big_cells", "fcc2048_regrow", "lj4000_3_cells"])
def test_both_list_kernels_build_the_fp64_lists(ljmd, kind, case):
    # the quad kernel (candidates over lanes) and the lane kernel (particles
    # over lanes) build the same sets, equal to the FP64 definition; big
    # cells (62 particles a cell) take the lane kernel's two-pass path, and a
    # capacity of 16 makes both overflow and regrow
    if case == "binary3000":
        s = inputs.binary_random_system(n=3000, seed=17)
        s.pos = oracle.fire(s.box, s.pos, _lj(s), s.type, maxit=300, ftol=1e-2)[0]
    elif case == "fcc2048_regrow":
        s = inputs.fcc_system(8, seed=3)
    else:
        s = inputs.lj4000()
    b = ljmd.from_system(s, "mixed_ds")
    b.list_kernel = kind
    assert b.list_kernel == kind
    if case == "lj4000_big_cells":
        b.set_layout(cell_scale=1.3)
    if case == "lj4000_3_cells":
        # 148 particles a cell: five passes of 32 lanes per cell; beyond the
        # quad kernel's tile
        if kind == "quads":
            pytest.skip("a 27-cell tile over 2048 particles: refused by the quad kernel")
        b.set_layout(cell_scale=1.7)
    if case == "fcc2048_regrow":
        b.set_tuning(capacity=16)
    b.neighbour_update(force=True)
    rl = float(np.max(s.rcut)) + s.skin
    check_lists(b, s, rl)
    f, e, w = b.force()
    lj = _lj(s)
    fo, eo, wo = oracle.forces(s.box, s.pos, lj, s.type)
    S = pair_scale(s.box, s.pos, lj, s.type)
    assert (np.linalg.norm(f - fo, axis=1) / S).max() <= 1e-5
    assert abs(e[0] - eo) <= 1e-5 * abs(eo)
