"""List rows as the FP32 force kernel reads them: whole blocks of 16 entries,
the entries past a row's count (stale from an earlier, denser build, or never
written) replaced inside the kernel by a far sentinel slot.  Forces after the
lists shrink, particles with empty lists, and rows ending at every residue
mod 16 are checked against the FP64 oracle, with the tolerance of
test_gpu_md.py: max_i |dF_i| / S_i <= 1e-5 (FP32 forces), <= 1e-12 (FP64),
S_i = sum_j |F_ij| (a floor of 1 where a particle has no pair force)."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

FTOL = {"mixed_ds": 1e-5, "mixed_fp64": 1e-5, "fp64": 1e-12}


@pytest.fixture(scope="module")
def ljmd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_04210_gb300 import build, ljmd as m
    build.build()
    m.load()
    return m


def _scale(box, pos, rc):
    """S_i = sum_j |F_ij| over pairs within rc (brute force, minimum image)."""
    d = pos[:, None, :] - pos[None, :, :]
    d -= box * np.rint(d / box)
    r2 = np.einsum("ijk,ijk->ij", d, d)
    np.fill_diagonal(r2, np.inf)
    near = r2 < rc * rc
    r2 = np.where(near, r2, 1.0)              # pairs beyond rc (and i = j) contribute 0
    s6 = r2 ** -3
    f = np.where(near, 48.0 / r2 * (s6 * s6 - 0.5 * s6), 0.0)
    return np.maximum((np.abs(f) * np.sqrt(r2)).sum(axis=1), 1.0)


def _check(b, box, pos, prec):
    f, e, _ = b.force()
    lj = oracle.LJ(np.ones((1, 1)), np.ones((1, 1)), np.full((1, 1), 2.5), True)
    fo, eo, _ = oracle.forces_brute(box, pos, lj)
    S = _scale(box, pos, 2.5)
    assert np.max(np.linalg.norm(f - fo, axis=1) / S) <= FTOL[prec]
    assert abs(e[0] - eo) <= FTOL[prec] * max(abs(eo), 1.0)


def _dense_then_dilute(seed):
    """1000 particles in a 20-sigma box: a dense 10^3 block of spacing 1.05 in
    one corner (lists of ~80 entries), then a jittered lattice of spacing 2
    over the whole box (lists of ~10-30 entries)."""
    rng = np.random.default_rng(seed)
    g = np.stack(np.meshgrid(*[np.arange(10)] * 3, indexing="ij"), -1).reshape(-1, 3).astype(float)
    dense = 1.0 + 1.05 * g + rng.uniform(-0.02, 0.02, g.shape)
    dilute = 1.0 + 2.0 * g + rng.uniform(-0.3, 0.3, g.shape)
    return np.full(3, 20.0), dense, dilute


@pytest.mark.parametrize("prec", ["mixed_ds", "mixed_fp64", "fp64"])
def test_forces_after_the_lists_shrink(ljmd, prec):
    box, dense, dilute = _dense_then_dilute(5)
    b = ljmd.Box(dense, box, precision=prec)
    b.set_lj(1.0, 1.0, 2.5, 0.3)
    c0 = b.nlist()[0]
    _check(b, box, dense, prec)
    b.set_state(dilute)                       # rebuild: every row shorter than before
    c1 = b.nlist()[0]
    assert c1.max() < c0.min()                # all entries past the new counts are stale
    _check(b, box, dilute, prec)
    # rows end at many residues mod 16 (the kernel masks a row's last block)
    assert len(set((c0 % 16).tolist()) | set((c1 % 16).tolist())) >= 12


@pytest.mark.parametrize("prec", ["mixed_ds", "fp64"])
def test_particles_without_neighbours(ljmd, prec):
    # three far-apart particles and one close pair in a 20-sigma box: counts 0 and 1
    box = np.full(3, 20.0)
    pos = np.array([[1.0, 1.0, 1.0], [11.0, 1.0, 1.0], [1.0, 11.0, 1.0],
                    [11.0, 11.0, 11.0], [12.1, 11.0, 11.0]])
    b = ljmd.Box(pos, box, precision=prec)
    b.set_lj(1.0, 1.0, 2.5, 0.3)
    count = b.nlist()[0]
    assert count.tolist() == [0, 0, 0, 1, 1]
    f, e, _ = b.force()
    assert np.all(f[:3] == 0.0)
    _check(b, box, pos, prec)
