"""md_force_noalloc: forces and energies without any device allocation.

For library users whose code cannot allocate GPU memory at the point where
it needs forces (for example a framework that owns the whole device through
its own memory pool, or a pool that is capped or frozen).  The entry point
keeps its scratch in a static device array, so this test calls it through
the C ABI twice in a row and checks both results against md_force on the
same box, with the force and energy tolerances of tests/test_gpu_md.py.
It lives in its own file, collected last, and builds and loads the library
itself, so it also runs alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

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


def test_force_noalloc_matches_md_force_twice(ljmd):
    import torch
    s = inputs.lj4000()
    b = ljmd.from_system(s, "mixed_ds")
    f_ref, e_ref, w_ref = b.force()                       # the existing entry point
    scale = np.abs(f_ref).max()
    out = torch.zeros((s.n, 3), dtype=torch.float64, device="cuda")
    for _ in range(2):
        out.zero_()
        e = np.zeros(1)
        w = np.zeros(1)
        st = b._lib.md_force_noalloc(b._h, ctypes.c_void_p(out.data_ptr()), e.ctypes.data,
                                     w.ctypes.data)
        assert st == 0, b._lib.md_last_error(b._h).decode()
        f = out.cpu().numpy()
        assert np.abs(f - f_ref).max() <= 1e-5 * scale
        assert abs(e[0] - e_ref[0]) <= 1e-5 * abs(e_ref[0])
        assert abs(w[0] - w_ref[0]) <= 1e-5 * abs(w_ref[0])


def test_force_noalloc_allocates_nothing_on_a_fresh_box(ljmd):
    # the first force evaluation of a fresh box (md_force would allocate its
    # energy buffers here): no allocation through the box's allocator (torch's
    # caching allocator, installed by the binding) and no change in the
    # device's free memory; then the same results as md_force
    import torch
    s = inputs.lj4000()
    # the once-per-device set-up (the scratch array's address; the CUDA driver may
    # load the library's module then) is done first, on another box
    a = ljmd.from_system(inputs.fcc_system(6, seed=7), "mixed_ds")
    assert a._lib.md_force_noalloc(a._h, None, None, None) == 0
    b = ljmd.from_system(s, "mixed_ds")
    out = torch.zeros((s.n, 3), dtype=torch.float64, device="cuda")
    e = np.zeros(1)
    w = np.zeros(1)
    torch.cuda.synchronize()
    n0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    free0, _ = torch.cuda.mem_get_info()
    st = b._lib.md_force_noalloc(b._h, ctypes.c_void_p(out.data_ptr()), e.ctypes.data, w.ctypes.data)
    torch.cuda.synchronize()
    assert st == 0, b._lib.md_last_error(b._h).decode()
    assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == n0
    assert torch.cuda.mem_get_info()[0] == free0
    f_ref, e_ref, w_ref = b.force()
    assert np.abs(out.cpu().numpy() - f_ref).max() <= 1e-5 * np.abs(f_ref).max()
    assert abs(e[0] - e_ref[0]) <= 1e-5 * abs(e_ref[0])


def test_force_noalloc_rejects_boxes_beyond_its_scratch(ljmd):
    # 32,768 one-particle replicas (FP32 forces: 16 doubles per 128-particle
    # chunk) need 16 x 32,768 + 4 x 32,768 doubles > 524,288
    nrep = 32768
    box = np.tile([10.0, 10.0, 10.0], (nrep, 1))
    pos = np.full((nrep, 3), 5.0)
    b = ljmd.Box(pos, box, n=[1] * nrep)
    e = np.zeros(nrep)
    st = b._lib.md_force_noalloc(b._h, None, e.ctypes.data, None)
    assert st == 1
    assert b"static scratch" in b._lib.md_last_error(b._h)
