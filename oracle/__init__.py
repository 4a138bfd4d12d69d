"""FP64 CPU oracle for truncated Lennard-Jones MD (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline /
reference arm may import this package.  It wraps ``ljmd_oracle.c`` (plain C,
FP64, sequential sums, compiled with ``-ffp-contract=off``) through ctypes and
shares nothing with the CUDA product path.

Parity status per function is listed in the header of ``ljmd_oracle.c``; every
function is pinned by ``tests/test_oracle.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ljmd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libljmd_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -O2, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math",
             "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_I64 = ctypes.POINTER(ctypes.c_int64)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.or_pair.argtypes = [ctypes.c_double] * 3 + [ctypes.c_int32, ctypes.c_double, _D]
            L.or_pair.restype = None
            L.or_min_image.argtypes = [ctypes.c_double, ctypes.c_double]
            L.or_min_image.restype = ctypes.c_double
            L.or_forces_brute.argtypes = [ctypes.c_int64, _D, ctypes.c_int32, _I32, _D,
                                          _D, _D, _D, ctypes.c_int32, _D, _D, _D]
            L.or_forces_brute.restype = ctypes.c_int32
            L.or_nlist.argtypes = [ctypes.c_int64, _D, _D, ctypes.c_double, ctypes.c_int32,
                                   ctypes.c_int64, _I32, _I64]
            L.or_nlist.restype = ctypes.c_int64
            L.or_forces_list.argtypes = [ctypes.c_int64, _D, ctypes.c_int32, _I32, _D,
                                         _D, _D, _D, ctypes.c_int32, _I32, _I64,
                                         ctypes.c_int64, _D, _D, _D]
            L.or_forces_list.restype = ctypes.c_int32
            L.or_hvp.argtypes = [ctypes.c_int64, _D, ctypes.c_int32, _I32, _D, _D, _D, _D,
                                 _I32, _I64, ctypes.c_int64, _D, _D]
            L.or_hvp.restype = ctypes.c_int32
            L.or_dforce_dparam.argtypes = [ctypes.c_int64, _D, ctypes.c_int32, _I32, _D, _D,
                                           _D, _D, _I32, _I64, ctypes.c_int64, _D, _D, _D]
            L.or_dforce_dparam.restype = ctypes.c_int32
            L.or_run.argtypes = [ctypes.c_int64, _D, ctypes.c_int32, _I32, _D, _D, _I32,
                                 _D, _D, _D, ctypes.c_int32, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_int64, _D, _D,
                                 ctypes.c_double, ctypes.c_double, ctypes.c_uint64]
            L.or_run.restype = ctypes.c_int64
            L.or_philox4x32.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            L.or_philox4x32.restype = None
            L.or_thermostat.argtypes = [ctypes.c_int64, _D, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_uint64, ctypes.c_int64]
            L.or_thermostat.restype = ctypes.c_int64
            L.or_hist.argtypes = [ctypes.c_int64, _D, _D, _I32, _I64, ctypes.c_int64,
                                  ctypes.c_double, ctypes.c_int32, ctypes.c_double,
                                  ctypes.c_double, _D]
            L.or_hist.restype = ctypes.c_int32
            L.or_hist_grad.argtypes = [ctypes.c_int64, _D, _D, _I32, _I64, ctypes.c_int64,
                                       ctypes.c_double, ctypes.c_int32, ctypes.c_double,
                                       ctypes.c_double, _D, _D]
            L.or_hist_grad.restype = ctypes.c_int32
            L.or_adjoint.argtypes = [ctypes.c_int64, _D, ctypes.c_int32, _I32, _D, _D, _D,
                                     _D, ctypes.c_double, ctypes.c_int64, _D, _D, _D, _D,
                                     _D, _D]
            L.or_adjoint.restype = ctypes.c_int32
            L.or_fire.argtypes = [ctypes.c_int64, _D, ctypes.c_int32, _I32, _D, _D, _D, _D,
                                  ctypes.c_int64, ctypes.c_double, ctypes.c_double, _D]
            L.or_fire.restype = ctypes.c_int64
            _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_D)


def _i32(a):
    return a.ctypes.data_as(_I32)


def _i64(a):
    return a.ctypes.data_as(_I64)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


class LJ:
    """Pair parameter tables (ntypes x ntypes, symmetric) and energy shift."""

    def __init__(self, eps, sigma, rcut, shift=True):
        self.eps = _f64(np.atleast_2d(eps))
        self.sigma = _f64(np.atleast_2d(sigma))
        self.rcut = _f64(np.atleast_2d(rcut))
        self.ntypes = self.eps.shape[0]
        self.shift = 1 if shift else 0

    @classmethod
    def single(cls, eps=1.0, sigma=1.0, rcut=2.5, shift=True):
        return cls([[eps]], [[sigma]], [[rcut]], shift)


def pair(eps, sigma, rcut, shift, r2):
    """(f = -phi'/r, U, phi'', phi'/r) of one pair at squared distance r2."""
    out = np.zeros(4)
    lib().or_pair(eps, sigma, rcut, int(shift), r2, _d(out))
    return out


def min_image(d, L):
    return lib().or_min_image(float(d), float(L))


def _types(type_, n):
    if type_ is None:
        return np.zeros(n, dtype=np.int32)
    return np.ascontiguousarray(type_, dtype=np.int32)


def forces_brute(box, pos, lj: LJ, type_=None):
    pos = _f64(pos, (-1, 3))
    n = pos.shape[0]
    t = _types(type_, n)
    f = np.zeros((n, 3))
    e = np.zeros(1)
    w = np.zeros(1)
    lib().or_forces_brute(n, _d(_f64(box)), lj.ntypes, _i32(t), _d(pos), _d(lj.eps),
                          _d(lj.sigma), _d(lj.rcut), lj.shift, _d(f), _d(e), _d(w))
    return f, float(e[0]), float(w[0])


class NList:
    def __init__(self, count, list_, cap):
        self.count, self.list, self.cap = count, list_, cap

    def sets(self):
        return [self.list[i, : self.count[i]].copy() for i in range(len(self.count))]


def nlist(box, pos, rl, use_cells=True, cap=64):
    pos = _f64(pos, (-1, 3))
    n = pos.shape[0]
    box = _f64(box)
    while True:
        count = np.zeros(n, dtype=np.int32)
        lst = np.full((n, cap), -1, dtype=np.int64)
        m = lib().or_nlist(n, _d(box), _d(pos), float(rl), 1 if use_cells else 0, cap,
                           _i32(count), _i64(lst))
        if m < 0:
            raise MemoryError("oracle nlist")
        if m <= cap:
            return NList(count, lst, cap)
        cap = int(m) + 8


def forces_list(box, pos, lj: LJ, nl: NList, type_=None):
    pos = _f64(pos, (-1, 3))
    n = pos.shape[0]
    t = _types(type_, n)
    f = np.zeros((n, 3))
    e = np.zeros(1)
    w = np.zeros(1)
    lib().or_forces_list(n, _d(_f64(box)), lj.ntypes, _i32(t), _d(pos), _d(lj.eps),
                         _d(lj.sigma), _d(lj.rcut), lj.shift, _i32(nl.count),
                         _i64(nl.list), nl.cap, _d(f), _d(e), _d(w))
    return f, float(e[0]), float(w[0])


def forces(box, pos, lj: LJ, type_=None, use_cells=True):
    """Forces, E_pot, W at pos from a fresh cutoff list."""
    nl = nlist(box, pos, float(lj.rcut.max()), use_cells)
    return forces_list(box, pos, lj, nl, type_)


def hvp(box, pos, lj: LJ, u, type_=None, nl: NList | None = None):
    pos = _f64(pos, (-1, 3))
    n = pos.shape[0]
    if nl is None:
        nl = nlist(box, pos, float(lj.rcut.max()))
    t = _types(type_, n)
    u = _f64(u, (n, 3))
    out = np.zeros((n, 3))
    lib().or_hvp(n, _d(_f64(box)), lj.ntypes, _i32(t), _d(pos), _d(lj.eps), _d(lj.sigma),
                 _d(lj.rcut), _i32(nl.count), _i64(nl.list), nl.cap, _d(u), _d(out))
    return out


def dforce_dparam(box, pos, lj: LJ, lam, type_=None, nl: NList | None = None):
    pos = _f64(pos, (-1, 3))
    n = pos.shape[0]
    if nl is None:
        nl = nlist(box, pos, float(lj.rcut.max()))
    t = _types(type_, n)
    lam = _f64(lam, (n, 3))
    ge = np.zeros((lj.ntypes, lj.ntypes))
    gs = np.zeros((lj.ntypes, lj.ntypes))
    lib().or_dforce_dparam(n, _d(_f64(box)), lj.ntypes, _i32(t), _d(pos), _d(lj.eps),
                           _d(lj.sigma), _d(lj.rcut), _i32(nl.count), _i64(nl.list),
                           nl.cap, _d(lam), _d(ge), _d(gs))
    return ge, gs


def run(box, pos, vel, lj: LJ, skin, dt, nsteps, type_=None, img=None, traj=False, thermostat=None):
    """Velocity-Verlet MD.  Returns dict(pos, vel, img, thermo, builds[, traj]).
    thermostat = (T_bath, rate, seed): Andersen-like collisions after every
    finalize (see or_thermostat).  Every lj.rcut infinite: all pairs, no lists."""
    pos = _f64(pos, (-1, 3)).copy()
    vel = _f64(vel, (-1, 3)).copy()
    n = pos.shape[0]
    t = _types(type_, n)
    img = np.zeros((n, 3), dtype=np.int32) if img is None else np.array(img, dtype=np.int32)
    thermo = np.zeros((max(nsteps, 1), 4))
    tr = np.zeros((nsteps + 1, n, 3)) if traj else None
    T_bath, rate, seed = thermostat if thermostat is not None else (0.0, 0.0, 0)
    b = lib().or_run(n, _d(_f64(box)), lj.ntypes, _i32(t), _d(pos), _d(vel), _i32(img),
                     _d(lj.eps), _d(lj.sigma), _d(lj.rcut), lj.shift, float(skin),
                     float(dt), int(nsteps), _d(thermo), _d(tr) if traj else None,
                     float(T_bath), float(rate), ctypes.c_uint64(int(seed)))
    if b < 0:
        raise RuntimeError(f"oracle run failed ({b})")
    out = dict(pos=pos, vel=vel, img=img, thermo=thermo[:nsteps], builds=int(b))
    if traj:
        out["traj"] = tr
    return out


def philox4x32(ctr, key):
    """Philox4x32-10 of one 4-word counter and 2-word key (uint32)."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    o = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32(c.ctypes.data, k.ctypes.data, o.ctypes.data)
    return o


def thermostat(vel, T_bath, rate, dt, seed, step):
    """One thermostat application to a copy of vel; returns (vel, collisions)."""
    v = _f64(vel, (-1, 3)).copy()
    hits = lib().or_thermostat(v.shape[0], _d(v), float(T_bath), float(rate), float(dt),
                               ctypes.c_uint64(int(seed)), int(step))
    return v, int(hits)


def hist(box, pos, nbins=64, rhist=2.5, w=None, rmax_pairs=2.8):
    pos = _f64(pos, (-1, 3))
    n = pos.shape[0]
    w = rhist / nbins if w is None else w
    nl = nlist(box, pos, rmax_pairs)
    h = np.zeros(nbins)
    lib().or_hist(n, _d(_f64(box)), _d(pos), _i32(nl.count), _i64(nl.list), nl.cap,
                  float(rmax_pairs), int(nbins), float(rhist), float(w), _d(h))
    return h


def hist_grad(box, pos, coef, nbins=64, rhist=2.5, w=None, rmax_pairs=2.8):
    pos = _f64(pos, (-1, 3))
    n = pos.shape[0]
    w = rhist / nbins if w is None else w
    nl = nlist(box, pos, rmax_pairs)
    g = np.zeros((n, 3))
    lib().or_hist_grad(n, _d(_f64(box)), _d(pos), _i32(nl.count), _i64(nl.list), nl.cap,
                       float(rmax_pairs), int(nbins), float(rhist), float(w),
                       _d(_f64(coef)), _d(g))
    return g


def hist_loss(box, pos, target, nbins=64, rhist=2.5, w=None, rmax_pairs=2.8):
    """L = (1/nbins) sum_k (h_k - target_k)^2 and dL/dx."""
    h = hist(box, pos, nbins, rhist, w, rmax_pairs)
    diff = h - np.asarray(target, dtype=np.float64)
    loss = float(np.mean(diff * diff))
    g = hist_grad(box, pos, 2.0 * diff / nbins, nbins, rhist, w, rmax_pairs)
    return loss, g, h


def adjoint(box, traj, lj: LJ, dt, lx_T, lv_T, type_=None):
    traj = _f64(traj)
    nsteps = traj.shape[0] - 1
    n = traj.shape[1]
    t = _types(type_, n)
    lx0 = np.zeros((n, 3))
    lv0 = np.zeros((n, 3))
    ge = np.zeros((lj.ntypes, lj.ntypes))
    gs = np.zeros((lj.ntypes, lj.ntypes))
    rc = lib().or_adjoint(n, _d(_f64(box)), lj.ntypes, _i32(t), _d(traj), _d(lj.eps),
                          _d(lj.sigma), _d(lj.rcut), float(dt), nsteps,
                          _d(_f64(lx_T, (n, 3))), _d(_f64(lv_T, (n, 3))), _d(lx0), _d(lv0),
                          _d(ge), _d(gs))
    if rc != 0:
        raise RuntimeError(f"oracle adjoint failed ({rc})")
    return lx0, lv0, ge, gs


def fire(box, pos, lj: LJ, type_=None, maxit=2000, ftol=1e-3, dt0=0.002):
    pos = _f64(pos, (-1, 3)).copy()
    n = pos.shape[0]
    t = _types(type_, n)
    fm = np.zeros(1)
    it = lib().or_fire(n, _d(_f64(box)), lj.ntypes, _i32(t), _d(pos), _d(lj.eps),
                       _d(lj.sigma), _d(lj.rcut), int(maxit), float(ftol), float(dt0), _d(fm))
    if it < 0:
        raise RuntimeError("oracle fire failed")
    return pos, int(it), float(fm[0])


def thermo_T(vel):
    v = _f64(vel, (-1, 3))
    n = v.shape[0]
    return float(np.sum(v * v)) / (3.0 * n - 3.0)
