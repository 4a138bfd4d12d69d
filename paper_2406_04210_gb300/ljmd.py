"""Thin ctypes binding of libljmd.so (the C ABI of include/ljmd.h).

Argument marshalling only: every step of the MD path runs in the library's
CUDA kernels.  Array arguments may be numpy arrays (host) or torch CUDA
tensors (device); results are returned as numpy arrays unless a torch tensor
is passed to be filled.  Device memory of a box comes from PyTorch's caching
allocator through the library's allocator hook, and calls are ordered on the
current torch CUDA stream.

The library is loaded on first use; a missing library raises
:class:`LibraryMissing` (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "libljmd.so")

PREC = {"mixed_ds": 0, "mixed_fp64": 1, "fp64": 2}
STATUS = {0: "MD_OK", 1: "MD_ERR_ARG", 2: "MD_ERR_CUDA", 3: "MD_ERR_OOM", 4: "MD_ERR_CAPACITY",
          5: "MD_ERR_BOX_TOO_SMALL", 6: "MD_ERR_NONFINITE", 7: "MD_ERR_TIMEOUT",
          8: "MD_ERR_STATE"}

EXPORTS = ["md_set_allocator", "md_batch_create", "md_box_create", "md_box_destroy",
           "md_set_lj", "md_neighbour_update", "md_force", "md_integrate", "md_adjoint",
           "md_get_state", "md_set_state", "md_get_nlist", "md_get_info", "md_set_tuning",
           "md_get_tuning", "md_autotune", "md_set_layout", "md_get_layout",
           "md_set_list_kernel", "md_get_list_kernel", "md_set_force_kernel",
           "md_get_force_kernel", "md_set_graph_conditional",
           "md_get_graph_conditional",
           "md_set_profiling", "md_get_profile", "md_pair_hist", "md_force_noalloc",
           "md_set_thermostat",
           "md_last_error", "md_status_string"]


class LibraryMissing(RuntimeError):
    pass


class MDError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Info(ctypes.Structure):
    _fields_ = [("n_total", ctypes.c_int64), ("nrep", ctypes.c_int32),
                ("ntypes", ctypes.c_int32), ("capacity", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("ncell_total", ctypes.c_int64),
                ("rebuilds", ctypes.c_int64), ("steps", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("rlist", ctypes.c_double),
                ("launches", ctypes.c_int64), ("list_entries", ctypes.c_int64),
                ("record_id", ctypes.c_int64)]


_lock = threading.Lock()
_lib = None
_ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
_cb = []


def library_path() -> str:
    return _SO


def load(path: str | None = None):
    """Load libljmd.so (raises LibraryMissing if it was not built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or _SO
        if not os.path.exists(p):
            raise LibraryMissing(
                f"{p} is missing: build it with `python -m paper_2406_04210_gb300.build`")
        L = ctypes.CDLL(p)
        vp, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        L.md_set_allocator.argtypes = [_ALLOC, _FREE, vp]
        L.md_batch_create.argtypes = [ctypes.POINTER(vp), i32, vp, vp, vp, vp, vp, i32, vp]
        L.md_box_create.argtypes = [ctypes.POINTER(vp), i64, vp, vp, vp, vp, i32, vp]
        L.md_box_destroy.argtypes = [vp]
        L.md_set_lj.argtypes = [vp, i32, vp, vp, vp, d, i32]
        L.md_neighbour_update.argtypes = [vp, i32, vp]
        L.md_force.argtypes = [vp, vp, vp, vp]
        L.md_integrate.argtypes = [vp, d, i64, i32, vp]
        L.md_adjoint.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.md_get_state.argtypes = [vp, vp, vp, vp]
        L.md_set_state.argtypes = [vp, vp, vp]
        L.md_get_nlist.argtypes = [vp, vp, vp, i64, vp]
        L.md_get_info.argtypes = [vp, ctypes.POINTER(Info)]
        L.md_set_tuning.argtypes = [vp, vp]
        L.md_get_tuning.argtypes = [vp, vp]
        L.md_autotune.argtypes = [vp, i32, vp]
        L.md_set_layout.argtypes = [vp, d, i32]
        L.md_get_layout.argtypes = [vp, vp, vp]
        L.md_set_list_kernel.argtypes = [vp, i32]
        L.md_get_list_kernel.argtypes = [vp, vp]
        L.md_set_force_kernel.argtypes = [vp, i32]
        L.md_get_force_kernel.argtypes = [vp, vp]
        L.md_set_graph_conditional.argtypes = [vp, i32]
        L.md_get_graph_conditional.argtypes = [vp, vp]
        L.md_set_profiling.argtypes = [vp, i32]
        L.md_pair_hist.argtypes = [vp, i32, d, d, d, vp, vp, vp]
        L.md_force_noalloc.argtypes = [vp, vp, vp, vp]
        L.md_get_profile.argtypes = [vp, vp, vp]
        L.md_set_thermostat.argtypes = [vp, vp, d, ctypes.c_uint64]
        L.md_last_error.argtypes = [vp]
        L.md_last_error.restype = ctypes.c_char_p
        L.md_status_string.argtypes = [i32]
        L.md_status_string.restype = ctypes.c_char_p
        for name in EXPORTS:
            if name not in ("md_last_error", "md_status_string"):
                getattr(L, name).restype = i32
        _lib = L
        _install_torch_allocator(L)
        return L


def _install_torch_allocator(L):
    """Route the library's device allocations through torch's caching allocator."""
    try:
        import torch
    except ImportError:
        return
    if not torch.cuda.is_available():
        return

    def _alloc(nbytes, ctx):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes)))
        except Exception:   # out of memory: report NULL to the library
            return 0

    def _free(ptr, ctx):
        try:
            torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:
            pass

    a, f = _ALLOC(_alloc), _FREE(_free)
    _cb.extend([a, f])
    L.md_set_allocator(a, f, None)


def _ptr(x):
    """(pointer, keepalive) of a numpy array or torch tensor; None -> NULL."""
    if x is None:
        return None, None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            x = np.ascontiguousarray(x)
        return x.ctypes.data, x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor arguments must be contiguous")
        return x.data_ptr(), x
    raise TypeError(f"unsupported array type {type(x)}")


def _stream_handle(stream=None):
    try:
        import torch
        if torch.cuda.is_available():
            s = stream if stream is not None else torch.cuda.current_stream()
            return s.cuda_stream
    except ImportError:
        pass
    return None


class Box:
    """A batch of nrep periodic LJ boxes advanced by libljmd on one GPU."""

    def __init__(self, pos, box, vel=None, type=None, n=None, precision="mixed_ds",
                 stream=None):
        L = load()
        box = np.ascontiguousarray(np.atleast_2d(np.asarray(box, dtype=np.float64)))
        nrep = box.shape[0]
        if n is None:
            if nrep != 1:
                raise ValueError("n (particles per replica) is required for nrep > 1")
            n = [int(pos.shape[0])]
        n = np.ascontiguousarray(np.asarray(n, dtype=np.int64))
        self.nrep, self.n_total = nrep, int(n.sum())
        self.n = n
        pos = _as_f64(pos)
        vel = _as_f64(vel) if vel is not None else None
        type = _as_i32(type) if type is not None else None
        pp, kp = _ptr(pos)
        pv, kv = _ptr(vel)
        pt, kt = _ptr(type)
        h = ctypes.c_void_p()
        st = L.md_batch_create(ctypes.byref(h), nrep, n.ctypes.data, box.ctypes.data, pt, pp,
                               pv, PREC[precision], _stream_handle(stream))
        if st != 0:
            raise MDError(st, "md_batch_create failed")
        self._h = h
        self._lib = L
        self.precision = precision
        self.box = box

    # -- helpers --
    def _check(self, st, what):
        if st != 0:
            raise MDError(st, f"{what}: {self._lib.md_last_error(self._h).decode()}")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.md_box_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- ABI wrappers --
    def set_lj(self, eps=1.0, sigma=1.0, rcut=2.5, skin=0.3, shift=True):
        self._rcut, self._skin = rcut, skin
        eps = np.ascontiguousarray(np.atleast_2d(eps), dtype=np.float64)
        sigma = np.ascontiguousarray(np.atleast_2d(sigma), dtype=np.float64)
        rcut = np.ascontiguousarray(np.atleast_2d(rcut), dtype=np.float64)
        nt = eps.shape[0]
        self._check(self._lib.md_set_lj(self._h, nt, eps.ctypes.data, sigma.ctypes.data,
                                        rcut.ctypes.data, float(skin), 1 if shift else 0),
                    "md_set_lj")
        return self

    def set_thermostat(self, T_bath=None, rate=0.0, seed=0):
        """Andersen-like collisions at `rate` per unit time with a bath at
        T_bath (scalar or one value per replica); rate 0 switches it off."""
        if rate and T_bath is None:
            raise ValueError("T_bath is required with rate > 0")
        t = None
        if T_bath is not None:
            t = np.ascontiguousarray(np.broadcast_to(np.asarray(T_bath, dtype=np.float64), (self.nrep,)))
        self._check(self._lib.md_set_thermostat(self._h, t.ctypes.data if t is not None else None,
                                                float(rate), ctypes.c_uint64(int(seed))),
                    "md_set_thermostat")
        return self

    def neighbour_update(self, force=False):
        r = ctypes.c_int32(0)
        self._check(self._lib.md_neighbour_update(self._h, 1 if force else 0, ctypes.byref(r)),
                    "md_neighbour_update")
        return r.value

    def force(self, out=None):
        f = np.zeros((self.n_total, 3)) if out is None else out
        e = np.zeros(self.nrep)
        w = np.zeros(self.nrep)
        pf, kf = _ptr(f)
        self._check(self._lib.md_force(self._h, pf, e.ctypes.data, w.ctypes.data), "md_force")
        return f, e, w

    def integrate(self, dt, nsteps, thermo=True, ckpt_every=0, out=None):
        th = None
        if thermo:
            th = np.zeros((nsteps, self.nrep, 4)) if out is None else out
        pt, kt = _ptr(th)
        self._check(self._lib.md_integrate(self._h, float(dt), int(nsteps), int(ckpt_every), pt),
                    "md_integrate")
        return th

    def adjoint(self, lam_x, lam_v, out=None):
        lx0 = np.zeros((self.n_total, 3))
        lv0 = np.zeros((self.n_total, 3))
        info = self.info()
        ge = np.zeros((info.ntypes, info.ntypes))
        gs = np.zeros((info.ntypes, info.ntypes))
        a, ka = _ptr(_as_f64(lam_x))
        b, kb = _ptr(_as_f64(lam_v))
        self._check(self._lib.md_adjoint(self._h, a, b, lx0.ctypes.data, lv0.ctypes.data,
                                         ge.ctypes.data, gs.ctypes.data), "md_adjoint")
        return lx0, lv0, ge, gs

    def pair_hist(self, nbins=64, rhist=2.5, width=None, rmax=2.8, coef=None):
        """Smoothed pair-distance histogram (nrep x nbins) and, with coef, the
        gradient of sum(coef * h) with respect to the positions."""
        width = rhist / nbins if width is None else width
        h = np.zeros((self.nrep, nbins))
        g = np.zeros((self.n_total, 3)) if coef is not None else None
        c = np.ascontiguousarray(np.broadcast_to(np.asarray(coef, dtype=np.float64),
                                                 (self.nrep, nbins))) if coef is not None else None
        pc, kc = _ptr(c)
        pg, kg = _ptr(g)
        self._check(self._lib.md_pair_hist(self._h, int(nbins), float(rhist), float(width),
                                           float(rmax), pc, h.ctypes.data, pg), "md_pair_hist")
        return h, g

    def get_state(self):
        pos = np.zeros((self.n_total, 3))
        vel = np.zeros((self.n_total, 3))
        img = np.zeros((self.n_total, 3), dtype=np.int32)
        self._check(self._lib.md_get_state(self._h, pos.ctypes.data, vel.ctypes.data,
                                           img.ctypes.data), "md_get_state")
        return pos, vel, img

    def set_state(self, pos, vel=None):
        pp, kp = _ptr(_as_f64(pos))
        pv, kv = _ptr(_as_f64(vel) if vel is not None else None)
        self._check(self._lib.md_set_state(self._h, pp, pv), "md_set_state")

    def nlist(self, cap=None):
        count = np.zeros(self.n_total, dtype=np.int32)
        info = self.info()
        cap = cap or info.capacity
        nbr = np.full((self.n_total, cap), -1, dtype=np.int64)
        pos = np.zeros((self.n_total, 3))
        self._check(self._lib.md_get_nlist(self._h, count.ctypes.data, nbr.ctypes.data, cap,
                                           pos.ctypes.data), "md_get_nlist")
        return count, nbr, pos

    def info(self) -> Info:
        i = Info()
        self._check(self._lib.md_get_info(self._h, ctypes.byref(i)), "md_get_info")
        return i

    TUNING = ("force_blocks_per_sm", "list_blocks_per_sm", "segment_cells", "capacity")

    def tuning(self):
        t = np.zeros(4, dtype=np.int32)
        self._check(self._lib.md_get_tuning(self._h, t.ctypes.data), "md_get_tuning")
        return dict(zip(self.TUNING, (int(x) for x in t)))

    def set_tuning(self, **kw):
        """Set any of force_blocks_per_sm, list_blocks_per_sm, segment_cells,
        capacity (0 = automatic); the others keep their current values."""
        cur = self.tuning()
        unknown = set(kw) - set(self.TUNING)
        if unknown:
            raise TypeError(f"unknown tuning keys {sorted(unknown)}")
        cur.update(kw)
        t = np.array([cur[k] for k in self.TUNING], dtype=np.int32)
        self._check(self._lib.md_set_tuning(self._h, t.ctypes.data), "md_set_tuning")

    ORDERS = {"zrun": 0, "morton": 1}

    def layout(self):
        """The cell layout: {"cell_scale": float, "order": "zrun" | "morton"}."""
        sc = ctypes.c_double()
        od = ctypes.c_int32()
        self._check(self._lib.md_get_layout(self._h, ctypes.byref(sc), ctypes.byref(od)), "md_get_layout")
        return {"cell_scale": sc.value, "order": {v: k for k, v in self.ORDERS.items()}[od.value]}

    def set_layout(self, cell_scale=None, order=None):
        """Cell edge over the list radius (>= 1) and the order inside cells
        ("zrun" or "morton"); unspecified values keep their current setting."""
        cur = self.layout()
        sc = cur["cell_scale"] if cell_scale is None else float(cell_scale)
        od = self.ORDERS[cur["order"] if order is None else order]
        self._check(self._lib.md_set_layout(self._h, sc, od), "md_set_layout")

    LIST_KERNELS = {"auto": 0, "quads": 1, "lanes": 2}

    @property
    def list_kernel(self):
        """List-build kernel: "auto", "quads" or "lanes" (md_set_list_kernel)."""
        k = ctypes.c_int32()
        self._check(self._lib.md_get_list_kernel(self._h, ctypes.byref(k)), "md_get_list_kernel")
        return {v: n for n, v in self.LIST_KERNELS.items()}[k.value]

    @list_kernel.setter
    def list_kernel(self, kind):
        self._check(self._lib.md_set_list_kernel(self._h, self.LIST_KERNELS[kind]), "md_set_list_kernel")

    FORCE_KERNELS = {"auto": 0, "chunks": 1, "tiles": 2}

    @property
    def force_kernel(self):
        """FP32 list-form force kernel: "auto", "chunks" or "tiles"
        (md_set_force_kernel)."""
        k = ctypes.c_int32()
        self._check(self._lib.md_get_force_kernel(self._h, ctypes.byref(k)), "md_get_force_kernel")
        return {v: n for n, v in self.FORCE_KERNELS.items()}[k.value]

    @force_kernel.setter
    def force_kernel(self, kind):
        self._check(self._lib.md_set_force_kernel(self._h, self.FORCE_KERNELS[kind]), "md_set_force_kernel")

    @property
    def graph_conditional(self):
        """True when step graphs hold the list update as a conditional node
        (md_set_graph_conditional)."""
        k = ctypes.c_int32()
        self._check(self._lib.md_get_graph_conditional(self._h, ctypes.byref(k)), "md_get_graph_conditional")
        return bool(k.value)

    @graph_conditional.setter
    def graph_conditional(self, on):
        self._check(self._lib.md_set_graph_conditional(self._h, 1 if on else 0), "md_set_graph_conditional")

    def autotune(self, reps=5, cache=True):
        """Measure and apply the fastest launch/layout settings (md_autotune).
        With cache, results are kept per (GPU, replicas, log2 N, density) in
        $XDG_CACHE_HOME/paper_2406_04210_gb300/autotune.json (default
        ~/.cache/...) and reused instead of re-measuring."""
        import json
        key = None
        path = None
        if cache:
            try:
                import torch
                gpu = torch.cuda.get_device_name()
            except Exception:
                gpu = "cuda"
            vol = float(np.prod(self.box, axis=1).sum())
            key = f"{gpu}|{self.precision}|{self.nrep}|{int(np.log2(max(self.n_total, 1)))}|{self.n_total / vol:.2f}"
            base = os.environ.get("XDG_CACHE_HOME", os.path.join(os.path.expanduser("~"), ".cache"))
            path = os.path.join(base, "paper_2406_04210_gb300", "autotune.json")
            try:
                with open(path) as f:
                    table = json.load(f)
            except Exception:
                table = {}
            if key in table:
                ent = dict(table[key])
                lay = {k: ent.pop(k) for k in ("cell_scale", "order") if k in ent}
                kind = ent.pop("list_kernel", None)
                if kind is not None:
                    self.list_kernel = kind
                fkind = ent.pop("force_kernel", None)
                if fkind is not None:
                    self.force_kernel = fkind
                self.set_tuning(**ent)
                if lay:
                    self.set_layout(**lay)
                return table[key]
        t = np.zeros(4, dtype=np.int32)
        self._check(self._lib.md_autotune(self._h, int(reps), t.ctypes.data), "md_autotune")
        res = dict(zip(self.TUNING, (int(x) for x in t)))
        res.update(self.layout())
        res["list_kernel"] = self.list_kernel
        res["force_kernel"] = self.force_kernel
        if cache and path:
            try:
                os.makedirs(os.path.dirname(path), exist_ok=True)
                try:
                    with open(path) as f:
                        table = json.load(f)
                except Exception:
                    table = {}
                table[key] = res
                with open(path, "w") as f:
                    json.dump(table, f, indent=1)
            except OSError:
                pass
        return res

    def set_profiling(self, on=True):
        self._check(self._lib.md_set_profiling(self._h, 1 if on else 0), "md_set_profiling")

    PHASES = ("integrate", "list_update", "force", "thermo")

    def profile(self):
        ms = np.zeros(4)
        cnt = np.zeros(4, dtype=np.int64)
        self._check(self._lib.md_get_profile(self._h, ms.ctypes.data, cnt.ctypes.data),
                    "md_get_profile")
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(self.PHASES)}


def _as_f64(a):
    if a is None or hasattr(a, "data_ptr"):
        return a
    return np.ascontiguousarray(a, dtype=np.float64)


def _as_i32(a):
    if a is None or hasattr(a, "data_ptr"):
        return a
    return np.ascontiguousarray(a, dtype=np.int32)


def from_system(s, precision="mixed_ds"):
    """Box from an inputs.System, with its LJ parameters set."""
    b = Box(s.pos, s.box, s.vel, s.type, precision=precision)
    b.set_lj(s.eps, s.sigma, s.rcut, s.skin, True)
    return b


# ---------------------------------------------------------------------------
# torch.autograd bridge: trajectories and the pair-histogram loss
# ---------------------------------------------------------------------------
def _torch():
    import torch
    return torch


class TrajectoryFn:
    """x_T, v_T = TrajectoryFn.apply(x0, v0, eps, sigma, box, dt, nsteps, ckpt_every)

    Forward: md_set_state(x0, v0), md_set_lj(eps, sigma) (monatomic: scalar
    tensors; the box's cutoff and skin are kept), then a recorded
    md_integrate.  Backward: md_adjoint.  x0, v0 are (n, 3) float64 CUDA
    tensors; eps, sigma are 0-d float64 tensors.  The box keeps one record:
    a backward whose forward record was replaced (another forward on the same
    box, a state or parameter change) raises MDError(MD_ERR_STATE) instead of
    differentiating the other run."""

    _fn = None

    @classmethod
    def apply(cls, *args):
        if cls._fn is None:
            torch = _torch()

            class _F(torch.autograd.Function):
                @staticmethod
                def forward(ctx, x0, v0, eps, sigma, box, dt, nsteps, ckpt_every):
                    box.set_lj(float(eps), float(sigma), box._rcut, box._skin, True)
                    box.set_state(x0.detach().contiguous(), v0.detach().contiguous())
                    box.integrate(dt, nsteps, thermo=False, ckpt_every=ckpt_every)
                    xT = torch.empty_like(x0)
                    vT = torch.empty_like(v0)
                    box._check(box._lib.md_get_state(box._h, xT.data_ptr(), vT.data_ptr(), None),
                               "md_get_state")
                    ctx.box = box
                    ctx.record = box.info().record_id
                    return xT, vT

                @staticmethod
                def backward(ctx, gx, gv):
                    box = ctx.box
                    if box.info().record_id != ctx.record:
                        raise MDError(8, "TrajectoryFn.backward: the box no longer holds this forward "
                                         "run's record (another forward, state or parameter change)")
                    gx = torch.zeros_like(gv) if gx is None else gx.contiguous()
                    gv = torch.zeros_like(gx) if gv is None else gv.contiguous()
                    lx0, lv0, ge, gs = box.adjoint(gx, gv)
                    dev = gx.device
                    return (torch.from_numpy(lx0).to(dev), torch.from_numpy(lv0).to(dev),
                            torch.tensor(ge[0, 0], dtype=torch.float64, device=dev),
                            torch.tensor(gs[0, 0], dtype=torch.float64, device=dev),
                            None, None, None, None)

            cls._fn = _F
        return cls._fn.apply(*args)


def _holds(box, x, tol=1e-8):
    """Raise ValueError unless the box's current positions are x (to within
    `tol`, minimum image: a list rebuild re-centres the stored offsets, which
    moves the positions by rounding only)."""
    torch = _torch()
    cur = torch.empty((box.n_total, 3), dtype=torch.float64, device=x.device)
    box._check(box._lib.md_get_state(box._h, cur.data_ptr(), None, None), "md_get_state")
    L = torch.as_tensor(np.repeat(box.box, box.n, axis=0), dtype=torch.float64, device=x.device)
    d = cur - x.detach().to(torch.float64).reshape(-1, 3)
    d = d - L * torch.round(d / L)
    if d.numel() and float(d.abs().max()) > tol:
        raise ValueError("PairHistLossFn: x is not the state the box holds")


class PairHistLossFn:
    """loss = mean_k (h_k(x) - target_k)^2 of the box's current positions,
    which must be x (e.g. the x_T a TrajectoryFn returned): forward and
    backward check that the box still holds x and raise ValueError if not."""

    _fn = None

    @classmethod
    def apply(cls, *args):
        if cls._fn is None:
            torch = _torch()

            class _F(torch.autograd.Function):
                @staticmethod
                def forward(ctx, x, box, target, nbins, rhist, width, rmax):
                    _holds(box, x)
                    h, _ = box.pair_hist(nbins, rhist, width, rmax)
                    t = target.detach().cpu().numpy().reshape(1, -1)
                    diff = h - t
                    ctx.box, ctx.args, ctx.diff = box, (nbins, rhist, width, rmax), diff
                    ctx.save_for_backward(x)
                    return torch.tensor(float(np.mean(diff * diff)), dtype=torch.float64,
                                        device=x.device)

                @staticmethod
                def backward(ctx, g):
                    nbins, rhist, width, rmax = ctx.args
                    _holds(ctx.box, ctx.saved_tensors[0])
                    coef = 2.0 * ctx.diff / nbins * float(g)
                    _, grad = ctx.box.pair_hist(nbins, rhist, width, rmax, coef=coef)
                    return (torch.from_numpy(grad).to(g.device), None, None, None, None, None, None)

            cls._fn = _F
        return cls._fn.apply(*args)
