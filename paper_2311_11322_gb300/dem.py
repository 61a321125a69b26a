"""Python binding of the C ABI in include/dem.h (ctypes; argument marshalling only).

Every function of the header is exposed under the same name; ``World`` wraps
them for numpy users.  All computation happens in libdem.so's CUDA kernels:
if the library is missing this module raises instead of falling back.

PyTorch provides the device memory (its caching allocator, through
dem_set_allocator) and the CUDA stream (the current torch stream by default).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdem.so")

DEM_OK, DEM_ERR_ARG, DEM_ERR_OOM, DEM_ERR_CUDA, DEM_ERR_OVERLAP = 0, 1, 2, 3, 4
DEM_ERR_SLOTS, DEM_ERR_NONFINITE, DEM_ERR_TIMEOUT, DEM_ERR_STATE = 5, 6, 7, 8
STATUS_NAMES = {0: "DEM_OK", 1: "DEM_ERR_ARG", 2: "DEM_ERR_OOM", 3: "DEM_ERR_CUDA",
                4: "DEM_ERR_OVERLAP", 5: "DEM_ERR_SLOTS", 6: "DEM_ERR_NONFINITE",
                7: "DEM_ERR_TIMEOUT", 8: "DEM_ERR_STATE"}
DEM_FP64, DEM_MIXED = 0, 1
DEM_FLAG_SLOTS, DEM_FLAG_NONFINITE, DEM_FLAG_OVERLAP, DEM_FLAG_TREE, DEM_FLAG_GRAV_RANGE = 1, 2, 4, 8, 16

FIELDS = {  # name: (id, rows ('A' aggregates / 'N' spheres / int), cols)
    "COM": (0, "A", 3), "VEL": (1, "A", 3), "QUAT": (2, "A", 4), "OMEGA": (3, "A", 3),
    "SPHERE_POS": (4, "N", 3), "FORCE": (5, "A", 3), "TORQUE": (6, "A", 3),
    "CONTACTS": (7, "N", None), "FORCE_CONTACT": (8, "A", 3), "TORQUE_CONTACT": (9, "A", 3),
    "FORCE_GRAV": (10, "A", 3), "TORQUE_GRAV": (11, "A", 3), "FORCE_EXT": (12, "A", 3),
    "TORQUE_EXT": (13, "A", 3), "SPHERE_FC": (14, "N", 3), "SPHERE_TC": (15, "N", 3),
    "SPHERE_FG": (16, "N", 3), "ACC": (17, "A", 3), "PLANET": (18, 9, None), "MASS": (19, "A", 1),
    "BODY_OFFSETS": (20, "N", 3), "OMEGA_BODY": (21, "A", 3), "INFO": (22, 20, None),
    "FRAME": (23, 6, None), "TORQUE_STORED": (24, "A", 3),
}
# record of dem_pile_bulk (enum dem_bulk): name -> (offset, length)
BULK = {"mass": (0, 1), "com": (1, 3), "vcom": (4, 3), "axes": (7, 3), "radius": (10, 1),
        "density": (11, 1), "spin": (12, 3), "period": (15, 1), "p_crit": (16, 1),
        "planet_dist": (17, 1), "L": (18, 3), "moments": (21, 3)}
DEM_BULK_LEN, DEM_WATCH_LEN = 24, 52
KERNELS = {"AGG_BEGIN": 0, "PILE_BEGIN": 1, "KEYS": 2, "SCAN": 3, "SCATTER": 4,
           "CELL_ORDER": 5, "GATHER": 6, "CONTACT": 7, "GRAVITY": 8, "AGG_END": 9,
           "PILE_END": 10}


class dem_params(C.Structure):
    _fields_ = [("G", C.c_double), ("dt", C.c_double), ("kn", C.c_double), ("kt", C.c_double),
                ("cn", C.c_double), ("ct", C.c_double), ("mu_s", C.c_double),
                ("mu_r", C.c_double), ("mu_t", C.c_double), ("w0", C.c_double),
                ("eps_soft", C.c_double), ("precision", C.c_int32),
                ("max_contacts", C.c_int32), ("cell_size", C.c_double),
                ("ext_mass", C.c_double), ("ext_pos", C.c_double * 3),
                ("ext_vel", C.c_double * 3), ("spin_inc", C.c_double * 3),
                ("rot_tol", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)

_lib = None


def load():
    """Load libdem.so (built by ``__graft_entry__.build()``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built; run __graft_entry__.build() "
                           "(there is no CPU fallback)")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, dbl, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_size_t
    sig = {
        "dem_create": (i32, [vp, sz, C.POINTER(vp)]),
        "dem_set_allocator": (i32, [vp, ALLOC_FN, FREE_FN, vp]),
        "dem_add_aggregates": (i32, [vp, C.POINTER(dem_params), i64, vp, vp, vp, vp, vp, vp,
                                     C.POINTER(i32)]),
        "dem_step": (i32, [vp, vp, i32, i64]),
        "dem_sync": (i32, [vp]),
        "dem_step_profiled": (i32, [vp, i64, i32, vp]),
        "dem_read_state": (i32, [vp, i32, i32, vp, i64]),
        "dem_read_state_async": (i32, [vp, i32, i32, vp, i64]),
        "dem_read_wait": (i32, [vp]),
        "dem_pile_flags": (i32, [vp, i32, C.POINTER(i32)]),
        "dem_remove_pile": (i32, [vp, i32]),
        "dem_set_tuning": (i32, [vp, C.c_char_p, dbl]),
        "dem_get_tuning": (i32, [vp, C.c_char_p, C.POINTER(dbl)]),
        "dem_autotune": (i32, [vp, i32, C.POINTER(dbl)]),
        "dem_footprint_bytes": (sz, [i64, i64, i32, i32]),
        "dem_world_bytes": (sz, [vp]),
        "dem_last_error": (C.c_char_p, [vp]),
        "dem_destroy": (None, [vp]),
        "dem_set_timed_kernel": (i32, [vp, i32]),
        "dem_step_timed": (i32, [vp, C.POINTER(C.c_float), C.POINTER(C.c_float)]),
        "dem_graph_kernel_count": (i32, [vp, C.POINTER(i32)]),
        "dem_gravity_noalloc": (i32, [vp, vp, vp, i32, dbl, dbl, vp, vp, C.c_char_p, sz]),
        "dem_probe_peak": (i32, [i32, i64, i32, vp, vp, vp, C.POINTER(dbl), C.POINTER(dbl),
                                 C.POINTER(i32), C.c_char_p, sz]),
        "dem_write_state": (i32, [vp, i32, i32, vp, i64]),
        "dem_pile_bulk": (i32, [vp, i32, vp, i64]),
        "dem_watch": (i32, [vp, i32, dbl, i64]),
        "dem_watch_result": (i32, [vp, i32, vp, i64]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


class DemError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def make_params(p) -> dem_params:
    """dem_params from a ``workloads.Params``-like object."""
    P = dem_params()
    for f in ("G", "dt", "kn", "kt", "cn", "ct", "mu_s", "mu_r", "mu_t", "w0"):
        setattr(P, f, float(getattr(p, f)))
    P.eps_soft = float(p.eps)
    P.precision = int(p.precision)
    P.max_contacts = int(p.max_contacts)
    P.cell_size = float(getattr(p, "cell_size", 0.0))
    P.ext_mass = float(getattr(p, "ext_mass", 0.0))
    for k in range(3):
        P.ext_pos[k] = float(p.ext_pos[k])
        P.ext_vel[k] = float(p.ext_vel[k])
        P.spin_inc[k] = float(p.spin_inc[k])
    P.rot_tol = float(getattr(p, "rot_tol", 0.0))
    return P


# ---- the C functions under their own names ---------------------------------
def dem_create(stream: int = 0, budget: int = 0):
    w = C.c_void_p()
    s = load().dem_create(C.c_void_p(stream), budget, C.byref(w))
    if s != DEM_OK:
        raise DemError(s, "dem_create failed")
    return w


def dem_footprint_bytes(n_spheres, n_agg, max_contacts, precision):
    return int(load().dem_footprint_bytes(n_spheres, n_agg, max_contacts, precision))


PROBES = {"FMA32": 0, "FMA32X2": 1, "FMA64": 2, "COPY": 3}


def dem_probe_peak(kind: str, size: int, reps: int, src_ptr: int, dst_ptr: int, stream: int = 0):
    """Peak-rate probe (include/dem.h): returns (rate per s, fastest ms, SM count)."""
    rate, ms, sms = C.c_double(), C.c_double(), C.c_int32()
    msg = C.create_string_buffer(256)
    s = load().dem_probe_peak(PROBES[kind], int(size), int(reps), C.c_void_p(src_ptr),
                              C.c_void_p(dst_ptr), C.c_void_p(stream), C.byref(rate), C.byref(ms),
                              C.byref(sms), msg, len(msg))
    if s != DEM_OK:
        raise DemError(s, msg.value.decode())
    return rate.value, ms.value, sms.value


def dem_last_error(w) -> str:
    return load().dem_last_error(w).decode()


def _torch_allocator():
    import torch

    def alloc(nbytes, stream, ctx):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0)))
        except Exception:
            return None

    def free(ptr, ctx):
        try:
            torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:
            pass

    return ALLOC_FN(alloc), FREE_FN(free)


class World:
    """A set of rubble piles stepped together on one GPU through libdem.so."""

    def __init__(self, stream=None, budget: int = 0, torch_memory: bool = True):
        L = load()
        self._torch_stream = None
        if stream is None:
            import torch
            self._torch_stream = torch.cuda.Stream()
            stream = self._torch_stream.cuda_stream
        self._L = L
        self.stream = int(stream)
        self.w = dem_create(self.stream, budget)
        self._cb = None
        if torch_memory:
            self._cb = _torch_allocator()
            self._check(L.dem_set_allocator(self.w, self._cb[0], self._cb[1], None))
        self.piles = {}
        self._static = {}
        self._pending = []   # destinations of read_async copies in flight

    def _check(self, s):
        if s != DEM_OK:
            raise DemError(s, dem_last_error(self.w))
        return s

    # ---- piles
    def add_pile(self, ic, params) -> int:
        P = make_params(params)
        counts = np.ascontiguousarray(ic.counts, np.int32)
        pos = np.ascontiguousarray(ic.pos, np.float64)
        rad = np.ascontiguousarray(ic.radius, np.float64)
        den = np.ascontiguousarray(ic.density, np.float64)
        vel = None if ic.vel is None else np.ascontiguousarray(ic.vel, np.float64)
        om = None if ic.omega is None else np.ascontiguousarray(ic.omega, np.float64)
        pid = C.c_int32()
        self._check(self._L.dem_add_aggregates(self.w, C.byref(P), len(counts), _ptr(counts),
                                               _ptr(pos), _ptr(rad), _ptr(den), _ptr(vel),
                                               _ptr(om), C.byref(pid)))
        self.piles[pid.value] = (len(counts), len(rad), int(params.max_contacts))
        self._static[pid.value] = (counts.copy(), rad.copy(), den.copy())
        return pid.value

    def ic_of(self, pile):
        """The pile's current state as initial conditions for add_pile (sphere
        positions, aggregate COM velocities and spins; history not carried)."""
        from .workloads import PileIC
        counts, rad, den = self._static[pile]
        return PileIC(counts=counts.copy(), pos=self.read(pile, "SPHERE_POS"), radius=rad.copy(),
                      density=den.copy(), vel=self.read(pile, "VEL"), omega=self.read(pile, "OMEGA"))

    def remove(self, pile):
        self._check(self._L.dem_remove_pile(self.w, pile))
        self.piles.pop(pile, None)
        self._static.pop(pile, None)

    # ---- stepping
    def step(self, n=1, piles=None, check=True):
        ids = None if piles is None else np.ascontiguousarray(piles, np.int32)
        s = self._L.dem_step(self.w, _ptr(ids), 0 if ids is None else len(ids), int(n))
        return self._check(s) if check else s

    def sync(self, check=True):
        s = self._L.dem_sync(self.w)
        return self._check(s) if check else s

    def set_timed_kernel(self, kernel):
        self._check(self._L.dem_set_timed_kernel(self.w, -1 if kernel is None else KERNELS[kernel]))

    def step_timed(self):
        """One graph-launched step; returns (step_ms, timed_kernel_ms)."""
        a, b = C.c_float(), C.c_float()
        self._check(self._L.dem_step_timed(self.w, C.byref(a), C.byref(b)))
        return a.value, b.value

    def graph_kernel_count(self) -> int:
        n = C.c_int32()
        self._check(self._L.dem_graph_kernel_count(self.w, C.byref(n)))
        return n.value

    def step_profiled(self, n, kernel="GRAVITY"):
        ms = np.zeros(int(n), np.float32)
        self._check(self._L.dem_step_profiled(self.w, int(n), KERNELS[kernel], _ptr(ms)))
        return ms

    # ---- readout
    def read(self, pile, field, out=None):
        """One field of a pile as float64; `out` (optional): a C-contiguous
        float64 array of the field's shape to fill instead of a new one (for
        repeated reads, e.g. into pinned host memory)."""
        fid, rows, cols = FIELDS[field]
        if pile not in self.piles:   # let the library report the unknown id
            buf = np.zeros(16)
            self._check(self._L.dem_read_state(self.w, int(pile), fid, _ptr(buf), buf.size))
        A, N, K = self.piles[pile]
        if field == "CONTACTS":
            shape = (N, 1 + 4 * K)
        elif isinstance(rows, int):
            shape = (rows,)
        else:
            n = A if rows == "A" else N
            shape = (n, cols) if cols > 1 else (n,)
        if out is None:
            out = np.zeros(shape)
        elif out.shape != shape or out.dtype != np.float64 or not out.flags.c_contiguous:
            raise ValueError(f"out must be a C-contiguous float64 array of shape {shape}")
        self._check(self._L.dem_read_state(self.w, pile, fid, _ptr(out), out.size))
        return out

    # fields dem_read_state_async accepts
    ASYNC_FIELDS = ("COM", "VEL", "QUAT", "OMEGA_BODY", "ACC", "TORQUE_STORED", "MASS")

    def read_async(self, pile, field, out):
        """Enqueue a read of a per-aggregate state field into `out` (a
        C-contiguous float64 array of the field's shape, best in pinned memory)
        and return at once; `out` holds the values after read_wait()."""
        fid, rows, cols = FIELDS[field]
        if pile not in self.piles:   # let the library report the unknown id
            self._check(self._L.dem_read_state_async(self.w, int(pile), fid, None, 0))
        A = self.piles[pile][0]
        shape = (A, cols) if cols > 1 else (A,)
        if out.shape != shape or out.dtype != np.float64 or not out.flags.c_contiguous:
            raise ValueError(f"out must be a C-contiguous float64 array of shape {shape}")
        self._pending.append(out)   # kept alive until read_wait
        self._check(self._L.dem_read_state_async(self.w, int(pile), fid, _ptr(out), out.size))

    def read_wait(self):
        """Wait for the pending read_async copies (not for later steps) and
        convert them to FP64 in place."""
        try:
            self._check(self._L.dem_read_wait(self.w))
        finally:
            self._pending.clear()

    def write(self, pile, field, values):
        fid = FIELDS[field][0]
        v = np.ascontiguousarray(values, np.float64)
        self._check(self._L.dem_write_state(self.w, int(pile), fid, _ptr(v), v.size))

    def checkpoint(self, pile):
        """Everything the next step reads, as host arrays (bit-exact restore)."""
        names = ("COM", "VEL", "QUAT", "OMEGA_BODY", "ACC", "TORQUE_STORED", "CONTACTS",
                 "PLANET", "FRAME")
        return {n: self.read(pile, n) for n in names}

    def restore(self, pile, ck):
        for n, v in ck.items():
            self.write(pile, n, v)

    def contacts(self, pile):
        """Contact pairs (i < j, pile-local sphere indices) and their S vectors."""
        raw = self.read(pile, "CONTACTS")
        K = self.piles[pile][2]
        pairs, S = [], []
        for i in range(raw.shape[0]):
            n = int(raw[i, 0])
            for t in range(n):
                j = int(raw[i, 1 + 4 * t])
                if i < j:
                    pairs.append((i, j))
                    S.append(raw[i, 2 + 4 * t:5 + 4 * t])
        return pairs, np.array(S).reshape(-1, 3)

    # ---- bulk shape and spin (Sec. 4.1, 4.2), computed on the device
    @staticmethod
    def _bulk_dict(v):
        return {k: (float(v[o]) if n == 1 else v[o:o + n].copy()) for k, (o, n) in BULK.items()}

    def bulk(self, pile) -> dict:
        """Bulk record of a pile after the last step (see ``BULK`` for the keys)."""
        out = np.zeros(DEM_BULK_LEN)
        self._check(self._L.dem_pile_bulk(self.w, int(pile), _ptr(out), out.size))
        return self._bulk_dict(out)

    def watch(self, pile, growth, every=1):
        """Arm (growth > 0) or disarm (0) the device-side radius-growth watch."""
        self._check(self._L.dem_watch(self.w, int(pile), float(growth), int(every)))

    def watch_result(self, pile) -> dict:
        out = np.zeros(DEM_WATCH_LEN)
        self._check(self._L.dem_watch_result(self.w, int(pile), _ptr(out), out.size))
        fired = int(out[0])
        return {"fired_step": fired if fired >= 0 else None, "growth": float(out[1]),
                "every": int(out[2]), "armed": bool(out[3]),
                "at_arm": self._bulk_dict(out[4:4 + DEM_BULK_LEN]),
                "at_fire": self._bulk_dict(out[4 + DEM_BULK_LEN:]) if fired >= 0 else None}

    def flags(self, pile) -> int:
        f = C.c_int32()
        self._check(self._L.dem_pile_flags(self.w, pile, C.byref(f)))
        return f.value

    def info(self, pile) -> dict:
        v = self.read(pile, "INFO")
        keys = ("n_agg", "n_sph", "steps", "flags", "nx", "ny", "nz", "cell", "K", "precision",
                "Ox", "Oy", "Oz", "failed", "parity", "M_total", "rebuilds", "skin",
                "rebuild_next", "reserved")
        return dict(zip(keys, v.tolist()))

    # ---- tuning
    def set_tuning(self, key, value):
        self._check(self._L.dem_set_tuning(self.w, key.encode(), float(value)))

    def get_tuning(self, key) -> float:
        v = C.c_double()
        self._check(self._L.dem_get_tuning(self.w, key.encode(), C.byref(v)))
        return v.value

    def autotune(self, trial_steps=3):
        best = C.c_double()
        self._check(self._L.dem_autotune(self.w, int(trial_steps), C.byref(best)))
        return best.value

    def bytes(self) -> int:
        return int(self._L.dem_world_bytes(self.w))

    def close(self):
        if self.w:
            self._L.dem_destroy(self.w)
            self.w = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
