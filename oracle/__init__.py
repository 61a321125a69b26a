"""Plain FP64 CPU oracle for bonded-sphere aggregate DEM (arXiv 2311.11322).

TEST INFRASTRUCTURE.  Only the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library and never imports it; the two meet only through the
seeded input generators in ``paper_2311_11322_gb300.workloads``.

The arithmetic lives in ``dem_oracle.c`` (double precision, brute-force pair
search, plain O(N^2) gravity).  This module compiles it with gcc on first use
and wraps it with ctypes and numpy.  Section and equation citations are in the
C source beside each function.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dem_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

HCAP = 64  # history capacity per sphere as canonical owner


def build(force: bool = False) -> str:
    """Compile dem_oracle.c into liboracle.so next to it (gcc, OpenMP)."""
    with _lock:
        stale = (not os.path.exists(_LIB_PATH)
                 or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
        if force or stale:
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared",
                   "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(C.Structure):
    _fields_ = [("G", C.c_double), ("dt", C.c_double), ("kn", C.c_double),
                ("kt", C.c_double), ("cn", C.c_double), ("ct", C.c_double),
                ("mu_s", C.c_double), ("mu_r", C.c_double), ("mu_t", C.c_double),
                ("w0", C.c_double), ("eps", C.c_double), ("ext_mass", C.c_double),
                ("spin_inc", C.c_double * 3), ("rot_tol", C.c_double)]


class _Sim(C.Structure):
    _fields_ = [("n_agg", C.c_int64), ("n_sph", C.c_int64), ("hcap", C.c_int32),
                ("first", C.c_void_p), ("count", C.c_void_p),
                ("M", C.c_void_p), ("I", C.c_void_p), ("Iinv", C.c_void_p),
                ("r", C.c_void_p), ("v", C.c_void_p), ("q", C.c_void_p), ("wb", C.c_void_p),
                ("acc", C.c_void_p), ("torque", C.c_void_p),
                ("agg_of", C.c_void_p), ("m", C.c_void_p), ("s", C.c_void_p), ("b", C.c_void_p),
                ("h_n", C.c_void_p), ("h_partner", C.c_void_p), ("h_S", C.c_void_p),
                ("sph_pos", C.c_void_p), ("sph_vel", C.c_void_p), ("sph_w", C.c_void_p),
                ("Fc", C.c_void_p), ("Tc", C.c_void_p), ("Fg", C.c_void_p), ("Fe", C.c_void_p),
                ("FA_c", C.c_void_p), ("NA_c", C.c_void_p), ("FA_g", C.c_void_p),
                ("NA_g", C.c_void_p), ("FA_e", C.c_void_p), ("NA_e", C.c_void_p),
                ("planet", C.c_void_p), ("scaleF", C.c_void_p), ("scaleN", C.c_void_p),
                ("pairs", C.c_void_p), ("pair_x", C.c_void_p), ("pair_cap", C.c_int64),
                ("n_pairs", C.c_int64), ("sph_Fmc", C.c_void_p), ("sph_Tmc", C.c_void_p),
                ("sph_Fmg", C.c_void_p)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int32, C.c_double
        L.ora_threads.restype = C.c_int
        L.ora_build.restype = C.c_int
        L.ora_build.argtypes = [i64] + [vp] * 12
        L.ora_contacts.restype = i64
        L.ora_contacts.argtypes = [i64, vp, vp, vp, vp, vp, C.POINTER(Params), i32,
                                   vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, i64]
        L.ora_gravity.restype = None
        L.ora_gravity.argtypes = [i64, vp, vp, vp, dbl, dbl, C.c_int, i64, vp, vp, vp]
        L.ora_rotate.restype = None
        L.ora_rotate.argtypes = [vp, vp, vp, vp, vp, dbl]
        L.ora_rotate_adaptive.restype = C.c_int
        L.ora_rotate_adaptive.argtypes = [vp, vp, vp, vp, dbl, dbl]
        L.ora_spin_kick.restype = None
        L.ora_spin_kick.argtypes = [vp, vp, vp, vp, dbl]
        L.ora_rotmat.restype = None
        L.ora_rotmat.argtypes = [vp, vp]
        L.ora_step.restype = C.c_int
        L.ora_step.argtypes = [C.POINTER(_Sim), C.POINTER(Params), C.c_int]
        L.ora_step_sampled.restype = C.c_int
        L.ora_step_sampled.argtypes = [C.POINTER(_Sim), C.POINTER(Params), i64, vp,
                                       vp, vp, vp, vp, vp, vp]
        _lib = L
    return _lib


def threads() -> int:
    """OpenMP threads the oracle uses."""
    return int(lib().ora_threads())


def _p(a):
    return None if a is None else a.ctypes.data


def make_params(p) -> Params:
    """Oracle parameter block from a ``workloads.Params``-like object."""
    P = Params()
    for f in ("G", "dt", "kn", "kt", "cn", "ct", "mu_s", "mu_r", "mu_t", "w0", "eps",
              "ext_mass"):
        setattr(P, f, float(getattr(p, f)))
    si = getattr(p, "spin_inc", (0.0, 0.0, 0.0))
    for k in range(3):
        P.spin_inc[k] = float(si[k])
    P.rot_tol = float(getattr(p, "rot_tol", 0.0))
    return P


def build_aggregates(counts, pos, radius, density):
    """Mass, COM, inertia and body offsets (Sec. 2.2.1).  Returns a dict."""
    counts = np.ascontiguousarray(counts, np.int32)
    pos = np.ascontiguousarray(pos, np.float64).reshape(-1, 3)
    radius = np.ascontiguousarray(radius, np.float64)
    density = np.ascontiguousarray(density, np.float64)
    A, N = len(counts), len(radius)
    if int(counts.sum()) != N:
        raise ValueError("counts do not sum to the number of spheres")
    out = dict(first=np.zeros(A, np.int32), agg_of=np.zeros(N, np.int32),
               m=np.zeros(N), b=np.zeros((N, 3)), M=np.zeros(A), com=np.zeros((A, 3)),
               I=np.zeros((A, 3, 3)), Iinv=np.zeros((A, 3, 3)))
    rc = lib().ora_build(A, _p(counts), _p(pos), _p(radius), _p(density), _p(out["first"]),
                         _p(out["agg_of"]), _p(out["m"]), _p(out["b"]), _p(out["M"]),
                         _p(out["com"]), _p(out["I"]), _p(out["Iinv"]))
    if rc != 0:
        raise ValueError(f"ora_build failed ({rc})")
    return out


def gravity(pos, m, agg_of, G, eps, exclude_same_agg=False, rows=None, want_mag=False):
    """Eq. (particle_gravity), softened; rows=None computes every sphere."""
    pos = np.ascontiguousarray(pos, np.float64).reshape(-1, 3)
    m = np.ascontiguousarray(m, np.float64)
    agg_of = np.ascontiguousarray(agg_of, np.int32)
    n = len(m)
    if rows is not None:
        rows = np.ascontiguousarray(rows, np.int64)
        nr = len(rows)
    else:
        nr = n
    F = np.zeros((nr, 3))
    Fm = np.zeros(nr) if want_mag else None
    lib().ora_gravity(n, _p(pos), _p(m), _p(agg_of), float(G), float(eps),
                      int(bool(exclude_same_agg)), nr, _p(rows), _p(F), _p(Fm))
    return (F, Fm) if want_mag else F


def contacts(pos, vel, w, radius, agg_of, params, hist=None, hcap=HCAP):
    """One brute-force contact pass (Sec. 2.1, 2.2.4).

    Returns dict with Fc, Tc, Fmag, Tmag (per sphere), pairs (P,2), x (P,),
    and the new history (h_n, h_partner, h_S).
    """
    pos = np.ascontiguousarray(pos, np.float64).reshape(-1, 3)
    vel = np.ascontiguousarray(vel, np.float64).reshape(-1, 3)
    w = np.ascontiguousarray(w, np.float64).reshape(-1, 3)
    radius = np.ascontiguousarray(radius, np.float64)
    agg_of = np.ascontiguousarray(agg_of, np.int32)
    n = len(radius)
    if hist is None:
        hist = (np.zeros(n, np.int32), np.zeros(n * hcap, np.int32), np.zeros(n * hcap * 3))
    hn_new = np.zeros(n, np.int32)
    hp_new = np.zeros(n * hcap, np.int32)
    hS_new = np.zeros(n * hcap * 3)
    Fc, Tc = np.zeros((n, 3)), np.zeros((n, 3))
    Fm, Tm = np.zeros(n), np.zeros(n)
    cap = max(16, 16 * n)
    pairs = np.zeros((cap, 2), np.int32)
    px = np.zeros(cap)
    P = make_params(params)
    np_ = lib().ora_contacts(n, _p(pos), _p(vel), _p(w), _p(radius), _p(agg_of), C.byref(P),
                             hcap, _p(hist[0]), _p(hist[1]), _p(hist[2]), _p(hn_new),
                             _p(hp_new), _p(hS_new), _p(Fc), _p(Tc), _p(Fm), _p(Tm),
                             _p(pairs), _p(px), cap)
    if np_ < 0:
        raise RuntimeError("oracle contact history overflow")
    k = min(int(np_), cap)
    return dict(Fc=Fc, Tc=Tc, Fmag=Fm, Tmag=Tm, pairs=pairs[:k].copy(), x=px[:k].copy(),
                hist=(hn_new, hp_new, hS_new))


def rotmat(q):
    q = np.ascontiguousarray(q, np.float64)
    R = np.zeros(9)
    lib().ora_rotmat(_p(q), _p(R))
    return R.reshape(3, 3)


def rotate(q, wb, I, Iinv, N_space, h):
    """One RK4 rotation step (Sec. 2.2.1 reading); returns new (q, wb)."""
    q = np.array(q, np.float64)
    wb = np.array(wb, np.float64)
    I = np.ascontiguousarray(I, np.float64)
    Iinv = np.ascontiguousarray(Iinv, np.float64)
    N = np.ascontiguousarray(N_space, np.float64)
    lib().ora_rotate(_p(q), _p(wb), _p(I), _p(Iinv), _p(N), float(h))
    return q, wb


def rotate_adaptive(q, wb, I, Iinv, h, tol):
    """Torque-free rotation over h by the adaptive embedded RK5(4) (Sec. 2.2.1);
    returns new (q, wb, accepted substeps)."""
    q = np.array(q, np.float64)
    wb = np.array(wb, np.float64)
    I = np.ascontiguousarray(I, np.float64)
    Iinv = np.ascontiguousarray(Iinv, np.float64)
    n = lib().ora_rotate_adaptive(_p(q), _p(wb), _p(I), _p(Iinv), float(h), float(tol))
    return q, wb, int(n)


BULK_KEYS = ("mass", "com", "vcom", "axes", "radius", "density", "spin", "period", "p_crit",
             "planet_dist", "L", "moments")


def bulk(M, I, r, v, q, wb, G, planet_pos=None):
    """Bulk shape and spin of a pile of rigid aggregates (Sec. 4.1, 4.2).

    Reading: the paper measures the growth of a pile's radius and uses its
    bulk density without defining either; both are taken from the uniform
    ellipsoid with the pile's mass and principal moments of inertia about its
    COM.  Inertia of the pile: every aggregate's own tensor rotated to space
    plus its COM's orbital term; spin: the rigid rotation I^-1 L that carries
    the pile's angular momentum about its COM; nominal critical period
    sqrt(3 pi / (G rho)) of a rigid sphere of that bulk density (Sec. 4.1).
    M [A], I [A][3][3] body frame, r, v [A][3], q [A][4], wb [A][3] body spin.
    """
    M = np.asarray(M, np.float64)
    r = np.asarray(r, np.float64).reshape(-1, 3)
    v = np.asarray(v, np.float64).reshape(-1, 3)
    I = np.asarray(I, np.float64).reshape(-1, 3, 3)
    wb = np.asarray(wb, np.float64).reshape(-1, 3)
    Mt = float(M.sum())
    c = (M[:, None] * r).sum(0) / Mt
    vc = (M[:, None] * v).sum(0) / Mt
    Ip = np.zeros((3, 3))
    L = np.zeros(3)
    for a in range(len(M)):
        R = rotmat(q[a])
        x = r[a] - c
        Ip += M[a] * (np.dot(x, x) * np.eye(3) - np.outer(x, x)) + R @ I[a] @ R.T
        L += M[a] * np.cross(x, v[a] - vc) + R @ (I[a] @ wb[a])
    mom = np.linalg.eigvalsh(Ip)                       # ascending
    k = 5.0 / (2.0 * Mt)
    ax2 = k * np.array([mom[1] + mom[2] - mom[0], mom[0] + mom[2] - mom[1], mom[0] + mom[1] - mom[2]])
    axes = np.sqrt(np.maximum(ax2, 0.0))
    vol = float(np.prod(axes))
    rho = 3.0 * Mt / (4.0 * np.pi * vol) if vol > 0 else np.inf
    w = np.linalg.solve(Ip, L)
    wn = float(np.linalg.norm(w))
    dist = 0.0 if planet_pos is None else float(np.linalg.norm(np.asarray(planet_pos) - c))
    return {"mass": Mt, "com": c, "vcom": vc, "axes": axes, "radius": vol ** (1.0 / 3.0),
            "density": rho, "spin": w, "period": 2 * np.pi / wn if wn > 0 else np.inf,
            "p_crit": float(np.sqrt(3 * np.pi / (G * rho))) if G > 0 and np.isfinite(rho) else np.inf,
            "planet_dist": dist, "L": L, "moments": mom}


def roche_distance(R_primary, rho_primary, rho_pile):
    """Nominal disruption distance 1.26 R (rho_M / rho_m)^(1/3) (Sec. 4.2)."""
    return 1.26 * R_primary * (rho_primary / rho_pile) ** (1.0 / 3.0)


class Pile:
    """One rubble pile advanced by the oracle's leapfrog (Sec. 2.1, 2.2)."""

    def __init__(self, ic, params, want_scales=False, pair_cap=None):
        self.params = params
        self.P = make_params(params)
        agg = build_aggregates(ic.counts, ic.pos, ic.radius, ic.density)
        A, N = len(ic.counts), len(ic.radius)
        self.A, self.N = A, N
        self.counts = np.ascontiguousarray(ic.counts, np.int32)
        self.first = agg["first"]
        self.agg_of = agg["agg_of"]
        self.m, self.b, self.M = agg["m"], agg["b"], agg["M"]
        self.s = np.ascontiguousarray(ic.radius, np.float64)
        self.I, self.Iinv = agg["I"], agg["Iinv"]
        self.r = agg["com"].copy()
        self.v = np.zeros((A, 3)) if ic.vel is None else np.array(ic.vel, np.float64).reshape(A, 3)
        self.q = np.zeros((A, 4))
        self.q[:, 0] = 1.0
        self.wb = (np.zeros((A, 3)) if ic.omega is None
                   else np.array(ic.omega, np.float64).reshape(A, 3))
        self.acc = np.zeros((A, 3))
        self.torque = np.zeros((A, 3))
        self.h_n = np.zeros(N, np.int32)
        self.h_partner = np.zeros(N * HCAP, np.int32)
        self.h_S = np.zeros(N * HCAP * 3)
        for name in ("sph_pos", "sph_vel", "sph_w", "Fc", "Tc", "Fg", "Fe"):
            setattr(self, name, np.zeros((N, 3)))
        for name in ("FA_c", "NA_c", "FA_g", "NA_g", "FA_e", "NA_e"):
            setattr(self, name, np.zeros((A, 3)))
        self.planet = np.zeros(9)
        if getattr(params, "ext_mass", 0.0) > 0:
            self.planet[0:3] = params.ext_pos
            self.planet[3:6] = params.ext_vel
        self.want_scales = want_scales
        self.scaleF = np.zeros(A) if want_scales else None
        self.scaleN = np.zeros(A) if want_scales else None
        self.sph_Fmc = np.zeros(N) if want_scales else None
        self.sph_Tmc = np.zeros(N) if want_scales else None
        self.sph_Fmg = np.zeros(N) if want_scales else None
        cap = pair_cap if pair_cap is not None else 8 * N + 16
        self.pairs = np.zeros((cap, 2), np.int32)
        self.pair_x = np.zeros(cap)
        self.steps = 0
        self._sim = self._make_sim(cap)

    def _make_sim(self, cap):
        S = _Sim()
        S.n_agg, S.n_sph, S.hcap = self.A, self.N, HCAP
        for f in ("first", "M", "I", "Iinv", "r", "v", "q", "wb", "acc", "torque", "agg_of", "m",
                  "s", "b", "h_n", "h_partner", "h_S", "sph_pos", "sph_vel", "sph_w", "Fc", "Tc",
                  "Fg", "Fe", "FA_c", "NA_c", "FA_g", "NA_g", "FA_e", "NA_e", "planet", "scaleF",
                  "scaleN", "pairs", "pair_x", "sph_Fmc", "sph_Tmc", "sph_Fmg"):
            setattr(S, f, _p(getattr(self, f)))
        S.count = _p(self.counts)
        S.pair_cap = cap
        return S

    def step(self, n=1):
        for _ in range(n):
            rc = lib().ora_step(C.byref(self._sim), C.byref(self.P), int(self.want_scales))
            if rc != 0:
                raise RuntimeError(f"oracle step failed ({rc})")
            self.steps += 1

    def contact_pairs(self):
        k = min(int(self._sim.n_pairs), len(self.pair_x))
        return self.pairs[:k].copy(), self.pair_x[:k].copy()

    def step_sampled(self, rows):
        """First-step forces for the listed spheres only (see ora_step_sampled)."""
        rows = np.ascontiguousarray(rows, np.int64)
        k = len(rows)
        out = {n: np.zeros((k, 3)) for n in ("Fc", "Tc", "Fg", "Fe")}
        out["Fmag"], out["Tmag"] = np.zeros(k), np.zeros(k)
        rc = lib().ora_step_sampled(C.byref(self._sim), C.byref(self.P), k, _p(rows),
                                    _p(out["Fc"]), _p(out["Tc"]), _p(out["Fg"]), _p(out["Fe"]),
                                    _p(out["Fmag"]), _p(out["Tmag"]))
        if rc != 0:
            raise RuntimeError("oracle sampled step failed")
        return out

    # derived quantities -------------------------------------------------
    def omega_space(self):
        out = np.zeros((self.A, 3))
        for a in range(self.A):
            out[a] = rotmat(self.q[a]) @ self.wb[a]
        return out

    def kinetic_energy(self):
        ws = self.wb
        Iw = np.einsum("aij,aj->ai", self.I, ws)
        return 0.5 * float(np.sum(self.M[:, None] * self.v ** 2)) + 0.5 * float(np.sum(ws * Iw))

    def linear_momentum(self):
        return np.sum(self.M[:, None] * self.v, axis=0)

    def bulk(self):
        """Bulk shape and spin of this pile (module function ``bulk``)."""
        planet = self.planet[:3] if getattr(self.params, "ext_mass", 0.0) > 0 else None
        return bulk(self.M, self.I, self.r, self.v, self.q, self.wb, self.params.G, planet)

    def angular_momentum(self, about=None):
        about = np.zeros(3) if about is None else np.asarray(about, np.float64)
        L = np.zeros(3)
        for a in range(self.A):
            R = rotmat(self.q[a])
            L += self.M[a] * np.cross(self.r[a] - about, self.v[a])
            L += R @ (self.I[a] @ self.wb[a])
        return L
