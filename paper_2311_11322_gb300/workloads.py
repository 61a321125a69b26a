"""Seeded synthetic inputs: rubble piles of bonded-sphere aggregates.

This module only draws initial conditions and parameter values; it holds none
of the step's arithmetic and imports neither the CUDA library nor the oracle,
so both can be fed the same inputs.  Every generator is deterministic in its
seed (numpy PCG64).

Shapes (touching spheres of radius s, offsets from the shape centre):
  dumbbell (2): (+-s, 0, 0)
  rod3     (3): (-2s, 0, 0), (0, 0, 0), (2s, 0, 0)
  tetra    (4): regular tetrahedron of edge 2s
  square   (4): (+-s, +-s, 0)
  rod4     (4): (-3s, 0, 0), (-s, 0, 0), (s, 0, 0), (3s, 0, 0)
  diamond  (4): planar rhombus, (0, +-s, 0), (+-sqrt(3) s, 0, 0)
  cube8    (8): (+-s, +-s, +-s)
  single   (1): a free sphere (an aggregate of one)
These are the simple shapes the paper builds its grains from (Sec. 2.2 figure,
Sec. 3, Sec. 4.1).  Orientation is uniform on SO(3) (normalised 4-D Gaussian quaternion).

Parameter recipe (the paper delegates the force-law constants to earlier
work; these are the calibration rules used for the synthetic workloads):
  sphere mass m = rho 4/3 pi s^3;  mu_ref = (mean aggregate mass) / 2;
  k_n = mu_ref v_max^2 / (0.01 R_med)^2 so that the largest overlap is ~1% R;
  v_max = sqrt(2 G M_tot / R_cloud) (collapse speed) for free clouds, the
  escape speed plus any surface spin speed for settled piles;
  damping from restitution e: zeta = -ln e / sqrt(pi^2 + ln^2 e),
  c = 2 zeta sqrt(mu_ref k);  k_t = 2/7 k_n, c_t from e_t with k_t;
  contact time t_c = pi / (omega_0 sqrt(1 - zeta^2)), omega_0 = sqrt(k_n/mu_ref);
  h = t_c / 50;  rolling regularisation w0 = 1e-2 v_max / R_med.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field

import numpy as np

G_SI = 6.67430e-11          # CODATA 2018
EARTH_MASS = 5.972e24
EARTH_RADIUS = 6.371e6

PRECISION_FP64 = 0
PRECISION_MIXED = 1

SHAPES = ("dumbbell", "rod3", "tetra", "square")
# the grain shapes of the paper's profiling and spin-up runs (Sec. 3, Sec. 4.1)
E_SHAPES = ("dumbbell", "diamond", "rod4", "tetra", "cube8")
SHAPE_SIZE = {"dumbbell": 2, "rod3": 3, "tetra": 4, "square": 4, "rod4": 4, "diamond": 4,
              "cube8": 8, "single": 1}


@dataclass
class Params:
    G: float = G_SI
    dt: float = 0.1
    kn: float = 1.0
    kt: float = 2.0 / 7.0
    cn: float = 0.0
    ct: float = 0.0
    mu_s: float = 0.5
    mu_r: float = 0.0
    mu_t: float = 0.0
    w0: float = 1e-6
    eps: float = 0.1
    ext_mass: float = 0.0
    ext_pos: tuple = (0.0, 0.0, 0.0)
    ext_vel: tuple = (0.0, 0.0, 0.0)
    spin_inc: tuple = (0.0, 0.0, 0.0)
    precision: int = PRECISION_MIXED
    max_contacts: int = 16
    cell_size: float = 0.0
    rot_tol: float = 0.0        # 0: RK4 rotation; > 0: adaptive RK5(4) to this tolerance

    def replace(self, **kw) -> "Params":
        return dataclasses.replace(self, **kw)


@dataclass
class PileIC:
    """Initial conditions of one pile: aggregates of touching spheres."""
    counts: np.ndarray          # int32 [A]
    pos: np.ndarray             # float64 [N, 3], space frame
    radius: np.ndarray          # float64 [N]
    density: np.ndarray         # float64 [N]
    vel: np.ndarray | None = None    # float64 [A, 3] COM velocity
    omega: np.ndarray | None = None  # float64 [A, 3] spin (space frame)
    meta: dict = field(default_factory=dict)

    @property
    def n_agg(self) -> int:
        return int(len(self.counts))

    @property
    def n_sph(self) -> int:
        return int(len(self.radius))


# ---------------------------------------------------------------------------
# shapes and orientations
# ---------------------------------------------------------------------------
def shape_offsets(name: str, s: float) -> np.ndarray:
    if name == "dumbbell":
        o = np.array([[1, 0, 0], [-1, 0, 0]], float) * s
    elif name == "rod3":
        o = np.array([[-2, 0, 0], [0, 0, 0], [2, 0, 0]], float) * s
    elif name == "tetra":
        o = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], float) * (s / math.sqrt(2.0))
    elif name == "square":
        o = np.array([[1, 1, 0], [1, -1, 0], [-1, 1, 0], [-1, -1, 0]], float) * s
    elif name == "rod4":
        o = np.array([[-3, 0, 0], [-1, 0, 0], [1, 0, 0], [3, 0, 0]], float) * s
    elif name == "diamond":
        r3 = math.sqrt(3.0)
        o = np.array([[0, 1, 0], [0, -1, 0], [r3, 0, 0], [-r3, 0, 0]], float) * s
    elif name == "cube8":
        o = np.array([[i, j, k] for i in (-1, 1) for j in (-1, 1) for k in (-1, 1)], float) * s
    elif name == "single":
        o = np.zeros((1, 3))
    else:
        raise ValueError(name)
    return o


def bounding_radius(name: str, s: float) -> float:
    o = shape_offsets(name, s)
    return float(np.max(np.linalg.norm(o, axis=1)) + s)


def random_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z); R[:, 0, 1] = 2 * (x * y - w * z); R[:, 0, 2] = 2 * (x * z + w * y)
    R[:, 1, 0] = 2 * (x * y + w * z); R[:, 1, 1] = 1 - 2 * (x * x + z * z); R[:, 1, 2] = 2 * (y * z - w * x)
    R[:, 2, 0] = 2 * (x * z - w * y); R[:, 2, 1] = 2 * (y * z + w * x); R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def uniform_in_ball(rng, n, radius):
    v = rng.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    r = radius * rng.random(n) ** (1.0 / 3.0)
    return v * r[:, None]


def place_nonoverlapping(rng, bound_r: np.ndarray, ball_radius: float, max_tries=200) -> np.ndarray:
    """COMs uniform in a ball whose bounding spheres do not overlap (rejection)."""
    n = len(bound_r)
    cell = 2.0 * float(bound_r.max())
    grid: dict = {}
    out = np.empty((n, 3))
    for k in range(n):
        for _ in range(max_tries):
            c = uniform_in_ball(rng, 1, ball_radius - bound_r[k])[0]
            key = tuple(np.floor(c / cell).astype(int))
            ok = True
            for dx in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dz in (-1, 0, 1):
                        for j in grid.get((key[0] + dx, key[1] + dy, key[2] + dz), ()):
                            if np.sum((out[j] - c) ** 2) < (bound_r[j] + bound_r[k]) ** 2:
                                ok = False
                                break
                        if not ok:
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if ok:
                out[k] = c
                grid.setdefault(key, []).append(k)
                break
        else:
            raise RuntimeError("could not place aggregate without overlap; ball too small")
    return out


def assemble(shapes, sizes, coms, rots, density) -> PileIC:
    counts = np.array([SHAPE_SIZE.get(sh, 1) for sh in shapes], np.int32)
    N = int(counts.sum())
    pos = np.empty((N, 3))
    rad = np.empty(N)
    k = 0
    for a, sh in enumerate(shapes):
        o = shape_offsets(sh, sizes[a]) @ rots[a].T
        c = counts[a]
        pos[k:k + c] = coms[a] + o
        rad[k:k + c] = sizes[a]
        k += c
    return PileIC(counts=counts, pos=pos, radius=rad, density=np.full(N, float(density)),
                  vel=np.zeros((len(shapes), 3)), omega=np.zeros((len(shapes), 3)))


# ---------------------------------------------------------------------------
# parameter calibration
# ---------------------------------------------------------------------------
def damping_for_restitution(e: float, mu: float, k: float) -> float:
    if e >= 1.0:
        return 0.0
    L = -math.log(e)
    zeta = L / math.sqrt(math.pi ** 2 + L ** 2)
    return 2.0 * zeta * math.sqrt(mu * k)


def contact_time(k: float, c: float, mu: float) -> float:
    w0 = math.sqrt(k / mu)
    zeta = c / (2.0 * math.sqrt(mu * k))
    return math.pi / (w0 * math.sqrt(1.0 - zeta * zeta))


def sphere_mass(s, rho):
    return rho * 4.0 / 3.0 * math.pi * np.asarray(s, float) ** 3


def calibrate(ic: PileIC, *, v_max: float, r_med: float, e_n=0.5, e_t=0.5, mu_s=0.5, mu_r=0.1,
              mu_t=0.0, eps=None, overlap_frac=0.01, steps_per_contact=50,
              precision=PRECISION_MIXED, max_contacts=16, G=G_SI) -> Params:
    m = sphere_mass(ic.radius, ic.density)
    agg_mass = np.add.reduceat(m, np.concatenate([[0], np.cumsum(ic.counts)[:-1]]))
    mu_ref = 0.5 * float(agg_mass.mean())
    kn = mu_ref * v_max ** 2 / (overlap_frac * r_med) ** 2
    kt = 2.0 / 7.0 * kn
    cn = damping_for_restitution(e_n, mu_ref, kn)
    ct = damping_for_restitution(e_t, mu_ref, kt)
    tc = contact_time(kn, cn, mu_ref)
    return Params(G=G, dt=tc / steps_per_contact, kn=kn, kt=kt, cn=cn, ct=ct, mu_s=mu_s, mu_r=mu_r,
                  mu_t=mu_t, w0=1e-2 * v_max / r_med, eps=(0.1 * r_med if eps is None else eps),
                  precision=precision, max_contacts=max_contacts)


def total_mass(ic: PileIC) -> float:
    return float(np.sum(sphere_mass(ic.radius, ic.density)))


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
def config1(seed=0, precision=PRECISION_FP64, n_agg=250, ball=40.0):
    """250 tetrahedra, s = 1 m x U(0.9, 1.1), rho = 2500, COMs in a 40 m ball, at rest."""
    rng = np.random.default_rng(seed)
    sizes = 1.0 * rng.uniform(0.9, 1.1, n_agg)
    shapes = ["tetra"] * n_agg
    bound = np.array([bounding_radius("tetra", s) for s in sizes])
    coms = place_nonoverlapping(rng, bound, ball)
    ic = assemble(shapes, sizes, coms, random_rotations(rng, n_agg), 2500.0)
    vmax = math.sqrt(2 * G_SI * total_mass(ic) / ball)
    p = calibrate(ic, v_max=vmax, r_med=1.0, eps=0.1, precision=precision)
    ic.meta = dict(name="config1", seed=seed, steps=1000, ball=ball)
    return ic, p


def draw_shapes_exact(rng, n_spheres):
    """Shapes uniform from the four simple ones until the sphere count is exact."""
    out, left = [], n_spheres
    while left > 0:
        if left >= 6:
            sh = SHAPES[rng.integers(0, 4)]
        elif left == 5:
            sh = "dumbbell"
        elif left == 4:
            sh = ("tetra", "square")[rng.integers(0, 2)]
        elif left == 3:
            sh = "rod3"
        elif left == 2:
            sh = "dumbbell"
        else:
            raise AssertionError
        out.append(sh)
        left -= SHAPE_SIZE[sh]
    return out


def lognormal_truncated(rng, n, median, sigma, nsig=3.0):
    x = np.exp(np.clip(rng.standard_normal(n), -nsig, nsig) * sigma) * median
    return x


def config2(seed=0, precision=PRECISION_MIXED, n_spheres=100_000, ball=2000.0):
    """Collapse of a 2 km cloud: mixed simple shapes, radii lognormal(5 m, 0.2), at rest."""
    rng = np.random.default_rng(seed)
    shapes = draw_shapes_exact(rng, n_spheres)
    A = len(shapes)
    sizes = lognormal_truncated(rng, A, 5.0, 0.2)
    bound = np.array([bounding_radius(sh, s) for sh, s in zip(shapes, sizes)])
    coms = place_nonoverlapping(rng, bound, ball)
    ic = assemble(shapes, sizes, coms, random_rotations(rng, A), 2500.0)
    vmax = math.sqrt(2 * G_SI * total_mass(ic) / ball)
    p = calibrate(ic, v_max=vmax, r_med=5.0, eps=0.5, precision=precision)
    ic.meta = dict(name="config2", seed=seed, ball=ball)
    return ic, p


def e2_collapse(kind="mixed", seed=0, precision=PRECISION_MIXED, n_spheres=20_000, s=50.0,
                ball=None):
    """The paper's self-gravity profiling collapse (Sec. 3): N = 2e4 equal spheres of
    radius 50 m, all free ("spheres"), all bonded into one shape (one of E_SHAPES:
    2,500 cubes ... 10,000 dumbbells), or a uniform mix of the five shapes ("mixed",
    topped up with free spheres to the exact count); COMs uniform in a ball (bounding
    spheres disjoint), at rest, random orientations.  The paper does not give the
    cloud size: the ball is 3 km, or larger where the bounding spheres would fill
    more than 15% of it (random placement fails much above that), so contacts form
    as the cloud collapses."""
    rng = np.random.default_rng(seed)
    if kind == "spheres":
        shapes = ["single"] * n_spheres
    elif kind == "mixed":
        shapes, left = [], n_spheres
        while left > 0:
            sh = E_SHAPES[rng.integers(0, len(E_SHAPES))]
            if SHAPE_SIZE[sh] > left:
                sh = "single"
            shapes.append(sh)
            left -= SHAPE_SIZE[sh]
    elif kind in E_SHAPES:
        if n_spheres % SHAPE_SIZE[kind]:
            raise ValueError("sphere count not a multiple of the shape size")
        shapes = [kind] * (n_spheres // SHAPE_SIZE[kind])
    else:
        raise ValueError(kind)
    A = len(shapes)
    sizes = np.full(A, float(s))
    bound = np.array([bounding_radius(sh, s) for sh in shapes])
    if ball is None:
        ball = max(3000.0 * s / 50.0, float(np.sum(bound ** 3) / 0.15) ** (1.0 / 3.0))
    coms = place_nonoverlapping(rng, bound, ball)
    ic = assemble(shapes, sizes, coms, random_rotations(rng, A), 2500.0)
    vmax = math.sqrt(2 * G_SI * total_mass(ic) / ball)
    p = calibrate(ic, v_max=vmax, r_med=s, eps=0.1 * s, precision=precision)
    ic.meta = dict(name=f"e2_{kind}", seed=seed, ball=ball, steps=10_000)
    return ic, p


def lattice_pile(rng, n_agg, s_med=1.0, s_jit=0.1, shapes=("tetra",), spacing_factor=1.0,
                 center=(0.0, 0.0, 0.0), rho=2500.0):
    """Aggregates on a jittered cubic lattice inside a sphere, bounding spheres disjoint."""
    sh = [shapes[rng.integers(0, len(shapes))] for _ in range(n_agg)]
    sizes = s_med * rng.uniform(1 - s_jit, 1 + s_jit, n_agg)
    bmax = max(bounding_radius(x, s_med * (1 + s_jit)) for x in set(sh))
    a = 2.0 * bmax * spacing_factor
    # enough lattice points in a ball
    R = a * (3.0 * n_agg / (4.0 * math.pi)) ** (1.0 / 3.0) * 1.1 + a
    n1 = int(math.ceil(R / a))
    g = np.arange(-n1, n1 + 1) * a
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    pts = pts[np.argsort(np.linalg.norm(pts, axis=1), kind="stable")][:n_agg]
    jit = (a - 2.0 * bmax) * 0.5
    pts = pts + (rng.uniform(-jit, jit, pts.shape) if jit > 0 else 0.0) + np.asarray(center)
    return assemble(sh, sizes, pts, random_rotations(rng, n_agg), rho)


def settled_params(ic: PileIC, r_med: float, extra_speed=0.0, precision=PRECISION_MIXED, **kw):
    """Parameters for a bound pile: v_max from the escape speed (+ extra)."""
    com = np.average(ic.pos, axis=0, weights=sphere_mass(ic.radius, ic.density))
    Rp = float(np.max(np.linalg.norm(ic.pos - com, axis=1)))
    vesc = math.sqrt(2 * G_SI * total_mass(ic) / Rp)
    return calibrate(ic, v_max=vesc + extra_speed, r_med=r_med, precision=precision, **kw)


def config3(seed=0, precision=PRECISION_MIXED, n_spheres=200_000):
    """Spin-up pile: 2-8-sphere touching clusters in a 3:2:1.5 ellipsoid, YORP ramp.

    Clusters are grown by tangent attachment; COMs on a jittered lattice
    clipped to the ellipsoid.  Spin increment: 1e-6 rad/s per 1,000 steps
    about the pile's shortest axis (z here).
    """
    rng = np.random.default_rng(seed)
    counts, offs = [], []
    left = n_spheres
    while left > 0:
        k = int(rng.integers(2, 9))
        if left - k == 1:
            k += 1
        k = min(k, left)
        if k < 2:
            k = 2
        counts.append(k)
        offs.append(_touching_cluster(rng, k))
        left -= k
    A = len(counts)
    s = 1.0 * rng.uniform(0.9, 1.1, A)
    bound = np.array([np.max(np.linalg.norm(o, axis=1)) + 1.0 for o in offs]) * s
    a = 2.0 * float(bound.max())
    # lattice clipped to an ellipsoid with axes 3:2:1.5
    scale = 1.0
    while True:
        ax = np.array([3.0, 2.0, 1.5]) * scale
        n1 = [int(math.ceil(x / a)) for x in ax]
        g = [np.arange(-n, n + 1) * a for n in n1]
        X, Y, Z = np.meshgrid(*g, indexing="ij")
        pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
        inside = np.sum((pts / ax) ** 2, 1) <= 1.0
        if inside.sum() >= A:
            pts = pts[inside]
            break
        scale *= 1.05
    order = np.argsort(np.sum((pts / ax) ** 2, 1), kind="stable")[:A]
    coms = pts[order]
    rots = random_rotations(rng, A)
    N = int(sum(counts))
    pos = np.empty((N, 3))
    rad = np.empty(N)
    k = 0
    for i in range(A):
        c = counts[i]
        pos[k:k + c] = coms[i] + (offs[i] * s[i]) @ rots[i].T
        rad[k:k + c] = s[i]
        k += c
    ic = PileIC(counts=np.array(counts, np.int32), pos=pos, radius=rad, density=np.full(N, 2500.0),
                vel=np.zeros((A, 3)), omega=np.zeros((A, 3)))
    p = settled_params(ic, 1.0, precision=precision, eps=0.1)
    p = p.replace(spin_inc=(0.0, 0.0, 1e-9))
    ic.meta = dict(name="config3", seed=seed)
    return ic, p


def config3_settled(seed=0, precision=PRECISION_MIXED, n_spheres=200_000, overlap=1e-5):
    """Spin-up pile, pre-settled: equal spheres (s = 1 m) on a face-centred cubic
    packing clipped to a 3:2:1.5 ellipsoid, neighbours overlapping by
    `overlap` x s (about what the pile's own weight presses into the contacts
    at its centre), so nearly every sphere starts with contacts.  The sites
    are cut into aggregates of 2-8 face-adjacent spheres (size uniform, grown
    from a random seed site by random attachment to the cluster; a site left
    with no free neighbour joins an adjacent aggregate of fewer than 8, else
    stays a single sphere).  At rest; spin increment 1e-6 rad/s per 1,000
    steps about the shortest axis (z).  A geometric stand-in for a pile
    settled by the dynamics (settling with this library would make the
    oracle's input a product of the CUDA path)."""
    rng = np.random.default_rng(seed)
    s = 1.0
    h = s * (1.0 - overlap / 2.0) * math.sqrt(2.0)      # half the cubic cell: site (i, j, k) * h
    ax = np.array([3.0, 2.0, 1.5])
    c = (n_spheres * 2.0 * h ** 3 / (4.0 / 3.0 * math.pi * 9.0)) ** (1.0 / 3.0) * 1.05
    while True:
        n = [int(math.ceil(x * c / h)) + 1 for x in ax]
        g = [np.arange(-m, m + 1) for m in n]
        I, J, K = np.meshgrid(*g, indexing="ij")
        ijk = np.stack([I.ravel(), J.ravel(), K.ravel()], 1)
        ijk = ijk[(ijk.sum(1) % 2) == 0]
        e2 = np.sum((ijk * h / (ax * c)) ** 2, 1)
        if int((e2 <= 1.0).sum()) >= n_spheres:
            break
        c *= 1.05
    order = np.lexsort((ijk[:, 2], ijk[:, 1], ijk[:, 0], e2))[:n_spheres]
    ijk = ijk[order]
    site = {tuple(v): t for t, v in enumerate(ijk.tolist())}
    nb = np.array([(a, b, 0) for a in (-1, 1) for b in (-1, 1)] + [(a, 0, b) for a in (-1, 1) for b in (-1, 1)]
                  + [(0, a, b) for a in (-1, 1) for b in (-1, 1)])
    N = n_spheres
    adj = np.full((N, 12), -1, np.int64)
    for t, v in enumerate(ijk):
        for q, d in enumerate(nb):
            adj[t, q] = site.get((v[0] + d[0], v[1] + d[1], v[2] + d[2]), -1)
    owner = np.full(N, -1, np.int64)
    members = []
    for t in rng.permutation(N):
        if owner[t] >= 0:
            continue
        want = int(rng.integers(2, 9))
        cl = [int(t)]
        owner[t] = len(members)
        while len(cl) < want:
            front = [u for m in cl for u in adj[m] if u >= 0 and owner[u] < 0]
            if not front:
                break
            u = int(front[rng.integers(0, len(front))])
            owner[u] = len(members)
            cl.append(u)
        if len(cl) == 1:
            near = [owner[u] for u in adj[t] if u >= 0 and owner[u] >= 0 and owner[u] != len(members)
                    and len(members[owner[u]]) < 8]
            if near:
                g_ = int(min(near, key=lambda x: (len(members[x]), x)))
                owner[t] = g_
                members[g_].append(int(t))
                continue
        members.append(cl)
    counts = np.array([len(m) for m in members], np.int32)
    flat = np.concatenate([np.array(sorted(m), np.int64) for m in members])
    pos = (ijk[flat] * h).astype(np.float64)
    A = len(members)
    ic = PileIC(counts=counts, pos=pos, radius=np.full(N, s), density=np.full(N, 2500.0),
                vel=np.zeros((A, 3)), omega=np.zeros((A, 3)))
    p = settled_params(ic, s, precision=precision, eps=0.1 * s)
    p = p.replace(spin_inc=(0.0, 0.0, 1e-9))
    ic.meta = dict(name="config3_settled", seed=seed, overlap=overlap)
    return ic, p


def _touching_cluster(rng, k):
    """Offsets (unit radius) of k spheres grown by tangent attachment to a random
    member without overlapping any other member; centred on the mean."""
    pts = [np.zeros(3)]
    while len(pts) < k:
        base = pts[rng.integers(0, len(pts))]
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        c = base + 2.0 * d
        if all(np.linalg.norm(c - p) >= 2.0 - 1e-9 for p in pts):
            pts.append(c)
    P = np.array(pts)
    return P - P.mean(0)


def pile_sizes_config4(rng, n_piles=256, median=3000.0, lo=500, hi=20000):
    sigma = math.log(hi / lo) / 4.0
    out = []
    while len(out) < n_piles:
        x = int(round(median * math.exp(sigma * rng.standard_normal())))
        if lo <= x <= hi:
            out.append(x - x % 4)
    return out


def config4(seed=0, precision=PRECISION_MIXED, n_piles=256):
    """256 independent piles of tetrahedra, sizes lognormal in [500, 20000] spheres."""
    rng = np.random.default_rng(seed)
    sizes = pile_sizes_config4(rng, n_piles)
    piles = []
    for k, n in enumerate(sizes):
        ic = lattice_pile(rng, n // 4, shapes=("tetra",), spacing_factor=1.0)
        p = settled_params(ic, 1.0, precision=precision, eps=0.1)
        ic.meta = dict(name="config4", seed=seed, index=k)
        piles.append((ic, p))
    return piles


def dense_lattice(n_spheres=100_000, seed=0, overlap=0.005, precision=PRECISION_MIXED, s=1.0,
                  jitter=0.1, speed=1e-3):
    """Contact-stress case: tetrahedra from the 4-sphere basis of an FCC lattice whose
    nearest neighbours overlap by `overlap` x R; each aggregate gets a small rigid jitter
    and a random velocity and spin so that normal, tangential and rolling terms are live."""
    rng = np.random.default_rng(seed)
    n_cells = max(1, n_spheres // 4)
    d_nn = 2.0 * s * (1.0 - overlap / 2.0)          # neighbour distance
    a = d_nn * math.sqrt(2.0)                        # cubic cell edge
    n1 = int(math.ceil(n_cells ** (1.0 / 3.0)))
    idx = np.array([(i, j, k) for i in range(n1) for j in range(n1) for k in range(n1)], float)
    idx = idx[np.argsort(np.linalg.norm(idx - (n1 - 1) / 2.0, axis=1), kind="stable")][:n_cells]
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]]) * a
    centre = basis.mean(0)
    A = n_cells
    pos = np.empty((4 * A, 3))
    jit = rng.uniform(-1, 1, (A, 3)) * jitter * overlap * s
    for c in range(A):
        pos[4 * c:4 * c + 4] = idx[c] * a + basis - centre + jit[c]
    ic = PileIC(counts=np.full(A, 4, np.int32), pos=pos, radius=np.full(4 * A, s),
                density=np.full(4 * A, 2500.0),
                vel=rng.standard_normal((A, 3)) * speed,
                omega=rng.standard_normal((A, 3)) * speed / s)
    p = calibrate(ic, v_max=max(speed * 10, 1e-6), r_med=s, eps=0.1 * s, precision=precision,
                  overlap_frac=0.02)
    ic.meta = dict(name="dense_lattice", seed=seed)
    return ic, p


def planet_flyby(ic: PileIC, rng, periapsis_rp=(1.5, 4.0), v_inf_kms=(1.0, 10.0),
                 start_roche=10.0, rho_planet=5514.0):
    """Planet (Earth) on a hyperbola relative to the pile COM, started at 10x the
    Roche distance on the incoming branch (Sec. 4.2 setting).  Returns (mass,
    pos, vel) in the pile's frame (pile COM at rest at the origin)."""
    q = rng.uniform(*periapsis_rp) * EARTH_RADIUS
    vinf = rng.uniform(*v_inf_kms) * 1e3
    rho_pile = 2500.0 * 0.6
    d_roche = 1.26 * EARTH_RADIUS * (rho_planet / rho_pile) ** (1.0 / 3.0)
    r0 = start_roche * d_roche
    mu = G_SI * EARTH_MASS
    a = -mu / vinf ** 2                     # semi-major axis (negative)
    e = 1.0 - q / a                         # eccentricity > 1
    p = a * (1 - e * e)
    cosf = (p / r0 - 1.0) / e
    f = -math.acos(max(-1.0, min(1.0, cosf)))   # incoming branch
    r = p / (1 + e * math.cos(f))
    pos = np.array([r * math.cos(f), r * math.sin(f), 0.0])
    h = math.sqrt(mu * p)
    vel = np.array([-mu / h * math.sin(f), mu / h * (e + math.cos(f)), 0.0])
    # planet position/velocity relative to the pile = minus the pile's relative orbit
    return EARTH_MASS, -pos, -vel, dict(q=q, vinf=vinf, e=e)


def config5_trace(seed=0, n_arrivals=64, rate=4.0, n_lo=1000, n_hi=100_000, steps=20_000,
                  precision=PRECISION_MIXED):
    """Poisson arrivals of tidal-encounter simulations (log-uniform sizes)."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    for k in range(n_arrivals):
        t += rng.exponential(1.0 / rate)
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        n -= n % 4
        out.append(dict(t_arrival=t, n_spheres=max(n, 4), seed=int(rng.integers(2 ** 31)),
                        steps=steps))
    return out


def config5_pile(req, precision=PRECISION_MIXED):
    rng = np.random.default_rng(req["seed"])
    ic = lattice_pile(rng, req["n_spheres"] // 4, shapes=("tetra",), spacing_factor=1.0)
    p = settled_params(ic, 1.0, precision=precision, eps=0.1)
    mP, xP, vP, orb = planet_flyby(ic, rng)
    com = np.average(ic.pos, axis=0, weights=sphere_mass(ic.radius, ic.density))
    p = p.replace(ext_mass=mP, ext_pos=tuple(com + xP), ext_vel=tuple(vP))
    ic.meta = dict(name="config5", orbit=orb, **req)
    return ic, p


def tiny_pair(s1=1.0, s2=1.0, gap=-0.01, v=0.0, rho=2500.0, b=0.0):
    """Two single-sphere aggregates on the x axis, approaching at relative speed v.
    gap < 0 means initial overlap; b is an impact parameter along y."""
    pos = np.array([[0.0, 0.0, 0.0], [s1 + s2 + gap, b, 0.0]])
    return PileIC(counts=np.array([1, 1], np.int32), pos=pos, radius=np.array([s1, s2]),
                  density=np.full(2, rho), vel=np.array([[0.5 * v, 0, 0], [-0.5 * v, 0, 0]]),
                  omega=np.zeros((2, 3)))


def random_cluster(seed, n_agg=40, shapes=SHAPES, s=1.0, box=6.0, speed=0.05,
                   precision=PRECISION_FP64):
    """Small random set of aggregates in a box, allowed to overlap (for contact tests)."""
    rng = np.random.default_rng(seed)
    sh = [shapes[rng.integers(0, len(shapes))] for _ in range(n_agg)]
    sizes = s * rng.uniform(0.8, 1.2, n_agg)
    coms = rng.uniform(-box, box, (n_agg, 3))
    ic = assemble(sh, sizes, coms, random_rotations(rng, n_agg), 2500.0)
    ic.vel = rng.standard_normal((n_agg, 3)) * speed
    ic.omega = rng.standard_normal((n_agg, 3)) * speed / s
    p = calibrate(ic, v_max=speed * 5, r_med=s, eps=0.1 * s, precision=precision, overlap_frac=0.05,
                  max_contacts=32)
    return ic, p
