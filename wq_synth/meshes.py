"""Seeded synthetic control meshes (input data only).

This module builds quad control meshes and nothing else: vertex positions,
CCW quads and, for every face, the index of the initial-mesh face it descends
from (``level0_face``; -1 for faces of an added passive ring).  It holds none
of the weighted-quadrature arithmetic: no spline construction, classification,
quadrature or weights.  Both the CPU oracle and the GPU library read its
output.

Stand-ins for the paper's meshes (Sec. 6: unit square with two EPs, Fig. 4;
hemisphere, Fig. 10; aircraft nose, Fig. 11), whose control nets are not
published:

* ``disk``      -- mu quad sectors of n x n faces around one EP of valence mu
                   (polar layout, seeded jitter), the 180-face valence-5 disk at
                   mu=5, n=6.
* ``rotated``   -- a rectangular core grid with random interior edge rotations
                   (which create valence 3/5/6 EPs), Tutte-embedded, refined
                   uniformly and wrapped in one passive ring.
* ``cube_sphere`` -- a cube net subdivided and projected to a perturbed sphere
                   (closed surface, eight valence-3 EPs).
* ``grid``      -- an EP-free rectangular grid wrapped in one passive ring.

Every generator takes an explicit ``seed`` and uses NumPy's PCG64.
"""
from __future__ import annotations

import numpy as np


# ----------------------------------------------------------------------------
# small helpers (topology bookkeeping only)
# ----------------------------------------------------------------------------

def _edge_key(a, b):
    return (a, b) if a < b else (b, a)


def refine(xyz, quads, level0_face):
    """Uniform topological refinement: each quad -> 4 quads.

    New vertices sit at edge midpoints and face centroids (bilinear
    positions); children keep their parent's ``level0_face``.
    """
    xyz = [tuple(p) for p in np.asarray(xyz, dtype=np.float64)]
    quads = np.asarray(quads)
    mid = {}
    new_quads = []
    new_l0 = []

    def midpoint(a, b):
        k = _edge_key(a, b)
        if k not in mid:
            pa, pb = np.array(xyz[a]), np.array(xyz[b])
            xyz.append(tuple(0.5 * (pa + pb)))
            mid[k] = len(xyz) - 1
        return mid[k]

    for f, (v0, v1, v2, v3) in enumerate(quads):
        m01, m12 = midpoint(v0, v1), midpoint(v1, v2)
        m23, m30 = midpoint(v2, v3), midpoint(v3, v0)
        c = np.mean([xyz[v0], xyz[v1], xyz[v2], xyz[v3]], axis=0)
        xyz.append(tuple(c))
        ci = len(xyz) - 1
        for q in ((v0, m01, ci, m30), (m01, v1, m12, ci), (ci, m12, v2, m23), (m30, ci, m23, v3)):
            new_quads.append(q)
            new_l0.append(level0_face[f])
    return (np.array(xyz, dtype=np.float64), np.array(new_quads, dtype=np.int32),
            np.array(new_l0, dtype=np.int32))


def _boundary_loop(quads):
    """Ordered boundary loop (CCW for CCW faces) of a disk-topology quad mesh."""
    cnt = {}
    directed = {}
    for q in quads:
        for k in range(4):
            a, b = int(q[k]), int(q[(k + 1) % 4])
            cnt[_edge_key(a, b)] = cnt.get(_edge_key(a, b), 0) + 1
            directed[(a, b)] = True
    nxt = {}
    for q in quads:
        for k in range(4):
            a, b = int(q[k]), int(q[(k + 1) % 4])
            if cnt[_edge_key(a, b)] == 1:
                nxt[a] = b
    start = min(nxt)
    loop = [start]
    while True:
        n = nxt[loop[-1]]
        if n == start:
            break
        loop.append(n)
    return loop


def wrap_passive_ring(xyz, quads, level0_face, h):
    """Add one ring of quads around the boundary of a planar disk mesh.

    Boundary vertices of valence 3 get one outward edge; valence-2 corners get
    two outward edges and a corner quad, so that every old boundary vertex is
    interior with valence 4 afterwards.  New vertices are placed at distance
    ``h`` along the outward normal(s).  New faces get ``level0_face = -1``.
    """
    xyz = np.asarray(xyz, dtype=np.float64)
    quads = np.asarray(quads)
    loop = _boundary_loop(quads)
    nb = len(loop)
    deg = {}
    for q in quads:
        for k in range(4):
            a, b = int(q[k]), int(q[(k + 1) % 4])
            for v, w in ((a, b), (b, a)):
                deg.setdefault(v, set()).add(w)
    pts = list(map(tuple, xyz))
    outer_first, outer_last, corner_vertex = {}, {}, {}

    def normal(a, b):
        d = xyz[b, :2] - xyz[a, :2]
        n = np.array([d[1], -d[0]])          # right of a->b; outward for a CCW loop
        return n / np.linalg.norm(n)

    for i, v in enumerate(loop):
        prev_v, next_v = loop[i - 1], loop[(i + 1) % nb]
        n_in, n_out = normal(prev_v, v), normal(v, next_v)
        val = len(deg[v])
        base = xyz[v].copy()
        if val == 3:
            nrm = n_in + n_out
            nrm /= np.linalg.norm(nrm)
            p = base.copy()
            p[:2] += h * nrm
            pts.append(tuple(p))
            outer_first[v] = outer_last[v] = len(pts) - 1
        elif val == 2:
            p1, p2, pc = base.copy(), base.copy(), base.copy()
            p1[:2] += h * n_in
            p2[:2] += h * n_out
            pc[:2] += h * (n_in + n_out)
            pts.append(tuple(p1)); o1 = len(pts) - 1
            pts.append(tuple(pc)); oc = len(pts) - 1
            pts.append(tuple(p2)); o2 = len(pts) - 1
            outer_first[v], corner_vertex[v], outer_last[v] = o1, oc, o2
        else:
            raise ValueError("boundary vertex of valence %d cannot be wrapped" % val)
    new_quads = [tuple(q) for q in quads]
    new_l0 = list(level0_face)
    for i, v in enumerate(loop):
        w = loop[(i + 1) % nb]
        # quad on boundary edge v->w (CCW loop => outward side on the right)
        new_quads.append((w, v, outer_last[v], outer_first[w]))
        new_l0.append(-1)
        if v in corner_vertex:
            new_quads.append((v, outer_first[v], corner_vertex[v], outer_last[v]))
            new_l0.append(-1)
    return (np.array(pts, dtype=np.float64), np.array(new_quads, dtype=np.int32),
            np.array(new_l0, dtype=np.int32))


def _pack(xyz, quads, level0_face, dim, name, **extra):
    d = {"xyz": np.ascontiguousarray(xyz, dtype=np.float64),
         "quads": np.ascontiguousarray(quads, dtype=np.int32),
         "level0_face": np.ascontiguousarray(level0_face, dtype=np.int32),
         "dim": int(dim), "name": name}
    d.update(extra)
    return d


# ----------------------------------------------------------------------------
# generators
# ----------------------------------------------------------------------------

def grid(nx, ny, seed=0, jitter=0.0, levels=0):
    """EP-free nx x ny core grid on [0,1]x[0,ny/nx], refined, wrapped in a passive ring."""
    rng = np.random.Generator(np.random.PCG64(seed))
    xs, ys = np.meshgrid(np.arange(nx + 1) / nx, np.arange(ny + 1) / nx, indexing="ij")
    xyz = np.stack([xs.ravel(), ys.ravel(), np.zeros(xs.size)], axis=1)
    vid = lambda i, j: i * (ny + 1) + j
    quads = [(vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1))
             for i in range(nx) for j in range(ny)]
    l0 = np.arange(len(quads), dtype=np.int32)
    xyz, quads, l0 = np.asarray(xyz), np.asarray(quads, dtype=np.int32), l0
    for _ in range(levels):
        xyz, quads, l0 = refine(xyz, quads, l0)
    h = 1.0 / (nx * 2 ** levels)
    if jitter > 0:
        bnd = set(_boundary_loop(quads))
        for v in range(len(xyz)):
            if v not in bnd:
                xyz[v, :2] += rng.uniform(-jitter * h, jitter * h, size=2)
    xyz, quads, l0 = wrap_passive_ring(xyz, quads, l0, h)
    return _pack(xyz, quads, l0, 2, "grid%dx%d_L%d" % (nx, ny, levels))


def disk(mu=5, n=6, seed=1001, jitter=0.01, levels=0):
    """mu sectors of n x n faces around one EP of valence mu.

    Sector s holds vertices (a, b) in [0, N]^2 (N = n * 2**levels) with the EP
    at (0, 0); vertex (a, b) goes to radius max(a, b)/N and angle
    2 pi s/mu + (2 pi/mu) b/(a+b).  Non-EP interior vertices get
    U(-jitter/N, jitter/N) per coordinate.  Faces of the fine grid record the
    coarse (n x n per sector) face they descend from, so the region around the
    EP keeps its initial size under refinement.  The outermost face ring
    touches the boundary (passive).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    N = n * 2 ** levels
    ids, coords = {}, []

    def vid(s, a, b):
        # shared spokes: (a, 0) of sector s is (0, a) of sector s-1
        if a == 0 and b == 0:
            key = ("ep",)
        elif a == 0:
            key = ((s + 1) % mu, b, 0)
        else:
            key = (s % mu, a, b)
        if key not in ids:
            ids[key] = len(coords)
            coords.append((key[0] if len(key) == 3 else 0, key[1] if len(key) == 3 else 0,
                           key[2] if len(key) == 3 else 0))
        return ids[key]

    quads, l0 = [], []
    for s in range(mu):
        for a in range(N):
            for b in range(N):
                quads.append((vid(s, a, b), vid(s, a + 1, b), vid(s, a + 1, b + 1), vid(s, a, b + 1)))
                l0.append(s * n * n + (a >> levels) * n + (b >> levels))
    xyz = np.zeros((len(coords), 3))
    for v, (s, a, b) in enumerate(coords):
        if a == 0 and b == 0:
            continue
        r = max(a, b) / N
        phi = 2 * np.pi * s / mu + (2 * np.pi / mu) * b / (a + b)
        xyz[v, 0], xyz[v, 1] = r * np.cos(phi), r * np.sin(phi)
    for v, (s, a, b) in enumerate(coords):
        if (a == 0 and b == 0) or max(a, b) == N:
            continue
        xyz[v, :2] += rng.uniform(-jitter / N, jitter / N, size=2)
    return _pack(xyz, np.array(quads, dtype=np.int32), np.array(l0, dtype=np.int32), 2,
                 "disk_mu%d_n%d_L%d" % (mu, n, levels))


def _valences(quads, nv):
    nbrs = [set() for _ in range(nv)]
    for q in quads:
        for k in range(4):
            a, b = q[k], q[(k + 1) % 4]
            nbrs[a].add(b); nbrs[b].add(a)
    return np.array([len(s) for s in nbrs])


def _try_rotate(quads, e2f, a, b, rng):
    """Rotate interior edge (a, b) inside the hexagon of its two quads."""
    fs = e2f.get(_edge_key(a, b), [])
    if len(fs) != 2:
        return None
    f1, f2 = fs
    q1, q2 = list(quads[f1]), list(quads[f2])
    # orient q1 so it starts a -> b
    k = q1.index(a)
    q1 = q1[k:] + q1[:k]
    if q1[1] != b:
        return None
    k = q2.index(b)
    q2 = q2[k:] + q2[:k]
    if q2[1] != a:
        return None
    # q1 = [a, b, c, d], q2 = [b, a, e, f]; hexagon (CCW) = b, c, d, a, e, f
    hexa = [q1[1], q1[2], q1[3], q1[0], q2[2], q2[3]]
    if len(set(hexa)) != 6:
        return None
    r = rng.integers(2)
    if r == 0:   # diagonal h1-h4
        n1 = [hexa[1], hexa[2], hexa[3], hexa[4]]
        n2 = [hexa[4], hexa[5], hexa[0], hexa[1]]
    else:        # diagonal h2-h5
        n1 = [hexa[2], hexa[3], hexa[4], hexa[5]]
        n2 = [hexa[5], hexa[0], hexa[1], hexa[2]]
    return f1, f2, n1, n2


def _tutte(nv, quads, fixed_pos):
    """Tutte (barycentric) embedding with the given fixed boundary positions."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    nbrs = [set() for _ in range(nv)]
    for q in quads:
        for k in range(4):
            a, b = q[k], q[(k + 1) % 4]
            nbrs[a].add(b); nbrs[b].add(a)
    free = [v for v in range(nv) if v not in fixed_pos]
    idx = {v: i for i, v in enumerate(free)}
    rows, cols, vals = [], [], []
    rhs = np.zeros((len(free), 2))
    for v in free:
        i = idx[v]
        rows.append(i); cols.append(i); vals.append(float(len(nbrs[v])))
        for w in nbrs[v]:
            if w in idx:
                rows.append(i); cols.append(idx[w]); vals.append(-1.0)
            else:
                rhs[i] += fixed_pos[w]
    L = sp.csr_matrix((vals, (rows, cols)), shape=(len(free), len(free)))
    pos = np.zeros((nv, 2))
    for v, p in fixed_pos.items():
        pos[v] = p
    sol = np.column_stack([spla.spsolve(L.tocsc(), rhs[:, 0]), spla.spsolve(L.tocsc(), rhs[:, 1])])
    for v in free:
        pos[v] = sol[idx[v]]
    return pos


def _quads_convex(pos, quads, min_sin=0.15):
    for q in quads:
        p = pos[list(q)]
        for k in range(4):
            a, b, c = p[k - 1], p[k], p[(k + 1) % 4]
            u, w = b - a, c - b
            cr = u[0] * w[1] - u[1] * w[0]
            if cr <= min_sin * np.linalg.norm(u) * np.linalg.norm(w):
                return False
    return True


def rotated(nx=8, ny=5, n_ep=12, valences=(3, 5, 6), levels=4, seed=2001, jitter=0.02,
            max_tries=2000):
    """Planar core grid with random interior edge rotations, refined and wrapped.

    The nx x ny core keeps its boundary vertices regular; random edge rotations
    among core-interior vertices are drawn until exactly ``n_ep`` interior
    vertices have valence != 4, all in ``valences``.  The core is Tutte-embedded
    (boundary fixed on the rectangle [0, nx] x [0, ny]), refined ``levels`` times
    (bilinear positions), jittered by U(+-jitter * h) with h the fine spacing
    (core-boundary vertices stay fixed) and wrapped in one passive ring.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    vid = lambda i, j: i * (ny + 1) + j
    nv = (nx + 1) * (ny + 1)
    base = [(vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)) for i in range(nx) for j in range(ny)]
    core_bnd = {vid(i, j) for i in range(nx + 1) for j in range(ny + 1)
                if i in (0, nx) or j in (0, ny)}
    fixed = {vid(i, j): np.array([float(i), float(j)]) for i in range(nx + 1) for j in range(ny + 1)
             if vid(i, j) in core_bnd}
    base_val = _valences(base, nv)
    for _ in range(max_tries):
        quads = [list(q) for q in base]
        for _step in range(400):
            e2f = {}
            for f, q in enumerate(quads):
                for k in range(4):
                    e2f.setdefault(_edge_key(q[k], q[(k + 1) % 4]), []).append(f)
            edges = [e for e, fs in e2f.items() if len(fs) == 2
                     and e[0] not in core_bnd and e[1] not in core_bnd]
            a, b = edges[rng.integers(len(edges))]
            r = _try_rotate(quads, e2f, a, b, rng)
            if r is None:
                continue
            f1, f2, n1, n2 = r
            trial = [list(q) for q in quads]
            trial[f1], trial[f2] = n1, n2
            val = _valences(trial, nv)
            bad = False
            for v in core_bnd:
                if val[v] != base_val[v]:
                    bad = True
                    break
            if bad or any(val[v] < 3 or val[v] > max(valences) for v in range(nv) if v not in core_bnd):
                continue
            # no two faces may share two edges
            ok = True
            for f in (f1, f2):
                for g, q in enumerate(trial):
                    if g != f and len(set(q) & set(trial[f])) > 2:
                        ok = False
            if not ok:
                continue
            quads = trial
            eps = [v for v in range(nv) if v not in core_bnd and val[v] != 4]
            if len(eps) >= n_ep:
                break
        val = _valences(quads, nv)
        eps = [v for v in range(nv) if v not in core_bnd and val[v] != 4]
        if len(eps) != n_ep or any(val[v] not in valences for v in eps):
            continue
        pos = _tutte(nv, quads, fixed)
        if not _quads_convex(pos, quads):
            continue
        xyz = np.zeros((nv, 3))
        xyz[:, :2] = pos
        q = np.array(quads, dtype=np.int32)
        l0 = np.arange(len(q), dtype=np.int32)
        for _l in range(levels):
            xyz, q, l0 = refine(xyz, q, l0)
        h = 1.0 / 2 ** levels
        bnd = set(_boundary_loop(q))
        for v in range(len(xyz)):
            if v not in bnd:
                xyz[v, :2] += rng.uniform(-jitter * h, jitter * h, size=2)
        xyz, q, l0 = wrap_passive_ring(xyz, q, l0, h)
        return _pack(xyz, q, l0, 2, "rotated%dx%d_ep%d_L%d" % (nx, ny, n_ep, levels),
                     n_coarse_faces=nx * ny)
    raise RuntimeError("could not draw a valid rotated core mesh")


def cube_sphere(pre=3, levels=3, seed=3001, amp=0.05, n_bumps=8):
    """Cube net subdivided ``pre`` times (initial mesh), refined ``levels`` times,
    projected to the sphere of radius 1 + amp * h(x), h a sum of Gaussian bumps
    scaled to max |h| = 1.  Closed surface with eight valence-3 EPs."""
    rng = np.random.Generator(np.random.PCG64(seed))
    m = 2 ** pre * 2 ** levels          # cells per cube edge at the final level
    m0 = 2 ** pre
    ids = {}
    pts = []

    def vid(p):
        key = tuple(int(round(c)) for c in p)
        if key not in ids:
            ids[key] = len(pts)
            pts.append(key)
        return ids[key]

    quads, l0 = [], []
    # each cube face: fixed axis k at +-m/2, other two axes spanning [-m/2, m/2]
    faces = []
    for k in range(3):
        for sgn in (-1, 1):
            faces.append((k, sgn))
    for fi, (k, sgn) in enumerate(faces):
        a1, a2 = [ax for ax in range(3) if ax != k]
        for i in range(m):
            for j in range(m):
                def P(ii, jj):
                    p = [0, 0, 0]
                    p[k] = sgn * m
                    p[a1] = 2 * ii - m
                    p[a2] = 2 * jj - m
                    return vid(p)
                q = [P(i, j), P(i + 1, j), P(i + 1, j + 1), P(i, j + 1)]
                # outward orientation: normal along sgn * e_k
                e1 = np.zeros(3); e1[a1] = 1
                e2 = np.zeros(3); e2[a2] = 1
                if np.dot(np.cross(e1, e2), np.eye(3)[k]) * sgn < 0:
                    q = q[::-1]
                quads.append(q)
                l0.append(fi * m0 * m0 + (i * m0 // m) * m0 + (j * m0 // m))
    xyz = np.array(pts, dtype=np.float64)
    u = xyz / np.linalg.norm(xyz, axis=1, keepdims=True)
    centers = rng.normal(size=(n_bumps, 3))
    centers /= np.linalg.norm(centers, axis=1, keepdims=True)
    signs = rng.choice([-1.0, 1.0], size=n_bumps)
    hfield = np.zeros(len(u))
    for c, s in zip(centers, signs):
        hfield += s * np.exp(-np.sum((u - c) ** 2, axis=1) / (2 * 0.3 ** 2))
    hfield /= np.max(np.abs(hfield))
    xyz = u * (1.0 + amp * hfield)[:, None]
    return _pack(xyz, np.array(quads, dtype=np.int32), np.array(l0, dtype=np.int32), 3,
                 "cube_sphere_pre%d_L%d" % (pre, levels))


# ----------------------------------------------------------------------------
# coefficient fields (data evaluated at physical points)
# ----------------------------------------------------------------------------

def kappa_sines(x):
    """kappa(x, y) = 1 + 0.5 sin(pi x) sin(pi y)."""
    x = np.asarray(x)
    return 1.0 + 0.5 * np.sin(np.pi * x[..., 0]) * np.sin(np.pi * x[..., 1])


class LogNormalField:
    """kappa = exp(0.5 g), g = (1/16) sum_{k in [0,16)^2} a_k cos(2 pi k.xh) + b_k sin(2 pi k.xh),
    with a, b ~ N(0, 1) and xh the bounding-box-normalised point (Var g = 1)."""

    def __init__(self, seed, lo, hi, nk=16, sigma=0.5):
        rng = np.random.Generator(np.random.PCG64(seed))
        self.a = rng.normal(size=(nk, nk))
        self.b = rng.normal(size=(nk, nk))
        self.lo = np.asarray(lo, dtype=np.float64)[:2]
        self.hi = np.asarray(hi, dtype=np.float64)[:2]
        self.nk = nk
        self.sigma = sigma

    def __call__(self, x):
        x = np.asarray(x, dtype=np.float64)
        xh = (x[..., :2] - self.lo) / (self.hi - self.lo)
        k = np.arange(self.nk)
        ph = 2 * np.pi * (xh[..., 0, None, None] * k[:, None] + xh[..., 1, None, None] * k[None, :])
        g = (np.sum(self.a * np.cos(ph), axis=(-2, -1)) + np.sum(self.b * np.sin(ph), axis=(-2, -1))) / self.nk
        return np.exp(self.sigma * g)


def gaussian_bumps(seed, lo, hi, n=8, amp=0.5, width=0.1):
    """u0(x) = sum_m amp * exp(-|x - c_m|^2 / (2 (width * diam)^2)), c_m uniform in the bbox."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lo = np.asarray(lo, dtype=np.float64)[:2]
    hi = np.asarray(hi, dtype=np.float64)[:2]
    c = lo + rng.uniform(size=(n, 2)) * (hi - lo)
    s = width * float(np.linalg.norm(hi - lo))

    def f(x):
        x = np.asarray(x, dtype=np.float64)[..., :2]
        d2 = np.sum((x[..., None, :] - c) ** 2, axis=-1)
        return amp * np.sum(np.exp(-d2 / (2 * s * s)), axis=-1)
    return f


def instance_specs(seed, count, e_min=500, e_max=50000):
    """The drawn parameters of ``instances`` (all random draws happen here, in order):
    a list of ("rotated", nx, ny, n_ep, levels, sub) or ("disk", mu, n, levels, sub)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for k in range(count):
        target = float(np.exp(rng.uniform(np.log(e_min), np.log(e_max))))
        sub = int(rng.integers(1 << 30))
        if rng.uniform() < 0.6:
            nx, ny = int(rng.integers(4, 11)), int(rng.integers(4, 11))
            interior = (nx - 1) * (ny - 1)
            n_ep = int(min(20, max(2, 2 * int(rng.integers(1, max(2, interior // 3) + 1)))))
            n_ep = min(n_ep, 2 * (interior // 3)) if interior >= 6 else 0
            levels = int(np.clip(np.round(np.log(target / (nx * ny)) / np.log(4.0)), 0, 6))
            out.append(("rotated", nx, ny, n_ep, levels, sub))
        else:
            mu = int(rng.integers(3, 9))
            n = int(rng.integers(3, 7))
            levels = int(np.clip(np.round(np.log(target / (mu * n * n)) / np.log(4.0)), 0, 6))
            out.append(("disk", mu, n, levels, sub))
    return out


def make_instance(spec):
    """The mesh of one entry of ``instance_specs`` (no random draws beyond its seed)."""
    if spec[0] == "disk":
        _, mu, n, levels, sub = spec
        return disk(mu=mu, n=n, seed=sub, levels=levels)
    _, nx, ny, n_ep, levels, sub = spec
    mesh = None
    while mesh is None and n_ep >= 2:
        try:
            mesh = rotated(nx=nx, ny=ny, n_ep=n_ep, levels=levels, seed=sub, max_tries=40)
        except RuntimeError:
            n_ep -= 2                       # fewer EPs when none can be drawn
    return mesh if mesh is not None else grid(nx, ny, seed=sub, jitter=0.02, levels=levels)


def instances(seed, count, e_min=500, e_max=50000, workers=1):
    """Independent planar instances of uneven size for batched assembly.

    Element counts are drawn log-uniform in [e_min, e_max].  Each instance is
    either a rotated-core mesh (nx, ny in 4..10, an even number of EPs of valence
    3/5/6 up to 20) or a disk around one EP of valence 3..8, refined until its
    size is nearest to the drawn count.  Returns a list of mesh dicts.  workers > 1
    builds the meshes in that many spawned processes (the same meshes).
    """
    specs = instance_specs(seed, count, e_min, e_max)
    if workers <= 1:
        return [make_instance(sp) for sp in specs]
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(make_instance, specs))
