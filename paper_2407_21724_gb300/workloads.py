"""Seeded synthetic metasurface workloads (inputs only, no solver arithmetic).

Both the CUDA path and the FP64 oracle take their scenes from here.  The
module draws lattices, radii and incidences and builds particle meshes
(geometry only); it computes nothing of the MLFMA-SMR method itself.

All lengths are in vacuum wavelengths.  The particles are dielectric
(eps_r = 4, mu_r = 1) in vacuum on a square lattice of pitch 0.5 (or off it:
a jittered lattice, a golden-angle spiral), either
spheres (closed-form static modes) or nanopillars: circular cylinders of
height 0.6 given as closed 600-triangle meshes, whose static modes the
solver computes (N_perp transverse and N_par longitudinal per shape).  Radii
are quantised to 8 values in [0.08, 0.20].  The paper's gold spheres, bricks
and TiO2 nanofins need permittivity tables and meshers that are not
available here; these lattices stand in for them with the same particle
counts, the same 8-shape structure and the same unknown counts.
"""
import numpy as np

PITCH = 0.5
EPS_IN = 4.0
RADII8 = np.linspace(0.08, 0.20, 8)
PILLAR_HEIGHT = 0.6


def pillar(radius, modes, height=PILLAR_HEIGHT):
    """A nanopillar shape: the 600-triangle cylinder mesh of ``cylinder_mesh``
    with `modes` transverse and `modes` longitudinal static modes."""
    V, T = cylinder_mesh(radius, height)
    return dict(kind='mesh', verts=V, tris=T, n_perp=modes, n_par=modes, radius=float(radius),
                height=height, label=f'cylinder r={radius:.4f} h={height}, {len(T)} triangles')


def shapes8(kind, modes):
    """The 8 radii of RADII8 as spheres (radius, n_perp, n_par) or pillars."""
    if kind == 'pillar':
        return [pillar(r, modes) for r in RADII8]
    return [(r, modes, modes) for r in RADII8]


def lattice(nx, ny, pitch=PITCH):
    """Centred nx x ny lattice, row-major (x fastest); (p, 3) array."""
    xs = (np.arange(nx) - (nx - 1) / 2.0) * pitch
    ys = (np.arange(ny) - (ny - 1) / 2.0) * pitch
    X, Y = np.meshgrid(xs, ys, indexing='xy')
    return np.stack([X.ravel(), Y.ravel(), np.zeros(nx * ny)], axis=1)


def incidence(theta_deg=0.0, phi_deg=0.0, pol='x'):
    """Plane wave direction khat and the unit projection of x_hat or y_hat
    onto the plane orthogonal to khat."""
    t, f = np.radians(theta_deg), np.radians(phi_deg)
    k = np.array([np.sin(t) * np.cos(f), np.sin(t) * np.sin(f), np.cos(t)])
    e = np.array([1.0, 0.0, 0.0]) if pol == 'x' else np.array([0.0, 1.0, 0.0])
    e = e - k * (k @ e)
    return k, (e / np.linalg.norm(e)).astype(complex)


def incidence_grid64():
    """64 incidences: theta in linspace(0, 40 deg, 8), phi in {0,90,180,270},
    x and y polarisations (duplicates at theta = 0 kept)."""
    out = []
    for t in np.linspace(0.0, 40.0, 8):
        for f in (0.0, 90.0, 180.0, 270.0):
            for pol in ('x', 'y'):
                out.append(incidence(t, f, pol))
    return out


def metalens_bins(centres, focal, n_bins=8):
    """Radius bin per site from the hyperbolic lens phase
    phi = 2 pi (f - sqrt(f^2 + x^2 + y^2)) mod 2 pi, bin = floor(n phi / 2 pi)."""
    x, y = centres[:, 0], centres[:, 1]
    ph = np.mod(2 * np.pi * (focal - np.sqrt(focal ** 2 + x ** 2 + y ** 2)), 2 * np.pi)
    return np.minimum((n_bins * ph / (2 * np.pi)).astype(int), n_bins - 1)


def make(name, **kw):
    """Workload dict: centres, shape_ids, shapes [(radius, n_perp, n_par)],
    eps_in, pitch, incidences [(khat, pol)], label."""
    if name == 'spheres8x8':
        # 8x8 identical spheres r = 0.15, 12 + 12 modes per current: 3,072 unknowns
        C = lattice(8, 8)
        return dict(label='8x8 spheres r=0.15, 24 modes/current, 3072 unknowns',
                    centres=C, shape_ids=np.zeros(64, dtype=np.int32),
                    shapes=[(0.15, 12, 12)], eps_in=EPS_IN, pitch=PITCH,
                    incidences=[incidence(0, 0, 'x')])
    shape = kw.get('shape', 'sphere')
    what = 'pillars (600-triangle cylinder meshes, h=0.6)' if shape == 'pillar' else 'spheres'
    if name == 'random':
        # n x n lattice, radius index uniform over 8 values from a seed
        n = kw.get('n', 40)
        seed = kw.get('seed', 21724)
        modes = kw.get('modes', 16)
        rng = np.random.default_rng(seed)
        ids = rng.integers(0, 8, size=n * n).astype(np.int32)
        inc = kw.get('incidences') or [incidence(0, 0, 'x')]
        return dict(label=f'{n}x{n} random-radius {what} (8 radii), {2*modes} modes/current, '
                          f'{n*n*4*modes} unknowns',
                    centres=lattice(n, n), shape_ids=ids,
                    shapes=shapes8(shape, modes), eps_in=EPS_IN,
                    pitch=PITCH, incidences=inc)
    if name == 'metalens':
        # n x n hyperbolic-phase lens, focal length f, radii quantised to 8 bins
        n = kw.get('n', 200)
        f = kw.get('focal', 50.0)
        modes = kw.get('modes', 16)
        C = lattice(n, n)
        ids = metalens_bins(C, f).astype(np.int32)
        return dict(label=f'{n}x{n} metalens of {what}, f={f}, {2*modes} modes/current, '
                          f'{n*n*4*modes} unknowns',
                    centres=C, shape_ids=ids,
                    shapes=shapes8(shape, modes), eps_in=EPS_IN,
                    pitch=PITCH, incidences=[incidence(0, 0, 'x')], focal=f)
    if name == 'sparse':
        # n x n random-radius lattice thinned to a seeded fraction of its
        # sites: the tree depth and the upper levels' box counts of a full
        # n x n array with few particles
        w = make('random', n=kw.get('n', 200), seed=kw.get('seed', 21727), modes=kw.get('modes', 16),
                 shape=shape)
        keep = np.random.default_rng(kw.get('seed', 21727) + 1).random(len(w['centres'])) < kw.get('fill', 0.02)
        w['centres'], w['shape_ids'] = w['centres'][keep], w['shape_ids'][keep]
        w['label'] = f"{w['label']} thinned to {int(keep.sum())} sites"
        return w
    if name == 'jittered':
        # n x n random-radius lattice, each centre moved by a seeded uniform
        # in-plane displacement of at most `jitter` wavelengths per axis
        w = make('random', n=kw.get('n', 40), seed=kw.get('seed', 21728), modes=kw.get('modes', 16),
                 shape=shape)
        j = kw.get('jitter', 0.02)
        rng = np.random.default_rng(kw.get('seed', 21728) + 1)
        C = w['centres'].copy()
        C[:, :2] += rng.uniform(-j, j, size=(len(C), 2))
        w['centres'] = C
        w['label'] = f"{w['label']}, centres jittered by up to {j} per axis"
        return w
    if name == 'spiral':
        # golden-angle spiral of n particles, i = 1 .. n at r_i = c sqrt(i) and
        # angle i * 2 pi / phi^2 (the validation geometry of Sec. V), with c
        # set so that the closest two centres are `d_min` apart (sparser than
        # the paper's c = sqrt(3) R); radii from the three smallest of the 8
        # values, drawn from a seed.  With the pitch below d_min / sqrt(2)
        # every lattice cell holds at most one centre.
        n = kw.get('n', 400)
        d_min = kw.get('d_min', 0.75)
        modes = kw.get('modes', 16)
        i = np.arange(1, n + 1, dtype=float)
        ga = 2 * np.pi / ((1 + np.sqrt(5)) / 2) ** 2
        P = np.stack([np.sqrt(i) * np.cos(i * ga), np.sqrt(i) * np.sin(i * ga)], axis=1)
        d2 = np.sum((P[:, None, :] - P[None, :, :]) ** 2, axis=2) if n <= 4000 else None
        if d2 is None:
            raise ValueError('spiral: n <= 4000')
        np.fill_diagonal(d2, np.inf)
        P *= d_min / np.sqrt(d2.min())
        C = np.zeros((n, 3))
        C[:, :2] = P
        ids = np.random.default_rng(kw.get('seed', 21729)).integers(0, 3, size=n).astype(np.int32)
        inc = kw.get('incidences') or [incidence(0, 0, 'x')]
        return dict(label=f'golden-angle spiral of {n} {what} (3 radii), closest centres {d_min} apart, '
                          f'{2*modes} modes/current, {n*4*modes} unknowns',
                    centres=C, shape_ids=ids, shapes=shapes8(shape, modes)[:3], eps_in=EPS_IN,
                    pitch=PITCH, incidences=inc)
    if name == 'spiral_dense':
        # the paper's spiral spacing, c = sqrt(3) R, for n identical spheres
        # of radius R: neighbours about 1.4 diameters apart, so a lattice cell
        # of 0.5 wavelengths holds up to three centres
        n = kw.get('n', 2000)
        R = kw.get('R', 0.1)
        modes = kw.get('modes', 16)
        i = np.arange(1, n + 1, dtype=float)
        ga = 2 * np.pi / ((1 + np.sqrt(5)) / 2) ** 2
        c = np.sqrt(3.0) * R
        C = np.zeros((n, 3))
        C[:, 0], C[:, 1] = c * np.sqrt(i) * np.cos(i * ga), c * np.sqrt(i) * np.sin(i * ga)
        inc = kw.get('incidences') or [incidence(0, 0, 'x')]
        return dict(label=f'golden-angle spiral of {n} spheres R={R}, c = sqrt(3) R, {2*modes} modes/current, '
                          f'{n*4*modes} unknowns',
                    centres=C, shape_ids=np.zeros(n, dtype=np.int32), shapes=[(R, modes, modes)],
                    eps_in=EPS_IN, pitch=PITCH, incidences=inc)
    if name == 'spiral_bricks':
        # the paper's largest spiral (Sec. V): n bricks on the golden-angle
        # spiral with c = sqrt(3) R, R = 1/6 wavelength (100 nm at 600 nm; 115
        # wavelengths across at n = 40,000), brick i turned about z by
        # 2 pi (i - 1) / n, rounded to one of `bins` angles (rotated copies of
        # one box mesh).  The paper's 200 x 200 x 100 nm superellipsoid bricks
        # are stood in for by 0.3 x 0.3 x 0.15 wavelength boxes, whose corners
        # stay clear of the closest neighbours; cells of 0.9 wavelengths keep
        # every brick within a cell size of its cell centre, L0 = 16.
        n = kw.get('n', 40000)
        bins = kw.get('bins', 64)
        modes = kw.get('modes', 10)
        R = 1.0 / 6.0
        i = np.arange(1, n + 1, dtype=float)
        ga = 2 * np.pi / ((1 + np.sqrt(5)) / 2) ** 2
        c = np.sqrt(3.0) * R
        C = np.zeros((n, 3))
        C[:, 0], C[:, 1] = c * np.sqrt(i) * np.cos(i * ga), c * np.sqrt(i) * np.sin(i * ga)
        theta = 2 * np.pi * (i - 1) / n
        ids = (np.rint(theta / (2 * np.pi / bins)).astype(np.int64) % bins).astype(np.int32)
        V, T = box_mesh(0.3, 0.3, 0.15, 4, 4, 2)
        shapes = [dict(kind='mesh', verts=V, tris=T, n_perp=modes, n_par=modes,
                       label=f'brick 0.3 x 0.3 x 0.15, {len(T)} triangles')]
        shapes += [dict(kind='rotated', base=0, angle=b * 2 * np.pi / bins) for b in range(1, bins)]
        return dict(label=f'golden-angle spiral of {n} bricks (c = sqrt(3) R, R = 1/6), each turned by '
                          f'2 pi (i-1)/n in {bins} steps, {2*modes} modes/current, {n*4*modes} unknowns',
                    centres=C, shape_ids=ids, shapes=shapes, eps_in=EPS_IN, pitch=0.9, L0=16,
                    incidences=kw.get('incidences') or [incidence(0, 0, 'x')])
    if name == 'moire':
        # two-layer Moire superlattice (the 2.5D example of Sec. V): the
        # vertices of a honeycomb of side `side` (m x m unit cells, two
        # vertices each) at z = -h/2, and the same honeycomb turned by
        # `twist` degrees about z at z = +h/2; nanodisks of radius `radius`
        # and height radius / 2 (cylinder meshes), or spheres.  Lengths in
        # wavelengths from the paper's 400 / 300 / 100 nm at 600 nm.  Cells of
        # 0.85 wavelengths keep every disk within a cell size of its cell
        # centre; L0 = 16 for those cells.
        m = kw.get('m', 16)
        side = kw.get('side', 400 / 600)
        h = kw.get('h', 300 / 600)
        R = kw.get('radius', 100 / 600)
        twist = np.radians(kw.get('twist', 5.0))
        modes = kw.get('modes', 10)
        a1 = np.array([np.sqrt(3) * side, 0.0])
        a2 = np.array([np.sqrt(3) * side / 2, 1.5 * side])
        g = np.arange(m) - (m - 1) / 2.0
        I, J = np.meshgrid(g, g, indexing='xy')
        base = I.ravel()[:, None] * a1 + J.ravel()[:, None] * a2
        layer = np.vstack([base, base + [0.0, side]])
        layer -= layer.mean(axis=0)
        rot = np.array([[np.cos(twist), -np.sin(twist)], [np.sin(twist), np.cos(twist)]])
        C = np.zeros((2 * len(layer), 3))
        C[:len(layer), :2], C[:len(layer), 2] = layer, -h / 2
        C[len(layer):, :2], C[len(layer):, 2] = layer @ rot.T, h / 2
        if kw.get('shape', 'disk') == 'sphere':
            shapes = [(R, modes, modes)]
        else:
            V, T = cylinder_mesh(R, R / 2, n_phi=16, n_z=1, n_r=2)
            shapes = [dict(kind='mesh', verts=V, tris=T, n_perp=modes, n_par=modes,
                           label=f'disk r={R:.4f} h={R / 2:.4f}, {len(T)} triangles')]
        n = len(C)
        return dict(label=f'two-layer Moire lattice of {n} {"spheres" if kw.get("shape") == "sphere" else "nanodisks"} '
                          f'(honeycomb side {side:.3f}, layers {h} apart, twist {np.degrees(twist):.1f} deg), '
                          f'{2*modes} modes/current, {n*4*modes} unknowns',
                    centres=C, shape_ids=np.zeros(n, dtype=np.int32), shapes=shapes, eps_in=EPS_IN,
                    pitch=kw.get('pitch', 0.85), L0=kw.get('L0', 16),
                    incidences=kw.get('incidences') or [incidence(0, 0, 'x')])
    if name == 'pbfins':
        # n x n geometric-phase (PB) metalens of identical nanofins, each
        # turned about z by its pb_angles value rounded to one of `bins`
        # angles b pi / bins (the rotated copies of one meshed fin), focal
        # length for NA 0.8 over the aperture, circularly polarised incidence
        n = kw.get('n', 100)
        bins = kw.get('bins', 16)
        modes = kw.get('modes', 10)
        C = lattice(n, n)
        f = kw.get('focal', 0.75 * n * PITCH / 2)
        ids = (np.rint(pb_angles(C, f) / (np.pi / bins)).astype(np.int64) % bins).astype(np.int32)
        shapes = [nanofin(modes)] + [dict(kind='rotated', base=0, angle=b * np.pi / bins)
                                     for b in range(1, bins)]
        k = np.array([0.0, 0.0, 1.0])
        pol = np.array([1.0, 1.0j, 0.0]) / np.sqrt(2.0)
        return dict(label=f'{n}x{n} geometric-phase metalens of nanofins {FIN} ({bins} rotations of one '
                          f'656-triangle box mesh), f={f}, {2*modes} modes/current, {n*n*4*modes} unknowns',
                    centres=C, shape_ids=ids, shapes=shapes, eps_in=EPS_IN, pitch=PITCH,
                    incidences=[(k, pol)], focal=f)
    if name == 'ragged16':
        # 16 arrays of n_i = round(10 + 50 i / 15) pillars per side, seeds 21726 + i
        return [make('random', n=int(round(10 + 50 * i / 15)), seed=21726 + i,
                     modes=kw.get('modes', 16), shape=shape) for i in range(16)]
    raise KeyError(name)


def _orient_outward(V, T):
    """Order each triangle's vertices so that its normal points away from the
    origin (the meshes below are star-shaped about it)."""
    T = T.copy()
    p0, p1, p2 = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    n = np.cross(p1 - p0, p2 - p0)
    flip = np.sum(n * (p0 + p1 + p2), axis=1) < 0
    T[flip, 1], T[flip, 2] = T[flip, 2].copy(), T[flip, 1].copy()
    return T


def icosphere(radius, level):
    """Closed triangle mesh of a sphere: the icosahedron with every triangle
    split into four `level` times, vertices pushed onto the sphere.  Returns
    (verts (nv,3) float64, tris (nt,3) int32), nt = 20 * 4**level, outward
    vertex order."""
    g = (1.0 + np.sqrt(5.0)) / 2.0
    V = [(-1, g, 0), (1, g, 0), (-1, -g, 0), (1, -g, 0), (0, -1, g), (0, 1, g),
         (0, -1, -g), (0, 1, -g), (g, 0, -1), (g, 0, 1), (-g, 0, -1), (-g, 0, 1)]
    T = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
         (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
         (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    V = [np.array(v, dtype=float) / np.linalg.norm(v) for v in V]
    for _ in range(level):
        mid = {}

        def m(a, b):
            key = (min(a, b), max(a, b))
            if key not in mid:
                v = V[a] + V[b]
                V.append(v / np.linalg.norm(v))
                mid[key] = len(V) - 1
            return mid[key]
        T = [t for (a, b, c) in T for t in
             ((a, m(a, b), m(c, a)), (b, m(b, c), m(a, b)), (c, m(c, a), m(b, c)),
              (m(a, b), m(b, c), m(c, a)))]
    V = radius * np.array(V)
    return V, _orient_outward(V, np.array(T, dtype=np.int32))


def cylinder_mesh(radius, height, n_phi=20, n_z=10, n_r=3):
    """Closed triangle mesh of a circular cylinder (a nanopillar) centred at
    the origin, axis z: n_z rows of n_phi quads (two triangles each) on the
    side, and on each cap a centre fan inside n_r - 1 rings.  600 triangles,
    302 vertices and 900 edges at the defaults.  Returns (verts, tris) with
    outward vertex order."""
    ang = 2.0 * np.pi * np.arange(n_phi) / n_phi
    ring = np.stack([np.cos(ang), np.sin(ang)], axis=1)
    V, T = [], []

    def add_ring(r, z):
        base = len(V)
        V.extend(np.column_stack([r * ring, np.full(n_phi, z)]))
        return base

    side = [add_ring(radius, -height / 2 + height * k / n_z) for k in range(n_z + 1)]
    for k in range(n_z):
        a, b = side[k], side[k + 1]
        for j in range(n_phi):
            j1 = (j + 1) % n_phi
            T += [(a + j, a + j1, b + j1), (a + j, b + j1, b + j)]
    for z, outer in ((height / 2, side[-1]), (-height / 2, side[0])):
        rings = [add_ring(radius * i / n_r, z) for i in range(1, n_r)] + [outer]
        centre = len(V)
        V.append(np.array([0.0, 0.0, z]))
        for j in range(n_phi):
            T.append((centre, rings[0] + j, rings[0] + (j + 1) % n_phi))
        for i in range(n_r - 1):
            a, b = rings[i], rings[i + 1]
            for j in range(n_phi):
                j1 = (j + 1) % n_phi
                T += [(a + j, b + j, b + j1), (a + j, b + j1, a + j1)]
    V = np.array(V, dtype=float)
    return V, _orient_outward(V, np.array(T, dtype=np.int32))


def box_mesh(lx, ly, lz, nx, ny, nz):
    """Closed triangle mesh of a rectangular box (a brick or nanofin) of sides
    lx, ly, lz centred at the origin: each face an (n x n) grid of quads, two
    triangles each, 4 (nx ny + ny nz + nx nz) triangles.  Returns (verts,
    tris) with outward vertex order."""
    ids, V, T = {}, [], []
    n = (nx, ny, nz)
    L = np.array([lx, ly, lz], dtype=float)

    def vid(g):
        if g not in ids:
            ids[g] = len(V)
            V.append((np.array(g, dtype=float) / n - 0.5) * L)
        return ids[g]
    for ax in range(3):
        u, v = (ax + 1) % 3, (ax + 2) % 3
        for side in (0, n[ax]):
            for i in range(n[u]):
                for j in range(n[v]):
                    q = []
                    for di, dj in ((0, 0), (1, 0), (1, 1), (0, 1)):
                        g = [0, 0, 0]
                        g[ax], g[u], g[v] = side, i + di, j + dj
                        q.append(vid(tuple(g)))
                    T += [(q[0], q[1], q[2]), (q[0], q[2], q[3])]
    V = np.array(V, dtype=float)
    return V, _orient_outward(V, np.array(T, dtype=np.int32))


FIN = (0.31, 0.064, 0.45)        # nanofin sides (x, y, z) in wavelengths


def nanofin(modes):
    """A nanofin shape: the 656-triangle box mesh of FIN with `modes`
    transverse and `modes` longitudinal static modes."""
    V, T = box_mesh(*FIN, 10, 2, 12)
    return dict(kind='mesh', verts=V, tris=T, n_perp=modes, n_par=modes,
                label=f'nanofin {FIN[0]} x {FIN[1]} x {FIN[2]}, {len(T)} triangles')


def pb_angles(centres, focal):
    """Geometric-phase lens rotation of each fin: theta = pi (f - sqrt(f^2 +
    x^2 + y^2)) (wavelength 1), taken modulo pi (a fin turned by pi is the
    same fin)."""
    r2 = centres[:, 0] ** 2 + centres[:, 1] ** 2
    return np.mod(np.pi * (focal - np.sqrt(focal ** 2 + r2)), np.pi)


def mlp_params(dims, seed):
    """Seeded MLP parameters (layer by layer, W [in][out] then b) whose values
    are exactly representable in bfloat16 (the top 16 bits of a float32)."""
    rng = np.random.default_rng(seed)
    parts = []
    for l in range(4):
        a = np.sqrt(6.0 / (dims[l] + dims[l + 1]))
        parts.append(rng.uniform(-a, a, size=dims[l] * dims[l + 1]))
        parts.append(rng.uniform(-0.1, 0.1, size=dims[l + 1]))
    p = np.concatenate(parts).astype(np.float32)
    return (p.view(np.uint32) & np.uint32(0xFFFF0000)).view(np.float32)


def training_arrays(count, n=20, seed0=100000, modes=16, shape='sphere'):
    """Random n x n arrays for the learned initial guess: radius index
    U{0..7} and one incidence per array (theta ~ U[0, 40 deg), phi ~ U[0,
    360 deg), x or y polarisation), array i drawn from seed seed0 + i."""
    out = []
    shapes = shapes8(shape, modes)
    for i in range(count):
        rng = np.random.default_rng(seed0 + i)
        ids = rng.integers(0, 8, size=n * n).astype(np.int32)
        th, ph = rng.uniform(0.0, 40.0), rng.uniform(0.0, 360.0)
        pol = 'x' if rng.integers(0, 2) == 0 else 'y'
        out.append(dict(label=f'{n}x{n} training array {seed0 + i}', centres=lattice(n, n),
                        shape_ids=ids, shapes=shapes,
                        eps_in=EPS_IN, pitch=PITCH, incidences=[incidence(th, ph, pol)]))
    return out
