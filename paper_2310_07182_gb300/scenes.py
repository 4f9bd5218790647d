"""Seeded synthetic scenes and cameras: the input generators shared by the CUDA path's
tests/bench and by the CPU oracle's tests.

This module holds input *data* only (triangle soups, terrain, rooms, material tables,
camera placements).  It contains none of the path tracer's arithmetic: no ray
generation, no intersection, no sampling, no grouping.  Every generator draws from
``numpy.random.default_rng(seed)`` so the same seed gives the same arrays on any host.

The paper's scenes (Breakfast, Salle de Bain, Living room, Sibenik, Vokselia; Sec. 5)
are not available, so these stand in for them at their scale:

* ``landscape``: a 2.1M-triangle fBm heightfield, standing in for the Vokselia landscape
  (1.876M triangles).
* ``interior``: a closed room with 2,000 UV spheres (0.51M triangles), standing in for
  the dense indoor scenes (0.58M-1.35M triangles).
* ``tiny``: 1,024 random triangles over a ground plane, small enough for brute force.

Material types follow the paper's classes (Sec. 3.2): diffuse (Lambert), glossy (GGX)
and specular (mirror), plus area emitters for the interior light.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Material type codes (same numbering as ``cr_mat_type`` in include/cr.h).
MAT_LAMBERT = 0
MAT_GGX = 1
MAT_MIRROR = 2
MAT_EMITTER = 3
MAT_DIELECTRIC = 4   # smooth dielectric; the roughness slot holds the index of refraction
MAT_TRANSLUCENT = 5  # Lambertian transmission


@dataclass
class Camera:
    pos: tuple
    look_at: tuple
    up: tuple
    vfov_deg: float
    width: int
    height: int


@dataclass
class Scene:
    """Triangle soup with a per-triangle material index.

    tri_xyz:  float32 [n_tri, 9] (v0.xyz, v1.xyz, v2.xyz)
    tri_mat:  uint32  [n_tri]
    mat_type: uint32  [n_mat]   MAT_* codes
    mat_params: float32 [n_mat, 7]  albedo rgb, roughness (GGX alpha), emission rgb
    env:      float32 [3] constant environment radiance
    """
    name: str
    tri_xyz: np.ndarray
    tri_mat: np.ndarray
    mat_type: np.ndarray
    mat_params: np.ndarray
    env: np.ndarray
    camera: Camera | None = None
    meta: dict = field(default_factory=dict)

    @property
    def n_tri(self) -> int:
        return int(self.tri_xyz.shape[0])

    @property
    def n_mat(self) -> int:
        return int(self.mat_type.shape[0])


def _finish(name, tris, tri_mat, mat_type, mat_params, env, camera, **meta) -> Scene:
    return Scene(
        name=name,
        tri_xyz=np.ascontiguousarray(tris, dtype=np.float32).reshape(-1, 9),
        tri_mat=np.ascontiguousarray(tri_mat, dtype=np.uint32),
        mat_type=np.ascontiguousarray(mat_type, dtype=np.uint32),
        mat_params=np.ascontiguousarray(mat_params, dtype=np.float32).reshape(-1, 7),
        env=np.ascontiguousarray(env, dtype=np.float32).reshape(3),
        camera=camera,
        meta=dict(meta),
    )


def _ball_offsets(rng, n, radius):
    """n points uniform in a ball of the given radius (rejection-free: direction x r^(1/3))."""
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    r = radius * rng.random(n) ** (1.0 / 3.0)
    return v * r[:, None]


def ground_quad(y=-1.0, half=5.0):
    """Two triangles covering x,z in [-half, half] at height y."""
    a = (-half, y, -half)
    b = (half, y, -half)
    c = (half, y, half)
    d = (-half, y, half)
    return np.array([a + b + c, a + c + d], dtype=np.float64)


def soup_triangles(rng, n, centre_half=0.9, radius=0.1):
    """n random triangles: centroid uniform in [-centre_half, centre_half]^3, each vertex
    within ``radius`` of it, so every edge is at most 2*radius long."""
    c = rng.uniform(-centre_half, centre_half, size=(n, 3))
    v = np.stack([c + _ball_offsets(rng, n, radius) for _ in range(3)], axis=1)
    return v.reshape(n, 9)


def tiny(seed: int = 1, n_soup: int = 1024, width: int = 64, height: int = 64,
         material_mix: str = "lambert") -> Scene:
    """Tiny plain-method scene: random soup over a 2-triangle ground plane at y=-1,
    one Lambert material per triangle with albedo uniform in [0.2, 0.8] per channel,
    uniform white environment; camera at (0,0,-3) looking +z, 60 deg vertical FOV."""
    rng = np.random.default_rng(seed)
    tris = np.concatenate([soup_triangles(rng, n_soup), ground_quad()], axis=0)
    n = tris.shape[0]
    albedo = rng.uniform(0.2, 0.8, size=(n, 3))
    if material_mix == "lambert":
        mtype = np.full(n, MAT_LAMBERT, dtype=np.uint32)
    elif material_mix == "mixed":  # 60/30/10 Lambert/GGX/mirror, random per triangle
        u = rng.random(n)
        mtype = np.where(u < 0.6, MAT_LAMBERT, np.where(u < 0.9, MAT_GGX, MAT_MIRROR)).astype(np.uint32)
    elif material_mix == "glossy":  # GGX and mirror only
        u = rng.random(n)
        mtype = np.where(u < 0.75, MAT_GGX, MAT_MIRROR).astype(np.uint32)
    elif material_mix == "transmissive":  # 35/25/15/10/15 Lambert/translucent/GGX/mirror/dielectric
        u = rng.random(n)
        mtype = np.select([u < 0.35, u < 0.6, u < 0.75, u < 0.85], [MAT_LAMBERT, MAT_TRANSLUCENT, MAT_GGX, MAT_MIRROR],
                          MAT_DIELECTRIC).astype(np.uint32)
    else:
        raise ValueError(material_mix)
    rough = rng.uniform(0.05, 0.5, size=n)
    if material_mix == "transmissive":
        rough = np.where(mtype == MAT_DIELECTRIC, rng.uniform(1.3, 1.7, size=n), rough)
    params = np.zeros((n, 7))
    params[:, 0:3] = albedo
    params[:, 3] = rough
    cam = Camera((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 60.0, width, height)
    return _finish(f"tiny-{material_mix}", tris, np.arange(n), mtype, params, (1.0, 1.0, 1.0), cam,
                   seed=seed)


def soup(seed: int, n_tri: int, width: int = 512, height: int = 512) -> Scene:
    """Random-triangle soup of ``n_tri`` triangles (tiny generator at scale) over the
    ground plane, materials 60/30/10 Lambert/GGX/mirror from a palette."""
    rng = np.random.default_rng(seed)
    tris = np.concatenate([soup_triangles(rng, n_tri), ground_quad()], axis=0)
    mtype, params, tri_mat = _palette_assign(rng, tris.shape[0], rng.random(tris.shape[0]))
    cam = Camera((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 60.0, width, height)
    return _finish(f"soup{n_tri}", tris, tri_mat, mtype, params, (1.0, 1.0, 1.0), cam, seed=seed)


# ---------------------------------------------------------------------------------------
# Palette materials: a fixed table per class, each triangle picks one entry at random.
# Per-triangle albedo tables would cost 32 B/triangle of device memory for the 2M-10M
# triangle scenes; a 576-entry palette keeps the same value distributions.
N_PAL_LAMBERT, N_PAL_GGX, N_PAL_MIRROR = 256, 256, 64


def _palette(rng):
    n = N_PAL_LAMBERT + N_PAL_GGX + N_PAL_MIRROR
    mtype = np.empty(n, dtype=np.uint32)
    mtype[:N_PAL_LAMBERT] = MAT_LAMBERT
    mtype[N_PAL_LAMBERT:N_PAL_LAMBERT + N_PAL_GGX] = MAT_GGX
    mtype[N_PAL_LAMBERT + N_PAL_GGX:] = MAT_MIRROR
    params = np.zeros((n, 7))
    params[:, 0:3] = rng.uniform(0.2, 0.8, size=(n, 3))
    params[:, 3] = rng.uniform(0.05, 0.5, size=n)
    return mtype, params


def _palette_assign(rng, n_tri, u):
    """Class by thresholding ``u`` at its 60th/90th percentiles (60/30/10 split), then a
    random palette entry of that class."""
    mtype, params = _palette(rng)
    p60, p90 = np.quantile(u, [0.6, 0.9])
    cls = np.where(u < p60, 0, np.where(u < p90, 1, 2))
    base = np.array([0, N_PAL_LAMBERT, N_PAL_LAMBERT + N_PAL_GGX])
    size = np.array([N_PAL_LAMBERT, N_PAL_GGX, N_PAL_MIRROR])
    tri_mat = base[cls] + rng.integers(0, 1 << 30, size=n_tri) % size[cls]
    return mtype, params, tri_mat


# ---------------------------------------------------------------------------------------
# Value-noise fBm for the terrain (input data only).
def _value_noise(rng_table, x, z):
    xi = np.floor(x).astype(np.int64)
    zi = np.floor(z).astype(np.int64)
    fx = x - xi
    fz = z - zi
    ux = fx * fx * fx * (fx * (fx * 6.0 - 15.0) + 10.0)  # quintic fade
    uz = fz * fz * fz * (fz * (fz * 6.0 - 15.0) + 10.0)
    s = rng_table.shape[0]
    v00 = rng_table[xi % s, zi % s]
    v10 = rng_table[(xi + 1) % s, zi % s]
    v01 = rng_table[xi % s, (zi + 1) % s]
    v11 = rng_table[(xi + 1) % s, (zi + 1) % s]
    a = v00 + (v10 - v00) * ux
    b = v01 + (v11 - v01) * ux
    return (a + (b - a) * uz) * 2.0 - 1.0


def fbm(seed, x, z, octaves, lacunarity=2.0, gain=0.5):
    rng = np.random.default_rng(seed)
    tables = [rng.random((256, 256)) for _ in range(octaves)]
    total = np.zeros_like(x, dtype=np.float64)
    amp, freq = 1.0, 1.0
    for o in range(octaves):
        total += amp * _value_noise(tables[o], x * freq + 17.0 * o, z * freq - 31.0 * o)
        amp *= gain
        freq *= lacunarity
    return total


def heightfield_triangles(n_grid, half=100.0, height=25.0, scale=40.0, seed=7):
    g = np.linspace(-half, half, n_grid)
    X, Z = np.meshgrid(g, g, indexing="ij")
    Y = height * fbm(seed, X / scale, Z / scale, octaves=6)
    V = np.stack([X, Y, Z], axis=-1)
    v00 = V[:-1, :-1].reshape(-1, 3)
    v10 = V[1:, :-1].reshape(-1, 3)
    v11 = V[1:, 1:].reshape(-1, 3)
    v01 = V[:-1, 1:].reshape(-1, 3)
    t1 = np.concatenate([v00, v10, v11], axis=1)
    t2 = np.concatenate([v00, v11, v01], axis=1)
    return np.stack([t1, t2], axis=1).reshape(-1, 9)


def landscape(seed: int = 7, n_grid: int = 1024, width: int = 1920, height: int = 1080,
              mat_seed: int = 8) -> Scene:
    """fBm heightfield terrain (6 octaves, lacunarity 2, gain 0.5) on an n_grid^2 vertex grid
    over x,z in [-100,100], y = 25 fbm(x/40, z/40); constant sky; per-triangle materials from
    a 3-octave noise thresholded to 60% Lambert / 30% GGX / 10% mirror.  1024^2 grid gives
    2,093,058 triangles; camera at (0,30,-95) looking at (0,5,0), 50 deg vertical FOV."""
    tris = heightfield_triangles(n_grid, seed=seed)
    cen = (tris[:, 0:3] + tris[:, 3:6] + tris[:, 6:9]) / 3.0
    u = fbm(mat_seed, cen[:, 0] / 25.0, cen[:, 2] / 25.0, octaves=3)
    rng = np.random.default_rng(seed + 1000)
    mtype, params, tri_mat = _palette_assign(rng, tris.shape[0], u)
    cam = Camera((0.0, 30.0, -95.0), (0.0, 5.0, 0.0), (0.0, 1.0, 0.0), 50.0, width, height)
    return _finish(f"landscape{n_grid}", tris, tri_mat, mtype, params, (1.0, 1.0, 1.0), cam,
                   seed=seed)


# ---------------------------------------------------------------------------------------
def uv_sphere(centre, radius, slices=16, stacks=9):
    """UV sphere: triangle fans at the poles, quads (2 triangles) between; 16x9 -> 256 tris."""
    cx, cy, cz = centre
    tris = []

    def P(i, j):
        th = math.pi * i / stacks
        ph = 2.0 * math.pi * j / slices
        return (cx + radius * math.sin(th) * math.cos(ph), cy + radius * math.cos(th),
                cz + radius * math.sin(th) * math.sin(ph))

    for i in range(stacks):
        for j in range(slices):
            a, b = P(i, j), P(i, j + 1)
            c, d = P(i + 1, j + 1), P(i + 1, j)
            if i == 0:
                tris.append(a + c + d)
            elif i == stacks - 1:
                tris.append(a + b + c)
            else:
                tris.append(a + b + c)
                tris.append(a + c + d)
    return np.array(tris, dtype=np.float64)


def _box_room(lo, hi):
    x0, y0, z0 = lo
    x1, y1, z1 = hi
    c = [(x0, y0, z0), (x1, y0, z0), (x1, y1, z0), (x0, y1, z0),
         (x0, y0, z1), (x1, y0, z1), (x1, y1, z1), (x0, y1, z1)]
    faces = [(0, 1, 2, 3), (5, 4, 7, 6), (4, 0, 3, 7), (1, 5, 6, 2), (4, 5, 1, 0), (3, 2, 6, 7)]
    tris = []
    for a, b, cc, d in faces:
        tris.append(c[a] + c[b] + c[cc])
        tris.append(c[a] + c[cc] + c[d])
    return np.array(tris, dtype=np.float64)


def interior(seed: int = 11, n_spheres: int = 2000, width: int = 1280, height: int = 720) -> Scene:
    """Closed room [-4,4]x[0,4]x[-4,4] (12 triangles, Lambert 0.7) with n_spheres UV spheres
    (256 triangles each, radius uniform in [0.05,0.3], centres uniform in the room inset by
    the radius, redrawn if closer than 0.25 to the camera), materials 60/30/10 per sphere,
    and a 1.5x1.5 ceiling light at y=3.999 (emission 20).  2000 spheres give 512,014 triangles; camera at (0,2,-3.8) looking +z."""
    rng = np.random.default_rng(seed)
    room = _box_room((-4.0, 0.0, -4.0), (4.0, 4.0, 4.0))
    mtype, params = _palette(rng)
    # extra materials: room wall and the emitter
    wall = len(mtype)
    light = wall + 1
    mtype = np.concatenate([mtype, [MAT_LAMBERT, MAT_EMITTER]]).astype(np.uint32)
    params = np.concatenate([params, [[0.7, 0.7, 0.7, 0.0, 0, 0, 0], [0, 0, 0, 0, 20.0, 20.0, 20.0]]])
    sph = []
    sph_mat = []
    u = rng.random(n_spheres)
    cls = np.where(u < 0.6, 0, np.where(u < 0.9, 1, 2))
    base = np.array([0, N_PAL_LAMBERT, N_PAL_LAMBERT + N_PAL_GGX])
    size = np.array([N_PAL_LAMBERT, N_PAL_GGX, N_PAL_MIRROR])
    cam_pos = np.array([0.0, 2.0, -3.8])
    for s in range(n_spheres):
        while True:  # keep a 0.25 clearance around the camera (redraw otherwise)
            r = rng.uniform(0.05, 0.3)
            c = (rng.uniform(-4 + r, 4 - r), rng.uniform(0 + r, 4 - r), rng.uniform(-4 + r, 4 - r))
            if np.linalg.norm(np.array(c) - cam_pos) > r + 0.25:
                break
        t = uv_sphere(c, r)
        sph.append(t)
        m = base[cls[s]] + rng.integers(0, size[cls[s]])
        sph_mat.append(np.full(t.shape[0], m))
    h = 0.75
    y = 3.999
    lq = np.array([(-h, y, -h) + (h, y, -h) + (h, y, h), (-h, y, -h) + (h, y, h) + (-h, y, h)])
    tris = np.concatenate([room] + sph + [lq], axis=0)
    tri_mat = np.concatenate([np.full(12, wall)] + sph_mat + [np.full(2, light)])
    cam = Camera((0.0, 2.0, -3.8), (0.0, 2.0, 0.0), (0.0, 1.0, 0.0), 60.0, width, height)
    return _finish(f"interior{n_spheres}", tris, tri_mat, mtype, params, (0.0, 0.0, 0.0), cam,
                   seed=seed)


def emitter_box(floor=MAT_LAMBERT, floor_params=(0.6, 0.5, 0.4, 0.3), le=(1.0, 1.0, 1.0), n_spheres=0,
                seed: int = 3, width: int = 32, height: int = 32) -> Scene:
    """Closed box [-1,1]^3 lit by its own walls: the floor (y = -1, triangles 8 and 9) has the
    material ``floor`` (params: albedo rgb, roughness) and the five other faces emit ``le``;
    the environment is black.  Without occluders every floor point sees emitters over its
    whole upper hemisphere (irradiance pi * le), so a Lambert floor's outgoing radiance is
    exactly albedo * le.  ``n_spheres`` UV spheres (radius 0.1-0.25; Lambert, GGX and mirror
    in turn) add occlusion and all three material classes."""
    rng = np.random.default_rng(seed)
    box = _box_room((-1.0, -1.0, -1.0), (1.0, 1.0, 1.0))
    mtype = [floor, MAT_EMITTER, MAT_LAMBERT, MAT_GGX, MAT_MIRROR]
    params = np.zeros((5, 7))
    params[0, 0:4] = floor_params
    params[1, 4:7] = le
    params[2, 0:3] = (0.5, 0.6, 0.7)
    params[3, 0:4] = (0.8, 0.7, 0.5, 0.25)
    params[4, 0:3] = (0.9, 0.9, 0.9)
    tri_mat = np.full(12, 1)
    tri_mat[8:10] = 0
    sph, sph_mat = [], []
    for s in range(n_spheres):
        r = rng.uniform(0.1, 0.25)
        c = (rng.uniform(-1 + r, 1 - r), rng.uniform(-1 + r, 0.2), rng.uniform(-0.3, 1 - r))
        t = uv_sphere(c, r)
        sph.append(t)
        sph_mat.append(np.full(t.shape[0], 2 + s % 3))
    tris = np.concatenate([box] + sph, axis=0)
    tri_mat = np.concatenate([tri_mat] + sph_mat)
    cam = Camera((0.0, 0.5, -0.95), (0.0, -1.0, 0.4), (0.0, 1.0, 0.0), 60.0, width, height)
    return _finish(f"emitter_box{n_spheres}", tris, tri_mat, np.array(mtype), params, (0.0, 0.0, 0.0), cam,
                   seed=seed)


def terrain(seed: int = 51, n_grid: int = 2236, width: int = 1024, height: int = 1024) -> Scene:
    """Large terrain: the landscape generator on a 2236^2 grid (9,990,450 triangles)."""
    return landscape(seed=seed, n_grid=n_grid, width=width, height=height, mat_seed=seed + 1)


# ---------------------------------------------------------------------------------------
# Closed-form and hand-built test scenes.
def icosphere(subdiv: int = 2, radius: float = 1.0):
    t = (1.0 + 5 ** 0.5) / 2.0
    verts = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t),
             (0, 1, -t), (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    verts = [np.array(v, dtype=np.float64) / np.linalg.norm(v) for v in verts]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
             (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
             (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(subdiv):
        cache = {}

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    V = np.array(verts) * radius
    return np.array([np.concatenate([V[a], V[b], V[c]]) for a, b, c in faces])


def furnace(albedo=(0.5, 0.5, 0.5), env=(1.0, 1.0, 1.0), subdiv=2, width=32, height=32) -> Scene:
    """White furnace: a convex Lambert icosphere of uniform albedo inside a uniform
    environment.  Any path sees radiance albedo*env (hit) or env (miss), exactly."""
    tris = icosphere(subdiv)
    n = tris.shape[0]
    params = np.zeros((1, 7))
    params[0, 0:3] = albedo
    cam = Camera((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 45.0, width, height)
    return _finish("furnace", tris, np.zeros(n), [MAT_LAMBERT], params, env, cam)


def mixed_furnace(width=32, height=32) -> Scene:
    """A convex icosphere whose triangles alternate Lambert (albedo 0.5, 0.25, 0.75) with GGX
    (roughness 0.3) and mirror, in a uniform unit environment: every exit direction above a
    point escapes, so a Lambert point is exactly albedo * env whichever direction it takes,
    while most reuse groups are hybrid."""
    tris = icosphere(2)
    n = tris.shape[0]
    params = np.zeros((3, 7))
    params[0, 0:3] = (0.5, 0.25, 0.75)
    params[1, 0:4] = (0.8, 0.7, 0.6, 0.3)
    params[2, 0:3] = (0.9, 0.9, 0.9)
    cam = Camera((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 45.0, width, height)
    mat = np.array([0 if i % 2 == 0 else (1 if i % 4 == 1 else 2) for i in range(n)])
    return _finish("mixed_furnace", tris, mat, [MAT_LAMBERT, MAT_GGX, MAT_MIRROR], params, (1.0, 1.0, 1.0), cam)


def split_plane(width=32, height=32, left=MAT_LAMBERT, right=MAT_GGX, n_strips=1) -> Scene:
    """A plane z=0 seen head-on (orthogonal to the view axis) whose left half (x>0 seen from
    the camera at z=-2) is material ``left`` and right half ``right``; used to predict group
    categories from pixel positions alone.  With n_strips>1 the plane is cut into vertical
    strips alternating the two materials."""
    tris = []
    mats = []
    edges = np.linspace(-4.0, 4.0, 2 * n_strips + 1)
    for s in range(2 * n_strips):
        x0, x1 = edges[s], edges[s + 1]
        a, b, c, d = (x0, -4.0, 0.0), (x1, -4.0, 0.0), (x1, 4.0, 0.0), (x0, 4.0, 0.0)
        tris += [a + b + c, a + c + d]
        mats += [s % 2, s % 2]
    params = np.zeros((2, 7))
    params[:, 0:3] = [[0.6, 0.5, 0.4], [0.7, 0.7, 0.7]]
    params[:, 3] = 0.2
    cam = Camera((0.0, 0.0, -2.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 60.0, width, height)
    return _finish("split_plane", np.array(tris), np.array(mats), [left, right], params,
                   (1.0, 1.0, 1.0), cam)


def random_rays(seed: int, n: int, origin_box=(-1.5, 1.5), target_box=(-1.0, 1.0)):
    """Seeded fp32 rays (n, 8): o.xyz, tmin(=0), d.xyz (unit, from a point in origin_box^3
    towards a point in target_box^3), tmax(=inf)."""
    rng = np.random.default_rng(seed)
    o = rng.uniform(*origin_box, size=(n, 3))
    tgt = rng.uniform(*target_box, size=(n, 3))
    d = tgt - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = np.zeros((n, 8), dtype=np.float32)
    r[:, 0:3] = o
    r[:, 4:7] = d
    r[:, 7] = np.inf
    return r


CONFIGS = {
    "tiny": dict(make=tiny, spp=1, max_bounces=1, tile=(4, 4), k=16),
    "landscape": dict(make=landscape, spp=1, max_bounces=2, tile=(8, 8), k=8),
    "interior": dict(make=interior, spp=16, max_bounces=4, tile=(8, 8), k=8),
}
