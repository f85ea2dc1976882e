"""Seeded synthetic scenes shaped like the workloads of MARS (Meyer et al. 2024).

The paper evaluates on indoor scenes lit by small emitters with mixed glossy and
diffuse materials (Sec. 4.2 and Sec. 5.2).  Those scenes are not available, so
the generators below produce stand-ins with the same character:

* ``box_scene``         -- the Cornell-like box (the paper's own failure case,
                           Fig. "failure"): five diffuse quads and one small
                           ceiling light.
* ``guided_room_scene`` -- a closed room with seeded random spheres (GGX and
                           Lambertian) and four small ceiling lights; used with
                           three techniques (BSDF, NEE, guided).
* ``furnace_scene``     -- a closed, uniformly emitting, uniformly diffuse box
                           whose pixel values have a closed form.
* ``area_light_plane_scene`` -- one diffuse plane under one rectangular light,
                           whose first-bounce irradiance has a closed form.

Every coordinate and material value is rounded to float32 so that a float32
and a float64 consumer see exactly the same geometry.

Array layouts (all float64 unless stated):

* ``quads``      [nq, 9]  corner p0, edge e1, edge e2; the (one-sided) emission
                          normal of a quad is normalize(e1 x e2).
* ``spheres``    [ns, 4]  centre, radius.
* ``tris``       [nt, 9]  v0, v1, v2.
* ``*_mat``      int32    material index per primitive.
* ``materials``  [nm, 8]  type (0 Lambert, 1 GGX), colour rgb (albedo or F0),
                          GGX roughness alpha, emitted radiance rgb.
* ``camera``     [10]     origin, look-at point, up vector, vertical FOV (deg).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

MAT_LAMBERT = 0
MAT_GGX = 1

TECH_BSDF = 1
TECH_NEE = 2
TECH_GUIDED = 4
TECH_LIGHT = 8   # connections to light subpaths (the bidirectional application)

GUIDE_BINS = 256  # 16 (cos theta) x 16 (phi) cylindrical bins per cell


def _f32(a) -> np.ndarray:
    return np.asarray(a, dtype=np.float32).astype(np.float64)


@dataclasses.dataclass
class Scene:
    quads: np.ndarray
    quad_mat: np.ndarray
    spheres: np.ndarray
    sphere_mat: np.ndarray
    tris: np.ndarray
    tri_mat: np.ndarray
    materials: np.ndarray
    camera: np.ndarray
    width: int
    height: int
    name: str = "scene"

    @property
    def n_pixels(self) -> int:
        return self.width * self.height

    def n_prims(self) -> int:
        return len(self.quads) + len(self.spheres) + len(self.tris)

    def with_resolution(self, width: int, height: int) -> "Scene":
        return dataclasses.replace(self, width=int(width), height=int(height))


@dataclasses.dataclass
class WorkloadConfig:
    """Run parameters of one workload (a scene plus the MARS settings)."""

    scene: Scene
    max_depth: int
    grid_n: int
    techniques: int
    iterations: int
    warmup: int
    name: str

    @property
    def n_cells(self) -> int:
        return self.grid_n ** 3


def _mk(quads, quad_mat, spheres, sphere_mat, materials, camera, w, h, name):
    quads = _f32(np.asarray(quads, dtype=np.float64).reshape(-1, 9))
    spheres = _f32(np.asarray(spheres, dtype=np.float64).reshape(-1, 4))
    return Scene(
        quads=quads,
        quad_mat=np.asarray(quad_mat, dtype=np.int32).reshape(-1),
        spheres=spheres,
        sphere_mat=np.asarray(sphere_mat, dtype=np.int32).reshape(-1),
        tris=np.zeros((0, 9), dtype=np.float64),
        tri_mat=np.zeros((0,), dtype=np.int32),
        materials=_f32(np.asarray(materials, dtype=np.float64).reshape(-1, 8)),
        camera=_f32(np.asarray(camera, dtype=np.float64).reshape(10)),
        width=int(w),
        height=int(h),
        name=name,
    )


def _lambert(r, g, b, le=(0.0, 0.0, 0.0)):
    return [MAT_LAMBERT, r, g, b, 0.0, le[0], le[1], le[2]]


def _ggx(r, g, b, alpha):
    return [MAT_GGX, r, g, b, alpha, 0.0, 0.0, 0.0]


def box_scene(width: int = 64, height: int = 64) -> Scene:
    """Unit-cube box open at z = 0, red wall at x = 0, green wall at x = 1,
    0.25 x 0.25 ceiling light of radiance 15 facing down, pinhole camera at
    (0.5, 0.5, -1.4) looking +z with a 40 degree vertical field of view."""
    mats = [
        _lambert(0.7, 0.7, 0.7),          # 0 grey
        _lambert(0.63, 0.06, 0.05),       # 1 red
        _lambert(0.14, 0.45, 0.09),       # 2 green
        _lambert(0.0, 0.0, 0.0, (15.0, 15.0, 15.0)),  # 3 light (black, emits)
    ]
    y_light = 1.0 - 1e-4
    quads = [
        # floor y = 0
        [0, 0, 0, 1, 0, 0, 0, 0, 1],
        # ceiling y = 1
        [0, 1, 0, 0, 0, 1, 1, 0, 0],
        # back wall z = 1
        [0, 0, 1, 0, 1, 0, 1, 0, 0],
        # left wall x = 0 (red)
        [0, 0, 0, 0, 0, 1, 0, 1, 0],
        # right wall x = 1 (green)
        [1, 0, 0, 0, 1, 0, 0, 0, 1],
        # light: e1 x e2 points down (-y)
        [0.375, y_light, 0.375, 0.25, 0, 0, 0, 0, 0.25],
    ]
    quad_mat = [0, 0, 0, 1, 2, 3]
    cam = [0.5, 0.5, -1.4, 0.5, 0.5, 0.0, 0.0, 1.0, 0.0, 40.0]
    return _mk(quads, quad_mat, [], [], mats, cam, width, height, "box")


def furnace_scene(albedo: float = 0.5, radiance: float = 1.0,
                  width: int = 16, height: int = 16) -> Scene:
    """Closed unit cube; every face is Lambertian with ``albedo`` and emits
    ``radiance`` towards the inside.  The camera sits at the centre.  Every
    pixel's expected value with at most D path segments is
    radiance * (1 - albedo**D) / (1 - albedo)."""
    mats = [_lambert(albedo, albedo, albedo, (radiance, radiance, radiance))]
    # each quad's e1 x e2 points into the cube
    quads = [
        [0, 0, 0, 0, 0, 1, 1, 0, 0],   # y = 0, normal +y
        [0, 1, 0, 1, 0, 0, 0, 0, 1],   # y = 1, normal -y
        [0, 0, 0, 1, 0, 0, 0, 1, 0],   # z = 0, normal +z
        [0, 0, 1, 0, 1, 0, 1, 0, 0],   # z = 1, normal -z
        [0, 0, 0, 0, 1, 0, 0, 0, 1],   # x = 0, normal +x
        [1, 0, 0, 0, 0, 1, 0, 1, 0],   # x = 1, normal -x
    ]
    cam = [0.5, 0.5, 0.5, 0.5, 0.5, 1.0, 0.0, 1.0, 0.0, 60.0]
    return _mk(quads, [0] * 6, [], [], mats, cam, width, height, "furnace")


def area_light_plane_scene(width: int = 4, height: int = 4,
                           light_y: float = 1.0, light_half: float = 0.5,
                           albedo: float = 0.5, radiance: float = 2.0) -> Scene:
    """A large diffuse floor (y = 0, albedo ``albedo``) under a square light of
    half-size ``light_half`` centred above the origin at height ``light_y``,
    facing down.  The floor spans [-1, 1]^2.  The camera looks straight down at
    the floor from just below the light plane, so with two path segments every
    pixel sees only the floor's first-bounce radiance, which has a closed form
    (irradiance from a polygonal Lambertian emitter)."""
    mats = [
        _lambert(albedo, albedo, albedo),
        _lambert(0.0, 0.0, 0.0, (radiance, radiance, radiance)),
    ]
    big = 1.0
    h = light_half
    quads = [
        [-big, 0.0, -big, 0.0, 0.0, 2 * big, 2 * big, 0.0, 0.0],
        [-h, light_y, -h, 2 * h, 0.0, 0.0, 0.0, 0.0, 2 * h],  # e1 x e2 = -y
    ]
    # camera below the light, looking down at the origin with a narrow field
    cam = [0.0, 0.5 * light_y, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0, 2.0]
    return _mk(quads, [0, 1], [], [], mats, cam, width, height, "area_light_plane")


def occluded_light_plane_scene(width: int = 1, height: int = 1, fov: float = 30.0,
                               occluder_x1: float = 0.0) -> Scene:
    """The floor of ``area_light_plane_scene`` (y = 0, [-1, 1]^2, albedo 0.5)
    under a 0.5 x 0.5 light of radiance 2 at height 1, with a black occluder
    quad at height 0.7 over x in [-0.5, occluder_x1], z in [-0.5, 0.5] that
    hides part of the light from the floor below the camera, so that both NEE
    (visibility) and BSDF sampling (hitting the light) have a large relative
    variance.  The camera looks straight down from (0, 0.5, 0) with vertical
    field of view ``fov``: one pixel covers a patch of floor whose irradiance
    varies across it."""
    mats = [
        _lambert(0.5, 0.5, 0.5),
        _lambert(0.0, 0.0, 0.0),
        _lambert(0.0, 0.0, 0.0, (2.0, 2.0, 2.0)),
    ]
    quads = [
        [-1.0, 0.0, -1.0, 0.0, 0.0, 2.0, 2.0, 0.0, 0.0],
        [-0.5, 0.7, -0.5, 0.0, 0.0, 1.0, occluder_x1 + 0.5, 0.0, 0.0],
        [-0.25, 1.0, -0.25, 0.5, 0.0, 0.0, 0.0, 0.0, 0.5],  # e1 x e2 = -y
    ]
    cam = [0.0, 0.5, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0, fov]
    return _mk(quads, [0, 1, 2], [], [], mats, cam, width, height, "occluded_light_plane")


def light_step_scene(floor_ggx_alpha: float = 0.0) -> Scene:
    """A floor (y = 0, [-1, 1]^2; Lambertian of albedo 0.5, or GGX of roughness
    ``floor_ggx_alpha`` > 0 and colour 0.5), a Lambertian wall at x = 1 (y in
    [0, 2], z in [-1, 1], albedo 0.5) and a 0.5 x 0.5 light of radiance 2 at
    height 1 facing down (light 0): the geometry of the checks of light subpath
    steps (emission from the light, one bounce on the floor towards the wall)."""
    floor = _ggx(0.5, 0.5, 0.5, floor_ggx_alpha) if floor_ggx_alpha > 0.0 else _lambert(0.5, 0.5, 0.5)
    mats = [floor, _lambert(0.5, 0.5, 0.5), _lambert(0.0, 0.0, 0.0, (2.0, 2.0, 2.0))]
    quads = [
        [-1.0, 0.0, -1.0, 0.0, 0.0, 2.0, 2.0, 0.0, 0.0],
        [1.0, 0.0, -1.0, 0.0, 0.0, 2.0, 0.0, 2.0, 0.0],
        [-0.25, 1.0, -0.25, 0.5, 0.0, 0.0, 0.0, 0.0, 0.5],  # e1 x e2 = -y
    ]
    cam = [0.0, 0.5, -2.0, 0.0, 0.5, 0.0, 0.0, 1.0, 0.0, 40.0]
    return _mk(quads, [0, 1, 2], [], [], mats, cam, 1, 1, "light_step")


def guided_room_scene(seed: int = 0, width: int = 512, height: int = 512,
                      n_spheres: int = 64, n_lights: int = 4) -> Scene:
    """Closed 4 x 4 x 4 room (albedo 0.7) with ``n_spheres`` seeded spheres
    (centres uniform in the room, radius U[0.05, 0.5], scaled by (64 /
    n_spheres)^(1/3) beyond 64 spheres so that they fill the room no more than
    64 do; a sphere that would hold the camera shrinks to 0.9 of its distance
    from it); 70 % GGX with roughness U[0.05, 0.5] and 30 % Lambertian, colour
    U[0.2, 0.9] per channel; and ``n_lights`` 0.3 x 0.3 ceiling lights with
    radiance log-uniform in [1, 100]."""
    rng = np.random.Generator(np.random.Philox(key=seed))
    L = 4.0
    cam = [2.0, 2.0, 0.05, 2.0, 1.6, 4.0, 0.0, 1.0, 0.0, 65.0]
    rscale = (64.0 / n_spheres) ** (1.0 / 3.0) if n_spheres > 64 else 1.0
    mats = [_lambert(0.7, 0.7, 0.7)]
    quads = [
        [0, 0, 0, 0, 0, L, L, 0, 0],   # floor
        [0, L, 0, L, 0, 0, 0, 0, L],   # ceiling
        [0, 0, 0, L, 0, 0, 0, L, 0],   # z = 0
        [0, 0, L, 0, L, 0, L, 0, 0],   # z = L
        [0, 0, 0, 0, L, 0, 0, 0, L],   # x = 0
        [L, 0, 0, 0, 0, L, 0, L, 0],   # x = L
    ]
    quad_mat = [0] * 6
    spheres = []
    sphere_mat = []
    for _ in range(n_spheres):
        c = rng.uniform(0.0, L, size=3)
        r = rng.uniform(0.05, 0.5) * rscale
        dcam = math.sqrt(sum((c[k] - cam[k]) ** 2 for k in range(3)))
        if dcam <= r:
            r = 0.9 * dcam
        col = rng.uniform(0.2, 0.9, size=3)
        if rng.uniform() < 0.7:
            mats.append(_ggx(col[0], col[1], col[2], rng.uniform(0.05, 0.5)))
        else:
            mats.append(_lambert(col[0], col[1], col[2]))
        spheres.append([c[0], c[1], c[2], r])
        sphere_mat.append(len(mats) - 1)
    s = 0.3
    y_light = L - 1e-4 * L
    for _ in range(n_lights):
        x, z = rng.uniform(0.3, L - 0.3 - s, size=2)
        le = math.exp(rng.uniform(math.log(1.0), math.log(100.0)))
        mats.append(_lambert(0.0, 0.0, 0.0, (le, le, le)))
        quads.append([x, y_light, z, s, 0, 0, 0, 0, s])  # e1 x e2 = -y
        quad_mat.append(len(mats) - 1)
    return _mk(quads, quad_mat, spheres, sphere_mat, mats, cam, width, height, "guided_room")


def heightfield_scene(seed: int = 0, n: int = 256, width: int = 1024, height: int = 1024,
                      n_spheres: int = 200, size: float = 8.0, n_lights: int = 0,
                      ggx_fraction: float = 0.6) -> Scene:
    """A seeded heightfield of n x n quads (2 n^2 triangles, heights from three
    octaves of bilinearly interpolated value noise, Lambertian albedo 0.6) over a
    size x size square, with ``n_spheres`` spheres resting above it (radius
    U[0.05, 0.3], a fraction ``ggx_fraction`` GGX with roughness U[0.05, 0.5],
    the rest Lambertian), and one small 0.2 x 0.2 emitter of radiance 200 facing
    down, hidden low between two large occluding spheres so that little of the
    terrain sees it directly -- the geometry of the bidirectional workloads, here
    lit for the unidirectional tracer.  With ``n_lights`` > 0 the hidden emitter
    is replaced by that many 0.3 x 0.3 emitters facing down at heights
    U[2.5, 3.5] over the terrain, grey radiance log-uniform in [0.5, 500]."""
    rng = np.random.Generator(np.random.Philox(key=seed + 7))

    def noise(cells):
        g = rng.uniform(0.0, 1.0, size=(cells + 1, cells + 1))
        x = np.linspace(0.0, cells, n + 1)
        i = np.minimum(x.astype(int), cells - 1)
        f = x - i
        a = g[i][:, i] * (1 - f)[None, :] + g[i][:, i + 1] * f[None, :]
        b = g[i + 1][:, i] * (1 - f)[None, :] + g[i + 1][:, i + 1] * f[None, :]
        return a * (1 - f)[:, None] + b * f[:, None]

    h = 0.8 * noise(4) + 0.3 * noise(16) + 0.08 * noise(64)
    xs = np.linspace(0.0, size, n + 1)
    P = np.stack(np.meshgrid(xs, xs, indexing="ij"), axis=-1)         # [n+1, n+1, (x, z)]
    V = np.stack([P[..., 0], h, P[..., 1]], axis=-1)                   # vertices
    a, b = V[:-1, :-1].reshape(-1, 3), V[1:, :-1].reshape(-1, 3)
    c, d = V[1:, 1:].reshape(-1, 3), V[:-1, 1:].reshape(-1, 3)
    # both triangles wound so that the normal points up (+y)
    tris = np.concatenate([np.concatenate([a, d, c], 1), np.concatenate([a, c, b], 1)], 0)
    mats = [_lambert(0.6, 0.6, 0.6)]
    spheres, sphere_mat = [], []
    for _ in range(n_spheres):
        x, z = rng.uniform(0.2, size - 0.2, size=2)
        r = rng.uniform(0.05, 0.3)
        col = rng.uniform(0.2, 0.9, size=3)
        if rng.uniform() < ggx_fraction:
            mats.append(_ggx(col[0], col[1], col[2], rng.uniform(0.05, 0.5)))
        else:
            mats.append(_lambert(col[0], col[1], col[2]))
        spheres.append([x, 1.2 + r + rng.uniform(0.0, 0.4), z, r])
        sphere_mat.append(len(mats) - 1)
    if n_lights > 0:
        quads, quad_mat = [], []
        for _ in range(n_lights):
            lx, lz = rng.uniform(0.5, size - 0.8, size=2)
            ly = rng.uniform(2.5, 3.5)
            le = math.exp(rng.uniform(math.log(0.5), math.log(500.0)))
            mats.append(_lambert(0.0, 0.0, 0.0, (le, le, le)))
            quads.append([lx, ly, lz, 0.3, 0, 0, 0, 0, 0.3])            # e1 x e2 = -y: faces down
            quad_mat.append(len(mats) - 1)
    else:
        # the hidden emitter: low above the middle, between two big spheres
        mats.append(_lambert(0.0, 0.0, 0.0, (200.0, 200.0, 200.0)))
        lx, lz, ly = 0.5 * size - 0.1, 0.5 * size - 0.1, 1.45
        quads = [[lx, ly, lz, 0.2, 0, 0, 0, 0, 0.2]]                   # e1 x e2 = -y: faces down
        quad_mat = [len(mats) - 1]
        occ = len(mats)
        mats.append(_lambert(0.5, 0.5, 0.5))
        for dx in (-0.45, 0.65):
            spheres.append([0.5 * size + dx, 1.45, 0.5 * size, 0.4])
            sphere_mat.append(occ)
    cam = [0.5 * size, 4.0, -2.5, 0.5 * size, 0.6, 0.5 * size, 0.0, 1.0, 0.0, 50.0]
    sc = _mk(quads, quad_mat, spheres, sphere_mat, mats, cam, width, height, "heightfield")
    sc.tris = _f32(tris)
    sc.tri_mat = np.zeros(len(tris), dtype=np.int32)
    return sc


def config_heightfield(width: int = 1024, height: int = 1024, seed: int = 0) -> WorkloadConfig:
    """Heightfield 256 x 256 quads (131k triangles) + 200 spheres, 1024^2, D = 10,
    BSDF + NEE + guided, 32^3 grid (the geometry of the bidirectional workload,
    rendered unidirectionally)."""
    return WorkloadConfig(heightfield_scene(seed, 256, width, height), max_depth=10, grid_n=32,
                          techniques=TECH_BSDF | TECH_NEE | TECH_GUIDED, iterations=16, warmup=3,
                          name=f"heightfield_256q_{width}x{height}_D10_bsdf+nee+guided_grid32")


def config_large(width: int = 2048, height: int = 2048, seed: int = 0) -> WorkloadConfig:
    """Heightfield 512 x 512 quads (524k triangles) + 4096 GGX spheres, 8 area
    lights with radiance log-U[0.5, 500], 2048^2, D = 12, BSDF + NEE (the
    bidirectional application has no guiding), 32^3 grid: the geometry of the
    large bidirectional workload, rendered unidirectionally."""
    return WorkloadConfig(heightfield_scene(seed, 512, width, height, n_spheres=4096, n_lights=8, ggx_fraction=1.0),
                          max_depth=12, grid_n=32, techniques=TECH_BSDF | TECH_NEE, iterations=64,
                          warmup=3, name=f"heightfield_512q_{width}x{height}_D12_bsdf+nee_grid32")


def config_bdpt_heightfield(width: int = 1024, height: int = 1024, seed: int = 0) -> WorkloadConfig:
    """The bidirectional workload: the heightfield of 256 x 256 quads (131k
    triangles) with 200 spheres and one small emitter hidden between two
    occluding spheres, 1024^2, D = 10, BSDF + NEE + light connections (light
    subpaths of at most 6 vertices), 32^3 grid refined as an adaptive octree of
    at most 64k leaves, 32 iterations, 3 warm-up."""
    return WorkloadConfig(heightfield_scene(seed, 256, width, height), max_depth=10, grid_n=32,
                          techniques=TECH_BSDF | TECH_NEE | TECH_LIGHT, iterations=32, warmup=3,
                          name=f"bdpt_heightfield_256q_{width}x{height}_D10_bsdf+nee+light_octree64k")


def config_bdpt_large(width: int = 2048, height: int = 2048, seed: int = 0) -> WorkloadConfig:
    """The large bidirectional workload: 512 x 512 quads (524k triangles) + 4096
    GGX spheres, 8 area lights with radiance log-U[0.5, 500], 2048^2, D = 12,
    BSDF + NEE + light connections, adaptive octree of at most 64k leaves, 64
    iterations at 1 spp, 3 warm-up."""
    return WorkloadConfig(heightfield_scene(seed, 512, width, height, n_spheres=4096, n_lights=8, ggx_fraction=1.0),
                          max_depth=12, grid_n=32, techniques=TECH_BSDF | TECH_NEE | TECH_LIGHT, iterations=64,
                          warmup=3, name=f"bdpt_heightfield_512q_{width}x{height}_D12_bsdf+nee+light_octree64k")


def config_box(width: int = 64, height: int = 64) -> WorkloadConfig:
    """Box scene, 64 x 64, D = 5, BSDF + NEE, 8^3 grid, 4 iterations, 1 warm-up."""
    return WorkloadConfig(box_scene(width, height), max_depth=5, grid_n=8,
                          techniques=TECH_BSDF | TECH_NEE, iterations=4, warmup=1,
                          name=f"box_{width}x{height}_D5_bsdf+nee_grid8")


def config_guided(width: int = 512, height: int = 512, seed: int = 0) -> WorkloadConfig:
    """Guided room, 512 x 512, D = 10, BSDF + NEE + guided, 32^3 grid,
    16 iterations, 3 warm-up."""
    return WorkloadConfig(guided_room_scene(seed, width, height), max_depth=10, grid_n=32,
                          techniques=TECH_BSDF | TECH_NEE | TECH_GUIDED, iterations=16,
                          warmup=3, name=f"guided_room_{width}x{height}_D10_bsdf+nee+guided_grid32")


def random_count_fields(n_cells: int, seed: int, lo: float = 0.05, hi: float = 4.0,
                        p_valid: float = 0.8):
    """Seeded random count factors q^RR >= q^S >= 0 per (cell, technique, channel)
    and validity flags per (cell, technique), in the cache layout
    [cell][technique slot 0..2][channel]."""
    rng = np.random.default_rng(seed)
    q_rr = np.exp(rng.uniform(np.log(lo), np.log(hi), size=(n_cells, 3, 3))).astype(np.float32)
    frac = rng.uniform(0.0, 1.0, size=(n_cells, 3, 3)).astype(np.float32)
    q_s = (q_rr * frac).astype(np.float32)
    valid = (rng.uniform(size=(n_cells, 3)) < p_valid).astype(np.uint8)
    return q_rr, q_s, valid


def random_guide_cdf(n_cells: int, seed: int, sparsity: float = 0.7) -> np.ndarray:
    """Seeded per-cell inclusive CDFs over the 256 directional bins, in float32:
    a sparse random histogram plus a small positive floor, normalised, so that
    every bin has a positive probability and some bins dominate."""
    rng = np.random.default_rng(seed)
    h = rng.exponential(1.0, size=(n_cells, GUIDE_BINS))
    h[rng.uniform(size=h.shape) < sparsity] = 0.0
    h += rng.uniform(0.005, 0.05, size=(n_cells, 1))
    cdf = np.cumsum(h / h.sum(axis=1, keepdims=True), axis=1)
    cdf[:, -1] = 1.0
    return cdf.astype(np.float32)


def serving_requests(n: int = 256, rate: float = 20.0, seed: int = 0,
                     resolutions=(64, 128, 256, 512), spheres=(16, 4096), iterations=(4, 16),
                     warmup: int = 3):
    """A seeded stream of render requests: Poisson arrivals at ``rate`` per
    second (exponential gaps), a square resolution drawn uniformly from
    ``resolutions`` (log-uniform over 64^2 .. 512^2), a room with a log-uniform
    number of spheres in ``spheres`` and 4 ceiling lights, and a uniform number
    of fixed-point iterations in ``iterations`` (at least warmup + 1).  Every
    request carries its own scene seed and Philox key.  The statistics grid is
    as fine as the job's camera samples allow: about 64 of them per cell over
    the job (N^3 cells, N = round((pixels x iterations / 64)^(1/3)) between 8
    and 32) -- a 32^3 grid for a 128^2 job of 16 iterations would hold about
    eight samples per cell, too few for any count to be learned."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for k in range(n):
        t += rng.exponential(1.0 / rate)
        res = int(resolutions[rng.integers(len(resolutions))])
        ns = int(round(math.exp(rng.uniform(math.log(spheres[0]), math.log(spheres[1])))))
        iters = int(rng.integers(iterations[0], iterations[1] + 1))
        scene_seed = int(rng.integers(1, 2 ** 31))
        sc = guided_room_scene(scene_seed, res, res, n_spheres=ns)
        sc.name = f"room{ns}_{res}x{res}"
        iters = max(iters, warmup + 1)
        grid_n = int(min(32, max(8, round((res * res * iters / 64.0) ** (1.0 / 3.0)))))
        out.append({"arrival_s": t, "scene": sc, "iterations": iters, "warmup": warmup,
                    "seed": scene_seed & 0xFFFFFFFF, "key": k + 1, "grid_n": grid_n, "max_depth": 10,
                    "techniques": TECH_BSDF | TECH_NEE | TECH_GUIDED})
    return out


def random_pixel_estimate(n_pixels: int, seed: int, lo: float = 0.05, hi: float = 2.0) -> np.ndarray:
    """Seeded positive per-pixel estimates [pixel][channel] in float32."""
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=(n_pixels, 3))).astype(np.float32)
