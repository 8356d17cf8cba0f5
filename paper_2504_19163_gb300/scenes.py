"""Seeded synthetic scene generators (input data only).

This module builds the meshes, emitters, receivers and shading points that both
the CUDA path and the CPU oracle consume.  It holds none of the bounding,
sampling or solving arithmetic: every array it returns is plain input data,
generated in float64 with numpy and stored as float32 (the precision the
kernels read).  The paper's scenes (Plane, Sphere, Slab, Pool; Sec. 6, Table
"tab:perf") are not available, so these generators stand in for them with the
same kind of geometry:

* ``heightfield``   -- a mirror heightfield on [-1,1]^2 made of seeded
  sinusoids (+ optional per-vertex noise), standing in for the Plane scene
  (single reflection, interpolated normals).
* ``gerstner``      -- a water surface made of seeded Gerstner waves over a
  pool floor, standing in for the Pool scene (single refraction).
* ``slab``          -- a glass slab whose top and bottom faces are seeded
  heightfields, standing in for the Slab scene (two refractions).

Triangles use the (N+1)^2 vertex grid with the quad diagonal alternating by
quad parity; all triangles are counter-clockwise seen from +z.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, Optional

import numpy as np

SURFACE_REFLECT = 0
SURFACE_REFRACT = 1


@dataclasses.dataclass
class Surface:
    """Triangle mesh with per-vertex normals (SoA float32, int32 indices)."""
    px: np.ndarray
    py: np.ndarray
    pz: np.ndarray
    nx: np.ndarray
    ny: np.ndarray
    nz: np.ndarray
    i0: np.ndarray
    i1: np.ndarray
    i2: np.ndarray
    kind: int = SURFACE_REFLECT
    eta: float = 1.0   # ratio of indices of refraction, incident side / transmitted side

    @property
    def n_verts(self) -> int:
        return int(self.px.shape[0])

    @property
    def n_tris(self) -> int:
        return int(self.i0.shape[0])


@dataclasses.dataclass
class Receiver:
    """Planar receiver parallelogram p0 + u*e1 + v*e2, (u,v) in [0,1]^2."""
    p0: np.ndarray
    e1: np.ndarray
    e2: np.ndarray


@dataclasses.dataclass
class Emitters:
    """Point emitters (positions and isotropic intensities), float32."""
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    intensity: np.ndarray

    @property
    def n(self) -> int:
        return int(self.x.shape[0])


@dataclasses.dataclass
class Scene:
    name: str
    s1: Surface
    s2: Optional[Surface]
    receiver: Receiver
    emitters: Emitters
    depth: int
    su: np.ndarray          # shading points, receiver texture coordinates
    sv: np.ndarray
    grid_res: int = 512
    extra: Dict = dataclasses.field(default_factory=dict)


def _grid_triangles(n: int) -> np.ndarray:
    """Indices (2 n^2, 3) of the (n+1)^2 vertex grid; diagonal alternates per quad parity."""
    tris = np.empty((2 * n * n, 3), dtype=np.int64)
    k = 0
    for j in range(n):
        for i in range(n):
            v00 = j * (n + 1) + i
            v10 = v00 + 1
            v01 = v00 + (n + 1)
            v11 = v01 + 1
            if (i + j) % 2 == 0:
                tris[k] = (v00, v10, v11)
                tris[k + 1] = (v00, v11, v01)
            else:
                tris[k] = (v00, v10, v01)
                tris[k + 1] = (v10, v11, v01)
            k += 2
    return tris


def _sinusoids(rng: np.random.Generator, n_waves: int, amp_total: float):
    kmag = rng.uniform(math.pi, 3.0 * math.pi, n_waves)
    ang = rng.uniform(0.0, 2.0 * math.pi, n_waves)
    phase = rng.uniform(0.0, 2.0 * math.pi, n_waves)
    kx = kmag * np.cos(ang)
    ky = kmag * np.sin(ang)
    amp = np.full(n_waves, amp_total / n_waves)
    return kx, ky, phase, amp


def _face_average_normals(P: np.ndarray, tris: np.ndarray) -> np.ndarray:
    """Area-weighted average of face normals at each vertex, normalized."""
    e1 = P[tris[:, 1]] - P[tris[:, 0]]
    e2 = P[tris[:, 2]] - P[tris[:, 0]]
    fn = np.cross(e1, e2)            # length = 2 * area
    N = np.zeros_like(P)
    for c in range(3):
        np.add.at(N, tris[:, c], fn)
    return N / np.linalg.norm(N, axis=1, keepdims=True)


def _to_surface(P: np.ndarray, N: np.ndarray, tris: np.ndarray, kind: int, eta: float) -> Surface:
    f = np.float32
    return Surface(px=P[:, 0].astype(f), py=P[:, 1].astype(f), pz=P[:, 2].astype(f),
                   nx=N[:, 0].astype(f), ny=N[:, 1].astype(f), nz=N[:, 2].astype(f),
                   i0=tris[:, 0].astype(np.int32), i1=tris[:, 1].astype(np.int32),
                   i2=tris[:, 2].astype(np.int32), kind=kind, eta=float(eta))


def _value_noise(X: np.ndarray, Y: np.ndarray, extent: float, lattice: int, amp: float,
                 rng: np.random.Generator) -> np.ndarray:
    """Smooth value noise: U[-amp, amp] on a (lattice+3)^2 grid over [-extent, extent]^2,
    Catmull-Rom interpolated (C1) at the points."""
    V = rng.uniform(-amp, amp, (lattice + 3, lattice + 3))
    gx = (X + extent) / (2 * extent) * lattice + 1.0
    gy = (Y + extent) / (2 * extent) * lattice + 1.0
    ix = np.clip(np.floor(gx).astype(np.int64), 1, lattice)
    iy = np.clip(np.floor(gy).astype(np.int64), 1, lattice)
    tx, ty = gx - ix, gy - iy

    def w(t):
        return np.stack([(-t ** 3 + 2 * t ** 2 - t) / 2, (3 * t ** 3 - 5 * t ** 2 + 2) / 2,
                         (-3 * t ** 3 + 4 * t ** 2 + t) / 2, (t ** 3 - t ** 2) / 2], axis=0)
    wx, wy = w(tx), w(ty)
    out = np.zeros_like(X)
    for a in range(4):
        for b in range(4):
            out += wx[a] * wy[b] * V[ix - 1 + a, iy - 1 + b]
    return out


def heightfield(n: int, seed: int, n_waves: int = 4, amp_total: float = 0.05,
                noise: float = 0.0, normals: str = "analytic", extent: float = 1.0,
                z0: float = 0.0, kind: int = SURFACE_REFLECT, eta: float = 1.0,
                flip_normals: bool = False, noise_lattice: int = 0) -> Surface:
    """Heightfield z = z0 + sum_i A sin(k_i . (x,y) + phi_i) + noise on [-extent,extent]^2.

    Noise of amplitude ``noise``: with ``noise_lattice = 0`` independent U[-noise, noise] per
    vertex; otherwise smooth value noise on a ``noise_lattice``^2 lattice.
    ``normals='analytic'`` uses the normalized gradient normal of the sinusoid sum;
    ``'face'`` uses the normalized area-weighted average of the face normals (needed once
    noise is added).
    """
    rng = np.random.default_rng(seed)
    kx, ky, ph, amp = _sinusoids(rng, n_waves, amp_total)
    xs = np.linspace(-extent, extent, n + 1)
    X, Y = np.meshgrid(xs, xs, indexing="xy")     # row j = y index, column i = x index
    X = X.reshape(-1)
    Y = Y.reshape(-1)
    arg = np.outer(X, kx) + np.outer(Y, ky) + ph
    Z = z0 + (np.sin(arg) * amp).sum(axis=1)
    if noise > 0.0 and noise_lattice == 0:
        Z = Z + rng.uniform(-noise, noise, Z.shape[0])
    elif noise > 0.0:
        Z = Z + _value_noise(X, Y, extent, noise_lattice, noise, rng)
    P = np.stack([X, Y, Z], axis=1)
    tris = _grid_triangles(n)
    if normals == "analytic":
        zx = (np.cos(arg) * amp * kx).sum(axis=1)
        zy = (np.cos(arg) * amp * ky).sum(axis=1)
        N = np.stack([-zx, -zy, np.ones_like(zx)], axis=1)
        N /= np.linalg.norm(N, axis=1, keepdims=True)
    elif normals == "face":
        N = _face_average_normals(P, tris)
    elif normals == "flat_up":
        N = np.tile(np.array([0.0, 0.0, 1.0]), (P.shape[0], 1))
    else:
        raise ValueError(normals)
    if flip_normals:
        N = -N
    return _to_surface(P, N, tris, kind, eta)


def gerstner(n: int, seed: int, n_waves: int = 16, extent: float = 2.0, steep: float = 0.02,
             lam_lo: float = 0.2, lam_hi: float = 1.0, eta: float = 1.0 / 1.33) -> Surface:
    """Water surface as a sum of Gerstner waves (k_i A_i = steep, Q_i = 1) on [-extent,extent]^2.

    Normals are the analytic normals of the displaced surface, normalized.
    """
    rng = np.random.default_rng(seed)
    lam = rng.uniform(lam_lo, lam_hi, n_waves)
    k = 2.0 * math.pi / lam
    A = steep / k
    ang = rng.uniform(0.0, 2.0 * math.pi, n_waves)
    ph = rng.uniform(0.0, 2.0 * math.pi, n_waves)
    Dx, Dy = np.cos(ang), np.sin(ang)
    xs = np.linspace(-extent, extent, n + 1)
    X, Y = np.meshgrid(xs, xs, indexing="xy")
    X = X.reshape(-1)
    Y = Y.reshape(-1)
    arg = np.outer(X, k * Dx) + np.outer(Y, k * Dy) + ph
    C, S = np.cos(arg), np.sin(arg)
    Px = X + (A * Dx * C).sum(axis=1)
    Py = Y + (A * Dy * C).sum(axis=1)
    Pz = (A * S).sum(axis=1)
    # Tangents of the displaced surface; normal = dP/dx x dP/dy.
    WA = k * A
    tx = np.stack([1.0 - (WA * Dx * Dx * S).sum(1), -(WA * Dx * Dy * S).sum(1), (WA * Dx * C).sum(1)], 1)
    ty = np.stack([-(WA * Dx * Dy * S).sum(1), 1.0 - (WA * Dy * Dy * S).sum(1), (WA * Dy * C).sum(1)], 1)
    N = np.cross(tx, ty)
    N /= np.linalg.norm(N, axis=1, keepdims=True)
    P = np.stack([Px, Py, Pz], axis=1)
    return _to_surface(P, N, _grid_triangles(n), SURFACE_REFRACT, eta)


def slab(n: int, seed: int, amp_total: float = 0.02, thickness: float = 0.2, ior: float = 1.5,
         extent: float = 1.0, flat: bool = False):
    """Glass slab: top face z = h1 and bottom face z = -thickness + h2 over [-extent,extent]^2,
    each an n^2 heightfield of 4 seeded sinusoids (amplitude ``amp_total`` in all), analytic
    normals.  Rays enter through the top (eta' = 1/ior) and leave through the bottom (eta' = ior);
    both faces' normals point up, toward the incident side.  ``flat``: two planes with normals
    (0, 0, 1) (closed-form checks)."""
    if flat:
        top = heightfield(n, seed, n_waves=1, amp_total=0.0, normals="flat_up", extent=extent,
                          kind=SURFACE_REFRACT, eta=1.0 / ior)
        bot = heightfield(n, seed + 1, n_waves=1, amp_total=0.0, normals="flat_up", extent=extent,
                          z0=-thickness, kind=SURFACE_REFRACT, eta=ior)
        return top, bot
    top = heightfield(n, seed, n_waves=4, amp_total=amp_total, extent=extent, kind=SURFACE_REFRACT, eta=1.0 / ior)
    bot = heightfield(n, seed + 1000, n_waves=4, amp_total=amp_total, extent=extent, z0=-thickness,
                      kind=SURFACE_REFRACT, eta=ior)
    return top, bot


def point_emitters(positions, intensity=1.0) -> Emitters:
    P = np.asarray(positions, dtype=np.float64).reshape(-1, 3)
    I = np.broadcast_to(np.asarray(intensity, dtype=np.float64), (P.shape[0],))
    f = np.float32
    return Emitters(P[:, 0].astype(f), P[:, 1].astype(f), P[:, 2].astype(f), I.astype(f))


def area_quad_emitters(center, size: float, strata: int, seed: int) -> Emitters:
    """Axis-aligned horizontal quad light, one jittered sample per stratum, I0 = 1/strata^2 each."""
    rng = np.random.default_rng(seed)
    c = np.asarray(center, dtype=np.float64)
    pts = []
    for j in range(strata):
        for i in range(strata):
            a = (i + rng.uniform()) / strata - 0.5
            b = (j + rng.uniform()) / strata - 0.5
            pts.append((c[0] + a * size, c[1] + b * size, c[2]))
    return point_emitters(pts, 1.0 / (strata * strata))


def receiver_square(center_z: float, half: float, cx: float = 0.0, cy: float = 0.0,
                    half_y: Optional[float] = None) -> Receiver:
    hy = half if half_y is None else half_y
    p0 = np.array([cx - half, cy - hy, center_z], dtype=np.float32)
    e1 = np.array([2.0 * half, 0.0, 0.0], dtype=np.float32)
    e2 = np.array([0.0, 2.0 * hy, 0.0], dtype=np.float32)
    return Receiver(p0, e1, e2)


def shading_points(nx: int, ny: int, seed: int, jitter: float = 0.25):
    """Pixel centres of an nx x ny grid over [0,1]^2 plus a seeded jitter of +-jitter pixel."""
    rng = np.random.default_rng(seed)
    i = np.arange(nx, dtype=np.float64)
    j = np.arange(ny, dtype=np.float64)
    I, J = np.meshgrid(i, j, indexing="xy")
    su = (I.reshape(-1) + 0.5 + rng.uniform(-jitter, jitter, nx * ny)) / nx
    sv = (J.reshape(-1) + 0.5 + rng.uniform(-jitter, jitter, nx * ny)) / ny
    return su.astype(np.float32), sv.astype(np.float32)


# ---------------------------------------------------------------------------
# Workloads.  Sizes follow the paper-shaped configurations:
#   mirror32   : 32^2 mirror (2048 tris), light (0,0,2), 64^2 points, depth 2
#   mirror256  : 256^2 mirror (131,072 tris), 6 sinusoids + smooth noise of
#                amplitude 0.01, 0.2x0.2 area light with 4x4 strata at z=2,
#                1024^2 points, depth 3
#   mirror256_rough : the same with independent per-vertex noise (bound tests only)
#   water420   : 420^2 Gerstner water (352,800 tris), 4 lights, floor 1 below,
#                1920x1080 points, depth 3
#   slab48     : glass slab with two 48^2 faces, light (0,0,2), 512^2 points, depth 2
# Reflection receivers sit at z=+1 facing the mirror (reflected rays travel up).
# ---------------------------------------------------------------------------

def mirror(n: int, seed: int, n_waves: int, noise: float, normals: str, emitters: Emitters,
           points: int, depth: int, name: str, receiver_z: float = 1.0, point_seed: Optional[int] = None,
           points_y: Optional[int] = None, noise_lattice: int = 0) -> Scene:
    s1 = heightfield(n, seed, n_waves=n_waves, amp_total=0.05, noise=noise, normals=normals,
                     noise_lattice=noise_lattice)
    rec = receiver_square(receiver_z, 1.5)
    py = points if points_y is None else points_y
    su, sv = shading_points(points, py, seed + 1000 if point_seed is None else point_seed)
    return Scene(name, s1, None, rec, emitters, depth, su, sv)


def config(name: str, **kw) -> Scene:
    """Named workloads (see module docstring)."""
    if name == "mirror32":
        em = point_emitters([(0.0, 0.0, 2.0)], 1.0)
        return mirror(32, 1, 4, 0.0, "analytic", em, kw.get("points", 64), kw.get("depth", 2), name,
                      receiver_z=kw.get("receiver_z", 1.0))
    if name == "mirror256":
        # smooth value noise of amplitude 0.01 on a 16^2 lattice (see the module docstring)
        em = area_quad_emitters((0.0, 0.0, 2.0), 0.2, 4, seed=2)
        return mirror(256, 2, 6, 0.01, "face", em, kw.get("points", 1024), kw.get("depth", 3), name,
                      noise_lattice=kw.get("noise_lattice", 16))
    if name == "mirror256_rough":
        # per-vertex U[-0.01, 0.01] noise (slopes up to ~2.5): every cell's image spreads over
        # hundreds of grid cells; kept for the bound-pass tests only
        em = area_quad_emitters((0.0, 0.0, 2.0), 0.2, 4, seed=2)
        return mirror(256, 2, 6, 0.01, "face", em, kw.get("points", 1024), kw.get("depth", 3), name)
    if name == "water420":
        # 420^2 Gerstner water on [-2,2]^2 (352,800 tris), eta' = 1/1.33, pool floor 1 below over
        # [-2,2] x [-1.125,1.125], lights at (+-0.5, +-0.5, 2), 1920x1080 points, depth 3
        s1 = gerstner(420, 3)
        em = point_emitters([(-0.5, -0.5, 2.0), (0.5, -0.5, 2.0), (-0.5, 0.5, 2.0), (0.5, 0.5, 2.0)], 1.0)
        rec = receiver_square(-1.0, 2.0, half_y=1.125)
        su, sv = shading_points(kw.get("points_x", 1920), kw.get("points_y", 1080), 1003)
        return Scene(name, s1, None, rec, em, kw.get("depth", 3), su, sv)
    if name == "tir_wall":
        # near total internal reflection: a light under water (eta' 1.33, normals facing down, the
        # incident side) below an n^2 heightfield at z=0 over [-1,1]^2; the critical angle is reached
        # at ~0.57 from the light's foot, and the grazing transmitted rays hit a vertical wall
        # receiver at x=1.2 (y in [-1,1], z in [0,1])
        n = kw.get("n", 4)
        s1 = heightfield(n, kw.get("seed", 5), n_waves=4, amp_total=kw.get("amp", 0.02), extent=1.0,
                         flip_normals=True, kind=SURFACE_REFRACT, eta=1.33)
        em = point_emitters(kw.get("lights", [(0.02, -0.01, -0.5)]), 1.0)
        rec = Receiver(np.array([1.2, -1.0, 0.0], np.float32), np.array([0.0, 2.0, 0.0], np.float32),
                       np.array([0.0, 0.0, 1.0], np.float32))
        p = kw.get("points", 32)
        su, sv = shading_points(p, p, 1008)
        return Scene(name, s1, None, rec, em, kw.get("depth", 3), su, sv)
    if name == "water":
        # small refraction case: n^2 Gerstner water on [-ext,ext]^2, floor 1 below
        n = kw.get("n", 8)
        ext = kw.get("extent", 0.5)
        s1 = gerstner(n, kw.get("seed", 3), n_waves=kw.get("waves", 16), extent=ext, steep=kw.get("steep", 0.02),
                      lam_lo=kw.get("lam_lo", 0.2), lam_hi=kw.get("lam_hi", 1.0))
        em = point_emitters(kw.get("lights", [(0.1, -0.05, 2.0)]), 1.0)
        rec = receiver_square(-1.0, kw.get("rec_half", 0.8))
        p = kw.get("points", 32)
        su, sv = shading_points(p, p, 1004)
        return Scene(name, s1, None, rec, em, kw.get("depth", 1), su, sv)
    if name == "slab48":
        # glass slab (ior 1.5) with two 48^2 faces (4608 triangles each) over [-1,1]^2, 0.2 thick,
        # light (0,0,2), receiver [-1.5,1.5]^2 at z=-1, 512^2 points, depth 2
        top, bot = slab(48, 4)
        em = point_emitters([(0.0, 0.0, 2.0)], 1.0)
        su, sv = shading_points(kw.get("points", 512), kw.get("points", 512), 1005)
        return Scene(name, top, bot, receiver_square(-1.0, 1.5), em, kw.get("depth", 2), su, sv)
    if name == "slab":
        # small slab: n^2 faces over [-ext,ext]^2 (same law as slab48), receiver [-rec,rec]^2 at z=-1
        n = kw.get("n", 4)
        ext = kw.get("extent", 0.5)
        top, bot = slab(n, kw.get("seed", 4), amp_total=kw.get("amp", 0.02), extent=ext,
                        thickness=kw.get("thickness", 0.2), flat=kw.get("flat", False))
        em = point_emitters(kw.get("lights", [(0.05, -0.03, 2.0)]), 1.0)
        p = kw.get("points", 32)
        su, sv = shading_points(p, p, 1006)
        return Scene(name, top, bot, receiver_square(-1.0, kw.get("rec_half", 0.8)), em, kw.get("depth", 1), su, sv)
    if name in ("periscope", "mirror_glass"):
        # two specular vertices with reflection: a mirror heightfield at z=0 (normals up) lit from
        # above, then at z=1 either a second mirror facing down (periscope; receiver between them at
        # z=0.5) or a refracting interface into glass (eta' 1/1.5, normals facing down, the incident
        # side; receiver above at z=1.5); n^2 faces over [-ext, ext]^2, 4 sinusoids each
        n = kw.get("n", 3)
        ext = kw.get("extent", 0.5)
        flat = kw.get("flat", False)
        amp = kw.get("amp", 0.02)
        mk = lambda seed, **a: (heightfield(n, seed, n_waves=1, amp_total=0.0, normals="flat_up", extent=ext, **a)
                                if flat else heightfield(n, seed, n_waves=4, amp_total=amp, extent=ext, **a))
        bottom = mk(kw.get("seed", 8))
        if name == "periscope":
            top = mk(kw.get("seed", 8) + 1000, z0=1.0, flip_normals=True)
            rec = receiver_square(0.5, kw.get("rec_half", 1.0))
        else:
            top = mk(kw.get("seed", 8) + 1000, z0=1.0, flip_normals=True, kind=SURFACE_REFRACT, eta=1.0 / 1.5)
            rec = receiver_square(1.5, kw.get("rec_half", 1.0))
        em = point_emitters(kw.get("lights", [(0.05, -0.03, 2.0)]), 1.0)
        p = kw.get("points", 32)
        su, sv = shading_points(p, p, 1007)
        return Scene(name, bottom, top, rec, em, kw.get("depth", 1), su, sv)
    if name == "tiny":
        # A few triangles: exhaustive enumeration fits in milliseconds.
        n = kw.get("n", 4)
        em = point_emitters(kw.get("lights", [(0.1, -0.05, 2.0)]), 1.0)
        return mirror(n, kw.get("seed", 7), 4, 0.0, "analytic", em, kw.get("points", 16),
                      kw.get("depth", 1), name)
    if name == "flat":
        # Flat mirror z=0 with flat normals: the image-point closed form applies.
        n = kw.get("n", 4)
        s1 = heightfield(n, 0, n_waves=1, amp_total=0.0, normals="flat_up")
        h = kw.get("h", 2.0)
        em = point_emitters([(0.0, 0.0, h)], 1.0)
        rec = receiver_square(kw.get("c", 1.0), 1.5)
        su, sv = shading_points(kw.get("points", 16), kw.get("points", 16), 3)
        return Scene(name, s1, None, rec, em, kw.get("depth", 1), su, sv)
    raise KeyError(name)


def emitter_pool(center, half: float, n: int, seed: int) -> Emitters:
    """n point lights drawn uniformly (seeded) over a horizontal square of half-size `half`
    centred at `center`, each of intensity 1/n."""
    rng = np.random.default_rng(seed)
    c = np.asarray(center, dtype=np.float64)
    xy = rng.uniform(-half, half, (n, 2))
    pts = np.stack([c[0] + xy[:, 0], c[1] + xy[:, 1], np.full(n, c[2])], axis=1)
    return point_emitters(pts, 1.0 / n)


# Serving catalogue: the three single-specular-vertex mesh sizes of the rendering workloads, each
# with a fixed pool of 8 point lights; a request renders a subset of a scene's pool.
SERVING_SCENES = ("serve32", "serve256", "serve420")
SERVING_POOL = 8


def serving_scene(name: str) -> Scene:
    """A scene of the serving catalogue (mesh, receiver, emitter pool, bound depth).

    serve32  : the 32^2 mirror heightfield (2048 tris), depth 2
    serve256 : the 256^2 mirror heightfield with smooth noise (131,072 tris), depth 3
    serve420 : the 420^2 Gerstner water surface (352,800 tris) as a mirror, receiver 1 above
               over [-2,2]^2, depth 3 (single reflection: the refracting variant of this mesh is
               not part of the rendering pass)
    Shading points are per request; the scene's own point set is a small placeholder."""
    su, sv = shading_points(8, 8, 0)
    if name == "serve32":
        s1 = heightfield(32, 1, n_waves=4, amp_total=0.05, normals="analytic")
        em = emitter_pool((0.0, 0.0, 2.0), 0.3, SERVING_POOL, seed=51)
        return Scene(name, s1, None, receiver_square(1.0, 1.5), em, 2, su, sv)
    if name == "serve256":
        s1 = heightfield(256, 2, n_waves=6, amp_total=0.05, noise=0.01, normals="face", noise_lattice=16)
        em = emitter_pool((0.0, 0.0, 2.0), 0.3, SERVING_POOL, seed=52)
        return Scene(name, s1, None, receiver_square(1.0, 1.5), em, 3, su, sv)
    if name == "serve420":
        s1 = gerstner(420, 3)
        s1 = dataclasses.replace(s1, kind=SURFACE_REFLECT, eta=1.0)
        em = emitter_pool((0.0, 0.0, 2.0), 0.5, SERVING_POOL, seed=53)
        return Scene(name, s1, None, receiver_square(1.0, 2.0), em, 3, su, sv)
    raise KeyError(name)


def synthetic_cell_records(n_tuples: int, depth: int, n_tris: int, n_emitters: int, n_overflow: int, seed: int,
                           grid_res: int = 512):
    """Seeded synthetic bound records (float32 SoA) in the record layout of the bound pass:
    4^depth contiguous base records per tuple, then `n_overflow` extra records that repeat
    tuples of the base part (as split children do).  Boxes cluster per tuple; some edges sit
    exactly on grid lines, at 0 or at 1; some records are culled; some bounds are +inf."""
    rng = np.random.default_rng(seed)
    cpt = 4 ** depth
    n_base = n_tuples * cpt
    n = n_base + n_overflow
    em = np.empty(n, np.int32)
    t0 = np.empty(n, np.int32)
    tup_e = rng.integers(0, n_emitters, n_tuples)
    tup_t = rng.permutation(n_tris)[:n_tuples] if n_tuples <= n_tris else rng.integers(0, n_tris, n_tuples)
    em[:n_base] = np.repeat(tup_e, cpt)
    t0[:n_base] = np.repeat(tup_t, cpt)
    pick = rng.integers(0, n_tuples, n_overflow)
    em[n_base:] = tup_e[pick]
    t0[n_base:] = tup_t[pick]
    centre = rng.uniform(-0.05, 1.05, (n_tuples, 2))
    c = np.concatenate([np.repeat(centre, cpt, axis=0), centre[pick]], axis=0)
    c = c + rng.normal(0, 0.004, c.shape)
    half = rng.exponential(0.002, (n, 2)) + rng.choice([0.0, 0.02], (n, 2), p=[0.97, 0.03])
    lo = c - half
    hi = c + half
    # snap some edges onto grid lines and onto the region boundary
    snap = rng.random((n, 2)) < 0.05
    lo[snap] = np.floor(lo[snap] * grid_res) / grid_res
    snap = rng.random((n, 2)) < 0.05
    hi[snap] = np.ceil(hi[snap] * grid_res) / grid_res
    lo = np.clip(lo, 0.0, 1.0).astype(np.float32)
    hi = np.clip(hi, 0.0, 1.0).astype(np.float32)
    flags = np.full(n, 1, np.uint32)
    empty = (lo > hi).any(axis=1)
    flags[empty] = 8
    cull = rng.random(n) < 0.05
    flags[cull] = 4
    e_hi = rng.lognormal(0.0, 1.0, n).astype(np.float32)
    e_hi[rng.random(n) < 0.01] = np.inf
    depths = np.concatenate([np.full(n_base, depth), np.full(n_overflow, depth + 1)]).astype(np.uint32)
    flags = flags | (depths << np.uint32(24))
    return dict(u_lo=lo[:, 0], u_hi=hi[:, 0], v_lo=lo[:, 1], v_hi=hi[:, 1], e_lo=np.zeros(n, np.float32),
                e_hi=e_hi, emitter=em, tri0=t0, tri1=np.full(n, -1, np.int32),
                cell=np.zeros(n, np.uint32), flags=flags, n_base=n_base, depth=depth)
