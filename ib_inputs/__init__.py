"""Seeded synthetic inputs for the spreading / interpolation workloads.

This module is shared by the oracle tests, the CUDA parity tests and the
benchmark.  It holds only input synthesis: random numbers, point clouds,
membrane geometry, force and velocity fields, job mixes and arrival times.
It contains none of the method's arithmetic (no kernel, no cell map, no
spreading or interpolation), so neither side of a parity comparison can
borrow a step from the other through it.

Random numbers come from a counter-based SplitMix64 stream (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
value k of stream `key` is mix64(key + (k + 1) * 0x9E3779B97F4A7C15).  A
stream is addressed by (seed, purpose string), so every array can be
regenerated on its own, on any machine, without shipping files.

Workload shapes follow the paper's experiments: randomly placed points in a
triply periodic box under a shear flow (Section 4.1), and red-blood-cell
membranes with the Omori reference shape (Section 4.2, the RBC equation).
"""

from __future__ import annotations

import functools
import math
from dataclasses import dataclass

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _fnv1a64(text: str) -> int:
    h = 0xCBF29CE484222325
    for byte in text.encode():
        h ^= byte
        h = (h * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
    return h


def stream_key(seed: int, purpose: str) -> int:
    """64-bit key of the stream named `purpose` under `seed`."""
    z = np.array([(_fnv1a64(purpose) ^ (int(seed) * 0x2545F4914F6CDD1D)) & 0xFFFFFFFFFFFFFFFF],
                 dtype=np.uint64)
    with np.errstate(over="ignore"):
        return int(_mix64(z)[0])


def u64(key: int, n: int, offset: int = 0) -> np.ndarray:
    """Values offset .. offset+n-1 of the SplitMix64 stream `key`."""
    ctr = np.arange(offset, offset + n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(np.uint64(key) + (ctr + np.uint64(1)) * _GOLDEN)


def uniform(key: int, n: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1) with 53 random bits."""
    return (u64(key, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(key: int, n: int) -> np.ndarray:
    """N(0, 1) doubles by the Box-Muller transform on two uniform streams."""
    u1 = ((u64(key, n, 0) >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)  # (0, 1]
    u2 = uniform(key ^ 0x5DEECE66D, n)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def _round_into_box(x: np.ndarray, L: np.ndarray, dtype) -> np.ndarray:
    """Round positions to `dtype` once and keep them inside [0, L)."""
    out = x.astype(dtype)
    Lt = np.asarray(L, dtype=dtype)
    over = out >= Lt
    if np.any(over):
        below = np.nextafter(Lt, np.zeros_like(Lt)).astype(dtype)
        out = np.where(over, np.broadcast_to(below, out.shape), out)
    return out


def uniform_points(seed: int, n: int, L, dim: int, dtype=np.float32, purpose: str = "X") -> np.ndarray:
    """n points uniform in the box [0, L_0) x ... x [0, L_{d-1}), shape (n, dim), row-major."""
    L = np.asarray(L, dtype=np.float64)[:dim]
    raw = uniform(stream_key(seed, purpose), n * dim).reshape(n, dim) * L
    return _round_into_box(raw, L, dtype)


def normal_array(seed: int, shape, dtype=np.float32, purpose: str = "G") -> np.ndarray:
    """N(0, 1) array of the given shape, generated in FP64 and rounded once to dtype."""
    count = int(np.prod(shape))
    return normal(stream_key(seed, purpose), count).reshape(shape).astype(dtype)


def shear_field_mac(N: int, L: float, gamma: float, dtype=np.float32) -> np.ndarray:
    """The paper's shear flow u = (0, 0, gamma (y - L/2)) on a 3-D MAC grid (Section 4).

    Component-major array [3][N][N][N] (z, y, x; x fastest).  The z-velocity
    lives on z-faces, whose nodes sit at y = h (j + 1/2); the x and y
    components are zero.  The flow jumps at the periodic seam y = 0.
    """
    h = L / N
    y = h * (np.arange(N, dtype=np.float64) + 0.5)
    u = np.zeros((3, N, N, N), dtype=np.float64)
    u[2] = (gamma * (y - 0.5 * L))[None, :, None]
    return u.astype(dtype)


def uniform_array(seed: int, shape, lo: float = -1.0, hi: float = 1.0, dtype=np.float32,
                  purpose: str = "G") -> np.ndarray:
    """Uniform [lo, hi) array of the given shape, generated in FP64 and rounded once to dtype
    (a cheaper stand-in for normal_array on very large inputs)."""
    count = int(np.prod(shape))
    return (lo + (hi - lo) * uniform(stream_key(seed, purpose), count)).reshape(shape).astype(dtype)


def wave_field(N: int, ncomp: int = 3, dtype=np.float32) -> np.ndarray:
    """A deterministic grid field [ncomp][N][N][N] of plane waves up to the Nyquist range:
    u_a = sin(2 pi (k_a x + l_a y + m_a z) / N + phase_a) over node indices, with wavenumbers
    that make neighbouring nodes differ strongly (for interpolation checks on grids too
    large for a random field to be generated quickly)."""
    waves = [(3, 251, 17, 0.3), (199, 5, 101, 1.1), (61, 127, 233, 2.0), (255, 64, 7, 0.7)]
    i = np.arange(N, dtype=np.float64) * (2.0 * np.pi / N)
    out = np.empty((ncomp, N, N, N), dtype=dtype)
    for a in range(ncomp):
        k, l, m, ph = waves[a % len(waves)]
        for z in range(N):
            out[a, z] = np.sin(k * i[None, :] + l * i[:, None] + (m * i[z] + ph))
    return out


# ---------------------------------------------------------------------------
# Red-blood-cell membranes (Section 4.2, Omori reference shape)
# ---------------------------------------------------------------------------

RBC_R0_UM = 3.91          # reference radius R0 in micrometres (Section 4.2)
BOX_UM = 16.0             # side of the paper's triply periodic box


@functools.lru_cache(maxsize=8)
def icosphere(subdivisions: int) -> np.ndarray:
    """Vertices of a subdivided icosahedron on the unit sphere (10*4^k + 2 of them)."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    verts = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
             (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
             (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    verts = [np.array(v, dtype=np.float64) / np.linalg.norm(v) for v in verts]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
             (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
             (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
             (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(subdivisions):
        cache = {}

        def midpoint(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        new_faces = []
        for a, b, c in faces:
            ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
            new_faces += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = new_faces
    out = np.array(verts)
    out.setflags(write=False)
    return out


def _omori_p(r):
    return 0.105 + r * r - 0.56 * r ** 4


@functools.lru_cache(maxsize=16)
def rbc_surface(R0: float, subdivisions: int = 4) -> np.ndarray:
    """Omori RBC surface points in the body frame, from an icosphere by (theta, phi) = (atan2(y,x), asin z)."""
    s = icosphere(subdivisions)
    theta = np.arctan2(s[:, 1], s[:, 0])
    phi = np.arcsin(np.clip(s[:, 2], -1.0, 1.0))
    cphi = np.cos(phi)
    out = np.stack([R0 * np.cos(theta) * cphi,
                    R0 * np.sin(theta) * cphi,
                    R0 * _omori_p(cphi) * np.sin(phi)], axis=1)
    out.setflags(write=False)
    return out


def rbc_half_thickness(rho: np.ndarray, R0: float) -> np.ndarray:
    r = np.clip(rho / R0, 0.0, 1.0)
    return R0 * _omori_p(r) * np.sqrt(np.maximum(0.0, 1.0 - r * r))


def rbc_inside(p: np.ndarray, R0: float) -> np.ndarray:
    """Points (body frame) strictly inside the RBC body {|z| < h(rho), rho < R0}."""
    rho = np.hypot(p[:, 0], p[:, 1])
    return (rho < R0) & (np.abs(p[:, 2]) < rbc_half_thickness(rho, R0))


def rbc_volume(R0: float, samples: int = 20000) -> float:
    """Volume of the RBC body by the midpoint rule in rho (2 pi rho * 2 h(rho))."""
    rho = (np.arange(samples) + 0.5) * (R0 / samples)
    return float(np.sum(2.0 * np.pi * rho * 2.0 * rbc_half_thickness(rho, R0)) * (R0 / samples))


def random_rotation(key: int, k: int) -> np.ndarray:
    """Uniform random rotation (Shoemake's quaternion method), number k of stream `key`."""
    u1, u2, u3 = uniform(key, 3, offset=3 * k)
    q = np.array([math.sqrt(1 - u1) * math.sin(2 * math.pi * u2),
                  math.sqrt(1 - u1) * math.cos(2 * math.pi * u2),
                  math.sqrt(u1) * math.sin(2 * math.pi * u3),
                  math.sqrt(u1) * math.cos(2 * math.pi * u3)])
    x, y, z, w = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


@dataclass
class Membranes:
    X: np.ndarray            # (n, 3) positions in [0, L)
    cell_of_point: np.ndarray
    centres: np.ndarray      # (ncells, 3)
    rotations: np.ndarray    # (ncells, 3, 3) body -> lab
    offsets: np.ndarray      # (n, 3) lab-frame offset of each point from its cell centre
    R0: float
    volume_fraction: float
    attempts: int


@functools.lru_cache(maxsize=8)
def fibonacci_sphere(n: int) -> np.ndarray:
    """n nearly uniform points on the unit sphere (golden-angle spiral), for point counts
    that are not icosphere counts (the paper's 8832 data sites per cell)."""
    k = np.arange(n, dtype=np.float64) + 0.5
    z = 1.0 - 2.0 * k / n
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = np.pi * (3.0 - math.sqrt(5.0)) * k
    out = np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)
    out.setflags(write=False)
    return out


def rbc_points(R0: float, sphere: np.ndarray) -> np.ndarray:
    """Omori RBC surface points (body frame) from unit-sphere points by (theta, phi) = (atan2(y,x), asin z)."""
    theta = np.arctan2(sphere[:, 1], sphere[:, 0])
    phi = np.arcsin(np.clip(sphere[:, 2], -1.0, 1.0))
    cphi = np.cos(phi)
    return np.stack([R0 * np.cos(theta) * cphi, R0 * np.sin(theta) * cphi,
                     R0 * _omori_p(cphi) * np.sin(phi)], axis=1)


def _small_rotation(u: np.ndarray, angle: float) -> np.ndarray:
    """Rotation by `angle` * u[3] about the axis of (u[0], u[1], u[2]) - 1/2 (Rodrigues)."""
    axis = u[:3] - 0.5
    nrm = np.linalg.norm(axis)
    axis = axis / nrm if nrm > 1e-12 else np.array([0.0, 0.0, 1.0])
    t = angle * (2.0 * u[3] - 1.0)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(t) * K + (1.0 - math.cos(t)) * (K @ K)


def pack_membranes(seed: int, L: float = 1.0, target_cells: int = 17, subdivisions: int = 4,
                   max_attempts: int = 20000, gap: float = 0.02, dtype=np.float32,
                   points_per_cell: int | None = None, max_sweeps: int = 600) -> Membranes:
    """Non-overlapping, randomly oriented RBCs in a periodic box, packed by compression.

    The box side L stands for the paper's 16 um, so R0 = 3.91/16 L.  Two cells
    overlap when a probe point of one (its surface inflated by `gap` R0) lies
    inside the other, over the nearest periodic image.  The cells are first
    placed by random sequential addition at a reduced size s R0 (s = 0.6),
    where `target_cells` of them fit easily, with uniform random orientations
    (Shoemake quaternions); then they are compressed: sweeps of Monte Carlo
    moves (a small random translation and rotation of each cell in turn,
    kept when it overlaps nothing) alternate with growing s to the largest
    overlap-free value, until s = 1 or `max_sweeps` sweeps.  A packing that
    cannot reach full size keeps the cells placed so far at s = 1 that do not
    overlap (dropping the others).  Every random number comes from the
    counter-based streams of this module, so the packing depends on `seed`
    only.  The surface points are the subdivision-`subdivisions` icosphere
    (2562 points for 4), or `points_per_cell` golden-spiral points, mapped
    onto the Omori shape; the achieved volume fraction is returned.
    """
    R0 = RBC_R0_UM / BOX_UM * L
    sphere = fibonacci_sphere(points_per_cell) if points_per_cell else icosphere(subdivisions)
    surf = rbc_points(R0, sphere)
    unit_probe = rbc_points(1.0, icosphere(3)) * (1.0 + gap)       # R0 = 1, inflated
    kc = stream_key(seed, "rbc-centre")
    kr = stream_key(seed, "rbc-rotation")
    km = stream_key(seed, "rbc-move")

    def near(d, sc):
        return np.linalg.norm(d) <= 2.0 * sc * R0 * (1.0 + gap)

    def overlap(c1, R1, c2, R2, sc):
        d = c1 - c2
        d -= L * np.round(d / L)
        if not near(d, sc):
            return False
        p1 = unit_probe * (sc * R0)
        if rbc_inside((p1 @ R1.T + d) @ R2, sc * R0).any():
            return True
        return bool(rbc_inside((p1 @ R2.T - d) @ R1, sc * R0).any())

    def free(i, c, R, cen, rot, sc):
        return not any(overlap(c, R, cen[j], rot[j], sc) for j in range(len(cen)) if j != i)

    # 1. random sequential addition at the reduced size
    s = 0.6
    centres, rots = [], []
    attempts = 0
    while len(centres) < target_cells and attempts < max_attempts:
        c = uniform(kc, 3, offset=3 * attempts) * L
        R = random_rotation(kr, attempts)
        attempts += 1
        if free(-1, c, R, centres, rots, s):
            centres.append(c)
            rots.append(R)
    # 2. compression: Monte Carlo sweeps, then the largest overlap-free size
    move = 0
    sweeps = 0
    step = 0.08
    while s < 1.0 and sweeps < max_sweeps and centres:
        for i in range(len(centres)):
            u = uniform(km, 7, offset=7 * move)
            move += 1
            c = centres[i] + (u[:3] - 0.5) * (2.0 * step * s * R0)
            c -= L * np.floor(c / L)
            R = _small_rotation(u[3:], 2.0 * step) @ rots[i]
            if free(i, c, R, centres, rots, s):
                centres[i], rots[i] = c, R
        sweeps += 1
        lo, hi = s, min(1.0, s * 1.03)
        for _ in range(5):
            mid = hi if _ == 0 else 0.5 * (lo + hi)
            ok = all(not overlap(centres[i], rots[i], centres[j], rots[j], mid)
                     for i in range(len(centres)) for j in range(i + 1, len(centres)))
            if ok:
                lo = mid
                if _ == 0:
                    break
            else:
                hi = mid
        s = lo
    if s < 1.0:   # not compressed to full size: keep the cells that fit at s = 1
        kept_c, kept_r = [], []
        for c, R in zip(centres, rots):
            if free(-1, c, R, kept_c, kept_r, 1.0):
                kept_c.append(c)
                kept_r.append(R)
        centres, rots = kept_c, kept_r
    pts, owner, offs = [], [], []
    for ci, (c, R) in enumerate(zip(centres, rots)):
        off = surf @ R.T
        pts.append(c + off)
        offs.append(off)
        owner.append(np.full(len(surf), ci, dtype=np.int64))
    X = np.concatenate(pts) if pts else np.zeros((0, 3))
    X = X - L * np.floor(X / L)
    X = _round_into_box(X, np.array([L, L, L]), dtype)
    vf = len(centres) * rbc_volume(R0) / L ** 3
    return Membranes(X=X, cell_of_point=np.concatenate(owner) if owner else np.zeros(0, np.int64),
                     centres=np.array(centres).reshape(-1, 3), rotations=np.array(rots).reshape(-1, 3, 3),
                     offsets=np.concatenate(offs) if offs else np.zeros((0, 3)), R0=R0,
                     volume_fraction=vf, attempts=attempts + sweeps)


def membrane_forces(seed: int, mem: Membranes, dtype=np.float32) -> np.ndarray:
    """Smooth random membrane forces: per cell, a sum of six plane waves over the body offset."""
    ncells = len(mem.centres)
    D = 2.0 * mem.R0
    key_m = stream_key(seed, "force-modes")
    key_a = stream_key(seed, "force-amps")
    key_p = stream_key(seed, "force-phase")
    F = np.zeros((len(mem.X), 3))
    for ci in range(ncells):
        sel = mem.cell_of_point == ci
        off = mem.offsets[sel]
        m = (u64(key_m, 18, offset=18 * ci) % np.uint64(5)).astype(np.int64).reshape(6, 3) - 2
        m[np.all(m == 0, axis=1)] = (1, 0, 0)
        A = normal(key_a ^ ci, 18).reshape(6, 3) / math.sqrt(6.0)
        psi = uniform(key_p, 6, offset=6 * ci) * 2.0 * math.pi
        phase = 2.0 * math.pi * (off @ m.T) / D + psi       # (npts, 6)
        F[sel] = np.sin(phase) @ A
    return F.astype(dtype)


# ---------------------------------------------------------------------------
# Served batch: job mix and arrivals
# ---------------------------------------------------------------------------

@dataclass
class JobSpec:
    N: int
    npts: int
    clustered: bool
    seed: int


def job_mix(seed: int, njobs: int, grids=(32, 64, 96, 128), n_lo: float = 1e3, n_hi: float = 1e5):
    """Independent jobs: grid side uniform over `grids`, point count log-uniform in [n_lo, n_hi]."""
    kg = stream_key(seed, "job-grid")
    kn = stream_key(seed, "job-npts")
    kk = stream_key(seed, "job-kind")
    g = u64(kg, njobs) % np.uint64(len(grids))
    un = uniform(kn, njobs)
    npts = np.floor(np.exp(math.log(n_lo) + un * (math.log(n_hi) - math.log(n_lo)))).astype(np.int64)
    kind = uniform(kk, njobs) < 0.5
    return [JobSpec(N=int(grids[int(g[i])]), npts=int(npts[i]), clustered=bool(kind[i]),
                    seed=int(seed) * 1000003 + i) for i in range(njobs)]


def job_points(spec: JobSpec, L: float = 1.0, dtype=np.float32) -> np.ndarray:
    """Positions for one served job: uniform, or clustered on a few randomly placed RBC shells."""
    if not spec.clustered:
        return uniform_points(spec.seed, spec.npts, [L, L, L], 3, dtype)
    R0 = RBC_R0_UM / BOX_UM * L
    surf = rbc_surface(R0, 4)
    ncell = max(1, -(-spec.npts // len(surf)))
    kc = stream_key(spec.seed, "job-centre")
    kr = stream_key(spec.seed, "job-rot")
    kp = stream_key(spec.seed, "job-pick")
    per = [spec.npts // ncell + (1 if i < spec.npts % ncell else 0) for i in range(ncell)]
    pts = []
    for ci in range(ncell):
        order = np.argsort(u64(kp ^ ci, len(surf)), kind="stable")[:per[ci]]
        c = uniform(kc, 3, offset=3 * ci) * L
        pts.append(c + surf[order] @ random_rotation(kr, ci).T)
    X = np.concatenate(pts)
    X = X - L * np.floor(X / L)
    return _round_into_box(X, np.array([L, L, L]), dtype)


def poisson_arrivals(seed: int, njobs: int, rate_per_s: float) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process with the given rate."""
    u = 1.0 - uniform(stream_key(seed, "arrivals"), njobs)        # (0, 1]
    return np.cumsum(-np.log(u) / rate_per_s)
