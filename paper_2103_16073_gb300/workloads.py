"""Seeded synthetic inputs: room meshes, sources, receivers, admittances.

This module only produces geometry and random numbers.  It holds none of the
boundary-element or FMM arithmetic: no normals, areas, quadrature points or
kernel values are computed here.  Both the CUDA path and the CPU oracle take
its arrays as plain inputs.

Geometry follows the rooms of Sec. 4 (a shoebox room and an L-shaped room,
walls meshed with flat triangles).  Every wall is split into a structured grid
of rectangles and every rectangle into two right triangles.  The vertex order
of every triangle is counter-clockwise seen from OUTSIDE the room, so the
right-hand normal points out of the room, as Eq. (sp3) requires.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SOUND_SPEED = 343.0  # m/s, the speed of sound used for the rooms of Sec. 4


def wavenumber(freq_hz: float, c: float = SOUND_SPEED) -> float:
    """k = omega / c (Eq. sp2)."""
    return 2.0 * math.pi * freq_hz / c


def _grid_face(origin, ea, eb, na, nb):
    """Vertices and triangles of one planar rectangular wall.

    origin, ea, eb: 3-vectors; the wall is origin + s*ea + t*eb, s,t in [0,1].
    Triangles are ordered so that (ea x eb) is their right-hand normal.
    """
    return _grid_face_st(origin, ea, eb, np.linspace(0.0, 1.0, na + 1), np.linspace(0.0, 1.0, nb + 1))


def _grid_face_st(origin, ea, eb, s, t):
    """As _grid_face with explicit grid lines s[0..na], t[0..nb] in [0,1].
    Rectangle (i, j) = [s_i, s_i+1] x [t_j, t_j+1] gives triangles 2(i nb + j)
    and 2(i nb + j) + 1."""
    S, T = np.meshgrid(s, t, indexing="ij")
    na, nb = s.size - 1, t.size - 1
    verts = (np.asarray(origin, float)[None, None, :]
             + S[..., None] * np.asarray(ea, float)[None, None, :]
             + T[..., None] * np.asarray(eb, float)[None, None, :]).reshape(-1, 3)
    idx = np.arange((na + 1) * (nb + 1)).reshape(na + 1, nb + 1)
    v00 = idx[:-1, :-1].ravel()
    v10 = idx[1:, :-1].ravel()
    v01 = idx[:-1, 1:].ravel()
    v11 = idx[1:, 1:].ravel()
    t1 = np.stack([v00, v10, v11], axis=1)
    t2 = np.stack([v00, v11, v01], axis=1)
    tris = np.empty((2 * v00.size, 3), dtype=np.int64)
    tris[0::2] = t1
    tris[1::2] = t2
    return verts, tris


def _concat(parts):
    verts, tris, groups = [], [], []
    off = 0
    for g, (v, t) in enumerate(parts):
        verts.append(v)
        tris.append(t + off)
        groups.append(np.full(t.shape[0], g, dtype=np.int32))
        off += v.shape[0]
    return (np.concatenate(verts).astype(np.float64),
            np.concatenate(tris).astype(np.int32),
            np.concatenate(groups))


def shoebox_mesh(lx, ly, lz, nx, ny, nz):
    """Closed shoebox [0,lx]x[0,ly]x[0,lz]; nx,ny,nz rectangles per edge.

    Returns (verts[nv,3] f64, tris[nt,3] i32, wall[nt] i32) with
    nt = 4*(nx*ny + nx*nz + ny*nz).  Wall ids: 0 x=0, 1 x=lx, 2 y=0, 3 y=ly,
    4 z=0, 5 z=lz.  Outward normal = (v1-v0) x (v2-v0) direction.
    """
    X, Y, Z = np.eye(3)
    parts = [
        # x = 0, outward -x: ea x eb must be -x  -> ea = z, eb = y
        _grid_face([0, 0, 0], Z * lz, Y * ly, nz, ny),
        # x = lx, outward +x: ea = y, eb = z
        _grid_face([lx, 0, 0], Y * ly, Z * lz, ny, nz),
        # y = 0, outward -y: ea = x, eb = z
        _grid_face([0, 0, 0], X * lx, Z * lz, nx, nz),
        # y = ly, outward +y: ea = z, eb = x
        _grid_face([0, ly, 0], Z * lz, X * lx, nz, nx),
        # z = 0, outward -z: ea = y, eb = x
        _grid_face([0, 0, 0], Y * ly, X * lx, ny, nx),
        # z = lz, outward +z: ea = x, eb = y
        _grid_face([0, 0, lz], X * lx, Y * ly, nx, ny),
    ]
    return _concat(parts)


def shoebox_counts_for_h(lx, ly, lz, h):
    """Rectangle counts per edge for leg length at most h."""
    return tuple(max(1, int(math.ceil(L / h - 1e-9))) for L in (lx, ly, lz))


def _rect_wall(origin, ea, eb, ha, hb):
    na = max(1, int(math.ceil(np.linalg.norm(ea) / ha - 1e-9)))
    nb = max(1, int(math.ceil(np.linalg.norm(eb) / hb - 1e-9)))
    return _grid_face(origin, ea, eb, na, nb)


def lroom_mesh(h):
    """L-shaped room: box A=[0,5]x[0,4]x[0,3] joined to B=[5,8]x[0,3]x[0,3].

    The shared 3x3 m face at x=5, y in [0,3] is open.  All walls are meshed
    with legs <= h.  Wall ids are the part indices below.
    """
    X, Y, Z = np.eye(3)
    parts = [
        _rect_wall([0, 0, 0], Z * 3, Y * 4, h, h),            # x=0  (-x)
        _rect_wall([0, 0, 0], X * 8, Z * 3, h, h),            # y=0  (-y), both boxes
        _rect_wall([0, 4, 0], Z * 3, X * 5, h, h),            # y=4  (+y), box A
        _rect_wall([5, 3, 0], Z * 3, X * 3, h, h),            # y=3  (+y), box B
        _rect_wall([5, 3, 0], Y * 1, Z * 3, h, h),            # x=5, y in [3,4] (+x)
        _rect_wall([8, 0, 0], Y * 3, Z * 3, h, h),            # x=8  (+x)
        _rect_wall([0, 0, 0], Y * 4, X * 5, h, h),            # z=0 box A (-z)
        _rect_wall([5, 0, 0], Y * 3, X * 3, h, h),            # z=0 box B (-z)
        _rect_wall([0, 0, 3], X * 5, Y * 4, h, h),            # z=3 box A (+z)
        _rect_wall([5, 0, 3], X * 3, Y * 3, h, h),            # z=3 box B (+z)
    ]
    return _concat(parts)


def lroom_inside(p, margin=0.0):
    p = np.atleast_2d(p)
    inA = ((p[:, 0] > margin) & (p[:, 0] < 5 + margin) & (p[:, 1] > margin)
           & (p[:, 1] < 4 - margin) & (p[:, 2] > margin) & (p[:, 2] < 3 - margin))
    inB = ((p[:, 0] > 5 - margin) & (p[:, 0] < 8 - margin) & (p[:, 1] > margin)
           & (p[:, 1] < 3 - margin) & (p[:, 2] > margin) & (p[:, 2] < 3 - margin))
    return inA | inB


def _breaks(length, cuts, h):
    """Grid lines (as fractions of `length`) with every cut point a line and
    legs <= h between consecutive lines."""
    pts = [0.0] + sorted(cuts) + [float(length)]
    out = [0.0]
    for a, b in zip(pts[:-1], pts[1:]):
        n = max(1, int(math.ceil((b - a) / h - 1e-9)))
        out.extend(a + (b - a) * np.arange(1, n + 1) / n)
    out = np.asarray(out) / float(length)
    out[-1] = 1.0
    return out


# Room with a door and a free-standing baffle (the learned-preconditioner
# geometry of Sec. 4's scale): shoebox 5x4x3 m, door on the wall y = 0 at
# x in [0.5, 1.4], z in [0, 2.0]; baffle in the plane x = 2.5 over
# y in [1.0, 3.0], z in [0.5, 2.0].
BAFFLE_ROOM = (5.0, 4.0, 3.0)
DOOR_X = (0.5, 1.4)
DOOR_Z = (0.0, 2.0)
BAFFLE_X = 2.5
BAFFLE_Y = (1.0, 3.0)
BAFFLE_Z = (0.5, 2.0)
WALL_DOOR = 6
WALL_BAFFLE = 7


def baffle_room_mesh(h, thickness=0.02):
    """The door-and-baffle room meshed with legs <= h.

    thickness > 0 (the direct formulation, which needs a closed boundary):
    the baffle is a closed box of that thickness centred on its plane
    (x in 2.5 -/+ t/2), every normal pointing out of the air: out of the room
    on the walls, into the baffle's box on its six faces.
    thickness = 0 (the indirect formulation): the baffle is one sheet in the
    plane x = 2.5 with normal +x (its + side faces +x).
    The wall y = 0 has grid lines on the door's edges; its door rectangles
    get wall id 6, the baffle id 7, the walls ids 0..5 as in shoebox_mesh.
    Returns (verts f64, tris i32, wall i32)."""
    lx, ly, lz = BAFFLE_ROOM
    X, Y, Z = np.eye(3)
    parts, ids = [], []

    def add(vt, wid):
        parts.append(vt)
        ids.append(wid if np.ndim(wid) else np.full(vt[1].shape[0], wid, np.int32))

    add(_rect_wall([0, 0, 0], Z * lz, Y * ly, h, h), 0)
    add(_rect_wall([lx, 0, 0], Y * ly, Z * lz, h, h), 1)
    s = _breaks(lx, list(DOOR_X), h)
    t = _breaks(lz, [DOOR_Z[1]], h)
    v, tr = _grid_face_st([0, 0, 0], X * lx, Z * lz, s, t)
    sm = 0.5 * (s[:-1] + s[1:]) * lx
    tm = 0.5 * (t[:-1] + t[1:]) * lz
    door = ((sm[:, None] > DOOR_X[0]) & (sm[:, None] < DOOR_X[1])
            & (tm[None, :] > DOOR_Z[0]) & (tm[None, :] < DOOR_Z[1])).ravel()
    add((v, tr), np.where(np.repeat(door, 2), WALL_DOOR, 2).astype(np.int32))
    add(_rect_wall([0, ly, 0], Z * lz, X * lx, h, h), 3)
    add(_rect_wall([0, 0, 0], Y * ly, X * lx, h, h), 4)
    add(_rect_wall([0, 0, lz], X * lx, Y * ly, h, h), 5)
    x0, x1 = BAFFLE_X - 0.5 * thickness, BAFFLE_X + 0.5 * thickness
    wy, wz = BAFFLE_Y[1] - BAFFLE_Y[0], BAFFLE_Z[1] - BAFFLE_Z[0]
    y0, z0, z1 = BAFFLE_Y[0], BAFFLE_Z[0], BAFFLE_Z[1]
    y1 = BAFFLE_Y[1]
    faces = [
        ([x0, y0, z0], Y * wy, Z * wz),          # x = x0, normal +x (into the box)
        ([x1, y0, z0], Z * wz, Y * wy),          # x = x1, normal -x
        ([x0, y0, z0], Z * wz, X * thickness),   # y = y0, normal +y
        ([x0, y1, z0], X * thickness, Z * wz),   # y = y1, normal -y
        ([x0, y0, z0], X * thickness, Y * wy),   # z = z0, normal +z
        ([x0, y0, z1], Y * wy, X * thickness),   # z = z1, normal -z
    ]
    if thickness == 0:
        faces = faces[:1]
    for o, ea, eb in faces:
        add(_rect_wall(o, ea, eb, h, h), WALL_BAFFLE)
    verts, tris, _ = _concat(parts)
    return verts, tris, np.concatenate(ids).astype(np.int32)


def baffle_room_inside(p, margin=0.0, thickness=0.02):
    """Points of the air at least `margin` from the walls and the baffle."""
    p = np.atleast_2d(p)
    lx, ly, lz = BAFFLE_ROOM
    inroom = np.all((p > margin) & (p < np.array([lx, ly, lz]) - margin), axis=1)
    lo = np.array([BAFFLE_X - 0.5 * thickness, BAFFLE_Y[0], BAFFLE_Z[0]]) - margin
    hi = np.array([BAFFLE_X + 0.5 * thickness, BAFFLE_Y[1], BAFFLE_Z[1]]) + margin
    inbaffle = np.all((p > lo) & (p < hi), axis=1)
    return inroom & ~inbaffle


def baffle_workload(freq_hz=2000.0, per_wavelength=10.0, nsrc=8, nrec=64, wall_beta=0.2,
                    door_beta=1.0, baffle_beta=1.0, thickness=0.02, h=None, config_index=3):
    """Door-and-baffle room at one frequency: walls admittance 0.2, door and
    baffle 1.0, legs h = lambda/per_wavelength (or the given h), `nsrc`
    sources and `nrec` receivers seeded uniform in the air (>= 0.25 m from
    walls and baffle, receivers >= 0.1 m from sources)."""
    if h is None:
        h = SOUND_SPEED / freq_hz / per_wavelength
    verts, tris, wall = baffle_room_mesh(h, thickness)
    beta = np.full(tris.shape[0], complex(wall_beta), dtype=np.complex128)
    beta[wall == WALL_DOOR] = door_beta
    beta[wall == WALL_BAFFLE] = baffle_beta
    rng = seeded_rng(config_index)
    pts = []
    while len(pts) < nsrc + nrec:
        p = np.array(BAFFLE_ROOM) * rng.random(3)
        if not baffle_room_inside(p, 0.25, thickness)[0]:
            continue
        if len(pts) >= nsrc and np.min(np.linalg.norm(np.asarray(pts[:nsrc]) - p, axis=1)) < 0.1:
            continue
        pts.append(p)
    pts = np.asarray(pts)
    return Workload(f"baffle-room-5x4x3-{freq_hz:.0f}Hz-N{tris.shape[0]}", verts, tris, wall, float(freq_hz),
                    wavenumber(freq_hz), beta, pts[:nsrc], pts[nsrc:], room=BAFFLE_ROOM,
                    extra={"h": h, "thickness": thickness})


def cfg_baffle(nsrc=8, nrec=64):
    """The door-and-baffle room at 2 kHz, legs lambda/10 (N = 685,272)."""
    return baffle_workload(2000.0, 10.0, nsrc, nrec)


def cfg_baffle_sub(nsrc=4, nrec=16):
    """Small instance of the same geometry for dense parity: 250 Hz, legs
    0.25 m."""
    return baffle_workload(250.0, h=0.25, nsrc=nsrc, nrec=nrec)


def cfg_largest(nrec=1024):
    """Largest room: shoebox 6.5 x 5.5 x 4.2 m at 5 kHz, legs lambda/6
    (569 x 482 x 368 rectangles, N = 2,644,104), one admittance per wall
    drawn uniform in [0.05, 0.3], a seeded monopole and `nrec` receivers
    (>= 0.25 m from the walls, >= 0.1 m from the source)."""
    lx, ly, lz = 6.5, 5.5, 4.2
    h = SOUND_SPEED / 5000.0 / 6.0
    rng = seeded_rng(4)
    beta_wall = rng.uniform(0.05, 0.3, size=6)
    src = uniform_points_in_box(rng, [0, 0, 0], [lx, ly, lz], 1, 0.25)
    wl = shoebox_workload(f"shoebox-{lx}x{ly}x{lz}-5kHz", lx, ly, lz, shoebox_counts_for_h(lx, ly, lz, h),
                          5000.0, 0.0, src[0], nrec, 4, beta_per_wall=beta_wall)
    wl.name += f"-N{wl.n}"
    return wl


IR_ROOM = (8.0, 6.0, 3.0)       # the rectangular room of Sec. 4's image-source comparison
IR_SOURCE = (3.0, 2.0, 1.75)
IR_ZETA = 9.0                   # R = (zeta - 1)/(zeta + 1) = 0.8


def ir_receivers(spacing=0.25, margin=0.25, z=1.75, avoid=IR_SOURCE, avoid_dist=0.1):
    """Receiver grid in the source's horizontal plane (Sec. 4 images the
    plane z = 1.75 m), `margin` from the walls, none within `avoid_dist` of
    the source."""
    lx, ly, _ = IR_ROOM
    xs = np.arange(margin, lx - margin + 1e-9, spacing)
    ys = np.arange(margin, ly - margin + 1e-9, spacing)
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    P = np.stack([X.ravel(), Y.ravel(), np.full(X.size, z)], 1)
    keep = np.linalg.norm(P - np.asarray(avoid), axis=1) >= avoid_dist
    return P[keep]


def ir_sweep(f_max=640.0, df=10.0, per_wavelength=8.0, h_max=0.5):
    """Equispaced frequencies f_m = m df (m = 1..f_max/df) for the broadband
    response of the 8 x 6 x 3 m room (uniform zeta = 9, source at
    (3, 2, 1.75) m), each meshed with legs min(lambda/per_wavelength, h_max)."""
    out = []
    rec = ir_receivers()
    for m in range(1, int(round(f_max / df)) + 1):
        f = m * df
        h = min(SOUND_SPEED / f / per_wavelength, h_max)
        counts = shoebox_counts_for_h(*IR_ROOM, h)
        verts, tris, wall = shoebox_mesh(*IR_ROOM, *counts)
        beta = np.full(tris.shape[0], 1.0 / IR_ZETA, dtype=np.complex128)
        out.append(Workload(f"ir-room-8x6x3-{f:.0f}Hz-N{tris.shape[0]}", verts, tris, wall, f, wavenumber(f), beta,
                            np.asarray([IR_SOURCE], dtype=np.float64), rec, room=IR_ROOM))
    return out


def seeded_rng(config_index: int) -> np.random.Generator:
    """numpy PCG64 seeded with 2103_16073 + config index."""
    return np.random.Generator(np.random.PCG64(2103_16073 + int(config_index)))


def uniform_points_in_box(rng, lo, hi, n, margin, avoid=None, avoid_dist=0.0):
    lo = np.asarray(lo, float) + margin
    hi = np.asarray(hi, float) - margin
    out = []
    while len(out) < n:
        p = lo + (hi - lo) * rng.random(3)
        if avoid is not None and len(avoid):
            if np.min(np.linalg.norm(np.asarray(avoid) - p, axis=1)) < avoid_dist:
                continue
        out.append(p)
    return np.asarray(out, dtype=np.float64)


@dataclass
class Workload:
    """One synthetic room problem (geometry + frequency + sources)."""
    name: str
    verts: np.ndarray
    tris: np.ndarray
    wall: np.ndarray
    freq_hz: float
    k: float
    beta: np.ndarray            # complex admittance per element (beta = 1/zeta)
    sources: np.ndarray         # [ns,3]
    receivers: np.ndarray       # [nr,3]
    room: tuple = ()
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.tris.shape[0])


def shoebox_workload(name, lx, ly, lz, counts, freq_hz, beta, source, nrec,
                     config_index, beta_per_wall=None):
    verts, tris, wall = shoebox_mesh(lx, ly, lz, *counts)
    rng = seeded_rng(config_index)
    if beta_per_wall is not None:
        b = np.asarray(beta_per_wall, dtype=np.complex128)[wall]
    else:
        b = np.full(tris.shape[0], complex(beta), dtype=np.complex128)
    src = np.atleast_2d(np.asarray(source, dtype=np.float64))
    rec = uniform_points_in_box(rng, [0, 0, 0], [lx, ly, lz], nrec, 0.25,
                                avoid=src, avoid_dist=0.1)
    return Workload(name, verts, tris, wall, float(freq_hz), wavenumber(freq_hz),
                    b, src, rec, room=(lx, ly, lz))


def cfg_small(nrec=64):
    """Shoebox 3.0x2.4x2.0 m, 125 Hz, 16x16 rectangles per wall -> N=3,072,
    uniform admittance 0.2, monopole at (0.7,0.6,0.5) m."""
    return shoebox_workload("shoebox-3.0x2.4x2.0-125Hz-N3072", 3.0, 2.4, 2.0,
                            (16, 16, 16), 125.0, 0.2, (0.7, 0.6, 0.5), nrec, 0)


def cfg_1khz(nrec=64):
    """Same shoebox at 1 kHz, legs lambda/8 -> 70x56x47 rectangles, N=39,368."""
    return shoebox_workload("shoebox-3.0x2.4x2.0-1kHz-N39368", 3.0, 2.4, 2.0,
                            (70, 56, 47), 1000.0, 0.2, (0.7, 0.6, 0.5), nrec, 1)


def cfg_1khz_sub(nrec=64):
    """4k-element sub-instance of the 1 kHz shoebox: 22x18x15 -> N=3,984."""
    return shoebox_workload("shoebox-3.0x2.4x2.0-1kHz-N3984", 3.0, 2.4, 2.0,
                            (22, 18, 15), 1000.0, 0.2, (0.7, 0.6, 0.5), nrec, 1)


def cfg_high_order(nrec=8):
    """Coarse mesh at a high frequency: the 3.0 x 2.4 x 2.0 m shoebox with
    16 x 16 x 16 rectangles per edge (N = 3,072) at 7.5 kHz, so the
    expansion orders (116 on level 2, 66 on level 3) exceed what one
    shared-memory tile holds."""
    return shoebox_workload("shoebox-3.0x2.4x2.0-7.5kHz-N3072", 3.0, 2.4, 2.0, (16, 16, 16), 7500.0, 0.2,
                            (0.7, 0.6, 0.5), nrec, 0)


def exterior_source(room, dist=0.5):
    """A point at least `dist` outside the room's bounding box (for the
    exterior-source test: its field is regular inside the room)."""
    lx, ly, lz = room
    return np.array([lx + dist + 0.13, 0.37 * ly, 0.61 * lz], dtype=np.float64)


def sphere_mesh(radius, subdiv):
    """Icosphere: the icosahedron with every triangle split into 4, `subdiv`
    times, vertices pushed onto the sphere.  N = 20 * 4**subdiv; normals out."""
    t = (1.0 + 5 ** 0.5) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t),
         (0, -1, -t), (0, 1, -t), (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
         (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
         (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    verts = [np.array(p, float) / np.linalg.norm(p) for p in v]
    faces = list(f)
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
    V = np.asarray(verts) * radius
    T = np.asarray(faces, dtype=np.int64)
    # orient every triangle so that its right-hand normal points away from 0
    cen = V[T].mean(axis=1)
    nrm = np.cross(V[T[:, 1]] - V[T[:, 0]], V[T[:, 2]] - V[T[:, 0]])
    flip = np.sum(nrm * cen, axis=1) < 0
    T[flip] = T[flip][:, [0, 2, 1]]
    return V.astype(np.float64), T.astype(np.int32), np.zeros(T.shape[0], np.int32)


def paper_shoebox_counts(lx=8.0, ly=6.0, lz=3.0, max_edge=0.02):
    """Rectangle counts for the 8x6x3 m room of Sec. 4 meshed with maximum
    edge (the hypotenuse) `max_edge`: legs max_edge/sqrt(2)."""
    return shoebox_counts_for_h(lx, ly, lz, max_edge / math.sqrt(2.0))


def lroom_sweep(nfreq=64, f_lo=100.0, f_hi=2000.0, nsrc=8, per_wavelength=8, config_index=2):
    """Batching workload: the L-shaped room (5x4x3 m box joined to a 3x3x3 m
    box) at `nfreq` log-spaced frequencies, each meshed with legs
    lambda/per_wavelength (uneven N), one admittance per wall part drawn
    uniform in [0.05, 0.5], `nsrc` seeded interior sources per frequency
    (>= 0.3 m from every wall)."""
    rng = seeded_rng(config_index)
    beta_wall = rng.uniform(0.05, 0.5, size=10)
    out = []
    for f in np.geomspace(f_lo, f_hi, nfreq):
        h = SOUND_SPEED / f / per_wavelength
        verts, tris, wall = lroom_mesh(h)
        src = []
        while len(src) < nsrc:
            p = np.array([8.0, 4.0, 3.0]) * rng.random(3)
            if lroom_inside(p, 0.3)[0]:
                src.append(p)
        out.append(Workload(f"lroom-{f:.1f}Hz-N{tris.shape[0]}", verts, tris, wall, float(f), wavenumber(f),
                            beta_wall[wall].astype(np.complex128), np.asarray(src), np.zeros((0, 3)),
                            room=(8.0, 4.0, 3.0)))
    return out
