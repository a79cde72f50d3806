"""Seeded synthetic urban scenes (input data only; no propagation arithmetic).

The paper evaluates on a 2x2 km city model with hundreds of building blocks
and SUMO-generated vehicle trajectories (Sec. IV); neither is available, so
this module generates scenes with the same shapes: Manhattan grids of convex
extruded buildings, a flat ground, metal vehicle boxes moving along lanes
(moving objects are fixed-size metal boxes, Sec. V-A factor 2), pedestrians
on sidewalks and receivers mounted on vehicles.  A static base station is
assumed (Sec. III-C).

Both the CUDA path and the CPU oracle consume these arrays; this module holds
none of the method's arithmetic (no planes, normals, reflections or fields).

Conventions
-----------
* Coordinates are metres, centred on the scene origin, rounded once to
  float32.  z is up; the ground is the plane z = 0.
* Static faces are convex planar polygons (ground rectangle, building walls,
  roofs, bottoms).  Vertices are listed counter-clockwise seen from outside
  the solid.  ``face_off[f]:face_off[f+1]`` indexes ``face_xyz``.
* ``tri_xyz`` is a triangle mesh that covers every static face exactly
  (fan triangulation; the ground is tiled into a grid of triangle pairs),
  with ``tri_face`` giving the face of each triangle.
* Vehicle v is the axis-aligned box ``pos[v] - half[v] .. pos[v] + half[v]``
  (float32 arithmetic).  Its faces have global IDs ``F_s + 6 v + j`` with
  j = 0..5 for -x, +x, -y, +y, -z, +z.
* The material table always has 8 entries (ground, metal, concrete, glass,
  brick and three seeded concrete variants).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

# ---------------------------------------------------------------------------
# material table
# ---------------------------------------------------------------------------
MAT_GROUND, MAT_METAL, MAT_CONCRETE, MAT_GLASS, MAT_BRICK = 0, 1, 2, 3, 4
N_MATERIALS = 8
MATERIAL_NAMES = ["ground", "metal", "concrete", "glass", "brick",
                  "concrete_b", "concrete_c", "concrete_d"]


def material_table(seed: int = 1234):
    """Relative permittivity, conductivity (S/m) and the constant reflection
    coefficient used in constant-Gamma mode (Table I: walls 0.8, metal 0.9).

    Glass and brick conductivities are not given anywhere; fixed values are
    chosen here and used identically by every consumer."""
    eps = np.array([15.0, 1.0, 5.31, 6.27, 3.75, 0, 0, 0], np.float64)
    sig = np.array([0.035, 1.0e7, 0.0326, 0.004, 0.038, 0, 0, 0], np.float64)
    rng = np.random.default_rng(seed)
    eps[5:] = rng.uniform(4.5, 6.5, 3)
    sig[5:] = rng.uniform(0.02, 0.05, 3)
    gam = np.full(N_MATERIALS, 0.8)
    gam[MAT_METAL] = 0.9
    return eps, sig, gam


# ---------------------------------------------------------------------------
# data containers
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Frame:
    veh_pos: np.ndarray  # float32 [V,3] box centres
    veh_vel: np.ndarray  # float32 [V,3]
    rx_pos: np.ndarray   # float32 [R,3]
    rx_vel: np.ndarray   # float32 [R,3]
    tx_pos: np.ndarray   # float32 [X,3]
    tx_vel: np.ndarray   # float32 [X,3]


@dataclasses.dataclass
class Scene:
    name: str
    face_off: np.ndarray    # uint32 [F_s+1]
    face_xyz: np.ndarray    # float32 [NV,3]
    face_mat: np.ndarray    # uint32 [F_s]
    tri_xyz: np.ndarray     # float32 [T,3,3]
    tri_face: np.ndarray    # uint32 [T]
    veh_half: np.ndarray    # float32 [V,3]
    veh_mat: int
    eps_r: np.ndarray       # float64 [8]
    sigma: np.ndarray       # float64 [8]
    gamma: np.ndarray       # float64 [8]
    n_rays: int
    max_depth: int
    freqs: List[float]
    tx_power_w: float
    dt: float
    n_frames: int
    # motion description (frame k is a pure function of these)
    lanes: Optional[dict] = None
    static_frame: Optional[Frame] = None

    @property
    def n_static_faces(self) -> int:
        return int(self.face_mat.shape[0])

    @property
    def n_vehicles(self) -> int:
        return int(self.veh_half.shape[0])

    @property
    def n_faces(self) -> int:
        return self.n_static_faces + 6 * self.n_vehicles

    def frame(self, k: int = 0) -> Frame:
        if self.lanes is None:
            return self.static_frame
        return _motion_frame(self.lanes, k * self.dt)


# ---------------------------------------------------------------------------
# geometry builders
# ---------------------------------------------------------------------------
class _FaceBuilder:
    def __init__(self):
        self.off = [0]
        self.xyz: List[np.ndarray] = []
        self.mat: List[int] = []
        self.tris: List[np.ndarray] = []
        self.tri_face: List[int] = []

    def add(self, poly, mat, tris=None):
        poly = np.asarray(poly, np.float32)
        f = len(self.mat)
        self.xyz.append(poly)
        self.off.append(self.off[-1] + len(poly))
        self.mat.append(mat)
        if tris is None:  # fan triangulation of a convex polygon
            tris = [np.stack([poly[0], poly[i], poly[i + 1]])
                    for i in range(1, len(poly) - 1)]
        for t in tris:
            self.tris.append(np.asarray(t, np.float32))
            self.tri_face.append(f)
        return f

    def add_ground(self, x0, x1, y0, y1, tiles):
        xs = np.linspace(x0, x1, tiles + 1).astype(np.float32)
        ys = np.linspace(y0, y1, tiles + 1).astype(np.float32)
        xs[0], xs[-1], ys[0], ys[-1] = x0, x1, y0, y1
        tris = []
        for i in range(tiles):
            for j in range(tiles):
                a = (xs[i], ys[j], 0.0)
                b = (xs[i + 1], ys[j], 0.0)
                c = (xs[i + 1], ys[j + 1], 0.0)
                d = (xs[i], ys[j + 1], 0.0)
                tris.append((a, b, c))
                tris.append((a, c, d))
        poly = [(x0, y0, 0.0), (x1, y0, 0.0), (x1, y1, 0.0), (x0, y1, 0.0)]
        return self.add(poly, MAT_GROUND, tris)

    def add_prism(self, foot_xy, height, mat):
        """Convex prism from a CCW (seen from +z) footprint: walls, roof and
        bottom faces."""
        foot = np.asarray(foot_xy, np.float32)
        h = np.float32(height)
        n = len(foot)
        for i in range(n):
            a, b = foot[i], foot[(i + 1) % n]
            self.add([(a[0], a[1], 0.0), (b[0], b[1], 0.0),
                      (b[0], b[1], h), (a[0], a[1], h)], mat)
        self.add([(p[0], p[1], h) for p in foot], mat)             # roof
        self.add([(p[0], p[1], 0.0) for p in foot[::-1]], mat)     # bottom

    def arrays(self):
        return (np.asarray(self.off, np.uint32),
                np.concatenate(self.xyz).astype(np.float32),
                np.asarray(self.mat, np.uint32),
                np.stack(self.tris).astype(np.float32),
                np.asarray(self.tri_face, np.uint32))


def _hull_ccw(pts):
    """Monotone-chain convex hull, CCW, collinear points dropped."""
    pts = sorted(set(map(tuple, pts)))

    def cross(o, a, b):
        return (a[0] - o[0]) * (b[1] - o[1]) - (a[1] - o[1]) * (b[0] - o[0])

    lower, upper = [], []
    for p in pts:
        while len(lower) >= 2 and cross(lower[-2], lower[-1], p) <= 0:
            lower.pop()
        lower.append(p)
    for p in reversed(pts):
        while len(upper) >= 2 and cross(upper[-2], upper[-1], p) <= 0:
            upper.pop()
        upper.append(p)
    return lower[:-1] + upper[:-1]


def _random_footprint(rng, cx, cy, half, n_lo=12, n_hi=17):
    """Random convex polygon (about n vertices) inside the square
    [cx-half, cx+half] x [cy-half, cy+half]; float32 vertices, CCW."""
    for _ in range(100):
        n = int(rng.integers(n_lo, n_hi + 1))
        ang = np.sort(rng.uniform(0, 2 * np.pi, n))
        a, b = rng.uniform(0.65, 1.0, 2) * half
        rot = rng.uniform(0, np.pi)
        r = rng.uniform(0.97, 1.0, n)
        x = a * r * np.cos(ang)
        y = b * r * np.sin(ang)
        xr = x * np.cos(rot) - y * np.sin(rot)
        yr = x * np.sin(rot) + y * np.cos(rot)
        s = max(np.abs(xr).max(), np.abs(yr).max()) / half
        if s > 1:
            xr, yr = xr / s, yr / s
        pts = np.stack([cx + xr, cy + yr], 1).astype(np.float32)
        hull = np.asarray(_hull_ccw(pts), np.float32)
        # drop nearly collinear vertices and very short edges
        keep = []
        m = len(hull)
        for i in range(m):
            p0, p1, p2 = hull[i - 1], hull[i], hull[(i + 1) % m]
            e0 = (p1 - p0).astype(np.float64)
            e1 = (p2 - p1).astype(np.float64)
            c = e0[0] * e1[1] - e0[1] * e1[0]
            if c > 0.02 * np.linalg.norm(e0) * np.linalg.norm(e1) and \
                    np.linalg.norm(e1) > 0.3:
                keep.append(p1)
        if len(keep) >= 4:
            return np.asarray(_hull_ccw(np.asarray(keep)), np.float32)
    raise RuntimeError("footprint generation failed")


def _box_footprint(x0, y0, x1, y1):
    return np.array([(x0, y0), (x1, y0), (x1, y1), (x0, y1)], np.float32)


# ---------------------------------------------------------------------------
# motion (vehicles on lanes, pedestrians on sidewalks; periodic wrap)
# ---------------------------------------------------------------------------
def _motion_frame(L: dict, t: float) -> Frame:
    """Positions at time t, computed in float64 and rounded once."""
    def along(s0, speed, length):
        return np.mod(s0 + speed * t, length)

    # vehicles
    s = along(L["veh_s0"], L["veh_speed"], L["veh_len"])
    p = L["veh_start"] + s[:, None] * L["veh_dir"]
    veh_pos = p.astype(np.float32)
    veh_vel = (L["veh_speed"][:, None] * L["veh_dir"]).astype(np.float32)
    # receivers on vehicles
    rv = L["rxv_veh"]
    rx_v = p[rv] + L["rxv_off"][:, None] * L["veh_dir"][rv]
    rx_v[:, 2] = L["rxv_z"]
    vel_v = veh_vel[rv]
    # pedestrians
    sp = along(L["ped_s0"], L["ped_speed"], L["ped_len"])
    rx_p = L["ped_start"] + sp[:, None] * L["ped_dir"]
    vel_p = L["ped_speed"][:, None] * L["ped_dir"]
    rx_pos = np.concatenate([rx_v, rx_p]).astype(np.float32)
    rx_vel = np.concatenate([vel_v, vel_p]).astype(np.float32)
    return Frame(veh_pos, veh_vel, rx_pos, rx_vel,
                 L["tx_pos"].astype(np.float32),
                 np.zeros_like(L["tx_pos"], dtype=np.float32))


def _grid_city(name, rng, blocks, pitch, block_size, n_veh, n_rx_veh, n_ped,
               tx_mode, n_tx, mats, ground_tile, n_rays, depth, freqs,
               n_frames, dt, veh_size=(4.5, 1.8, 1.5), lot_split=2,
               setback=1.0, tiny_height=None):
    half_w = blocks * pitch / 2.0
    fb = _FaceBuilder()
    fb.add_ground(-half_w, half_w, -half_w, half_w,
                  max(1, int(round(2 * half_w / ground_tile))))
    street = pitch - block_size
    lot = block_size / lot_split
    buildings = []  # (centroid xy, footprint, height)
    for bi in range(blocks):
        for bj in range(blocks):
            bx0 = -half_w + bi * pitch + street / 2
            by0 = -half_w + bj * pitch + street / 2
            for li in range(lot_split):
                for lj in range(lot_split):
                    cx = bx0 + (li + 0.5) * lot
                    cy = by0 + (lj + 0.5) * lot
                    foot = _random_footprint(rng, cx, cy, lot / 2 - setback)
                    h = float(np.clip(20.0 * np.exp(0.5 * rng.normal()),
                                      5.0, 120.0))
                    buildings.append([foot, h, int(rng.choice(mats))])
    # transmitters
    if tx_mode == "rooftop":
        idx = rng.choice(len(buildings), n_tx, replace=False)
        tx = []
        for k in idx:
            buildings[k][1] = 28.0
            c = buildings[k][0].astype(np.float64).mean(0)
            tx.append((c[0], c[1], 30.0))
        tx = np.asarray(tx)
    else:  # street intersections
        lines = -half_w + pitch * np.arange(1, blocks)
        tx = []
        used = set()
        while len(tx) < n_tx:
            i, j = rng.integers(0, len(lines), 2)
            if (i, j) in used:
                continue
            used.add((i, j))
            tx.append((lines[i], lines[j], rng.uniform(25.0, 40.0)))
        tx = np.asarray(tx)
    for foot, h, m in buildings:
        fb.add_prism(foot, h, m)
    off, xyz, fmat, tris, tface = fb.arrays()

    # lanes: street centrelines between blocks, both axes
    lines = -half_w + pitch * np.arange(1, blocks)
    lane_off = np.array([-7.5, -2.5, 2.5, 7.5])
    lane_dirsign = np.array([-1.0, -1.0, 1.0, 1.0])
    L_len = 2 * half_w
    vs0, vsp, vstart, vdir, vhalf = [], [], [], [], []
    hx, hy, hz = (np.float32(v / 2) for v in veh_size)
    for v in range(n_veh):
        axis = int(rng.integers(0, 2))
        line = lines[int(rng.integers(0, len(lines)))]
        k = int(rng.integers(0, 4))
        sgn = lane_dirsign[k]
        d = np.zeros(3)
        d[axis] = sgn
        start = np.zeros(3)
        start[axis] = -half_w if sgn > 0 else half_w
        start[1 - axis] = line + lane_off[k]
        start[2] = float(hz)
        vstart.append(start)
        vdir.append(d)
        vs0.append(rng.uniform(0, L_len))
        vsp.append(rng.uniform(5.0, 15.0))
        vhalf.append((hx, hy, hz) if axis == 0 else (hy, hx, hz))
    # receivers on vehicles: Rx j on vehicle j mod V, roof offsets 0, -1.5, +1.5
    rxv_veh = np.arange(n_rx_veh) % max(n_veh, 1)
    rxv_off = np.array([0.0, -1.5, 1.5])[(np.arange(n_rx_veh) // max(n_veh, 1)) % 3]
    rxv_z = 2 * float(hz) + 0.1
    # pedestrians on sidewalks (1 m from block edges), 1.5 m height
    ps0, psp, pstart, pdir = [], [], [], []
    for _ in range(n_ped):
        axis = int(rng.integers(0, 2))
        line = lines[int(rng.integers(0, len(lines)))]
        side = rng.choice([-1.0, 1.0]) * (street / 2 - 1.0)
        sgn = rng.choice([-1.0, 1.0])
        d = np.zeros(3)
        d[axis] = sgn
        start = np.zeros(3)
        start[axis] = -half_w if sgn > 0 else half_w
        start[1 - axis] = line + side
        start[2] = 1.5
        pstart.append(start)
        pdir.append(d)
        ps0.append(rng.uniform(0, L_len))
        psp.append(rng.uniform(1.0, 1.5))
    lanes = dict(
        veh_s0=np.asarray(vs0, np.float64), veh_speed=np.asarray(vsp, np.float64),
        veh_start=np.asarray(vstart, np.float64).reshape(-1, 3),
        veh_dir=np.asarray(vdir, np.float64).reshape(-1, 3),
        veh_len=L_len, rxv_veh=rxv_veh, rxv_off=rxv_off, rxv_z=rxv_z,
        ped_s0=np.asarray(ps0, np.float64), ped_speed=np.asarray(psp, np.float64),
        ped_start=np.asarray(pstart, np.float64).reshape(-1, 3),
        ped_dir=np.asarray(pdir, np.float64).reshape(-1, 3), ped_len=L_len,
        tx_pos=tx)
    eps, sig, gam = material_table()
    return Scene(name=name, face_off=off, face_xyz=xyz, face_mat=fmat,
                 tri_xyz=tris, tri_face=tface,
                 veh_half=np.asarray(vhalf, np.float32).reshape(-1, 3),
                 veh_mat=MAT_METAL, eps_r=eps, sigma=sig, gamma=gam,
                 n_rays=n_rays, max_depth=depth, freqs=list(freqs),
                 tx_power_w=100.0, dt=dt, n_frames=n_frames, lanes=lanes)


# ---------------------------------------------------------------------------
# the five workloads
# ---------------------------------------------------------------------------
def toy_scene(seed: int = 0, n_rays: int = 100_000, depth: int = 2) -> Scene:
    """Static toy scene: 200x200 m ground (2 triangles), 20 concrete box
    buildings (footprints 10-30 m, heights 8-40 m, 12 triangles each), one
    transmitter at (0, 0, 10) m, 16 receivers at 1.5 m, 3.5 GHz."""
    rng = np.random.default_rng(seed)
    fb = _FaceBuilder()
    fb.add_ground(-100.0, 100.0, -100.0, 100.0, 1)
    tx = np.array([[0.0, 0.0, 10.0]])
    boxes = []
    while len(boxes) < 20:
        w, d = rng.uniform(10, 30, 2)
        cx = rng.uniform(-100 + w / 2, 100 - w / 2)
        cy = rng.uniform(-100 + d / 2, 100 - d / 2)
        b = (cx - w / 2, cy - d / 2, cx + w / 2, cy + d / 2)
        if b[0] - 1 <= 0 <= b[2] + 1 and b[1] - 1 <= 0 <= b[3] + 1:
            continue
        if any(b[0] < o[2] + 2 and o[0] < b[2] + 2 and b[1] < o[3] + 2
               and o[1] < b[3] + 2 for o in boxes):
            continue
        boxes.append(b)
    for b in boxes:
        fb.add_prism(_box_footprint(*b), rng.uniform(8, 40), MAT_CONCRETE)
    rx = []
    while len(rx) < 16:
        x, y = rng.uniform(-99, 99, 2)
        if any(o[0] - 1 <= x <= o[2] + 1 and o[1] - 1 <= y <= o[3] + 1
               for o in boxes):
            continue
        rx.append((x, y, 1.5))
    off, xyz, fmat, tris, tface = fb.arrays()
    eps, sig, gam = material_table()
    fr = Frame(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32),
               np.asarray(rx, np.float32), np.zeros((16, 3), np.float32),
               tx.astype(np.float32), np.zeros((1, 3), np.float32))
    return Scene(name="toy", face_off=off, face_xyz=xyz, face_mat=fmat,
                 tri_xyz=tris, tri_face=tface,
                 veh_half=np.zeros((0, 3), np.float32), veh_mat=MAT_METAL,
                 eps_r=eps, sigma=sig, gamma=gam, n_rays=n_rays,
                 max_depth=depth, freqs=[3.5e9], tx_power_w=100.0, dt=0.1,
                 n_frames=1, static_frame=fr)


def tiny_scene(seed: int = 0, n_rays: int = 200_000, depth: int = 3) -> Scene:
    """Random tiny scene for property tests: 60x60 m ground, 2-4 concrete box
    buildings (6 faces each, at most 25 static faces in all), 0-2 metal
    vehicle boxes, 1-2 transmitters and 6 receivers placed outside the
    buildings, K = 3, 3.5 GHz."""
    rng = np.random.default_rng([seed, 777])
    fb = _FaceBuilder()
    fb.add_ground(-30.0, 30.0, -30.0, 30.0, 1)
    boxes = []
    n_b = int(rng.integers(2, 5))
    while len(boxes) < n_b:
        w, d = rng.uniform(5, 15, 2)
        cx, cy = rng.uniform(-22, 22, 2)
        b = (cx - w / 2, cy - d / 2, cx + w / 2, cy + d / 2)
        if any(b[0] < o[2] + 2 and o[0] < b[2] + 2 and b[1] < o[3] + 2
               and o[1] < b[3] + 2 for o in boxes):
            continue
        boxes.append(b)
    for b in boxes:
        fb.add_prism(_box_footprint(*b), rng.uniform(5, 20), MAT_CONCRETE)

    def outside(x, y, m=1.0):
        return not any(o[0] - m <= x <= o[2] + m and o[1] - m <= y <= o[3] + m for o in boxes)

    def free_points(n, z_lo, z_hi):
        pts = []
        while len(pts) < n:
            x, y = rng.uniform(-28, 28, 2)
            if outside(x, y, 3.0):
                pts.append((x, y, rng.uniform(z_lo, z_hi)))
        return np.asarray(pts, np.float32)

    tx = free_points(int(rng.integers(1, 3)), 4.0, 15.0)
    rx = free_points(6, 1.0, 3.0)
    vpos = free_points(int(rng.integers(0, 3)), 0.75, 0.75)
    off, xyz, fmat, tris, tface = fb.arrays()
    eps, sig, gam = material_table()
    z = lambda n: np.zeros((n, 3), np.float32)
    fr = Frame(vpos, z(len(vpos)), rx, z(len(rx)), tx, z(len(tx)))
    return Scene(name=f"tiny{seed}", face_off=off, face_xyz=xyz, face_mat=fmat,
                 tri_xyz=tris, tri_face=tface,
                 veh_half=np.tile(np.float32([[2.25, 0.9, 0.75]]), (len(vpos), 1)),
                 veh_mat=MAT_METAL, eps_r=eps, sigma=sig, gamma=gam, n_rays=n_rays,
                 max_depth=depth, freqs=[3.5e9], tx_power_w=1.0, dt=0.1,
                 n_frames=1, static_frame=fr)


def district_scene(seed: int = 0, n_rays: int = 1_000_000, depth: int = 3,
                   n_veh: int = 200, n_rx: int = 1000) -> Scene:
    """500x500 m grid, 400 convex extruded buildings (~20k triangles),
    200 metal vehicles at 5-15 m/s, 1000 receivers (half vehicle-mounted),
    2 rooftop transmitters at 30 m, 3.5 GHz, 100 frames at 10 Hz."""
    rng = np.random.default_rng(seed)
    return _grid_city("district", rng, blocks=10, pitch=50.0, block_size=30.0,
                      n_veh=n_veh, n_rx_veh=n_rx // 2, n_ped=n_rx - n_rx // 2,
                      tx_mode="rooftop", n_tx=2, mats=[2, 3, 4, 5, 6, 7],
                      ground_tile=25.0, n_rays=n_rays, depth=depth,
                      freqs=[3.5e9], n_frames=100, dt=0.1)


def city_scene(seed: int = 0, n_rays: int = 10_000_000, depth: int = 4,
               n_veh: int = 5000, n_rx: int = 10_000, blocks: int = 40) -> Scene:
    """2x2 km grid, 6400 buildings (~300k triangles; concrete, glass, brick),
    5000 metal vehicles, 10k receivers (5000 vehicle-mounted, 5000
    pedestrians), 4 transmitters at 25-40 m above street intersections,
    3.5 and 28 GHz, 300 frames at 10 Hz."""
    rng = np.random.default_rng(seed)
    return _grid_city("city", rng, blocks=blocks, pitch=50.0, block_size=30.0,
                      n_veh=n_veh, n_rx_veh=n_rx // 2, n_ped=n_rx - n_rx // 2,
                      tx_mode="intersection", n_tx=4, mats=[2, 3, 4],
                      ground_tile=50.0, n_rays=n_rays, depth=depth,
                      freqs=[3.5e9, 28e9], n_frames=300, dt=0.1)


def batched_scenes(seed: int = 0, n: int = 64) -> List[Scene]:
    """Uneven batch: 50-2000 buildings, 0-500 vehicles, 16-4000 receivers,
    1-4 transmitters, 2-4 reflections, 1e5-4e6 rays (log-uniform)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        nb = int(np.exp(rng.uniform(np.log(50), np.log(2000))))
        blocks = max(4, int(round(math.sqrt(nb / 4))))
        nveh = int(np.exp(rng.uniform(0, np.log(501)))) - 1
        nrx = int(np.exp(rng.uniform(np.log(16), np.log(4000))))
        ntx = int(rng.integers(1, 5))
        k = int(rng.integers(2, 5))
        nr = int(np.exp(rng.uniform(np.log(1e5), np.log(4e6))))
        s = _grid_city(f"batch{i}", np.random.default_rng([seed, i]),
                       blocks=blocks, pitch=50.0, block_size=30.0,
                       n_veh=nveh, n_rx_veh=min(nrx // 2, 3 * nveh),
                       n_ped=nrx - min(nrx // 2, 3 * nveh),
                       tx_mode="intersection", n_tx=ntx, mats=[2, 3, 4],
                       ground_tile=50.0, n_rays=nr, depth=k, freqs=[3.5e9],
                       n_frames=1, dt=0.1)
        out.append(s)
    return out


# ---------------------------------------------------------------------------
# small hand-built scenes used by the closed-form checks
# ---------------------------------------------------------------------------
def custom_scene(polys, mats, tx, rx, tx_vel=None, rx_vel=None,
                 boxes=None, box_vel=None, n_rays=100_000, depth=2,
                 freq=3.5e9) -> Scene:
    """Scene from explicit convex polygons (each CCW seen from the side the
    rays come from) and optional axis-aligned vehicle boxes (lo, hi)."""
    fb = _FaceBuilder()
    for p, m in zip(polys, mats):
        fb.add(p, m)
    if polys:
        off, xyz, fmat, tris, tface = fb.arrays()
    else:
        off = np.zeros(1, np.uint32)
        xyz = np.zeros((0, 3), np.float32)
        fmat = np.zeros(0, np.uint32)
        tris = np.zeros((0, 3, 3), np.float32)
        tface = np.zeros(0, np.uint32)
    boxes = [] if boxes is None else boxes
    half = np.array([(np.asarray(h, np.float64) - np.asarray(l)) / 2
                     for l, h in boxes], np.float32).reshape(-1, 3)
    pos = np.array([(np.asarray(h, np.float64) + np.asarray(l)) / 2
                    for l, h in boxes], np.float32).reshape(-1, 3)
    tx = np.asarray(tx, np.float32).reshape(-1, 3)
    rx = np.asarray(rx, np.float32).reshape(-1, 3)
    z = lambda a, n: (np.zeros((n, 3), np.float32) if a is None
                      else np.asarray(a, np.float32).reshape(n, 3))
    fr = Frame(pos, z(box_vel, len(boxes)), rx, z(rx_vel, len(rx)),
               tx, z(tx_vel, len(tx)))
    eps, sig, gam = material_table()
    return Scene(name="custom", face_off=off, face_xyz=xyz, face_mat=fmat,
                 tri_xyz=tris, tri_face=tface, veh_half=half,
                 veh_mat=MAT_METAL, eps_r=eps, sigma=sig, gamma=gam,
                 n_rays=n_rays, max_depth=depth, freqs=[freq],
                 tx_power_w=1.0, dt=0.1, n_frames=1, static_frame=fr)


def rect_xy(x0, y0, x1, y1, z=0.0, up=True):
    """Horizontal rectangle at height z, CCW seen from +z (up) or -z."""
    p = [(x0, y0, z), (x1, y0, z), (x1, y1, z), (x0, y1, z)]
    return p if up else p[::-1]


def rect_wall_x(x, y0, y1, z0, z1, facing=-1):
    """Vertical rectangle in the plane x = const, facing -x or +x."""
    p = [(x, y0, z0), (x, y0, z1), (x, y1, z1), (x, y1, z0)]
    return p if facing < 0 else p[::-1]
