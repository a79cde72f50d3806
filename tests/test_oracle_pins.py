"""Pins of the CPU oracle against results fixed by the paper and by
mathematics (no GPU).  Each test would fail under a plausible slip in the
oracle: a dropped term, a swapped polarisation, a wrong sign or index."""
import dataclasses
import math
import os

import numpy as np
import pytest

import oracle
from paper_2303_10521_gb300 import scenes as S

C = 299792458.0
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _lam(f):
    return C / f


def _one(tx, rx, polys=(), mats=(), boxes=None, box_vel=None, tx_vel=None,
         rx_vel=None, freq=3.5e9, const_gamma=False, eps=None, sig=None):
    sc = S.custom_scene(list(polys), list(mats), tx, rx, tx_vel=tx_vel,
                        rx_vel=rx_vel, boxes=boxes, box_vel=box_vel, freq=freq)
    o = oracle.OracleScene(sc, sc.frame(0), const_gamma=const_gamma,
                           eps_r=eps, sigma=sig)
    return sc, o


def _path(tx, rx, faces):
    p = np.zeros(1, oracle.PATH_DTYPE)
    p["tx"], p["rx"], p["depth"] = tx, rx, len(faces)
    p["face"][0] = [*faces, *([oracle.NO_FACE] * (4 - len(faces)))]
    return p


# ---------------------------------------------------------------------------
# ray set and reception radius
# ---------------------------------------------------------------------------
def test_ray_directions_unit_and_equal_area():
    n = 4096
    d = np.array([oracle.ray_dir(n, i) for i in range(n)], np.float64)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=2e-7)
    # Fibonacci sphere: z levels are the centres of N equal-area bands
    assert np.allclose(d[:, 2], 1 - (2 * np.arange(n) + 1) / n, atol=1e-7)
    assert np.linalg.norm(d.mean(0)) < 2e-3
    # consecutive azimuths advance by the golden angle
    phi = np.arctan2(d[:, 1], d[:, 0])
    step = np.mod(np.diff(phi), 2 * np.pi)
    assert np.allclose(step, np.pi * (3 - math.sqrt(5)), atol=1e-5)


@pytest.mark.parametrize("n", [2000, 20000])
def test_reception_radius_covers_every_direction(n):
    """Any direction has a ray within the reception angle r(L)/L, so a
    receiver on a specular path is inside the sphere of a nearby ray."""
    scipy_spatial = pytest.importorskip("scipy.spatial")
    d = np.array([oracle.ray_dir(n, i) for i in range(n)], np.float64)
    tree = scipy_spatial.cKDTree(d)
    rng = np.random.default_rng(0)
    q = rng.normal(size=(400_000, 3))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    # densify the polar caps where the lattice is least regular
    kap = oracle.radius_factor(n)
    cap = np.concatenate([rng.normal(size=(100_000, 2)) * 6 * kap,
                          np.ones((100_000, 1))], 1)
    cap /= np.linalg.norm(cap, axis=1, keepdims=True)
    cap[::2, 2] *= -1
    dist, _ = tree.query(np.concatenate([q, cap]))
    ang = 2 * np.arcsin(dist / 2)
    assert ang.max() <= oracle.radius_factor(n)
    # and the radius is not needlessly large (hexagonal bound times 1.25)
    assert oracle.radius_factor(n) == pytest.approx(
        1.25 * math.sqrt(8 * math.pi / (3 * math.sqrt(3) * n)), rel=1e-12)


# ---------------------------------------------------------------------------
# Fresnel coefficients
# ---------------------------------------------------------------------------
def test_fresnel_normal_incidence():
    for eps in (5.31 - 0.17j, 15.0, 2.25 - 1j):
        gs, gp = oracle.fresnel(eps, 1.0)
        n = np.sqrt(eps)
        assert gs == pytest.approx((1 - n) / (1 + n), abs=1e-14)
        # with p vectors defined as s x k the two agree up to sign at theta=0
        assert gp == pytest.approx(-gs, abs=1e-14)


def test_fresnel_brewster_and_grazing():
    for er in (2.0, 5.31, 15.0):
        tb = math.atan(math.sqrt(er))
        gs, gp = oracle.fresnel(complex(er, 0.0), math.cos(tb))
        assert abs(gp) < 1e-13
        assert abs(gs) > 0.1
        gs, gp = oracle.fresnel(complex(er, -0.3), 1e-9)
        assert gs == pytest.approx(-1, abs=1e-7)
        assert gp == pytest.approx(-1, abs=1e-6)


def test_fresnel_perfect_conductor_limit():
    f = 3.5e9
    eps = complex(1.0, -1e7 / (2 * math.pi * f * 8.8541878128e-12))
    for ct in (1.0, 0.5, 0.1):
        gs, gp = oracle.fresnel(eps, ct)
        assert abs(gs + 1) < 1e-3 and abs(gp - 1) < 1e-3 / ct


def test_fresnel_lossless_energy():
    # |Gamma| = 1 beyond the critical angle cannot occur from air; below it
    # a lossless dielectric conserves energy: |G|^2 + transmittance = 1
    er = 5.31
    for ct in np.linspace(0.05, 1, 7):
        st2 = 1 - ct * ct
        ct_t = math.sqrt(er - st2) / math.sqrt(er)
        n = math.sqrt(er)
        ts = 2 * ct / (ct + n * ct_t)
        gs, gp = oracle.fresnel(complex(er, 0), ct)
        assert abs(gs) ** 2 + (n * ct_t / ct) * ts ** 2 == pytest.approx(1, abs=1e-12)


# ---------------------------------------------------------------------------
# closed-form propagation
# ---------------------------------------------------------------------------
def test_friis_free_space():
    f = 3.5e9
    tx, rx = (1.0, -2.0, 10.0), (401.25, 37.5, 1.5)
    sc, o = _one(tx, rx, freq=f)
    paths = oracle.enumerate_paths(o, 2)
    assert len(paths) == 1 and paths["depth"][0] == 0
    a, tau, fd = oracle.field(o, paths, f)
    d = np.linalg.norm(np.float32(rx).astype(float) - np.float32(tx).astype(float))
    k = 2 * math.pi * f / C
    expect = _lam(f) / (4 * math.pi * d) * np.exp(-1j * k * d)
    assert abs(a[0] - expect) <= 1e-10 * abs(expect)  # k d ~ 3e4 rad in FP64
    assert tau[0] == pytest.approx(d / C, rel=1e-15)
    # received power ratio (lambda / 4 pi d)^2
    assert abs(a[0]) ** 2 == pytest.approx((_lam(f) / (4 * math.pi * d)) ** 2, rel=1e-12)


@pytest.mark.parametrize("D,ht,hr", [(50.0, 10.0, 1.5), (300.0, 30.0, 1.6), (20.0, 5.0, 5.0)])
def test_two_ray_ground(D, ht, hr):
    f = 3.5e9
    D, ht, hr = (float(np.float32(v)) for v in (D, ht, hr))  # scene inputs are float32
    ground = S.rect_xy(-1e4, -1e4, 1e4, 1e4, 0.0)
    eps, sig = np.array(S.material_table()[0]), np.array(S.material_table()[1])
    sc, o = _one((0, 0, ht), (D, 0, hr), [ground], [S.MAT_GROUND], freq=f)
    paths = oracle.enumerate_paths(o, 2)
    assert sorted(paths["depth"].tolist()) == [0, 1]
    a, tau, _ = oracle.field(o, paths, f)
    d1 = math.hypot(D, ht - hr)
    d2 = math.hypot(D, ht + hr)
    ct = (ht + hr) / d2
    ec = complex(eps[S.MAT_GROUND], -sig[S.MAT_GROUND] / (2 * math.pi * f * 8.8541878128e-12))
    root = np.sqrt(ec - (1 - ct * ct))
    gp = (ec * ct - root) / (ec * ct + root)
    k = 2 * math.pi * f / C
    h = _lam(f) / (4 * math.pi) * (np.exp(-1j * k * d1) / d1 + gp * np.exp(-1j * k * d2) / d2)
    assert abs(a.sum() - h) <= 1e-10 * abs(h) + 1e-15
    assert sorted(tau * C) == pytest.approx([d1, d2], rel=1e-13)


def test_brewster_ground_reflection_vanishes():
    """Lossless ground and a geometry at the Brewster angle: the vertically
    polarised ground bounce carries no field."""
    er = 4.0
    eps, sig = S.material_table()[:2]
    eps = eps.copy(); sig = sig.copy()
    eps[S.MAT_GROUND], sig[S.MAT_GROUND] = er, 0.0
    ht = hr = 10.0
    D = (ht + hr) * math.sqrt(er)      # tan(theta) = D / (ht + hr)
    ground = S.rect_xy(-1e3, -1e3, 1e3, 1e3, 0.0)
    sc, o = _one((0, 0, ht), (D, 0, hr), [ground], [S.MAT_GROUND], eps=eps, sig=sig)
    paths = oracle.enumerate_paths(o, 1)
    a, _, _ = oracle.field(o, paths, 3.5e9)
    los = a[paths["depth"] == 0][0]
    refl = a[paths["depth"] == 1][0]
    assert abs(refl) < 1e-6 * abs(los)


def test_single_wall_s_polarised():
    """Vertical wall, Tx and Rx at equal height, no ground: the field is
    purely s-polarised and the image source gives the path length."""
    f = 28e9
    wall = S.rect_wall_x(20.0, -100, 100, -50, 50, facing=-1)
    eps, sig = S.material_table()[:2]
    tx, rx = (0.0, 0.0, 5.0), (3.0, 40.0, 5.0)
    sc, o = _one(tx, rx, [wall], [S.MAT_CONCRETE], freq=f)
    paths = oracle.enumerate_paths(o, 2)
    assert sorted(paths["depth"].tolist()) == [0, 1]
    acc, marg, pts = oracle.validate(o, paths, points=True)
    one = np.nonzero(paths["depth"] == 1)[0][0]
    # reflection point: y = y_t + (y_r - y_t) * (20 - x_t) / ((20 - x_t) + (20 - x_r))
    yp = 0.0 + 40.0 * 20.0 / (20.0 + 17.0)
    assert pts[one, 0] == pytest.approx([20.0, yp, 5.0], abs=1e-12)
    a, tau, _ = oracle.field(o, paths[one:one + 1], f)
    d2 = math.hypot(40.0 - 0.0, (20 - 0.0) + (20 - 3.0))
    ct = (40.0 - 3.0 + 3.0) / d2  # |k . n|: x-travel over length
    ct = 37.0 / d2
    ec = complex(eps[S.MAT_CONCRETE], -sig[S.MAT_CONCRETE] / (2 * math.pi * f * 8.8541878128e-12))
    root = np.sqrt(ec - (1 - ct * ct))
    gs = (ct - root) / (ct + root)
    k = 2 * math.pi * f / C
    expect = gs * _lam(f) / (4 * math.pi * d2) * np.exp(-1j * k * d2)
    assert abs(a[0] - expect) <= 1e-10 * abs(expect)


def _read_golden(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#")[0].split()
        if line:
            rows.append(line)
    return rows


def test_table1_constant_reflection_coefficients():
    """Table I constant-coefficient mode: a one-bounce path off a wall
    (concrete) or a vehicle (metal) has |a| = Gamma * lambda / (4 pi L)."""
    g = {r[0]: float(r[1]) for r in _read_golden("table1_constant_gamma.txt")}
    f = 3.5e9
    tx, rx = (0.0, 0.0, 1.0), (4.0, 30.0, 1.0)
    wall = S.rect_wall_x(20.0, -100, 100, -50, 50, facing=-1)
    sc, o = _one(tx, rx, [wall], [S.MAT_CONCRETE], const_gamma=True, freq=f)
    paths = oracle.enumerate_paths(o, 1)
    one = paths[paths["depth"] == 1]
    a, tau, _ = oracle.field(o, one, f)
    assert abs(a[0]) == pytest.approx(g["wall"] * _lam(f) / (4 * math.pi * tau[0] * C), rel=1e-12)
    # metal: a vehicle box face (+x side of a box) as the reflector
    box = ((30.0, -10.0, 0.0), (34.5, 10.0, 1.5))
    sc, o = _one((40.0, 0.0, 1.0), (42.0, 6.0, 1.0), boxes=[box], const_gamma=True, freq=f)
    paths = oracle.enumerate_paths(o, 1)
    one = paths[paths["depth"] == 1]
    assert one["face"][0, 0] == 1  # vehicle 0, face +x
    a, tau, _ = oracle.field(o, one, f)
    assert abs(a[0]) == pytest.approx(g["metal"] * _lam(f) / (4 * math.pi * tau[0] * C), rel=1e-12)


def test_corner_double_bounce_length():
    """Two perpendicular walls: the doubly mirrored source is the point
    reflection of Tx through the corner line."""
    w1 = S.rect_wall_x(0.0, 0.0, 200.0, -50, 50, facing=+1)                 # x = 0, faces +x
    w2 = [(0, 0, -50), (0, 0, 50), (200, 0, 50), (200, 0, -50)]            # y = 0, faces +y
    tx, rx = (10.0, 30.0, 2.0), (50.0, 7.0, 2.0)
    sc, o = _one(tx, rx, [w1, w2], [S.MAT_CONCRETE, S.MAT_CONCRETE])
    assert o.face_plane(0)[:3] == pytest.approx([1, 0, 0])
    assert o.face_plane(1)[:3] == pytest.approx([0, 1, 0])
    paths = oracle.enumerate_paths(o, 2)
    two = paths[paths["depth"] == 2]
    # of the two orders only x-wall-then-y-wall lands on both half-walls:
    # the other order's line from the double image crosses x = 0 at y < 0
    assert len(two) == 1 and list(two["face"][0, :2]) == [0, 1]
    _, tau, _ = oracle.field(o, two, 3.5e9)
    d = math.dist((-10.0, -30.0, 2.0), rx)
    assert tau[0] * C == pytest.approx(d, rel=1e-13)


def test_occluding_wall_blocks_line_of_sight():
    blocker = S.rect_wall_x(10.0, -5, 5, 0, 20, facing=-1)
    sc, o = _one((0, 0, 5), (20, 0, 5), [blocker], [S.MAT_CONCRETE])
    assert len(oracle.enumerate_paths(o, 0)) == 0
    sc, o = _one((0, 0, 5), (20, 0, 40), [blocker], [S.MAT_CONCRETE])  # passes over
    assert len(oracle.enumerate_paths(o, 0)) == 1


# ---------------------------------------------------------------------------
# Doppler
# ---------------------------------------------------------------------------
def test_doppler_los_eq3():
    rows = _read_golden("eq3_doppler_los.txt")
    for fc, v, th in ((float(r[0]), float(r[1]), float(r[2])) for r in rows):
        tx = (0.0, 0.0, 10.0)
        rx = np.array([120.0, -35.0, 10.0])
        u = (np.array(tx) - rx) / np.linalg.norm(np.array(tx) - rx)  # Rx -> Tx
        w = np.cross(u, [0, 0, 1.0]); w /= np.linalg.norm(w)
        t = math.radians(th)
        vel = v * (math.cos(t) * u + math.sin(t) * w)
        sc, o = _one(tx, rx, rx_vel=vel, freq=fc)
        paths = oracle.enumerate_paths(o, 0)
        _, _, fd = oracle.field(o, paths, fc)
        vel32 = np.float32(vel).astype(float)
        v32 = np.linalg.norm(vel32)
        cos_t = vel32 @ u / v32
        assert fd[0] == pytest.approx(fc * v32 / C * cos_t, abs=1e-9 * fc * v / C + 1e-12)


def test_doppler_moving_mirror():
    """A reflector translating along its normal: dL/dh = -2 cos(theta)."""
    f = 28e9
    box = ((-50.0, -50.0, -1.0), (50.0, 50.0, 0.0))    # top face z = 0
    vz = 3.0
    tx, rx = (0.0, 0.0, 10.0), (30.0, 5.0, 4.0)
    sc, o = _one(tx, rx, boxes=[box], box_vel=[(0.0, 0.0, vz)], freq=f)
    paths = oracle.enumerate_paths(o, 1)
    one = paths[paths["depth"] == 1]
    assert one["face"][0, 0] == 5  # +z face
    _, tau, fd = oracle.field(o, one, f)
    L = tau[0] * C
    cos_t = (10.0 + 4.0) / L
    assert fd[0] == pytest.approx(-(f / C) * (-2 * cos_t * vz), rel=1e-12)
    # motion parallel to the face does not shift the frequency
    sc, o = _one(tx, rx, boxes=[box], box_vel=[(7.0, -2.0, 0.0)], freq=f)
    _, _, fd = oracle.field(o, one, f)
    assert abs(fd[0]) < 1e-9


def test_doppler_moving_transmitter_sign():
    f = 3.5e9
    tx, rx = (0.0, 0.0, 10.0), (100.0, 0.0, 10.0)
    sc, o = _one(tx, rx, tx_vel=(5.0, 0.0, 0.0), freq=f)   # towards Rx
    _, _, fd = oracle.field(o, oracle.enumerate_paths(o, 0), f)
    assert fd[0] == pytest.approx(f * 5.0 / C, rel=1e-12)


# ---------------------------------------------------------------------------
# reciprocity and exhaustive enumeration on the toy scene
# ---------------------------------------------------------------------------
def test_reciprocity_toy_scene():
    sc = S.toy_scene(seed=0)
    fr = sc.frame(0)
    o = oracle.OracleScene(sc, fr)
    fwd = oracle.enumerate_paths(o, 2)
    a_f, tau_f, _ = oracle.field(o, fwd, 3.5e9)
    checked = 0
    for r in range(0, 16, 3):
        fr2 = dataclasses.replace(fr, tx_pos=fr.rx_pos[r:r + 1], rx_pos=fr.tx_pos,
                                  tx_vel=fr.rx_vel[r:r + 1], rx_vel=fr.tx_vel)
        o2 = oracle.OracleScene(sc, fr2)
        rev = oracle.enumerate_paths(o2, 2)
        a_r, tau_r, _ = oracle.field(o2, rev, 3.5e9)
        mine = np.nonzero(fwd["rx"] == r)[0]
        assert len(mine) == len(rev)
        table = {}
        for i, p in enumerate(rev):
            table[tuple(p["face"][:p["depth"]][::-1])] = i
        for i in mine:
            key = tuple(fwd["face"][i][:fwd["depth"][i]])
            j = table[key]
            assert tau_r[j] == pytest.approx(tau_f[i], rel=1e-13)
            assert abs(a_r[j] - a_f[i]) <= 1e-9 * abs(a_f[i])
            checked += 1
    assert checked > 10


def test_sbr_discovery_matches_exhaustive_enumeration():
    """Shooting-and-bouncing with reception spheres finds (almost) every path
    that exhaustive image enumeration proves valid, and nothing else."""
    sc = S.toy_scene(seed=0)
    o = oracle.OracleScene(sc, sc.frame(0))
    exact = oracle.enumerate_paths(o, 2)
    cands, marg, segs = oracle.trace(o, sc.n_rays, 2)
    uniq = oracle.dedup(cands)
    acc, vmarg = oracle.validate(o, uniq)
    found = uniq[acc]
    k_exact = {tuple(r) for r in oracle.key_fields(exact)}
    k_found = {tuple(r) for r in oracle.key_fields(found)}
    assert k_found <= k_exact
    a, _, _ = oracle.field(o, exact, 3.5e9)
    w = np.abs(a) ** 2
    hit = np.array([tuple(r) in k_found for r in oracle.key_fields(exact)])
    assert w[hit].sum() / w.sum() > 0.99
    assert hit.mean() > 0.9


def test_sbr_candidates_follow_the_ray():
    """Brute force on a single-bounce scene: the reflected ray that
    discovers the wall path starts on the wall and its face list is the wall."""
    wall = S.rect_wall_x(30.0, -60, 60, 0, 40, facing=-1)
    sc, o = _one((0.0, 0.0, 10.0), [(5.0, 20.0, 10.0), (-5, -3, 2)], [wall],
                 [S.MAT_CONCRETE])
    cands, _, _ = oracle.trace(o, 20000, 2)
    u = oracle.dedup(cands)
    acc, _ = oracle.validate(o, u)
    keys = {(int(p["rx"]), int(p["depth"]), int(p["face"][0])) for p in u[acc]}
    assert keys == {(0, 0, oracle.NO_FACE), (0, 1, 0), (1, 0, oracle.NO_FACE), (1, 1, 0)}


def test_validation_margin_flags_points_near_edges():
    wall = S.rect_wall_x(20.0, -10, 10, 0, 20, facing=-1)
    # the reflection point lies 5e-5 m inside the wall's y = 10 edge
    yp = 10.0 - 5e-5
    tx = (0.0, yp, 5.0)
    rx = (0.0, yp, 15.0)
    sc, o = _one(tx, rx, [wall], [S.MAT_CONCRETE])
    p = _path(0, 0, [0])
    acc, marg = oracle.validate(o, p)
    assert acc[0] and marg[0] & 1
    acc, marg = oracle.validate(o, p, eps_abs=1e-6)
    assert acc[0] and not marg[0]


def test_vehicle_face_numbering():
    box = ((1.0, 2.0, 0.0), (5.5, 3.8, 1.5))
    sc, o = _one((0, 0, 10), (20, 0, 1), polys=[S.rect_xy(-50, -50, 50, 50)],
                 mats=[S.MAT_GROUND], boxes=[box])
    normals = [o.face_plane(1 + j)[:3] for j in range(6)]
    expect = [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]
    for n, e in zip(normals, expect):
        assert n == pytest.approx(e)
    assert o.face_plane(2)[3] == pytest.approx(5.5)
    assert o.face_plane(6)[3] == pytest.approx(1.5)


# ---------------------------------------------------------------------------
# reduction and gradient helpers
# ---------------------------------------------------------------------------
def test_reduction_statistics():
    p = np.zeros(3, oracle.PATH_DTYPE)
    p["tx"] = [0, 0, 0]
    p["rx"] = [1, 1, 0]
    a = np.array([1.0 + 0j, 1j, 0.5])
    tau = np.array([1e-6, 3e-6, 2e-6])
    fd = np.array([-40.0, 40.0, 7.0])
    st = oracle.reduce(p, a, tau, fd, 1, 2)
    assert st[0, 1, 0:3] == pytest.approx([1.0, 1.0, 2.0])
    assert st[0, 1, 3] == pytest.approx(0.0, abs=1e-12)
    assert st[0, 1, 4] == pytest.approx(40.0)
    assert st[0, 1, 5] == pytest.approx(2e-6)
    assert st[0, 1, 6] == pytest.approx(1e-6)
    assert st[0, 0, 3:8] == pytest.approx([7.0, 0.0, 2e-6, 0.0, 1.0])


def test_fermat_gradient_of_path_length():
    """dL/dTx = -k0 (unit direction of the first segment) for any valid path."""
    sc = S.toy_scene(seed=0)
    fr = sc.frame(0)
    o = oracle.OracleScene(sc, fr)
    paths = oracle.enumerate_paths(o, 2)
    acc, marg, pts = oracle.validate(o, paths, points=True)
    sel = np.nonzero(acc & (paths["depth"] > 0))[0][:6]
    for i in sel:
        x = np.float32(fr.tx_pos[0, 0])
        h = 2.0 ** -12  # exact offset for |x| < 2048 m in float32
        def L(dx):
            tx = fr.tx_pos.copy(); tx[0, 0] = np.float32(float(x) + dx)
            oo = oracle.OracleScene(sc, dataclasses.replace(fr, tx_pos=tx))
            return oracle.field(oo, paths[i:i + 1], 3.5e9)[1][0] * C
        g = (L(h) - L(-h)) / (2 * h)
        q1 = pts[i, 0]
        k0 = (q1 - fr.tx_pos[0].astype(float)) / np.linalg.norm(q1 - fr.tx_pos[0].astype(float))
        assert g == pytest.approx(-k0[0], abs=1e-6)


def test_table1_constant_mode_two_ray_sum():
    """Constant-coefficient mode with a vertically polarised ground bounce:
    the bounce enters the coherent sum with +gamma (a scaled perfect
    conductor keeps the p component's sign)."""
    g = {r[0]: float(r[1]) for r in _read_golden("table1_constant_gamma.txt")}
    f = 3.5e9
    D, ht, hr = 40.0, 12.0, 1.5
    ground = S.rect_xy(-1e3, -1e3, 1e3, 1e3, 0.0)
    sc, o = _one((0, 0, ht), (D, 0, hr), [ground], [S.MAT_GROUND], const_gamma=True, freq=f)
    paths = oracle.enumerate_paths(o, 1)
    a, _, _ = oracle.field(o, paths, f)
    d1, d2 = math.hypot(D, ht - hr), math.hypot(D, ht + hr)
    k = 2 * math.pi * f / C
    h = _lam(f) / (4 * math.pi) * (np.exp(-1j * k * d1) / d1 + g["wall"] * np.exp(-1j * k * d2) / d2)
    assert abs(a.sum() - h) <= 1e-10 * abs(h)


# ---------------------------------------------------------------------------
# backward tracing (Sec. II-A): role exchange and record reversal
# ---------------------------------------------------------------------------
def test_reverse_paths_brute_force():
    NO = oracle.NO_FACE
    p = np.zeros(4, oracle.PATH_DTYPE)
    p["tx"] = [0, 1, 2, 1]
    p["rx"] = [3, 0, 1, 2]
    p["depth"] = [0, 1, 3, 4]
    p["face"] = [[NO, NO, NO, NO], [7, NO, NO, NO], [5, 9, 2, NO], [1, 2, 3, 4]]
    p["ray"] = [11, 12, 13, 14]
    p["flag"] = [0, 1, 2, 0]
    r = oracle.reverse_paths(p, rx_ids=[10, 20, 30])
    assert r["tx"].tolist() == [3, 0, 1, 2]
    assert r["rx"].tolist() == [10, 20, 30, 20]
    assert r["face"].tolist() == [[NO, NO, NO, NO], [7, NO, NO, NO], [2, 9, 5, NO],
                                  [4, 3, 2, 1]]
    assert r["depth"].tolist() == [0, 1, 3, 4]
    assert r["ray"].tolist() == [11, 12, 13, 14] and r["flag"].tolist() == [0, 1, 2, 0]
    # without an id list the source index is the receiver; turning a record
    # round twice gives it back
    q = oracle.reverse_paths(oracle.reverse_paths(p))
    assert (q == p).all()


def test_backward_discovery_matches_exhaustive_enumeration():
    """Shooting from the receivers finds (almost) every path that the forward
    exhaustive image enumeration proves valid, and nothing else."""
    sc = S.toy_scene(seed=0)
    fr = sc.frame(0)
    ids = [0, 5, 10, 15]
    o = oracle.OracleScene(sc, fr)
    exact = oracle.enumerate_paths(o, 2)
    exact = exact[np.isin(exact["rx"], ids)]
    cands, marg, segs = oracle.trace_backward(sc, fr, sc.n_rays, 2, rx_ids=ids)
    assert marg.shape == (len(ids), sc.n_rays)
    assert set(cands["rx"].tolist()) <= set(ids) and set(cands["tx"].tolist()) == {0}
    uniq = oracle.dedup(cands)
    acc, _ = oracle.validate(o, uniq)
    found = uniq[acc]
    k_exact = {tuple(r) for r in oracle.key_fields(exact)}
    k_found = {tuple(r) for r in oracle.key_fields(found)}
    assert k_found <= k_exact
    a, _, _ = oracle.field(o, exact, 3.5e9)
    w = np.abs(a) ** 2
    hit = np.array([tuple(r) in k_found for r in oracle.key_fields(exact)])
    assert w[hit].sum() / w.sum() > 0.99
    assert hit.mean() > 0.9
    # the same paths as forward discovery, up to the rays that miss a path
    fc, _, _ = oracle.trace(o, sc.n_rays, 2)
    fu = oracle.dedup(fc[np.isin(fc["rx"], ids)])
    fa, _ = oracle.validate(o, fu)
    k_fwd = {tuple(r) for r in oracle.key_fields(fu[fa])}
    both = k_fwd & k_found
    wk = dict(zip([tuple(r) for r in oracle.key_fields(exact)], w))
    assert sum(wk[k] for k in both) / w.sum() > 0.98


def test_backward_subset_is_the_restriction_of_the_full_set():
    """Receivers shoot independently: tracing from a subset gives exactly the
    full backward candidates of those receivers (same rays, same indices)."""
    sc = S.toy_scene(seed=2)
    fr = sc.frame(0)
    full, _, _ = oracle.trace_backward(sc, fr, 20000, 2)
    sub, _, _ = oracle.trace_backward(sc, fr, 20000, 2, rx_ids=[3, 11])
    ref = full[np.isin(full["rx"], [3, 11])]
    key = lambda p: sorted(map(tuple, np.concatenate(
        [oracle.key_fields(p), p["ray"][:, None].astype(np.int64)], 1).tolist()))
    assert len(ref) > 10 and key(sub) == key(ref)


# ---------------------------------------------------------------------------
# per-receiver re-discovery schedule (Sec. III-A segments, Sec. III-B Eq. 2)
# ---------------------------------------------------------------------------
def test_refresh_schedule_rule_by_hand():
    f, dt = 3.5e9, 1e-3
    tx = (0.0, 0.0, 10.0)
    rx = [(50.0, 0.0, 10.0),     # at rest: reused up to max_interval
          (0.0, 60.0, 10.0),     # moves across the Tx direction at 1 m/s
          (-40.0, 0.0, 10.0)]    # LoS blocked later by a vehicle
    vel = [(0.0, 0.0, 0.0), (1.0, 0.0, 0.0), (0.0, 0.0, 0.0)]
    box = ((-22.0, -1.0, 0.0), (-18.0, 1.0, 20.0))
    sc = S.custom_scene([], [], tx, rx, rx_vel=vel, boxes=[box], freq=f)
    fr = sc.frame(0)
    far = dataclasses.replace(fr, veh_pos=np.float32([[300.0, 300.0, 10.0]]))
    o = oracle.OracleScene(sc, far)
    state = np.full((3, 4), -1.0, np.float32)
    ref = np.zeros((1, 3), np.uint8)
    # Eq. 2 by hand for receiver 1: theta = pi/2, f_D = f * 1 / c, R = 0.5
    tc = math.sqrt(1 / 0.5 ** 4 - 1) / (2 * math.pi * f / C * (math.pi / 2) ** 2)
    assert 0.021 < tc < 0.022          # 21 frames of 1 ms
    due, state, ref = oracle.refresh_schedule(o, state, ref, f, 0.5, dt, 10.0, 50)
    assert due.tolist() == [0, 1, 2] and ref.tolist() == [[1, 1, 1]]
    assert state[:, 3].tolist() == [0, 0, 0]
    for k in range(1, 21):             # frames 1..20: nothing due
        due, state, ref = oracle.refresh_schedule(o, state, ref, f, 0.5, dt, 10.0, 50)
        assert due.tolist() == [], k
    due, state, ref = oracle.refresh_schedule(o, state, ref, f, 0.5, dt, 10.0, 50)
    assert due.tolist() == [1]         # frame 21 reaches floor(T_c / dt)
    # the vehicle moves onto the line of sight of receiver 2
    o2 = oracle.OracleScene(sc, fr)
    due, state, ref = oracle.refresh_schedule(o2, state, ref, f, 0.5, dt, 10.0, 50)
    assert due.tolist() == [2] and ref.tolist() == [[1, 1, 0]]
    # segment length: moved exactly 10 m is due, 9.5 m is not
    moved = dataclasses.replace(fr, rx_pos=np.float32([[60.0, 0.0, 10.0], [0.0, 60.0, 10.0],
                                                       [-49.5, 0.0, 10.0]]))
    o3 = oracle.OracleScene(sc, moved)
    due, state, ref = oracle.refresh_schedule(o3, state, ref, f, 0.5, dt, 10.0, 50)
    assert 0 in due.tolist() and 2 not in due.tolist()
    # max_interval caps the reuse of a receiver at rest
    st = np.zeros((3, 4), np.float32)
    st[:, :3] = moved.rx_pos
    st[:, 3] = 49                      # this frame is the 50th since discovery
    due, _, _ = oracle.refresh_schedule(o3, st, np.array([[1, 1, 0]], np.uint8), f, 0.5, dt,
                                        10.0, 50)
    assert 0 in due.tolist() and 2 in due.tolist()
    st[:, 3] = 48
    due, _, _ = oracle.refresh_schedule(o3, st, np.array([[1, 1, 0]], np.uint8), f, 0.5, dt,
                                        10.0, 50)
    assert 0 not in due.tolist() and 2 not in due.tolist()


# ---------------------------------------------------------------------------
# received power, the loss of the differentiable-field workload and its
# central finite differences (Sec. IV: transmit power and received power;
# gradient over a frozen path topology)
# ---------------------------------------------------------------------------
def _hand_paths():
    """Five hand-made paths on 2 Tx x 3 Rx with amplitudes chosen so that the
    coherent per-Tx sum, the incoherent sum over Tx and a fully coherent sum
    over Tx all differ."""
    p = np.zeros(5, oracle.PATH_DTYPE)
    p["tx"] = [0, 0, 1, 0, 0]
    p["rx"] = [0, 0, 0, 1, 1]
    a = np.array([1e-3, 1e-3, 1e-3, 2e-3, -2e-3], complex)
    return p, a


def test_rx_power_coherent_per_tx_incoherent_over_tx():
    p, a = _hand_paths()
    z = np.zeros(len(p))
    st = oracle.reduce(p, a, z, z, 2, 3)
    coh, inc = oracle.rx_power(st, 0.25)
    # rx 0: tx 0 adds 1e-3 + 1e-3 in phase (|h|^2 = 4e-6), tx 1 adds 1e-6
    # as power; rx 1: the two tx-0 paths cancel; rx 2 has no path
    assert coh == pytest.approx([0.25 * 5e-6, 0.0, 0.0], rel=1e-14, abs=1e-30)
    assert inc == pytest.approx([0.25 * 3e-6, 0.25 * 8e-6, 0.0], rel=1e-14, abs=1e-30)
    # the same from a hand-written statistics array (Re h, Im h, sum |a|^2)
    st2 = np.zeros((2, 3, 8))
    st2[0, 0, :3] = (2e-3, 0.0, 2e-6)
    st2[1, 0, :3] = (0.0, 1e-3, 1e-6)
    st2[0, 2, :3] = (3e-3, -4e-3, 1e-5)
    coh2, inc2 = oracle.rx_power(st2, 2.0)
    assert coh2 == pytest.approx([2.0 * 5e-6, 0.0, 2.0 * 25e-6], rel=1e-14)
    assert inc2 == pytest.approx([2.0 * 3e-6, 0.0, 2.0 * 1e-5], rel=1e-14)


def test_power_loss_closed_form():
    p, a = _hand_paths()
    # add a third receiver reached by tx 1 only
    p = np.concatenate([p, p[:1]])
    p["tx"][-1], p["rx"][-1] = 1, 2
    a = np.concatenate([a, [1e-3 * np.exp(0.7j)]])
    pt = 0.25
    target = np.array([-31.0, 0.0, -40.0])
    mask = np.array([True, False, True])
    got = oracle.power_loss(p, a, 2, 3, pt, target, mask)
    p0 = pt * (4e-6 + 1e-6)      # coherent within tx 0, power of tx 1 added
    p2 = pt * 1e-6
    dbm = [10 * math.log10(p0 * 1e3), 10 * math.log10(p2 * 1e3)]
    expect = (dbm[0] + 31.0) ** 2 + (dbm[1] + 40.0) ** 2
    assert got == pytest.approx(expect, rel=1e-13)
    # receiver 1 (its two paths cancel: zero power) is masked out and adds
    # nothing; unmasking a receiver with power adds its term
    mask2 = np.array([True, False, False])
    assert oracle.power_loss(p, a, 2, 3, pt, target, mask2) == pytest.approx(
        (dbm[0] + 31.0) ** 2, rel=1e-13)


def _wall_los_scene(f):
    wall = S.rect_wall_x(20.0, -100, 100, -50, 50, facing=-1)
    tx, rx = (0.0, 0.0, 5.0), (3.0, 40.0, 5.0)
    return _one(tx, rx, [wall], [S.MAT_CONCRETE], freq=f)


def test_fd_gradient_materials_single_wall_closed_form():
    """LoS + one s-polarised wall bounce, coherently summed: the derivative
    of |h|^2 w.r.t. the wall's eps_r and sigma follows from
    dGamma_s / d eps_c = -cos(theta) / (s (cos(theta) + s)^2),
    s = sqrt(eps_c - sin^2 theta), eps_c = eps_r - j sigma / (2 pi f eps0)."""
    f = 28e9
    sc, o = _wall_los_scene(f)
    fr = sc.frame(0)
    paths = oracle.enumerate_paths(o, 1)
    assert sorted(paths["depth"].tolist()) == [0, 1]
    eps, sig = S.material_table()[:2]
    e0 = 8.8541878128e-12
    k = 2 * math.pi * f / C
    d1 = math.hypot(3.0, 40.0)
    d2 = math.hypot(40.0, 37.0)
    ct = 37.0 / d2
    ec = complex(eps[S.MAT_CONCRETE], -sig[S.MAT_CONCRETE] / (2 * math.pi * f * e0))
    s = np.sqrt(ec - (1 - ct * ct))
    gs = (ct - s) / (ct + s)
    dg = -ct / (s * (ct + s) ** 2)
    a_los = _lam(f) / (4 * math.pi * d1) * np.exp(-1j * k * d1)
    a_w = gs * _lam(f) / (4 * math.pi * d2) * np.exp(-1j * k * d2)
    h = a_los + a_w
    pt = 10.0 ** ((50 - 30) / 10)  # 50 dBm
    dbm = 10 * math.log10(pt * abs(h) ** 2 * 1e3)
    target = np.array([dbm - 3.0])
    mask = np.array([True])
    # d loss / d|h|^2 = 2 (dBm - target) 10 / (ln 10 |h|^2)
    dl = 2 * 3.0 * 10 / (math.log(10) * abs(h) ** 2)
    dh_deps = a_w / gs * dg
    dh_dsig = dh_deps * (-1j / (2 * math.pi * f * e0))
    g_eps_cf = dl * 2 * (np.conj(h) * dh_deps).real
    g_sig_cf = dl * 2 * (np.conj(h) * dh_dsig).real
    # the coherent sum matters: the incoherent one gives another value
    g_inc = dl * 2 * (np.conj(a_w) * dh_deps).real * abs(h) ** 2 / (abs(a_los) ** 2 + abs(a_w) ** 2)
    assert abs(g_inc - g_eps_cf) > 0.05 * abs(g_eps_cf)
    g_eps, g_sig, g_tx = oracle.fd_gradient(sc, fr, paths, f, pt, target, mask)
    assert g_eps[S.MAT_CONCRETE] == pytest.approx(g_eps_cf, rel=1e-6)
    assert g_sig[S.MAT_CONCRETE] == pytest.approx(g_sig_cf, rel=1e-6)
    # materials the paths never meet have zero gradient (no other term)
    others = np.arange(len(eps)) != S.MAT_CONCRETE
    assert np.all(g_eps[others] == 0.0) and np.all(g_sig[others] == 0.0)


def test_fd_gradient_tx_position_friis():
    """LoS only: P = P_t (lambda / 4 pi d)^2, so d loss / d Tx =
    2 (dBm - target) (-20 / (d ln 10)) (Tx - Rx) / d; no material enters."""
    f = 3.5e9
    tx, rx = (1.0, -2.0, 10.0), (401.25, 37.5, 1.5)
    sc, o = _one(tx, rx, freq=f)
    fr = sc.frame(0)
    paths = oracle.enumerate_paths(o, 2)
    assert len(paths) == 1
    t = np.float32(tx).astype(float)
    r = np.float32(rx).astype(float)
    d = np.linalg.norm(t - r)
    pt = 100.0
    dbm = 10 * math.log10(pt * (_lam(f) / (4 * math.pi * d)) ** 2 * 1e3)
    target = np.array([dbm + 2.0])
    g_eps, g_sig, g_tx = oracle.fd_gradient(sc, fr, paths, f, pt, target, np.array([True]))
    expect = 2 * (-2.0) * (-20 / (d * math.log(10))) * (t - r) / d
    assert g_tx[0] == pytest.approx(expect, rel=1e-6)
    assert np.all(g_eps == 0.0) and np.all(g_sig == 0.0)
