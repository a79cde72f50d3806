"""CPU oracle for dynamic urban EM ray tracing (arXiv 2303.10521).

TEST INFRASTRUCTURE ONLY.  A plain FP64 restatement of the method (brute
force over every face, no BVH) used by the tests, the smoke check and the
benchmark's CPU-baseline leg to check and time the CUDA path.  Nothing in the
product package imports it, and it imports nothing from the product package.

The compiled part lives in ``emrt_oracle.c`` (discovery, image-method
acceptance, field, enumeration).  This module adds the steps that are plain
array bookkeeping: deduplication of candidates (Sec. II-A: a path is a face-ID
sequence stored once), the per-(transmitter, receiver) reduction of Table III
statistics (Sec. V-D), the received-power loss and its central finite
differences.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
(closed forms, reciprocity, exhaustive enumeration, covering property).
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "emrt_oracle.c")
MAX_DEPTH = 4
C_LIGHT = 299792458.0

PATH_DTYPE = np.dtype([("tx", "<u4"), ("rx", "<u4"), ("depth", "<u4"),
                       ("face", "<u4", (MAX_DEPTH,)), ("ray", "<u4"),
                       ("flag", "<u4")])
NO_FACE = 0xFFFFFFFF


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, so x86 and Arm agree)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off",
                           "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC,
                           "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Desc(C.Structure):
    _fields_ = [("n_static_faces", C.c_int), ("face_off", C.c_void_p),
                ("face_xyz", C.c_void_p), ("face_mat", C.c_void_p),
                ("n_veh", C.c_int), ("veh_half", C.c_void_p),
                ("veh_pos", C.c_void_p), ("veh_vel", C.c_void_p),
                ("veh_mat", C.c_uint32), ("n_rx", C.c_int),
                ("rx_pos", C.c_void_p), ("rx_vel", C.c_void_p),
                ("n_tx", C.c_int), ("tx_pos", C.c_void_p),
                ("tx_vel", C.c_void_p), ("n_mat", C.c_int),
                ("eps_r", C.c_void_p), ("sigma", C.c_void_p),
                ("gamma", C.c_void_p), ("const_gamma", C.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        vp, i64, u64, d = C.c_void_p, C.c_int64, C.c_uint64, C.c_double
        L.orc_scene_create.restype = vp
        L.orc_scene_create.argtypes = [vp]
        L.orc_scene_destroy.argtypes = [vp]
        L.orc_scene_n_faces.argtypes = [vp]
        L.orc_face_plane.argtypes = [vp, C.c_int, vp]
        L.orc_ray_dir.argtypes = [u64, u64, vp]
        L.orc_radius_factor.restype = d
        L.orc_radius_factor.argtypes = [u64]
        L.orc_trace.restype = i64
        L.orc_trace.argtypes = [vp, u64, C.c_int, u64, u64, u64, d, d, C.c_int,
                                vp, i64, vp, vp]
        L.orc_trace_list.restype = i64
        L.orc_trace_list.argtypes = [vp, u64, C.c_int, vp, u64, d, d, C.c_int, vp, i64, vp, vp]
        L.orc_validate.argtypes = [vp, i64, vp, d, d, C.c_int, vp, vp, vp]
        L.orc_field.argtypes = [vp, i64, vp, d, C.c_int, vp, vp, vp]
        L.orc_fresnel.argtypes = [d, d, d, vp]
        L.orc_enumerate.restype = i64
        L.orc_enumerate.argtypes = [vp, C.c_int, C.c_int, vp, i64]
    return _lib


def n_threads() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None and a.size else None


class OracleScene:
    """One frame of a scene (geometry, vehicle poses, Rx and Tx) on the CPU."""

    def __init__(self, scene, frame, const_gamma: bool = False,
                 eps_r=None, sigma=None):
        f32 = lambda a: np.ascontiguousarray(a, np.float32)
        self._keep = dict(
            off=np.ascontiguousarray(scene.face_off, np.uint32),
            xyz=f32(scene.face_xyz),
            mat=np.ascontiguousarray(scene.face_mat, np.uint32),
            half=f32(scene.veh_half), vpos=f32(frame.veh_pos),
            vvel=f32(frame.veh_vel), rx=f32(frame.rx_pos), rxv=f32(frame.rx_vel),
            tx=f32(frame.tx_pos), txv=f32(frame.tx_vel),
            eps=np.ascontiguousarray(scene.eps_r if eps_r is None else eps_r, np.float64),
            sig=np.ascontiguousarray(scene.sigma if sigma is None else sigma, np.float64),
            gam=np.ascontiguousarray(scene.gamma, np.float64))
        k = self._keep
        d = _Desc(scene.n_static_faces, _ptr(k["off"]), _ptr(k["xyz"]),
                  _ptr(k["mat"]), scene.n_vehicles, _ptr(k["half"]),
                  _ptr(k["vpos"]), _ptr(k["vvel"]), scene.veh_mat,
                  len(k["rx"]), _ptr(k["rx"]), _ptr(k["rxv"]), len(k["tx"]),
                  _ptr(k["tx"]), _ptr(k["txv"]), len(k["eps"]), _ptr(k["eps"]),
                  _ptr(k["sig"]), _ptr(k["gam"]), int(const_gamma))
        self.h = lib().orc_scene_create(C.byref(d))
        self.n_faces = lib().orc_scene_n_faces(self.h)
        self.n_rx = len(k["rx"])
        self.n_tx = len(k["tx"])

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_scene_destroy(self.h)
            self.h = None

    def face_plane(self, f):
        out = np.zeros(4)
        lib().orc_face_plane(self.h, int(f), _ptr(out))
        return out


# ---------------------------------------------------------------------------
def ray_dir(n_rays: int, i: int) -> np.ndarray:
    out = np.zeros(3, np.float32)
    lib().orc_ray_dir(n_rays, i, _ptr(out))
    return out


def radius_factor(n_rays: int) -> float:
    return lib().orc_radius_factor(n_rays)


def fresnel(eps_c: complex, cos_t: float):
    out = np.zeros(4)
    lib().orc_fresnel(eps_c.real, eps_c.imag, cos_t, _ptr(out))
    return complex(out[0], out[1]), complex(out[2], out[3])


def trace(os_: OracleScene, n_rays, max_depth, offset=0, stride=1, count=None,
          eps_abs=1e-4, eps_rel=0.0, threads=None):
    """SBR discovery (not deduplicated).  Returns (candidates, ray_marg,
    ray_segs); ray_marg[tx, j] = first segment within the margin (255: none)."""
    if count is None:
        count = (n_rays - offset + stride - 1) // stride
    threads = threads or n_threads()
    cap = max(1024, 4 * count * os_.n_tx)
    marg = np.zeros((os_.n_tx, count), np.uint8)
    segs = np.zeros((os_.n_tx, count), np.uint8)
    while True:
        out = np.zeros(cap, PATH_DTYPE)
        n = lib().orc_trace(os_.h, n_rays, max_depth, offset, stride, count,
                            eps_abs, eps_rel, threads, _ptr(out), cap,
                            _ptr(marg), _ptr(segs))
        if n <= cap:
            return out[:n], marg, segs
        cap = int(n)


def trace_list(os_, n_rays, max_depth, ray_idx, eps_abs=1e-4, eps_rel=0.0, threads=None):
    """SBR discovery for an explicit list of ray indices (same outputs as
    trace; candidate and ray_marg indices refer to positions in the list)."""
    idx = np.ascontiguousarray(ray_idx, np.uint64)
    count = len(idx)
    threads = threads or n_threads()
    cap = max(1024, 4 * count * os_.n_tx)
    marg = np.zeros((os_.n_tx, count), np.uint8)
    segs = np.zeros((os_.n_tx, count), np.uint8)
    while True:
        out = np.zeros(cap, PATH_DTYPE)
        n = lib().orc_trace_list(os_.h, n_rays, max_depth, _ptr(idx), count, eps_abs, eps_rel,
                                 threads, _ptr(out), cap, _ptr(marg), _ptr(segs))
        if n <= cap:
            return out[:n], marg, segs
        cap = int(n)


# ---------------------------------------------------------------------------
# Backward tracing (Sec. II-A: rays shot from the receiver side).  A path is
# reciprocal -- the same face sequence joins Tx and Rx in either direction --
# so backward discovery is forward discovery in the frame with the roles
# exchanged, followed by turning each record round.
def backward_scene(scene, frame, rx_ids=None, **kw) -> OracleScene:
    """The frame with the roles exchanged: the receivers rx_ids (all when
    None) shoot as transmitters, the transmitters receive."""
    ids = np.arange(len(frame.rx_pos)) if rx_ids is None else np.asarray(rx_ids, np.int64)
    fr = dataclasses.replace(frame, tx_pos=np.asarray(frame.rx_pos)[ids],
                             tx_vel=np.asarray(frame.rx_vel)[ids],
                             rx_pos=frame.tx_pos, rx_vel=frame.tx_vel)
    return OracleScene(scene, fr, **kw)


def reverse_paths(p, rx_ids=None):
    """Records of the role-exchanged frame (tx = shooting receiver's position
    in rx_ids, rx = transmitter, faces in the order met from the receiver)
    in forward orientation: tx first, rx = rx_ids[source], faces reversed."""
    out = np.array(p, PATH_DTYPE, copy=True)
    src = p["tx"].astype(np.int64)
    out["tx"] = p["rx"]
    out["rx"] = src if rx_ids is None else np.asarray(rx_ids, np.int64)[src]
    for d in range(1, MAX_DEPTH + 1):
        sel = p["depth"] == d
        for k in range(d):
            out["face"][sel, k] = p["face"][sel, d - 1 - k]
    return out


def trace_backward(scene, frame, n_rays, max_depth, rx_ids=None, offset=0, stride=1,
                   count=None, eps_abs=1e-4, eps_rel=0.0, threads=None):
    """Backward SBR discovery from the receivers rx_ids with reception spheres
    at the transmitters.  Returns (candidates in forward orientation,
    ray_marg, ray_segs); ray_marg rows are positions in rx_ids."""
    ob = backward_scene(scene, frame, rx_ids)
    c, marg, segs = trace(ob, n_rays, max_depth, offset=offset, stride=stride, count=count,
                          eps_abs=eps_abs, eps_rel=eps_rel, threads=threads)
    return reverse_paths(c, rx_ids), marg, segs


def key_fields(p):
    return np.stack([p["tx"], p["rx"], p["depth"]] +
                    [p["face"][:, j] for j in range(MAX_DEPTH)], 1).astype(np.int64)


def dedup(cands):
    """Unique candidates in canonical (tx, rx, depth, faces) order.  The
    merged record keeps the smallest ray index and the most robust flag."""
    if len(cands) == 0:
        return cands.copy()
    k = key_fields(cands)
    order = np.lexsort(tuple(k[:, j] for j in range(k.shape[1] - 1, -1, -1)))
    ks = k[order]
    first = np.ones(len(ks), bool)
    first[1:] = np.any(ks[1:] != ks[:-1], axis=1)
    grp = np.cumsum(first) - 1
    out = cands[order][first].copy()
    ray = np.full(len(out), np.iinfo(np.uint32).max, np.uint64)
    np.minimum.at(ray, grp, cands["ray"][order].astype(np.uint64))
    flag = np.full(len(out), 3, np.uint32)
    np.minimum.at(flag, grp, cands["flag"][order])
    out["ray"] = ray.astype(np.uint32)
    out["flag"] = flag
    return out


def validate(os_: OracleScene, paths, eps_abs=1e-4, eps_rel=0.0, threads=None,
             points=False):
    paths = np.ascontiguousarray(paths, PATH_DTYPE)
    n = len(paths)
    acc = np.zeros(n, np.uint8)
    marg = np.zeros(n, np.uint8)
    pts = np.zeros((n, MAX_DEPTH, 3)) if points else None
    if n:
        lib().orc_validate(os_.h, n, _ptr(paths), eps_abs, eps_rel,
                           threads or n_threads(), _ptr(acc), _ptr(marg),
                           _ptr(pts) if points else None)
    return (acc.astype(bool), marg, pts) if points else (acc.astype(bool), marg)


def field(os_: OracleScene, paths, freq, threads=None):
    """Per path: complex amplitude (1 W transmit power), delay (s), Doppler (Hz)."""
    paths = np.ascontiguousarray(paths, PATH_DTYPE)
    n = len(paths)
    a = np.zeros((n, 2))
    tau = np.zeros(n)
    fd = np.zeros(n)
    if n:
        lib().orc_field(os_.h, n, _ptr(paths), float(freq),
                        threads or n_threads(), _ptr(a), _ptr(tau), _ptr(fd))
    return a[:, 0] + 1j * a[:, 1], tau, fd


def enumerate_paths(os_: OracleScene, max_depth, threads=None):
    cap = 1 << 16
    while True:
        out = np.zeros(cap, PATH_DTYPE)
        n = lib().orc_enumerate(os_.h, max_depth, threads or n_threads(),
                                _ptr(out), cap)
        if n <= cap:
            return out[:n]
        cap = int(n)


def reduce(paths, a, tau, fd, n_tx, n_rx):
    """Per (tx, rx): coherent sum h, incoherent power, power-weighted mean
    Doppler shift and RMS Doppler spread (Table III), mean delay and RMS delay
    spread, path count.  Returns an array [n_tx, n_rx, 8]:
    (Re h, Im h, sum|a|^2, fd_mean, fd_rms, tau_mean, tau_rms, count)."""
    out = np.zeros((n_tx, n_rx, 8))
    for i in range(len(paths)):
        t, r = int(paths["tx"][i]), int(paths["rx"][i])
        w = abs(a[i]) ** 2
        o = out[t, r]
        o[0] += a[i].real
        o[1] += a[i].imag
        o[2] += w
        o[3] += w * fd[i]
        o[4] += w * fd[i] ** 2
        o[5] += w * tau[i]
        o[6] += w * tau[i] ** 2
        o[7] += 1
    p = out[..., 2]
    safe = np.where(p > 0, p, 1.0)
    for m, m2 in ((3, 4), (5, 6)):
        mean = np.where(p > 0, out[..., m] / safe, 0.0)
        var = np.where(p > 0, out[..., m2] / safe - mean ** 2, 0.0)
        out[..., m] = mean
        out[..., m2] = np.sqrt(np.maximum(var, 0.0))
    return out


def rx_power(stats, tx_power_w):
    """Received power per receiver (W): coherent per transmitter, summed
    incoherently over transmitters; and the fully incoherent sum."""
    coh = tx_power_w * (stats[..., 0] ** 2 + stats[..., 1] ** 2).sum(0)
    inc = tx_power_w * stats[..., 2].sum(0)
    return coh, inc


def power_loss(paths, a, n_tx, n_rx, tx_power_w, target_dbm, mask):
    """Sum over receivers in ``mask`` of (P_dBm - target)^2."""
    h = np.zeros((n_tx, n_rx), complex)
    np.add.at(h, (paths["tx"].astype(int), paths["rx"].astype(int)), a)
    p = tx_power_w * (np.abs(h) ** 2).sum(0)
    dbm = 10 * np.log10(np.where(mask, p, 1.0) * 1e3)
    return float(np.sum(np.where(mask, (dbm - target_dbm) ** 2, 0.0)))


def fd_gradient(scene, frame, paths, freq, tx_power_w, target_dbm, mask,
                h_rel=1e-4, eps_r=None, sigma=None, tx_h=1e-4):
    """Central finite differences (relative step h_rel) of power_loss with
    respect to eps_r[m], sigma[m] (m over the material table) and each
    transmitter position (step near tx_h metres), over a frozen path
    topology."""
    eps0 = np.array(scene.eps_r if eps_r is None else eps_r, np.float64)
    sig0 = np.array(scene.sigma if sigma is None else sigma, np.float64)
    n_tx, n_rx = len(frame.tx_pos), len(frame.rx_pos)

    def loss(eps, sig, fr):
        o = OracleScene(scene, fr, eps_r=eps, sigma=sig)
        a, _, _ = field(o, paths, freq)
        return power_loss(paths, a, n_tx, n_rx, tx_power_w, target_dbm, mask)

    g_eps = np.zeros_like(eps0)
    g_sig = np.zeros_like(sig0)
    for m in range(len(eps0)):
        for arr, g in ((eps0, g_eps), (sig0, g_sig)):
            h = h_rel * abs(arr[m])
            up, dn = arr.copy(), arr.copy()
            up[m] += h
            dn[m] -= h
            if arr is eps0:
                g[m] = (loss(up, sig0, frame) - loss(dn, sig0, frame)) / (2 * h)
            else:
                g[m] = (loss(eps0, up, frame) - loss(eps0, dn, frame)) / (2 * h)
    g_tx = np.zeros((n_tx, 3))
    import dataclasses
    for t in range(n_tx):
        for c in range(3):
            # positions are float32 inputs: the step is a power-of-two number
            # of float32 ulps near tx_h, so both perturbed positions are
            # exact and the difference stays centred
            x = np.float32(frame.tx_pos[t, c])
            ulp = float(np.spacing(np.abs(x)))
            h = ulp * 2.0 ** max(0, int(np.floor(np.log2(tx_h / ulp))))
            up = frame.tx_pos.copy()
            dn = frame.tx_pos.copy()
            up[t, c] = np.float32(float(x) + h)
            dn[t, c] = np.float32(float(x) - h)
            assert float(up[t, c]) - float(x) == h == float(x) - float(dn[t, c])
            fu = dataclasses.replace(frame, tx_pos=up)
            fdn = dataclasses.replace(frame, tx_pos=dn)
            g_tx[t, c] = (loss(eps0, sig0, fu) - loss(eps0, sig0, fdn)) / (2 * h)
    return g_eps, g_sig, g_tx


# ---------------------------------------------------------------------------
# channel statistics over time (Sec. III-B)
def channel_correlation(h, max_lag):
    """Eq. 1 read as the normalised autocovariance of g(t) = |h(t)| over the
    frames t (the printed denominator E[g^2] E[g]^2 is dimensionally
    inconsistent): R(tau) = (mean_{t<F-tau} g(t) g(t+tau) - mu^2) /
    (mean_t g^2 - mu^2).  h: complex [F, P]; returns [P, max_lag + 1]; a
    constant |h| gives 0."""
    g = np.abs(np.asarray(h))
    F, P = g.shape
    R = np.zeros((P, max_lag + 1))
    for p in range(P):
        mu = g[:, p].mean()
        var = (g[:, p] ** 2).mean() - mu ** 2
        for tau in range(max_lag + 1):
            n = F - tau
            if n <= 0 or var <= 0:
                continue
            R[p, tau] = (np.dot(g[:n, p], g[tau:, p]) / n - mu ** 2) / var
    return R


def coherence_time(tx_pos, rx_pos, rx_vel, freq, r_threshold):
    """Eq. 2 as printed: T_c = sqrt(1/R^4 - 1) / (2 pi f_D theta^2) per
    (tx, rx), f_D = f |v| / c, theta the angle between the receiver's motion
    and the direction from transmitter to receiver; infinite when f_D theta^2
    is zero."""
    tx = np.asarray(tx_pos, np.float64)
    rx = np.asarray(rx_pos, np.float64)
    v = np.asarray(rx_vel, np.float64)
    out = np.full((len(tx), len(rx)), np.inf)
    num = np.sqrt(max(0.0, 1.0 / r_threshold ** 4 - 1.0))
    for t in range(len(tx)):
        for r in range(len(rx)):
            k = rx[r] - tx[t]
            kn, vn = np.linalg.norm(k), np.linalg.norm(v[r])
            if kn == 0 or vn == 0:
                continue
            th = np.arccos(np.clip(np.dot(k, v[r]) / (kn * vn), -1.0, 1.0))
            den = 2 * np.pi * (freq * vn / C_LIGHT) * th * th
            if den > 0:
                out[t, r] = num / den
    return out


def refresh_schedule(os_: OracleScene, state, los_ref, freq, r_threshold, dt, d_seg,
                     max_interval):
    """Per-receiver re-discovery rule (Sec. III-A trajectory segments where
    the LoS condition or position changes; Sec. III-B reuse within the Eq. 2
    coherence time).  Receiver r is due when never discovered (state w < 0),
    when the LoS of one of its pairs (direct path through the acceptance
    test) differs from los_ref, when it moved d_seg or more since its last
    discovery, or when the frames since then plus this one reach
    min(max_interval, max(1, floor(min_tx T_c / dt))) (dt = 0: max_interval).  Returns (due ids,
    new state, new los_ref); inputs are not modified."""
    k = os_._keep
    rx = k["rx"].astype(np.float64)
    n_tx, n_rx = os_.n_tx, os_.n_rx
    direct = np.zeros(n_tx * n_rx, PATH_DTYPE)
    direct["tx"] = np.repeat(np.arange(n_tx), n_rx)
    direct["rx"] = np.tile(np.arange(n_rx), n_tx)
    direct["face"] = NO_FACE
    los, _ = validate(os_, direct)
    los = los.reshape(n_tx, n_rx).astype(np.uint8)
    tc = coherence_time(k["tx"], k["rx"], k["rxv"], freq, r_threshold).min(axis=0)
    state = np.array(state, np.float32, copy=True)
    ref = np.array(los_ref, np.uint8, copy=True)
    due = []
    for r in range(n_rx):
        never = state[r, 3] < 0
        frames = 0 if never else int(state[r, 3]) + 1
        moved2 = float(np.sum((rx[r] - state[r, :3].astype(np.float64)) ** 2))
        iv = np.floor(tc[r] / dt) if dt > 0 else np.inf
        interval = max_interval if iv >= max_interval else int(max(1.0, iv))
        d = (never or bool(np.any(los[:, r] != ref[:, r])) or moved2 >= float(np.float32(d_seg)) ** 2
             or frames >= interval)
        if d:
            due.append(r)
            state[r] = (k["rx"][r][0], k["rx"][r][1], k["rx"][r][2], 0.0)
            ref[:, r] = los[:, r]
        else:
            state[r, 3] = frames
    return np.asarray(due, np.int64), state, ref
