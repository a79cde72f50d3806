"""Python front end of the emrt C-ABI: device memory and streams come from
PyTorch; every computation runs in libemrt.so's CUDA kernels.

    sc = Scene(scenes.city_scene())           # static BVH built once
    sc.update(sc_desc.frame(k))               # per frame: vehicles, Rx, Tx
    paths = sc.trace()                         # plain discovery + acceptance
    ch = sc.channel(paths, 3.5e9)              # per-path field, per-Rx stats
    sc.revalidate(paths)                       # cached frame
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from typing import Optional

import numpy as np
import torch

from . import _native as N


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _dev(a, dtype, device) -> torch.Tensor:
    if isinstance(a, torch.Tensor):
        t = a.to(device=device, dtype=dtype)
    else:
        t = torch.as_tensor(np.ascontiguousarray(a), dtype=dtype).to(device, non_blocking=False)
    return t.contiguous()


def _u32(a, device):
    return _dev(np.asarray(a, np.uint32).view(np.int32), torch.int32, device)


def _ptr(t: Optional[torch.Tensor]):
    return C.c_void_p(t.data_ptr()) if t is not None and t.numel() else None


class Paths:
    """Caller-owned path set on the device: ``rec`` int32 [capacity, 8]
    (uint32 records, see include/emrt.h) and ``count`` int32 [1]."""

    def __init__(self, capacity: int, device):
        self.capacity = int(capacity)
        self.rec = torch.empty((max(self.capacity, 1), N.PATH_WORDS), dtype=torch.int32,
                               device=device)
        self.count = torch.zeros(1, dtype=torch.int32, device=device)

    def c(self) -> N.PathsC:
        return N.PathsC(self.rec.data_ptr(), self.capacity, self.count.data_ptr())

    def n(self) -> int:
        return int(self.count.item())

    def records(self) -> np.ndarray:
        """uint32 [n, 8] copy on the host (n clamped to the capacity)."""
        n = min(self.n(), self.capacity)
        return self.rec[:n].cpu().numpy().view(np.uint32)

    def save(self, path: str):
        """Checkpoint of the path set (e.g. the cache of a frame sequence):
        its canonical records as a uint32 [n, 8] .npy file."""
        np.save(path, self.records())

    @classmethod
    def load(cls, path: str, device, capacity: Optional[int] = None) -> "Paths":
        """A path set from save(), on `device`, with room for `capacity`
        records (default: the records saved)."""
        r = np.load(path).astype(np.uint32).reshape(-1, N.PATH_WORDS)
        p = cls(max(len(r), capacity or 0), device)
        if len(r):
            p.rec[:len(r)] = torch.from_numpy(r.view(np.int32)).to(device)
        p.count.fill_(len(r))
        return p


@dataclass
class ChannelResult:
    path: torch.Tensor   # [capacity, 4] float64: Re a, Im a, tau, f_D
    pair: torch.Tensor   # [n_tx, n_rx, 8] float64
    rx: torch.Tensor     # [n_rx, 2] float64 W: coherent, incoherent


def rx_dbm(ch: ChannelResult, coherent: bool = True) -> np.ndarray:
    """Received power per receiver in dBm from a channel result (coherent
    per Tx and summed over Tx, or the fully incoherent sum); -inf where no
    path arrives."""
    p = ch.rx[:, 0 if coherent else 1].detach().to("cpu", torch.float64).numpy()
    with np.errstate(divide="ignore"):
        return 10.0 * np.log10(p) + 30.0


def save_heatmap(path: str, ch: ChannelResult, rx_pos=None, coherent: bool = True):
    """Per-receiver received power as a .npy heat-map array: float64
    [n_rx, 4] (x, y, z, dBm) when rx_pos ([n_rx, 3]) is given, else [n_rx]
    dBm."""
    dbm = rx_dbm(ch, coherent)
    if rx_pos is not None:
        xyz = np.asarray(rx_pos.detach().cpu() if torch.is_tensor(rx_pos) else rx_pos,
                         dtype=np.float64).reshape(-1, 3)
        np.save(path, np.concatenate([xyz, dbm[:, None]], axis=1))
    else:
        np.save(path, dbm)


class Scene:
    """A scene on one GPU: static geometry (with its BVH), per-frame
    dynamic state, scratch buffers.  Wraps ``emrt_scene``."""

    def __init__(self, scene, device=None, max_rx: Optional[int] = None,
                 max_tx: Optional[int] = None, rebuild_every: int = 1, stream=None):
        self.lib = N.load()
        self.device = torch.device(device if device is not None else "cuda")
        self.desc = scene
        d = self.device
        self._static = dict(
            off=_u32(scene.face_off, d), xyz=_dev(scene.face_xyz, torch.float32, d),
            mat=_u32(scene.face_mat, d), tri=_dev(scene.tri_xyz, torch.float32, d),
            tface=_u32(scene.tri_face, d), half=_dev(scene.veh_half, torch.float32, d))
        s = self._static
        fr0 = scene.frame(0)
        self.max_rx = int(max_rx or len(fr0.rx_pos))
        self.max_tx = int(max_tx or len(fr0.tx_pos))
        desc = N.SceneDesc(scene.n_static_faces, _ptr(s["off"]), _ptr(s["xyz"]), _ptr(s["mat"]),
                           int(scene.tri_xyz.shape[0]), _ptr(s["tri"]), _ptr(s["tface"]),
                           scene.n_vehicles, _ptr(s["half"]), int(scene.veh_mat),
                           self.max_rx, self.max_tx, int(rebuild_every))
        h = C.c_void_p()
        torch.cuda.synchronize(d)
        N.check(self.lib.emrt_scene_create(C.byref(desc), _stream(stream), C.byref(h)),
                "emrt_scene_create")
        self.h = h
        self.n_rx = self.n_tx = 0
        self.materials(scene.eps_r, scene.sigma, scene.gamma)
        self._frame = None

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            try:
                torch.cuda.synchronize(self.device)
            except Exception:
                pass
            self.lib.emrt_scene_destroy(h)
            self.h = None

    # ------------------------------------------------------------------
    def materials(self, eps_r, sigma, gamma=None):
        d = self.device
        self.eps_r = _dev(eps_r, torch.float64, d)
        self.sigma = _dev(sigma, torch.float64, d)
        self.gamma = _dev(gamma if gamma is not None else np.zeros(len(eps_r)), torch.float64, d)

    def _mat(self, const_gamma=False, eps_r=None, sigma=None):
        e = self.eps_r if eps_r is None else eps_r
        s = self.sigma if sigma is None else sigma
        return N.Materials(int(e.numel()), _ptr(e), _ptr(s), _ptr(self.gamma), int(const_gamma))

    def update(self, frame, stream=None):
        """Per-frame dynamic state from a scenes.Frame (numpy or torch)."""
        d = self.device
        t = {k: _dev(getattr(frame, k), torch.float32, d)
             for k in ("veh_pos", "veh_vel", "rx_pos", "rx_vel", "tx_pos", "tx_vel")}
        self._frame = t
        self.n_rx, self.n_tx = int(t["rx_pos"].shape[0]), int(t["tx_pos"].shape[0])
        N.check(self.lib.emrt_scene_update_dynamic(
            self.h, _ptr(t["veh_pos"]), _ptr(t["veh_vel"]), _ptr(t["rx_pos"]), _ptr(t["rx_vel"]),
            self.n_rx, _ptr(t["tx_pos"]), _ptr(t["tx_vel"]), self.n_tx, _stream(stream)),
            "emrt_scene_update_dynamic")

    def set_transmitters(self, tx_pos, stream=None):
        """Moves the transmitters to tx_pos (rounded to float32), keeping the
        rest of the current frame; no call when they are already there."""
        t = _dev(tx_pos, torch.float32, self.device).reshape(-1, 3).contiguous()
        if t.shape == self._frame["tx_pos"].shape and torch.equal(t, self._frame["tx_pos"]):
            return
        fr = dict(self._frame)
        fr["tx_pos"] = t
        self.update(type("Frame", (), fr), stream)

    def trace_async(self, out: Paths, n_rays=None, max_depth=None, offset=0, stride=1, count=0,
                    keep_rejected=False, sort_rays=True, stream=None, wide_bvh=False,
                    static_cache=False, breadth_first=False):
        """Plain discovery into out (no sync).  static_cache: reuse the static
        closest hits of earlier calls with this ray set; breadth_first: trace
        bounce by bounce (sort_rays applies to that form) instead of
        depth-first chains; wide_bvh: static closest hits through the
        compressed 8-wide tree.  Identical output either way."""
        p = N.TraceParams(int(self.desc.max_depth if max_depth is None else max_depth),
                          int(self.desc.n_rays if n_rays is None else n_rays), int(offset),
                          int(stride), int(count),
                          (N.TRACE_KEEP_REJECTED if keep_rejected else 0) |
                          (N.TRACE_SORT_RAYS if sort_rays else 0) |
                          (N.TRACE_WIDE_BVH if wide_bvh else 0) |
                          (N.TRACE_STATIC_CACHE if static_cache else 0) |
                          (N.TRACE_BREADTH_FIRST if breadth_first else 0))
        pc = out.c()
        N.check(self.lib.emrt_trace(self.h, C.byref(p), C.byref(pc), _stream(stream)),
                "emrt_trace")

    def trace(self, n_rays=None, max_depth=None, offset=0, stride=1, count=0,
              keep_rejected=False, capacity=None, stream=None, retries=3,
              sort_rays=True, wide_bvh=False, static_cache=False,
              breadth_first=False) -> Paths:
        """Plain discovery; grows scratch and output on capacity errors."""
        return self._retry(lambda out: self.trace_async(
            out, n_rays, max_depth, offset, stride, count, keep_rejected, sort_rays=sort_rays,
            stream=stream, wide_bvh=wide_bvh, static_cache=static_cache,
            breadth_first=breadth_first), capacity, stream, retries, "emrt_trace")

    def trace_backward_async(self, out: Paths, rx_ids: Optional[torch.Tensor] = None,
                             n_rays=None, max_depth=None, offset=0, stride=1, count=0,
                             keep_rejected=False, sort_rays=True, stream=None,
                             breadth_first=False, wide_bvh=False):
        """Backward discovery from the receivers rx_ids (device int tensor;
        None = every receiver); paths come out in forward orientation."""
        p = N.TraceParams(int(self.desc.max_depth if max_depth is None else max_depth),
                          int(self.desc.n_rays if n_rays is None else n_rays), int(offset),
                          int(stride), int(count),
                          (N.TRACE_KEEP_REJECTED if keep_rejected else 0) |
                          (N.TRACE_SORT_RAYS if sort_rays else 0) |
                          (N.TRACE_WIDE_BVH if wide_bvh else 0) |
                          (N.TRACE_BREADTH_FIRST if breadth_first else 0))
        ids, n_ids = None, 0
        if rx_ids is not None:
            ids = rx_ids.to(device=self.device, dtype=torch.int32).contiguous()
            n_ids = int(ids.numel())
            if n_ids == 0:  # an empty tensor has no address to pass
                raise N.EmrtError(1, "emrt_trace_backward: empty receiver list")
            self._keep_ids = ids  # alive until the stream has used it
        pc = out.c()
        N.check(self.lib.emrt_trace_backward(self.h, C.byref(p), _ptr(ids) if ids is not None
                                             else None, n_ids, C.byref(pc), _stream(stream)),
                "emrt_trace_backward")

    def trace_backward(self, rx_ids: Optional[torch.Tensor] = None, n_rays=None, max_depth=None,
                       offset=0, stride=1, count=0, keep_rejected=False, capacity=None,
                       stream=None, retries=3, sort_rays=True,
                       breadth_first=False, wide_bvh=False) -> Paths:
        """Backward discovery; grows scratch and output on capacity errors."""
        return self._retry(lambda out: self.trace_backward_async(
            out, rx_ids, n_rays, max_depth, offset, stride, count, keep_rejected,
            sort_rays=sort_rays, stream=stream, breadth_first=breadth_first, wide_bvh=wide_bvh),
            capacity, stream, retries, "emrt_trace_backward")

    def _retry(self, launch, capacity, stream, retries, name) -> Paths:
        cap = capacity or max(4096, 8 * self.n_tx * self.n_rx)
        for _ in range(retries + 1):
            out = Paths(cap, self.device)
            launch(out)
            try:
                self.last_stats = self.sync(stream)
                return out
            except N.EmrtError as e:
                if e.code != 4:
                    raise
                cap = max(cap, int(out.n()) + 1024)
        raise N.EmrtError(4, name + " (after retries)")

    def rediscover(self, cache: Paths, n_rays=None, max_depth=None, offset=0, stride=1, count=0,
                   sort_rays=True, stream=None, static_cache=False, breadth_first=False,
                   revalidate=False):
        """cache <- cache | accepted paths of a discovery with this ray set
        (no sync).  The cache must have been revalidated with the current
        poses (revalidate=True: done by this call, on a side stream during
        the discovery): the candidates it holds are not validated again.
        Same records as revalidate, trace_async into a separate output and
        merge."""
        p = N.TraceParams(int(self.desc.max_depth if max_depth is None else max_depth),
                          int(self.desc.n_rays if n_rays is None else n_rays), int(offset),
                          int(stride), int(count),
                          (N.TRACE_SORT_RAYS if sort_rays else 0) |
                          (N.TRACE_STATIC_CACHE if static_cache else 0) |
                          (N.TRACE_BREADTH_FIRST if breadth_first else 0) |
                          (N.TRACE_REVALIDATE_FIRST if revalidate else 0))
        pc = cache.c()
        N.check(self.lib.emrt_rediscover(self.h, C.byref(p), C.byref(pc), _stream(stream)),
                "emrt_rediscover")

    def revalidate(self, cache: Paths, keep=False, stream=None):
        pc = cache.c()
        N.check(self.lib.emrt_revalidate(self.h, C.byref(pc),
                                         N.REVALIDATE_KEEP if keep else 0, _stream(stream)),
                "emrt_revalidate")

    def revalidate_cache(self, cache: Paths, stream=None) -> torch.Tensor:
        """revalidate (invalid paths removed); returns the device count of
        records evicted."""
        ev = torch.zeros(1, dtype=torch.int32, device=self.device)
        pc = cache.c()
        N.check(self.lib.emrt_revalidate_cache(self.h, C.byref(pc), _ptr(ev), _stream(stream)),
                "emrt_revalidate_cache")
        return ev

    def merge(self, cache: Paths, fresh: Paths, stream=None):
        a, b = cache.c(), fresh.c()
        N.check(self.lib.emrt_cache_merge(self.h, C.byref(a), C.byref(b), _stream(stream)),
                "emrt_cache_merge")

    def channel(self, paths: Paths, freq: float, tx_power_w: Optional[float] = None,
                const_gamma=False, eps_r=None, sigma=None, out: Optional[ChannelResult] = None,
                stream=None) -> ChannelResult:
        d = self.device
        if out is None:
            out = ChannelResult(
                torch.empty((max(paths.capacity, 1), 4), dtype=torch.float64, device=d),
                torch.empty((self.n_tx, self.n_rx, 8), dtype=torch.float64, device=d),
                torch.empty((self.n_rx, 2), dtype=torch.float64, device=d))
        m = self._mat(const_gamma, eps_r, sigma)
        co = N.ChannelOut(out.path.data_ptr(), out.pair.data_ptr(), out.rx.data_ptr())
        pc = paths.c()
        pt = self.desc.tx_power_w if tx_power_w is None else tx_power_w
        N.check(self.lib.emrt_channel(self.h, C.byref(pc), C.byref(m), float(freq), float(pt),
                                      C.byref(co), _stream(stream)), "emrt_channel")
        return out

    def channels(self, paths: Paths, freqs, tx_power_w: Optional[float] = None,
                 const_gamma=False, eps_r=None, sigma=None, outs=None,
                 stream=None) -> list:
        """channel() at several frequencies in one pass (emrt_channel_multi);
        outs: optional list of ChannelResult to reuse."""
        d = self.device
        freqs = [float(f) for f in freqs]
        outs = list(outs) if outs is not None else [None] * len(freqs)
        for q, o in enumerate(outs):
            if o is None:
                outs[q] = ChannelResult(
                    torch.empty((max(paths.capacity, 1), 4), dtype=torch.float64, device=d),
                    torch.empty((self.n_tx, self.n_rx, 8), dtype=torch.float64, device=d),
                    torch.empty((self.n_rx, 2), dtype=torch.float64, device=d))
        m = self._mat(const_gamma, eps_r, sigma)
        cos = (N.ChannelOut * len(freqs))(*[N.ChannelOut(o.path.data_ptr(), o.pair.data_ptr(),
                                                          o.rx.data_ptr()) for o in outs])
        fa = (C.c_double * len(freqs))(*freqs)
        pc = paths.c()
        pt = self.desc.tx_power_w if tx_power_w is None else tx_power_w
        N.check(self.lib.emrt_channel_multi(self.h, C.byref(pc), C.byref(m), fa, len(freqs),
                                            float(pt), cos, _stream(stream)), "emrt_channel_multi")
        return outs

    def channel_backward(self, paths: Paths, freq: float, dloss_dh: torch.Tensor,
                         const_gamma=False, eps_r=None, sigma=None, stream=None):
        d = self.device
        m = self._mat(const_gamma, eps_r, sigma)
        ge = torch.empty(int(m.n_mat), dtype=torch.float64, device=d)
        gs = torch.empty_like(ge)
        gt = torch.empty((self.n_tx, 3), dtype=torch.float64, device=d)
        g = dloss_dh.to(device=d, dtype=torch.float64).contiguous()
        pc = paths.c()
        N.check(self.lib.emrt_channel_backward(self.h, C.byref(pc), C.byref(m), float(freq),
                                               _ptr(g), _ptr(ge), _ptr(gs), _ptr(gt),
                                               _stream(stream)), "emrt_channel_backward")
        return ge, gs, gt

    def coherence_time(self, freq: float, r_threshold: float = 0.5, stream=None) -> torch.Tensor:
        """Eq. 2 coherence time (s) per (tx, rx) for the current frame."""
        tc = torch.empty((self.n_tx, self.n_rx), dtype=torch.float64, device=self.device)
        N.check(self.lib.emrt_coherence_time(self.h, float(freq), float(r_threshold),
                                             _ptr(tc), _stream(stream)), "emrt_coherence_time")
        return tc

    def refresh_schedule(self, sched: "RefreshSchedule", stream=None):
        """Due receivers of this frame (emrt_refresh_schedule): fills
        sched.ids[:n] and sched.n_due (device) and updates sched's state."""
        N.check(self.lib.emrt_refresh_schedule(
            self.h, _ptr(sched.state), _ptr(sched.los_ref), float(sched.freq),
            float(sched.r_threshold), float(sched.dt), float(sched.d_seg),
            int(sched.max_interval), _ptr(sched.ids), _ptr(sched.n_due), _stream(stream)),
            "emrt_refresh_schedule")

    def refresh_interval(self, freq: float, dt: float, r_threshold: float = 0.5,
                         quantile: float = 0.5) -> int:
        """Frames a cached path set stays within the coherence time:
        max(1, floor(T_c / dt)) with T_c the given quantile over the pairs."""
        tc = self.coherence_time(freq, r_threshold).flatten()
        q = float(torch.quantile(tc[torch.isfinite(tc)], quantile)) if torch.isfinite(tc).any() \
            else float("inf")
        return max(1, int(q // dt)) if q != float("inf") else 1 << 30

    def sync(self, stream=None) -> dict:
        st = N.Stats()
        code = self.lib.emrt_sync(self.h, _stream(stream), C.byref(st))
        out = {f: getattr(st, f) for f, _ in N.Stats._fields_}
        out["segments"] = list(st.segments)
        self.last_stats = out
        N.check(code, "emrt_sync")
        return out


class RefreshSchedule:
    """Caller-owned state of the per-receiver re-discovery schedule: each
    receiver's position and frame count at its last discovery and the LoS
    condition of its pairs then (device tensors), with the rule's
    parameters: segment length d_seg (m), Eq. 2 frequency and correlation
    threshold, frame interval dt (s) and the longest reuse in frames."""

    def __init__(self, n_tx: int, n_rx: int, device, freq: float, dt: float,
                 d_seg: float = 10.0, r_threshold: float = 0.5, max_interval: int = 50):
        self.state = torch.full((n_rx, 4), -1.0, dtype=torch.float32, device=device)
        self.los_ref = torch.zeros((n_tx, n_rx), dtype=torch.uint8, device=device)
        self.ids = torch.zeros(n_rx, dtype=torch.int32, device=device)
        self.n_due = torch.zeros(1, dtype=torch.int32, device=device)
        self.freq, self.dt, self.d_seg = freq, dt, d_seg
        self.r_threshold, self.max_interval = r_threshold, max_interval

    def due(self) -> torch.Tensor:
        """Due receiver ids of the last call (synchronises on the count)."""
        return self.ids[:int(self.n_due.item())]


class Batch:
    """Batched discovery over several Scenes (wraps ``emrt_batch``):
    traversal launches over all scenes (depth-first by default, one launch per
    bounce with breadth_first), replayed from a CUDA graph."""

    def __init__(self, scenes, params=None, capacity=None, autotune=False, stream=None,
                 breadth_first=False):
        self.lib = N.load()
        self.scenes = list(scenes)
        n = len(self.scenes)
        self.device = self.scenes[0].device
        self.outs = []
        ps = []
        for i, sc in enumerate(self.scenes):
            p = dict(n_rays=sc.desc.n_rays, max_depth=sc.desc.max_depth, offset=0, stride=1,
                     count=0)
            if params is not None:
                p.update(params[i])
            ps.append(N.TraceParams(int(p["max_depth"]), int(p["n_rays"]), int(p["offset"]),
                                    int(p["stride"]), int(p["count"]), 0))
            cap = capacity[i] if isinstance(capacity, (list, tuple)) else \
                (capacity or max(4096, 8 * sc.n_tx * sc.n_rx))
            self.outs.append(Paths(cap, self.device))
        self._params = (N.TraceParams * n)(*ps)
        self._outs = (N.PathsC * n)(*[o.c() for o in self.outs])
        self._scenes = (C.c_void_p * n)(*[sc.h.value for sc in self.scenes])
        h = C.c_void_p()
        N.check(self.lib.emrt_batch_create(self._scenes, n, self._params, self._outs,
                                           (N.BATCH_AUTOTUNE if autotune else 0) |
                                           (N.BATCH_BREADTH_FIRST if breadth_first else 0),
                                           _stream(stream),
                                           C.byref(h)), "emrt_batch_create")
        self.h = h

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            try:
                torch.cuda.synchronize(self.device)
            except Exception:
                pass
            self.lib.emrt_batch_destroy(h)
            self.h = None

    def trace_async(self, stream=None):
        N.check(self.lib.emrt_batch_trace(self.h, _stream(stream)), "emrt_batch_trace")

    def sync(self, stream=None) -> dict:
        st = N.Stats()
        code = self.lib.emrt_batch_sync(self.h, _stream(stream), C.byref(st))
        out = {f: getattr(st, f) for f, _ in N.Stats._fields_}
        out["segments"] = list(st.segments)
        N.check(code, "emrt_batch_sync")
        return out

    def config(self) -> str:
        buf = C.create_string_buffer(128)
        N.check(self.lib.emrt_batch_config(self.h, buf, 128), "emrt_batch_config")
        return buf.value.decode()


def trace_batched(scenes, outs, params=None, stream=None):
    """One-call batched discovery (emrt_trace_batched) into the caller's Paths
    outs[i]; the graph is captured on the first call with these scenes,
    params and outputs and replayed afterwards.  Synchronises."""
    lib = N.load()
    n = len(scenes)
    ps = []
    for i, sc in enumerate(scenes):
        p = dict(n_rays=sc.desc.n_rays, max_depth=sc.desc.max_depth, offset=0, stride=1,
                 count=0)
        if params is not None:
            p.update(params[i])
        ps.append(N.TraceParams(int(p["max_depth"]), int(p["n_rays"]), int(p["offset"]),
                                int(p["stride"]), int(p["count"]), 0))
    hs = (C.c_void_p * n)(*[sc.h for sc in scenes])
    pa = (N.TraceParams * n)(*ps)
    oa = (N.PathsC * n)(*[o.c() for o in outs])
    N.check(lib.emrt_trace_batched(hs, n, pa, oa, _stream(stream)), "emrt_trace_batched")
    return outs


def channel_correlation(h_series: torch.Tensor, max_lag: int, stream=None) -> torch.Tensor:
    """Eq. 1 over frames: h_series [n_frames, n_pairs, 2] float64 (device) ->
    R [n_pairs, max_lag + 1]."""
    lib = N.load()
    h = h_series.to(torch.float64).contiguous()
    F, P = int(h.shape[0]), int(h.shape[1])
    R = torch.empty((P, max_lag + 1), dtype=torch.float64, device=h.device)
    N.check(lib.emrt_channel_correlation(_ptr(h), F, P, int(max_lag), _ptr(R), _stream(stream)),
            "emrt_channel_correlation")
    return R
