"""UAV streams through the serving form (pilot_serve_*): the localisation stage of the online
system (Supp. "Runtime Analysis") for many concurrent streams on one GPU.

For every frame of a stream the client makes, on the device, the reference crop around the
stream's previous estimate (pilot_crop_reference: every valid crop pixel a geo-anchor), takes
the frame's features from the network (`StreamNetwork`, the feature extractor's stand-in),
stores them as BF16 (pilot_quantize_features), writes the hypothesis grid around the
previous estimate (pilot_seed_hypotheses), and submits the frame; the server admits it when
a slot, hypothesis room and arena memory are free and runs it with whatever else it is
serving.  The frames due at one time are prepared together (one network pass per query
pyramid for all of them) on a high-priority stream; a server that leaves a few SMs outside
its rounds (pilot_serve_set_reserved_sms) lets this work run beside a round instead of after
it, as the paper's map-preparation and localisation threads run side by side.  A stream has at most one frame in the server: when its result arrives, the
client takes the stream's newest arrived frame and drops the ones that arrived meanwhile
(a tracker keeps the latest image), so latency stays bounded under overload and the
completed rate is the sustainable one.  This module only orders the library calls and
keeps the statistics.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field
from types import SimpleNamespace

import numpy as np

from . import binding as B


@dataclass
class StreamState:
    gt: np.ndarray                     # (n_frames, 12) ground truth, world -> camera
    sensors: list                      # per frame (gravity in the camera frame, laser range)
    arrivals: np.ndarray               # arrival time of each frame, seconds from the start
    estimate: np.ndarray               # latest estimate (world); the first frame starts from its truth
    next_t: int = 0                    # first frame not yet accounted for (completed, dropped or failed)
    in_flight: tuple | None = None     # (ticket, t, arrival, keep-alive)
    done: list = field(default_factory=list)


def grid_values(n: int, span: float) -> tuple:
    """n values evenly spread over [-span, span] (n = 1: 0)."""
    if n == 1:
        return (0.0,)
    return tuple(float(v) for v in np.linspace(-span, span, n))


class StreamClient:
    """Prepares and submits stream frames (see the module docstring)."""

    def __init__(self, server: B.Server, gmap, dsm_dev, sc, network, cam, ray_step: float = 0.25,
                 ray_samples: int = 12000, dsm_window: int = 1024):
        import torch
        self.torch = torch
        self.server, self.gmap, self.sc, self.net, self.cam = server, gmap, sc, network, cam
        self.dsm_dev = dsm_dev
        self.map = B.MapArgs(dsm_dev, None, gmap.x0, gmap.y0, gmap.gsd)
        self.ray_step, self.ray_samples, self.win = ray_step, ray_samples, dsm_window
        self.bank16 = [[B.quantize_features(q, B.BF16)[0] for q in pyr] for pyr in network.bank32]
        torch.cuda.synchronize()
        # frames are prepared on a high-priority stream, so that their small kernels are
        # dispatched ahead of the server's queued level launches
        self.stream = torch.cuda.Stream(priority=-1)

    def _dsm_window(self, T_prev: np.ndarray, origin):
        """A window of the global DSM for the range prior: win x win cells centred where the
        previous estimate's optical axis meets the plane at the DSM height under the crop
        origin (the laser point of the frame lies well inside it)."""
        g = self.gmap
        A = np.asarray(T_prev, np.float64).reshape(3, 4)
        R, t = A[:, :3], A[:, 3]
        C, d = -R.T @ t, R[2]
        side = g.dsm.shape[0]
        oc = int(np.clip((origin[0] - g.x0) / g.gsd, 0, side - 1))
        orr = int(np.clip((origin[1] - g.y0) / g.gsd, 0, side - 1))
        h = float(g.dsm[orr, oc])
        s = (h - C[2]) / d[2] if d[2] < -1e-6 else 0.0
        px, py = C[0] + s * d[0], C[1] + s * d[1]
        c0 = int(np.clip((px - g.x0) / g.gsd - self.win // 2, 0, side - self.win))
        r0 = int(np.clip((py - g.y0) / g.gsd - self.win // 2, 0, side - self.win))
        return self.dsm_dev[r0:r0 + self.win, c0:c0 + self.win].contiguous(), g.x0 + c0 * g.gsd, g.y0 + r0 * g.gsd

    def prepare(self, sid: int, st: StreamState, t: int):
        """Frame t of stream sid around the stream's current estimate: (FrameArgs, origin,
        keep-alive) or None when the crop fails."""
        return self.prepare_batch([(sid, st, t)])[0]

    def prepare_batch(self, jobs: list) -> list:
        """prepare() for several (stream id, state, frame) at once, with one host wait for all
        the crops' geometry and one before the frames are handed to the server."""
        from . import scenes as S
        torch = self.torch
        sc, cam = self.sc, self.cam
        out = []
        with torch.cuda.stream(self.stream):
            crops = []
            for sid, st, t in jobs:
                side, n_xy, n_yaw = S.stream_frame_shape(sc, sid, t)
                p = B.crop_params(st.estimate, cam.fx, cam.fy, cam.cx, cam.cy, cam.img_w, cam.img_h, 0.0,
                                  self.ray_step, self.ray_samples, side)
                crop = B.crop_reference(self.map, p, with_rgb=False, stream=self.stream)
                crops.append((crop, (n_xy, n_yaw)))
            geos = torch.stack([c["geometry"] for c, _ in crops]).cpu().numpy()   # one wait for all
            # the frames whose crop succeeded, described together by the network
            keep = [k for k, geo in enumerate(geos) if geo[27] == 1.0]
            items = []
            for k in keep:
                sid, st, t = jobs[k]
                ox, oy = float(geos[k][9]), float(geos[k][10])
                items.append((t % len(self.bank16), crops[k][0]["points"], B.pose_reorigin(st.gt[t], ox, oy),
                              (sid << 20) + t))
            described = dict(zip(keep, self.net.descriptors_batch(items)))
            for k, ((sid, st, t), (crop, (n_xy, n_yaw)), geo) in enumerate(zip(jobs, crops, geos)):
                if k not in described:
                    out.append(None)
                    continue
                ox, oy = float(geo[9]), float(geo[10])
                prior = st.estimate
                b = t % len(self.bank16)
                refs32 = described[k]
                refs16 = [B.quantize_features(r, B.BF16, stream=self.stream)[0] for r in refs32]
                seeds = B.seed_hypotheses(B.seed_params(prior, grid_values(n_xy, sc.xy_span),
                                                        grid_values(n_yaw, sc.yaw_span_deg), (ox, oy)),
                                          stream=self.stream)
                dsm, wx0, wy0 = self._dsm_window(prior, (ox, oy))
                g_cam, rng = st.sensors[t]
                scal = SimpleNamespace(fx=cam.fx, fy=cam.fy, cx=cam.cx, cy=cam.cy, use_gravity=True,
                                       gravity_cam=g_cam, gravity_world=np.array([0.0, 0.0, -1.0]),
                                       w_grav=sc.w_grav, use_range=True, range_m=rng, w_range=sc.w_range,
                                       dsm_x0=wx0 - ox, dsm_y0=wy0 - oy, dsm_gsd=self.gmap.gsd)
                arrays = dict(points=crop["points"], point_valid=crop["valid"], point_weight=None,
                              ref_feat=refs16, qry_feat=self.bank16[b], T_cw=seeds, dsm=dsm)
                out.append((B.FrameArgs(scal, arrays, is_device=True, dtype=B.BF16), (ox, oy), (crop, refs32)))
        self.stream.synchronize()          # the server stages the frames on its own stream
        return out

    def run(self, streams: list, duration_s: float, poll_s: float = 0.0005) -> dict:
        """Serve `streams` for duration_s seconds of arrivals (then drain the frames in the
        server); returns the statistics of the completed frames."""
        t0 = time.perf_counter()
        lat, srv_lat, units, dropped, crop_failed, rejected = [], [], 0, 0, 0, 0
        prep_s = 0.0                          # host time spent preparing frames
        errs = []
        pending = {}                          # sid -> prepared frame waiting for admission
        while True:
            now = time.perf_counter() - t0
            active = False
            # the newest arrived frame of every stream with nothing in the server, prepared
            # together
            due = []
            for sid, st in enumerate(streams):
                if st.in_flight is not None or now > duration_s:
                    continue
                k = int(np.searchsorted(st.arrivals, now, side="right")) - 1
                if st.next_t <= k < len(st.arrivals) and (sid not in pending or pending[sid][0] != k):
                    due.append((sid, st, k))
            if due:
                tp = time.perf_counter()
                prepared = self.prepare_batch(due)
                prep_s += time.perf_counter() - tp
                for (sid, st, k), prep in zip(due, prepared):
                    # frames next_t .. k - 1 are dropped (among them a prepared frame that was
                    # waiting for admission); frame k is accounted for from here on
                    dropped += k - st.next_t
                    st.next_t = k
                    if prep is None:
                        crop_failed += 1
                        st.next_t = k + 1
                        pending.pop(sid, None)
                        continue
                    pending[sid] = (k, prep)
            for sid, st in enumerate(streams):
                if st.in_flight is not None:
                    active = True
                    tk, t, arr, keep = st.in_flight
                    ok, r, l_ = self.server.poll(tk)
                    if ok:
                        st.in_flight = None
                        lat.append(1e3 * (time.perf_counter() - t0 - arr))
                        srv_lat.append(l_)
                        units += r.hyp_iters
                        if r.best >= 0:
                            est = B.pose_reorigin(r.T_cw[r.best], -keep[1][0], -keep[1][1])
                            st.estimate = est
                            A, G = est.reshape(3, 4), st.gt[t].reshape(3, 4)
                            errs.append(float(np.linalg.norm(A[:, :3].T @ A[:, 3] - G[:, :3].T @ G[:, 3])))
                        st.done.append(t)
                    continue
                if now > duration_s:
                    continue
                # newest frame that has arrived; the ones before it are dropped
                k = int(np.searchsorted(st.arrivals, now, side="right")) - 1
                if k < st.next_t or k >= len(st.arrivals):
                    active = active or k < len(st.arrivals)
                    continue
                active = True
                if sid not in pending:
                    continue
                k, (fa, origin, keep) = pending[sid]
                try:
                    tk = self.server.submit(fa)
                except B.PilotError as e:
                    if e.status != B.PILOT_EBUSY:
                        raise
                    rejected += 1
                    continue
                del pending[sid]
                st.in_flight = (tk, k, float(st.arrivals[k]), (keep, origin, fa))
                st.next_t = k + 1
            if not active and all(st.in_flight is None for st in streams):
                break
            time.sleep(poll_s)
        span = time.perf_counter() - t0
        n_done = len(lat)
        offered = sum(int(np.searchsorted(st.arrivals, duration_s, side="right")) for st in streams)
        pct = lambda a, q: float(np.percentile(a, q)) if a else None
        return {"streams": len(streams), "duration_s": duration_s, "span_s": span, "offered_frames": offered,
                "completed_frames": n_done, "dropped_frames": dropped, "crop_failed": crop_failed,
                "ebusy_retries": rejected, "offered_fps": offered / duration_s, "completed_fps": n_done / span,
                "hyp_iter_per_s": units / span, "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99),
                "server_p50_ms": pct(srv_lat, 50), "server_p99_ms": pct(srv_lat, 99),
                "client_prepare_busy": prep_s / span,
                "median_error_m": float(np.median(errs)) if errs else None}
