"""Serving: continuous batching of log-likelihood and kriging requests over
resident datasets.

Each dataset's locations, observations and a factor of its covariance at a
fitted theta stay resident on the device.  Log-likelihood requests (a dataset
and a theta) need a tile store of their own for the factorization; kriging
requests (a dataset and new locations) use the resident factor.

The request loop runs in real time and keeps several launches on the device
at once:

* The SMs are split into `lanes` shares, each with its own stream.  Whenever a
  lane is free, the queued log-likelihood requests whose stores fit the HBM
  budget are admitted together and evaluated in one batched persistent launch
  on that lane's share of the SMs (geo.Batch with `ctas`): their tasks share
  the launch's queues and overlap on its SMs.  Requests that arrive while a
  launch is on the device join the next free lane at once, so a short request
  does not wait for a long one to finish, and its work overlaps the long one's
  on the device.
* Kriging requests run as soon as they arrive, on a stream of their own,
  beside the likelihood launches.
* HBM budget: the resident kriging factors, every tile store (pooled or busy)
  and every in-flight launch's workspace count against it.  Stores are pooled
  per dataset; free stores of other datasets are released when the budget
  needs room.  A request whose store can never fit beside the resident factors
  is rejected; one that fits later waits in the queue.

Per request the arithmetic is that of the single-problem path, so every result
is the same alone and in any mix.
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass

import numpy as np

from . import geo


@dataclass
class Request:
    kind: str                      # "loglik" or "krige"
    dataset: int
    theta: geo.Theta = None        # loglik
    xnew: np.ndarray = None        # krige: new locations (host arrays)
    ynew: np.ndarray = None
    t_arrival: float = 0.0         # seconds after the start of the run
    id: int = -1


@dataclass
class Result:
    id: int
    kind: str
    dataset: int
    value: object                  # (l, log|Sigma|, Q) or predictions
    t_arrival: float
    t_admit: float
    t_done: float
    batch: int
    status: int = 0
    lane: int = -1                 # the lane of a likelihood launch (-1: kriging stream)

    @property
    def latency(self):
        return self.t_done - self.t_arrival


def store_bytes(n: int, nb: int, band: int) -> int:
    lay = geo.layout(n, nb, band, geo.GEO_LP_SPLIT_BF16)
    return int(lay.bytes_dp + lay.bytes_sp + lay.bytes_planes + lay.bytes_meta)


class Server:
    def __init__(self, datasets, hbm_budget_bytes: int, nb: int = 256, band: int = 1, max_batch: int = 256,
                 lanes: int = 2, device="cuda"):
        """datasets: list of dicts with host arrays x, y, z (Morton-ordered), the
        theta of the resident kriging factor, optional per-dataset nb and
        krige=False to keep no resident factor (log-likelihood requests only).
        lanes: concurrent likelihood launches, each on an equal share of the SMs
        (at most SM count / GEO_MIN_CTAS lanes)."""
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.budget = int(hbm_budget_bytes)
        self.band = band
        self.max_batch = max_batch
        self.ds = []
        for d in datasets:
            nbd = int(d.get("nb", nb))
            X, Y, Z = (torch.as_tensor(np.ascontiguousarray(d[k]), dtype=torch.float64, device=self.device)
                       for k in ("x", "y", "z"))
            n = int(Z.shape[0])
            krig = None
            if d.get("krige", True):
                krig = geo.TileStore(n, nbd, band, geo.GEO_LP_SPLIT_BF16, device=self.device)
                krig.matern(X, Y, d["theta"])
                try:
                    krig.potrf()
                except geo.NotSPDError:
                    krig = None        # no resident factor: its kriging requests are rejected
            self.ds.append(dict(x=X, y=Y, z=Z, n=n, nb=nbd, theta=d["theta"], krig=krig,
                                bytes=store_bytes(n, nbd, band)))
        self.resident_bytes = sum(d["bytes"] for d in self.ds if d["krig"] is not None)
        self.pool = collections.defaultdict(list)      # dataset -> free stores
        self.allocated = self.resident_bytes           # resident factors + pooled/busy stores + workspaces
        nsm = torch.cuda.get_device_properties(self.device).multi_processor_count
        self.nlanes = max(1, min(int(lanes), nsm // geo.GEO_MIN_CTAS))   # each share >= GEO_MIN_CTAS SMs
        share = [nsm // self.nlanes + (1 if q < nsm % self.nlanes else 0) for q in range(self.nlanes)]
        self.lanes = [dict(stream=torch.cuda.Stream(device=self.device),
                           ctas=0 if self.nlanes == 1 else share[q], inflight=None) for q in range(self.nlanes)]
        self.krige_stream = torch.cuda.Stream(device=self.device)
        self.batches = 0

    # ---- store pool -------------------------------------------------------
    def _take_store(self, dsi):
        d = self.ds[dsi]
        if self.pool[dsi]:
            return self.pool[dsi].pop()
        need = d["bytes"]
        if need > self.budget - self.resident_bytes:
            return "reject"                      # can never fit beside the resident factors
        while self.allocated + need > self.budget:
            victim = next((k for k, v in self.pool.items() if v and k != dsi), None)
            if victim is None:
                return None                      # wait for busy stores to come back
            self.pool[victim].pop()
            self.allocated -= self.ds[victim]["bytes"]
        self.allocated += need
        return geo.TileStore(d["n"], d["nb"], self.band, geo.GEO_LP_SPLIT_BF16, device=self.device)

    def _give_back(self, dsi, ts):
        self.pool[dsi].append(ts)

    # ---- launches -----------------------------------------------------------
    def _launch_lik(self, lane, reqs, now):
        torch = self.torch
        with torch.cuda.stream(lane["stream"]):
            probs = [dict(x=self.ds[r.dataset]["x"], y=self.ds[r.dataset]["y"], z=self.ds[r.dataset]["z"],
                          store=s) for r, s in reqs]
            batch = geo.Batch(probs, device=self.device, ctas=lane["ctas"])
            batch.set_theta([r.theta for r, _ in reqs])
            batch.loglik_async(lane["stream"])
            ev = torch.cuda.Event()
            ev.record(lane["stream"])
        self.allocated += batch.nbytes()
        self.batches += 1
        lane["inflight"] = dict(lik=reqs, batch=batch, event=ev, t_admit=now, id=self.batches)

    def _harvest_lik(self, q, lane, now, results):
        fl = lane["inflight"]
        out = fl["batch"].out.cpu().numpy()
        for b, (r, s) in enumerate(fl["lik"]):
            code, _ = s.status()
            results.append(Result(r.id, r.kind, r.dataset, tuple(out[b]), r.t_arrival, fl["t_admit"], now,
                                  fl["id"], code, q))
            self._give_back(r.dataset, s)
        self.allocated -= fl["batch"].nbytes()
        lane["inflight"] = None

    def _launch_krige(self, r, now):
        torch = self.torch
        d = self.ds[r.dataset]
        with torch.cuda.stream(self.krige_stream):
            xn = torch.as_tensor(np.ascontiguousarray(r.xnew), dtype=torch.float64, device=self.device)
            yn = torch.as_tensor(np.ascontiguousarray(r.ynew), dtype=torch.float64, device=self.device)
            z = d["krig"].krige(d["x"], d["y"], d["z"], d["theta"], xn, yn, stream=self.krige_stream)
            ev = torch.cuda.Event()
            ev.record(self.krige_stream)
        work = 8 * (2 * d["krig"].p * d["krig"].nb + 3 * len(r.xnew))   # solve scratch, new points, predictions
        self.allocated += work
        return dict(req=r, z=z, event=ev, t_admit=now, bytes=work)

    # ---- the request loop -------------------------------------------------
    def run(self, requests, admit_until: float = math.inf):
        """Serve `requests` (their t_arrival fields, seconds from now) in real time.
        Requests arriving after `admit_until` are not admitted (counted as
        queued).  Returns (results, stats)."""
        pending = collections.deque(sorted(requests, key=lambda r: r.t_arrival))
        queue = collections.deque()
        results, rejected, kinflight = [], [], []
        t0 = time.perf_counter()
        overlap = 0                               # launches admitted while another was on the device
        while True:
            now = time.perf_counter() - t0
            while pending and pending[0].t_arrival <= now:
                queue.append(pending.popleft())
            for q, lane in enumerate(self.lanes):
                if lane["inflight"] is not None and lane["inflight"]["event"].query():
                    self._harvest_lik(q, lane, time.perf_counter() - t0, results)
            while kinflight and kinflight[0]["event"].query():
                k = kinflight.pop(0)
                self.allocated -= k["bytes"]
                r = k["req"]
                results.append(Result(r.id, r.kind, r.dataset, k["z"].cpu().numpy(), r.t_arrival, k["t_admit"],
                                      time.perf_counter() - t0, 0, 0, -1))
            if now <= admit_until and queue:
                # kriging: at once, on its own stream
                keep = collections.deque()
                for r in queue:
                    if r.kind != "krige":
                        keep.append(r)
                    elif self.ds[r.dataset]["krig"] is None:
                        rejected.append(r)        # no resident factor for this dataset
                    else:
                        kinflight.append(self._launch_krige(r, now))
                queue = keep
                # likelihoods: into every free lane
                for lane in self.lanes:
                    if lane["inflight"] is not None or not queue:
                        continue
                    admitted, keep = [], collections.deque()
                    while queue and len(admitted) < self.max_batch:
                        r = queue.popleft()
                        s = self._take_store(r.dataset)
                        if s == "reject":
                            rejected.append(r)
                        elif s is None:
                            keep.append(r)
                        else:
                            admitted.append((r, s))
                    queue.extendleft(reversed(keep))
                    if admitted:
                        if any(ln["inflight"] is not None for ln in self.lanes) or kinflight:
                            overlap += 1
                        self._launch_lik(lane, admitted, now)
            busy = any(ln["inflight"] is not None for ln in self.lanes) or kinflight
            if not busy and (not queue or now > admit_until) and (not pending or now > admit_until):
                break
            nxt = pending[0].t_arrival - now if pending else 1e-3
            time.sleep(max(0.0, min(nxt, 2e-4)))
        wall = time.perf_counter() - t0
        lat = np.array([r.latency for r in results]) if results else np.zeros(0)
        nl = sum(1 for r in results if r.kind == "loglik")
        stats = dict(completed=len(results), loglik_completed=nl,
                     krige_completed=len(results) - nl, rejected=len(rejected),
                     queued=len(queue) + len(pending), launches=self.batches, lanes=self.nlanes,
                     launches_overlapping=overlap, wall_s=wall,
                     evals_per_s=nl / wall if wall > 0 else 0.0,
                     p50_ms=float(np.percentile(lat, 50) * 1e3) if lat.size else None,
                     p99_ms=float(np.percentile(lat, 99) * 1e3) if lat.size else None)
        return results, stats
