"""Serving: continuous batching of log-likelihood and kriging requests over
resident datasets.

Each dataset's locations, observations and a factor of its covariance at a
fitted theta stay resident on the device.  Log-likelihood requests (a dataset
and a theta) need a tile store of their own for the factorization; kriging
requests (a dataset and new locations) use the resident factor.  The request
loop runs in real time: arrivals join a queue; whenever the device is idle,
the queued log-likelihood requests whose stores fit the HBM budget are
admitted together and evaluated in one batched launch (geo.Batch: their tasks
share the device's queues and overlap on the SMs), the queued kriging requests
run right after on the same stream, and requests that arrive meanwhile wait
for the next launch.  Stores are pooled per dataset; free stores of other
datasets are released when the budget needs room.  A request whose store alone
exceeds the budget is rejected.
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field

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

    @property
    def latency(self):
        return self.t_done - self.t_arrival


def store_bytes(n: int, nb: int, band: int) -> int:
    lay = geo.layout(n, nb, band, geo.GEO_LP_SPLIT_BF16)
    return int(lay.bytes_dp + lay.bytes_sp + lay.bytes_planes + lay.bytes_meta)


class Server:
    def __init__(self, datasets, hbm_budget_bytes: int, nb: int = 256, band: int = 1, max_batch: int = 256,
                 device="cuda"):
        """datasets: list of dicts with host arrays x, y, z (Morton-ordered), the
        theta of the resident kriging factor, optional per-dataset nb and
        krige=False to keep no resident factor (log-likelihood requests only)."""
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
        self.allocated = 0                              # bytes of pooled + busy stores
        self.stream = torch.cuda.Stream(device=self.device)
        self.batches = 0

    # ---- store pool -------------------------------------------------------
    def _take_store(self, dsi):
        d = self.ds[dsi]
        if self.pool[dsi]:
            return self.pool[dsi].pop()
        need = d["bytes"]
        if need > self.budget:
            return "reject"
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

    # ---- one launch -------------------------------------------------------
    def _launch(self, reqs, now):
        torch = self.torch
        lik = [(r, s) for r, s in reqs if r.kind == "loglik"]
        krg = [r for r, _ in reqs if r.kind == "krige"]
        with torch.cuda.stream(self.stream):
            batch = None
            if lik:
                probs = [dict(x=self.ds[r.dataset]["x"], y=self.ds[r.dataset]["y"], z=self.ds[r.dataset]["z"],
                              store=s) for r, s in lik]
                batch = geo.Batch(probs, device=self.device)
                batch.set_theta([r.theta for r, _ in lik])
                batch.loglik_async(self.stream)
            kout = []
            for r in krg:
                d = self.ds[r.dataset]
                xn = torch.as_tensor(np.ascontiguousarray(r.xnew), dtype=torch.float64, device=self.device)
                yn = torch.as_tensor(np.ascontiguousarray(r.ynew), dtype=torch.float64, device=self.device)
                kout.append(d["krig"].krige(d["x"], d["y"], d["z"], d["theta"], xn, yn, stream=self.stream))
            ev = torch.cuda.Event()
            ev.record(self.stream)
        self.batches += 1
        return dict(lik=lik, krg=krg, batch=batch, kout=kout, event=ev, t_admit=now, id=self.batches)

    def _harvest(self, fl, now, results):
        if fl["batch"] is not None:
            out = fl["batch"].out.cpu().numpy()
            for b, (r, s) in enumerate(fl["lik"]):
                code, _ = s.status()
                results.append(Result(r.id, r.kind, r.dataset, tuple(out[b]), r.t_arrival, fl["t_admit"], now,
                                      fl["id"], code))
                self._give_back(r.dataset, s)
        for r, z in zip(fl["krg"], fl["kout"]):
            results.append(Result(r.id, r.kind, r.dataset, z.cpu().numpy(), r.t_arrival, fl["t_admit"], now,
                                  fl["id"], 0))

    # ---- the request loop -------------------------------------------------
    def run(self, requests, admit_until: float = math.inf):
        """Serve `requests` (their t_arrival fields, seconds from now) in real time.
        Requests arriving after `admit_until` are not admitted (counted as
        queued).  Returns (results, stats)."""
        pending = collections.deque(sorted(requests, key=lambda r: r.t_arrival))
        queue = collections.deque()
        results, rejected = [], []
        inflight = None
        t0 = time.perf_counter()
        while pending or queue or inflight is not None:
            now = time.perf_counter() - t0
            while pending and pending[0].t_arrival <= now:
                queue.append(pending.popleft())
            if inflight is not None and inflight["event"].query():
                self._harvest(inflight, time.perf_counter() - t0, results)
                inflight = None
            if inflight is None and queue and now <= admit_until:
                admitted, keep = [], collections.deque()
                while queue and len(admitted) < self.max_batch:
                    r = queue.popleft()
                    if r.kind == "krige":
                        if self.ds[r.dataset]["krig"] is None:
                            rejected.append(r)          # no resident factor for this dataset
                        else:
                            admitted.append((r, None))
                        continue
                    s = self._take_store(r.dataset)
                    if s == "reject":
                        rejected.append(r)
                    elif s is None:
                        keep.append(r)
                    else:
                        admitted.append((r, s))
                queue.extendleft(reversed(keep))
                if admitted:
                    inflight = self._launch(admitted, now)
                    continue
            if inflight is None and (not queue or now > admit_until) and (not pending or now > admit_until):
                break
            nxt = pending[0].t_arrival - now if pending else 1e-3
            time.sleep(max(0.0, min(nxt, 5e-4)))
        wall = time.perf_counter() - t0
        lat = np.array([r.latency for r in results]) if results else np.zeros(0)
        nl = sum(1 for r in results if r.kind == "loglik")
        stats = dict(completed=len(results), loglik_completed=nl,
                     krige_completed=len(results) - nl, rejected=len(rejected),
                     queued=len(queue) + len(pending), launches=self.batches, wall_s=wall,
                     evals_per_s=nl / wall if wall > 0 else 0.0,
                     p50_ms=float(np.percentile(lat, 50) * 1e3) if lat.size else None,
                     p99_ms=float(np.percentile(lat, 99) * 1e3) if lat.size else None)
        return results, stats
