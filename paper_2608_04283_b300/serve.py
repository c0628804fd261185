"""Continuous-batching server for VKLB simulations (the served form).

Requests (system, grid side, step count, initial data) arrive over time.  The
server admits them first-in first-out while their device memory fits under an
HBM budget, keeps every simulation in the moment form (all families run at
omega = 1, where U alone is the state: 2p instead of 10p values a cell), keeps
every admitted simulation's state resident on the GPU, and advances all active
simulations of one system family together with a
single batched launch per step (``vklb_batch_step``); the three families run on
their own CUDA streams, so their work overlaps on the device.  A tick advances
a family by K steps, K = min(tick_steps, fewest steps any member still needs);
when it completes, that family's finished simulations are read back and freed,
waiting requests are admitted into the freed memory and its next tick is
launched, without waiting for the other families' ticks.  Every request's result is the
same as when it is served alone: the batched kernel computes each tile of each
member independently, with the family's fixed tiling.

All arithmetic runs in libvklb.so; this module only schedules.
"""
from __future__ import annotations

import json
import time
from dataclasses import dataclass, field

import numpy as np

from . import inputs
from . import vklb

FAMILY = {
    # system: (Sim keyword arguments, domain side)
    "swe": (dict(omega=1.0, cfl=0.3, g=9.81), 1.0),
    "euler": (dict(omega=1.0, cfl=0.3, gamma=1.4), 1.0),
    "mhd_glm": (dict(omega=1.0, cfl=0.3, gamma=5.0 / 3.0, ch_factor=6.0), 2.0 * np.pi),
}
FIELDS = {"swe": 3, "euler": 4, "mhd_glm": 9}


def device_bytes(system, n, precision="fp32", form="moments", tile_x=128):
    """Device memory one simulation holds: two state buffers (p or 5p values a
    cell), the double staging array used by set_state / moments, and for
    MHD-GLM the two buffers of its tiles' edge columns (tiles tile_x wide)."""
    s = {"fp32": 4, "bf16": 2, "fp64": 8}[precision]
    pitch = ((n + 31) // 32) * 32
    p = FIELDS[system]
    q = 1 if form == "moments" else 5
    halo = 2 * (-(-n // tile_x)) * 2 * n * q * p * s if system == "mhd_glm" else 0
    return 2 * q * p * pitch * n * s + p * n * n * 8 + halo


@dataclass
class Job:
    req: inputs.Request
    sim: object = None
    left: int = 0
    t_admit: float = 0.0
    t_done: float = 0.0
    result: np.ndarray = None
    status: str = "queued"


@dataclass
class Report:
    jobs: list = field(default_factory=list)
    wall_s: float = 0.0

    def summary(self):
        done = [j for j in self.jobs if j.status == "done"]
        lat = np.array([j.t_done - j.req.arrival for j in done]) if done else np.zeros(1)
        wait = np.array([j.t_admit - j.req.arrival for j in done]) if done else np.zeros(1)
        lups = sum(j.req.n * j.req.n * j.req.steps for j in done)
        return {"requests": len(self.jobs), "completed": len(done),
                "failed": sum(j.status == "failed" for j in self.jobs),
                "wall_s": self.wall_s, "solves_per_s": len(done) / self.wall_s if self.wall_s > 0 else 0.0,
                "MLUPS": lups / self.wall_s / 1e6 if self.wall_s > 0 else 0.0,
                "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
                "queue_p50_s": float(np.percentile(wait, 50)), "queue_p99_s": float(np.percentile(wait, 99))}


class Server:
    """``max_side``: grids up to this side have their results read back through a
    pinned host buffer per family (allocated here, one direct copy per result;
    the result a caller keeps is copied out of it); larger ones through a fresh
    pageable array.  ``log``: a text stream that receives one JSON line per
    finished request (id, system, side, steps, arrival, admission and finish
    times, status)."""

    def __init__(self, budget_bytes=120e9, tick_steps=50, precision="fp32", tiles=None, keep_results=False,
                 clock=None, form="moments", max_side=2048, device_ic=False, log=None):
        import torch
        self.torch = torch
        self.budget = float(budget_bytes)
        self.tick = int(tick_steps)
        self.precision = precision
        self.tiles = tiles or {"swe": (64, 16), "euler": (64, 16), "mhd_glm": (128, 16)}
        self.keep = keep_results
        self.form = form
        self.device_ic = device_ic
        self.log = log
        self.streams = {k: torch.cuda.Stream() for k in FAMILY}
        self.clock = clock or time.perf_counter
        self.staging = {k: torch.empty(FIELDS[k] * max_side * max_side, dtype=torch.float64,
                                       pin_memory=True).numpy() for k in FAMILY}

    def _result(self, fam, sim):
        """Read a finished simulation's U back (into the family's pinned buffer
        when it fits)."""
        shape = sim.shape
        size = int(np.prod(shape))
        if size > self.staging[fam].size:
            return sim.moments()
        U = sim.moments(out=self.staging[fam][:size].reshape(shape))
        return U.copy() if self.keep else U

    def _make(self, req, U0=None):
        kw, side = FAMILY[req.system]
        sim = vklb.Sim(req.system, (req.n, req.n), (0.0, 0.0), (side, side), precision=self.precision,
                       stream=self.streams[req.system], form=self.form, **kw)
        sim.set_tiling(*self.tiles[req.system])
        if U0 is None and self.device_ic:
            # the request's analytic initial data evaluated on the device, on the
            # family's stream (the state's copy is ordered after it)
            with self.torch.cuda.stream(self.streams[req.system]):
                sim.set_state(inputs.request_initial_state_torch(req, self.torch))
            return sim
        if U0 is None:
            U0 = inputs.request_initial_state(req)
        sim.set_state(np.ascontiguousarray(U0))
        return sim

    def run(self, requests, realtime=True, payloads=None):
        """Serve ``requests`` (sorted by arrival).  With realtime, arrivals are
        honoured against the wall clock from the start; otherwise everything is
        available at once.  ``payloads`` optionally maps a request id to its
        initial state U_0 (the data a client sends with the request); without
        it the server generates U_0 itself (on the device with ``device_ic``,
        from the request's system, side and phases).  Returns a Report.

        Each family has at most one tick in flight on its stream, and a family
        is served as soon as its own tick completes (its finished requests read
        back and freed, waiting requests admitted, its next tick launched),
        while the other families' ticks keep the GPU busy."""
        torch = self.torch
        t0 = self.clock()
        now = lambda: self.clock() - t0
        jobs = [Job(req=r, left=r.steps) for r in requests]
        queue, active = [], {k: [] for k in FAMILY}
        batches = {}
        inflight = {}   # family -> (event, members stepped, k), in launch order
        used = 0.0
        peak = 0.0
        qi = 0
        while qi < len(jobs) or queue or any(active.values()):
            t = now()
            while qi < len(jobs) and (not realtime or jobs[qi].req.arrival <= t):
                queue.append(jobs[qi])
                qi += 1
            # admission: first in, first out, under the memory budget
            while queue:
                j = queue[0]
                need = device_bytes(j.req.system, j.req.n, self.precision, self.form)
                if used + need > self.budget and any(active.values()):
                    break
                queue.pop(0)
                j.sim = self._make(j.req, None if payloads is None else payloads.get(j.req.rid))
                j.t_admit = now()
                j.status = "running"
                j.need = need
                used += need
                peak = max(peak, used)
                active[j.req.system].append(j)
            if not any(active.values()):
                if qi < len(jobs):
                    time.sleep(max(0.0, min(0.01, jobs[qi].req.arrival - now())))
                continue
            # launch a tick of every family that has none in flight; a family's
            # batch is rebuilt only when its membership changed
            for fam, js in active.items():
                if not js or fam in inflight:
                    continue
                key = tuple(j.req.rid for j in js)
                if batches.get(fam, (None,))[0] != key:
                    if fam in batches:
                        batches[fam][1].close()
                    batches[fam] = (key, vklb.Batch([j.sim for j in js], tile=self.tiles[fam]))
                k = min(self.tick, min(j.left for j in js))
                batches[fam][1].step(k, graph=False)
                ev = torch.cuda.Event()
                ev.record(self.streams[fam])
                inflight[fam] = (ev, list(js), k)
            # serve the families whose tick has completed (polled, so that the
            # first family to finish is served first), or admit an arrival
            done = [fam for fam, (ev, _, _) in inflight.items() if ev.query()]
            while not done and inflight:
                if realtime and qi < len(jobs) and jobs[qi].req.arrival <= now():
                    break
                if len(inflight) == 1:
                    next(iter(inflight.values()))[0].synchronize()
                else:
                    time.sleep(1e-4)
                done = [fam for fam, (ev, _, _) in inflight.items() if ev.query()]
            for fam in done:
                _, stepped, k = inflight.pop(fam)
                for j in stepped:
                    j.left -= k
                if any(j.left == 0 for j in stepped):
                    batches.pop(fam)[1].close()
                still = []
                for j in active[fam]:
                    if j.left > 0:
                        still.append(j)
                        continue
                    try:
                        U = self._result(fam, j.sim)
                        j.status = "done"
                        if self.keep:
                            j.result = U
                    except vklb.VKLBError:
                        j.status = "failed"
                    j.t_done = now()
                    if self.log is not None:
                        r = j.req
                        self.log.write(json.dumps({"rid": r.rid, "system": r.system, "n": r.n, "steps": r.steps,
                                                   "arrival_s": r.arrival, "admitted_s": j.t_admit,
                                                   "done_s": j.t_done, "status": j.status}) + "\n")
                    j.sim.close()
                    j.sim = None
                    used -= j.need
                active[fam] = still
        for key, b in batches.values():
            b.close()
        rep = Report(jobs=jobs, wall_s=now())
        rep.peak_bytes = peak
        return rep


def serve_alone(req, **kw):
    """The same request served on its own (a batch of one)."""
    srv = Server(keep_results=True, **kw)
    r = inputs.Request(rid=req.rid, arrival=0.0, system=req.system, n=req.n, steps=req.steps, phase=req.phase)
    rep = srv.run([r], realtime=False)
    return rep.jobs[0].result


def run_plain(requests, precision="fp32", tiles=None, form="moments", payloads=None, max_side=2048,
              device_ic=False):
    """Baseline: the same requests one at a time, one launch per step each, the
    results read back through a pinned buffer as the server reads them.  Each
    simulation takes the library's default launch shape for its grid (128 wide,
    height fitted to whole waves) unless ``tiles`` names one per system.  The
    initial state comes from ``payloads``, or is built on the device
    (``device_ic``) or on the host, as the server builds it."""
    import torch
    staging = torch.empty(max(FIELDS.values()) * max_side * max_side, dtype=torch.float64, pin_memory=True).numpy()
    t0 = time.perf_counter()
    for r in requests:
        kw, side = FAMILY[r.system]
        sim = vklb.Sim(r.system, (r.n, r.n), (0.0, 0.0), (side, side), precision=precision, form=form, **kw)
        if tiles:
            sim.set_tiling(*tiles[r.system])
        if payloads is not None:
            sim.set_state(np.ascontiguousarray(payloads[r.rid]))
        elif device_ic:
            sim.set_state(inputs.request_initial_state_torch(r, torch))
        else:
            sim.set_state(np.ascontiguousarray(inputs.request_initial_state(r)))
        sim.step(r.steps)
        size = int(np.prod(sim.shape))
        if size <= staging.size:
            sim.moments(out=staging[:size].reshape(sim.shape))
        else:
            sim.moments()
        sim.close()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    lups = sum(r.n * r.n * r.steps for r in requests)
    return {"requests": len(requests), "wall_s": wall, "solves_per_s": len(requests) / wall,
            "MLUPS": lups / wall / 1e6}
