"""Continuous-batching server of configuration-generation requests.

A request asks for n_sweeps sweeps (1 heatbath + n_overrelax overrelaxation
steps, re-unitarization) of an SU(Nc) chain on an L^4 lattice from a Haar
start, and gets back its plaquette and Polyakov-loop history.  The server keeps
every admitted chain's links and random state (seed, heatbath counter) resident
on the GPU, admits waiting requests in arrival order as soon as their device
footprint fits the memory budget, and advances chains together: each tick is
one batched run (sun_batch_run) over the chains the scheduling policy picks,
chains of different Nc on their own streams.  Requests that arrive while others
are on the GPU join at the next tick; finished chains leave and free their
memory.  A chain's results do not depend on which ticks and batches it ran in.

The plain path (serve_plain) runs the same trace one request at a time, each
chain alone (sun_run), in arrival order or shortest request first.
"""
import dataclasses
import time
from typing import List, Optional

import numpy as np

from . import sun


@dataclasses.dataclass
class Request:
    rid: int
    nc: int
    L: int
    beta: float
    n_sweeps: int
    seed: int
    arrival: float  # seconds after the start of the trace
    t_admit: Optional[float] = None
    t_done: Optional[float] = None
    plaquette: Optional[np.ndarray] = None
    polyakov: Optional[np.ndarray] = None

    @property
    def dims(self):
        return (self.L, self.L, self.L, self.L)

    @property
    def latency(self):
        return None if self.t_done is None else self.t_done - self.arrival


def poisson_trace(n, rate=20.0, seed=0, ncs=(2, 3, 4, 6), Ls=(8, 12, 16, 20, 24), sweeps=(20, 200)):
    """n requests with exponential inter-arrival times of mean 1/rate; Nc and L
    uniform over the given sets; beta uniform in [2.2, 2.5] for SU(2) and
    0.7 Nc^2 x U[0.95, 1.05] otherwise; n_sweeps uniform in the given range."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        nc = int(rng.choice(ncs))
        L = int(rng.choice(Ls))
        beta = float(rng.uniform(2.2, 2.5)) if nc == 2 else float(0.7 * nc * nc * rng.uniform(0.95, 1.05))
        ns = int(rng.integers(sweeps[0], sweeps[1] + 1))
        out.append(Request(i, nc, L, beta, ns, 1000 + i, t))
    return out


def _clone(reqs):
    return [dataclasses.replace(r, t_admit=None, t_done=None, plaquette=None, polyakov=None) for r in reqs]


def footprint(req, precision=32):
    return sun.footprint_bytes(req.nc, req.dims, precision, 0)


# Scheduling estimate of one sweep (1 heatbath + 4 overrelaxation, FP32), in ms
# per lattice site: a default measured on a GB300 on 24^4 lattices, replaced by
# measure_sweep_costs() on the GPU at hand.
SWEEP_MS_PER_SITE = {2: 1.4e-6, 3: 4.2e-6, 4: 1.3e-5, 6: 6.7e-5}


def sweep_cost_ms(req, costs=None):
    table = SWEEP_MS_PER_SITE if costs is None else costs
    c = table.get(req.nc, table.get(6, 6.7e-5) * (req.nc / 6.0) ** 3)
    return c * float(np.prod(req.dims))


def measure_sweep_costs(ncs=(2, 3, 4, 6), L=24, sweeps=3, n_overrelax=4, precision=32):
    """ms per lattice site of one sweep for each Nc, measured on the current GPU
    (an L^4 lattice alone, after one untimed sweep; CUDA events on its stream)."""
    import torch
    out = {}
    for nc in ncs:
        beta = 2.3 if nc == 2 else 0.7 * nc * nc
        with sun.Lattice(nc, (L,) * 4, beta, hot_start=True, seed=1, precision=precision) as lat:
            lat.run(1, 1, n_overrelax, plaquette=False, polyakov=False)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(lat.stream)
            lat.run(sweeps, 1, n_overrelax)
            b.record(lat.stream)
            b.synchronize()
            out[nc] = a.elapsed_time(b) / sweeps / float(L ** 4)
    return out


class Server:
    """Continuous batching over a device-memory budget (bytes).

    Admission: waiting requests are admitted in arrival order as soon as their
    footprint fits the budget; an admitted chain keeps its links and random
    state resident until it has all its sweeps.
    Each tick: the server picks which resident chains to advance and runs them
    as one batch (sun_batch_run) for k sweeps.  policy "srpt" takes chains in
    order of least remaining work (remaining sweeps x predicted sweep time),
    "fifo" in admission order; both add chains while the predicted time of one
    sweep of the selection stays within work_cap_ms (the first chain always
    runs).  k is as many sweeps as fill about tick_ms of predicted GPU time, at
    most the fewest remaining sweeps of the selection.  Under srpt a large
    request no longer holds small ones behind it: they run beside it or
    between its ticks, and leave as soon as they are done."""

    def __init__(self, hbm_budget, n_overrelax=4, sweeps_per_tick=None, precision=32, use_graphs=True,
                 work_cap_ms=8.0, tick_ms=40.0, policy="srpt", graph_sweeps=16, clock=time.perf_counter,
                 costs=None):
        if policy not in ("srpt", "fifo"):
            raise ValueError("policy must be 'srpt' or 'fifo'")
        self.work_cap = work_cap_ms
        self.budget = int(hbm_budget)
        self.n_or = int(n_overrelax)
        self.max_k = None if sweeps_per_tick is None else int(sweeps_per_tick)
        self.tick_ms = float(tick_ms)
        self.policy = policy
        self.precision = precision
        self.use_graphs = use_graphs
        # sweeps per graph launch: a tick of small chains runs up to hundreds of
        # sweeps of a few microseconds each
        self.graph_sweeps = int(graph_sweeps)
        self.clock = clock
        self.costs = costs  # ms per site of a sweep by Nc (None: the default table)
        self.ticks = 0
        self.batches_built = 0
        self.link_updates = 0

    def _select(self, active):
        if self.policy == "srpt":
            order = sorted(active, key=lambda a: ((a[0].n_sweeps - a[2]) * sweep_cost_ms(a[0], self.costs),
                                                  a[0].arrival))
        else:
            order = list(active)
        sel, cost = [], 0.0
        for a in order:
            c = sweep_cost_ms(a[0], self.costs)
            if sel and self.work_cap is not None and cost + c > self.work_cap:
                continue
            sel.append(a)
            cost += c
        return sel, cost

    def run(self, trace: List[Request]):
        """Serve the trace in real time; returns the requests with their results."""
        reqs = _clone(trace)
        pending = sorted(reqs, key=lambda r: r.arrival)
        active = []  # [request, lattice, sweeps done, plaquette list, polyakov list, footprint]
        used = 0
        batch = None
        members = None
        t0 = self.clock()
        while pending or active:
            now = self.clock() - t0
            # admit in arrival order while the head of the queue fits the budget
            while pending and pending[0].arrival <= now and used + footprint(pending[0], self.precision) <= self.budget:
                r = pending.pop(0)
                fp = footprint(r, self.precision)
                lat = sun.Lattice(r.nc, r.dims, r.beta, hot_start=True, seed=r.seed, precision=self.precision,
                                  graph_sweeps=self.graph_sweeps)
                r.t_admit = self.clock() - t0
                active.append([r, lat, 0, [], [], fp])
                used += fp
            if not active:
                if pending[0].arrival <= now:
                    raise RuntimeError(f"request {pending[0].rid} does not fit the memory budget")
                time.sleep(min(pending[0].arrival - now, 0.05))
                continue
            sel, cost = self._select(active)
            ids = tuple(id(a[1]) for a in sel)
            if ids != members:
                if batch is not None:
                    batch.close()
                batch = sun.Batch([a[1] for a in sel], use_graphs=self.use_graphs)
                self.batches_built += 1
                members = ids
            k = min(a[0].n_sweeps - a[2] for a in sel)
            k = min(k, max(1, int(self.tick_ms / max(cost, 1e-6))))
            if self.max_k is not None:
                k = min(k, self.max_k)
            plaq, poly = batch.run(k, 1, self.n_or)
            self.ticks += 1
            for j, a in enumerate(sel):
                a[2] += k
                a[3].extend(plaq[:, j].tolist())
                a[4].extend(poly[:, j].tolist())
                self.link_updates += k * (1 + self.n_or) * 4 * int(np.prod(a[0].dims))
            done = [a for a in sel if a[2] >= a[0].n_sweeps]
            if done:
                t = self.clock() - t0
                for a in done:
                    r = a[0]
                    r.t_done = t
                    r.plaquette = np.array(a[3])
                    r.polyakov = np.array(a[4])
                    used -= a[5]
                active = [a for a in active if a[2] < a[0].n_sweeps]
                batch.close()
                batch = None
                members = None
                for a in done:
                    a[1].close()
        if batch is not None:
            batch.close()
        self.wall = self.clock() - t0
        return reqs


def serve_plain(trace: List[Request], n_overrelax=4, precision=32, clock=time.perf_counter, order="fifo",
                costs=None):
    """One request at a time, each chain alone (sun_run).  order "fifo" takes
    requests in arrival order; "srpt" takes, among the requests that have
    arrived, the one with the least predicted work (sweeps x sweep time), as
    the server's policy does, but without batching or preemption."""
    if order not in ("fifo", "srpt"):
        raise ValueError("order must be 'fifo' or 'srpt'")
    reqs = _clone(trace)
    queue = sorted(reqs, key=lambda q: q.arrival)
    t0 = clock()
    updates = 0
    while queue:
        now = clock() - t0
        if queue[0].arrival > now:
            time.sleep(queue[0].arrival - now)
            now = clock() - t0
        if order == "srpt":
            arrived = [q for q in queue if q.arrival <= now]
            r = min(arrived, key=lambda q: (q.n_sweeps * sweep_cost_ms(q, costs), q.arrival))
        else:
            r = queue[0]
        queue.remove(r)
        r.t_admit = clock() - t0
        with sun.Lattice(r.nc, r.dims, r.beta, hot_start=True, seed=r.seed, precision=precision) as lat:
            plaq, poly = lat.run(r.n_sweeps, 1, n_overrelax)
        r.t_done = clock() - t0
        r.plaquette, r.polyakov = plaq, poly
        updates += r.n_sweeps * (1 + n_overrelax) * 4 * int(np.prod(r.dims))
    return reqs, clock() - t0, updates


def latency_stats(reqs):
    lat = np.array([r.latency for r in reqs if r.latency is not None])
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "max_s": float(lat.max()), "completed": int(len(lat))}
