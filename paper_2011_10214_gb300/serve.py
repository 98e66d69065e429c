"""Continuous-batching server for independent charging simulations.

Requests (one sphere-charging problem each) arrive over time.  The server
admits a request as soon as its estimated device memory fits the HBM budget
next to the running ones, sets it up (load, initial field solve, leapfrog
start) and adds it to one pifepic batch; every round advances all running
members with one CUDA graph launch per step, so requests that arrive while
others run share the device.  A member finishes after `max_steps` steps or
once its area-mean surface potential changed by less than `rel_change` over
the last `window` steps (the charging has reached its floating potential,
Sec. 3.1.2).  Latency = finish time - arrival time.

Admission overlaps the running work (overlap=True): a worker thread creates
each admitted request and loads its particles on its own CUDA stream while the
main thread keeps stepping the batch; at the next round the main thread runs
the request's initial field solve and leapfrog start (a persistent solve over
the whole device, which must not run beside the batch's clustered solves) and
adds it to the batch.  With overlap=False the whole set-up runs between rounds
on the batch's stream and every running member waits for it.

Host-side orchestration only (admission, batch membership, stop tests); every
step of every member runs in libpifepic's kernels.
"""
import math
import queue
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import capi
from . import workloads as wl


def estimate_bytes(cfg, precision=capi.MIXED):
    """Device memory of one instance: particle bins with slack, mover lists,
    mesh, field and solver arrays (a conservative estimate)."""
    n = cfg["n"]
    cells = n[0] * n[1] * n[2]
    nodes = (n[0] + 1) * (n[1] + 1) * (n[2] + 1)
    per_p = 28 if precision == capi.MIXED else 48
    parts = sum(sp["ppc"] for sp in cfg["species"]) * cells
    bins = parts * per_p * 1.25 + len(cfg["species"]) * (cells // 64 + 1) * 64 * per_p
    movers = len(cfg["species"]) * 2 * max(1 << 16, parts // len(cfg["species"]) // 8 + 4096) * per_p
    mesh = nodes * (8 * 20 + 4 * 12 + 8 * 8 * 8) + cells * 16
    return int(bins + movers + mesh + (4 << 20))


def request_distribution(rng, count, big_fraction=0.05):
    """Sphere-charging requests: n ~ U{16..48} cells per side (h = 0.5),
    R ~ U[1, 8] Debye lengths clamped to fit the box, eps_in ~ U[2, 10],
    ppc ~ U{16..64}; a fraction at 96^3 cells with 64 ppc."""
    out = []
    for _ in range(count):
        if rng.random() < big_fraction:
            n, ppc = 96, 64
        else:
            n, ppc = int(rng.integers(16, 49)), int(rng.integers(16, 65))
        box = n * 0.5
        R = float(min(rng.uniform(1.0, 8.0), 0.3 * box))
        eps = float(rng.uniform(2.0, 10.0))
        out.append(wl.sphere_config(n, R, ppc, 500, eps_in=eps, seed_offset=int(rng.integers(100, 10**6))))
    return out


@dataclass
class Member:
    rid: int
    cfg: dict
    arrival: float
    sim: object
    admitted: float
    steps: int = 0
    pushed: int = 0
    history: list = field(default_factory=list)   # (step, surface potential)


class Server:
    """stream: the batch's CUDA stream (handle); admit_stream: the stream the
    admission worker sets requests up on (overlap=True; None = the batch's);
    bin_edges: particle-bin edge per size class (autotune_bin_edge's picks;
    classes not listed use the library's default)."""

    def __init__(self, hbm_budget, precision=capi.MIXED, steps_per_round=10, max_steps=500, window=50,
                 rel_change=0.01, pcg_tol=1e-6, cta_nodes=8192, stream=None, keep_phi=False, overlap=True,
                 admit_stream=None, bin_edges=None):
        self.budget = int(hbm_budget)
        self.precision = precision
        self.k = int(steps_per_round)
        self.max_steps = int(max_steps)
        self.window = int(window)
        self.rel = float(rel_change)
        self.pcg_tol = pcg_tol
        self.batch = capi.Batch(stream=stream)
        self.batch.set_cta_nodes(cta_nodes)
        self.stream = stream
        self.running = []
        self.used = 0
        self.results = []
        self.keep_phi = keep_phi
        self.bin_edges = dict(bin_edges or {})   # size class -> particle-bin edge (autotune_bin_edge)
        self.overlap = bool(overlap)
        self.inflight = 0            # handed to the admission worker, not yet in the batch
        if self.overlap:
            self.admit_stream = admit_stream if admit_stream is not None else stream
            try:                     # the worker thread must use this thread's device
                import torch
                self.device = torch.cuda.current_device()
            except Exception:
                self.device = None
            self._todo = queue.Queue()
            self._ready = queue.Queue()
            self._worker = threading.Thread(target=self._work, daemon=True)
            self._worker.start()

    def _create(self, cfg, stream):
        """Context, object, species, particle load and injection (no solve)."""
        return capi.from_config(cfg, precision=self.precision, pcg_tol=self.pcg_tol, stream=stream,
                                bin_edge=self.bin_edges.get(size_class(cfg)))

    @staticmethod
    def _start(sim):
        """The initial field solve and the leapfrog start."""
        sim.solve()
        sim.leapfrog_init()

    def _setup(self, cfg, stream):
        sim = self._create(cfg, stream)
        self._start(sim)
        return sim

    def _work(self):
        """Admission worker: creates and loads handed-over requests on the
        admission stream, in arrival order, while the main thread steps the
        batch (the main thread starts them at the join)."""
        if self.device is not None:
            import torch
            torch.cuda.set_device(self.device)
        while True:
            item = self._todo.get()
            if item is None:
                return
            rid, cfg, arrival = item
            try:
                self._ready.put((rid, cfg, arrival, self._create(cfg, self.admit_stream), None))
            except Exception as e:          # reported by the main thread
                self._ready.put((rid, cfg, arrival, None, e))

    def _join(self, rid, cfg, arrival, sim):
        self.batch.add(sim)
        m = Member(rid, cfg, arrival, sim, time.perf_counter())
        self.running.append(m)
        return m

    def _join_ready(self, block=False):
        """Add the requests the worker has finished setting up to the batch."""
        while self.inflight:
            try:
                rid, cfg, arrival, sim, err = self._ready.get(block=block, timeout=0.05 if block else None)
            except queue.Empty:
                return
            block = False
            self.inflight -= 1
            if err is not None:
                raise err
            self._start(sim)
            self._join(rid, cfg, arrival, sim)

    def _admit(self, rid, cfg, arrival):
        self.used += estimate_bytes(cfg, self.precision)
        if self.overlap:
            self.inflight += 1
            self._todo.put((rid, cfg, arrival))
            return None
        return self._join(rid, cfg, arrival, self._setup(cfg, self.stream))

    def _done(self, m):
        if m.steps >= self.max_steps:
            return True
        past = [v for s, v in m.history if s <= m.steps - self.window]
        if not past or not m.history:
            return False
        v0, v1 = past[-1], m.history[-1][1]
        return abs(v1 - v0) <= self.rel * max(abs(v0), 1e-30)

    def run(self, requests, arrivals, time_limit=None):
        """requests: list of workload dicts; arrivals: seconds after start.
        Returns per-request results and aggregate throughput."""
        t_start = time.perf_counter()
        pending = sorted(zip(arrivals, range(len(requests)), requests), key=lambda t: (t[0], t[1]))
        pushed_total = 0
        waiting = []
        while pending or waiting or self.running or self.inflight:
            now = time.perf_counter() - t_start
            if time_limit is not None and now > time_limit:
                break
            while pending and pending[0][0] <= now:
                waiting.append(pending.pop(0))
            # admission by HBM budget, first come first served
            while waiting:
                arr, rid, cfg = waiting[0]
                need = estimate_bytes(cfg, self.precision)
                if (self.running or self.inflight) and self.used + need > self.budget:
                    break
                waiting.pop(0)
                self._admit(rid, cfg, t_start + arr)
            if self.overlap:
                self._join_ready(block=not self.running)
            if not self.running:
                if pending and not self.inflight:
                    time.sleep(max(0.0, min(0.05, pending[0][0] - (time.perf_counter() - t_start))))
                continue
            stats = self.batch.step(self.k)
            for m, st in zip(list(self.running), stats):
                m.steps += self.k
                pushed = int(sum(st["pushed"]))
                m.pushed += pushed
                pushed_total += pushed
                m.history.append((m.steps, st["surface_potential"]))
            for m in [m for m in self.running if self._done(m)]:
                t = time.perf_counter()
                self.batch.remove(m.sim)
                self.results.append(dict(rid=m.rid, n=m.cfg["n"][0], steps=m.steps, latency=t - m.arrival,
                                         queue_wait=m.admitted - m.arrival, pushed=m.pushed,
                                         surface_potential=m.history[-1][1],
                                         phi=m.sim.potential() if self.keep_phi else None))
                m.sim.close()
                self.running.remove(m)
                self.used -= estimate_bytes(m.cfg, self.precision)
        wall = time.perf_counter() - t_start
        lat = np.array([r["latency"] for r in self.results]) if self.results else np.zeros(1)
        return dict(completed=len(self.results), wall_s=wall, particle_steps=pushed_total,
                    particle_steps_per_s=pushed_total / wall if wall > 0 else 0.0,
                    p50_s=float(np.percentile(lat, 50)), p99_s=float(np.percentile(lat, 99)),
                    results=self.results)

    def close(self):
        if self.overlap:
            self._todo.put(None)
            self._worker.join()
            while not self._ready.empty():
                item = self._ready.get()
                if item[3] is not None:
                    item[3].close()
            self.inflight = 0
        for m in self.running:
            self.batch.remove(m.sim)
            m.sim.close()
        self.running = []
        self.batch.close()


def autotune_batch(batch, trial_steps=2, candidates=(8192, 4096, 2048),
                   preconds=(capi.PRECOND_MULTIGRID, capi.PRECOND_JACOBI)):
    """Pick the clustered solves' preconditioner (multigrid or Jacobi) and
    nodes per CTA (hence each member's cluster size) by timing real steps of
    the batch (the trial steps advance the members like any other step).
    Returns (preconditioner, nodes per CTA, seconds per step of the pick)."""
    best, best_t = None, math.inf
    for pc in preconds:
        batch.set_preconditioner(pc)
        for cn in candidates:
            batch.set_cta_nodes(cn)
            batch.step(1, stats=False)            # graph rebuild + warm-up
            t0 = time.perf_counter()
            batch.step(trial_steps, stats=False)
            t = time.perf_counter() - t0
            if t < best_t:
                best, best_t = (pc, cn), t
    batch.set_preconditioner(best[0])
    batch.set_cta_nodes(best[1])
    return best[0], best[1], best_t / trial_steps


def size_class(cfg):
    """The tuner's instance classes: cells per side (below 32 or not) and
    particles per cell and species (up to 32, up to 48, more)."""
    n = cfg["n"][0]
    ppc = max(sp["ppc"] for sp in cfg["species"])
    return (0 if n < 32 else 1, 0 if ppc <= 32 else (1 if ppc <= 48 else 2))


BIN_MAX = 32767   # particles of one species a bin holds (the rest waits in the mover list)


def fits_bin(ppc, edge):
    """A bin of edge^3 cells at ppc particles per cell and species, with the
    library's 25 % + 64 slack, stays within BIN_MAX (else its overflow would
    travel through the mover list every step)."""
    return ppc * edge ** 3 * 1.25 + 64 <= BIN_MAX


def autotune_bin_edge(cfgs, precision=capi.MIXED, edges=(4, 8), per_class=8, trial_steps=3, stream=None):
    """Pick the particle-bin edge per size class by timing: up to per_class
    members of the class, set up with each edge whose full bins fit (fits_bin
    at the class's largest ppc), are stepped as one batch (graph rebuilt and
    warmed first) and timed with CUDA events on the batch's stream.  Returns
    ({class: edge}, {class: {edge: ms per step}})."""
    import torch
    st = torch.cuda.Stream() if stream is None else None
    handle = st.cuda_stream if st is not None else stream
    ev_stream = st if st is not None else torch.cuda.ExternalStream(stream)
    classes = {}
    for c in cfgs:
        classes.setdefault(size_class(c), []).append(c)
    picks, times = {}, {}
    for k, members in sorted(classes.items()):
        trial = members[:per_class]
        times[k] = {}
        ppc = max(sp["ppc"] for c in members for sp in c["species"])
        for e in edges:
            if not fits_bin(ppc, e):
                continue
            sims = []
            try:
                for c in trial:
                    sim = capi.from_config(c, precision=precision, stream=handle, bin_edge=e)
                    sim.solve()
                    sim.leapfrog_init()
                    sims.append(sim)
                batch = capi.Batch(sims, stream=handle)
                batch.step(1, stats=False)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(ev_stream)
                batch.step(trial_steps, stats=False)
                e1.record(ev_stream)
                torch.cuda.synchronize()
                times[k][e] = e0.elapsed_time(e1) / trial_steps
                batch.close()
            finally:
                for sim in sims:
                    sim.close()
        picks[k] = min(times[k], key=times[k].get)
    return picks, times


def poisson_arrivals(rng, rate, horizon):
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t > horizon:
            return out
        out.append(t)
