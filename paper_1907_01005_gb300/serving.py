"""Request loop for apply_H + P^T Y + P^T P with continuous batching.

A `Server` owns one GPU.  Workloads ("payloads": a mesh, a block pattern and
the values of P) are registered once; the server keeps each payload's mesh
geometry, DoF map, potential, P (values and work lists), Y and the two Gram
matrices resident in device memory while the payload is in use, and evicts
idle payloads (least recently used first) when the memory budget is needed.

Requests name a payload (and may bring new values of P from host memory).
A queued request is admitted as soon as
  * a stream slot is free (at most `slots` requests are on the GPU), and
  * the payload is resident or its device footprint fits in the budget
    (after evicting idle payloads).
Among the queued requests the predicted shortest goes first (the prediction
is a running mean of the payload's observed service time, seeded from its
DoF x column count), except that a request which has waited more than
`age_factor` times its own prediction (at least `min_age_s`) is aged and
goes ahead of all unaged ones, in arrival order, so large requests cannot
starve.  The last free slot is kept for small requests (predicted at most
the median of the registered payloads) unless the request is aged, so that
small requests do not queue behind a GPU full of large ones.  On the
device, small requests run on high-priority streams (their CTAs are
scheduled before the pending CTAs of large ones), and the persistent kernels
of large requests are capped to all but `reserve_sms` SMs, so that a small
request finds SMs free while a large request's Gram products run.  Requests
that arrive while others run join them on the device: each
admitted request runs `fe_apply_H_gram` on its own CUDA stream and the
kernels of different requests overlap.  A request completes when its Gram
matrices (and, if asked, Y) are back in host memory; its latency is measured
from its arrival to that moment.

All arithmetic runs in libfe_mf.so; this module only schedules calls and
moves buffers.  One payload is on the GPU for at most one request at a time
(its device buffers are the request's workspace); a later request for a busy
payload waits while other requests may overtake it.
"""
from __future__ import annotations

import collections
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import api, harness


def _nbytes(t) -> int:
    return t.numel() * t.element_size()


@dataclass
class Payload:
    """A registered workload: host-side problem plus (when resident) device state."""
    pid: int
    problem: harness.Problem
    mesh_key: tuple
    dev: dict | None = None
    host: dict | None = None
    busy: bool = False
    last_used: float = 0.0
    service_s: float = 0.0        # running estimate of one request's service time

    @property
    def dofs_cols(self) -> float:
        return float(self.problem.mesh.n_dofs) * float(self.problem.n_cols)

    def footprint(self) -> int:
        """Device bytes of the payload's own buffers (the mesh is counted apart)."""
        i = self.problem.P.info
        m = self.problem.n_cols
        return int(2 * i.value_bytes + max(256, i.table_bytes) + 2 * m * m * 8)


@dataclass
class Request:
    rid: int
    pid: int
    arrival: float
    p_host: object = None          # pinned torch tensor of new P values, or None
    want_y: bool = False
    admitted: float = 0.0
    done: float = 0.0
    stream: object = None
    event: object = None
    result: dict = field(default_factory=dict)

    @property
    def latency(self) -> float:
        return self.done - self.arrival


class Server:
    """Continuous-batching server on one GPU (see the module docstring)."""

    def __init__(self, budget_bytes: int | None = None, slots: int = 4, device: str = "cuda",
                 age_factor: float = 4.0, min_age_s: float = 2e-3, seed_rate: float = 1e11,
                 reserve_sms: int = 16, priority_small: bool = True):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        free, _total = torch.cuda.mem_get_info(self.device)
        self.budget = int(budget_bytes if budget_bytes is not None else 0.8 * free)
        self.slots = slots
        # per slot a normal stream (large requests) and a high-priority one
        # (small requests: their CTAs are scheduled ahead of pending large ones)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(slots)]
        self.streams_hi = [torch.cuda.Stream(device=self.device, priority=-8) for _ in range(slots)]
        n_sms = torch.cuda.get_device_properties(self.device).multi_processor_count
        # large requests' persistent kernels leave reserve_sms SMs to the small ones
        self.large_sm_limit = max(1, n_sms - reserve_sms) if reserve_sms > 0 else 0
        self.priority_small = priority_small
        self.free_streams = list(range(slots))
        self.payloads: dict[int, Payload] = {}
        self.meshes: dict[tuple, dict] = {}       # mesh key -> {"mesh": Mesh, "bytes": int, "users": set}
        self.used = 0
        self.peak_used = 0
        self.evictions = 0
        self.queue: collections.deque[Request] = collections.deque()
        self.running: list[Request] = []
        self.finished: list[Request] = []
        self._next_rid = 0
        self._lock = threading.Lock()
        self.age_factor = age_factor
        self.min_age_s = min_age_s
        self.seed_rate = seed_rate                 # DoF*columns/s that seeds the service estimates
        self.small_s = 0.0                         # the median service estimate of the payloads

    # ---- registration ---------------------------------------------------------
    def register(self, problem: harness.Problem) -> int:
        """Registers a host-built problem (harness.build_problem) as a payload."""
        pid = len(self.payloads)
        key = (id(problem.mesh),)
        pl = Payload(pid, problem, key)
        pl.service_s = pl.dofs_cols / self.seed_rate
        self.payloads[pid] = pl
        self._update_small()
        return pid

    def _update_small(self):
        est = sorted(p.service_s for p in self.payloads.values())
        self.small_s = est[(len(est) - 1) // 2] if est else 0.0

    # ---- memory -----------------------------------------------------------------
    def _mesh_resident(self, pl: Payload) -> int:
        """Uploads the payload's mesh (geometry, DoF map, potential) if needed;
        returns the bytes it added."""
        if pl.mesh_key in self.meshes:
            self.meshes[pl.mesh_key]["users"].add(pl.pid)
            return 0
        pb = pl.problem
        torch = self.torch
        pb.mesh.upload(self.device)
        vq = torch.from_numpy(pb.vq.astype(api.np_dtype(pb.dtype))).to(self.device)
        pb.mesh.set_potential(vq, pb.dtype)
        nbytes = _nbytes(pb.mesh._ws) + _nbytes(vq)
        self.meshes[pl.mesh_key] = {"bytes": nbytes, "users": {pl.pid}, "vq": vq}
        return nbytes

    def _mesh_bytes_needed(self, pl: Payload) -> int:
        if pl.mesh_key in self.meshes:
            return 0
        pb = pl.problem
        return int(pb.mesh.info.n_q) * (8 if pb.dtype == api.FE_F64 else 4) + 4096

    def _make_resident(self, pl: Payload):
        torch = self.torch
        pb = pl.problem
        self.used += self._mesh_resident(pl)
        pv, pt = pb.P.alloc(self.device, with_tables=True)
        yv, _ = pb.Y.alloc(self.device, with_tables=False)
        pv.copy_(torch.from_numpy(pb.P_host))
        pb.P.bind(pv, pt)
        pb.Y.bind(yv, None)
        m = pb.n_cols
        pl.dev = {"P": pv, "Pt": pt, "Y": yv,
                  "G_PY": torch.zeros((m, m), dtype=torch.float64, device=self.device),
                  "G_PP": torch.zeros((m, m), dtype=torch.float64, device=self.device)}
        if pl.host is None:                        # pinned result buffers, kept across residencies
            pl.host = {"G_PY": torch.empty((m, m), dtype=torch.float64).pin_memory(),
                       "G_PP": torch.empty((m, m), dtype=torch.float64).pin_memory()}
        torch.cuda.synchronize(self.device)
        self.used += pl.footprint()
        self.peak_used = max(self.peak_used, self.used)

    def _evict(self, pl: Payload):
        pl.dev = None                              # the handles are re-bound before their next use
        self.used -= pl.footprint()
        self.evictions += 1
        users = self.meshes[pl.mesh_key]["users"]
        users.discard(pl.pid)
        if not users:
            self.used -= self.meshes[pl.mesh_key]["bytes"]
            del self.meshes[pl.mesh_key]
            pl.problem.mesh._ws = None
            pl.problem.mesh._vq = {}

    def _fits(self, pl: Payload) -> bool:
        """True once the payload is resident, evicting idle payloads if needed."""
        if pl.dev is not None:
            return True
        need = pl.footprint() + self._mesh_bytes_needed(pl)
        if need > self.budget:
            raise MemoryError(f"payload {pl.pid} needs {need} bytes, budget {self.budget}")
        idle = sorted((q for q in self.payloads.values() if q.dev is not None and not q.busy and q is not pl),
                      key=lambda q: q.last_used)
        while self.used + need > self.budget and idle:
            self._evict(idle.pop(0))
        if self.used + need > self.budget:
            return False
        self._make_resident(pl)
        return True

    # ---- requests ---------------------------------------------------------------
    def submit(self, pid: int, p_host=None, want_y: bool = False, arrival: float | None = None) -> Request:
        with self._lock:
            r = Request(self._next_rid, pid, time.perf_counter() if arrival is None else arrival, p_host, want_y)
            self._next_rid += 1
            self.queue.append(r)
        return r

    def _launch(self, r: Request):
        torch = self.torch
        pl = self.payloads[r.pid]
        pb = pl.problem
        si = self.free_streams.pop()
        small = pl.service_s <= self.small_s
        s = self.streams_hi[si] if small and self.priority_small else self.streams[si]
        r.stream = si
        pb.P.set_sm_limit(0 if small else self.large_sm_limit)
        d = pl.dev
        with torch.cuda.stream(s):
            if r.p_host is not None:
                d["P"].copy_(r.p_host, non_blocking=True)
            api.apply_H_gram(pb.mesh, pb.P, pb.Y, d["G_PY"], d["G_PP"], s)
            pl.host["G_PY"].copy_(d["G_PY"], non_blocking=True)
            pl.host["G_PP"].copy_(d["G_PP"], non_blocking=True)
            if r.want_y:
                if "Y" not in pl.host:
                    pl.host["Y"] = torch.empty(d["Y"].shape, dtype=d["Y"].dtype).pin_memory()
                pl.host["Y"].copy_(d["Y"], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s)
        r.event = ev
        r.admitted = time.perf_counter()
        pl.busy = True
        pl.last_used = r.admitted
        self.running.append(r)

    def step(self) -> int:
        """One scheduling round: retire finished requests, admit queued ones.
        Returns the number of requests retired."""
        n = 0
        for r in list(self.running):
            if r.event.query():
                r.done = time.perf_counter()
                pl = self.payloads[r.pid]
                for k in ("G_PY", "G_PP") + (("Y",) if r.want_y else ()):
                    r.result[k] = pl.host[k].numpy().copy()
                self.running.remove(r)
                self.free_streams.append(r.stream)
                pl.busy = False
                pl.last_used = r.done
                pl.service_s = 0.7 * pl.service_s + 0.3 * (r.done - r.admitted)
                self.finished.append(r)
                n += 1
        if n:
            self._update_small()
        with self._lock:
            pending = list(self.queue)
        now = time.perf_counter()
        service = {pid: pl.service_s for pid, pl in self.payloads.items()}
        order = admission_order(pending, service, now, self.age_factor, self.min_age_s)
        admitted = []
        busy_now = set()
        for r, old in order:
            if not self.free_streams:
                break
            pl = self.payloads[r.pid]
            if pl.busy or r.pid in busy_now:
                continue
            if not may_take_slot(len(self.free_streams), self.slots, old, pl.service_s, self.small_s):
                continue                       # the last slot waits for a small or an aged request
            if not self._fits(pl):
                if old:
                    break                      # memory frees up for the aged request first
                continue
            self._launch(r)
            admitted.append(r)
            busy_now.add(r.pid)
        if admitted:
            with self._lock:
                for r in admitted:
                    self.queue.remove(r)
        return n

    def drain(self, timeout_s: float = 600.0):
        t0 = time.perf_counter()
        while self.queue or self.running:
            if self.step() == 0:
                time.sleep(20e-6)
            if time.perf_counter() - t0 > timeout_s:
                raise TimeoutError("serving drain timed out")

    def run_trace(self, trace, p_hosts=None, want_y: bool = False, timeout_s: float = 600.0):
        """Replays (arrival offset in s, payload id) pairs in real time and
        returns the finished requests in arrival order."""
        t0 = time.perf_counter()
        order = sorted(range(len(trace)), key=lambda i: trace[i][0])
        reqs = [None] * len(trace)
        k = 0
        while k < len(order) or self.queue or self.running:
            now = time.perf_counter()
            while k < len(order) and t0 + trace[order[k]][0] <= now:
                i = order[k]
                ph = None if p_hosts is None else p_hosts[i]
                reqs[i] = self.submit(trace[i][1], ph, want_y, arrival=t0 + trace[i][0])
                k += 1
            if self.step() == 0:
                time.sleep(20e-6)
            if now - t0 > timeout_s:
                raise TimeoutError("serving trace timed out")
        return reqs


def admission_order(pending, service_s, now, age_factor, min_age_s):
    """The order in which queued requests are considered, with their aged
    flag: a request is aged when it has waited more than age_factor times
    its payload's predicted service time (and at least min_age_s); aged
    requests come first in arrival order, then the others by predicted
    service time (ties by arrival)."""
    def aged(r):
        return now - r.arrival > max(age_factor * service_s[r.pid], min_age_s)
    flagged = [(r, aged(r)) for r in pending]
    return sorted(flagged, key=lambda x: (0, x[0].arrival, 0.0) if x[1] else (1, service_s[x[0].pid], x[0].arrival))


def may_take_slot(free_slots, slots, aged, service_s, small_s):
    """The last free slot (of more than one) goes to a small request (predicted
    at most small_s) or to an aged one only."""
    return not (free_slots == 1 and slots > 1 and not aged and service_s > small_s)


def latency_stats(reqs, dofs_cols, classes=None, alone_ms=None) -> dict:
    """p50/p99 latency (ms) and aggregate DoF*columns/s of finished requests;
    with `classes` (name -> (low, high) DoF*column bounds) also per size class,
    beside the class's one-at-a-time latency when `alone_ms` (payload id ->
    ms) is given."""
    lat = np.array([r.latency for r in reqs]) * 1e3
    span = max(r.done for r in reqs) - min(r.arrival for r in reqs)
    work = float(sum(dofs_cols[r.pid] for r in reqs))
    out = {"requests": len(reqs), "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
           "mean_ms": float(lat.mean()), "dof_cols_per_s": work / span, "span_s": span}
    if classes:
        per = {}
        for name, (lo, hi) in classes.items():
            sel = [i for i, r in enumerate(reqs) if lo <= dofs_cols[r.pid] < hi]
            if not sel:
                continue
            cl = lat[sel]
            d = {"requests": len(sel), "p50_ms": float(np.percentile(cl, 50)), "p99_ms": float(np.percentile(cl, 99))}
            if alone_ms:
                a = [alone_ms[reqs[i].pid] for i in sel]
                d["alone_ms_median"] = float(np.median(a))
                d["p99_over_alone"] = d["p99_ms"] / max(float(np.median(a)), 1e-9)
            per[name] = d
        out["classes"] = per
    return out
