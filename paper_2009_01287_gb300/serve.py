"""Continuous-batching solve server on top of the C ABI.

Requests (a mesh, a right-hand side, a tolerance) arrive over time.  A
dispatcher admits them into solver slots as slots and device memory free up:
every slot is a host thread with its own CUDA stream, so the solves of
different slots overlap on the GPU while new requests keep arriving.  The
device state of a mesh (operator data and preconditioner) stays resident in
an LRU cache bounded by a device-memory budget, so later requests on the same
mesh skip the setup.  A handle is used by one slot at a time.

Every request is solved by the same calls as a standalone solve
(dg_rhs_sine + dg_pcg_solve on its own preconditioner handle), so its result
does not depend on what else is in flight.

Latency = completion time - arrival time; the report gives p50 / p99 and the
aggregate DOF-iterations per second.
"""
from __future__ import annotations

import dataclasses
import hashlib
import heapq
import threading
import time
from collections import OrderedDict
from typing import Dict, List, Optional

import numpy as np

from . import binding as B
from .inputs import MeshDesc, SineRHS

BYTES_PER_DOF_ESTIMATE = 600  # device bytes per DOF of one resident mesh + preconditioner + solve


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the run
    mesh: MeshDesc
    rhs: SineRHS
    tol: float = 1e-8
    maxit: int = 5000


@dataclasses.dataclass
class Result:
    rid: int
    ok: bool
    error: str = ""
    iters: int = 0
    rel_res: float = 0.0
    n_dofs: int = 0
    arrival: float = 0.0
    admitted: float = 0.0
    finished: float = 0.0
    solve_ms: float = 0.0
    setup_s: float = 0.0
    x: Optional[np.ndarray] = None

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def mesh_key(m: MeshDesc) -> str:
    h = hashlib.sha1()
    for a in (m.lo, m.size, m.p, np.asarray(m.extent)):
        h.update(np.ascontiguousarray(a).tobytes())
    h.update(repr((m.dim, m.lattice_h)).encode())
    return h.hexdigest()


class _Resident:
    def __init__(self, mesh: MeshDesc, opts):
        t = time.perf_counter()
        self.mesh = B.Mesh(mesh, opts)
        self.pc = B.Precond(self.mesh, opts)
        self.setup_s = time.perf_counter() - t
        self.n_dofs = self.mesh.n_dofs
        self.lock = threading.Lock()
        self.bytes = BYTES_PER_DOF_ESTIMATE * self.n_dofs

    def close(self):
        self.pc.close()
        self.mesh.close()


class Server:
    def __init__(self, slots: int = 8, precision: int = B.DG_PREC_MIXED,
                 memory_budget: Optional[int] = None, keep_solutions: bool = False,
                 cache_entries: int = 64):
        import torch
        self.torch = torch
        self.slots = slots
        self.opts = B.make_options(precision=precision)
        free, _ = torch.cuda.mem_get_info()
        self.budget = int(0.8 * free) if memory_budget is None else int(memory_budget)
        self.keep = keep_solutions
        self.cache: "OrderedDict[str, _Resident]" = OrderedDict()
        self.cache_entries = cache_entries
        self.lock = threading.Condition()
        self.in_use_bytes = 0
        self.peak_bytes = 0
        self.max_inflight = 0

    # ---------------------------------------------------------------- memory
    def _cached_bytes(self) -> int:
        return sum(r.bytes for r in self.cache.values())

    def _evict_for(self, need: int) -> bool:
        """Drop idle cache entries (LRU) until `need` more bytes fit."""
        while self.in_use_bytes + self._cached_bytes() + need > self.budget or \
                len(self.cache) >= self.cache_entries:
            victim = None
            for k, r in self.cache.items():
                if not r.lock.locked():
                    victim = k
                    break
            if victim is None:
                return False
            self.cache.pop(victim).close()
        return True

    # ---------------------------------------------------------------- run
    def run(self, requests: List[Request], realtime: bool = True) -> List[Result]:
        torch = self.torch
        pending = sorted(requests, key=lambda r: r.arrival)
        ready: List = []   # heap of (arrival, rid, request)
        results: Dict[int, Result] = {}
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        active = [0]
        done = threading.Event()

        def worker(slot: int):
            stream = torch.cuda.Stream()
            while True:
                with self.lock:
                    while True:
                        while pending and (not realtime or pending[0].arrival <= now()):
                            rq = pending.pop(0)
                            heapq.heappush(ready, (rq.arrival, rq.rid, rq))
                        if ready:
                            rq = ready[0][2]
                            need = BYTES_PER_DOF_ESTIMATE * rq.mesh.n_dofs()
                            key = mesh_key(rq.mesh)
                            hit = key in self.cache
                            if hit or self._evict_for(need) or self.in_use_bytes == 0:
                                heapq.heappop(ready)
                                self.in_use_bytes += 0 if hit else need
                                self.peak_bytes = max(self.peak_bytes, self.in_use_bytes + self._cached_bytes())
                                active[0] += 1
                                self.max_inflight = max(self.max_inflight, active[0])
                                break
                        if not pending and not ready:
                            return
                        wait = 0.05
                        if realtime and pending and not ready:
                            wait = max(0.0, min(wait, pending[0].arrival - now()))
                        self.lock.wait(timeout=wait)
                res = Result(rid=rq.rid, ok=False, arrival=rq.arrival, admitted=now())
                entry = None
                try:
                    with self.lock:
                        entry = self.cache.get(key)
                        if entry is not None:
                            self.cache.move_to_end(key)
                    if entry is None:
                        entry = _Resident(rq.mesh, self.opts)
                        res.setup_s = entry.setup_s
                    with entry.lock:
                        with torch.cuda.stream(stream):
                            b = torch.empty(entry.n_dofs, dtype=torch.float64, device="cuda")
                            x = torch.empty_like(b)
                            B.dg_rhs_sine(entry.mesh.h, rq.rhs.amps, rq.rhs.waves, b, stream)
                            info = B.dg_pcg_solve(entry.mesh.h, entry.pc.h, b, x, rq.tol, rq.maxit, stream,
                                                  raise_on_notconv=False)
                            if self.keep:
                                res.x = x.cpu().numpy()
                            stream.synchronize()
                    res.ok = info.status == B.DG_OK
                    res.iters, res.rel_res, res.solve_ms = info.iters, info.rel_res, info.solve_ms
                    res.n_dofs = entry.n_dofs
                    if not res.ok:
                        res.error = "not converged"
                except Exception as e:   # a failed request does not stop the server
                    res.error = str(e)
                res.finished = now()
                with self.lock:
                    if not hit:
                        self.in_use_bytes -= need
                    if entry is not None and key not in self.cache:
                        self.cache[key] = entry
                    active[0] -= 1
                    results[rq.rid] = res
                    self.lock.notify_all()

        threads = [threading.Thread(target=worker, args=(i,), daemon=True) for i in range(self.slots)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        return [results[r.rid] for r in sorted(requests, key=lambda r: r.rid)]

    def close(self):
        for r in self.cache.values():
            r.close()
        self.cache.clear()


def report(results: List[Result], wall_s: float) -> dict:
    ok = [r for r in results if r.ok]
    lat = sorted(r.latency for r in ok)

    def pct(q):
        if not lat:
            return None
        i = min(len(lat) - 1, max(0, int(round(q * (len(lat) - 1)))))
        return lat[i]

    dofit = sum(r.n_dofs * r.iters for r in ok)
    return {"requests": len(results), "ok": len(ok), "p50_latency_s": pct(0.5), "p99_latency_s": pct(0.99),
            "dof_iters_per_s": dofit / wall_s if wall_s > 0 else None, "wall_s": wall_s}


def poisson_stream(n: int, rate: float, meshes: List[MeshDesc], seed: int = 0, tol: float = 1e-8
                   ) -> List[Request]:
    """Poisson arrivals at `rate` per second; each request picks one of the
    given meshes and its own seeded sine right-hand side."""
    from .inputs import sine_rhs
    rng = np.random.Generator(np.random.PCG64(seed))
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    pick = rng.integers(0, len(meshes), size=n)
    return [Request(rid=i, arrival=float(t[i]), mesh=meshes[int(pick[i])], rhs=sine_rhs(2, 5000 + i), tol=tol)
            for i in range(n)]
