"""Continuous-batching solve server on top of the C ABI.

Requests (a mesh of squares or cubes, a right-hand side, a tolerance) arrive
over time.  A dispatcher admits them into solver slots as slots and device
memory free up: every slot is a host thread with its own CUDA stream, so the
solves of different slots overlap on the GPU while new requests keep arriving.
The device state of a mesh (operator data, preconditioner, and the PCG
workspace and solve graph that dg_precond_setup creates with it) stays
resident in an LRU cache, so later requests on the same mesh skip the setup
and their solves allocate nothing.

Memory.  A resident entry is charged the device bytes its handles report
(dg_mesh_stats.device_bytes + dg_precond_stats.device_bytes).  A request on a
mesh that is not resident is admitted only when an estimate of its bytes (the
largest bytes per DOF seen so far for its dimension, or a conservative default)
fits both under the budget, next to the resident entries and the builds in
flight, and under the device's current free memory (cudaMemGetInfo) less a
reserve; idle entries are evicted, least recently used first, to make room.
An entry in use by a slot, or waited for, is pinned by a reference count taken
under the server lock and is never evicted.

Every request is solved by the same calls as a standalone solve
(dg_rhs_sine + dg_pcg_solve on its own handles), so its result does not
depend on what else is in flight.

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

# bytes per DOF assumed for a mesh of a dimension not yet seen (measured
# handles are below these: about 0.9 kB / DOF in 2D, 2.3 kB in 3D)
DEFAULT_BYTES_PER_DOF = {2: 2000, 3: 4000}
FREE_RESERVE = 512 << 20   # device memory left free for everything else


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
    dim: int = 2
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
    """Cache key of a mesh: its boxes, degrees, coefficient and geometry (the
    corners' values; a caller's map by the identity of the map object, which
    must not change while the server holds the mesh)."""
    h = hashlib.sha1()
    for a in (m.lo, m.size, m.p, np.asarray(m.extent)):
        h.update(np.ascontiguousarray(a).tobytes())
    if m.coeff is not None:
        h.update(b"coeff")
        h.update(np.ascontiguousarray(m.coeff, dtype=np.float64).tobytes())
    if getattr(m, "corners", None) is not None:
        h.update(b"corners")
        h.update(np.ascontiguousarray(m.corners, dtype=np.float64).tobytes())
    if getattr(m, "mapping", None) is not None:
        h.update(b"map%d" % id(m.mapping))
    h.update(repr((m.dim, m.lattice_h)).encode())
    return h.hexdigest()


class _Resident:
    """Mesh + preconditioner handles of one mesh.  refs (guarded by the
    server's lock) counts the slots using or waiting for it; lock serialises
    the solves on its handles (a handle is not thread-safe)."""

    def __init__(self, mesh: MeshDesc, opts):
        t = time.perf_counter()
        self.mesh = B.Mesh(mesh, opts)
        try:
            self.pc = B.Precond(self.mesh, opts)
        except Exception:
            self.mesh.close()
            raise
        self.setup_s = time.perf_counter() - t
        self.n_dofs = self.mesh.n_dofs
        self.dim = mesh.dim
        self.bytes = int(self.mesh.stats.device_bytes) + int(self.pc.stats.device_bytes)
        self.refs = 0
        self.lock = threading.Lock()

    def close(self):
        self.pc.close()
        self.mesh.close()


class Server:
    def __init__(self, slots: int = 8, precision: int = B.DG_PREC_MIXED,
                 memory_budget: Optional[int] = None, keep_solutions: bool = False,
                 cache_entries: int = 64, forms=None):
        import torch
        self.torch = torch
        self.slots = slots
        forms = forms or {2: B.DG_FORM_SIPG, 3: B.DG_FORM_BR2}
        self.opts = {d: B.make_options(form=f, precision=precision) for d, f in forms.items()}
        free, _ = torch.cuda.mem_get_info()
        self.budget = int(0.8 * free) if memory_budget is None else int(memory_budget)
        self.keep = keep_solutions
        self.cache: "OrderedDict[str, _Resident]" = OrderedDict()
        self.building: Dict[str, threading.Event] = {}
        self.waiters: Dict[str, int] = {}   # slots waiting for a build, per key
        self.reserved = 0          # estimated bytes of the builds in flight
        self.cache_entries = cache_entries
        self.bytes_per_dof: Dict[int, float] = {}
        self.lock = threading.Condition()
        self.peak_bytes = 0
        self.max_inflight = 0
        self.evictions = 0
        self.refused_for_memory = 0

    # ---------------------------------------------------------------- memory
    def _resident_bytes(self) -> int:
        return sum(r.bytes for r in self.cache.values())

    def estimate(self, mesh: MeshDesc) -> int:
        bpd = self.bytes_per_dof.get(mesh.dim, DEFAULT_BYTES_PER_DOF.get(mesh.dim, 4000))
        return int(bpd * mesh.n_dofs())

    def _evict_one(self) -> bool:
        """Close the least recently used idle entry (lock held)."""
        for k, r in self.cache.items():
            if r.refs == 0:
                self.cache.pop(k).close()
                self.evictions += 1
                return True
        return False

    def _make_room(self, need: int) -> bool:
        """Evict idle entries until `need` more bytes fit under the budget and
        the device's free memory, and the cache has a free entry (lock held)."""
        torch = self.torch
        while True:
            fits_budget = self._resident_bytes() + self.reserved + need <= self.budget
            fits_count = len(self.cache) + len(self.building) < self.cache_entries
            fits_device = True
            if fits_budget and fits_count:
                free, _ = torch.cuda.mem_get_info()
                fits_device = need + FREE_RESERVE <= free
                if fits_device:
                    return True
            if not self._evict_one():   # cudaFree returns the memory before it returns
                return False

    # ---------------------------------------------------------------- run
    def run(self, requests: List[Request], realtime: bool = True) -> List[Result]:
        torch = self.torch
        pending = sorted(requests, key=lambda r: r.arrival)
        ready: List = []   # heap of (arrival, rid, request)
        results: Dict[int, Result] = {}
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        state = {"active": 0}

        def admit():
            """Next request to start, as (request, key, mode, entry, event,
            need); mode: "hit" (entry pinned), "wait" (another slot builds the
            mesh; event set when done) or "build" (this slot builds it, need
            bytes reserved).  None when the run is over.  Lock held."""
            while True:
                while pending and (not realtime or pending[0].arrival <= now()):
                    rq = pending.pop(0)
                    heapq.heappush(ready, (rq.arrival, rq.rid, rq))
                if ready:
                    rq = ready[0][2]
                    key = mesh_key(rq.mesh)
                    entry = self.cache.get(key)
                    if entry is not None:
                        heapq.heappop(ready)
                        entry.refs += 1
                        self.cache.move_to_end(key)
                        return rq, key, "hit", entry, None, 0
                    if key in self.building:
                        # the builder pins the entry for every waiter
                        heapq.heappop(ready)
                        self.waiters[key] = self.waiters.get(key, 0) + 1
                        return rq, key, "wait", None, self.building[key], 0
                    need = self.estimate(rq.mesh)
                    idle = state["active"] == 0 and not self.building
                    room = self._make_room(need)
                    if room or idle:
                        if not room:
                            # nothing else is in flight: try anyway, the
                            # library reports DG_ENOMEM if it does not fit
                            while self._evict_one():
                                pass
                        heapq.heappop(ready)
                        ev = threading.Event()
                        self.building[key] = ev
                        self.reserved += need
                        return rq, key, "build", None, ev, need
                    self.refused_for_memory += 1
                if not pending and not ready:
                    return None
                wait = 0.05
                if realtime and pending and not ready:
                    wait = max(0.0, min(wait, pending[0].arrival - now()))
                self.lock.wait(timeout=wait)

        def worker(slot: int):
            stream = torch.cuda.Stream()
            while True:
                with self.lock:
                    got = admit()
                    if got is None:
                        return
                    rq, key, mode, entry, ev, need = got
                    state["active"] += 1
                    self.max_inflight = max(self.max_inflight, state["active"])
                res = Result(rid=rq.rid, ok=False, arrival=rq.arrival, admitted=now(), dim=rq.mesh.dim)
                try:
                    if mode == "wait":
                        ev.wait()
                        with self.lock:
                            entry = self.cache.get(key)   # pinned for this slot by the builder
                        if entry is None:
                            raise RuntimeError("setup of this mesh failed in another slot")
                    elif mode == "build":
                        built = None
                        try:
                            built = _Resident(rq.mesh, self.opts[rq.mesh.dim])
                            res.setup_s = built.setup_s
                        finally:
                            with self.lock:
                                self.reserved -= need
                                n_wait = self.waiters.pop(key, 0)
                                if built is not None:
                                    built.refs = 1 + n_wait
                                    self.cache[key] = built
                                    bpd = built.bytes / max(built.n_dofs, 1)
                                    self.bytes_per_dof[built.dim] = max(self.bytes_per_dof.get(built.dim, 0.0),
                                                                        bpd)
                                    self.peak_bytes = max(self.peak_bytes, self._resident_bytes())
                                del self.building[key]
                                ev.set()
                                self.lock.notify_all()
                        entry = built
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
                    if entry is not None:
                        entry.refs -= 1
                    state["active"] -= 1
                    results[rq.rid] = res
                    self.lock.notify_all()

        threads = [threading.Thread(target=worker, args=(i,), daemon=True) for i in range(self.slots)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        return [results[r.rid] for r in sorted(requests, key=lambda r: r.rid)]

    def close(self):
        with self.lock:
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
            "dof_iters_per_s": dofit / wall_s if wall_s > 0 else None, "wall_s": wall_s,
            "requests_3d": sum(1 for r in results if r.dim == 3)}


def poisson_stream(n: int, rate: float, meshes: List[MeshDesc], seed: int = 0, tol: float = 1e-8
                   ) -> List[Request]:
    """Poisson arrivals at `rate` per second; each request picks one of the
    given meshes (squares or cubes) and its own seeded sine right-hand side."""
    from .inputs import sine_rhs
    rng = np.random.Generator(np.random.PCG64(seed))
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    pick = rng.integers(0, len(meshes), size=n)
    out = []
    for i in range(n):
        m = meshes[int(pick[i])]
        out.append(Request(rid=i, arrival=float(t[i]), mesh=m, rhs=sine_rhs(m.dim, 5000 + i), tol=tol))
    return out
