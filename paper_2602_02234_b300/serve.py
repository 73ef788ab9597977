"""Serving driver: feed timed requests to a ``dp_server`` and collect latencies.

Requests arrive on the wall clock (each has ``arrival_s``); the loop submits
every request whose time has come, runs one server tick (one MD step of all
resident systems), and collects finished results.  Returns per-request
latencies and the server's tick statistics.
"""
from __future__ import annotations

import time

import numpy as np

from . import Server


def run(server: Server, requests, velocities, timeout_s: float = 600.0):
    """requests: objects with .system (coords, types, box), .n_steps, .arrival_s;
    velocities: list of (n, 3) arrays.  Returns (results, stats)."""
    order = sorted(range(len(requests)), key=lambda k: requests[k].arrival_s)
    ids = {}
    results = {}
    t0 = time.perf_counter()
    nxt = 0
    pending = set()
    while len(results) < len(requests):
        now = time.perf_counter() - t0
        if now > timeout_s:
            raise TimeoutError("serving run did not finish")
        while nxt < len(order) and requests[order[nxt]].arrival_s <= now:
            k = order[nxt]
            r = requests[k]
            ids[k] = server.submit(r.system.types, r.system.box, r.system.coords, velocities[k],
                                   r.n_steps)
            pending.add(k)
            nxt += 1
        n_active, n_queued = server.tick()
        for k in list(pending):
            out = server.poll(ids[k])
            if out is not None:
                results[k] = out
                pending.discard(k)
        if n_active == 0 and n_queued == 0 and nxt < len(order):
            time.sleep(max(0.0, min(0.01, requests[order[nxt]].arrival_s - now)))
    wall = time.perf_counter() - t0
    st = server.stats()
    lat = np.array([results[k][3]["total_ms"] for k in results])
    st.update(wall_s=wall, request_p50_ms=float(np.percentile(lat, 50)),
              request_p99_ms=float(np.percentile(lat, 99)),
              atom_steps_per_s=st["atom_steps"] / (st["busy_ms"] / 1e3) if st["busy_ms"] else 0.0)
    return results, st
