"""Serving loop: independent periodic D3Q19 solves arriving as a Poisson stream.

Two schedulers over the same seeded request trace:
  * ``serve_pool``  -- continuous batching on the pool (``lbm_pool_*``): requests are
    admitted while the arena has room, every resident request advances inside the same
    batched kernel launches, finished ones leave at chunk boundaries and new ones join;
  * ``serve_plain`` -- first in, first out, one request at a time on the single-lattice
    kernel (``lbm_create`` / ``lbm_step`` / ``lbm_get_moments``), the comparison baseline.
Latency of a request = time its result reaches the host minus its arrival time.

Trace (seeded): cube side round(exp(U(ln 32, ln 128))), tau ~ U[0.52, 1.0], Taylor-Green
u0 ~ U[0.01, 0.08], steps ~ U{100..2000}, Poisson arrivals at ``rate`` per second.
"""
import collections
import math
import queue
import threading
import time

import numpy as np

from . import fields, lbm

T0_D3Q19 = 1.0 / 3.0


def make_trace(n, rate=50.0, config_index=4, salt=0, side=(32, 128), tau=(0.52, 1.0), u0=(0.01, 0.08),
               steps=(100, 2000)):
    g = fields.rng(config_index, salt)
    gaps = g.exponential(1.0 / rate, size=n)
    arrivals = np.cumsum(gaps) - gaps[0]
    sides = np.rint(np.exp(g.uniform(math.log(side[0]), math.log(side[1]), size=n))).astype(int)
    taus = g.uniform(tau[0], tau[1], size=n)
    u0s = g.uniform(u0[0], u0[1], size=n)
    nsteps = g.integers(steps[0], steps[1] + 1, size=n)
    return [{"i": i, "arrival": float(arrivals[i]), "side": int(sides[i]), "tau": float(taus[i]),
             "u0": float(u0s[i]), "steps": int(nsteps[i])} for i in range(n)]


def request_fields(r):
    d = (r["side"],) * 3
    return fields.taylor_green_3d(d, r["u0"], T0_D3Q19)


class Producer:
    """Client side: generates each request's initial fields ahead of its arrival, in arrival
    order, on a background thread (bounded look-ahead), so that the scheduler loop only
    admits, advances and collects."""

    def __init__(self, trace, ahead=32):
        self.order = sorted(trace, key=lambda r: r["arrival"])
        self.q = queue.Queue(maxsize=ahead)
        self.thread = threading.Thread(target=self._run, daemon=True)
        self.thread.start()

    def _run(self):
        for r in self.order:
            self.q.put((r, request_fields(r)))

    def next(self):
        return self.q.get()


def _summary(lat, t_total, cells):
    lat = np.array(sorted(lat))
    return {"solves": int(len(lat)), "seconds": t_total, "solves_per_s": len(lat) / t_total,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "mean_latency_s": float(lat.mean()), "glups": cells / t_total / 1e9}


def serve_pool(trace, K=3, storage="f32", arena_bytes=48 << 30, max_slots=512, chunk=50, keep=None,
               autotune=True, storage_range=None):
    """Continuous batching.  keep: optional set of request indices whose results are returned.
    storage_range: range of a fixed-point pool ("q16")."""
    pool = lbm.Pool("D3Q19", K, storage, arena_bytes, max_slots, storage_range=storage_range)
    producer = Producer(trace)
    pending = collections.deque(sorted(trace, key=lambda r: r["arrival"]))
    waiting = collections.deque()
    ready = {}
    active = {}
    lat, results = [], {}
    cells = 0
    tuned = not autotune
    t0 = time.perf_counter()
    while pending or waiting or active:
        now = time.perf_counter() - t0
        while pending and pending[0]["arrival"] <= now:
            waiting.append(pending.popleft())
        while waiting:
            r = waiting[0]
            while r["i"] not in ready:
                rr, fl = producer.next()
                ready[rr["i"]] = fl
            rho, u = ready[r["i"]]
            rid = pool.submit((r["side"],) * 3, r["tau"], rho, u, r["steps"])
            if rid is None:
                break
            del ready[r["i"]]
            active[rid] = r
            waiting.popleft()
        if not tuned and len(active) >= 8:
            lbm.lbm_pool_autotune(pool.handle, 3)
            tuned = True
        n = pool.advance(chunk) if active else 0
        for rid in list(active):
            done, _ = pool.poll(rid)
            if done:
                r = active.pop(rid)
                C = r["side"] ** 3
                rho, u = pool.result(rid, C)
                lat.append(time.perf_counter() - t0 - r["arrival"])
                cells += C * r["steps"]
                if keep is not None and r["i"] in keep:
                    results[r["i"]] = (rho, u)
        if n == 0 and not active:
            if pending and not waiting:
                time.sleep(max(0.0, min(0.01, pending[0]["arrival"] - (time.perf_counter() - t0))))
        elif n == 0:
            pool.sync()
    t_total = time.perf_counter() - t0
    pool.close()
    out = _summary(lat, t_total, cells)
    out["chunk"] = chunk
    return out, results


def serve_plain(trace, K=3, storage="f32", keep=None):
    """FIFO, one request at a time on the single-lattice kernel (one reused workspace)."""
    import torch

    stream = torch.cuda.current_stream()
    smax = max(r["side"] for r in trace)
    ws_bytes = lbm.lbm_workspace_bytes("D3Q19", (smax,) * 3, storage)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    producer = Producer(trace)
    lat, results = [], {}
    cells = 0
    t0 = time.perf_counter()
    for _ in range(len(trace)):
        r, (rho, u) = producer.next()
        now = time.perf_counter() - t0
        if r["arrival"] > now:
            time.sleep(r["arrival"] - now)
        d = (r["side"],) * 3
        C = r["side"] ** 3
        h = lbm.lbm_create("D3Q19", d, r["tau"], K, storage, 1.0, ws.data_ptr(), ws_bytes, stream.cuda_stream)
        lbm.lbm_set_fields(h, rho, u)
        lbm.lbm_step(h, r["steps"])
        ro = np.empty(C)
        uo = np.empty((3, C))
        lbm.lbm_get_moments(h, ro, uo)
        lbm.lbm_destroy(h)
        lat.append(time.perf_counter() - t0 - r["arrival"])
        cells += C * r["steps"]
        if keep is not None and r["i"] in keep:
            results[r["i"]] = (ro, uo)
    t_total = time.perf_counter() - t0
    return _summary(lat, t_total, cells), results


def batched_rate(n=40, steps=200, storage="f32", K=3, chunk=50, salt=5, autotune=True, kernel=None):
    """Throughput of the batched step alone: n resident D3Q19 Taylor-Green lattices drawn like
    the trace (sides log-uniform 32-128, tau, u0), every one with more steps left than are run,
    advanced `steps` steps in chunks of `chunk`; timed with CUDA events on the pool's compute
    stream after one untimed chunk (and the autotuner, unless a kernel (cells per thread,
    block) is given).  Returns MLUPS, bytes per update and the kernel configuration."""
    import torch

    trace = make_trace(n, salt=salt)
    cells = sum(r["side"] ** 3 for r in trace)
    Q = lbm.lbm_lattice_info("D3Q19")["Q"]
    arena = sum(lbm.lbm_pool_request_bytes("D3Q19", (r["side"],) * 3, storage) for r in trace) + (64 << 20)
    pool = lbm.Pool("D3Q19", K, storage, arena, max(n, 1))
    try:
        for r in trace:
            rho, u = request_fields(r)
            if pool.submit((r["side"],) * 3, r["tau"], rho, u, 10 * (steps + chunk)) is None:
                raise RuntimeError("pool refused a request of the batched workload")
        if kernel is not None:
            lbm.lbm_pool_set_kernel(pool.handle, *kernel)
        pool.advance(chunk)
        if autotune and kernel is None:
            lbm.lbm_pool_autotune(pool.handle, 20)
        pool.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(pool.compute)
        done = 0
        while done < steps:
            m = min(chunk, steps - done)
            pool.advance(m)
            done += m
        e1.record(pool.compute)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        cpt, block = lbm.lbm_pool_get_kernel(pool.handle)
    finally:
        pool.close()
    return {"workload": "%d resident D3Q19 lattices (sides log-uniform 32-128, %d cells), %s, K=%d, %d steps"
                        % (n, cells, storage, K, steps),
            "MLUPS": cells * steps / (ms / 1e3) / 1e6, "bytes_per_update": 2 * Q * lbm.STORAGE_BYTES[storage],
            "ms_per_step": ms / steps, "kernel": {"cells_per_thread": cpt, "block": block}}


def served_accuracy(n=24, salt=7, forms=(("f32", None), ("f16", None), ("bf16", None), ("q16", 0.5), ("q16", 0.0))):
    """Accuracy of served results per storage form: n requests drawn like the trace, all offered at
    once, served by a pool of each form; u compared with the FP32 single-lattice solver on the same
    request (which matches the FP64 oracle within 1e-5).  Two measures per form: max|du| / max|u| on
    the requests whose flow still holds at least a tenth of its initial amplitude u0 (many requests
    decay by orders of magnitude over their steps, and then any rounding is large next to u), and
    max|du| / u0 on every request.  The fixed-point pools run with one range, 1/2 (it holds the
    trace's flows: |h| below about 0.3 for u0 <= 0.08), and with each request's own range chosen
    at admission (range 0)."""
    trace = [dict(r, arrival=0.0) for r in make_trace(n, salt=salt)]
    keep = {r["i"] for r in trace}
    _, ref = serve_plain(trace, keep=keep)
    live = [r["i"] for r in trace if np.max(np.abs(ref[r["i"]][1])) >= 0.1 * r["u0"]]
    out = {"requests": n, "live_requests": len(live),
           "reference": "FP32 single-lattice solver, same requests"}
    for storage, R in forms:
        _, res = serve_pool(trace, storage=storage, keep=keep, storage_range=R)
        rel = [float(np.max(np.abs(res[i][1] - ref[i][1])) / np.max(np.abs(ref[i][1]))) for i in live]
        by_u0 = [float(np.max(np.abs(res[r["i"]][1] - ref[r["i"]][1])) / r["u0"]) for r in trace]
        key = storage if R is None else ("%s (range auto)" % storage if R == 0.0 else "%s (range %g)" % (storage, R))
        out[key] = {"max_rel_u_live": max(rel) if rel else None,
                    "median_rel_u_live": float(np.median(rel)) if rel else None,
                    "max_du_over_u0": max(by_u0)}
    return out
