"""Simulated MPC controllers driving the serving loop (prism_server_*).

Each controller has a fixed (J, H, N) drawn like the uneven multi-problem
workload and issues one projection request per control step of 20 ms, with
an exponential (Poisson-process) delay of mean ``jitter_ms`` after its step
boundary.  Every ``burst_every_s`` seconds all controllers fire within
``burst_window_ms`` (32 controllers in 6.4 ms is a 5 000 req/s burst).
Requests are submitted at their arrival times from one thread and collected
from another; latency is measured by the server from submission to the
completion of the result copy.
"""
from __future__ import annotations

import math
import threading
import time

import numpy as np

from . import prism_proj as pp
from . import workloads


def make_controllers(n: int = 32, seed: int = 1004, n_lo: int = 128, n_hi: int = 8192,
                     prec: int = pp.PREC_TF32X3, pool: int = 3, iters: int = 150):
    """Controllers with (J, H, N, dt, bounds scale) drawn like the uneven workload,
    each with ``pool`` pinned sample / result buffers that its requests cycle."""
    import torch
    probs = workloads.batched_problems(n, seed=seed, n_lo=n_lo, n_hi=n_hi)
    ctrls = []
    for k, pr in enumerate(probs):
        P = pp.Projector(pr.J, pr.H, pr.dt, pr.bounds)
        P.factor(1.0, pp.MODE_ADMM, pp.SCALE_ROWNORM,
                 prec if pr.H <= pp.TC_MAX_H else pp.PREC_FP32)
        xs = []
        for q in range(pool):
            b = workloads.draw_batch(np.random.default_rng([seed, k, q]), pr.N, pr.J, pr.H, pr.bounds)
            xs.append(torch.from_numpy(b["xi"]).pin_memory())
        ctrls.append({"proj": P, "N": pr.N, "J": pr.J, "H": pr.H, "iters": iters,
                      "q0": torch.from_numpy(pr.q0).pin_memory(), "v0": torch.from_numpy(pr.v0).pin_memory(),
                      "xs": xs, "outs": [torch.empty_like(x).pin_memory() for x in xs]})
    return ctrls


def arrival_times(n_ctrl: int, steps: int, period_ms: float = 20.0, jitter_ms: float = 2.0,
                  burst_every_s: float = 1.0, burst_window_ms: float = 6.4, seed: int = 7):
    """Sorted (time_s, controller, step) arrivals."""
    rng = np.random.default_rng(seed)
    phase = rng.uniform(0, period_ms, n_ctrl)
    out = []
    burst_steps = max(1, int(round(burst_every_s * 1e3 / period_ms)))
    for c in range(n_ctrl):
        for k in range(steps):
            if k > 0 and k % burst_steps == 0:
                t = k * period_ms + rng.uniform(0, burst_window_ms)
            else:
                t = k * period_ms + phase[c] + rng.exponential(jitter_ms)
            out.append((t / 1e3, c, k))
    out.sort()
    return out


def run(server: pp.Server, ctrls, steps: int, **arrival_kw) -> dict:
    """Drive ``steps`` requests per controller through ``server``; returns stats."""
    ids = [server.add_controller(c["proj"], c["N"], c["iters"], warm=True) for c in ctrls]
    arrivals = arrival_times(len(ctrls), steps, **arrival_kw)
    tickets = []
    lock = threading.Lock()
    done_submitting = threading.Event()
    results = {"states": {}}

    def collector():
        k = 0
        while True:
            with lock:
                pending = tickets[k:]
            if not pending:
                if done_submitting.is_set():
                    with lock:
                        if k >= len(tickets):
                            return
                time.sleep(0.0005)
                continue
            for t in pending:
                try:
                    st, _ = server.wait(t)
                except pp.PrismError:
                    st = "failed"
                results["states"][st] = results["states"].get(st, 0) + 1
                k += 1

    th = threading.Thread(target=collector, daemon=True)
    th.start()
    server.reset_stats()
    t0 = time.perf_counter() + 0.05
    for (ta, c, k) in arrivals:
        delay = t0 + ta - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        cc = ctrls[c]
        slot = k % len(cc["xs"])
        t = server.submit(ids[c], cc["q0"], cc["v0"], cc["xs"][slot], cc["outs"][slot])
        with lock:
            tickets.append(t)
    done_submitting.set()
    th.join()
    wall = time.perf_counter() - t0
    st = server.stats()
    st["requests"] = len(arrivals)
    st["offered_req_per_s"] = len(arrivals) / (arrivals[-1][0] + 1e-9)
    st["wall_s"] = wall
    st["states"] = results["states"]
    return st
