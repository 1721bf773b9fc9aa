"""Driver of the request loop: submits a stream of steady solves at their arrival times to
an ``emg_server`` and collects time-to-converge statistics.

All scheduling decisions (admission by slots and memory, one V-cycle in flight per solve,
convergence checks) are made by the library; this module only keeps the arrival clock.
"""
import time

import numpy as np

from ._lib import Server


def percentile(xs, q):
    return float(np.percentile(np.asarray(xs, dtype=np.float64), q)) if len(xs) else float("nan")


def serve_stream(requests, make_mesh, max_active=8, mem_budget=0, drop=1e-10, max_cycles=3000, prec=1,
                 keep_state=False, idle_sleep=1e-4, stall_cycles=0):
    """Run ``requests`` (objects with arrival, p, mach and a mesh key understood by
    ``make_mesh``) through one server.  Returns (per-request results in stream order,
    summary).  Time-to-converge counts from the nominal arrival time, so any lag of the
    submission itself is included."""
    srv = Server(max_active=max_active, mem_budget=mem_budget, drop=drop, max_cycles=max_cycles,
                 keep_state=keep_state, stall_cycles=stall_cycles)
    order = sorted(range(len(requests)), key=lambda k: requests[k].arrival)
    by_id, out, states = {}, [None] * len(requests), {}
    t0 = srv.clock()
    nxt = 0
    peak_active = 0
    while any(r is None for r in out):
        now = srv.clock() - t0
        while nxt < len(order) and requests[order[nxt]].arrival <= now:
            k = order[nxt]
            rq = requests[k]
            rid = srv.submit(make_mesh(rq), p_max=rq.p, mach=rq.mach, prec=prec)
            by_id[rid] = k
            nxt += 1
        active, queued = srv.step()
        peak_active = max(peak_active, active)
        got = srv.results()
        for res in got:
            k = by_id[res["id"]]
            res["arrival"] = t0 + requests[k].arrival
            res["time_to_converge"] = res["t_done"] - res["arrival"]
            out[k] = res
            if keep_state and res["status"] == 0:
                states[k] = srv.take_state(res["id"])
        if not got:
            time.sleep(idle_sleep)
    srv.close()
    ok = [r for r in out if r["status"] == 0]
    ttc = [r["time_to_converge"] for r in ok]
    span = max(r["t_done"] for r in out) - t0
    summary = {"requests": len(requests), "converged": len(ok), "p50_s": percentile(ttc, 50),
               "p99_s": percentile(ttc, 99), "makespan_s": span, "solves_per_s": len(ok) / span if span > 0 else 0.0,
               "peak_active": peak_active, "max_active": max_active,
               "cycles_total": int(sum(r["cycles"] for r in out))}
    if keep_state:
        return out, summary, states
    return out, summary
