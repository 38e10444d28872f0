"""Open-loop Poisson load for a tt_server: requests arrive at exponential
gaps of mean 1/rate, are uploaded and submitted by one host thread at
their arrival instants and collected by another, so a slow request never
delays later arrivals.  Latency runs from the arrival instant to the
instant the server finished the request (both on the host's monotonic
clock), so it includes upload, queueing and service."""
import threading
import time

import numpy as np

from . import ttgb as T


def poisson_load(server, ctx, requests, rate, basis_ids, seed=0):
    """requests: dicts with kind ("round" | "orth"), cores (host FP64), delta,
    and for "orth" k, scheme and the (d, n) key into basis_ids.  Returns a
    dict of latency percentiles (ms), throughput (requests/s) and counts."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=len(requests))
    lock = threading.Lock()  # the context is driven by one host thread at a time
    inflight = []
    cv = threading.Condition()
    done_submitting = [False]
    errors = []
    t0 = time.monotonic() + 0.05
    arrivals = t0 + np.cumsum(gaps)

    def submitter():
        for q, ta in zip(requests, arrivals):
            now = time.monotonic()
            if ta > now:
                time.sleep(ta - now)
            try:
                with lock:
                    x = T.tt_tensor_create(ctx, q["cores"])
                if q["kind"] == "round":
                    t = server.submit_round(x, q["delta"])
                else:
                    t = server.submit_orth(x, basis_ids[(q["d"], q["n"])], q["k"], q["scheme"], q["delta"])
            except T.TTError as e:
                errors.append(e.name)
                continue
            with cv:
                inflight.append((t, x, ta, q))
                cv.notify()
        with cv:
            done_submitting[0] = True
            cv.notify()

    lat, svc, que, fin = [], [], [], []

    def collector():
        while True:
            with cv:
                while not inflight and not done_submitting[0]:
                    cv.wait()
                if not inflight:
                    return
                t, x, ta, q = inflight.pop(0)
            try:
                y, _, (ts, tb, te) = server.wait(t, coef_cap=q.get("k", 0) + 1)
                lat.append(te - ta)
                svc.append(te - tb)
                que.append(tb - ts)
                fin.append(te)
                with lock:
                    y.free()
            except T.TTError as e:
                errors.append(e.name)
            with lock:
                x.free()

    th = [threading.Thread(target=submitter), threading.Thread(target=collector)]
    for h in th:
        h.start()
    for h in th:
        h.join()
    lat = np.array(lat)
    pct = (lambda a, p: float(np.percentile(a, p) * 1e3) if len(a) else None)
    span = (max(fin) - arrivals[0]) if fin else None
    return {
        "offered_rate": rate,
        "requests": len(requests),
        "completed": int(len(lat)),
        "errors": errors,
        "throughput": (len(lat) / span) if span else None,
        "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99), "max_ms": pct(lat, 100),
        "service_p50_ms": pct(np.array(svc), 50), "service_p99_ms": pct(np.array(svc), 99),
        "queue_p50_ms": pct(np.array(que), 50), "queue_p99_ms": pct(np.array(que), 99),
    }
