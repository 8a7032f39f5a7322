"""Workload and replay driver for the serving runtime (cqr_server_*).

A workload is a set of device-resident bases and a stream of requests with
Poisson arrival times:
  * basis b has m_b rows (log-uniform in [m_lo, m_hi]) and capacity n_max;
  * a factor request picks a basis, n uniform in [n_lo, n_hi] and kappa
    log-uniform in [1e2, 1e14]; its payload is G diag(s) V^T with G Gaussian
    (m_b x n, well conditioned for m_b >> n), s log-spaced 1 -> 1/kappa and V
    a seeded orthogonal matrix, so cond(A) ~ kappa (the recipe of Sec. 4.1
    with a Gaussian instead of an orthonormal left factor); its first columns
    mix in the basis's fixed subspace S_b;
  * an append request picks a basis and p uniform in [p_lo, p_hi]; its payload
    is S_b G 0.1 + N eta with eta log-uniform in [1e-12, 1] (near-dependent on
    the basis, like the basis-growth blocks); an append that would overflow the
    basis capacity becomes a factor request.
Payloads are generated on the device before the replay (they hold none of the
method's arithmetic) and stay caller-owned until their request completes.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from .synth import seed_for


@dataclass
class Req:
    kind: str            # "factor" or "append"
    basis: int
    width: int           # n or p
    kappa: float
    arrival: float       # seconds after the start of the replay
    payload: object = None
    ticket: int = -1
    result: dict = field(default_factory=dict)


@dataclass
class Workload:
    m: list
    n_max: int
    reqs: list


def make_workload(n_bases=64, n_requests=512, mean_gap_s=2e-3, m_lo=10_000, m_hi=2_000_000,
                  n_lo=8, n_hi=128, p_lo=4, p_hi=32, factor_frac=0.5, n_max=256, seed=0) -> Workload:
    rng = np.random.default_rng(seed_for(n_bases, n_requests, seed, 0x5E))
    m = [int(round(10 ** rng.uniform(math.log10(m_lo), math.log10(m_hi)))) for _ in range(n_bases)]
    width = [0] * n_bases
    reqs = []
    t = 0.0
    for _ in range(n_requests):
        t += rng.exponential(mean_gap_s)
        b = int(rng.integers(0, n_bases))
        if rng.random() < factor_frac:
            kind, w = "factor", int(rng.integers(n_lo, n_hi + 1))
        else:
            kind, w = "append", int(rng.integers(p_lo, p_hi + 1))
            if width[b] + w > n_max:
                kind, w = "factor", int(rng.integers(n_lo, n_hi + 1))
        w = min(w, m[b])
        kappa = 10.0 ** rng.uniform(2.0, 14.0)
        width[b] = w if kind == "factor" else width[b] + w
        reqs.append(Req(kind, b, w, kappa, t))
    return Workload(m, n_max, reqs)


def make_payloads(wl: Workload, seed=0, device="cuda"):
    """Device payloads for every request (column-major float64)."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(seed_for(len(wl.m), len(wl.reqs), seed, 0x70) & 0x7FFFFFFFFFFFFFFF)
    rng = np.random.default_rng(seed_for(len(wl.m), len(wl.reqs), seed, 0x71))
    S = [torch.randn((8, mb), generator=gen, device=device, dtype=torch.float64).t() for mb in wl.m]
    for r in wl.reqs:
        mb = wl.m[r.basis]
        if r.kind == "factor":
            n = r.width
            G = torch.randn((n, mb), generator=gen, device=device, dtype=torch.float64).t()
            k = min(8, n)
            G[:, :k] = S[r.basis][:, :k]
            s = torch.from_numpy(np.logspace(0.0, -math.log10(r.kappa), n)).to(device)
            V, _ = np.linalg.qr(rng.standard_normal((n, n)))
            Vt = torch.from_numpy(np.ascontiguousarray(V.T)).to(device)
            A = (G * s) @ Vt
        else:
            p = r.width
            N = torch.randn((p, mb), generator=gen, device=device, dtype=torch.float64).t()
            Gm = torch.randn((8, p), generator=gen, device=device, dtype=torch.float64)
            eta = 10.0 ** rng.uniform(-12.0, 0.0)
            A = S[r.basis] @ Gm * 0.1 + N * eta
        out = torch.empty((A.shape[1], A.shape[0]), dtype=torch.float64, device=device).t()
        out.copy_(A)
        r.payload = out
    torch.cuda.synchronize()
    return wl


def make_bases(cq, wl: Workload):
    return [cq.Basis(mb, wl.n_max) for mb in wl.m]


def replay(cq, server, bases, wl: Workload, realtime=True):
    """Submits every request at its arrival time (realtime) or back to back,
    then waits for all.  Returns per-request results with latencies."""
    t0 = server.now()
    lag = []
    for r in wl.reqs:
        if realtime:
            while server.now() - t0 < r.arrival:
                dt = r.arrival - (server.now() - t0)
                if dt > 2e-4:
                    time.sleep(dt - 1e-4)
            lag.append(server.now() - t0 - r.arrival)
        b = bases[r.basis]
        if r.kind == "factor":
            r.ticket = server.submit_factor(b, r.payload)
        else:
            r.ticket = server.submit_append(b, r.payload)
    for r in wl.reqs:
        r.result = server.wait(r.ticket)
    return {"submit_lag_max_s": max(lag) if lag else 0.0}


def run_alone(cq, server, bases, wl: Workload):
    """Each request submitted only after the previous one completed."""
    for r in wl.reqs:
        b = bases[r.basis]
        r.ticket = server.submit_factor(b, r.payload) if r.kind == "factor" else \
            server.submit_append(b, r.payload)
        r.result = server.wait(r.ticket)


def scale_arrivals(wl: Workload, factor: float):
    """Multiplies every arrival time by `factor`: a Poisson process of rate
    lambda becomes one of rate lambda / factor with the same request order."""
    for r in wl.reqs:
        r.arrival *= factor
    return wl


def service_times(wl: Workload):
    """Per-request service time (completion - submission) of a run_alone pass."""
    return np.array([r.result["t_done"] - r.result["t_submit"] for r in wl.reqs])


def latency_stats(wl: Workload):
    lat = np.array([r.result["t_done"] - r.result["t_submit"] for r in wl.reqs])
    ok = [r for r in wl.reqs if r.result["status"] >= 0]
    t_first = min(r.result["t_submit"] for r in wl.reqs)
    t_last = max(r.result["t_done"] for r in wl.reqs)
    rows_cols = sum(wl.m[r.basis] * r.width for r in ok)
    return {"rows_cols_per_s": rows_cols / max(t_last - t_first, 1e-9),"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "max_ms": float(lat.max() * 1e3),
            "completed": len(ok), "failed": len(wl.reqs) - len(ok),
            "makespan_s": t_last - t_first, "batched": sum(1 for r in wl.reqs if r.result["batched"]),
            "max_batch": max((r.result["batch_size"] for r in wl.reqs), default=0)}
