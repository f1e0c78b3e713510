"""Drive the request loop (wrs_server_*) with a timed request stream.

`replay` submits each operation of a stream (see inputs.serving_stream) at
its arrival time, from one submitting thread, while the server's worker runs
steps on the GPU; then waits for every request.  Weights are generated on
the device from each build's seed (seeded torch generator) so that the
submitter is not slowed by host-side generation; sample outputs go to
device buffers.
"""
from __future__ import annotations

import time

import torch


def make_weights(n: int, kind: str, seed: int) -> torch.Tensor:
    """Device weights of a serving build: U[0,1) or w = 1/rank (shuffled)."""
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    if kind == "uniform":
        return torch.rand(n, generator=g, device="cuda", dtype=torch.float32)
    rank = torch.randperm(n, generator=g, device="cuda").to(torch.float64) + 1.0
    return (1.0 / rank).to(torch.float32)


def replay(server, ops, realtime: bool = True):
    """Submit `ops` (arrival times in seconds from now) and wait for all.

    Returns (tickets, outputs, weights): per op index the server ticket, the
    sample output tensor (samples) and the weight tensor (builds)."""
    weights = {}
    for k, op in enumerate(ops):
        if op["op"] == "build":
            weights[k] = make_weights(op["n"], op["kind"], op["wseed"])
    torch.cuda.synchronize()
    outputs, tickets = {}, {}
    t0 = time.perf_counter()
    for k, op in enumerate(ops):
        if realtime:
            delay = op["t"] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
        if op["op"] == "build":
            tickets[k] = server.build(weights[k])
        elif op["op"] == "sample":
            out = torch.empty(max(op["count"], 1), dtype=torch.int32, device="cuda")
            outputs[k] = out
            tickets[k] = server.sample(tickets[op["table"]], op["count"], op["seed"], out,
                                       stream_lo=op["stream"])
        else:
            tickets[k] = server.release(tickets[op["table"]])
    status = {k: server.wait(t) for k, t in tickets.items()}
    return tickets, outputs, weights, status
