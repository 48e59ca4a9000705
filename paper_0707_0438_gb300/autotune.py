"""Autotuner of the force kernel's launch shape (j-groups per CTA x j-split CTAs).

Sect. 5 of the paper notes that the best number of threads and bundles
depends on the GPU and wishes CUDA picked them itself; Sect. 3.2 splits j when
the active block is small.  Here the candidates are timed on the device,
through the C ABI, for a ladder of active-block sizes, and the winners become
the context's launch table (kirin_set_launch_table).  Results are cached in a
JSON file keyed by GPU name, SM count, precision and n_j.

For batched ensembles, tune_batch times the work decompositions (i-block size
through the j-groups per CTA, and the longest j range of a work item) on the
ensemble itself and installs the fastest (kirin_batch_set_launch).
"""
from __future__ import annotations

import json
import os

import numpy as np

from .abi import CALL_KINDS, Kirin, KirinBatch, KirinError

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "kirin_gb300", "launch_table.json")
# Tables measured on this project's GPUs (python -m paper_0707_0438_gb300.autotune --n N --out FILE).
PACKAGED = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned_launch_tables.json")


def _ladder(n_j: int):
    """Active-block sizes timed: powers of two below n_j, and n_j."""
    out, n = [], 1
    while n < n_j:
        out.append(n)
        n *= 2
    out.append(n_j)
    return out


def _candidates(auto, ntiles, big):
    """Shapes to time: every j-group count with a ladder of splits (only a few splits
    when the block alone fills the GPU many times over)."""
    g0, s0 = auto
    cands = {(g0, s0)}
    splits = (1, 2, 3, 4) if big else (1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512,
                                       768, 1024)
    for g in (1, 2, 4, 8):
        for s in splits:
            if s <= ntiles:
                cands.add((g, s))
    for s in (max(1, s0 // 2), s0 * 2):
        if s <= ntiles:
            cands.add((g0, s))
    return sorted(cands)


def _seconds_per_call(k: Kirin, call, reps: int, torch) -> float:
    """Device time of one `call` (a force launch through the C ABI).

    Short calls are replayed from a captured CUDA graph of many calls, so the
    host's launch rate does not hide the difference between shapes; long ones
    are timed directly."""
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    call()  # warm-up: buffers and kernel attributes are set up outside any capture
    ev[0].record()
    call()
    ev[1].record()
    torch.cuda.synchronize()
    t1 = ev[0].elapsed_time(ev[1]) / 1e3
    if t1 > 5e-3:
        r = max(1, reps)
        ev[0].record()
        for _ in range(r):
            call()
        ev[1].record()
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]) / 1e3 / r
    r = int(min(100, max(reps, 2e-3 / max(t1, 1e-7))))
    orig = k.stream
    side = torch.cuda.Stream()
    k.set_stream(side.cuda_stream)
    try:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            for _ in range(r):
                call()
        with torch.cuda.stream(side):
            g.replay()  # warm; finished before the timed replay, which would otherwise queue behind it
            torch.cuda.synchronize()
            ev[0].record()
            g.replay()
            ev[1].record()
        torch.cuda.synchronize()
    finally:
        k.set_stream(orig)
    return ev[0].elapsed_time(ev[1]) / 1e3 / r


def _pick(timed, tie: float = 0.005):
    """The fastest (n_i, groups, n_split, seconds); among shapes within `tie` of it, the fewest splits
    (each split adds a partial sum per i to write and reduce), then the fewest groups."""
    t_best = min(e[3] for e in timed)
    close = [e for e in timed if e[3] <= t_best * (1.0 + tie)]
    return min(close, key=lambda e: (e[2], e[1], e[3]))


def tune(k: Kirin, n_j: int, reps: int = 3, seed: int = 5, quick: bool = True, device_name: str = "",
         cache: str | None = DEFAULT_CACHE, precision: str = "mixed"):
    """Time launch shapes for the particles already set in `k` (n_j of them) and install
    the best as its launch table; returns [(n_i_max, groups, n_split, seconds), ...]."""
    import torch

    key = f"{device_name}|{precision}|{n_j}"
    if cache and os.path.exists(cache):
        try:
            table = json.load(open(cache)).get(key)
        except (OSError, ValueError):
            table = None
        if table:
            k.set_launch_table([tuple(e[:3]) for e in table])
            return table
    dev = torch.device("cuda", torch.cuda.current_device())
    rng = np.random.default_rng(seed)
    ntiles = (n_j + 127) // 128
    table = []
    for n_i in _ladder(n_j):
        il = torch.tensor(np.sort(rng.choice(n_j, n_i, replace=False)).astype(np.int32), device=dev)
        acc = torch.empty((n_i, 3), dtype=torch.float64, device=dev)
        jerk = torch.empty_like(acc)
        pot = torch.empty(n_i, dtype=torch.float64, device=dev)
        k.set_launch(0, 0)
        k.set_launch_table([])
        auto = k.get_launch(n_i)
        if auto[0] == 0:  # the tiny-block kernel serves this size; time the regular shapes around 8 groups
            auto = (8, 1)
        nsm = torch.cuda.get_device_properties(dev).multi_processor_count
        cands = _candidates(auto, ntiles, big=n_i >= 16 * nsm * 512)
        if quick:  # prune: the groups the cost model chose and its neighbours
            cands = [c for c in cands if c == auto or abs(np.log2(c[0]) - np.log2(auto[0])) <= 1]
        timed = []
        for g, s in cands:
            k.set_launch(g, s)
            timed.append((n_i, g, s, _seconds_per_call(k, lambda: k.compute_forces_dev(il, acc, jerk, pot), reps,
                                                       torch)))
        table.append(_pick(timed))
    k.set_launch(0, 0)
    k.sync()
    # each timed size covers the sizes up to the geometric mean with the next one
    entries = []
    for a, b in zip(table, table[1:] + [None]):
        hi = int(np.sqrt(float(a[0]) * b[0])) if b is not None else n_j
        entries.append((int(max(hi, a[0])), int(a[1]), int(a[2]), float(a[3])))
    k.set_launch_table([e[:3] for e in entries])
    if cache:
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        try:
            data = json.load(open(cache)) if os.path.exists(cache) else {}
        except (OSError, ValueError):
            data = {}
        data[key] = entries
        with open(cache, "w") as f:
            json.dump(data, f)
    return entries


def _key(device_name: str, precision: str, n_j: int, kind: str = "forces") -> str:
    base = f"{device_name}|{precision}|{n_j}"
    return base if kind == "forces" else f"{base}|{kind}"


def tune_full(k: Kirin, m, x, kind: str, reps: int = 3, device_name: str = "", cache: str | None = DEFAULT_CACHE,
              precision: str = "mixed"):
    """Time launch shapes of full evaluations (every particle an i) of the acceleration-and-potential
    call ("acc_pot", as the leapfrog makes) or of the adjoint ("adjoint") for the particles (m, x) on
    the device, and install the best as that kind's table; returns [(n_j, groups, n_split, seconds)]."""
    import torch

    n_j = int(m.shape[0])
    key = _key(device_name, precision, n_j, kind)
    if cache and os.path.exists(cache):
        try:
            table = json.load(open(cache)).get(key)
        except (OSError, ValueError):
            table = None
        if table:
            k.set_launch_table([tuple(e[:3]) for e in table], CALL_KINDS[kind])
            return table
    acc = torch.empty_like(x)
    pot = torch.empty_like(m)
    g = torch.randn_like(x)
    gm = torch.zeros_like(m)
    if kind == "acc_pot":
        call = lambda: k.accel_dev(m, x, acc, pot)
    elif kind == "adjoint":
        call = lambda: k.accel_adjoint_dev(m, x, g, acc, gm)
    else:
        raise ValueError(f"kind must be acc_pot or adjoint, not {kind!r}")
    ntiles = (n_j + 127) // 128
    timed = []
    for groups in (1, 2, 4, 8):
        for n_split in (1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64):
            if n_split > ntiles:
                continue
            k.set_launch(groups, n_split)
            timed.append((n_j, groups, n_split, _seconds_per_call(k, call, reps, torch)))
    best = _pick(timed)
    k.set_launch(0, 0)
    k.sync()
    entries = [tuple(best)]
    k.set_launch_table([e[:3] for e in entries], CALL_KINDS[kind])
    if cache:
        os.makedirs(os.path.dirname(cache) or ".", exist_ok=True)
        try:
            data = json.load(open(cache)) if os.path.exists(cache) else {}
        except (OSError, ValueError):
            data = {}
        data[key] = entries
        with open(cache, "w") as f:
            json.dump(data, f)
    return entries


def install(k: Kirin, n_j: int, device_name: str, precision: str = "mixed", path: str = PACKAGED) -> bool:
    """Install the stored tables for this GPU, precision and n_j, one per kind of call that has one;
    returns whether the table of full (acc, jerk, pot) calls was among them."""
    try:
        data = json.load(open(path))
    except (OSError, ValueError):
        return False
    found = False
    for kind, code in CALL_KINDS.items():
        table = data.get(_key(device_name, precision, n_j, kind))
        if table:
            k.set_launch_table([tuple(e[:3]) for e in table], code)
            found = found or kind == "forces"
    return found


# Batched ensembles: (j-groups per CTA, longest j range of a work item in tiles of 128; 0 = whole clusters).
BATCH_CANDIDATES = tuple((g, jt) for g in (1, 2, 4) for jt in (0, 64, 32, 16))


def _pick_batch(timed, tie: float = 0.005):
    """The fastest (groups, j_tiles, seconds); among those within `tie` of it, whole clusters first (no
    partial sums), then the longest j ranges, then the fewest groups."""
    t_best = min(e[2] for e in timed)
    close = [e for e in timed if e[2] <= t_best * (1.0 + tie)]
    return min(close, key=lambda e: (e[1] != 0, -e[1], e[0], e[2]))


def tune_batch(b: KirinBatch, m, x, v, dt: float = 1.0 / 256, steps: int = 2, reps: int = 2,
               candidates=BATCH_CANDIDATES, tie: float = 0.005):
    """Time the work decompositions of a batched ensemble by replaying a captured `steps`-step leapfrog
    of it (the kick and drift kernels are the same for every candidate), install the fastest and put
    the state (m, x, v) back.  Returns (groups, j_tiles, [(groups, j_tiles, seconds per step)]);
    candidates whose partial sums would exceed the library's cap are skipped."""
    import time

    timed = []
    for g, jt in candidates:
        try:
            b.set_launch(g, jt)
        except KirinError:
            continue
        b.set_state(m, x, v)
        b.leapfrog(dt, steps)  # first evaluation and graph capture
        b.sync()
        best = float("inf")
        for _ in range(reps):
            t0 = time.perf_counter()
            b.leapfrog(dt, steps)
            b.sync()
            best = min(best, time.perf_counter() - t0)
        timed.append((g, jt, best / steps))
    if not timed:
        raise ValueError("tune_batch: no candidate decomposition could be installed")
    g, jt, _ = _pick_batch(timed, tie)
    b.set_launch(g, jt)
    b.set_state(m, x, v)
    return g, jt, timed


def main(argv=None):
    import argparse

    import torch

    from . import workloads
    ap = argparse.ArgumentParser(description="time launch shapes and store the winners")
    ap.add_argument("--n", type=int, nargs="+", default=[1 << 20, 65536])
    ap.add_argument("--kinds", nargs="+", default=["forces"], choices=sorted(CALL_KINDS))
    ap.add_argument("--out", default=PACKAGED)
    ap.add_argument("--reps", type=int, default=2)
    args = ap.parse_args(argv)
    name = torch.cuda.get_device_name(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    for n in args.n:
        p = workloads.config_large(n)
        k = Kirin(n, p.eps, stream=torch.cuda.current_stream().cuda_stream)
        k.set_j_particles(p.m, p.x, p.v)
        for kind in args.kinds:
            if os.path.exists(args.out):  # re-time: drop a stored entry for this key first
                data = json.load(open(args.out))
                data.pop(_key(name, "mixed", n, kind), None)
                json.dump(data, open(args.out, "w"), indent=0)
            if kind == "forces":
                entries = tune(k, n, reps=args.reps, device_name=name, cache=args.out)
            else:
                m = torch.tensor(p.m, dtype=torch.float64, device=dev)
                x = torch.tensor(p.x, dtype=torch.float64, device=dev)
                entries = tune_full(k, m, x, kind, reps=args.reps, device_name=name, cache=args.out)
            print(n, kind, [(e[0], e[1], e[2], round(n * min(e[0], n) / e[3] / 1e9, 1)) for e in entries],
                  flush=True)
        k.close()


if __name__ == "__main__":
    main()
