"""Autotuner of the planning parameters: the kernel each GEMM shape runs on
and the schedule of the grouped launches.

The planner's choices (include/symtensor.h, ``sym_tune``) trade off against
one another on a given machine and workload: how narrow a sector may be and
still run faster on the tensor cores than on the CUDA cores, how far long
reductions are split across CTAs, how many positions a direct-contraction
work item covers, in which order the tensor-core tiles go to the CTAs.  They
are chosen by measurement: a coordinate descent over ``SPACE`` in which every
candidate is timed on the caller's own step -- the step re-plans under the
candidate parameters (plan caches are keyed by the tuning epoch), then CUDA
events time ``reps`` replays of a CUDA graph of the step, each after an L2
flush, following ``warmup`` eager steps, median of ``trials`` -- and a
value replaces the incumbent only when it is faster by more than ``tol``
and, given a ``check``, when its results stay accurate.
The winner is stored per (device, workload) in a JSON table that later runs
load (``load`` / ``save``); ``tune`` leaves it installed.
"""
import json
import os
import time

from . import symtensor as st
from .symtensor import SymError

SPACE = {
    "tc_all": [0, 1],                         # every GEMM on the tensor cores (one launch per phase)
    "tc_min_mn": [16, 32, 48, 64, 96, 128],  # tensor cores vs CUDA cores (sector width)
    "tc_min_k": [16, 32, 48, 64, 96],         # ... (reduction depth)
    "direct_max": [0, 2, 4],                  # direct contraction of tiny-matrix sectors
    "direct_mixed": [0, 1],                   # ... also in contractions that have GEMM sectors
    "direct_chunk": [256, 512, 1024, 2048],   # positions per direct work item
    "rows_spans": [2, 4, 8, 16],              # rows kernel: runs per warp tile
    "splitk_ctas": [0, 1, 2, 4],              # CUDA-core tiles: split k up to this many CTAs per SM
    "thin_slice": [1024, 4096, 16384],        # thin GEMMs: reduction per CTA
    "tc_order": [0, 1],                       # tcgen05 tiles: longest reduction first / sector order
    "tc_group": [0, 4, 8, 16, 32],            # tcgen05 tiles: row tiles per group (L2 panel reuse)
}

# Whole configurations a single-parameter step cannot reach from each other
# (they change several parameters at once); the descent starts from the
# fastest of these, the defaults and any stored entry.
PRESETS = (
    {"tc_all": 1, "direct_max": 4, "direct_mixed": 0},  # one tensor-core launch per GEMM phase, MPO steps direct
    {"tc_all": 1, "direct_max": 4, "direct_mixed": 1},
    {"tc_all": 0, "direct_max": 0, "tc_min_mn": 16, "tc_min_k": 16},  # no direct path, narrow sectors on tensor cores
)

TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned.json")


def device_key():
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


def time_step(step, reps=5, warmup=2, trials=3, graph=True, flush_mb=256):
    """Median over `trials` of the mean device time (ms) of one step.

    With `graph`, the step is captured once into a CUDA graph and its replays
    are timed (what a graph-replaying caller sees: no host launch cost); with
    `flush_mb`, a buffer of that size is written before every step so that
    each one starts with a cold L2, and only the step itself is timed.
    """
    import torch
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    fn, g = step, None
    if graph:
        try:
            side = torch.cuda.Stream()
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                step()
            torch.cuda.current_stream().wait_stream(side)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                step()
            fn = g.replay
            fn()
        except Exception:  # a step that cannot be captured is timed eagerly, as its caller runs it
            g, fn = None, step
            torch.cuda.synchronize()
    flush = torch.empty(flush_mb * (1 << 20) // 4, device="cuda") if flush_mb else None
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    ts = []
    for _ in range(trials):
        for e0, e1 in ev:
            if flush is not None:
                flush.fill_(1.0)
            e0.record()
            fn()
            e1.record()
        torch.cuda.synchronize()
        ts.append(sum(e0.elapsed_time(e1) for e0, e1 in ev) / reps)
    del g, fn
    return sorted(ts)[len(ts) // 2]


def tune(step, space=None, start=None, reps=5, warmup=2, trials=3, rounds=2, tol=0.02, log=None, graph=True,
         starts=PRESETS, check=None):
    """Coordinate descent over `space` from `start` (default: the current parameters).

    step() runs one step of the workload (it must plan through the cached
    plan functions, so that it re-plans after every parameter change, and
    be capturable in a CUDA graph when `graph`).  `starts` are further
    starting points, each applied over the first one (by default the presets
    above; a caller adds e.g. an earlier table entry): the descent begins at
    the fastest of them, so a search never ends worse than a known point.
    check(), if given, runs with a faster candidate's parameters installed
    and returns whether its results are still accurate enough; a candidate
    it rejects never becomes the incumbent (the kernel choice changes the
    rounding of the split-BF16 path).
    Returns (parameters, ms per step, history); the parameters are installed.
    """
    space = SPACE if space is None else space
    base = dict(st.tune_get() if start is None else start)
    history = []

    def measure(params):
        try:
            st.tune_set(**params)
        except SymError:
            return None  # out of range for this combination (e.g. tc_max_k < tc_min_k)
        t0 = time.time()
        ms = time_step(step, reps, warmup, trials, graph=graph)
        history.append({"params": dict(params), "ms": round(ms, 5), "wall_s": round(time.time() - t0, 2)})
        if log:
            log(f"tune {json.dumps(params)} -> {ms:.4f} ms")
        return ms

    def accurate(params):
        if check is None:
            return True
        st.tune_set(**params)  # measure() left them installed; set them again for clarity
        ok = bool(check())
        history[-1]["accurate"] = ok
        if not ok and log:
            log(f"tune {json.dumps(params)} rejected: results not accurate enough")
        return ok

    best = measure(base)
    if best is None:
        raise ValueError("starting parameters are out of range")
    for other in starts:
        cand = dict(base, **other)
        ms = measure(cand)
        if ms is not None and ms < best and accurate(cand):
            base, best = cand, ms
    for _ in range(rounds):
        improved = False
        for name, values in space.items():
            for v in values:
                if v == base[name]:
                    continue
                cand = dict(base, **{name: v})
                ms = measure(cand)
                if ms is not None and ms < best * (1.0 - tol) and accurate(cand):
                    base, best, improved = cand, ms, True
        if not improved:
            break
    st.tune_set(**base)
    return base, best, history


def load(workload, path=TABLE, device=None):
    """Parameters stored for (device, workload), or None."""
    if not os.path.exists(path):
        return None
    with open(path) as f:
        table = json.load(f)
    entry = table.get(f"{device or device_key()}|{workload}")
    return None if entry is None else entry["params"]


def save(workload, params, ms, default_ms, evaluations, path=TABLE, device=None):
    table = {}
    if os.path.exists(path):
        with open(path) as f:
            table = json.load(f)
    table[f"{device or device_key()}|{workload}"] = {
        "params": params, "ms_per_step": round(ms, 5), "default_ms_per_step": round(default_ms, 5),
        "evaluations": evaluations}
    with open(path, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
