#!/usr/bin/env python
"""Benchmark: symmetric block-sparse contraction, forward + backward, on one GB300.

Default workload (the large-sector configuration, SU(2) with recoupling):
rank-4 SU(2)-invariant tensors whose legs carry 2j = 0..8 with degeneracies
drawn uniformly in 1..32 (seeded); A (comb tree, all legs out) is recoupled
by 6j coefficients into the matrix tree and its legs 1, 3 are contracted
with the dual legs 0, 1 of B.  One step = C = contract(A, B) forward and the
gradients of <G, C> with respect to A and B (autograd through the library's
adjoint), on N(0,1) blocks.  Other workloads (--workload): the U(1) MPS
effective-Hamiltonian apply, the 512-problem batch, the MERA gradient, the
fermionic and SU(2) x U(1) MPS chains, the blockwise SVD and the SU(2)
micro-benchmarks.

Metric: useful TFLOP/s = block-sparse GEMM flops (sum over sectors of 2 m n k,
forward + backward) / device time.  Reported for the split-BF16 x3 tcgen05
path (the value), next to the plain FP64 GPU path and the FP64 CPU oracle,
with the relative error against both.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload W]

Rank 0 prints one JSON line.  Under torchrun (N > 1) every rank runs the same
workload on its own GPU (replicas; weak scaling) and the slowest rank's time
is used.  L2 is flushed (a 256 MiB write) between timed steps; each step is
bracketed by CUDA events on the compute stream.
"""
import argparse
import inspect
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "useful TFLOP/s of symmetric block-sparse contraction fwd+bwd vs plain FP64 GPU"
SPLIT_BF16_TOL = 2e-5  # relative error bar of the split-BF16 x3 path against FP64
WORKLOAD = ("u1_mps_heff: ((L.A).W).R fwd+bwd, D=2048 over q=-20..20 (gaussian sigma=6), "
            "phys {0:1,1:1}, MPO w=5 {-1:1,0:3,+1:1}")
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--workload", choices=["u1_mps_heff", "su2_recouple", "u1_two_site_batch", "u1_mera_grad",
                                           "z2f_mps_heff", "su2u1_mps_heff", "u1_two_site_svd", "u1_two_site_eig",
                                           "su2_micro"],
                    default="su2_recouple",
                    help="su2_recouple (default: the large-sector SU(2) recoupling contraction at full size), "
                         "the U(1) MPS chain u1_mps_heff, the 512-problem u1_two_site_batch, the MERA gradient "
                         "u1_mera_grad, ...")
    ap.add_argument("--su2-dmax", type=int, default=32,
                    help="su2_recouple: largest degeneracy (32 = the full configuration; smaller sizes serve "
                         "profiler captures of the same kernels)")
    ap.add_argument("--steps", type=int, default=None, help="timed steps (default 20 for su2_recouple)")
    ap.add_argument("--warmup", type=int, default=None, help="warm-up steps (default 5)")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--fp64-steps", type=int, default=None, help="FP64 comparator steps (default 10; su2_recouple 1)")
    ap.add_argument("--cpu-sample-steps", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="launch eagerly instead of replaying a CUDA graph")
    ap.add_argument("--tune", choices=["table", "search", "off"], default="table",
                    help="planning parameters: the autotuned table entry for this device and workload (default; "
                         "the library defaults when there is none), a new autotuner search (stored in "
                         "--tune-table), or the library defaults")
    ap.add_argument("--tune-table", default=None, help="autotuner table (default paper_1203_2222_gb300/tuned.json)")
    ap.add_argument("--batch-n", type=int, default=512,
                    help="u1_two_site_batch: number of problems (512 at full size; fewer for a small profiling case)")
    ap.add_argument("--tune-space", default=None,
                    help="comma-separated planning parameters the search varies (default: all of autotune.SPACE)")
    args = ap.parse_args()
    wl = ({"u1_two_site_svd": SVDWorkload, "u1_two_site_eig": EigWorkload, "su2_micro": MicroWorkload}
          .get(args.workload) or WORKLOADS[args.workload])
    args.steps = wl.default_steps if args.steps is None else args.steps
    args.warmup = wl.default_warmup if args.warmup is None else args.warmup
    args.fp64_steps = wl.default_fp64_steps if args.fp64_steps is None else args.fp64_steps
    return args


# ----------------------------------------------------------------- helpers ---

L2_POLICY = "flushed between timed steps (256 MiB write)"


def bench_config(describe):
    """The `config` of both arms' JSON lines (the same dict, so that the two
    lines name the same configuration): the workload and the L2 policy of the
    GPU arm's timed steps."""
    return {"workload": describe, "l2": L2_POLICY}


def max_over_ranks(x, world, device=None):
    """The largest of every rank's x (a job takes as long as its slowest
    rank); x itself on one rank.  Every rank must call it."""
    if world <= 1:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank_step, steps, world, ms):
    """Units per second of the whole job: every rank (a replica) processes
    units_per_rank_step per step, and the job takes ms for `steps` steps."""
    return units_per_rank_step * steps * world / (ms * 1e-3)


def load_peaks():
    try:
        with open(PEAKS_PATH) as f:
            p = json.load(f)
        return p, "measured"
    except (OSError, ValueError):
        return dict(FALLBACK_PEAKS), "fallback"


class ClockSampler:
    """SM clock, power and clock-event reasons sampled during a timed region.

    Read-only NVML queries (through ctypes, no Python binding needed) from a
    thread polling every 2 ms, so that even a region of a few milliseconds
    gets samples; the device is looked up by UUID so that the index mapping
    of CUDA_VISIBLE_DEVICES cannot pick another GPU.  Falls back to
    ``nvidia-smi -lms 200`` when NVML cannot be loaded.
    """

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        import threading
        self.device = device
        self.rows = []
        self.stop_evt = threading.Event()
        self.thread = None
        self.proc = None
        self.nvml = self.handle = None
        self.source = None
        try:
            import ctypes
            import torch
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                raise OSError("nvmlInit failed")
            uuid = "GPU-" + str(torch.cuda.get_device_properties(device).uuid)
            h = ctypes.c_void_p()
            if lib.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(h)) != 0:
                raise OSError("device not found by UUID")
            self.nvml, self.handle, self.ct = lib, h, ctypes
            self.reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                lib.nvmlDeviceGetCurrentClocksThrottleReasons
            self.source = "nvml"
        except Exception:
            self.nvml = None

    def _poll(self):
        ct, lib, h = self.ct, self.nvml, self.handle
        clk, mx, mw, rs = ct.c_uint(), ct.c_uint(), ct.c_uint(), ct.c_ulonglong()
        while not self.stop_evt.is_set():
            ok = lib.nvmlDeviceGetClockInfo(h, 1, ct.byref(clk)) == 0  # NVML_CLOCK_SM
            ok = ok and lib.nvmlDeviceGetMaxClockInfo(h, 1, ct.byref(mx)) == 0
            ok = ok and self.reasons_fn(h, ct.byref(rs)) == 0
            if ok:
                pw = mw.value / 1000.0 if lib.nvmlDeviceGetPowerUsage(h, ct.byref(mw)) == 0 else None
                self.rows.append((float(clk.value), float(mx.value), pw, int(rs.value)))
            self.stop_evt.wait(0.002)

    def start(self):
        import threading
        if self.nvml is not None:
            self.thread = threading.Thread(target=self._poll, daemon=True)
            self.thread.start()
            return
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
            self.source = "nvidia-smi"
            time.sleep(1.0)  # let the first samples arrive before the region starts
        except OSError:
            self.proc = None

    def stop(self):
        if self.thread is not None:
            self.stop_evt.set()
            self.thread.join()
            sm = [r[0] for r in self.rows]
            mx = [r[1] for r in self.rows]
            pw = [r[2] for r in self.rows if r[2] is not None]
            reasons = sorted({n for r in self.rows for bit, n in self.REASONS.items() if r[3] & bit})
        elif self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()
            rows = []
            with open(self.path) as f:
                for line in f:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
            os.unlink(self.path)
            sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
            mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
            pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        else:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no clock source"], "samples": 0}
        load = [x for x in sm if mx and x >= 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_median": statistics.median(pw) if pw else None,
                "reasons": reasons, "samples": len(sm), "source": self.source}


def mps_structures(P, group="u1"):
    from paper_1203_2222_gb300 import synthetic
    m = {"u1": synthetic.u1_mps_heff, "z2f": synthetic.z2f_mps_heff, "su2u1": synthetic.su2u1_mps_heff}[group]()
    g = {"u1": P.U1, "z2f": P.Z2F, "su2u1": P.SU2U1}[group]
    S = {n: P.Structure(g, m[n]) for n in ("L", "A", "W", "R")}
    return m, S


def make_inputs(P, m, S, dtype, device):
    import torch
    from paper_1203_2222_gb300 import synthetic
    t = {}
    for n, s in S.items():
        v = torch.as_tensor(synthetic.normal(m["seeds"][n], s.numel)).to(dtype)
        t[n] = v.to(device)
    return t


def mps_step(P, S, data, G):
    """Y = ((L.A).W).R and d<G,Y>/d(L, A, W, R) through the public API."""
    import torch
    L = P.SymTensor(S["L"], data["L"])
    A = P.SymTensor(S["A"], data["A"])
    W = P.SymTensor(S["W"], data["W"])
    R = P.SymTensor(S["R"], data["R"])
    T1 = P.contract(L, A, [2], [0])
    T2 = P.contract(T1, W, [1, 2], [0, 2])
    Y = P.contract(T2, R, [1, 3], [2, 1])
    grads = torch.autograd.grad(Y.data, [data["L"], data["A"], data["W"], data["R"]], grad_outputs=G)
    return Y.data, grads


def step_flops(P, prec):
    """Useful flops of one step: forward GEMMs + backward GEMMs (dA and dB)."""
    tot = 0.0
    for p in P.cached_plans():
        if p.kind == "contract" and p.precision == prec:
            tot += 3.0 * p.stats()["flops_fwd"]
    return tot


def step_alg_bytes(P, prec):
    """Algorithmic bytes of one step: per contraction, A and B read and C written
    in the forward; dC, A and B read and dA, dB written in the backward."""
    tot = 0.0
    for p in P.cached_plans():
        if p.kind == "contract" and p.precision == prec:
            st = p.stats()
            tot += 3.0 * (st["bytes_a"] + st["bytes_b"]) + 2.0 * st["bytes_c"]
    return tot


class MPSWorkload:
    """U(1) MPS effective-Hamiltonian apply ((L.A).W).R, fwd + bwd."""
    name = "u1_mps_heff"
    describe = WORKLOAD
    default_steps, default_warmup, default_fp64_steps = 100, 5, 10
    group = "u1"

    def build(self, P, dev):
        import torch
        from paper_1203_2222_gb300 import synthetic
        self.m, self.S = mps_structures(P, self.group)
        self.data = make_inputs(P, self.m, self.S, torch.float32, dev)
        for v in self.data.values():
            v.requires_grad_(True)
        d = self.data
        Yt = P.contract(P.contract(P.contract(P.SymTensor(self.S["L"], d["L"]), P.SymTensor(self.S["A"], d["A"]),
                                              [2], [0]), P.SymTensor(self.S["W"], d["W"]), [1, 2], [0, 2]),
                        P.SymTensor(self.S["R"], d["R"]), [1, 3], [2, 1])
        self.G = torch.as_tensor(synthetic.normal(4242, Yt.structure.numel)).to(torch.float32).to(dev)

    def step(self, P, data, G):
        return mps_step(P, self.S, data, G)


class Z2FMPSWorkload(MPSWorkload):
    """The MPS chain with fermion-parity legs (swap signs on every gather):
    two large sectors per leg, so the GEMMs run at tensor-core size."""
    name = "z2f_mps_heff"
    describe = ("z2f_mps_heff: fermionic ((L.A).W).R fwd+bwd, fermion-parity legs: D=2048 as {0:1024, 1:1024}, "
                "phys {0:1, 1:1}, MPO {0:3, 1:2}; swap signs on every permutation")
    default_steps, default_warmup, default_fp64_steps = 50, 5, 2
    group = "z2f"


class SU2U1MPSWorkload(MPSWorkload):
    """The MPS chain with SU(2) x U(1) legs: every gather recouples the spins
    (6j coefficients) while the charges select the blocks."""
    name = "su2u1_mps_heff"
    describe = ("su2u1_mps_heff: ((L.A).W).R fwd+bwd with SU(2) x U(1) legs (labels (q, 2j)): Hubbard-like site "
                "{(0,0), (1,1), (2,0)}, MPO {(-1,1):2, (0,0):3, (1,1):2}, 1023 bond multiplets (dense 2459) over "
                "q = -8..8, 2j = 0..4")
    default_steps, default_warmup, default_fp64_steps = 50, 5, 2
    group = "su2u1"


class SU2Workload:
    """SU(2) recoupling contraction, fwd + bwd: rank-4 tensors, 2j = 0..8,
    degeneracies 1..32; A's legs 1, 3 contracted with B's dual legs 0, 1
    (A recoupled from the comb into the matrix tree by 6j coefficients)."""
    name = "su2_recouple"
    describe = ("su2_recouple: rank-4 SU(2), legs 2j=0..8 with degeneracies U{1..32} (seeded), "
                "A comb tree recoupled (6j) to the matrix tree, contract A(1,3) with B(0,1); fwd+bwd")
    # 20 timed steps of ~86 ms: a timed region long enough for the clock
    # sampler; one FP64 comparator step (~30 s on the CUDA cores' FP64 units)
    default_steps, default_warmup, default_fp64_steps = 20, 5, 1

    dmax = 32

    def build(self, P, dev):
        import torch
        from paper_1203_2222_gb300 import synthetic
        self.c = synthetic.su2_recouple(dmax=self.dmax, jmax2=8)
        self.S = {"A": P.Structure(P.SU2, self.c["A"]), "B": P.Structure(P.SU2, self.c["B"])}
        gen = torch.Generator(device=dev)
        gen.manual_seed(1236)
        self.data = {n: torch.randn(self.S[n].numel, device=dev, generator=gen).requires_grad_(True)
                     for n in ("A", "B")}
        C = P.contract(P.SymTensor(self.S["A"], self.data["A"]), P.SymTensor(self.S["B"], self.data["B"]),
                       self.c["pairsA"], self.c["pairsB"])
        self.G = torch.randn(C.structure.numel, device=dev, generator=gen)

    def step(self, P, data, G, on_forward=None):
        """C and the gradients; on_forward(C) is called between the forward
        and the backward (the end-to-end pass starts C's copy to the host
        there, so that it overlaps the backward)."""
        import torch
        C = P.contract(P.SymTensor(self.S["A"], data["A"]), P.SymTensor(self.S["B"], data["B"]),
                       self.c["pairsA"], self.c["pairsB"])
        if on_forward is not None:
            on_forward(C.data)
        grads = torch.autograd.grad(C.data, [data["A"], data["B"]], grad_outputs=G)
        return C.data, grads


BATCH_STREAMS = {"L": 1, "theta": 2, "W": 3, "R": 4}  # random sub-stream of each tensor role


class BatchWorkload:
    """512 independent two-site effective-Hamiltonian applies, fwd + bwd, as
    one batch plan per contraction of the chain (one launch per kernel and
    phase for all problems)."""
    name = "u1_two_site_batch"
    describe = ("u1_two_site_batch: 512 independent U(1) two-site H_eff applies (((L.theta).W1).W2).R fwd+bwd, "
                "D_i log-uniform in 64..1024 over q=-12..12 (Gaussian profile, sigma_i U(2,6)), seeded per problem; "
                "one batch plan per contraction")
    default_steps, default_warmup, default_fp64_steps = 50, 5, 3
    names = ("L", "theta", "W", "R")
    n = 512

    def build(self, P, dev):
        import torch
        from paper_1203_2222_gb300 import synthetic
        self.spec = synthetic.u1_two_site_batch(n=self.n)
        pr = self.spec["problems"]
        self.S = {n: [P.Structure(P.U1, p[n]) for p in pr] for n in self.names}
        plans = self.plans(P, P.BF16X3)
        self.offs = {"L": plans[0].off_a, "theta": plans[0].off_b, "W": plans[1].off_b, "R": plans[3].off_b}
        self.data = {}
        for n in self.names:
            parts = [synthetic.normal(p["seed"], self.offs[n][i + 1] - self.offs[n][i], stream=BATCH_STREAMS[n])
                     for i, p in enumerate(pr)]
            self.data[n] = torch.as_tensor(np.concatenate(parts)).to(torch.float32).to(dev).requires_grad_(True)
        self.G = torch.as_tensor(synthetic.normal(4243, plans[3].off_c[-1])).to(torch.float32).to(dev)

    def plans(self, P, prec):
        out, cur = [], self.S["L"]
        for an, bn, pa, pb in self.spec["steps"]:
            bp = P.contract_batch_plan(cur if an is None else self.S[an], self.S[bn], pa, pb, prec)
            out.append(bp)
            cur = bp.outs
        return out

    def step(self, P, data, G):
        import torch
        pl = self.plans(P, P.FP64 if data["L"].dtype == torch.float64 else P.BF16X3)
        t1 = P.contract_batch(pl[0], data["L"], data["theta"])
        t2 = P.contract_batch(pl[1], t1, data["W"])
        t3 = P.contract_batch(pl[2], t2, data["W"])
        y = P.contract_batch(pl[3], t3, data["R"])
        grads = torch.autograd.grad(y, [data[n] for n in self.names], grad_outputs=G)
        return y, grads


class MeraWorkload:
    """Energy E = <psi|h|psi>/<psi|psi> of a ternary-MERA patch (U(1), chi = 48)
    and its gradient with respect to the disentangler u and the isometry w,
    the environment checkpointed (recomputed in the backward pass)."""
    name = "u1_mera_grad"
    describe = ("u1_mera_grad: E of psi=(1x1xux1x1)(wxw)t, chi=48 over q=-4..4 (deg 5, +1 on q=-1,0,1), "
                "XXZ-like h on the bond under u, gradient w.r.t. u and w (environment checkpointed)")
    default_steps, default_warmup, default_fp64_steps = 50, 5, 5

    def build(self, P, dev):
        import torch
        from paper_1203_2222_gb300 import networks, synthetic
        self.spec = synthetic.u1_mera()
        self.S = networks.mera_structures(self.spec)
        h, one = networks.mera_h_and_identity(self.S, self.spec)
        scale = 1.0 / np.sqrt(self.spec["chi"])
        self.const = {}
        for n in ("t",):
            self.const[n] = torch.as_tensor(synthetic.normal(self.spec["seeds"][n], self.S[n].numel) * scale)
        self.const["h"], self.const["1"] = torch.as_tensor(h), torch.as_tensor(one)
        self.dev = dev
        self.data = {n: torch.as_tensor(synthetic.normal(self.spec["seeds"][n], self.S[n].numel) * scale)
                     .to(torch.float32).to(dev).requires_grad_(True) for n in ("w", "u")}
        self.G = torch.ones((), device=dev)
        self.step(P, self.data, self.G)  # plans

    def _const(self, dtype):
        cache = self.__dict__.setdefault("_by_dtype", {})
        if dtype not in cache:
            cache[dtype] = {n: v.to(dtype).to(self.dev) for n, v in self.const.items()}
        return cache[dtype]

    def step(self, P, data, G):
        import torch
        from paper_1203_2222_gb300 import networks
        c = self._const(data["w"].dtype)
        E = networks.mera_energy(self.S, c["t"], data["w"], data["u"], c["h"], c["1"], checkpoint=True)
        grads = torch.autograd.grad(E, [data["w"], data["u"]], grad_outputs=G.to(E.dtype))
        return E.reshape(1), grads

    def contractions(self, P, prec):
        """(plan, gradient w.r.t. A computed, w.r.t. B computed) of every contraction of the step."""
        S = self.S
        cp = lambda a, b, pa, pb: P.contract_plan(a, b, pa, pb, prec)
        top = cp(S["t"], S["t*"], [], [])
        w1 = cp(S["w"], S["w*"], [1, 2], [1, 2])
        w2 = cp(S["w"], S["w*"], [2, 3], [2, 3])
        x = cp(top.out, w1.out, [0, 2], [0, 2])
        rho = cp(x.out, w2.out, [0, 1], [0, 2])
        y = cp(S["u"], rho.out, [2, 3], [0, 2])
        rp = cp(y.out, S["u*"], [2, 3], [2, 3])
        num = cp(rp.out, S["h*"], [0, 1, 2, 3], [0, 1, 2, 3])
        den = cp(rp.out, S["1*"], [0, 1, 2, 3], [0, 1, 2, 3])
        # the environment is checkpointed: its forward contractions run twice
        env = [(top, False, False), (w1, True, True), (w2, True, True), (x, False, True), (rho, True, True)]
        rest = [(y, True, True), (rp, True, True), (num, True, False), (den, True, False)]
        return env + [(p, False, False) for p, _, _ in env] + rest

    def flops_and_bytes(self, P, prec):
        """Useful flops and algorithmic bytes of one step: each contraction's
        forward, plus one GEMM and its operands per gradient it computes."""
        fl = by = 0.0
        for p, ga, gb in self.contractions(P, prec):
            st = p.stats()
            a, b, c = st["bytes_a"], st["bytes_b"], st["bytes_c"]
            fl += st["flops_fwd"] * (1 + ga + gb)
            by += a + b + c + (c + b + a if ga else 0) + (c + a + b if gb else 0)
        return fl, by


WORKLOADS = {"u1_mps_heff": MPSWorkload, "su2_recouple": SU2Workload, "u1_two_site_batch": BatchWorkload,
             "u1_mera_grad": MeraWorkload, "z2f_mps_heff": Z2FMPSWorkload, "su2u1_mps_heff": SU2U1MPSWorkload}  # u1_two_site_svd: SVDWorkload below


# ---------------------------------------------------------------- roofline ---

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch of
# the dominant kernels of each workload, from one ncu pass (profiles/), with
# the SHA-256 of the kernel's sources at that time: once a source changes, the
# figure no longer applies and the bench reports null.  "ratio" entries come
# from a smaller case of the same workload: DRAM bytes / algorithmic bytes of
# the captured launches, applied to the full launch's algorithmic bytes.
TRAFFIC = {
    "u1_mps_heff": {  # profiles/traffic_u1_mps_heff.md
        "gemm_tc": {"bytes_per_launch": 13768640, "sha": "e8b8ba59c26dc3b8"},
        "box_flat": {"bytes_per_launch": 5856928, "sha": "b2745455cd736886"},
        "box": {"bytes_per_launch": 13080064, "sha": "b2745455cd736886"},
        "direct": {"bytes_per_launch": 11909291, "sha": "a481e530fd08e2e9"},
    },
    "su2_recouple": {  # profiles/gemm_tc_su2_recouple.md (full size, forward and backward launches)
        "gemm_tc": {"bytes_per_launch": 61145753344, "sha": "e8b8ba59c26dc3b8"},
    },
    "u1_two_site_batch": {  # profiles/direct_u1_two_site_batch.md (128 of the 512 problems)
        "direct": {"ratio": 0.96, "sha": "a481e530fd08e2e9"},
    },
    "u1_two_site_svd": {  # profiles/svd_u1_two_site_svd.md (full size, mean of 11 launches)
        "svd_jacobi": {"bytes_per_launch": 9013271, "sha": "96f8106d63b42dfd"},
    },
    "u1_two_site_eig": {  # profiles/eig_u1_two_site_eig.md (full size, mean of 11 launches)
        "svd_jacobi": {"bytes_per_launch": 8889972, "sha": "96f8106d63b42dfd"},
    },
    "z2f_mps_heff": {  # profiles/traffic_z2f_mps_heff_and_mera.md (full size, mean of 62 step launches)
        "gemm_tc": {"bytes_per_launch": 196322104, "sha": "e8b8ba59c26dc3b8"},
    },
    "u1_mera_grad": {  # profiles/traffic_z2f_mps_heff_and_mera.md (full size, mean of 663 launches)
        "box_flat": {"bytes_per_launch": 2139167, "sha": "b2745455cd736886"},
    },
}
KERNEL_SOURCES = {
    "box": ["box.cu", "kernels.h", "pdl.h"], "box_flat": ["box.cu", "kernels.h", "pdl.h"],
    "gemm_tc": ["gemm_tc.cu", "kernels.h", "pdl.h"],
    "gemm_tile": ["gemm_simt.cu", "kernels.h", "pdl.h"], "gemm_wide": ["gemm_simt.cu", "kernels.h", "pdl.h"],
    "gemm_thin": ["gemm_simt.cu", "kernels.h", "pdl.h"], "gemm_rows": ["gemm_simt.cu", "kernels.h", "pdl.h"],
    "direct": ["direct.cu", "kernels.h", "pdl.h"],
    "svd_jacobi": ["svd.cu"],
}


def kernel_source_sha(kern):
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kern]:
        with open(os.path.join(ROOT, "paper_1203_2222_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def roofline(prof, clk, sustained=False, workload="u1_mps_heff", full_size=True):
    """Roofline of the kernel with the largest summed device time.

    box kernels, the direct kernel and the rows / thin GEMMs: HBM-bound,
    algorithmic bytes (block data read once + written once) per launch / mean
    launch time vs the measured copy bandwidth;
    tcgen05: useful flops vs the measured bf16 peak / 3 (three BF16 passes);
    CUDA-core GEMMs: FP32 FMA peak from the unit count and the sampled clock.
    """
    if not prof:
        return None
    peaks, peak_src = load_peaks()
    dom = max(prof, key=lambda k: prof[k]["ms"])
    d = prof[dom]
    n = max(d["launches"], 1)
    sec = d["ms"] * 1e-3 / n  # mean launch duration
    if dom.startswith("box") or dom in ("direct", "gemm_rows", "gemm_thin"):
        # streaming kernels: block movement, the direct contraction of tiny
        # sectors, and the GEMMs with a side of at most 16 (A, B, C once)
        bound, unit, per = "hbm", "GB/s", d["bytes"] / n
        achieved, peak = per / sec / 1e9, peaks["hbm_gbs"]
        src = f"{peak_src} hbm_gbs"
    elif dom == "gemm_tc":
        bound, unit, per = "tensor", "TFLOP/s", d["flops"] / n
        key = "bf16_tflops_sustained" if sustained else "bf16_tflops"
        achieved, peak = per / sec / 1e12, peaks[key] / 3.0
        src = f"{peak_src} {key} ({'sustained: long step' if sustained else 'burst: short step'}) / 3 passes"
    else:
        mhz = clk.get("sm_mhz") or 2070.0
        bound, unit, per = "alu", "TFLOP/s", d["flops"] / n
        achieved, peak = per / sec / 1e12, 152 * 128 * 2 * mhz * 1e6 / 1e12
        src = "152 SMs x 128 FP32 FMA/clk x 2 flops x sampled SM clock"
    t = TRAFFIC.get(workload, {}).get(dom) if full_size else None  # the figures are the full-size launches
    traffic = None
    if t and t["sha"] == kernel_source_sha(dom):
        traffic = t["bytes_per_launch"] if "bytes_per_launch" in t else round(t["ratio"] * d["bytes"] / n)
    return {"bound": bound, "kernel": dom, "symbol": __import__("paper_1203_2222_gb300").KERNEL_SYMBOLS[dom],
            "achieved": round(achieved, 4), "peak": round(peak, 1), "unit": unit, "frac": round(achieved / peak, 4),
            "traffic": traffic, "algorithmic_per_launch": per, "launches_timed": d["launches"],
            "avg_launch_us": round(sec * 1e6, 2), "peak_source": src}


# -------------------------------------------------------------- our path ---

def run_ours(args, rank, world):
    import torch
    import paper_1203_2222_gb300 as P

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    wl = WORKLOADS[args.workload]()
    if args.workload == "su2_recouple":
        wl.dmax = args.su2_dmax
    if args.workload == "u1_two_site_batch":
        wl.n = args.batch_n

    # ---- planning parameters (autotuned table entry, search, or defaults)
    from paper_1203_2222_gb300 import autotune
    table = args.tune_table or autotune.TABLE
    tuning = {"source": "library defaults", "params": P.tune_get()}
    if args.tune == "table":
        params = autotune.load(args.workload, table)
        if params:
            tuning = {"source": "autotuned table", "params": P.tune_set(**params)}

    # ---- split-BF16 x3 path (the value); the first contraction builds the plans
    wl.build(P, dev)
    data, G = wl.data, wl.G

    def run_once(dt, Gt):
        return wl.step(P, dt, Gt)

    if args.tune == "search":
        t0 = time.time()
        space = autotune.SPACE if not args.tune_space else {k: autotune.SPACE[k] for k in args.tune_space.split(",")}
        known = autotune.load(args.workload, table)  # the search starts from the better of defaults and this
        # a candidate must keep the step within the split-BF16 bar of the FP64 path
        ref64 = wl.step(P, {n: v.detach().double().requires_grad_(True) for n, v in data.items()}, G.double())
        ref64 = [ref64[0].detach()] + [g.detach() for g in ref64[1]]

        def accurate():
            y, gs = run_once(data, G)
            outs = [y.detach()] + [g.detach() for g in gs]
            return max(float((a.double() - b).norm() / b.norm()) for a, b in zip(outs, ref64)) <= SPLIT_BF16_TOL

        params, ms_t, hist = autotune.tune(lambda: run_once(data, G), space=space, graph=not args.no_graph,
                                           starts=list(autotune.PRESETS) + ([known] if known else []),
                                           log=lambda m: print("# " + m, file=sys.stderr, flush=True),
                                           check=accurate)
        del ref64
        autotune.save(args.workload, params, ms_t, hist[0]["ms"], len(hist), path=table)
        tuning = {"source": "autotuner search", "params": params, "evaluations": len(hist),
                  "ms_per_step_defaults": hist[0]["ms"], "ms_per_step_tuned": round(ms_t, 5),
                  "search_s": round(time.time() - t0, 1), "table": os.path.relpath(table, ROOT)}
        run_once(data, G)  # plans under the installed parameters (the search's last change dropped the old ones)
        torch.cuda.synchronize()

    if hasattr(wl, "flops_and_bytes"):
        flops, alg_bytes = wl.flops_and_bytes(P, P.BF16X3)
    else:
        flops = step_flops(P, P.BF16X3)
        alg_bytes = step_alg_bytes(P, P.BF16X3)

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    use_graph = not args.no_graph
    graph = graph_prof = None
    static_out = None
    for _ in range(max(args.warmup, 1)):
        run_once(data, G)
    torch.cuda.synchronize()
    plans = P.cached_plans()
    # The library records a CUDA event pair around each of its own launches
    # (on the launch stream).  Captured into the graph, every replay re-records
    # them with the kernels' own device times.  While profiling, a phase's
    # GEMM kinds run one after another instead of concurrently, so that every
    # pair brackets one kernel alone (the timed graph keeps them concurrent).
    if use_graph:
        try:
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(s):
                for _ in range(2):
                    run_once(data, G)
            torch.cuda.current_stream().wait_stream(s)
            torch.cuda.synchronize()
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph):
                static_out = run_once(data, G)
            # a second graph of the same step with the library's event pairs
            # captured around every launch, for the per-kernel timing pass
            for p in plans:
                p.profile(True)
            graph_prof = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph_prof):
                run_once(data, G)
            for p in plans:
                p.profile(False)  # keep the captured events, record no more
            torch.cuda.synchronize()
            for _ in range(2):
                graph.replay()
                graph_prof.replay()
            torch.cuda.synchronize()
        except Exception as e:  # capture unsupported: fall back to eager launches
            print(f"# graph capture failed ({e}); timing eager launches", file=sys.stderr)
            graph = None
    if graph is None:
        for p in plans:
            p.profile(True)
        run_once(data, G)
        torch.cuda.synchronize()
    launches_per_step = sum(p.profile_read(ph)["launches"] for p in plans for ph in P.PHASES.values())
    if graph is None:
        for p in plans:
            p.profile(False)  # eager: the timed region runs without event records

    def one_step():
        if graph is not None:
            graph.replay()
        else:
            run_once(data, G)

    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev)
    clocks.start()
    evs = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        one_step()
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in evs)

    prof = {}

    def accumulate():
        for p in plans:
            for kern, kid in P.KERNELS.items():
                r = p.profile_kernel(kid)
                if r["launches"] == 0:
                    continue
                d = prof.setdefault(kern, {"launches": 0, "ms": 0.0, "bytes": 0.0, "flops": 0.0})
                for k in d:
                    d[k] += r[k]

    if graph is not None:
        # per-kernel device times: K replays of the instrumented graph, each
        # read back from the event pairs captured around every library launch
        for _ in range(args.steps):
            flush.fill_(1.0)
            graph_prof.replay()
            torch.cuda.synchronize()
            accumulate()
    else:
        # per-kernel device times: K more eager steps with the event pairs on
        for p in plans:
            p.profile(True)
        for _ in range(args.steps):
            flush.fill_(1.0)
            run_once(data, G)
        torch.cuda.synchronize()
        accumulate()
        for p in plans:
            p.profile(False)
    ms = max_over_ranks(ms, world, dev)
    ms_per_step = ms / args.steps
    value = whole_job_rate(flops, args.steps, world, ms) / 1e12

    # ---- accuracy against the FP64 path, and the FP64 GPU comparator
    launch_mode = "cuda graph replay" if graph is not None else "eager"
    y32, g32 = (static_out if graph is not None else run_once(data, G))
    y32, g32 = y32.detach().clone(), [g.detach().clone() for g in g32]
    torch.cuda.synchronize()
    # the graphs' memory pools are not needed any more (the FP64 comparator
    # and the end-to-end pass launch eagerly)
    del graph, graph_prof, static_out
    torch.cuda.empty_cache()
    data64 = {n: v.detach().double().requires_grad_(True) for n, v in data.items()}
    G64 = G.double()
    y64, g64 = wl.step(P, data64, G64)  # builds the FP64 plans
    torch.cuda.synchronize()

    def rel(a, b):
        return float((a.double() - b.detach()).norm() / b.detach().norm())

    err = max([rel(y32, y64)] + [rel(a, b) for a, b in zip(g32, g64)])
    del y64, g64
    # inputs and results on the host for the oracle's sampled check (rank 0)
    check = None
    if args.workload == "su2_recouple" and args.su2_dmax == 32 and rank == 0 and not args.no_cpu_baseline:
        check = {"A": data["A"].detach().cpu().numpy(), "B": data["B"].detach().cpu().numpy(),
                 "G": G.detach().cpu().numpy(), "C": y32.cpu().numpy(),
                 "dA": g32[0].cpu().numpy(), "dB": g32[1].cpu().numpy()}
    e64 = []
    for _ in range(args.fp64_steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out64 = wl.step(P, data64, G64)
        e1.record(stream)
        del out64
        e64.append((e0, e1))
    torch.cuda.synchronize()
    ms64 = sum(a.elapsed_time(b) for a, b in e64) / args.fp64_steps if e64 else None
    value64 = flops * world / (ms64 * 1e-3) / 1e12 if e64 else None
    del data64, G64

    # ---- end to end through the public API: pinned host inputs -> results on
    # the host.  Two slots (device input buffers, a CUDA graph of the step
    # captured on them, host result buffers) take turns, so that step i+1's
    # inputs go to the device and step i's results to the host on copy
    # streams while the next step computes; the host waits for every step's
    # results, one step behind.
    names = list(data.keys())
    host_in = {n: v.detach().cpu().pin_memory() for n, v in data.items()}
    h2d = sum(v.numel() * 4 for v in host_in.values())
    d2h = y32.numel() * 4 + sum(v.numel() * 4 for v in host_in.values())
    # workloads whose step exposes its forward result copy it to the host on
    # a side stream, forked inside the graph, while the backward runs
    overlap_y = "on_forward" in inspect.signature(wl.step).parameters
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()

    class Slot:
        pass

    def make_slot():
        sl = Slot()
        sl.dev_in = {n: torch.empty_like(v.detach()).requires_grad_(True) for n, v in data.items()}
        sl.host_y = torch.empty(y32.numel(), dtype=torch.float32).pin_memory()
        sl.host_g = {n: torch.empty(v.numel(), dtype=torch.float32).pin_memory() for n, v in data.items()}
        sl.s_copy = torch.cuda.Stream() if overlap_y else None
        sl.graph, sl.out = None, None
        sl.ev_in, sl.ev_done, sl.ev_out = torch.cuda.Event(), torch.cuda.Event(), torch.cuda.Event()
        for n in names:
            sl.dev_in[n].detach().copy_(data[n].detach())

        def copy_y(y):
            sl.s_copy.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(sl.s_copy):
                sl.host_y.copy_(y.detach(), non_blocking=True)

        sl.copy_y = copy_y
        if use_graph:
            try:
                s2 = torch.cuda.Stream()
                s2.wait_stream(torch.cuda.current_stream())
                with torch.cuda.stream(s2):
                    for _ in range(2):
                        wl.step(P, sl.dev_in, G)
                torch.cuda.current_stream().wait_stream(s2)
                torch.cuda.synchronize()
                sl.graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(sl.graph):
                    if overlap_y:
                        sl.out = wl.step(P, sl.dev_in, G, on_forward=copy_y)
                        torch.cuda.current_stream().wait_stream(sl.s_copy)  # join the copy inside the graph
                    else:
                        sl.out = wl.step(P, sl.dev_in, G)
            except Exception as e:
                print(f"# e2e graph capture failed ({e}); eager launches", file=sys.stderr)
                sl.graph = None
        sl.ev_done.record(stream)
        return sl

    slots = [make_slot(), make_slot()]
    e2e_launch = ("cuda graph replay" if all(sl.graph is not None for sl in slots) else "eager") + \
        ", two slots: the next step's inputs to the device and this step's results to the host on copy streams " \
        "during the following step" + (", the forward result during the backward" if overlap_y else "")

    def issue_in(sl):  # after the slot's previous step has finished with its inputs
        s_in.wait_event(sl.ev_done)
        with torch.cuda.stream(s_in), torch.no_grad():
            for n in names:
                sl.dev_in[n].copy_(host_in[n], non_blocking=True)
        sl.ev_in.record(s_in)

    def run(sl):
        stream.wait_event(sl.ev_in)
        flush.fill_(1.0)
        if sl.graph is not None:
            sl.graph.replay()  # with overlap_y the graph itself copies the result to host_y
            yy, gg = sl.out
        else:
            yy, gg = (wl.step(P, sl.dev_in, G, on_forward=sl.copy_y) if overlap_y else wl.step(P, sl.dev_in, G))
            if overlap_y:
                stream.wait_stream(sl.s_copy)
        sl.ev_done.record(stream)
        s_out.wait_event(sl.ev_done)
        with torch.cuda.stream(s_out):
            if not overlap_y:
                sl.host_y.copy_(yy.detach(), non_blocking=True)
            for n, gv in zip(names, gg):
                sl.host_g[n].copy_(gv, non_blocking=True)
        sl.ev_out.record(s_out)

    def e2e_run(k):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s_in.wait_event(e0)
        issue_in(slots[0])
        for i in range(k):
            run(slots[i % 2])
            if i + 1 < k:
                issue_in(slots[(i + 1) % 2])
            if i >= 1:
                slots[(i - 1) % 2].ev_out.synchronize()  # the host takes step i-1's results
        stream.wait_event(slots[(k - 1) % 2].ev_out)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1)

    e2e_run(2)
    torch.cuda.synchronize()
    ms_e2e = e2e_run(args.steps) / args.steps
    e2e_value = flops * world / (ms_e2e * 1e-3) / 1e12
    del slots

    # ---- roofline of the dominant kernel (largest summed device time), and of
    # the whole step: T_roof = max(useful flops / tensor peak, algorithmic
    # bytes / HBM bandwidth) against the measured step time
    long_step = ms_per_step > 20.0  # seconds-long timed region: the power cap applies
    full_size = not ((args.workload == "su2_recouple" and args.su2_dmax != 32) or
                     (args.workload == "u1_two_site_batch" and args.batch_n != 512))
    roof = roofline(prof, clk, sustained=long_step, workload=args.workload, full_size=full_size)
    peaks, peak_src = load_peaks()
    p_tensor = (peaks["bf16_tflops_sustained"] if long_step else peaks["bf16_tflops"]) / 3.0
    t_flop = flops / (p_tensor * 1e12)
    t_byte = alg_bytes / (peaks["hbm_gbs"] * 1e9)
    t_roof = max(t_flop, t_byte)
    step_roof = {"t_roof_ms": round(t_roof * 1e3, 5), "t_meas_ms": round(ms_per_step, 5),
                 "frac": round(t_roof / (ms_per_step * 1e-3), 4),
                 "bound": "tensor" if t_flop >= t_byte else "hbm",
                 "useful_flops": flops, "alg_bytes": alg_bytes,
                 "tensor_peak_tflops": round(p_tensor, 1), "hbm_gbs": peaks["hbm_gbs"],
                 "peak_source": f"{peak_src} {'bf16_tflops_sustained' if long_step else 'bf16_tflops'} / 3, hbm_gbs"}
    kernels = {k: {"symbol": P.KERNEL_SYMBOLS[k], "launches": v["launches"], "ms": round(v["ms"], 4),
                   "share": round(v["ms"] / max(sum(x["ms"] for x in prof.values()), 1e-12), 4)}
               for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])}

    out = {
        "metric": METRIC, "value": round(value, 4), "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16x3-f32acc", "data": "synthetic",
        "config": bench_config(wl.describe + (f" [dmax {args.su2_dmax}]" if args.workload == "su2_recouple" and
                                              args.su2_dmax != 32 else "")
                               + (f" [{args.batch_n} problems]" if args.workload == "u1_two_site_batch" and
                                  args.batch_n != 512 else "")),
        "precision": "split-BF16 x3 on tcgen05, FP32 accumulate, fp32 blocks",
        "useful_gflop_per_step": round(flops / 1e9, 4),
        "launch": launch_mode,
        "parallelism": f"replicas x{world}",
        "roofline": roof, "step_roofline": step_roof, "kernels": kernels,
        "fp64_gpu": ({"value": round(value64, 5), "unit": "TFLOP/s", "ms_per_step": round(ms64, 4)}
                     if value64 else None),
        "speedup_vs_fp64_gpu": round(value / value64 / world, 3) if value64 else None,
        "max_rel_err_vs_fp64": err,
        "e2e": {"value": round(e2e_value, 4), "unit": "TFLOP/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": round(ms_e2e, 4), "launch": e2e_launch},
        "clocks": clk, "gpu_launches": launches_per_step * args.steps,
        "tuning": tuning,
    }
    return out, flops, check


# ------------------------------------------------------------- blockwise SVD ---

SVD_METRIC = "blockwise FP64 SVD + truncation of the two-site tensor, per second"
# FP64 peak: 1.25 TFLOP/s nominal over 152 SMs at the 2070 MHz maximum clock
# is 4 flops (2 FMAs) per SM per clock, scaled to the sampled clock
FP64_FLOPS_PER_SM_CLK = 4.0
FP32_FLOPS_PER_SM_CLK = 256.0  # 128 FP32 FMAs per SM per clock


class SVDWorkload:
    describe = ("u1_two_site_svd: theta[a, s1, s2, b] of the MPS chain (D = 2048 over q = -20..20, Gaussian profile "
                "sigma 6; phys {0:1, 1:1}; total charge 0) as the matrix (a, s1) x (s2, b): 41 diagonal blocks up "
                "to 272 x 272, FP64 blockwise SVD, truncated to chi = 2048 singular values, factors U and S V")
    default_steps = 20
    default_warmup = 3
    default_fp64_steps = 0


EIG_METRIC = "blockwise FP64 symmetric eigendecomposition + truncation of the two-site density matrix, per second"


class EigWorkload:
    describe = ("u1_two_site_eig: rho = theta theta* over (a, s1) of the two-site tensor of u1_two_site_svd (D = 2048 "
                "over q = -20..20, Gaussian profile sigma 6; phys {0:1, 1:1}), 42 diagonal blocks up to 272 x 272, "
                "FP64 blockwise eigendecomposition, truncated to chi = 2048 eigenvalues of largest magnitude, "
                "eigenvectors U and their transposes")
    default_steps = 20
    default_warmup = 3
    default_fp64_steps = 0


def _svd_inputs(P):
    from paper_1203_2222_gb300 import synthetic
    w = synthetic.u1_two_site_svd()
    S = P.Structure(P.U1, w["theta"])
    return w, S, synthetic.normal(w["seed"], S.numel)


def _eig_inputs(P, dev):
    """rho = theta theta* contracted by the library in FP64 (not timed)."""
    import torch
    from paper_1203_2222_gb300 import networks, synthetic
    w = synthetic.u1_two_site_eig()
    S = P.Structure(P.U1, w["theta"])
    Sc = P.Structure(P.U1, networks.reversed_legs(w["theta"]))
    th = torch.as_tensor(synthetic.normal(w["seed"], S.numel)).to(dev)
    with torch.no_grad():
        rho = P.contract(P.SymTensor(S, th), P.SymTensor(Sc, th), *w["pairs"])
    torch.cuda.synchronize()
    return w, rho.structure, rho.data.contiguous()


def run_svd(args, rank, world):
    """Blockwise FP64 SVD workload: one step = P.svd(theta, 2, chi) -- the
    Jacobi launch, the singular values to the host for the truncation, and
    the factor launch writing U and S V.  With u1_two_site_eig, one step =
    P.eig(rho, 2, chi) on the density matrix, through the same kernels."""
    import torch
    import paper_1203_2222_gb300 as P

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    is_eig = args.workload == "u1_two_site_eig"
    if is_eig:
        w, S, data = _eig_inputs(P, dev)
        vals = data.cpu()
        T = P.SymTensor(S, data)
    else:
        w, S, vals = _svd_inputs(P)
        T = P.SymTensor(S, torch.as_tensor(vals).to(dev))
    chi, nrow = w["chi"], w["nrow"]
    plan = P.eig_plan(S, nrow) if is_eig else P.svd_plan(S, nrow)
    absorb = 0 if is_eig else 2

    def step(t):
        return (P.eig if is_eig else P.svd)(t, nrow, chi=chi, absorb=absorb)

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 1)):
        step(T)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(dev)
    clocks.start()
    evs = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(T)
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in evs)
    ms = max_over_ranks(ms, world, dev)
    ms_per_step = ms / args.steps
    value = whole_job_rate(1.0, args.steps, world, ms)

    # per-kernel device times (the same launches, timed one by one)
    kms = {"svd_jacobi": 0.0, "svd_factor": 0.0}
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        plan.execute(T.data)
        e1.record(stream)
        plan.factors(absorb)
        e2.record(stream)
        torch.cuda.synchronize()
        kms["svd_jacobi"] += e0.elapsed_time(e1)
        kms["svd_factor"] += e1.elapsed_time(e2)
    f64, f32 = plan.flops()
    sweeps64, _ = plan.stats()
    sweeps32, _ = plan.stats(fp32=True)
    kernels = {k: {"symbol": k + "_kernel", "launches": args.steps, "ms": round(v, 4),
                   "share": round(v / max(sum(kms.values()), 1e-12), 4)} for k, v in kms.items()}
    jac_s = kms["svd_jacobi"] * 1e-3 / args.steps
    mhz = clk.get("sm_mhz") or 2070.0
    peak64 = 152 * FP64_FLOPS_PER_SM_CLK * mhz * 1e6 / 1e12
    peak32 = 152 * FP32_FLOPS_PER_SM_CLK * mhz * 1e6 / 1e12
    roof = {"bound": "alu", "kernel": "svd_jacobi", "symbol": "svd_jacobi_kernel",
            "achieved": round(f64 / jac_s / 1e12, 5), "peak": round(peak64, 4), "unit": "TFLOP/s",
            "frac": round(f64 / jac_s / 1e12 / peak64, 4), "traffic": svd_traffic(args.workload),
            "algorithmic_per_launch": f64, "fp32_flops_per_launch": f32,
            "avg_launch_us": round(jac_s * 1e6, 2), "launches_timed": args.steps,
            "peak_source": "FP64 ALU: 152 SMs x 4 flops/clk (1.25 TFLOP/s nominal at 2070 MHz) x sampled SM clock",
            "sweeps_fp64_max": max(sweeps64), "sweeps_fp32_max": max(sweeps32)}
    # the step's floor: FP64 flops at the FP64 peak plus FP32 flops at the FP32 peak
    t_roof = f64 / (peak64 * 1e12) + f32 / (peak32 * 1e12)
    step_roof = {"t_roof_ms": round(t_roof * 1e3, 4), "t_meas_ms": round(ms_per_step, 4),
                 "frac": round(t_roof / (ms_per_step * 1e-3), 4), "bound": "alu",
                 "fp64_flops": f64, "fp32_flops": f32}

    # end to end: pinned host input -> device, the factorization, U, the values
    # and the second factor back to the host
    host_in = torch.as_tensor(vals).pin_memory()
    dev_in = torch.empty_like(T.data)
    Us, Vs = plan.bond(plan.truncation(plan.execute(T.data).cpu().numpy(), chi))
    host_u = torch.empty(Us.numel, dtype=torch.float64).pin_memory()
    host_v = torch.empty(Vs.numel, dtype=torch.float64).pin_memory()
    host_s = torch.empty(chi, dtype=torch.float64).pin_memory()
    h2d, d2h = host_in.numel() * 8, (host_u.numel() + host_v.numel() + host_s.numel()) * 8

    def e2e_step():
        dev_in.copy_(host_in, non_blocking=True)
        U, Sk, V = step(P.SymTensor(S, dev_in))
        host_u.copy_(U.data, non_blocking=True)
        host_v.copy_(V.data, non_blocking=True)
        host_s[:Sk.numel()].copy_(Sk, non_blocking=True)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    ee = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        e2e_step()
        e1.record(stream)
        e1.synchronize()
        ee.append((e0, e1))
    ms_e2e = sum(a.elapsed_time(b) for a, b in ee) / args.steps
    P.device_status()

    unit = "eig/s" if is_eig else "SVD/s"
    out = {
        "metric": EIG_METRIC if is_eig else SVD_METRIC, "value": round(value, 4), "unit": unit, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(EigWorkload.describe if is_eig else SVDWorkload.describe),
        "precision": "FP64 result: FP32 Jacobi sweeps seed FP64 Newton-Schulz + FP64 Jacobi sweeps"
                     + (" on the block's symmetric part shifted by its Frobenius norm" if is_eig else ""),
        "blocks": plan.nblocks, "singular_values": plan.nsv, "chi": chi,
        "launch": "eager (host truncation)",
        "parallelism": f"replicas x{world}",
        "roofline": roof, "step_roofline": step_roof, "kernels": kernels,
        "e2e": {"value": round(1e3 / ms_e2e * world, 4), "unit": unit, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": round(ms_e2e, 4)},
        "clocks": clk, "gpu_launches": 2 * args.steps,
    }
    vals_gpu = plan.execute(T.data).cpu().numpy()  # every block's values, for the oracle's comparison
    torch.cuda.synchronize()
    return out, (plan.labels, plan.m if is_eig else [min(a, b) for a, b in zip(plan.m, plan.n)], vals_gpu)


def svd_traffic(workload="u1_two_site_svd"):
    t = TRAFFIC[workload]["svd_jacobi"]
    return t["bytes_per_launch"] if t["sha"] == kernel_source_sha("svd_jacobi") else None


def _oracle_svd_step(w, To):
    from oracle import svd as osvd
    fac, _ = osvd.svd("u1", To, w["nrow"])
    keep = osvd.truncation({x: f[1] for x, f in fac.items()}, w["chi"])
    osvd.factors("u1", To, w["nrow"], keep, absorb=2, fac=fac)
    return fac


def _oracle_svd_inputs():
    from oracle import u1
    from paper_1203_2222_gb300 import synthetic
    w = synthetic.u1_two_site_svd()
    legs = [u1.Leg(*l) for l in w["theta"]]
    n = u1.layout(legs, 0)[2]
    return w, (legs, 0, synthetic.normal(w["seed"], n))


def _values_error(check, fac):
    """Largest difference of the GPU's values from the oracle's, block by
    block (each sorted), relative to the largest magnitude."""
    labels, sizes, vals = check
    off, worst, vmax = 0, 0.0, 0.0
    for x, k in zip(labels, sizes):
        ref = np.sort(fac[x][1])
        got = np.sort(vals[off:off + k])
        off += k
        worst = max(worst, float(np.max(np.abs(got - ref))))
        vmax = max(vmax, float(np.max(np.abs(ref))))
    return {"value": worst / vmax, "sample": "every value of every block, relative to the largest |value|"}


def cpu_baseline_svd(steps, check=None):
    w, To = _oracle_svd_inputs()
    n = max(steps, 1) * 3
    t0 = time.perf_counter()
    for _ in range(n):
        fac = _oracle_svd_step(w, To)
    dt = time.perf_counter() - t0
    base = {"value": round(n / dt, 4), "unit": "SVD/s", "cores": cpu_cores(), "kind": "oracle",
            "sample": f"{n} full steps of the same workload (numpy SVD of every block, truncation, factors), "
                      f"{dt:.1f} s"}
    return base, (_values_error(check, fac) if check else None)


def _oracle_eig_inputs():
    """rho = theta theta* by the oracle's dense contraction of the same theta."""
    from oracle import contract as oc
    from oracle import u1
    from paper_1203_2222_gb300 import synthetic
    w = synthetic.u1_two_site_eig()
    legs = [u1.Leg(*l) for l in w["theta"]]
    legs_c = [u1.Leg(l.labels, l.degens, -l.dir) for l in legs]
    th = synthetic.normal(w["seed"], u1.layout(legs, 0)[2])
    lr, qr, rho, _ = oc.contract("u1", (legs, 0, th), (legs_c, 0, th), *w["pairs"])
    return w, (lr, qr, rho)


def _oracle_eig_step(w, To):
    from oracle import eig as oeig
    fac, _ = oeig.eig("u1", To, w["nrow"])
    keep = oeig.truncation({x: f[1] for x, f in fac.items()}, w["chi"])
    oeig.factors("u1", To, w["nrow"], keep, absorb=0, fac=fac)
    return fac


def cpu_baseline_eig(steps, check=None):
    w, To = _oracle_eig_inputs()
    n = max(steps, 1) * 3
    t0 = time.perf_counter()
    for _ in range(n):
        fac = _oracle_eig_step(w, To)
    dt = time.perf_counter() - t0
    base = {"value": round(n / dt, 4), "unit": "eig/s", "cores": cpu_cores(), "kind": "oracle",
            "sample": f"{n} full steps of the same workload (numpy eigh of every block, truncation, factors; rho "
                      f"formed once by the oracle's dense contraction, untimed), {dt:.1f} s"}
    return base, (_values_error(check, fac) if check else None)


def run_reference_eig(args):
    """Oracle reference arm for u1_two_site_eig: each step is the oracle's blockwise
    eigendecomposition, truncation and factors of the same density matrix."""
    w, To = _oracle_eig_inputs()
    for _ in range(args.warmup):
        _oracle_eig_step(w, To)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _oracle_eig_step(w, To)
    dt = time.perf_counter() - t0
    value = args.steps / dt
    sample = "step = the oracle's blockwise eigendecomposition (numpy eigh, FP64) + truncation + factors of rho"
    return {
        "metric": EIG_METRIC, "value": round(value, 4), "unit": "eig/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(dt * 1e3 / args.steps, 2), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": bench_config(EigWorkload.describe), "sample": sample,
        "cpu_baseline": {"value": round(value, 4), "unit": "eig/s", "cores": cpu_cores(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 4), "unit": "eig/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_reference_svd(args):
    """Oracle reference arm for u1_two_site_svd: each step is the oracle's blockwise SVD,
    truncation and factors of the same tensor."""
    w, To = _oracle_svd_inputs()
    for _ in range(args.warmup):
        _oracle_svd_step(w, To)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _oracle_svd_step(w, To)
    dt = time.perf_counter() - t0
    value = args.steps / dt
    sample = "step = the oracle's blockwise SVD (numpy, FP64) + truncation + factors of the same tensor"
    return {
        "metric": SVD_METRIC, "value": round(value, 4), "unit": "SVD/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(dt * 1e3 / args.steps, 2), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": bench_config(SVDWorkload.describe), "sample": sample,
        "cpu_baseline": {"value": round(value, 4), "unit": "SVD/s", "cores": cpu_cores(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 4), "unit": "SVD/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


# ------------------------------------------- SU(2) vs regular micro-benchmarks ---

MICRO_METRIC = "SU(2)-invariant vs regular time ratio (regular / SU(2)), matrix multiply at the largest d"


class MicroWorkload:
    describe = ("su2_micro: the thesis's comparisons of SU(2)-invariant and regular tensors (Ch. 5, Figs. "
                "permutereshapecompare and multsvdcompare): permute two indices and fuse two indices of a rank-4 "
                "tensor whose legs have spins 0, 1, 2 with degeneracy d each (dense size 9d per leg), multiply and "
                "SVD 9d x 9d matrices (three d x d blocks); 'regular' = the same dense tensor as a one-charge "
                "tensor through the same kernels; plus the recoupling coefficients a permutation evaluates (Fig. sn1)")
    default_steps = 5
    default_warmup = 2
    default_fp64_steps = 0


def _time_ms(fn, steps, warmup, flush, stream):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return sorted(ts)[len(ts) // 2]


def run_su2_micro(args, rank, world):
    """Every comparison of SU(2)-invariant and regular tensors the thesis plots,
    on the library's kernels; one JSON line with every series."""
    import ctypes
    import itertools

    import torch
    import paper_1203_2222_gb300 as P
    from paper_1203_2222_gb300 import _lib as L

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    K, W = args.steps, args.warmup
    spins = [0, 2, 4]  # 2j: j = 0, 1, 2

    def su2_leg(d, dr):
        return (spins, [d] * 3, dr)

    def reg_leg(d, dr):
        return ([0], [9 * d], dr)

    def transform_ms(S, make_plan, dtype=torch.float64):
        plan = make_plan(S)
        x = torch.randn(S.numel, dtype=dtype, device=dev)
        y = torch.empty(plan.out.numel, dtype=dtype, device=dev)
        args_ = (plan._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                 ctypes.c_void_p(stream.cuda_stream))
        ms = _time_ms(lambda: L.check(L.lib.sym_plan_execute(*args_)), K, W, flush, stream)
        launches[0] += K * plan.launches()
        return ms, S.numel

    series = {"permute": [], "fuse": [], "matmul": [], "svd": []}
    launches = [0]  # the library's kernels launched by the timed calls
    for d in (2, 4, 8, 12, 16, 20):
        row = {"d": d}
        for kind, leg, grp in (("su2", su2_leg, P.SU2), ("regular", reg_leg, P.U1)):
            S = P.Structure(grp, [leg(d, 1)] * 4)
            ms, n = transform_ms(S, lambda S: P.permute_plan(S, [0, 2, 1, 3], None, P.FP64))
            row[kind + "_ms"], row[kind + "_coefficients"] = round(ms, 4), n
        row["ratio"] = round(row["regular_ms"] / row["su2_ms"], 3)
        series["permute"].append(row)
        row = {"d": d}
        for kind, leg, grp in (("su2", su2_leg, P.SU2), ("regular", reg_leg, P.U1)):
            S = P.Structure(grp, [leg(d, 1)] * 4)
            ms, n = transform_ms(S, lambda S: P.fuse_plan(S, 0, P.FP64))
            row[kind + "_ms"] = round(ms, 4)
        row["ratio"] = round(row["regular_ms"] / row["su2_ms"], 3)
        series["fuse"].append(row)
        torch.cuda.empty_cache()

    # (d <= 1024: a regular 9d x 9d product with 9d > 16384 would exceed the
    # planner's longest tensor-core reduction and run on the CUDA cores)
    for d in (64, 128, 256, 512, 1024):
        row = {"d": d}
        for kind, leg, grp in (("su2", su2_leg, P.SU2), ("regular", reg_leg, P.U1)):
            SA = P.Structure(grp, [leg(d, 1), leg(d, -1)])
            SB = P.Structure(grp, [leg(d, 1), leg(d, -1)])
            A = P.SymTensor(SA, torch.randn(SA.numel, device=dev))
            B = P.SymTensor(SB, torch.randn(SB.numel, device=dev))
            with torch.no_grad():
                row[kind + "_ms"] = round(_time_ms(lambda: P.contract(A, B, [1], [0]), K, W, flush, stream), 4)
            launches[0] += K * P.contract_plan(SA, SB, [1], [0], P.BF16X3).launches()
        row["ratio"] = round(row["regular_ms"] / row["su2_ms"], 3)
        row["dtype"] = "split-BF16 x3 (fp32 blocks)"
        series["matmul"].append(row)
        torch.cuda.empty_cache()

    for d in (8, 16, 32, 64):
        row = {"d": d}
        for kind, leg, grp in (("su2", su2_leg, P.SU2), ("regular", reg_leg, P.U1)):
            S = P.Structure(grp, [leg(d, 1), leg(d, -1)])
            T = P.SymTensor(S, torch.randn(S.numel, dtype=torch.float64, device=dev))
            row[kind + "_ms"] = round(_time_ms(lambda: P.svd(T, 1), K, W, flush, stream), 4)
            launches[0] += 2 * K  # the Jacobi and the factor launch
        Md = torch.randn(9 * d, 9 * d, dtype=torch.float64, device=dev)
        row["regular_library_ms"] = round(_time_ms(lambda: torch.linalg.svd(Md), K, W, flush, stream), 4)
        row["ratio"] = round(row["regular_ms"] / row["su2_ms"], 3)
        row["dtype"] = "f64"
        series["svd"].append(row)
    P.device_status()

    # Fig. sn1: recoupling coefficients (spin networks) a permutation of two
    # neighbouring legs evaluates, against the rank and the spins per leg
    sn = []
    for k in (3, 4, 5, 6):
        for nsp in (1, 2, 3, 4):
            sp = [2 * i for i in range(nsp)]
            S = P.Structure(P.SU2, [(sp, [1] * nsp, 1)] * k)
            t0 = time.perf_counter()
            plan = P.permute_plan(S, [0, 2, 1] + list(range(3, k)), None, P.FP64)
            dt = time.perf_counter() - t0
            n = 0
            for tup in itertools.product(sp, repeat=k):
                G, _, _ = P.su2_gamma(list(tup), None, [0, 2, 1] + list(range(3, k)), None)
                n += int(np.count_nonzero(np.abs(G) > 1e-12))  # exact zeros may round to ~1e-17
            sn.append({"rank": k, "spins_per_leg": nsp, "coefficients": n, "plan_ms": round(dt * 1e3, 3)})
    last = series["matmul"][-1]
    out = {
        "metric": MICRO_METRIC, "value": last["ratio"], "unit": "x", "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": last["su2_ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 (permute, fuse, svd), bf16x3-f32acc (matmul)", "data": "synthetic",
        "config": dict(bench_config(MicroWorkload.describe), l2="flushed before every timed call (256 MiB write)"),
        "timing": f"median of {K} calls after {W} warm-up calls, CUDA events",
        "series": series, "spin_networks": sn, "gpu_launches": launches[0],
    }
    return out


# ------------------------------------------------------------ oracle (CPU) ---

class OracleMPS:
    """The FP64 CPU oracle on the same workload (dense embedding, brute force)."""

    def __init__(self, group="u1"):
        from oracle import su2, su2u1, u1, z2f
        from paper_1203_2222_gb300 import synthetic
        mod = {"u1": u1, "z2f": z2f, "su2u1": su2u1}[group]
        m = {"u1": synthetic.u1_mps_heff, "z2f": synthetic.z2f_mps_heff, "su2u1": synthetic.su2u1_mps_heff}[group]()
        self.group = group
        self.legs = {n: [mod.Leg(*l) for l in m[n]] for n in ("L", "A", "W", "R")}
        # second member of a tensor: total charge, or (tree, total) for SU(2) x U(1)
        self.tot = {n: (su2.left_comb(len(self.legs[n])), 0) if group == "su2u1" else 0 for n in self.legs}
        self.data = {n: synthetic.normal(m["seeds"][n], mod.layout(self.legs[n], self.tot[n])[2]) for n in self.legs}
        self.steps = [("L", "A", [2], [0]), (None, "W", [1, 2], [0, 2]), (None, "R", [1, 3], [2, 1])]

    def contraction(self, i, a=None):
        """Forward + gradient of contraction i of the chain (i = 0, 1, 2)."""
        from oracle import contract as oc
        an, bn, pa, pb = self.steps[i]
        A = (self.legs[an], self.tot[an], self.data[an]) if an else a
        B = (self.legs[bn], self.tot[bn], self.data[bn])
        lc, qc, c, _ = oc.contract(self.group, A, B, pa, pb)
        g = np.random.default_rng(i).standard_normal(c.size)
        oc.contract_grad(self.group, A, B, pa, pb, g)
        return (lc, qc, c)

    def forward0(self):
        """Forward of the first contraction (L.A) alone."""
        from oracle import contract as oc
        return oc.contract(self.group, (self.legs["L"], self.tot["L"], self.data["L"]),
                           (self.legs["A"], self.tot["A"], self.data["A"]), [2], [0])

    def full_step(self):
        a = None
        for i in range(3):
            a = self.contraction(i, a)

    def inputs_of(self, i):
        """Input of contraction i (computed once, outside any timing)."""
        from oracle import contract as oc
        a = None
        for j in range(i):
            an, bn, pa, pb = self.steps[j]
            A = (self.legs[an], self.tot[an], self.data[an]) if an else a
            lc, qc, c, _ = oc.contract(self.group, A, (self.legs[bn], self.tot[bn], self.data[bn]), pa, pb)
            a = (lc, qc, c)
        return a


np = None


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


class LazyBlocks:
    """Block data of a tensor drawn on demand: the entries at [o, o + n) of a
    block starting at offset o are N(0,1) draws of PCG64(seed, stream o)."""

    def __init__(self, seed):
        self.seed = seed

    def __getitem__(self, sl):
        from paper_1203_2222_gb300 import synthetic
        return synthetic.normal(self.seed, sl.stop - sl.start, stream=sl.start)


class OracleSU2:
    """The FP64 CPU oracle on the SU(2) recoupling workload: dense elements of
    C = contract(A, B), each from two embedded slices (oracle.su2.embed_slice);
    the dense tensors (7.5e8 block entries for A) are never formed."""

    def __init__(self):
        from oracle import contract as oc
        from oracle import su2
        from paper_1203_2222_gb300 import synthetic
        c = synthetic.su2_recouple(dmax=32, jmax2=8)
        self.su2 = su2
        self.la = [su2.Leg(*l) for l in c["A"]]
        self.lb = [su2.Leg(*l) for l in c["B"]]
        self.lc = oc.result_legs(self.la, self.lb, c["pairsA"], c["pairsB"])
        self.nodes_c = oc.comb_pair_tree(2, 2)
        self.secs = su2.layout(self.lc, self.nodes_c)[0]
        self.loffs = [l.offsets() for l in self.lc]
        self.a, self.b = LazyBlocks(1236), LazyBlocks(1237)
        self.rng = np.random.default_rng(0)

    def element(self):
        su2 = self.su2
        sec = self.secs[int(self.rng.integers(len(self.secs)))]
        idx = [self.loffs[l][p] + int(self.rng.integers((self.lc[l].labels[p] + 1) * self.lc[l].degens[p]))
               for l, p in enumerate(sec[0])]
        sa = su2.embed_slice(self.la, su2.left_comb(4), self.a, {0: idx[0], 2: idx[1]})
        sb = su2.embed_slice(self.lb, su2.left_comb(4), self.b, {2: idx[2], 3: idx[3]})
        return float(np.sum(sa * sb))


def su2_oracle_check(h, flops, n):
    """The FP64 CPU oracle on the bench's own inputs and results: n dense
    elements each of C, dA and dB (oracle.sample: slices of the embedded
    inputs, summed), at indices drawn in uniformly chosen sectors, against
    the embedding of the GPU's result blocks at the same indices.  Returns
    the cpu_baseline (the oracle's elements timed on the host cores, each
    credited the useful flops per block entry of its tensor) and the relative
    error of each result over its sample."""
    from oracle import contract as oc
    from oracle import sample, su2
    from paper_1203_2222_gb300 import synthetic
    c = synthetic.su2_recouple(dmax=32, jmax2=8)
    la = [su2.Leg(*l) for l in c["A"]]
    lb = [su2.Leg(*l) for l in c["B"]]
    pa, pb = c["pairsA"], c["pairsB"]
    lc = oc.result_legs(la, lb, pa, pb)
    comb, nodes_c = su2.left_comb(4), oc.comb_pair_tree(2, 2)
    A, B, G = (la, comb, h["A"]), (lb, comb, h["B"]), (lc, nodes_c, h["G"])
    rng = np.random.default_rng(0)

    per_entry = {"C": flops / 3.0 / h["C"].size, "dA": flops / 3.0 / h["A"].size, "dB": flops / 3.0 / h["B"].size}
    kinds = {
        "C": (lambda i: sample.contraction_element(su2, A, B, pa, pb, i), (lc, nodes_c, h["C"]), (lc, nodes_c)),
        "dA": (lambda i: sample.grad_a_element(su2, A, B, pa, pb, G, i), (la, comb, h["dA"]), (la, comb)),
        "dB": (lambda i: sample.grad_b_element(su2, A, B, pa, pb, G, i), (lb, comb, h["dB"]), (lb, comb)),
    }
    t_ref, credited, errs = 0.0, 0.0, {}
    for name, (ref_fn, got_t, lay) in kinds.items():
        idxs = sample.draw_indices(su2, *lay, rng, n)
        t0 = time.perf_counter()
        ref = np.array([ref_fn(i) for i in idxs])
        t_ref += time.perf_counter() - t0
        credited += n * per_entry[name]
        got = np.array([sample.element(su2, got_t, i) for i in idxs])
        errs[name] = float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300))
    base = {"value": round(credited / t_ref / 1e12, 9), "unit": "TFLOP/s", "cores": cpu_cores(), "kind": "oracle",
            "sample": f"{n} dense elements each of C, dA and dB on the bench's own inputs (slices of the embedded "
                      f"tensors, FP64 numpy oracle), each credited the useful flops per block entry of its tensor; "
                      f"{t_ref:.1f} s"}
    err = {"value": max(errs.values()), "per_result": errs,
           "sample": f"relative Frobenius error over {n} sampled dense elements of each result"}
    return base, err


def su2_flops_per_entry():
    """Forward useful flops per block entry of C (host planning only)."""
    os.environ["SYM_PLAN_DRYRUN"] = "1"
    import paper_1203_2222_gb300 as P
    from paper_1203_2222_gb300 import synthetic
    c = synthetic.su2_recouple(dmax=32, jmax2=8)
    p = P.contract_plan(P.Structure(P.SU2, c["A"]), P.Structure(P.SU2, c["B"]), c["pairsA"], c["pairsB"], P.BF16X3)
    return p.stats()["flops_fwd"] / p.out.numel


SU2_SAMPLE = 4  # dense elements per oracle step (about 2-3 s of host work)


class OracleBatch:
    """The FP64 CPU oracle on the batch workload: the whole chain of one
    problem, forward and the gradients of <G, Y> (dense embedding, brute
    force), with the problem's own seeded inputs."""

    def __init__(self):
        from paper_1203_2222_gb300 import synthetic
        self.spec = synthetic.u1_two_site_batch()
        self.order = sorted(range(len(self.spec["problems"])), key=lambda i: self.spec["problems"][i]["D"])

    def problem_flops(self, i):
        """Useful flops of problem i's fwd + bwd (host planning only)."""
        os.environ["SYM_PLAN_DRYRUN"] = "1"
        try:
            import paper_1203_2222_gb300 as P
            p = self.spec["problems"][i]
            S = {n: P.Structure(P.U1, p[n]) for n in ("L", "theta", "W", "R")}
            tot, cur = 0.0, S["L"]
            for an, bn, pa, pb in self.spec["steps"]:
                pl = P.contract_plan(cur if an is None else S[an], S[bn], pa, pb, P.BF16X3)
                tot += 3.0 * pl.stats()["flops_fwd"]
                cur = pl.out
            return tot
        finally:
            del os.environ["SYM_PLAN_DRYRUN"]

    def step(self, i):
        from oracle import contract as oc
        from oracle import u1
        from paper_1203_2222_gb300 import synthetic
        p = self.spec["problems"][i]
        legs = {n: [u1.Leg(*l) for l in p[n]] for n in ("L", "theta", "W", "R")}
        data = {n: synthetic.normal(p["seed"], u1.layout(legs[n], 0)[2], stream=BATCH_STREAMS[n]) for n in legs}
        ins, cur = [], (legs["L"], 0, data["L"])
        for an, bn, pa, pb in self.spec["steps"]:
            a = cur if an is None else (legs[an], 0, data[an])
            b = (legs[bn], 0, data[bn])
            lc, qc, c, _ = oc.contract("u1", a, b, pa, pb)
            ins.append((a, b, pa, pb))
            cur = (lc, qc, c)
        dc = np.random.default_rng(i).standard_normal(cur[2].size)
        for a, b, pa, pb in reversed(ins):
            dc, _, _ = oc.contract_grad("u1", a, b, pa, pb, dc)


class OracleMera:
    """The FP64 CPU oracle on the MERA workload: the dense energy of the patch
    (oracle.mera.energy, reduced density matrices, numpy BLAS einsums)."""

    def __init__(self):
        from oracle import mera, u1
        from paper_1203_2222_gb300 import synthetic
        spec = synthetic.u1_mera()
        legs = {n: [u1.Leg(*l) for l in spec[n]] for n in ("t", "w", "u", "h")}
        scale = 1.0 / np.sqrt(spec["chi"])
        self.dense = {n: u1.embed(legs[n], 0, synthetic.normal(spec["seeds"][n], u1.layout(legs[n], 0)[2]) * scale)
                      for n in ("t", "w", "u")}
        self.H = mera.h_dense(legs["h"], lambda *a: synthetic.mera_h_entry(spec["delta"], *a))
        self.mera = mera

    def energy(self):
        d = self.dense
        return self.mera.energy(d["t"], d["w"], d["u"], self.H)


def mera_forward_flops():
    """Useful forward flops of the MERA energy (host planning only)."""
    os.environ["SYM_PLAN_DRYRUN"] = "1"
    try:
        import paper_1203_2222_gb300 as P
        wl = MeraWorkload()
        from paper_1203_2222_gb300 import networks, synthetic
        wl.spec = synthetic.u1_mera()
        wl.S = networks.mera_structures(wl.spec)
        uniq = {id(p): p for p, _, _ in wl.contractions(P, P.BF16X3)}
        return sum(p.stats()["flops_fwd"] for p in uniq.values())
    finally:
        del os.environ["SYM_PLAN_DRYRUN"]


BATCH_SAMPLE = 4  # problems per oracle step (the smallest ones, about a second of host work)
BATCH_BASELINE = 24  # problems of the cpu_baseline sample (about 10 s of host work)


def cpu_baseline(args, flops, steps):
    if args.workload == "u1_mera_grad":
        o = OracleMera()
        fwd = mera_forward_flops()
        n = max(steps, 1) * 3
        t0 = time.perf_counter()
        for _ in range(n):
            o.energy()
        dt = time.perf_counter() - t0
        return {"value": round(fwd * n / dt / 1e12, 9), "unit": "TFLOP/s", "cores": cpu_cores(), "kind": "oracle",
                "sample": f"{n} dense evaluations of the energy (no gradient: the oracle has none but finite "
                          f"differences), credited the forward useful flops of the block-sparse path; {dt:.1f} s"}
    if args.workload == "u1_two_site_batch":
        o = OracleBatch()
        probs = o.order[:BATCH_BASELINE * max(steps, 1)]
        fl = sum(o.problem_flops(i) for i in probs)
        t0 = time.perf_counter()
        for i in probs:
            o.step(i)
        dt = time.perf_counter() - t0
        return {"value": round(fl / dt / 1e12, 9), "unit": "TFLOP/s", "cores": cpu_cores(), "kind": "oracle",
                "sample": f"the {len(probs)} smallest problems of the batch (D = "
                          f"{', '.join(str(o.spec['problems'][i]['D']) for i in probs)}), whole chain fwd + grad, "
                          f"dense FP64 numpy oracle, credited their own useful flops; {dt:.1f} s"}
    if args.workload == "su2_recouple":
        o = OracleSU2()
        per = flops / 3.0 / su2_flops_per_entry_cached()
        o.element()
        t0 = time.perf_counter()
        n = SU2_SAMPLE * max(steps, 1)
        for _ in range(n):
            o.element()
        dt = time.perf_counter() - t0
        return {"value": round(n * per / dt / 1e12, 9), "unit": "TFLOP/s", "cores": cpu_cores(), "kind": "oracle",
                "sample": f"{n} dense elements of C from embedded slices of A and B (FP64 numpy oracle), each "
                          f"credited the forward useful flops per block entry of C; {dt:.1f} s"}
    if args.workload == "su2u1_mps_heff":
        o = OracleMPS("su2u1")
        f0 = contraction_flops_host("su2u1")[0]
        t0 = time.perf_counter()
        o.forward0()
        dt = time.perf_counter() - t0
        return {"value": round(f0 / dt / 1e12, 9), "unit": "TFLOP/s", "cores": cpu_cores(), "kind": "oracle",
                "sample": f"the forward of the first contraction (L.A) alone, dense FP64 oracle with CG trees, "
                          f"credited its own useful flops; {dt:.1f} s"}
    o = OracleMPS("z2f" if args.workload == "z2f_mps_heff" else "u1")
    t0 = time.perf_counter()
    for _ in range(steps):
        o.full_step()
    dt = time.perf_counter() - t0
    return {"value": round(flops * steps / dt / 1e12, 6), "unit": "TFLOP/s", "cores": cpu_cores(),
            "kind": "oracle",
            "sample": f"{steps} full fwd+bwd step(s) of the same workload, dense FP64 numpy oracle, "
                      f"{dt:.1f} s"}


_PER_ENTRY = []


def su2_flops_per_entry_cached():
    if not _PER_ENTRY:
        _PER_ENTRY.append(su2_flops_per_entry())
    return _PER_ENTRY[0]


def run_reference_mera(args):
    """Oracle reference arm for u1_mera_grad: each step is one dense energy evaluation."""
    fwd = mera_forward_flops()
    o = OracleMera()
    for _ in range(args.warmup):
        o.energy()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.energy()
    dt = time.perf_counter() - t0
    value = fwd * args.steps / dt / 1e12
    sample = ("step = one dense FP64 evaluation of the energy (numpy oracle, no gradient), credited the forward "
              "useful flops of the block-sparse path")
    return {
        "metric": METRIC, "value": round(value, 9), "unit": "TFLOP/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(dt * 1e3 / args.steps, 2), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": bench_config(MeraWorkload.describe), "sample": sample,
        "cpu_baseline": {"value": round(value, 9), "unit": "TFLOP/s", "cores": cpu_cores(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 9), "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_reference_batch(args):
    """Oracle reference arm for u1_two_site_batch: each step is BATCH_SAMPLE problems (smallest first, rotating)."""
    o = OracleBatch()
    pool = o.order[:16]
    fl_of = {i: o.problem_flops(i) for i in pool}
    for w in range(args.warmup):
        o.step(pool[w % len(pool)])
    t0 = time.perf_counter()
    fl = 0.0
    for s_ in range(args.steps):
        for q in range(BATCH_SAMPLE):
            i = pool[(s_ * BATCH_SAMPLE + q) % len(pool)]
            o.step(i)
            fl += fl_of[i]
    dt = time.perf_counter() - t0
    value = fl / dt / 1e12
    sample = (f"step = {BATCH_SAMPLE} of the 16 smallest problems of the batch, rotating, whole chain fwd + grad, "
              f"dense FP64 numpy oracle, credited their own useful flops")
    return {
        "metric": METRIC, "value": round(value, 9), "unit": "TFLOP/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(dt * 1e3 / args.steps, 2), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": bench_config(BatchWorkload.describe), "sample": sample,
        "cpu_baseline": {"value": round(value, 9), "unit": "TFLOP/s", "cores": cpu_cores(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 9), "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_reference_su2(args):
    """Oracle reference arm for su2_recouple: each step is SU2_SAMPLE dense elements."""
    per = su2_flops_per_entry()
    o = OracleSU2()
    for _ in range(args.warmup):
        for _ in range(SU2_SAMPLE):
            o.element()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for _ in range(SU2_SAMPLE):
            o.element()
    dt = time.perf_counter() - t0
    value = SU2_SAMPLE * args.steps * per / dt / 1e12
    sample = (f"step = {SU2_SAMPLE} dense elements of C from embedded slices (FP64 numpy oracle), "
              f"credited the forward useful flops per block entry of C")
    return {
        "metric": METRIC, "value": round(value, 9), "unit": "TFLOP/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(dt * 1e3 / args.steps, 2), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": bench_config(SU2Workload.describe), "sample": sample,
        "cpu_baseline": {"value": round(value, 9), "unit": "TFLOP/s", "cores": cpu_cores(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 9), "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_reference(args, flops_by_contraction, group="u1"):
    """The oracle as the reference arm: each step is one contraction of the chain (fwd + grad), rotating."""
    o = OracleMPS(group)
    ins = [o.inputs_of(i) for i in range(3)]
    for w in range(args.warmup):
        o.contraction(w % 3, ins[w % 3])
    t0 = time.perf_counter()
    fl = 0.0
    for s in range(args.steps):
        o.contraction(s % 3, ins[s % 3])
        fl += 3.0 * flops_by_contraction[s % 3]
    dt = time.perf_counter() - t0
    value = fl / dt / 1e12
    return {
        "metric": METRIC, "value": round(value, 6), "unit": "TFLOP/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(dt * 1e3 / args.steps, 2), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": bench_config(WORKLOAD if group == "u1" else Z2FMPSWorkload.describe),
        "sample": "step s = contraction (s mod 3) of the chain, fwd + grad",
        "cpu_baseline": {"value": round(value, 6), "unit": "TFLOP/s", "cores": cpu_cores(), "kind": "oracle",
                         "sample": "one contraction of ((L.A).W).R per step, rotating, dense FP64 numpy oracle"},
        "e2e": {"value": round(value, 6), "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_reference_su2u1(args):
    """Oracle reference arm for su2u1_mps_heff: each step is the forward of the
    first contraction (L.A) (the dense CG-tree oracle takes seconds per step)."""
    f0 = contraction_flops_host("su2u1")[0]
    o = OracleMPS("su2u1")
    for _ in range(args.warmup):
        o.forward0()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.forward0()
    dt = time.perf_counter() - t0
    value = f0 * args.steps / dt / 1e12
    sample = "step = forward of the first contraction (L.A), dense FP64 oracle with CG trees, its own useful flops"
    return {
        "metric": METRIC, "value": round(value, 9), "unit": "TFLOP/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(dt * 1e3 / args.steps, 2), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": bench_config(SU2U1MPSWorkload.describe), "sample": sample,
        "cpu_baseline": {"value": round(value, 9), "unit": "TFLOP/s", "cores": cpu_cores(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 9), "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def contraction_flops_host(group="u1"):
    """Useful forward flops of each contraction of the chain (host planning only)."""
    old = os.environ.get("SYM_PLAN_DRYRUN")
    os.environ["SYM_PLAN_DRYRUN"] = "1"
    try:
        import paper_1203_2222_gb300 as P
        m, S = mps_structures(P, group)
        t1 = P.contract_plan(S["L"], S["A"], [2], [0], P.BF16X3)
        t2 = P.contract_plan(t1.out, S["W"], [1, 2], [0, 2], P.BF16X3)
        t3 = P.contract_plan(t2.out, S["R"], [1, 3], [2, 1], P.BF16X3)
        return [t.stats()["flops_fwd"] for t in (t1, t2, t3)]
    finally:
        if old is None:
            del os.environ["SYM_PLAN_DRYRUN"]
        else:
            os.environ["SYM_PLAN_DRYRUN"] = old


def main():
    global np
    import numpy
    np = numpy
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        if rank != 0:
            return 0
        if args.workload == "su2_micro":
            out = {"impl": "reference", "unavailable": "su2_micro compares SU(2)-invariant and regular tensors on the "
                                                      "library's own kernels; the thesis's MATLAB timings have no values"}
        elif args.workload == "u1_two_site_svd":
            out = run_reference_svd(args)
        elif args.workload == "u1_two_site_eig":
            out = run_reference_eig(args)
        elif args.workload == "su2_recouple":
            out = run_reference_su2(args)
        elif args.workload == "u1_two_site_batch":
            out = run_reference_batch(args)
        elif args.workload == "u1_mera_grad":
            out = run_reference_mera(args)
        elif args.workload == "su2u1_mps_heff":
            out = run_reference_su2u1(args)
        else:
            g = "z2f" if args.workload == "z2f_mps_heff" else "u1"
            out = run_reference(args, contraction_flops_host(g), g)
        print(json.dumps(out))
        return 0
    import torch
    if world > 1:
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        torch.distributed.init_process_group("nccl")
    if args.workload == "su2_micro":
        out = run_su2_micro(args, rank, world)
    elif args.workload in ("u1_two_site_svd", "u1_two_site_eig"):
        out, check = run_svd(args, rank, world)
        if rank == 0 and not args.no_cpu_baseline:
            fn = cpu_baseline_eig if args.workload == "u1_two_site_eig" else cpu_baseline_svd
            out["cpu_baseline"], out["max_rel_err_vs_oracle"] = fn(args.cpu_sample_steps, check)
    else:
        out, flops, check = run_ours(args, rank, world)
        if rank == 0 and not args.no_cpu_baseline:
            if check is not None:
                out["cpu_baseline"], out["max_rel_err_vs_oracle"] = su2_oracle_check(
                    check, flops, SU2_SAMPLE * max(args.cpu_sample_steps, 1))
            else:
                out["cpu_baseline"] = cpu_baseline(args, flops, args.cpu_sample_steps)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
