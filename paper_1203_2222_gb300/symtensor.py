"""Python front end of the GB300 symmetric block-sparse tensor library.

Thin layer over the C ABI (``include/symtensor.h``): structures and plans are
host handles; block data are 1-D torch tensors on the GPU (float32 for the
split-BF16 tensor-core path, float64 for the plain FP64 path).  Every step of
every operation runs in the library's kernels; PyTorch provides device memory,
the current CUDA stream and autograd bookkeeping.

    A = SymTensor.randn(Structure(U1, legs_a, total=0), seed, dtype=torch.float32)
    C = contract(A, B, pairsA=[2, 3], pairsB=[0, 1])     # autograd-aware
"""
import ctypes

import numpy as np
import torch

from . import _lib as L

U1, SU2, Z2F, SU2U1 = L.SYM_U1, L.SYM_SU2, L.SYM_Z2F, L.SYM_SU2U1


def su2u1_label(q, spin2):
    """The C ABI's SU(2) x U(1) label of charge q and doubled spin 2j (include/symtensor.h)."""
    if not 0 <= spin2 < 64:
        raise ValueError("2j must be in 0..63")
    return 64 * int(q) + int(spin2)


def su2u1_pair(label):
    return ((label - label % 64) // 64, label % 64)
FP64, BF16X3 = L.SYM_PREC_FP64, L.SYM_PREC_BF16X3
SymError = L.SymError


def _byref(x):
    return ctypes.byref(x)


class Structure:
    """Sector table of a symmetric tensor (legs, total charge or tree); host only.

    ``legs`` is a sequence of ``(labels, degens, dir)`` (U(1) charges, SU(2)
    doubled spins, fermion parities 0/1, or SU(2) x U(1) pairs (q, 2j);
    strictly increasing; dir +1 out, -1 in).  ``tree`` (SU(2), SU(2) x U(1))
    is a list of ``(left, right)`` node children, None for the left comb.
    ``legs`` of an SU(2) x U(1) structure read back as (q, 2j) pairs.
    """

    def __init__(self, group, legs=None, total=0, tree=None, _handle=None):
        self.group = int(group)
        if _handle is None:
            if self.group == SU2U1:
                legs = [([su2u1_label(q, j) for q, j in lab], deg, d) for lab, deg, d in legs]
            arr, _keep = L.leg_array(legs)
            h = ctypes.c_void_p()
            L.check(L.lib.sym_tensor_create(self.group, len(legs), arr, int(total),
                                            L.tree_array(tree), _byref(h)))
            self._h = h
        else:
            self._h = _handle
        self.total = 0 if self.group == SU2 else int(total)
        g, r, n, ns = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64()
        L.check(L.lib.sym_tensor_info(self._h, _byref(g), _byref(r), _byref(n), _byref(ns)))
        self.rank, self.numel, self.nsec = r.value, n.value, ns.value
        self.legs = [self._leg(i) for i in range(self.rank)]
        self.tree = None
        if self.group in (SU2, SU2U1) and self.rank >= 2:
            buf = (ctypes.c_int * (2 * (self.rank - 1)))()
            L.check(L.lib.sym_tensor_tree(self._h, buf))
            self.tree = [(buf[2 * i], buf[2 * i + 1]) for i in range(self.rank - 1)]

    def _leg(self, i):
        n, d = ctypes.c_int(), ctypes.c_int()
        L.check(L.lib.sym_tensor_leg(self._h, i, _byref(n), None, None, _byref(d)))
        la = (ctypes.c_int * n.value)()
        de = (ctypes.c_int * n.value)()
        L.check(L.lib.sym_tensor_leg(self._h, i, None, la, de, None))
        labels = tuple(su2u1_pair(x) for x in la) if self.group == SU2U1 else tuple(la)
        return (labels, tuple(de), d.value)

    def sectors(self):
        """(labels[nsec, rank + max(rank-2,0)] int32, offsets[nsec+1] int64)."""
        w = self.rank + (max(self.rank - 2, 0) if self.group in (SU2, SU2U1) else 0)
        lab = np.zeros((self.nsec, w), dtype=np.int32)
        off = np.zeros(self.nsec + 1, dtype=np.int64)
        L.check(L.lib.sym_tensor_sectors(self._h, lab.ctypes.data_as(L._IP) if lab.size else None,
                                         off.ctypes.data_as(L._LP)))
        return lab, off

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and L is not None and L.lib is not None:
            L.lib.sym_tensor_destroy(h)
            self._h = None


class Plan:
    """Precomputed tables + scratch of one operation (owned handle)."""

    def __init__(self, handle, out, kind, precision=None):
        self._h = handle
        self.out = out
        self.kind = kind
        self.precision = precision

    @property
    def c_numel(self):
        """Elements of the result (of all problems, for a batch plan)."""
        return self.out.numel

    def stats(self):
        f = ctypes.c_double()
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        L.check(L.lib.sym_plan_stats(self._h, _byref(f), _byref(a), _byref(b), _byref(c)))
        return {"flops_fwd": f.value, "bytes_a": a.value, "bytes_b": b.value, "bytes_c": c.value}

    def launches(self):
        n = ctypes.c_int()
        L.check(L.lib.sym_plan_launches(self._h, _byref(n)))
        return n.value

    def gemm_shapes(self):
        """(m, n, k, kernel) of every GEMM; kernel 0 = tcgen05, 1 = CUDA cores."""
        n = ctypes.c_int()
        L.check(L.lib.sym_plan_gemm_shapes(self._h, _byref(n), None))
        buf = (ctypes.c_int * max(4 * n.value, 1))()
        L.check(L.lib.sym_plan_gemm_shapes(self._h, _byref(n), buf))
        return [tuple(buf[4 * i:4 * i + 4]) for i in range(n.value)]

    def profile(self, enable=True):
        """Start (clear) or stop recording device time of this plan's launches."""
        L.check(L.lib.sym_plan_profile(self._h, 1 if enable else 0))

    def profile_read(self, phase):
        """{launches, ms, bytes, flops} recorded for one phase (see SYM_PHASE_*)."""
        n = ctypes.c_int()
        ms, by, fl = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        L.check(L.lib.sym_plan_profile_read(self._h, int(phase), _byref(n), _byref(ms), _byref(by), _byref(fl)))
        return {"launches": n.value, "ms": ms.value, "bytes": by.value, "flops": fl.value}

    def profile_kernel(self, kernel):
        """{launches, ms, bytes, flops} recorded for one kernel (see SYM_KERNEL_*)."""
        n = ctypes.c_int()
        ms, by, fl = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        L.check(L.lib.sym_plan_profile_kernel(self._h, int(kernel), _byref(n), _byref(ms), _byref(by), _byref(fl)))
        return {"launches": n.value, "ms": ms.value, "bytes": by.value, "flops": fl.value}

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and L is not None and L.lib is not None:
            L.lib.sym_plan_destroy(h)
            self._h = None


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _precision(dtype):
    if dtype == torch.float64:
        return FP64
    if dtype == torch.float32:
        return BF16X3
    raise TypeError("block data must be float32 (split-BF16 path) or float64 (FP64 path)")


_PLANS = {}

# phases of a plan's launches (include/symtensor.h, SYM_PHASE_*)
PHASES = {"fwd_gather": 0, "fwd_gemm_tc": 1, "fwd_scatter": 2, "bwd_gather": 3, "bwd_gemm_tc": 4,
          "bwd_scatter": 5, "transform": 6, "fwd_gemm_cuda_cores": 7, "bwd_gemm_cuda_cores": 8,
          "fwd_direct": 9, "bwd_direct": 10}
# kernels of a plan's launches (include/symtensor.h, SYM_KERNEL_*), with the
# name of the CUDA kernel each one launches
KERNELS = {"box": 0, "box_flat": 1, "gemm_tc": 2, "gemm_tile": 3, "gemm_wide": 4, "gemm_thin": 5, "gemm_rows": 6,
           "direct": 7}
KERNEL_SYMBOLS = {"box": "box_kernel<T, T, 0 | 2>", "box_flat": "box_kernel<T, T, 1>",
                  "gemm_tc": "gemm_tc_kernel", "gemm_tile": "gemm_tile_kernel<T, 64, 64>",
                  "gemm_wide": "gemm_tile_kernel<T, 256, 16>", "gemm_thin": "gemm_thin_kernel<T>",
                  "gemm_rows": "gemm_rows_kernel<T>", "direct": "direct_kernel<T>"}


def _fuse_total(group, a, b):
    """Total charge of a contraction's result: U(1) sum, fermion parity sum mod 2."""
    return (a ^ b) if group == Z2F else a + b


def tune_get():
    """Current planning parameters (include/symtensor.h, sym_tune) as a dict."""
    t = L.sym_tune()
    L.check(L.lib.sym_tune_get(_byref(t)))
    return {f: int(getattr(t, f)) for f in L.TUNE_FIELDS}


def tune_set(**params):
    """Change planning parameters; plans built afterwards use them (the plan
    caches below are keyed by the tuning epoch, so later calls re-plan)."""
    cur = tune_get()
    unknown = set(params) - set(cur)
    if unknown:
        raise KeyError(f"unknown planning parameters: {sorted(unknown)}")
    cur.update({k: int(v) for k, v in params.items()})
    L.check(L.lib.sym_tune_set(_byref(L.sym_tune(**cur))))
    # plans of older epochs are never looked up again: release them (their
    # device scratch) unless a caller still holds them
    e = tune_epoch()
    for key in [k for k in _PLANS if k[0] in ("c", "b") and k[-1] != e]:
        del _PLANS[key]
    return cur


def tune_epoch():
    e = ctypes.c_int()
    L.check(L.lib.sym_tune_epoch(_byref(e)))
    return e.value


def cached_plans():
    """Every plan built so far (for profiling and statistics)."""
    return [v[0] for v in _PLANS.values()]


def contract_plan(A, B, pairsA, pairsB, precision=BF16X3, tree_c=None):
    """Plan (cached) of contracting structure A's legs pairsA with B's pairsB."""
    key = ("c", id(A), id(B), tuple(pairsA), tuple(pairsB), precision,
           None if tree_c is None else tuple(map(tuple, tree_c)), tune_epoch())
    hit = _PLANS.get(key)
    if hit is not None:
        return hit[0]
    c, p = ctypes.c_void_p(), ctypes.c_void_p()
    L.check(L.lib.sym_contract_plan(A._h, B._h, len(pairsA), L.int_array(pairsA), L.int_array(pairsB),
                                    L.tree_array(tree_c), int(precision), _byref(c), _byref(p)))
    out = Structure(A.group, total=_fuse_total(A.group, A.total, B.total), _handle=c)
    plan = Plan(p, out, "contract", int(precision))
    _PLANS[key] = (plan, A, B)
    return plan


class BatchPlan(Plan):
    """One plan over many independent contractions on packed buffers.

    ``outs[i]`` is problem i's result structure; ``off_a``, ``off_b``,
    ``off_c`` (length n + 1) are the element offsets of each problem in the
    packed A, B and C (the last entry is the packed size).
    """

    def __init__(self, handle, outs, offsets, precision):
        super().__init__(handle, None, "contract", precision)
        n = len(outs)
        self.outs = outs
        self.off_a = [int(x) for x in offsets[:n + 1]]
        self.off_b = [int(x) for x in offsets[n + 1:2 * (n + 1)]]
        self.off_c = [int(x) for x in offsets[2 * (n + 1):]]

    @property
    def c_numel(self):
        return self.off_c[-1]


def contract_batch_plan(As, Bs, pairsA, pairsB, precision=BF16X3):
    """Plan (cached) of contracting As[i] with Bs[i] over the same leg pairs, all i at once."""
    key = ("b", tuple(id(a) for a in As), tuple(id(b) for b in Bs), tuple(pairsA), tuple(pairsB), precision,
           tune_epoch())
    hit = _PLANS.get(key)
    if hit is not None:
        return hit[0]
    n = len(As)
    if n != len(Bs) or n < 1:
        raise ValueError("As and Bs must be non-empty lists of equal length")
    Ah = (ctypes.c_void_p * n)(*[a._h for a in As])
    Bh = (ctypes.c_void_p * n)(*[b._h for b in Bs])
    Ch = (ctypes.c_void_p * n)()
    offs = np.zeros(3 * (n + 1), dtype=np.int64)
    p = ctypes.c_void_p()
    L.check(L.lib.sym_contract_batch_plan(n, Ah, Bh, len(pairsA), L.int_array(pairsA), L.int_array(pairsB),
                                          int(precision), Ch, offs.ctypes.data_as(L._LP), _byref(p)))
    outs = [Structure(As[i].group, total=_fuse_total(As[i].group, As[i].total, Bs[i].total),
                      _handle=ctypes.c_void_p(Ch[i]))
            for i in range(n)]
    plan = BatchPlan(p, outs, offs, int(precision))
    _PLANS[key] = (plan, tuple(As), tuple(Bs))
    return plan


def contract_batch(plan, a, b):
    """Packed results of a batch plan: c[off_c[i]:off_c[i+1]] = contract(problem i) (autograd-aware)."""
    if a.numel() != plan.off_a[-1] or b.numel() != plan.off_b[-1]:
        raise ValueError("packed inputs do not match the batch plan")
    if _precision(a.dtype) != plan.precision or b.dtype != a.dtype:
        raise TypeError("packed inputs must have the plan's precision")
    return _Contract.apply(plan, a.contiguous(), b.contiguous())


def _transform_plan(key, make):
    hit = _PLANS.get(key)
    if hit is not None:
        return hit[0]
    o, p = ctypes.c_void_p(), ctypes.c_void_p()
    total = make(o, p)
    plan = Plan(p, None, key[0])
    plan.out = Structure(key[-1].group, total=total, _handle=o)
    _PLANS[key] = (plan,)
    return plan


def permute_plan(S, perm, tree=None, precision=BF16X3):
    key = ("p", id(S), tuple(perm), None if tree is None else tuple(map(tuple, tree)), precision, S)
    return _transform_plan(key, lambda o, p: (L.check(L.lib.sym_permute_plan(
        S._h, L.int_array(perm), L.tree_array(tree), int(precision), _byref(o), _byref(p))), S.total)[1])


def fuse_plan(S, first, precision=BF16X3, nlegs=2):
    """Plan (cached) of fusing legs first..first+nlegs-1 of structure S."""
    key = ("f", id(S), int(first), int(nlegs), precision, S)
    if nlegs == 2:
        return _transform_plan(key, lambda o, p: (L.check(L.lib.sym_fuse_plan(
            S._h, int(first), int(precision), _byref(o), _byref(p))), S.total)[1])
    return _transform_plan(key, lambda o, p: (L.check(L.lib.sym_fuse_n_plan(
        S._h, int(first), int(nlegs), int(precision), _byref(o), _byref(p))), S.total)[1])


def split_plan(S, leg, parts, precision=BF16X3):
    key = ("s", id(S), int(leg), tuple((tuple(a), tuple(b), int(c)) for a, b, c in parts), precision, S)

    def make(o, p):
        ps = parts
        if S.group == SU2U1:
            ps = [([su2u1_label(q, j) for q, j in lab], deg, d) for lab, deg, d in parts]
        arr, _keep = L.leg_array(ps)
        L.check(L.lib.sym_split_plan(S._h, int(leg), arr, int(precision), _byref(o), _byref(p)))
        return S.total

    return _transform_plan(key, make)


class _Contract(torch.autograd.Function):
    @staticmethod
    def forward(ctx, plan, a, b):
        c = torch.empty(plan.c_numel, dtype=a.dtype, device=a.device)
        L.check(L.lib.sym_contract(plan._h, _ptr(a), _ptr(b), _ptr(c), _stream()))
        ctx.plan = plan
        ctx.save_for_backward(a, b)
        return c

    @staticmethod
    def backward(ctx, dc):
        a, b = ctx.saved_tensors
        dc = dc.contiguous()
        da = torch.empty_like(a) if ctx.needs_input_grad[1] else None
        db = torch.empty_like(b) if ctx.needs_input_grad[2] else None
        L.check(L.lib.sym_contract_backward(ctx.plan._h, _ptr(a), _ptr(b), _ptr(dc), _ptr(da), _ptr(db),
                                            _stream()))
        return None, da, db


class SymTensor:
    """A symmetric tensor: structure + its block data (1-D CUDA tensor)."""

    def __init__(self, structure, data):
        if not (isinstance(data, torch.Tensor) and data.is_cuda):
            raise TypeError("block data must be a CUDA tensor")
        if data.dim() != 1 or data.numel() != structure.numel:
            raise ValueError(f"data must be 1-D with {structure.numel} elements, got {tuple(data.shape)}")
        _precision(data.dtype)
        self.structure = structure
        self.data = data if data.is_contiguous() else data.contiguous()

    @property
    def group(self):
        return self.structure.group

    @property
    def legs(self):
        return self.structure.legs

    @staticmethod
    def zeros(structure, dtype=torch.float32, device="cuda"):
        return SymTensor(structure, torch.zeros(structure.numel, dtype=dtype, device=device))

    @staticmethod
    def from_numpy(structure, values, dtype=torch.float32, device="cuda"):
        t = torch.as_tensor(np.asarray(values, dtype=np.float64)).to(dtype)
        return SymTensor(structure, t.to(device))


def contract(A, B, pairsA, pairsB, tree_c=None):
    """C = contract(A, B) summing A's legs pairsA with B's legs pairsB (autograd-aware)."""
    prec = _precision(A.data.dtype)
    if B.data.dtype != A.data.dtype:
        raise TypeError("A and B must share a dtype")
    plan = contract_plan(A.structure, B.structure, pairsA, pairsB, prec, tree_c)
    return SymTensor(plan.out, _Contract.apply(plan, A.data, B.data))


def _run_transform(plan, T):
    out = torch.empty(plan.out.numel, dtype=T.data.dtype, device=T.data.device)
    L.check(L.lib.sym_plan_execute(plan._h, _ptr(T.data), _ptr(out), _stream()))
    return SymTensor(plan.out, out)


def permute(T, perm, tree=None):
    """PERMUTE: output leg n is input leg perm[n] (SU(2): recoupled into ``tree``)."""
    return _run_transform(permute_plan(T.structure, perm, tree, _precision(T.data.dtype)), T)


def fuse(T, first, nlegs=2):
    """FUSE legs first..first+nlegs-1 into one leg (pairwise from the left)."""
    return _run_transform(fuse_plan(T.structure, first, _precision(T.data.dtype), nlegs), T)


def split(T, leg, parts):
    """SPLIT leg ``leg`` into the two legs ``parts`` (which must fuse to it)."""
    return _run_transform(split_plan(T.structure, leg, parts, _precision(T.data.dtype)), T)


def device_status():
    """Raise SymError(SYM_ERR_TIMEOUT) if a bounded device wait expired."""
    L.check(L.lib.sym_device_status())


def su2_F(jd, je, ja, jb, jc, J):
    out = ctypes.c_double()
    L.check(L.lib.sym_su2_F(jd, je, ja, jb, jc, J, _byref(out)))
    return out.value


def su2_gamma(spins, tree_in, perm, tree_out):
    """(G[n_out, n_in], labels_in, labels_out) of the host Gamma builder."""
    k = len(spins)
    ni, no = ctypes.c_int(), ctypes.c_int()
    args = (k, L.int_array(spins), L.tree_array(tree_in), L.int_array(perm), L.tree_array(tree_out))
    L.check(L.lib.sym_su2_gamma(*args, _byref(ni), _byref(no), None, None, None))
    w = max(k - 2, 1)
    G = np.zeros(max(ni.value * no.value, 1))
    li = np.zeros(max(ni.value * w, 1), dtype=np.int32)
    lo = np.zeros(max(no.value * w, 1), dtype=np.int32)
    L.check(L.lib.sym_su2_gamma(*args, None, None, G.ctypes.data_as(L._DP), li.ctypes.data_as(L._IP),
                                lo.ctypes.data_as(L._IP)))
    wk = max(k - 2, 0)
    return (G[:ni.value * no.value].reshape(no.value, ni.value),
            li[:ni.value * wk].reshape(ni.value, wk), lo[:no.value * wk].reshape(no.value, wk))


class SVDPlan:
    """Blockwise SVD of tensors with structure ``S``, rows = legs 0..nrow-1
    (include/symtensor.h, sym_svd_*; Ch. 5, Eq. svd0 and svd1)."""

    _plan_fn = "sym_svd_plan"

    def __init__(self, S, nrow):
        h, nb, ns = ctypes.c_void_p(), ctypes.c_int(), ctypes.c_int64()
        L.check(getattr(L.lib, self._plan_fn)(S._h, int(nrow), _byref(h), _byref(nb), _byref(ns)))
        self._h = h
        self.structure, self.nrow = S, int(nrow)
        self.nblocks, self.nsv = nb.value, ns.value
        x, m, n = [(ctypes.c_int * self.nblocks)() for _ in range(3)]
        L.check(L.lib.sym_svd_blocks(self._h, x, m, n))
        self.labels, self.m, self.n = list(x), list(m), list(n)
        self.full = [min(a, b) for a, b in zip(self.m, self.n)]
        self._bond = None

    def execute(self, data):
        """S (device, float64, nsv): every block's singular values, descending."""
        if data.dtype != torch.float64 or not data.is_cuda or data.numel() != self.structure.numel:
            raise TypeError("SVD input must be the tensor's float64 CUDA blocks")
        S = torch.empty(self.nsv, dtype=torch.float64, device=data.device)
        L.check(L.lib.sym_svd_execute(self._h, _ptr(data.contiguous()), _ptr(S), _stream()))
        return S

    def stats(self, fp32=False):
        """(sweeps, rotations) per block of the last execute, of its FP64
        sweeps or (fp32) of its FP32 sweeps (synchronizes)."""
        sw = (ctypes.c_int * self.nblocks)()
        rot = (ctypes.c_int64 * self.nblocks)()
        L.check(L.lib.sym_svd_stats(self._h, 1 if fp32 else 0, sw, rot))
        return list(sw), list(rot)

    def flops(self):
        """(FP64 flops, FP32 flops) of the last execute (synchronizes).

        Per sweep one FMA per row of every pair visited and the squared
        column norms (one FMA per element of W) when the kernel carries the
        norms through the rotations (blocks of at most 384 rows), else three
        FMAs per row of every pair visited; per rotation 4 multiply-adds per
        row of W and V; in FP64 also the two Newton-Schulz steps (2 C^3 FMAs
        each), W = A V (R C^2) and the column norms.  An FMA counts 2."""
        out = []
        for fp32 in (False, True):
            sweeps, rotations = self.stats(fp32)
            f = 0.0
            for m, n, sw, rot in zip(self.m, self.n, sweeps, rotations):
                R, C = max(m, n), min(m, n)
                if R <= 384:
                    f += sw * ((C * (C - 1) // 2) * 2.0 * R + 2.0 * R * C)
                else:
                    f += sw * (C * (C - 1) // 2) * 6.0 * R
                f += rot * 6.0 * (R + C)
                if not fp32:
                    f += 2.0 * (4.0 * C ** 3 + R * C * C + R * C)
            out.append(f)
        return tuple(out)

    def truncation(self, S_host, chi=None, cutoff=0.0):
        """keep per block (ascending x) for a host copy of execute's S."""
        S_host = np.ascontiguousarray(S_host, dtype=np.float64)
        keep = (ctypes.c_int * self.nblocks)()
        L.check(L.lib.sym_svd_truncation(self._h, S_host.ctypes.data_as(L._DP), -1 if chi is None else int(chi),
                                         float(cutoff), keep))
        return list(keep)

    def bond(self, keep):
        """(U structure, V structure) for ``keep`` vectors per block (cached for the last keep)."""
        keep = tuple(int(k) for k in keep)
        if self._bond is None or self._bond[0] != keep:
            u, v = ctypes.c_void_p(), ctypes.c_void_p()
            L.check(L.lib.sym_svd_bond(self._h, L.int_array(keep), _byref(u), _byref(v)))
            self._bond = (keep, Structure(self.structure.group, total=0, _handle=u),
                          Structure(self.structure.group, total=self.structure.total, _handle=v))
        return self._bond[1], self._bond[2]

    def factors(self, absorb=0):
        """(U data, V data, kept S) of the last execute for the last bond."""
        keep, Us, Vs = self._bond
        U = torch.empty(Us.numel, dtype=torch.float64, device="cuda")
        V = torch.empty(Vs.numel, dtype=torch.float64, device="cuda")
        Sk = torch.empty(sum(keep), dtype=torch.float64, device="cuda")
        L.check(L.lib.sym_svd_factors(self._h, int(absorb), _ptr(U), _ptr(V), _ptr(Sk), _stream()))
        return U, V, Sk

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and L is not None and L.lib is not None:
            L.lib.sym_svd_destroy(h)
            self._h = None


class EigPlan(SVDPlan):
    """Blockwise symmetric eigendecomposition of tensors with structure ``S``
    seen as a square matrix, rows = legs 0..nrow-1, columns = the row legs
    reversed (include/symtensor.h, sym_eig_*; Ch. 5, Eq. spectral by blocks).
    ``execute`` returns the eigenvalues (|lambda| descending per block);
    ``bond`` / ``factors`` give U (eigenvectors) and V (their transposes)."""

    _plan_fn = "sym_eig_plan"

    def execute(self, data):
        """lambda (device, float64, nev): every block's eigenvalues."""
        if data.dtype != torch.float64 or not data.is_cuda or data.numel() != self.structure.numel:
            raise TypeError("eigendecomposition input must be the tensor's float64 CUDA blocks")
        lam = torch.empty(self.nsv, dtype=torch.float64, device=data.device)
        L.check(L.lib.sym_eig_execute(self._h, _ptr(data.contiguous()), _ptr(lam), _stream()))
        return lam

    def truncation(self, lam_host, chi=None, cutoff=0.0):
        """keep per block (ascending x) for a host copy of execute's lambda (by |lambda|)."""
        lam_host = np.ascontiguousarray(lam_host, dtype=np.float64)
        keep = (ctypes.c_int * self.nblocks)()
        L.check(L.lib.sym_eig_truncation(self._h, lam_host.ctypes.data_as(L._DP), -1 if chi is None else int(chi),
                                         float(cutoff), keep))
        return list(keep)


_SVD_PLANS = {}


def eig_plan(S, nrow):
    """Eigendecomposition plan (cached) of structure S with rows = legs 0..nrow-1."""
    key = ("eig", id(S), int(nrow))
    hit = _SVD_PLANS.get(key)
    if hit is None or hit[1] is not S:
        hit = (EigPlan(S, nrow), S)
        _SVD_PLANS[key] = hit
    return hit[0]


def eig(T, nrow, chi=None, cutoff=0.0, absorb=0):
    """Blockwise eigendecomposition T = U diag(lambda) V of a symmetric float64
    tensor (rows = legs 0..nrow-1, columns = the row legs reversed; blocks
    taken as symmetric), truncated to the ``chi`` eigenvalues of largest
    magnitude above ``cutoff`` times the largest (include/symtensor.h,
    sym_eig_truncation).

    Returns (U, lambda, V): U has the row legs and an incoming bond leg (its
    columns are the eigenvectors), V an outgoing bond leg and the column
    legs, lambda the kept eigenvalues in bond order; absorb = 1 / 2 multiplies
    lambda into U / V.  Without chi or cutoff nothing is truncated and no host
    synchronisation happens.
    """
    plan = eig_plan(T.structure, nrow)
    lam = plan.execute(T.data)
    if chi is None and not cutoff:
        keep = plan.full
    else:
        keep = plan.truncation(lam.cpu().numpy(), chi, cutoff)
    Us, Vs = plan.bond(keep)
    U, V, Lk = plan.factors(absorb)
    return SymTensor(Us, U), Lk, SymTensor(Vs, V)


def svd_plan(S, nrow):
    """SVD plan (cached) of structure S with rows = legs 0..nrow-1."""
    key = (id(S), int(nrow))
    hit = _SVD_PLANS.get(key)
    if hit is None or hit[1] is not S:
        hit = (SVDPlan(S, nrow), S)
        _SVD_PLANS[key] = hit
    return hit[0]


def svd(T, nrow, chi=None, cutoff=0.0, absorb=0):
    """Blockwise SVD T = U diag(S) V of a float64 U(1) or fermion-parity tensor
    (rows = legs 0..nrow-1), truncated to the ``chi`` largest singular values
    above ``cutoff`` times the largest (include/symtensor.h, sym_svd_truncation).

    Returns (U, S, V): U has the row legs and an incoming bond leg, V an
    outgoing bond leg and the column legs, S the kept values in bond order;
    absorb = 1 / 2 multiplies S into U / V.  Without chi or cutoff nothing is
    truncated and no host synchronisation happens.
    """
    plan = svd_plan(T.structure, nrow)
    S = plan.execute(T.data)
    if chi is None and not cutoff:
        keep = plan.full
    else:
        keep = plan.truncation(S.cpu().numpy(), chi, cutoff)
    Us, Vs = plan.bond(keep)
    U, V, Sk = plan.factors(absorb)
    return SymTensor(Us, U), Sk, SymTensor(Vs, V)
