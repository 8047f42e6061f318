"""Spawned host processes that evaluate the oracle's sampled elements of the
SU(2) recoupling contraction (test helper; imports numpy and oracle only, so
that the spawned interpreters start quickly and never touch CUDA).

The tensors are read from .npy files in a directory, memory-mapped, so that
the workers share the page cache instead of each receiving a copy."""
import multiprocessing as mp
import os

import numpy as np

_W = {}


def _init(dirname, c):
    from oracle import contract as oc
    from oracle import su2
    la = [su2.Leg(*l) for l in c["A"]]
    lb = [su2.Leg(*l) for l in c["B"]]
    lc = oc.result_legs(la, lb, c["pairsA"], c["pairsB"])
    arr = {n: np.load(os.path.join(dirname, n + ".npy"), mmap_mode="r") for n in ("A", "B", "G", "C", "dA", "dB")}
    comb, nodes_c = su2.left_comb(4), oc.comb_pair_tree(2, 2)
    _W.update(su2=su2, pa=c["pairsA"], pb=c["pairsB"], A=(la, comb, arr["A"]), B=(lb, comb, arr["B"]),
              G=(lc, nodes_c, arr["G"]), got={"C": (lc, nodes_c, arr["C"]), "dA": (la, comb, arr["dA"]),
                                              "dB": (lb, comb, arr["dB"])})


def _element(task):
    """(kind, oracle value, embedding of the tested result) at one index."""
    from oracle import sample
    kind, idx = task
    w = _W
    su2, A, B, G, pa, pb = w["su2"], w["A"], w["B"], w["G"], w["pa"], w["pb"]
    if kind == "C":
        ref = sample.contraction_element(su2, A, B, pa, pb, idx)
    elif kind == "dA":
        ref = sample.grad_a_element(su2, A, B, pa, pb, G, idx)
    else:
        ref = sample.grad_b_element(su2, A, B, pa, pb, G, idx)
    return kind, ref, sample.element(su2, w["got"][kind], idx)


def su2_elements(dirname, c, tasks, nproc=16, timeout=1200):
    """Evaluate tasks [(kind, idx)] with kind in C, dA, dB in a spawn pool;
    raises multiprocessing.TimeoutError after `timeout` seconds (a pool whose
    workers cannot start would otherwise wait for ever)."""
    nproc = max(1, min(nproc, os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(nproc, initializer=_init, initargs=(dirname, c)) as pool:
        return pool.map_async(_element, tasks, chunksize=4).get(timeout)
