"""The cross-rank exchange of the parallel modes (paper_2204_07485_gb300/replicas.py)
with two gloo ranks on the CPU.  The chunks run in a stand-in context that
applies the oracle's chunk (so no GPU is needed); the exchange is the real
code.  Both ranks must end with the same incumbent, equal to a sequential
simulation of the same rounds."""
import math
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import bminputs as bi
import oracle as o

M, N, K, S = 3000, 3, 5, 300


class OracleContext:
    """Stand-in for a Big-means context: the oracle's chunk on chunk draws t."""

    def __init__(self, X, seed):
        self.X, self.seed = X, seed
        self.st = o.BigMeansState(K, N)
        self.t = 0

    # the subset of the binding that replicas.fit_replicas uses
    def bm_get_state(self, ctx, C, mask):
        C[:] = self.st.C.astype(np.float32)
        mask[:] = self.st.live.astype(np.uint8)
        return self.st.f_opt, self.t

    def bm_set_state(self, ctx, C, mask, f_opt, t):
        self.st.C = np.asarray(C, np.float64).copy()
        self.st.live = np.asarray(mask).astype(bool)
        self.st.f_opt = f_opt
        self.t = t

    def bm_fit_chunk(self, ctx, chunks):
        for _ in range(chunks):
            idx, uf, u = bi.chunk_draws(self.seed, self.t, M, S, K)
            o.big_means_chunk(self.X, self.st, idx, uf, u, t=self.t)
            self.t += 1


def _data():
    X, _ = bi.mixtures.isotropic_blobs(M, N, 8, 21)
    return X


def _replicas_module():
    # by path: the exchange is host code and needs no compiled library
    import importlib.util
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location(
        "replicas", os.path.join(root, "paper_2204_07485_gb300", "replicas.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _rank_main(rank, world, port, mode, rounds, cpr, out):
    import torch.distributed as dist
    replicas = _replicas_module()
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port,
                            rank=rank, world_size=world)
    try:
        ctx = OracleContext(_data(), seed=3)
        f, C, mask = replicas.fit_replicas(ctx, None, K, N, rounds, cpr, mode)
        # ties: equal objectives go to the lowest rank
        w, fb, _, _ = replicas.exchange_best(1.0, np.zeros((2, 2), np.float32),
                                             np.zeros(2, np.uint8))
        out.put((rank, f, C, mask, w, fb))
    finally:
        dist.destroy_process_group()


def _sequential(mode, world, rounds, cpr):
    X = _data()
    ranks = [o.BigMeansState(K, N) for _ in range(world)]
    for r in range(rounds):
        for q in range(world):
            for c in range(cpr):
                t = (r * world + q) * cpr + c
                idx, uf, u = bi.chunk_draws(3, t, M, S, K)
                o.big_means_chunk(X, ranks[q], idx, uf, u, t=t)
        if mode == "collective" or r == rounds - 1:
            best = min(range(world), key=lambda q: (ranks[q].f_opt, q))
            win = ranks[best].copy()
            win.C = win.C.astype(np.float32).astype(np.float64)
            ranks = [win.copy() for _ in range(world)]
    return ranks[0]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


@pytest.mark.parametrize("mode", ["competitive", "collective"])
def test_two_gloo_ranks_agree_with_sequential_simulation(mode):
    world, rounds, cpr = 2, 3, 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, mode, rounds, cpr, out))
             for r in range(world)]
    for p in procs:
        p.start()
    res = sorted([out.get(timeout=120) for _ in range(world)], key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref = _sequential(mode, world, rounds, cpr)
    for rank, f, C, mask, w, fb in res:
        assert w == 0 and fb == 1.0                  # tie -> lowest rank
        assert f == res[0][1] and np.array_equal(C, res[0][2])
        assert np.array_equal(mask.astype(bool), ref.live)
        assert math.isclose(f, ref.f_opt, rel_tol=1e-12)
        np.testing.assert_array_equal(C, ref.C.astype(np.float32))
