"""Big-means across GPUs: the exchange of the paper's parallel modes (Sec. 3.5)
between ranks, one process per GPU.

Each rank runs its own Big-means context on its own samples.  The only data
exchanged is the incumbent: every rank contributes (f_opt, rank) and the
winner -- lowest f_opt, lowest rank on ties -- broadcasts its centroids and
mask.  Competitive mode (mode 2) exchanges once, after the last round;
collective mode (mode 3) exchanges after every round and every rank continues
from the winner.  Host-side logic over ``torch.distributed`` (any backend);
the chunks themselves run in the CUDA library.
"""
import numpy as np
import torch
import torch.distributed as dist

COMPETITIVE = "competitive"
COLLECTIVE = "collective"


def exchange_best(f_opt, C, mask, group=None):
    """All ranks agree on the best incumbent.

    f_opt: this rank's incumbent objective (float; +inf if none);
    C: k x n float32 array, mask: k uint8 array (this rank's incumbent).
    Returns (winner rank, f_opt, C, mask) of the winner, identical on every
    rank.
    """
    world = dist.get_world_size(group)
    mine = torch.tensor([float(f_opt), float(dist.get_rank(group))], dtype=torch.float64)
    allv = [torch.zeros(2, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(allv, mine, group=group)
    pairs = [(float(v[0]), int(v[1])) for v in allv]
    f_best, winner = min(pairs)          # lowest f_opt, then lowest rank
    payload = torch.from_numpy(np.concatenate([np.asarray(C, np.float32).ravel(),
                                               np.asarray(mask, np.float32).ravel()]))
    dist.broadcast(payload, src=winner, group=group)
    k, n = np.asarray(C).shape
    out = payload.numpy()
    return winner, f_best, out[:k * n].reshape(k, n).copy(), out[k * n:].astype(np.uint8)


def fit_replicas(bm, ctx, k, n, rounds, chunks_per_round, mode=COLLECTIVE, group=None):
    """Big-means on every rank with the exchange of ``mode``.

    Rank r processes chunks t = (round * world + r) * chunks_per_round + q of
    its context's sequence, so ranks never draw the same sample.  Returns
    the final (f_opt, C, mask), identical on every rank.
    """
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    C = np.zeros((k, n), np.float32)
    mask = np.zeros(k, np.uint8)
    for r in range(rounds):
        f_opt, _ = bm.bm_get_state(ctx, C, mask)
        bm.bm_set_state(ctx, C, mask, f_opt, (r * world + rank) * chunks_per_round)
        bm.bm_fit_chunk(ctx, chunks_per_round)
        if mode == COLLECTIVE or r == rounds - 1:
            f_opt, _ = bm.bm_get_state(ctx, C, mask)
            _, f_best, C_best, mask_best = exchange_best(f_opt, C, mask, group)
            bm.bm_set_state(ctx, C_best, mask_best, f_best, (r + 1) * world * chunks_per_round)
    f_opt, _ = bm.bm_get_state(ctx, C, mask)
    return f_opt, C, mask
