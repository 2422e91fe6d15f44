"""The distance-tile pipeline with resident operands (bm_tile_bench): its
checksum -- per row the argmin of ||c_j||^2 - 2 x.c_j and the count of ties
at the minimum, summed over rows, steps and CTAs -- must equal the exact
value computed here from the stated integer operand patterns, with and
without the split-BF16 planes (whose lo planes are zero here)."""
import numpy as np
import pytest

from gpu_helpers import require_gpu

pytestmark = pytest.mark.gpu


def _expected(n, k, tiles, steps, grid):
    r = np.arange(128)[:, None]
    f = np.arange(n)[None, :]
    B = ((np.arange(k)[:, None] * 11 + f * 13) % 7) - 3
    cc = (B * B).sum(axis=1)
    per_tile = []
    for t in range(tiles):
        A = ((r * 7 + f * 3 + t * 5) % 5) - 2
        D = cc[None, :] - 2 * (A @ B.T)
        j1 = D.argmin(axis=1)                         # lowest index on ties
        nc = (D == D.min(axis=1, keepdims=True)).sum(axis=1)
        per_tile.append(int(j1.sum() + 1024 * nc.sum()))
    total = sum(per_tile[s % tiles] for s in range(steps))
    return total * grid


@pytest.mark.parametrize("n,k,planes", [(64, 50, 1), (128, 50, 1), (128, 50, 2),
                                        (256, 33, 1), (192, 128, 1), (128, 7, 2)])
def test_tile_pipeline_checksum(n, k, planes):
    require_gpu()
    import paper_2204_07485_gb300 as bm
    steps = 37
    r = bm.bm_tile_bench(n, k, planes, steps, True)
    assert r["checksum"] == _expected(n, k, r["tiles"], steps, r["grid"])


def test_tile_pipeline_rejects_bad_shapes():
    require_gpu()
    import paper_2204_07485_gb300 as bm
    for args in [(100, 50, 1), (128, 0, 1), (128, 50, 3), (512, 50, 1)]:
        with pytest.raises(bm.BigMeansError) as e:
            bm.bm_tile_bench(*args, steps=4)
        assert e.value.status == bm.BM_EINVAL
