"""GPU parity of the grouped Lloyd launches (many independent Lloyd problems
advanced together, Sec. 2 with the stop rule of Sec. 5).

Every problem of a group must end where the oracle's Lloyd ends from the same
start: the same number of update steps, the same live set, objectives and
centroids within 1e-6 relative, labels equal except at exempt near-ties.
Cases are decisive (asserted from the oracle's own record).  The same
problems run alone through bm_lloyd must take the same decisions, and a
group's results must not depend on anything but its inputs.
"""
import numpy as np
import pytest

import bminputs as bi
import oracle as o
from gpu_helpers import (CEN_REL, OBJ_REL, centroids_close, dev, host, labels_match, rel,
                         require_gpu, torch)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bm():
    require_gpu()
    import paper_2204_07485_gb300 as lib
    return lib


# (s, n, k, components, seed): n spans the 4-aligned and ragged cases, k the
# one-group and two-group tables, s the one-tile and ragged-tail cases
SHAPES = [(3000, 16, 5, 8, 0), (5000, 32, 10, 14, 1), (2000, 64, 25, 30, 2),
          (4100, 128, 50, 60, 3), (700, 28, 7, 9, 4), (1500, 3, 2, 3, 5), (64, 5, 1, 2, 6),
          (2345, 33, 12, 15, 7)]


def _problem(s, n, k, comps, seed):
    P, _ = bi.mixtures.isotropic_blobs(s, n, comps, seed, box=8.0)
    rng = np.random.default_rng(1000 + seed)
    rows = rng.choice(s, size=k, replace=False)
    C0 = P[np.sort(rows)].astype(np.float32)
    return P, C0


def _oracle(P, C0, max_iter=300):
    res = o.lloyd(P, C0.astype(np.float64), np.ones(C0.shape[0], bool), max_iter=max_iter)
    assert res.min_gap >= 1e-5, "not decisive: near-tie in the oracle's assignments"
    assert res.stop_margin >= 1e-6, "not decisive: objective near the stop threshold"
    return res


def _group(bm, probs, balance=True, max_iter=300, stream="own", tiles=None, shapes_out=None):
    """probs: list of (P, C0); returns per problem (result, C, mask, labels), steps.
    tiles: tile-shape mode (None: the default autotuning); shapes_out (list)
    receives the shape each problem ran with."""
    specs, keep = [], []
    for P, C0 in probs:
        s, n = P.shape
        k = C0.shape[0]
        Pd, Cd = dev(P), dev(C0)
        md = torch.ones(k, dtype=torch.uint8, device="cuda:0")
        ld = torch.full((s,), -1, dtype=torch.int32, device="cuda:0")
        specs.append(dict(P=Pd, s=s, n=n, k=k, C=Cd, mask=md, labels=ld))
        keep.append((Pd, Cd, md, ld))
    torch.cuda.synchronize()   # the inputs are on the device before the group's stream reads them
    if stream == "own":
        stream = torch.cuda.Stream()
    g = bm.bm_group_create(specs, max_iter=max_iter, balance=balance, stream=stream)
    try:
        if tiles is not None:
            bm.bm_group_set_tiles(g, tiles)
        res, steps = bm.bm_group_run(g, len(specs))
        info = bm.bm_group_info(g)
        if shapes_out is not None:
            shapes_out.extend(bm.bm_group_tiles(g, len(specs)))
    finally:
        bm.bm_group_destroy(g)
    out = [(r, host(C), host(m).astype(bool), host(l)) for r, (_, C, m, l) in zip(res, keep)]
    return out, steps, info


def _check_against_oracle(P, res_o, r, C, mask, labels):
    assert r["iters"] == res_o.iters
    assert np.array_equal(mask, res_o.live)
    assert r["live"] == int(res_o.live.sum())
    assert r["n_d"] == res_o.n_d
    assert rel(r["f"], res_o.f) <= OBJ_REL
    assert centroids_close(C, res_o.C, res_o.live) <= CEN_REL
    A, _, d1, d2 = o.final_assignment(P, res_o.C.astype(np.float32), res_o.live)
    bad, _ = labels_match(labels, A, d1, d2)
    assert bad == 0


def test_group_matches_oracle_per_problem(bm):
    probs = [_problem(*sh) for sh in SHAPES]
    refs = [_oracle(P, C0) for P, C0 in probs]
    out, steps, info = _group(bm, probs, stream="own")
    assert steps >= max(r.iters for r in refs) + 1
    assert info["segments"] >= len(probs)
    for (P, _), ro, (r, C, mask, labels) in zip(probs, refs, out):
        _check_against_oracle(P, ro, r, C, mask, labels)


def test_one_cta_per_problem_takes_the_same_decisions(bm):
    probs = [_problem(*sh) for sh in SHAPES[:5]]
    a, _, ia = _group(bm, probs, balance=True)
    b, _, ib = _group(bm, probs, balance=False)
    assert ib["grid"] == len(probs) and ib["segments"] == len(probs)
    for (ra, Ca, ma, la), (rb, Cb, mb, lb) in zip(a, b):
        assert ra["iters"] == rb["iters"] and np.array_equal(ma, mb)
        assert rel(ra["f"], rb["f"]) <= OBJ_REL
        assert centroids_close(Ca, Cb.astype(np.float64), ma) <= CEN_REL


def test_group_is_bitwise_reproducible(bm):
    probs = [_problem(*sh) for sh in SHAPES]
    a, _, _ = _group(bm, probs, stream="own")
    b, _, _ = _group(bm, probs, stream="own")
    for (ra, Ca, ma, la), (rb, Cb, mb, lb) in zip(a, b):
        assert ra == rb
        assert np.array_equal(Ca, Cb) and np.array_equal(ma, mb) and np.array_equal(la, lb)


def test_group_equals_problems_run_alone(bm):
    probs = [_problem(*sh) for sh in SHAPES[:4]]
    out, _, _ = _group(bm, probs)
    for (P, C0), (r, C, mask, _) in zip(probs, out):
        s, n = P.shape
        k = C0.shape[0]
        Cd = dev(C0)
        md = torch.ones(k, dtype=torch.uint8, device="cuda:0")
        f, iters = bm.bm_lloyd(dev(P), s, n, k, Cd, md)
        assert iters == r["iters"]
        assert np.array_equal(host(md).astype(bool), mask)
        assert rel(f, r["f"]) <= OBJ_REL
        assert centroids_close(C, host(Cd).astype(np.float64), mask) <= CEN_REL


def test_emptied_cluster_becomes_degenerate(bm):
    # a start centroid far from every row loses all members at the first
    # assignment and leaves the live set (Sec. 3.3)
    P, C0 = _problem(2000, 16, 6, 6, 11)
    C0[2] = 1e3
    ro = _oracle(P, C0)
    assert not ro.live[2]
    (r, C, mask, labels), = _group(bm, [(P, C0)])[0]
    _check_against_oracle(P, ro, r, C, mask, labels)


def test_iteration_cap(bm):
    probs = [_problem(*sh) for sh in SHAPES[:3]]
    refs = [o.lloyd(P, C0.astype(np.float64), np.ones(C0.shape[0], bool), max_iter=2)
            for P, C0 in probs]
    out, steps, _ = _group(bm, probs, max_iter=2)
    assert steps <= 2 + 3
    for ro, (r, C, mask, _) in zip(refs, out):
        assert r["iters"] == ro.iters <= 2
        assert rel(r["f"], ro.f) <= OBJ_REL
        assert centroids_close(C, ro.C, ro.live) <= CEN_REL


def test_legacy_stream_without_graphs(bm):
    probs = [_problem(*sh) for sh in SHAPES[5:]]
    refs = [_oracle(P, C0) for P, C0 in probs]
    out, _, _ = _group(bm, probs, stream=None)
    for (P, _), ro, (r, C, mask, labels) in zip(probs, refs, out):
        _check_against_oracle(P, ro, r, C, mask, labels)


def test_tile_shapes_give_the_same_bits(bm):
    """A lane per centroid, four lanes per row (k <= 16) and the autotuned
    choice: every problem's result identical bit for bit, and the oracle's."""
    shapes = [(3000, 16, 5, 8, 0), (5000, 32, 10, 14, 1), (2345, 33, 12, 15, 7),
              (1500, 3, 2, 3, 5), (4100, 64, 16, 20, 9), (2000, 64, 25, 30, 2)]
    probs = [_problem(*sh) for sh in shapes]
    refs = [_oracle(P, C0) for P, C0 in probs]
    runs, used = [], []
    for mode in (1, 2, 0):
        got = []
        out, steps, _ = _group(bm, probs, tiles=mode, shapes_out=got)
        runs.append(out)
        used.append(got)
    assert used[0] == [0] * len(shapes)
    assert used[1] == [1 if sh[2] <= 16 else 0 for sh in shapes]
    assert all(u == 0 or sh[2] <= 16 for u, sh in zip(used[2], shapes))
    for a, b in ((runs[0], runs[1]), (runs[0], runs[2])):
        for (ra, Ca, ma, la), (rb, Cb, mb, lb) in zip(a, b):
            assert ra == rb
            assert np.array_equal(Ca, Cb) and np.array_equal(ma, mb) and np.array_equal(la, lb)
    for (P, _), res_o, (r, C, mask, labels) in zip(probs, refs, runs[1]):
        _check_against_oracle(P, res_o, r, C, mask, labels)
