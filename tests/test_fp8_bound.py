"""The E4M3 screening bound of the tensor-core chunk kernel, checked on the
CPU against an independent E4M3 rounding (torch.float8_e4m3fn).

The kernel scales row x by 2^(7 - e_x) with 2^e_x <= max|x_f| < 2^(e_x + 1),
and every centroid of a chunk by cs = 2^(7 - e_M) with M >= every |c_f|,
rounds both to E4M3 and accumulates the products.  Its candidate rule
assumes, before accumulation error,

  |x~ . c~ - x . c| <= ||x|| ||c|| (2^-3 + 2^-8 + 1.07 2^-17 sqrt n)
                     + ||x|| M (1.07 2^-17 sqrt n + n 2^-34).

Adversarial inputs: midpoint mantissas (every operand rounds by almost
2^-4 in the same direction, so the relative term is nearly reached),
features down in the subnormal range of the row's scale, and a centroid
scale set by a value far larger than the centroid itself.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not hasattr(torch, "float8_e4m3fn"):
    pytest.skip("no float8_e4m3fn in this torch", allow_module_level=True)


def e4m3(v):
    return torch.from_numpy(np.asarray(v, np.float32)).to(torch.float8_e4m3fn) \
        .to(torch.float64).numpy()


def floor_log2(v):
    _, e = np.frexp(v)   # v = m 2^e, m in [0.5, 1)
    return e - 1


def quant_rows(X):
    mx = np.abs(X).max(axis=1)
    e = np.where(mx > 0, floor_log2(np.where(mx > 0, mx, 1.0)), 7)
    inv = np.ldexp(1.0, e - 7)[:, None]
    return e4m3(X / inv) * inv


def quant_cents(C, M):
    e = floor_log2(M) if M > 0 else 7
    cs = math.ldexp(1.0, 7 - int(e))
    return e4m3(C * cs) / cs


def bound(X, C, M):
    n = X.shape[1]
    nx = np.sqrt((X.astype(np.float64) ** 2).sum(1))[:, None]
    nc = np.sqrt((C.astype(np.float64) ** 2).sum(1))[None, :]
    rn = math.sqrt(n)
    return nx * nc * (2.0 ** -3 + 2.0 ** -8 + 1.07 * 2.0 ** -17 * rn) + \
        nx * M * (1.07 * 2.0 ** -17 * rn + n * 2.0 ** -34)


def errors(X, C, M):
    Xq = quant_rows(X)
    Cq = quant_cents(C, M)
    exact = X.astype(np.float64) @ C.astype(np.float64).T
    return np.abs(Xq @ Cq.T - exact), bound(X, C, M)


def test_e4m3_rounding_reference():
    # the rounding the test relies on: 3 mantissa bits, nearest-even, the
    # subnormal spacing 2^-9 below 2^-6, 448 the largest finite value
    assert e4m3([1.0625, 1.1875, 448.0, 2.0 ** -9, 3 * 2.0 ** -10]).tolist() == \
        [1.0, 1.25, 448.0, 2.0 ** -9, 2.0 ** -8]


@pytest.mark.parametrize("n", [33, 128, 384, 512])
def test_bound_holds_on_wide_magnitude_data(n):
    rng = np.random.default_rng(n)
    X = (rng.choice([-1.0, 1.0], (400, n)) *
         np.exp2(rng.uniform(-30, 10, (400, n)))).astype(np.float32)
    C = (rng.choice([-1.0, 1.0], (50, n)) *
         np.exp2(rng.uniform(-30, 10, (50, n)))).astype(np.float32)
    M = float(max(np.abs(X).max(), np.abs(C).max()))
    err, b = errors(X, C, M)
    assert (err <= b).all()


@pytest.mark.parametrize("n", [64, 384])
def test_relative_term_is_nearly_reached(n):
    # every feature at the midpoint 1.0625 rounds down to 1.0 (ties to even):
    # the product error is 2 * 0.0625 / 1.0625 + (0.0625 / 1.0625)^2 of ||x|| ||c||
    X = np.full((4, n), 1.0625, np.float32)   # scaled by 2^7: 136, halfway from 128 to 144
    C = np.full((3, n), 1.0625, np.float32)
    M = 1.0625
    err, b = errors(X, C, M)
    assert (err <= b).all()
    assert (err / b).min() > 0.85


def test_subnormal_features_and_a_far_scale():
    # one large feature per row puts the others below the row's normal range;
    # a far value M leaves the centroid down in the subnormal range
    rng = np.random.default_rng(7)
    n = 384
    X = rng.uniform(-1, 1, (300, n)).astype(np.float32) * np.float32(2.0 ** -12)
    X[:, 0] = 100.0
    C = rng.uniform(-1, 1, (40, n)).astype(np.float32)
    for M in (1.0, 2.0 ** 10, 2.0 ** 20):
        err, b = errors(X, C, M)
        assert (err <= b).all()
    # aligned rows and centroids flushed to zero by a far scale: the whole
    # dot product is lost, and only the M term covers it
    X = np.ones((2, n), np.float32)
    C = np.ones((2, n), np.float32)
    err, b = errors(X, C, 2.0 ** 20)
    assert (err <= b).all()
    rel_only = n * (2.0 ** -3 + 2.0 ** -8 + 1.07 * 2.0 ** -17 * math.sqrt(n))
    assert (err == n).all() and (err > rel_only).all()
