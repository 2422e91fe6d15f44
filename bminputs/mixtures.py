"""Seeded Gaussian-mixture datasets shaped like the paper's workloads.

The paper evaluates on public datasets (Table 1: e.g. HEPMASS with n = 28,
Gas Sensor Array Drift with n = 128) that are not available here; these
synthetic mixtures stand in for them with the same m, n, k ranges.  Every
generator is a pure function of its arguments and seed (numpy PCG64), emits
float32 row-major data and holds no clustering arithmetic.
"""
import numpy as np


def _weights(rng, comps, alpha):
    if alpha is None:
        return np.full(comps, 1.0 / comps)
    return rng.dirichlet(np.full(comps, float(alpha)))


def _haar_orthogonal(rng, n):
    """Haar-distributed orthogonal matrix (QR of a Gaussian, sign-fixed)."""
    a = rng.standard_normal((n, n))
    q, r = np.linalg.qr(a)
    return q * np.sign(np.diag(r))


def isotropic_blobs(m, n, comps, seed, sigma=1.0, box=10.0, alpha=None,
                    feature_scale=None, block=1 << 20):
    """m points from ``comps`` isotropic Gaussians, means U[-box, box]^n.

    alpha=None gives equal weights, otherwise Dirichlet(alpha) weights.
    ``feature_scale`` (optional length-n vector) multiplies every feature.
    Returns (X float32 m x n, component id int32 m).
    """
    rng = np.random.default_rng(seed)
    means = rng.uniform(-box, box, size=(comps, n))
    w = _weights(rng, comps, alpha)
    comp = rng.choice(comps, size=m, p=w).astype(np.int32)
    X = np.empty((m, n), dtype=np.float32)
    for a in range(0, m, block):
        b = min(m, a + block)
        z = rng.standard_normal((b - a, n), dtype=np.float32)
        blk = means[comp[a:b]].astype(np.float32) + np.float32(sigma) * z
        if feature_scale is not None:
            blk *= np.asarray(feature_scale, dtype=np.float32)
        X[a:b] = blk
    return X, comp


def anisotropic_with_outliers(m, n, comps, seed, box=10.0, alpha=1.0,
                              eig_lo=0.1, eig_hi=10.0, outlier_frac=0.01,
                              block=1 << 20):
    """Anisotropic mixture plus uniform outliers (the m = 1e6, n = 28 workload).

    Component c has mean U[-box, box]^n and covariance Q diag(lam) Q^T with
    Haar Q and lam log-uniform in [eig_lo, eig_hi]; weights Dirichlet(alpha).
    A fraction ``outlier_frac`` of the rows is replaced by points uniform in
    the bounding box of the inliers.  Returns (X float32, component id, -1 for
    outliers).
    """
    rng = np.random.default_rng(seed)
    means = rng.uniform(-box, box, size=(comps, n))
    lam = np.exp(rng.uniform(np.log(eig_lo), np.log(eig_hi), size=(comps, n)))
    factors = np.empty((comps, n, n))
    for c in range(comps):
        q = _haar_orthogonal(rng, n)
        factors[c] = q * np.sqrt(lam[c])          # Q diag(sqrt(lam))
    w = _weights(rng, comps, alpha)
    comp = rng.choice(comps, size=m, p=w).astype(np.int32)
    X = np.empty((m, n), dtype=np.float32)
    for a in range(0, m, block):
        b = min(m, a + block)
        z = rng.standard_normal((b - a, n))
        cc = comp[a:b]
        y = np.einsum("rij,rj->ri", factors[cc], z) + means[cc]
        X[a:b] = y.astype(np.float32)
    n_out = int(round(outlier_frac * m))
    if n_out:
        lo, hi = X.min(axis=0), X.max(axis=0)
        rows = rng.choice(m, size=n_out, replace=False)
        X[rows] = rng.uniform(lo, hi, size=(n_out, n)).astype(np.float32)
        comp[rows] = -1
    return X, comp


# ---- the workloads, by name -------------------------------------------------

def blobs_2d(seed=0, m=20_000):
    """m = 20,000, n = 2, ten equal-weight isotropic blobs, sigma 1 (k = 10)."""
    return isotropic_blobs(m, 2, 10, seed)[0]


def hepmass_like(seed=0, m=1_000_000):
    """m = 1e6, n = 28, 50 anisotropic components + 1 % outliers (k = 25)."""
    return anisotropic_with_outliers(m, 28, 50, seed)[0]


def gas_sensor_like(seed=0, m=10_000_000, n=128):
    """m = 1e7, n = 128, 100 isotropic components, Dirichlet(0.5) (k = 50)."""
    return isotropic_blobs(m, n, 100, seed, alpha=0.5)[0]


def scaled_384(seed=0, m=2_000_000):
    """m = 2e6, n = 384, 100 components, per-feature scales log-U[0.1, 10] (k = 100)."""
    rng = np.random.default_rng(seed + 7919)
    scale = np.exp(rng.uniform(np.log(0.1), np.log(10.0), size=384))
    return isotropic_blobs(m, 384, 100, seed, alpha=0.5, feature_scale=scale)[0]


def isotropic_blobs_device(m, n, comps, seed, sigma=1.0, box=10.0, alpha=None,
                           device="cuda", feature_scale=None):
    """isotropic_blobs generated on a CUDA device (for workloads of several GB).

    Means and weights come from numpy PCG64(seed) as in isotropic_blobs; the
    component ids and the Gaussian noise come from torch's CUDA generator
    seeded with `seed`, so the data is a deterministic function of the seed
    (but not the same numbers as isotropic_blobs).  Returns a float32 torch
    tensor on `device`.
    """
    import torch
    rng = np.random.default_rng(seed)
    means = rng.uniform(-box, box, size=(comps, n))
    w = _weights(rng, comps, alpha)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    mu = torch.tensor(means, dtype=torch.float32, device=device)
    probs = torch.tensor(w, dtype=torch.float32, device=device)
    X = torch.empty((m, n), dtype=torch.float32, device=device)
    block = 1 << 21
    for a in range(0, m, block):
        b = min(m, a + block)
        comp = torch.multinomial(probs, b - a, replacement=True, generator=g)
        X[a:b] = mu[comp] + sigma * torch.randn((b - a, n), generator=g, device=device)
    if feature_scale is not None:
        X *= torch.tensor(np.asarray(feature_scale), dtype=torch.float32, device=device)
    return X


def scaled_384_device(seed=0, m=2_000_000, device="cuda"):
    """scaled_384 generated on a CUDA device (same scales and mixture law)."""
    rng = np.random.default_rng(seed + 7919)
    scale = np.exp(rng.uniform(np.log(0.1), np.log(10.0), size=384))
    return isotropic_blobs_device(m, 384, 100, seed, alpha=0.5, device=device,
                                  feature_scale=scale)


def gas_sensor_like_device(seed=0, m=10_000_000, n=128, device="cuda"):
    """m = 1e7, n = 128, 100 isotropic components, Dirichlet(0.5) (k = 50), on device."""
    return isotropic_blobs_device(m, n, 100, seed, alpha=0.5, device=device)


def grouped_chunks_spec(seed=0, count=256):
    """Shapes of `count` independent chunks for the grouped Lloyd workload:
    s ~ U[4000, 64000], n ~ U{16, 32, 64, 128}, k ~ U{5, 10, 25, 50}.  Chunk i
    is a mixture of k_i isotropic components (sigma 1, means U[-10, 10]^n)
    drawn with seed i.  Returns a list of dicts (s, n, k, seed)."""
    rng = np.random.default_rng(seed)
    s = rng.integers(4000, 64001, size=count)
    n = rng.choice([16, 32, 64, 128], size=count)
    k = rng.choice([5, 10, 25, 50], size=count)
    return [dict(s=int(s[i]), n=int(n[i]), k=int(k[i]), seed=i) for i in range(count)]


def forgy_rows(s, k, seed):
    """k distinct row indices of an s-row chunk (a seeded Forgy start), ascending."""
    rng = np.random.default_rng(10_000 + seed)
    return np.sort(rng.choice(s, size=k, replace=False))
