"""Shared helpers of the GPU parity tests: device transfers and the parity rules.

Parity rules (FP32 GPU path vs the FP64 oracle on the same draws):
  * labels equal, except rows whose oracle top-two squared distances differ by
    less than 1e-5 relative (d2 - d1 < 1e-5 * d2);
  * objectives (sample f, SSE) within 1e-6 relative;
  * centroids within 1e-6 relative, per centroid in the Euclidean norm:
    ||c_gpu - c_ref|| <= 1e-6 * max(||c_ref||, 1);
  * per-row squared distances within (n + 2) * 2^-24 relative, the rounding
    bound of an n-term FP32 sum of squared FP32 differences;
  * integer work (sample indices, gathered rows, K-means++ picks) bit-exact.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

TIE_REL = 1e-5
OBJ_REL = 1e-6
CEN_REL = 1e-6


def require_gpu():
    if not torch.cuda.is_available():
        pytest.fail("GPU test selected but no CUDA device is visible")


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to("cuda:0")


def host(t):
    return t.detach().cpu().numpy()


def labels_match(gpu_labels, ref_labels, d1, d2, rel=TIE_REL):
    gpu_labels = np.asarray(gpu_labels)
    ref_labels = np.asarray(ref_labels)
    tie = (d2 - d1) < rel * d2
    bad = (gpu_labels != ref_labels) & ~tie
    return int(bad.sum()), int(tie.sum())


def centroids_close(C_gpu, C_ref, live, rel=CEN_REL):
    C_gpu = np.asarray(C_gpu, dtype=np.float64)[live]
    C_ref = np.asarray(C_ref, dtype=np.float64)[live]
    err = np.linalg.norm(C_gpu - C_ref, axis=1)
    scale = np.maximum(np.linalg.norm(C_ref, axis=1), 1.0)
    return float((err / scale).max()) if len(err) else 0.0


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)
