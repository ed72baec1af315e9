"""Shared helpers of the GPU tests (no arithmetic of the method here)."""
import numpy as np


def relerr(x, ref):
    """Norm-wise relative error ||x - ref||_F / ||ref||_F."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    d = np.linalg.norm((x - ref).ravel())
    n = np.linalg.norm(ref.ravel())
    return d / n if n > 0 else d


def cuda(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x)).cuda()


def problem(F, K, N, seed=1234):
    """Seeded gamma-model spectrogram V (N, F) and start dictionary W0 (K, F)."""
    import synth
    V = synth.spectrogram(F, K, N, seed=seed)
    W0 = synth.init_dictionary(F, K)
    return V, W0
