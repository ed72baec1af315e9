"""Seeded synthetic spectrograms from the IS-NMF generative model.

This module only draws inputs; it holds none of the factorization's
arithmetic and is shared by the oracle tests, the GPU tests and the
benchmark. The paper's audio tracks (Section 3) are not available, so this
gamma model stands in for power spectrograms:

    W* ~ Gamma(1, 1)            F x K
    H* ~ Gamma(0.5, 1)          K x N, each entry zeroed with probability 0.7
    E  ~ Exp(1)                 F x N
    V  = (W* H*) o E + 1e-9

and the initial dictionary W0 ~ Gamma(1, 1), columns scaled to sum to 1.
Frames are generated in independent chunks (one counter-based Philox stream
per chunk), so any chunk of a long stream can be drawn on its own.

Host arrays use the frame-major memory order of the CUDA library: V is
returned with shape (N, F) (row n = frame n = column n of the F x N matrix),
W with shape (K, F) (row k = column k of the F x K matrix).
"""
import numpy as np

DATA_SEED = 1234
INIT_SEED = 5678
FLOOR = 1e-9
ZERO_PROB = 0.7
H_SHAPE = 0.5


def _rng(seed, stream):
    key = np.array([seed & (2**64 - 1), stream & (2**64 - 1)], dtype=np.uint64)
    return np.random.Generator(np.random.Philox(key=key))


def dictionary(F, K, seed=DATA_SEED):
    """The generating dictionary W*, shape (K, F), float64."""
    return _rng(seed, 2**63).gamma(1.0, 1.0, size=(K, F))


def activations(K, n, seed=DATA_SEED, chunk=0):
    """Sparse activations H* of one chunk, shape (n, K), float64."""
    rng = _rng(seed, 2 * chunk)
    h = rng.gamma(H_SHAPE, 1.0, size=(n, K))
    keep = rng.random(size=(n, K)) >= ZERO_PROB
    return h * keep


def frames(F, K, n, seed=DATA_SEED, chunk=0, Wstar=None):
    """n frames of V = (W* H*) o E + 1e-9 as float32, shape (n, F)."""
    if Wstar is None:
        Wstar = dictionary(F, K, seed)
    H = activations(K, n, seed, chunk)
    E = _rng(seed, 2 * chunk + 1).exponential(1.0, size=(n, F))
    V = (H @ Wstar) * E + FLOOR
    return V.astype(np.float32)


def spectrogram(F, K, N, seed=DATA_SEED, chunk_frames=65536):
    """A whole F x N spectrogram, shape (N, F), drawn chunk by chunk."""
    Wstar = dictionary(F, K, seed)
    out = np.empty((N, F), dtype=np.float32)
    for c, s in enumerate(range(0, N, chunk_frames)):
        n = min(chunk_frames, N - s)
        out[s:s + n] = frames(F, K, n, seed, c, Wstar)
    return out


def init_dictionary(F, K, seed=INIT_SEED):
    """W0 ~ Gamma(1, 1) with unit column sums, shape (K, F), float32."""
    W = _rng(seed, 0).gamma(1.0, 1.0, size=(K, F))
    W /= W.sum(axis=1, keepdims=True)
    return W.astype(np.float32)


def device_frames(F, K, n, seed=DATA_SEED, chunk=0, Wstar=None, out=None,
                  device="cuda"):
    """n frames of the same model drawn on the GPU with torch's Philox
    generator (a different stream from the host draw, same distribution).
    Returns (or fills) a float32 CUDA tensor of shape (n, F)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed((seed * 1000003 + chunk) & (2**63 - 1))
    if Wstar is None:
        Wstar = torch.as_tensor(dictionary(F, K, seed), dtype=torch.float32,
                                device=device)
    alpha = torch.full((n, K), H_SHAPE, device=device)
    H = torch._standard_gamma(alpha, generator=g)
    keep = torch.rand((n, K), device=device, generator=g) >= ZERO_PROB
    H = H * keep
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        V = H @ Wstar
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    E = torch.empty((n, F), device=device).exponential_(generator=g)
    V = V * E + FLOOR
    if out is not None:
        out.copy_(V)
        return out
    return V
