"""The seeded input generator (synth): deterministic per seed and chunk,
chunk-independent, and drawing the stated model: W* ~ Gamma(1,1),
H* ~ Gamma(0.5,1) with each entry zeroed with probability 0.7,
E ~ Exp(1), V = (W* H*) o E + 1e-9, W0 ~ Gamma(1,1) with unit column sums.
Statistical checks use bounds of several standard errors."""
import numpy as np

import synth


def test_deterministic_and_chunk_independent():
    F, K = 65, 7
    a = synth.spectrogram(F, K, 1000, chunk_frames=300)
    b = synth.spectrogram(F, K, 1000, chunk_frames=300)
    assert np.array_equal(a, b)
    # any chunk can be drawn on its own
    Wstar = synth.dictionary(F, K)
    c2 = synth.frames(F, K, 300, chunk=2, Wstar=Wstar)
    assert np.array_equal(a[600:900], c2)
    assert not np.array_equal(a[:300], a[300:600])
    assert not np.array_equal(a, synth.spectrogram(F, K, 1000, seed=99, chunk_frames=300))


def test_model_statistics():
    K, n = 20, 50_000
    H = synth.activations(K, n)
    nz = H > 0
    assert abs((~nz).mean() - synth.ZERO_PROB) < 0.005  # se ~ 0.0006
    assert abs(H[nz].mean() - synth.H_SHAPE) < 0.01     # Gamma(0.5, 1): mean 0.5, se ~ 0.002
    W = synth.dictionary(513, 100)
    assert abs(W.mean() - 1.0) < 0.02 and np.all(W > 0)  # Gamma(1, 1)
    F = 129
    V = synth.frames(F, K, 4000)
    assert V.dtype == np.float32 and V.shape == (4000, F)
    assert np.all(np.isfinite(V)) and np.all(V >= np.float32(synth.FLOOR))
    # E ~ Exp(1): V / (W* H*) has mean 1 where W* H* > 0 (floor negligible)
    Hs = synth.activations(K, 4000)
    X = Hs @ synth.dictionary(F, K)
    m = X > 1e-3
    ratio = (V.astype(np.float64)[m] - synth.FLOOR) / X[m]
    assert abs(ratio.mean() - 1.0) < 0.02


def test_initial_dictionary_columns_sum_to_one():
    W0 = synth.init_dictionary(513, 100)
    assert W0.shape == (100, 513) and W0.dtype == np.float32
    assert np.all(W0 > 0)
    assert np.max(np.abs(W0.astype(np.float64).sum(axis=1) - 1.0)) < 1e-5
