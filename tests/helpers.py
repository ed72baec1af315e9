"""Shared helpers of the GPU tests (no arithmetic of the method here).

Parity measures (x: GPU result, ref: FP64 oracle, same shape):
  relerr     norm-wise  ||x - ref||_F / ||ref||_F
  entry_err  element-wise  max_i |x_i - ref_i| / (|ref_i| + FLOOR * mean|ref|):
             every entry is checked; the floor (a thousandth of the mean
             magnitude) keeps entries that are zero to rounding from
             dividing by zero, and nothing else
  row_errs   per frequency row f of an F x K matrix held as (K, F) (W, A, B):
             ||x[:, f] - ref[:, f]|| / ||ref[:, f]||, so that one wrong row
             (the F = 2^n + 1 tail row, a masked pad row) cannot hide in the
             norm of the others; the last row f = F - 1 is reported on its own
"""
import numpy as np

FLOOR = 1e-3


def relerr(x, ref):
    """Norm-wise relative error ||x - ref||_F / ||ref||_F."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    d = np.linalg.norm((x - ref).ravel())
    n = np.linalg.norm(ref.ravel())
    return d / n if n > 0 else d


def entry_err(x, ref, floor=FLOOR):
    """Largest element-wise relative error with an absolute floor of
    floor * mean|ref|."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if ref.size == 0:
        return 0.0
    scale = np.abs(ref) + floor * np.mean(np.abs(ref))
    d = np.abs(x - ref)
    with np.errstate(invalid="ignore", divide="ignore"):
        r = np.where(scale > 0, d / np.where(scale > 0, scale, 1.0), d)
    r = np.where(np.isfinite(r), r, np.inf)
    return float(np.max(r))


def row_errs(x, ref):
    """Per-frequency-row relative errors of (K, F) arrays: one value per f."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    d = np.linalg.norm(x - ref, axis=0)
    n = np.linalg.norm(ref, axis=0)
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.where(n > 0, d / np.where(n > 0, n, 1.0), d)


def parity(label, pairs, tol, rows=("W", "A", "B"), print_only=False):
    """Check GPU results against the oracle entry by entry and, for the
    F x K matrices named in `rows`, row by row with the last row on its own.

    pairs: {name: (x, ref)}; tol: one bound for all, or {name: bound} (a name
    missing from the dict is reported but not bounded). Scalars (the loss)
    are compared as relative differences. Returns the measured errors."""
    out = {}
    for name, (x, ref) in pairs.items():
        bound = tol.get(name) if isinstance(tol, dict) else tol
        if np.ndim(ref) == 0:
            e = abs(float(x) - float(ref)) / max(abs(float(ref)), 1e-300)
            out[name] = dict(rel=e)
            ok = bound is None or e <= bound
            assert print_only or ok, (label, name, e, bound)
            continue
        m = dict(norm=relerr(x, ref), entry=entry_err(x, ref))
        if name in rows:
            r = row_errs(x, ref)
            m["row_max"] = float(np.max(r))
            m["row_argmax"] = int(np.argmax(r))
            m["row_last"] = float(r[-1])
        out[name] = m
    line = "; ".join(
        "%s %s" % (k, " ".join("%s=%.2e" % (a, b) if isinstance(b, float) else "%s=%d" % (a, b)
                               for a, b in v.items()))
        for k, v in out.items())
    print("[parity] %s: %s" % (label, line))
    if print_only:
        return out
    for name, m in out.items():
        bound = tol.get(name) if isinstance(tol, dict) else tol
        if bound is None or "rel" in m:
            continue
        assert m["entry"] <= bound, (label, name, "entry", m)
        if "row_max" in m:
            assert m["row_max"] <= bound, (label, name, "row", m)
            assert m["row_last"] <= bound, (label, name, "last row f = F-1", m)
    return out


def cuda(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x)).cuda()


def problem(F, K, N, seed=1234):
    """Seeded gamma-model spectrogram V (N, F) and start dictionary W0 (K, F)."""
    import synth
    V = synth.spectrogram(F, K, N, seed=seed)
    W0 = synth.init_dictionary(F, K)
    return V, W0
