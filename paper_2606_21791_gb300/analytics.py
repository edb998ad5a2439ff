"""Campaign analytics on the engine's records (host side).

* Per-field severity (Table 2): footprint quantiles in percent of the frame,
  pooled over bits, and the catastrophe rate (Definition 2: non-finite, or a
  footprint above 1% of the frame averaged over the views) with a 95% Wilson
  score interval.
* Scaling law (Sec. 5 "A measured scaling law"): least-squares fit of
  log(error) = alpha log(N) + c, with its R^2, for the median and the mean
  single-upset error."""
import math

import numpy as np

# parameter fields by stored word (Sec. 3 "Parameter layout")
FIELDS = (("mean", range(0, 3)), ("log-scale", range(3, 6)), ("quat", range(6, 10)),
          ("opacity", range(10, 11)), ("color (DC)", range(11, 14)), ("color (SH)", range(14, 59)))
Z95 = 1.959963984540054   # two-sided 95% normal quantile


def wilson(k: int, n: int, z: float = Z95):
    """Wilson score interval (lo, hi) for k successes in n trials."""
    if n <= 0:
        return (0.0, 1.0)
    p = k / n
    den = 1.0 + z * z / n
    mid = (p + z * z / (2 * n)) / den
    half = z * math.sqrt(p * (1.0 - p) / n + z * z / (4.0 * n * n)) / den
    lo = 0.0 if k == 0 else max(0.0, mid - half)   # exactly 0 / 1 at the ends
    hi = 1.0 if k == n else min(1.0, mid + half)
    return (lo, hi)


def footprint_frac(records: np.ndarray, npix: int) -> np.ndarray:
    """Per variant: footprint averaged over the K views, as a fraction of the frame."""
    return records["footprint"].astype(np.float64).mean(axis=1) / npix


def catastrophic(records: np.ndarray, npix: int, threshold: float = 0.01) -> np.ndarray:
    """Definition 2 per variant: a non-finite pixel in any view, or a footprint
    above `threshold` of the frame (averaged over the views)."""
    return (records["nonfinite"] > 0).any(axis=1) | (footprint_frac(records, npix) > threshold)


def severity_table(flips: np.ndarray, records: np.ndarray, npix: int) -> dict:
    """Table 2: per field, footprint quantiles (% of frame) and the catastrophe
    rate (%) with its 95% Wilson interval."""
    fp = 100.0 * footprint_frac(records, npix)
    cat = catastrophic(records, npix)
    out = {}
    for name, words in FIELDS:
        sel = np.isin(flips["word"], list(words))
        n = int(sel.sum())
        if n == 0:
            continue
        k = int(cat[sel].sum())
        lo, hi = wilson(k, n)
        f = fp[sel]
        out[name] = {"n": n, "median": float(np.median(f)), "p95": float(np.percentile(f, 95)),
                     "p99": float(np.percentile(f, 99)), "max": float(f.max()), "mean": float(f.mean()),
                     "catastrophe_pct": 100.0 * k / n, "ci95_pct": [100.0 * lo, 100.0 * hi]}
    return out


def loglog_fit(x, y):
    """Least squares of log(y) = alpha log(x) + c over the points with y > 0:
    returns (alpha, c, r2)."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    m = (x > 0) & (y > 0)
    lx, ly = np.log(x[m]), np.log(y[m])
    A = np.stack([lx, np.ones_like(lx)], axis=1)
    (alpha, c), *_ = np.linalg.lstsq(A, ly, rcond=None)
    pred = alpha * lx + c
    ss_res = float(((ly - pred) ** 2).sum())
    ss_tot = float(((ly - ly.mean()) ** 2).sum())
    return float(alpha), float(c), (1.0 - ss_res / ss_tot) if ss_tot > 0 else 1.0
