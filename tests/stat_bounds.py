"""Acceptance thresholds of the statistical pins.

A single observable is accepted within 3 standard errors (the acceptance the
method's exact-mean check uses).  A check over m elements of a density at
once takes the Bonferroni threshold for a family-wise false-alarm rate alpha:
each element's z = (mean - exact) / (s / sqrt(V)) follows Student's t with
V - 1 degrees of freedom (the standard error is estimated from the same V
vectors), so the threshold is the t quantile at 1 - alpha / (2 m).
"""
from scipy import stats

SINGLE = 3.0


def familywise(m: int, vectors: int, alpha: float = 1e-3) -> float:
    """Largest |z| accepted over m elements whose standard errors come from
    `vectors` independent vectors."""
    m = max(1, int(m))
    return float(stats.t.ppf(1.0 - alpha / (2.0 * m), vectors - 1))
