"""The identities behind two shortcuts of the CUDA path, checked on the CPU.

- Merge candidate search: the residual cut |trunc(n / d)| <= MC is decided as
  |n| < (MC + 1) |d| before any division (integers, d != 0, MC >= 0).
- Cross-sector pair search: for a symmetric positive definite M,
  d^T M^-1 d >= d_i^2 / M_ii for every component i, so a pair whose y or zeta
  residual alone gives d_i^2 > 4 cut M_ii has chi2 > cut and is dropped before
  the full 5x5 solve.
"""
import numpy as np


def _trunc_div(n, d):
    q = abs(n) // abs(d)
    return q if (n >= 0) == (d > 0) else -q


def test_division_free_cut_matches_truncated_quotient():
    rng = np.random.default_rng(7)
    cases = 0
    for mc in (0, 1, 7, 384, 16383):
        for _ in range(4000):
            d = int(rng.integers(1, 1 << 19)) * (1 if rng.random() < 0.5 else -1)
            # numerators near the cut's boundaries as well as anywhere
            k = int(rng.integers(-3, 4))
            n = (mc + 1) * abs(d) + k if rng.random() < 0.5 else int(rng.integers(-(1 << 40), 1 << 40))
            n = n if rng.random() < 0.5 else -n
            within = abs(n) < (mc + 1) * abs(d)
            assert within == (abs(_trunc_div(n, d)) <= mc), (n, d, mc)
            cases += 1
    assert cases == 20000


def test_residual_bound_never_exceeds_chi2():
    rng = np.random.default_rng(11)
    for _ in range(2000):
        a = rng.normal(size=(5, 5))
        # strongly correlated covariances, like fitted tracks'
        scales = 10.0 ** rng.uniform(-4, 1, size=5)
        m = (a @ a.T + 1e-6 * np.eye(5)) * np.outer(scales, scales)
        d = rng.normal(size=5) * np.sqrt(np.diag(m)) * rng.uniform(0.1, 20)
        chi2 = float(d @ np.linalg.solve(m, d))
        for i in range(5):
            assert d[i] ** 2 / m[i, i] <= chi2 * (1 + 1e-9) + 1e-12
