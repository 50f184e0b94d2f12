"""Oracle: the error model of the AMA estimator (Sec. 2.1, eqs. ama1-ama3),
plain numpy FP64.

Test infrastructure only (see ``oracle/__init__``).

From measurements of one observable on n_conf configurations, with
Delta O = O - <O> and sigma = sqrt(<Delta O^2>) estimated by sample moments
over the configurations:

    sigma_AMA / sigma ~ sqrt(1/N_G + 2 Delta r + R)                    (ama1)
    Delta r = (1/N_org - 1/N_G) (1 - (1/N_org) sum_f
              <Delta O^f Delta O_appx^f> / (sigma^f sigma_appx^f))     (ama2)
    R = (1/N_G^2) sum_{g != g'} <Delta O_appx^g Delta O_appx^g'>
                                / (sigma_appx^g sigma_appx^g')         (ama3)

and, for comparison, the spread of the AMA estimate itself (eqs. caa1,
caa2) over the configurations relative to that of one exact measurement.
"""
from __future__ import annotations

import numpy as np


def _corr(a, b):
    """Sample correlation coefficient of two series (n_conf - 1 normalisation)."""
    da, db = a - a.mean(), b - b.mean()
    n = a.size - 1
    return (np.sum(da * db) / n) / np.sqrt((np.sum(da * da) / n) * (np.sum(db * db) / n))


def error_model(exact, appx_org, appx):
    """exact, appx_org: [n_conf, N_org]; appx: [n_conf, N_G].  Returns
    (Delta r, R, model sigma_AMA/sigma, measured sigma_AMA/sigma)."""
    exact, appx_org, appx = (np.asarray(x, dtype=np.float64) for x in (exact, appx_org, appx))
    n_org, n_g = exact.shape[1], appx.shape[1]
    rho = np.mean([_corr(exact[:, f], appx_org[:, f]) for f in range(n_org)])
    dr = (1.0 / n_org - 1.0 / n_g) * (1.0 - rho)
    R = sum(_corr(appx[:, g], appx[:, h]) for g in range(n_g) for h in range(n_g) if g != h) / n_g ** 2
    ama = np.mean(exact - appx_org, axis=1) + np.mean(appx, axis=1)
    measured = np.sqrt(np.var(ama, ddof=1) / np.mean(np.var(exact, axis=0, ddof=1)))
    return dr, R, np.sqrt(1.0 / n_g + 2.0 * dr + R), measured
