"""Fits of a bubble-size sweep to the functional forms of Fig. 3 (Sec. 4).

The paper fits its two-bubble runs with a quadratic critical film thickness
in the film-disc radius, h_c = a R_d^2 + b R_d + c, and a disc radius
logarithmic in the bubble radius, R_d = alpha ln(R_b) + beta (its
coefficients are in its own units).  ``fit_fig3`` fits the same forms by
least squares to the rows of a sweep (lbm.Ensemble results of the domains
whose criterion fired), so the trend of a sweep can be set beside the
paper's.
"""
from __future__ import annotations

import numpy as np


def fit_fig3(R_b, R_d, h_c):
    """Least-squares fits of h_c(R_d) (quadratic) and R_d(ln R_b) (linear)
    with their coefficients of determination, and the Pearson correlation
    of h_c with R_d.  Needs at least three rows."""
    R_b, R_d, h_c = (np.asarray(v, dtype=float) for v in (R_b, R_d, h_c))
    if len(h_c) < 3:
        raise ValueError("at least three fired domains are needed")

    def r2(y, yhat):
        ss = float(((y - y.mean()) ** 2).sum())
        return 1.0 - float(((y - yhat) ** 2).sum()) / ss if ss > 0 else 1.0

    q = np.polyfit(R_d, h_c, 2)
    lin = np.polyfit(np.log(R_b), R_d, 1)
    corr = float(np.corrcoef(R_d, h_c)[0, 1]) if R_d.std() > 0 and h_c.std() > 0 else 0.0
    return {"h_c_vs_R_d": {"a": float(q[0]), "b": float(q[1]), "c": float(q[2]),
                           "r2": r2(h_c, np.polyval(q, R_d))},
            "R_d_vs_ln_R_b": {"alpha": float(lin[0]), "beta": float(lin[1]),
                              "r2": r2(R_d, np.polyval(lin, np.log(R_b)))},
            "corr_h_c_R_d": corr, "n": int(len(h_c))}
