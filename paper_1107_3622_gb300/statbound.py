"""Statistical bound of a sort's run time (Section 3): ordinary least squares of the mean
time y on n log2 n and n with an intercept,

    y = a + b * n log2 n + c * n,

with the diagnostics Section 3 reports for eqs (1) and (2): standard errors, t ratios,
S, R-Sq, R-Sq(adj), PRESS, R-Sq(pred), the analysis of variance with sequential sums of
squares (n log2 n entered first), variance inflation factors, and per observation the fit,
its standard error, the residual and the standardised residual. Eq (3) of Section 4 is the
coefficient-wise difference of two fits (`difference`).

Plain numpy on the host; it only consumes measured times."""
from __future__ import annotations

import math

import numpy as np

PREDICTORS = ("constant", "nlog2n", "n")


def design(ns) -> np.ndarray:
    """The model's design matrix: columns 1, n log2 n, n (Section 3.1)."""
    n = np.asarray(ns, dtype=np.float64)
    return np.stack([np.ones_like(n), n * np.log2(n), n], axis=1)


def _p_two_sided(t: float, df: int):
    """Two-sided p value of a t ratio (scipy's Student t; None without scipy)."""
    try:
        from scipy.special import stdtr
    except ImportError:
        return None
    return float(2.0 * stdtr(df, -abs(t)))


def _p_f(f: float, dfn: int, dfd: int):
    try:
        from scipy.special import fdtrc
    except ImportError:
        return None
    return float(fdtrc(dfn, dfd, f))


def fit(ns, ys) -> dict:
    """Least-squares fit of y = a + b n log2 n + c n with Section 3's diagnostics."""
    X = design(ns)
    y = np.asarray(ys, dtype=np.float64)
    m, p = X.shape
    if m <= p:
        raise ValueError("the model has 3 coefficients: at least 4 observations are needed")
    # QR keeps the conditioning of the n log2 n / n pair (VIF ~ 2e3) out of the normal
    # equations; R^-1 gives (X'X)^-1 = R^-1 R^-T.
    Q, R = np.linalg.qr(X)
    coef = np.linalg.solve(R, Q.T @ y)
    Rinv = np.linalg.solve(R, np.eye(p))
    xtx_inv = Rinv @ Rinv.T
    fitted = X @ coef
    res = y - fitted
    sse = float(res @ res)
    dfe = m - p
    mse = sse / dfe
    s = math.sqrt(mse)
    se = np.sqrt(np.diag(xtx_inv) * mse)
    sst = float(((y - y.mean()) ** 2).sum())
    ssr = sst - sse
    h = np.einsum("ij,jk,ik->i", X, xtx_inv, X)        # leverages
    press = float(((res / (1.0 - h)) ** 2).sum())
    # sequential sums of squares: n log2 n alone, then n added to it
    X1 = X[:, :2]
    c1, *_ = np.linalg.lstsq(X1, y, rcond=None)
    r1 = y - X1 @ c1
    seq1 = sst - float(r1 @ r1)
    # variance inflation of the two slopes (they share one VIF with two predictors)
    z = X[:, 1:]
    corr = np.corrcoef(z[:, 0], z[:, 1])[0, 1]
    vif = 1.0 / (1.0 - corr * corr)
    t = coef / se
    st_resid = res / np.sqrt(mse * (1.0 - h))
    return {
        "a": float(coef[0]), "b_nlog2n": float(coef[1]), "c_n": float(coef[2]),
        "coef": coef.tolist(), "se_coef": se.tolist(), "t": t.tolist(),
        "p": [_p_two_sided(v, dfe) for v in t], "vif": float(vif),
        "s": s, "r2": 1.0 - sse / sst, "r2_adj": 1.0 - mse / (sst / (m - 1)),
        "press": press, "r2_pred": 1.0 - press / sst,
        "anova": {"regression": {"df": p - 1, "ss": ssr, "ms": ssr / (p - 1)},
                  "residual": {"df": dfe, "ss": sse, "ms": mse},
                  "total": {"df": m - 1, "ss": sst},
                  "f": (ssr / (p - 1)) / mse, "p": _p_f((ssr / (p - 1)) / mse, p - 1, dfe),
                  "seq_ss": {"nlog2n": seq1, "n": ssr - seq1}},
        "obs": {"nlog2n": X[:, 1].tolist(), "y": y.tolist(), "fit": fitted.tolist(),
                "se_fit": np.sqrt(h * mse).tolist(), "residual": res.tolist(),
                "st_resid": st_resid.tolist(),
                # observations flagged for a large standardised residual (|value| > 2)
                "large": [int(i) for i in np.nonzero(np.abs(st_resid) > 2.0)[0]]},
    }


def predict(f: dict, n) -> np.ndarray:
    """The fitted time at sizes n (Section 4's use of eqs (1)-(3) beyond the measured range)."""
    return design(np.atleast_1d(n)) @ np.asarray(f["coef"])


def difference(fk: dict, fh: dict) -> dict:
    """Eq (3): the difference of two fitted equations, coefficient by coefficient."""
    d = [a - b for a, b in zip(fk["coef"], fh["coef"])]
    return {"a": d[0], "b_nlog2n": d[1], "c_n": d[2], "coef": d}


def summary(f: dict, digits: int = 6) -> dict:
    """The compact form bench.py records: coefficients, SE, R-Sq, R-Sq(adj), S."""
    g = lambda v: float(f"{v:.{digits}g}")  # noqa: E731
    return {"a": g(f["a"]), "b_nlog2n": g(f["b_nlog2n"]), "c_n": g(f["c_n"]),
            "se_coef": [g(v) for v in f["se_coef"]], "s": g(f["s"]),
            "r2": round(f["r2"], 4), "r2_adj": round(f["r2_adj"], 4)}
