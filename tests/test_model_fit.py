"""The statistical bound of Section 3: y = a + b n log2 n + c n fitted by least squares,
with the diagnostics Sections 3.1 and 3.2 print. Refitting the paper's own Table 1 mean
times (K-sort and Heap sort) must give back every printed number at its printed
precision: eqs (1) and (2) with SE, t, p, VIF, S, R-Sq, R-Sq(adj), PRESS, R-Sq(pred), the
analysis of variance, the sequential sums of squares and the ten observation rows. Eq (3)
of Section 4 is their difference. Then properties that hold for any data."""
import math
import os

import numpy as np
import pytest

from paper_1107_3622_gb300 import statbound as sb

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "section3_regression.txt")


def _golden():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def _close(got, printed: str, pct=False):
    """True when `got` rounds to the printed string (half a unit of its last digit)."""
    want = float(printed)
    dec = len(printed.split(".")[1]) if "." in printed else 0
    tol = 0.5 * 10.0 ** -dec * (1 + 1e-9) + 1e-15
    g = got * 100.0 if pct else got
    return abs(g - want) <= tol


def _table1():
    rows = [r for r in _golden() if r[0] == "table1"]
    ns = [int(r[1]) for r in rows]
    return ns, [float(r[2]) for r in rows], [float(r[3]) for r in rows]


def _fits():
    ns, k, h = _table1()
    return {"K": sb.fit(ns, k), "H": sb.fit(ns, h)}


def test_table1_nlog2n_column():
    got = {n: v for n, v in zip(_table1()[0], sb.design(_table1()[0])[:, 1])}
    for r in _golden():
        if r[0] == "table1_nlog2n":
            assert _close(got[int(r[1])], r[2]), r


@pytest.mark.parametrize("model", ["K", "H"])
def test_refit_reproduces_printed_regression(model):
    f = _fits()[model]
    checked = 0
    for r in _golden():
        if r[0] != model:
            continue
        field, vals = r[1], r[2:]
        if field in ("coef", "se_coef", "t"):
            for g, w in zip(f[field], vals):
                assert _close(g, w), (model, field, g, w)
        elif field == "p":
            pytest.importorskip("scipy")
            for g, w in zip(f["p"], vals):
                assert _close(g, w), (model, field, g, w)
        elif field in ("vif", "s", "press"):
            assert _close(f[field], vals[0]), (model, field)
        elif field.endswith("_pct"):
            assert _close(f[field[:-4]], vals[0], pct=True), (model, field)
        elif field.startswith("anova_"):
            row = f["anova"][field[6:]]
            assert row["df"] == int(vals[0]) and _close(row["ss"], vals[1]), (model, field)
            if len(vals) > 2:
                assert _close(row["ms"], vals[2]), (model, field)
            if len(vals) > 3:
                assert _close(f["anova"]["f"], vals[3]), (model, "F")
                if f["anova"]["p"] is not None:
                    assert _close(f["anova"]["p"], vals[4]), (model, "P")
        elif field == "seq_ss":
            assert _close(f["anova"]["seq_ss"]["nlog2n"], vals[0])
            assert _close(f["anova"]["seq_ss"]["n"], vals[1])
        elif field == "obs":
            i = int(vals[0]) - 1
            o = f["obs"]
            for key, w in zip(("nlog2n", "y", "fit", "se_fit", "residual", "st_resid"),
                              vals[1:]):
                assert _close(o[key][i], w), (model, "obs", i + 1, key, o[key][i], w)
        elif field == "large":
            assert [i + 1 for i in f["obs"]["large"]] == [int(v) for v in vals]
        else:
            raise AssertionError(f"unknown golden field {field}")
        checked += 1
    assert checked >= 25


def test_equation_3_is_the_difference():
    g = {r[0]: r[1:] for r in _golden() if r[0].startswith("eq3")}
    d = sb.difference(*(_fits()[m] for m in ("K", "H")))
    printed = g["eq3_printed"]
    # the slopes: difference of the fits rounds to the printed eq (3) slopes
    assert _close(d["b_nlog2n"], printed[1]) and _close(d["c_n"], printed[2])
    # the constant: the difference of eqs (1) and (2) as printed (0.7516 - 0.12574)
    k = [float(v) for v in next(r for r in _golden() if r[:2] == ["K", "coef"])[2:]]
    h = [float(v) for v in next(r for r in _golden() if r[:2] == ["H", "coef"])[2:]]
    assert k[0] - h[0] == pytest.approx(float(g["eq3_constant_as_read"][0]), abs=1e-12)
    assert _close(d["a"], "0.626")          # the fits' own difference, to 3 decimals
    assert not _close(k[0] - h[0], printed[0])  # the printed 0.52586 is not the difference


def test_fit_is_exact_on_model_data():
    ns = [1e5, 5e5, 1e6, 2.5e6, 5e6, 1e7]
    ys = [0.2 + 3e-8 * n * math.log2(n) + 1e-7 * n for n in ns]
    f = sb.fit(ns, ys)
    assert f["a"] == pytest.approx(0.2, rel=1e-6)
    assert f["b_nlog2n"] == pytest.approx(3e-8, rel=1e-6)
    assert f["c_n"] == pytest.approx(1e-7, rel=1e-5)
    assert f["r2"] == pytest.approx(1.0)
    assert np.allclose(sb.predict(f, ns), ys, rtol=1e-9)


def test_identities_on_random_data():
    rng = np.random.default_rng(3)
    ns = np.sort(rng.uniform(1e4, 1e7, 12))
    ys = 1e-8 * ns * np.log2(ns) + rng.normal(0, 0.05, ns.size)
    f = sb.fit(ns, ys)
    a = f["anova"]
    # SS decomposition, sequential SS sum, R^2 forms
    assert a["regression"]["ss"] + a["residual"]["ss"] == pytest.approx(a["total"]["ss"])
    assert a["seq_ss"]["nlog2n"] + a["seq_ss"]["n"] == pytest.approx(a["regression"]["ss"])
    assert f["r2"] == pytest.approx(a["regression"]["ss"] / a["total"]["ss"])
    # residuals orthogonal to the design; leverages sum to the coefficient count
    X = sb.design(ns)
    assert np.abs(X.T @ np.array(f["obs"]["residual"])).max() < 1e-6 * np.abs(X).max()
    h = (np.array(f["obs"]["se_fit"]) ** 2) / a["residual"]["ms"]
    assert h.sum() == pytest.approx(3.0)
    # PRESS equals the leave-one-out prediction errors computed by refitting
    loo = 0.0
    for i in range(ns.size):
        keep = np.arange(ns.size) != i
        fi = sb.fit(ns[keep], ys[keep])
        loo += float(ys[i] - sb.predict(fi, ns[i])[0]) ** 2
    assert f["press"] == pytest.approx(loo, rel=1e-6)


def test_too_few_observations():
    with pytest.raises(ValueError):
        sb.fit([1e5, 1e6, 1e7], [1, 2, 3])
