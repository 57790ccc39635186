"""Small statistics helpers shared by the tests."""
import numpy as np
import scipy.stats as st


def chisq_pvalue(codes, p, min_expected=5.0):
    """Chi-square goodness of fit of integer-coded samples against the law p.

    Bins with expected count below min_expected are pooled into one bin."""
    codes = np.asarray(codes, np.int64)
    M = codes.size
    obs = np.bincount(codes, minlength=len(p)).astype(float)
    exp = np.asarray(p, float) * M
    big = exp >= min_expected
    o = np.append(obs[big], obs[~big].sum())
    e = np.append(exp[big], exp[~big].sum())
    if e[-1] < min_expected:
        o, e = o[:-1], e[:-1]
        o[-1] += obs[~big].sum()
        e[-1] += exp[~big].sum()
    e = e * o.sum() / e.sum()
    return float(st.chisquare(o, e).pvalue)
