"""Exact-rational brute force of one DVL update -- TEST INFRASTRUCTURE.

An independent second statement of the per-update computation for tiny inputs,
in exact rational arithmetic (``fractions.Fraction``) and pure Python loops,
written straight from the paper's definitions rather than from the C oracle:

* Sec. 3.3: the field value is normalised to t in [0, 1] and looked up in the
  alpha transfer function (T equal buckets).
* Eq. 1: V = max_m alpha_m - min_m alpha_m.
* Eq. 5/6: max V approximated from the TF entries the data range reaches.
* Eq. 3: f = (max(V / max V, m) * 2^L)^P (minimum importance m of Eq. 2).
* Eq. 4: F(h) = sum of f up to h; xf1 = F(h-1)/F(max) * W, xf2 = F(h)/F(max) * W.
* Sec. 3.2: a cell adds its value to every pixel its [xf1, xf2) span touches,
  a per-pixel counter counts the additions, the mean is sum / count.

Only integer P is supported (a half-integer P makes f irrational).  The C
oracle's results agree with this exactly when every float32 operation it
performs is exact, which tests arrange by choosing dyadic inputs; with
``widths`` given, the brute force instead places cells with those integer
widths, which checks the oracle's position and binning arithmetic on any input.
"""
from __future__ import annotations

from fractions import Fraction
from math import floor, ceil


def _bucket(t: Fraction, T: int) -> int:
    return min(floor(t * T), T - 1)


def brute_update(fields, level, alpha, W, P=1, min_importance=Fraction(1, 32), dom_lo=None,
                 dom_hi=None, min_imp_mode=0, width_mode=0, widths=None):
    """fields: list of M lists of numbers; level: list; alpha: M lists of T numbers.

    Returns dict(f, b1, b2, count, sum, min, max, vmax) with exact values."""
    M, n = len(fields), len(level)
    T = len(alpha[0])
    F_ = Fraction
    vals = [[F_(v) for v in fl] for fl in fields]
    alp = [[F_(a) for a in al] for al in alpha]
    lo, hi = [], []
    for m in range(M):
        if dom_lo is None or dom_lo[m] is None:
            lo.append(min(vals[m]) if n else F_(0))
            hi.append(max(vals[m]) if n else F_(0))
        else:
            lo.append(F_(dom_lo[m]))
            hi.append(F_(dom_hi[m]))

    def norm(m, v):
        if hi[m] <= lo[m]:
            return F_(0)
        return min(max((v - lo[m]) / (hi[m] - lo[m]), F_(0)), F_(1))

    # Eq. 5 / Eq. 6
    i_g = min(_bucket(norm(m, min(vals[m])), T) for m in range(M)) if n else 0
    j_g = max(_bucket(norm(m, max(vals[m])), T) for m in range(M)) if n else 0
    vmax = max((max(alp[m][a] for m in range(M)) - min(alp[m][a] for m in range(M))
                for a in range(i_g, j_g + 1)), default=F_(0))

    t = [[norm(m, vals[m][c]) for c in range(n)] for m in range(M)]
    f = []
    for c in range(n):
        al = [alp[m][_bucket(t[m][c], T)] for m in range(M)]
        V = max(al) - min(al)                                   # Eq. 1
        r = V / vmax if vmax > 0 else F_(0)
        scale = F_(2) ** (level[c] * (3 if width_mode else 1))
        mi = F_(min_importance)
        if min_imp_mode == 0:
            fc = (max(r, mi) * scale) ** P                      # Eq. 3
        else:
            fc = max((r * scale) ** P, mi)
        f.append(fc)

    w = [F_(x) for x in widths] if widths is not None else f
    total = sum(w, F_(0))
    if total == 0 and n:
        w = [F_(1)] * n
        total = F_(n)
    b1, b2 = [], []
    count = [0] * W
    s = [[F_(0)] * W for _ in range(M)]
    mn = [[None] * W for _ in range(M)]
    mx = [[None] * W for _ in range(M)]
    acc = F_(0)
    for c in range(n):
        xf1 = acc / total * W                                   # Eq. 4
        acc += w[c]
        xf2 = acc / total * W
        k1 = min(floor(xf1), W - 1)
        k2 = min(ceil(xf2) - 1, W - 1) if xf2 > xf1 else k1
        b1.append(k1)
        b2.append(k2)
        for p in range(k1, k2 + 1):
            count[p] += 1
            for m in range(M):
                v = t[m][c]
                s[m][p] += v
                mn[m][p] = v if mn[m][p] is None else min(mn[m][p], v)
                mx[m][p] = v if mx[m][p] is None else max(mx[m][p], v)
    return dict(f=f, b1=b1, b2=b2, count=count, sum=s, min=mn, max=mx, vmax=vmax, i=i_g, j=j_g)
