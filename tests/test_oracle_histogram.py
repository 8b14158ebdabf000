"""Pins for the oracle's muPDF (Sec. 5.3, Eq. weighthisto): brute-force
binning against edges computed in 50-digit decimal arithmetic, exact integer
weights, and the weighted moments from their definitions."""
import math
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np

import inputs
import oracle


def _edges(mu_min, mu_max, bins):
    getcontext().prec = 50
    lo, hi = Decimal(mu_min).ln(), Decimal(mu_max).ln()
    return [float((lo + (hi - lo) * Decimal(i) / Decimal(bins)).exp()) for i in range(bins + 1)], \
        [(lo + (hi - lo) * Decimal(i) / Decimal(bins)).exp() for i in range(bins + 1)]


def test_histogram_against_brute_force():
    g = inputs.rng(42)
    n, bins, mu_min, mu_max = 5000, 200, 0.5, 5.0
    mu = np.exp(g.uniform(math.log(0.3), math.log(8.0), n))
    mu[::7] *= -1.0                      # negative parity, binned by |mu|
    flags = np.zeros(n, np.int32)
    flags[3] = oracle.F_NOCROSS
    mu[5] = np.nan
    _, edges = _edges(mu_min, mu_max, bins)
    # keep values clear of the bin edges (the FP64 decision is then unambiguous)
    getcontext().prec = 50
    keep = []
    for i, m in enumerate(mu):
        if not np.isfinite(m):
            keep.append(True)
            continue
        d = min(abs(Decimal(abs(float(m))) / e - 1) for e in edges)
        keep.append(d > Decimal("1e-9"))
    mu = mu[np.array(keep)]
    flags = flags[np.array(keep)]
    counts, wfix, sc = oracle.histogram(mu, flags, bins, mu_min, mu_max)

    ref_c = [0] * bins
    ref_w = [0] * bins
    under = over = neg = used = bad = 0
    invs = []
    for m, fl in zip(mu, flags):
        if fl or not np.isfinite(m):
            bad += 1
            continue
        used += 1
        a = abs(float(m))
        neg += m < 0
        invs.append(1.0 / a)
        da = Decimal(a)
        if da < edges[0]:
            under += 1
        elif da >= edges[-1]:
            over += 1
        else:
            k = max(i for i in range(bins) if edges[i] <= da)
            ref_c[k] += 1
            ref_w[k] += round(Fraction(2 ** 32) / Fraction(a))  # round half to even
    assert counts.tolist() == ref_c
    assert wfix.tolist() == ref_w
    assert (sc["n_used"], sc["n_under"], sc["n_over"], sc["n_neg"], sc["n_bad"]) == (used, under, over, neg, bad)
    assert sum(ref_c) + under + over == used
    W = math.fsum(invs)
    assert abs(sc["W_total"] / W - 1) < 1e-14
    # weighted mean with w = 1/|mu|: sum(w |mu|) / sum(w) = n / sum(1/|mu|)
    assert abs(sc["mean_w"] / (used / W) - 1) < 1e-13
    absmu = [1 / w for w in invs]
    mean = used / W
    var = math.fsum((a - mean) ** 2 / a for a in absmu) / W
    assert abs(sc["sigma_w"] / math.sqrt(var) - 1) < 1e-12


def test_histogram_normalisation_and_edges():
    bins, mu_min, mu_max = 10, 1.0, 10.0
    mu = np.array([1.0, 1.5, 9.99, 10.0, 0.999, 3.0])
    counts, wfix, sc = oracle.histogram(mu, None, bins, mu_min, mu_max)
    assert counts[0] == 1                 # mu = mu_min sits in the first bin
    assert sc["n_over"] == 1 and sc["n_under"] == 1
    edges, _ = _edges(mu_min, mu_max, bins)
    dmu = np.diff(edges)
    W = wfix.astype(np.float64) / 2 ** 32
    # P(mu) d mu = F / mu (Eq. weighthisto), normalised over the binned range
    P = W / (W.sum() * dmu)
    assert abs(np.sum(P * dmu) - 1) < 1e-12


def test_flux_conservation_weighting():
    # for a population whose image-plane areas are mu_i, the 1/mu-weighted mean
    # magnification is n / sum(1/mu) (Eqs. fluxconserve, weighthisto)
    mu = np.array([0.9, 0.95, 1.0, 1.2, 2.0])
    _, _, sc = oracle.histogram(mu, None, 20, 0.5, 5.0)
    assert abs(sc["mean_w"] - len(mu) / np.sum(1 / mu)) < 1e-15


def test_shear_histogram_against_brute_force():
    # shear PDF (Sec. 5.4): |gamma| binned in log10, weight 1/|mu|, checked
    # against 50-digit edges and exact integer weights
    g = inputs.rng(43)
    n, bins, g_min, g_max = 4000, 120, 1e-3, 0.5
    gam = np.exp(g.uniform(math.log(3e-4), math.log(0.9), n))
    ang = g.uniform(0, 2 * math.pi, n)
    g1, g2 = gam * np.cos(ang), gam * np.sin(ang)
    mu = np.exp(g.uniform(math.log(0.5), math.log(3.0), n))
    mu[::11] *= -1.0
    g1[4], g2[4] = 0.0, 0.0          # no shear: underflow
    flags = np.zeros(n, np.int32)
    flags[9] = oracle.F_NONFINITE
    getcontext().prec = 50
    _, edges = _edges(g_min, g_max, bins)
    gabs = [Decimal(float(a)) ** 2 + Decimal(float(b)) ** 2 for a, b in zip(g1, g2)]
    gabs = [x.sqrt() for x in gabs]
    keep = np.array([x == 0 or min(abs(x / e - 1) for e in edges) > Decimal("1e-9") for x in gabs])
    mu, g1, g2, flags = mu[keep], g1[keep], g2[keep], flags[keep]
    gabs = [x for x, k in zip(gabs, keep) if k]
    counts, wfix, sc = oracle.shear_histogram(mu, g1, g2, flags, bins, g_min, g_max)
    ref_c, ref_w = [0] * bins, [0] * bins
    under = over = neg = used = bad = 0
    W, S1 = [], []
    for m, x, fl in zip(mu, gabs, flags):
        if fl:
            bad += 1
            continue
        used += 1
        neg += m < 0
        w = 1.0 / abs(float(m))
        W.append(w)
        S1.append(w * float(x))
        if x < edges[0]:
            under += 1
        elif x >= edges[-1]:
            over += 1
        else:
            k = max(i for i in range(bins) if edges[i] <= x)
            ref_c[k] += 1
            ref_w[k] += round(Fraction(2 ** 32) / Fraction(abs(float(m))))
    assert counts.tolist() == ref_c and wfix.tolist() == ref_w
    assert (sc["n_used"], sc["n_under"], sc["n_over"], sc["n_neg"], sc["n_bad"]) == (used, under, over, neg, bad)
    assert abs(sc["mean_w"] / (math.fsum(S1) / math.fsum(W)) - 1) < 1e-13
