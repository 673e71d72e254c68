"""The density tag's exponent shortcut (tag_kernel, Sec. 3.4 indicator)
never contradicts the test as written: whenever the exponents of the
differences, of rho_C and of tol^2 alone say that
(rho_E - rho_W)^2 + (rho_N - rho_S)^2 <= tol^2 (2 rho_C)^2 / 2, the rounded
binary64 test (rho_E - rho_W)^2 + (rho_N - rho_S)^2 > tol^2 (2 rho_C)^2 is
false.  The predicate is restated here from its definition (binary
exponents of the operands, the bounds 2 Ed + 3 <= Et + 2 Ec + 1 and
|Ed|, |Ec|, |Et| <= 200) and checked on random and adversarial operands."""
import numpy as np


def bexp(x):
    return ((np.asarray(x, dtype=np.float64).view(np.uint64) >> np.uint64(52)) & np.uint64(0x7FF)).astype(np.int64)


def below(d1, d2, rc, tol2):
    et = bexp(tol2) - 1023
    ec = bexp(rc) - 1023
    ed = np.maximum(bexp(d1), bexp(d2)) - 1023
    ok = (et >= -200) & (et <= 200) & (ec >= -200) & (ec <= 200) & (ed <= 200) & (tol2 > 0)
    return ok & (2 * ed + 3 <= et + 2 * ec + 1)


def full(d1, d2, rc, tol2):
    with np.errstate(all="ignore"):
        num = d1 * d1 + d2 * d2
        t = 2.0 * rc
        return num > tol2 * (t * t)


def test_shortcut_never_contradicts_the_test():
    rng = np.random.default_rng(7)
    n = 2_000_000
    rc = np.exp(rng.uniform(-60, 60, n)) * rng.choice([1.0, -1.0], n)
    tol2 = np.exp(rng.uniform(-40, 10, n))
    # differences around the threshold tol * 2 rc, spread over many binades
    scale = np.sqrt(tol2) * 2 * np.abs(rc)
    d1 = scale * np.exp(rng.uniform(-30, 3, n)) * rng.choice([1.0, -1.0], n)
    d2 = scale * np.exp(rng.uniform(-30, 3, n)) * rng.choice([1.0, -1.0], n)
    d2[::7] = 0.0
    d1[::11] = 5e-324  # subnormal
    b = below(d1, d2, rc, tol2)
    f = full(d1, d2, rc, tol2)
    assert not np.any(b & f)
    assert b.sum() > n // 4 and f.sum() > n // 10  # both outcomes are exercised
    # right at the bound: the largest differences the shortcut accepts
    for et in (-12, -3, 0, 5):
        for ec in (-5, 0, 3):
            ed = (et + 2 * ec + 1 - 3) // 2
            d = np.nextafter(2.0 ** (ed + 1), 0.0)
            r = 2.0 ** ec
            t2 = 2.0 ** et
            assert below(np.array([d]), np.array([d]), np.array([r]), np.array([t2]))[0]
            assert not full(np.array([d]), np.array([d]), np.array([r]), np.array([t2]))[0]


def test_shortcut_stands_aside_for_extremes():
    """Zeros, NaN, infinities and far exponents go to the full test."""
    one = np.array([1.0])
    for rc in (0.0, np.nan, np.inf, 2.0 ** -300, 2.0 ** 300):
        assert not below(one * 1e-9, one * 1e-9, np.array([rc]), np.array([4e-4]))[0]
    for tol2 in (0.0, 2.0 ** -300, np.inf, np.nan):
        assert not below(one * 1e-9, one * 1e-9, one, np.array([tol2]))[0]
    assert not below(np.array([np.nan]), one * 0.0, one, np.array([4e-4]))[0]
    assert below(one * 0.0, one * 0.0, one, np.array([4e-4]))[0]  # zero differences: never tagged
