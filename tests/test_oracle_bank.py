"""Pins of the oracle's template-bank generators (Sec. 2: cubic lattice and
uniform random banks) to facts that do not come from the oracle itself:
numpy's own Philox4x64-10 implementation, hand-written lattice values, the
uniform distribution (Kolmogorov-Smirnov) and the slicing property that lets
a bank of 1e8-1e9 templates be produced in independent ranges."""
import numpy as np
import pytest

import oracle

LO = (500.0, 3500.0, 3.0)
HI = (3000.0, 35000.0, 7.0)


@pytest.mark.parametrize("counter,key", [((0, 0, 0, 0), (0, 0)), ((5, 7, 0, 0), (123, 456)),
                                         ((2**64 - 2, 2**63, 1, 2**40), (2**64 - 1, 99)),
                                         ((10**12, 0, 0, 0), (20250715, 0))])
def test_philox_matches_numpy(counter, key):
    """numpy.random.Philox is Philox4x64-10; it increments its 256-bit counter
    before producing each block, so block c comes from Philox(counter=c - 1)."""
    c = list(counter)
    prev = c[:]
    for w in range(4):                # 256-bit decrement
        if prev[w] > 0:
            prev[w] -= 1
            break
        prev[w] = 2**64 - 1
    bg = np.random.Philox(counter=np.array(prev, np.uint64), key=np.array(key, np.uint64))
    np.testing.assert_array_equal(oracle.philox4x64_10(c, key), bg.random_raw(4).astype(np.uint64))


def test_lattice_hand_values():
    """3 x 2 x 2 lattice, f0 fastest: every point written out by hand."""
    f0, tau, n = oracle.bank_templates(0, 0, 12, (500.0, 3500.0, 3.0), (600.0, 35000.0, 7.0),
                                       n_f0=3, n_tau=2, n_n=2)
    exp = [(f, t, m) for m in (3.0, 7.0) for t in (3500.0, 35000.0) for f in (500.0, 550.0, 600.0)]
    assert list(zip(f0, tau, n)) == exp


def test_lattice_axis_spacing_and_endpoints():
    m = 1001
    f0, tau, n = oracle.bank_templates(0, 0, m, LO, HI, n_f0=m)
    assert f0[0] == LO[0] and f0[-1] == HI[0]
    step = (HI[0] - LO[0]) / (m - 1)
    np.testing.assert_allclose(np.diff(f0), step, rtol=1e-11)
    assert np.all(tau == LO[1]) and np.all(n == LO[2])      # other axes at their first point
    # a single-point axis sits at its lower bound
    f0, _, _ = oracle.bank_templates(0, 0, 1, LO, HI, n_f0=1)
    assert f0[0] == LO[0]


def test_random_bank_from_numpy_philox():
    """Template t uses block (t, 0, 0, 0) under key (seed, 0); value = lo + (hi - lo) u
    with u = (x >> 11) 2^-53, recomputed here from numpy's Philox (within one ulp:
    the oracle rounds the product and sum once, by fma)."""
    seed, first, count = 777, 1000, 64
    f0, tau, n = oracle.bank_templates(1, first, count, LO, HI, seed=seed)
    bg = np.random.Philox(counter=np.array([first - 1, 0, 0, 0], np.uint64), key=np.array([seed, 0], np.uint64))
    raw = bg.random_raw(4 * count).astype(np.uint64).reshape(count, 4)
    u = (raw[:, :3] >> np.uint64(11)).astype(np.float64) * 2.0**-53
    for a, got in enumerate((f0, tau, n)):
        ref = (HI[a] - LO[a]) * u[:, a] + LO[a]
        assert np.all(np.abs(got - ref) <= np.spacing(ref))


def test_random_bank_uniform_and_sliceable():
    scipy_stats = pytest.importorskip("scipy.stats")
    N = 100000
    f0, tau, n = oracle.bank_templates(1, 0, N, LO, HI, seed=20250715)
    for a, v in enumerate((f0, tau, n)):
        assert v.min() >= LO[a] and v.max() <= HI[a]
        assert scipy_stats.kstest((v - LO[a]) / (HI[a] - LO[a]), "uniform").pvalue > 1e-4
    assert abs(np.corrcoef(f0, tau)[0, 1]) < 0.02 and abs(np.corrcoef(tau, n)[0, 1]) < 0.02
    # any range equals the same slice of the whole bank
    g = oracle.bank_templates(1, 31337, 777, LO, HI, seed=20250715)
    for a, v in enumerate((f0, tau, n)):
        np.testing.assert_array_equal(g[a], v[31337:31337 + 777])
    # a different seed gives a different bank
    h = oracle.bank_templates(1, 0, 100, LO, HI, seed=20250716)
    assert not np.array_equal(h[0], f0[:100])
