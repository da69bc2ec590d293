"""Pins of the FP64 oracle to facts that do not come from the oracle itself.

Each test names the passage of the paper it checks and the independent fact it
uses: hand-derived closed forms, the braking-law ODE, detector positions,
special geometries, exact library sorts, statistical invariants, and recovery
of a signal synthesised without the search's closed forms.
"""
import math
import os

import numpy as np
import pytest

import oracle
import tcw_synth as syn

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_rows(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#", 1)[0].strip()
        if line:
            rows.append(line.split())
    return rows


# ---------------------------------------------------------------- Eq. 1 ----
def test_track_golden_closed_forms():
    """Eq. 1 at times where the base is an exact power (hand-derived values)."""
    for f0, tau, n, dt, fexp in _read_rows("track_closed_form.txt"):
        f0, tau, n, dt, fexp = map(float, (f0, tau, n, dt, fexp))
        T0 = 1.4e9
        got = oracle.track_frequency(f0, tau, n, T0, T0 + dt)
        assert got == pytest.approx(fexp, rel=4e-15), (f0, tau, n, dt)


def test_track_special_exponents():
    """n = 3, 5 and 2 reduce Eq. 1 to square roots and a reciprocal."""
    r = syn.rng(1)
    for _ in range(200):
        f0 = r.uniform(500, 3000)
        tau = r.uniform(3500, 35000)
        T0 = 1.4e9
        dt = (T0 + r.uniform(0, 1e5)) - T0      # exactly representable offset
        x = dt / tau
        assert oracle.track_frequency(f0, tau, 3.0, T0, T0 + dt) == pytest.approx(
            f0 / math.sqrt(1 + x), rel=4e-16 * 8)
        assert oracle.track_frequency(f0, tau, 5.0, T0, T0 + dt) == pytest.approx(
            f0 / math.sqrt(math.sqrt(1 + x)), rel=4e-16 * 8)
        assert oracle.track_frequency(f0, tau, 2.0, T0, T0 + dt) == pytest.approx(
            f0 / (1 + x), rel=4e-16 * 8)


def test_track_starts_at_f0_and_decreases():
    r = syn.rng(2)
    for _ in range(100):
        f0, tau, n = r.uniform(500, 3000), r.uniform(3500, 35000), r.uniform(3, 7)
        T0 = 1.4e9
        assert oracle.track_frequency(f0, tau, n, T0, T0) == f0
        ts = T0 + np.linspace(0, 2e5, 64)
        fs = [oracle.track_frequency(f0, tau, n, T0, t) for t in ts]
        assert all(a >= b for a, b in zip(fs, fs[1:]))


def test_track_matches_braking_law_integration():
    """Eq. 1 is the solution of df/dt = -f^n/((n-1) tau f0^(n-1)) (RK4 reference)."""
    r = syn.rng(3)
    for _ in range(6):
        f0, tau, n = r.uniform(500, 3000), r.uniform(3500, 35000), r.uniform(3, 7)
        T0 = 1.4e9
        t = T0 + np.sort(r.uniform(0, 4e4, 40))
        ode = syn.spindown_frequency(f0, tau, n, T0, t)
        ora = np.array([oracle.track_frequency(f0, tau, n, T0, x) for x in t])
        np.testing.assert_allclose(ora, ode, rtol=1e-10)


# ---------------------------------------------------------------- Eq. 2 ----
def test_doppler_geometry():
    """Perpendicular motion gives no shift; motion toward the source gives f(1+|v|/c)."""
    v = np.array([12000.0, -25000.0, 3000.0])
    u = v / np.linalg.norm(v)
    perp = np.cross(u, [0.0, 0.0, 1.0])
    perp /= np.linalg.norm(perp)
    assert oracle.doppler_frequency(1000.0, v, perp) == pytest.approx(1000.0, rel=1e-15)
    assert oracle.doppler_frequency(1000.0, v, u) == pytest.approx(
        1000.0 * (1 + np.linalg.norm(v) / 299792458.0), rel=1e-15)
    assert oracle.doppler_frequency(1000.0, v, -u) < 1000.0


def test_earth_motion_model():
    """Orbital speed 2 pi AU / yr = 29.78 km/s; velocity is d(position)/dt."""
    det = syn.Detector(latitude=0.3, longitude=1.0, orbit_phase=2.0)
    t = syn.GPS_EPOCH0 + np.linspace(0, 86400, 50)
    v = det.velocity(t)
    orb = 2 * math.pi * syn.AU / syn.YEAR
    assert orb == pytest.approx(29785.0, rel=1e-3)
    speeds = np.linalg.norm(v, axis=1)
    assert speeds.min() > orb - 466 and speeds.max() < orb + 466
    h = 1.0
    fd = (det.position(t + h) - det.position(t - h)) / (2 * h)
    np.testing.assert_allclose(fd, v, atol=2e-3)


def test_doppler_matches_arrival_delay_derivative():
    """Eq. 2 equals f times d/dt of the arrival delay r(t).nhat/c (from positions)."""
    r = syn.rng(4)
    det = syn.random_detectors(r, 1)[0]
    t = syn.GPS_EPOCH0 + np.linspace(0, 4e4, 30)
    v = det.velocity(t)
    for nhat in syn.random_sky(r, 8):
        ref = syn.detector_frame_frequency(np.full(t.shape, 1500.0), det, nhat, t)
        got = np.array([oracle.doppler_frequency(1500.0, v[i], nhat) for i in range(t.size)])
        # FP64 positions of ~1 AU limit the finite difference to a few 1e-12; a sign
        # or factor error in Eq. 2 would show at the 1e-4 level.
        np.testing.assert_allclose(got, ref, rtol=5e-12)


# ------------------------------------------------------------- binning ----
def test_bin_rounding_hand_cases():
    f_min, df = 500.0, 0.25
    cases = [(500.0, 0), (500.12, 0), (500.125, 1), (500.13, 1), (500.25, 1),
             (499.875, 0), (499.87, -1), (503.0, 12), (502.874, 11), (502.875, 12)]
    for fh, k in cases:
        assert oracle.bin_index(fh, f_min, df) == k, fh


def test_out_of_band_and_pre_T0_fixture():
    """Hand-computed S, W1, W2 with band edges and a segment before T0."""
    kv = {row[0]: row[1:] for row in _read_rows("out_of_band_case.txt")}
    t = np.array(list(map(float, kv["t_mid"])))
    w = np.array([list(map(float, kv["weights"]))], np.float32)
    n_bin = int(kv["n_bin"][0])
    rho = np.zeros((1, t.size, n_bin), np.float32)
    for j in range(t.size):
        rho[0, j] = 1 + j + np.arange(n_bin) / 100.0
    vel = np.zeros((1, t.size, 3))
    S, W1, W2, Psi = oracle.search_stats(
        rho, float(kv["f_min"][0]), float(kv["df"][0]), t, w, vel,
        np.array([[0.0, 0.0, 1.0]]), [float(kv["f0"][0])], [float(kv["tau"][0])],
        [float(kv["n"][0])], float(kv["T0"][0]))
    assert S[0, 0] == pytest.approx(float(kv["S"][0]), rel=1e-6)
    assert W1[0, 0] == pytest.approx(float(kv["W1"][0]), rel=1e-12)
    assert W2[0, 0] == pytest.approx(float(kv["W2"][0]), rel=1e-12)
    assert Psi[0, 0] == pytest.approx((7.23 - 2.75) / math.sqrt(4.3125), rel=1e-6)
    x = oracle.track_coordinates(1, float(kv["f_min"][0]), float(kv["df"][0]), t, vel,
                                 np.array([[0.0, 0.0, 1.0]]), [100.0], [1000.0], [3.0],
                                 5000.0, [[0, 0]])[0, 0]
    bins = [-1 if not np.isfinite(v) else int(math.floor(v + 0.5)) for v in x]
    bins = [b if 0 <= b < n_bin else -1 for b in bins]
    assert bins == list(map(int, kv["bins"]))


def test_amplitude_weight_fixture():
    """Eq. 3 amplitude weight (f/f0)^4 on the hand-computed band-edge case:
    exact rational S, W1, W2 derived by hand from (1 + dt/tau)^-2 for n = 3."""
    kv = {row[0]: row[1:] for row in _read_rows("out_of_band_case.txt")}
    amp = {row[0]: row[1:] for row in _read_rows("amplitude_weight_case.txt")}
    t = np.array(list(map(float, kv["t_mid"])))
    w = np.array([list(map(float, kv["weights"]))], np.float32)
    n_bin = int(kv["n_bin"][0])
    rho = np.zeros((1, t.size, n_bin), np.float32)
    for j in range(t.size):
        rho[0, j] = 1 + j + np.arange(n_bin) / 100.0
    S, W1, W2, Psi = oracle.search_stats(
        rho, float(kv["f_min"][0]), float(kv["df"][0]), t, w, np.zeros((1, t.size, 3)),
        np.array([[0.0, 0.0, 1.0]]), [float(kv["f0"][0])], [float(kv["tau"][0])],
        [float(kv["n"][0])], float(kv["T0"][0]), amp_power=int(amp["amp_power"][0]))
    ex = {k: int(amp[k + "_num"][0]) / int(amp[k + "_den"][0]) for k in ("S", "W1", "W2")}
    assert S[0, 0] == pytest.approx(ex["S"], rel=1e-6)       # rho is float32
    assert W1[0, 0] == pytest.approx(ex["W1"], rel=1e-12)
    assert W2[0, 0] == pytest.approx(ex["W2"], rel=1e-12)
    assert Psi[0, 0] == pytest.approx((ex["S"] - ex["W1"]) / math.sqrt(ex["W2"]), rel=1e-6)


def test_amplitude_weight_closed_form_n5():
    """For n = 5, (f/f0)^4 = tau / (tau + t - T0) exactly (Eq. 1 and Eq. 3), so
    with unit power in every bin S = W1 = sum_j w_j tau/(tau + dt_j) and
    W2 = sum_j (w_j tau/(tau + dt_j))^2.  amp_power = 0 recovers the plain sums."""
    r = syn.rng(21)
    n_seg, n_bin = 40, 4096
    t = syn.segment_times(n_seg, 600.0)
    T0 = t[0] - 10.0
    rho = np.ones((2, n_seg, n_bin), np.float32)
    w = syn.uniform_weights(r, 2, n_seg, 0.2, 2.0)
    vel = np.zeros((2, n_seg, 3))
    f0 = r.uniform(900.0, 1000.0, 6)
    tau = r.uniform(3500.0, 35000.0, 6)
    n = np.full(6, 5.0)
    S, W1, W2, Psi = oracle.search_stats(rho, 500.0, 0.125, t, w, vel, np.array([[0, 0, 1.0]]),
                                         f0, tau, n, T0, amp_power=4)
    S0, W10, W20, _ = oracle.search_stats(rho, 500.0, 0.125, t, w, vel, np.array([[0, 0, 1.0]]),
                                          f0, tau, n, T0)
    wd = w.astype(np.float64)
    for b in range(6):
        a = tau[b] / (tau[b] + (t - T0))
        assert W1[0, b] == pytest.approx((wd * a).sum(), rel=1e-13)
        assert W2[0, b] == pytest.approx(((wd * a) ** 2).sum(), rel=1e-13)
        assert S[0, b] == pytest.approx(W1[0, b], rel=1e-13)
        assert Psi[0, b] == pytest.approx(0.0, abs=1e-12)
        assert W10[0, b] == pytest.approx(wd.sum(), rel=1e-13)
        assert W20[0, b] == pytest.approx((wd ** 2).sum(), rel=1e-13)
    # the weight decays: the template's own later segments count for less
    assert (W1 < W10).all()


def _band_edge_case(**kw):
    kv = {row[0]: row[1:] for row in _read_rows("out_of_band_case.txt")}
    t = np.array(list(map(float, kv["t_mid"])))
    w = np.array([list(map(float, kv["weights"]))], np.float32)
    n_bin = int(kv["n_bin"][0])
    rho = np.zeros((1, t.size, n_bin), np.float32)
    for j in range(t.size):
        rho[0, j] = 1 + j + np.arange(n_bin) / 100.0
    out = oracle.search_stats(
        rho, float(kv["f_min"][0]), float(kv["df"][0]), t, w, np.zeros((1, t.size, 3)),
        np.array([[0.0, 0.0, 1.0]]), [float(kv["f0"][0])], [float(kv["tau"][0])],
        [float(kv["n"][0])], float(kv["T0"][0]), **kw)
    return tuple(float(x[0, 0]) for x in out)


def test_number_count_fixture():
    """Number count on the hand-computed band-edge case: nu = [rho > rho_th],
    S = sum w nu, Psi with the Bernoulli(exp(-rho_th)) mean and variance."""
    kv = {row[0]: row[1:] for row in _read_rows("number_count_case.txt")}
    th = float(kv["rho_th"][0])
    S, W1, W2, Psi = _band_edge_case(rho_th=th)
    assert S == float(kv["S"][0])
    assert W1 == pytest.approx(float(kv["W1"][0]), rel=1e-12)
    assert W2 == pytest.approx(float(kv["W2"][0]), rel=1e-12)
    q = math.exp(-th)
    assert Psi == pytest.approx((0.75 - q * 2.75) / math.sqrt(q * (1 - q) * 4.3125), rel=1e-12)


def test_number_count_threshold_is_strict_in_double():
    """rho equal to rho_th counts 0 and the compare is made in double: a
    threshold one double ulp below the float power 3.01f counts it."""
    r301 = float(np.float32(3.01))
    assert _band_edge_case(rho_th=r301)[0] == 0.25               # 3.01f == rho_th: not counted
    assert _band_edge_case(rho_th=math.nextafter(r301, 0.0))[0] == 0.75
    r61 = float(np.float32(6.1))                                  # 6.0999999046..., below 6.1
    assert _band_edge_case(rho_th=6.1)[0] == 0.0
    assert _band_edge_case(rho_th=r61)[0] == 0.0
    assert _band_edge_case(rho_th=math.nextafter(r61, 0.0))[0] == 0.25


def test_number_count_noise_mean_zero_variance_one():
    """Under Exp(1) noise nu is Bernoulli(exp(-rho_th)): the weighted count's
    Psi has mean 0 and variance 1 over disjoint tracks (binomial moments)."""
    vals = []
    r = syn.rng(23)
    n_seg, n_bin = 48, 2048
    t = syn.segment_times(n_seg, 32.0)
    T0 = t[0] - 16.0
    vel = np.zeros((1, n_seg, 3))
    f0 = 510.0 + 1.25 * np.arange(48)
    tau = np.full(f0.shape, 35000.0)
    n = np.full(f0.shape, 5.0)
    for _ in range(300):
        rho = syn.exponential_noise(r, (1, n_seg, n_bin))
        w = syn.uniform_weights(r, 1, n_seg, 0.2, 2.0)
        vals.append(oracle.search_stats(rho, 500.0, 1 / 32, t, w, vel, np.array([[0, 0, 1.0]]),
                                        f0, tau, n, T0, rho_th=1.6)[3].ravel())
    v = np.concatenate(vals)
    N = v.size
    assert abs(v.mean()) < 4.0 / math.sqrt(N)
    assert abs(v.var() - 1.0) < 4.0 * math.sqrt(3.0 / N)


def test_number_count_is_the_power_sum_of_the_thresholded_map():
    """S and W of the count equal the power statistic of the 0/1 map [rho > rho_th]
    (brute-force threshold in numpy), with and without the amplitude weight."""
    p = syn.config_small(seed=24, n_seg=40, n_bin=1024, n_f0=6, n_tau=3, snr=8, weights=True)
    nu = (p.rho.astype(np.float64) > 1.6).astype(np.float32)
    for amp in (0, 4):
        a = oracle.search_stats(p.rho, p.f_min, p.df, p.t_mid, p.weights, p.velocity, p.nhat,
                                p.bank.f0, p.bank.tau, p.bank.n, p.T0, amp_power=amp, rho_th=1.6)
        b = oracle.search_stats(nu, p.f_min, p.df, p.t_mid, p.weights, p.velocity, p.nhat,
                                p.bank.f0, p.bank.tau, p.bank.n, p.T0, amp_power=amp)
        for x, y in zip(a[:3], b[:3]):
            np.testing.assert_array_equal(x, y)
        q = math.exp(-1.6)
        fin = b[2] > 0
        np.testing.assert_allclose(a[3][fin], (b[0][fin] - q * b[1][fin]) / np.sqrt(q * (1 - q) * b[2][fin]),
                                   rtol=1e-13, atol=1e-13)


def test_two_bin_fixture():
    """Two-bin lookups on the hand-computed band-edge case: the pair floor(x),
    floor(x) + 1 (not the nearest bin), both in band; Eq. 4 with 2 W1, 2 W2."""
    kv = {row[0]: row[1:] for row in _read_rows("two_bin_case.txt")}
    S, W1, W2, Psi = _band_edge_case(track_bins=2)
    ex = float(kv["S"][0])
    assert S == pytest.approx(ex, rel=1e-6)                        # float32 powers
    assert W1 == pytest.approx(float(kv["W1"][0]), rel=1e-12)
    assert W2 == pytest.approx(float(kv["W2"][0]), rel=1e-12)
    assert Psi == pytest.approx((ex - 2 * 2.75) / math.sqrt(2 * 4.3125), rel=1e-6)
    # the pair must lie in the band: x = 15.3 in a 16-bin band
    f0 = float(kv["edge_f0"][0])
    rho = np.zeros((1, 1, 16), np.float32)
    rho[0, 0] = 1 + np.arange(16) / 100.0
    args = (90.0, 1.0, np.array([5000.0]), None, np.zeros((1, 1, 3)), np.array([[0.0, 0.0, 1.0]]),
            [f0], [1000.0], [3.0], 5000.0)
    one = oracle.search_stats(rho, *args)
    two = oracle.search_stats(rho, *args, track_bins=2)
    assert one[0][0, 0] == pytest.approx(float(kv["edge_S1"][0]), rel=1e-6)
    assert two[2][0, 0] == 0.0 and two[3][0, 0] == -math.inf


def test_two_bin_noise_mean_zero_variance_one():
    """Two independent Exp(1) bins per lookup: Psi with mean 2 W1 and variance
    2 W2 has mean 0 and variance 1 under noise (power and count)."""
    r = syn.rng(25)
    n_seg, n_bin = 48, 2048
    t = syn.segment_times(n_seg, 32.0)
    T0 = t[0] - 16.0
    vel = np.zeros((1, n_seg, 3))
    f0 = 510.0 + 1.25 * np.arange(48)
    tau = np.full(f0.shape, 35000.0)
    n = np.full(f0.shape, 5.0)
    for kw in ({}, {"rho_th": 1.6}):
        vals = []
        for _ in range(300):
            rho = syn.exponential_noise(r, (1, n_seg, n_bin))
            w = syn.uniform_weights(r, 1, n_seg, 0.2, 2.0)
            vals.append(oracle.search_stats(rho, 500.0, 1 / 32, t, w, vel, np.array([[0, 0, 1.0]]),
                                            f0, tau, n, T0, track_bins=2, **kw)[3].ravel())
        v = np.concatenate(vals)
        N = v.size
        assert abs(v.mean()) < 4.0 / math.sqrt(N), kw
        assert abs(v.var() - 1.0) < 4.0 * math.sqrt(3.0 / N), kw


def test_pre_T0_segments_are_dropped():
    """Statistic with T0 mid-way equals the statistic of the map cut at T0."""
    p = syn.config_small(seed=11, n_seg=64, n_bin=1024, n_f0=4, n_tau=4, snr=0, weights=True)
    cut = 20
    T0 = p.t_mid[cut] - 1.0
    full = oracle.search_stats(p.rho, p.f_min, p.df, p.t_mid, p.weights, p.velocity,
                               p.nhat, p.bank.f0, p.bank.tau, p.bank.n, T0)
    part = oracle.search_stats(p.rho[:, cut:], p.f_min, p.df, p.t_mid[cut:],
                               p.weights[:, cut:], p.velocity[:, cut:], p.nhat,
                               p.bank.f0, p.bank.tau, p.bank.n, T0)
    for a, b in zip(full, part):
        np.testing.assert_allclose(a, b, rtol=1e-14)


# ------------------------------------------------------------ Eq. 4 -------
def test_psi_invariant_under_weight_scaling():
    """Psi = (S - W1)/sqrt(W2) is unchanged by w -> c w; a wrong mean or sigma is not."""
    p = syn.config_small(seed=12, n_seg=64, n_bin=1024, n_f0=8, n_tau=4, snr=0, weights=True)
    a = oracle.search_stats(p.rho, p.f_min, p.df, p.t_mid, p.weights, p.velocity,
                            p.nhat, p.bank.f0, p.bank.tau, p.bank.n, p.T0)[3]
    b = oracle.search_stats(p.rho, p.f_min, p.df, p.t_mid, p.weights * np.float32(4.0),
                            p.velocity, p.nhat, p.bank.f0, p.bank.tau, p.bank.n, p.T0)[3]
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)


def test_pure_noise_mean_zero_variance_one():
    """Sum of N unit-mean exponential powers has mean N and variance N: with
    weights, Psi over independent noise has mean 0 and variance 1 (Eq. 4)."""
    vals = []
    r = syn.rng(13)
    n_seg, n_bin = 48, 2048
    t = syn.segment_times(n_seg, 32.0)
    T0 = t[0] - 16.0
    vel = np.zeros((1, n_seg, 3))
    f0 = 510.0 + 1.25 * np.arange(48)        # 40 bins apart: disjoint tracks
    tau = np.full(f0.shape, 35000.0)
    n = np.full(f0.shape, 5.0)
    for _ in range(300):
        rho = syn.exponential_noise(r, (1, n_seg, n_bin))
        w = syn.uniform_weights(r, 1, n_seg, 0.2, 2.0)
        vals.append(oracle.search_stats(rho, 500.0, 1 / 32, t, w, vel,
                                        np.array([[0, 0, 1.0]]), f0, tau, n, T0)[3].ravel())
    v = np.concatenate(vals)
    N = v.size
    assert abs(v.mean()) < 4.0 / math.sqrt(N)
    assert abs(v.var() - 1.0) < 4.0 * math.sqrt(2.3 / N)


# ------------------------------------------------------------- top-k ------
def test_topk_matches_exact_sort_with_ties():
    r = syn.rng(14)
    psi = np.round(r.normal(size=(5, 3000)), 1)      # many exact ties
    psi[0, :] = 1.0
    psi[1, 10] = np.inf
    psi[2, :50] = -np.inf
    idx, val = oracle.topk(psi, 100)
    for row in range(psi.shape[0]):
        ref = sorted(range(psi.shape[1]), key=lambda b: (-psi[row, b], b))[:100]
        assert list(idx[row]) == ref
        np.testing.assert_array_equal(val[row], psi[row, ref])


# --------------------------------------------------------- injection -----
def test_injected_signal_peaks_at_true_template_and_sky():
    """A track synthesised by ODE + arrival-delay Doppler peaks at its own
    template (Sec. 3: exact tracks give the maximum sensitivity), beats the
    noise-only maximum (detection rule of Sec. 3), and the wrong sky loses."""
    p = syn.config_small(seed=15, snr=10.0)
    inj = p.injections[0]
    sky = np.vstack([inj.nhat, -inj.nhat])
    S, W1, W2, Psi = oracle.search_stats(p.rho, p.f_min, p.df, p.t_mid, p.weights,
                                         p.velocity, sky, p.bank.f0, p.bank.tau,
                                         p.bank.n, p.T0)
    best = int(np.argmax(Psi[0]))
    xb = oracle.track_coordinates(1, p.f_min, p.df, p.t_mid, p.velocity, sky,
                                  p.bank.f0, p.bank.tau, p.bank.n, p.T0,
                                  [[0, best], [0, inj.template]])
    kb = np.floor(xb + 0.5)
    same = np.array_equal(kb[0], kb[1])
    assert best == inj.template or same
    assert Psi[0].max() > 6.0
    assert Psi[0, inj.template] > Psi[1, inj.template] + 3.0
    noise = syn.config_small(seed=16, snr=0)
    Pn = oracle.search_stats(noise.rho, p.f_min, p.df, p.t_mid, None, noise.velocity,
                             sky[:1], p.bank.f0, p.bank.tau, p.bank.n, p.T0)[3]
    assert Psi[0].max() > Pn.max()


def test_high_precision_bins_agree_outside_tie_band():
    """FP64 bin indices equal a 40-digit recomputation except within 2^-30 of a tie."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    p = syn.config_small(seed=17, n_seg=32, n_bin=4096, n_f0=4, n_tau=4, snr=0, n_sky=3)
    pairs = [(s, b) for s in range(3) for b in range(0, len(p.bank), 7)]
    x = oracle.track_coordinates(1, p.f_min, p.df, p.t_mid, p.velocity, p.nhat,
                                 p.bank.f0, p.bank.tau, p.bank.n, p.T0, pairs)
    c = mp.mpf(299792458)
    checked = 0
    for i, (s, b) in enumerate(pairs):
        f0, tau, n = (mp.mpf(float(a)) for a in (p.bank.f0[b], p.bank.tau[b], p.bank.n[b]))
        for j in range(p.t_mid.size):
            t = mp.mpf(float(p.t_mid[j])) - mp.mpf(float(p.T0))
            f = f0 * mp.power(t / tau + 1, 1 / (1 - n))
            vn = sum(mp.mpf(float(p.velocity[0, j, a])) * mp.mpf(float(p.nhat[s, a]))
                     for a in range(3))
            xe = (f * (1 + vn / c) - mp.mpf(float(p.f_min))) / mp.mpf(float(p.df))
            fr = xe - mp.floor(xe)
            if abs(fr - mp.mpf(0.5)) <= mp.mpf(2) ** -30:
                continue
            assert math.floor(x[i, 0, j] + 0.5) == int(mp.floor(xe + mp.mpf(0.5)))
            checked += 1
    assert checked > 1000
