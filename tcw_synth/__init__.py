"""Seeded synthetic inputs for the tCW track-statistic search.

This module is shared by the tests, the benchmark and the smoke check.  It
holds none of the search's arithmetic (no Eq. 1 closed form, no Eq. 2
Doppler factor applied to a template, no statistic): it only draws inputs.

* Detector motion: circular Earth orbit (1 AU, 1 sidereal-ish year of
  365.25 d) in the ecliptic, rotated to equatorial coordinates by the
  obliquity, plus diurnal rotation of 465 m/s x cos(latitude) at the sidereal
  rate.  Positions and velocities are both analytic; the velocity is the exact
  time derivative of the position.
* Sky: Fibonacci-sphere lattice (equal area for any count).
* Banks: cubic lattice and uniform random over (f0, tau, n) (Sec. 2 of the
  paper; parameter ranges from Sec. 1).
* Noise: whitened data, so normalized power is Exponential(1).
* Signals: the source frequency is obtained by integrating the braking law
  df/dt = -f^n / ((n-1) tau f0^(n-1)) with a fourth-order Runge-Kutta scheme,
  and the detector-frame frequency by multiplying with the time derivative of
  the arrival-time delay (r(t).nhat/c), taken by central differences of the
  detector POSITION.  Neither step evaluates the closed forms the search uses,
  so an injection recovered by the search is an independent check of them.
  Power in a signal bin is ((x + mu)^2 + y^2)/2 with x, y ~ N(0, 1), whose mean
  is 1 + mu^2/2; mu follows h0 ~ f^2 (Eq. 3).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

C_LIGHT = 299792458.0
AU = 1.495978707e11
YEAR = 365.25 * 86400.0
OBLIQUITY = math.radians(23.4393)
SIDEREAL_RATE = 7.2921159e-5
ROT_SPEED_EQ = 465.0                      # m/s at the equator
EARTH_RADIUS = ROT_SPEED_EQ / SIDEREAL_RATE
ORBIT_RATE = 2.0 * math.pi / YEAR
GPS_EPOCH0 = 1.4e9                        # start time used by the configs, s


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# --------------------------------------------------------------------------
# detector motion
# --------------------------------------------------------------------------
@dataclass
class Detector:
    latitude: float       # rad
    longitude: float      # rad (rotation phase at t = 0)
    orbit_phase: float    # rad (orbital phase at t = 0)

    def _ecl_to_eq(self, x, y, z):
        ce, se = math.cos(OBLIQUITY), math.sin(OBLIQUITY)
        return x, ce * y - se * z, se * y + ce * z

    def position(self, t):
        """Detector position w.r.t. the solar-system barycentre, m, [N][3]."""
        t = np.asarray(t, np.float64)
        a = ORBIT_RATE * t + self.orbit_phase
        ox, oy, oz = self._ecl_to_eq(AU * np.cos(a), AU * np.sin(a), 0.0 * a)
        b = SIDEREAL_RATE * t + self.longitude
        cl, sl = math.cos(self.latitude), math.sin(self.latitude)
        rx = EARTH_RADIUS * cl * np.cos(b)
        ry = EARTH_RADIUS * cl * np.sin(b)
        rz = EARTH_RADIUS * sl + 0.0 * b
        return np.stack([ox + rx, oy + ry, oz + rz], axis=-1)

    def velocity(self, t):
        """Exact time derivative of position(), m/s, [N][3]."""
        t = np.asarray(t, np.float64)
        a = ORBIT_RATE * t + self.orbit_phase
        vx, vy, vz = self._ecl_to_eq(-AU * ORBIT_RATE * np.sin(a),
                                     AU * ORBIT_RATE * np.cos(a), 0.0 * a)
        b = SIDEREAL_RATE * t + self.longitude
        cl = math.cos(self.latitude)
        rx = -EARTH_RADIUS * SIDEREAL_RATE * cl * np.sin(b)
        ry = EARTH_RADIUS * SIDEREAL_RATE * cl * np.cos(b)
        return np.stack([vx + rx, vy + ry, vz + 0.0 * b], axis=-1)


def random_detectors(r: np.random.Generator, count: int):
    """Detectors with seeded latitude/longitude; they share the orbital phase."""
    orb = r.uniform(0.0, 2.0 * math.pi)
    return [Detector(latitude=r.uniform(-1.0, 1.0), longitude=r.uniform(0.0, 2.0 * math.pi),
                     orbit_phase=orb) for _ in range(count)]


def segment_times(n_seg: int, t_sft: float, t_start: float = GPS_EPOCH0):
    """Segment mid-times t_start + (j + 1/2) T_SFT."""
    return t_start + (np.arange(n_seg, dtype=np.float64) + 0.5) * t_sft


# --------------------------------------------------------------------------
# sky and banks
# --------------------------------------------------------------------------
def fibonacci_sky(count: int):
    """Unit vectors on a Fibonacci-sphere lattice, [count][3]."""
    i = np.arange(count, dtype=np.float64) + 0.5
    z = 1.0 - 2.0 * i / count
    phi = i * math.pi * (3.0 - math.sqrt(5.0))
    rxy = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    v = np.stack([rxy * np.cos(phi), rxy * np.sin(phi), z], axis=-1)
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def random_sky(r: np.random.Generator, count: int):
    v = r.normal(size=(count, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


@dataclass
class Bank:
    f0: np.ndarray
    tau: np.ndarray
    n: np.ndarray

    def __len__(self):
        return int(self.f0.shape[0])

    def subset(self, idx):
        return Bank(self.f0[idx].copy(), self.tau[idx].copy(), self.n[idx].copy())


def lattice_bank(f0_values, tau_values, n_values) -> Bank:
    """Cubic lattice; f0 varies fastest, then tau, then n."""
    nn, tt, ff = np.meshgrid(np.asarray(n_values, np.float64),
                             np.asarray(tau_values, np.float64),
                             np.asarray(f0_values, np.float64), indexing="ij")
    return Bank(ff.ravel().copy(), tt.ravel().copy(), nn.ravel().copy())


def random_bank(r: np.random.Generator, count: int, f0_range=(500.0, 3000.0),
                tau_range=(3500.0, 35000.0), n_range=(3.0, 7.0)) -> Bank:
    """Uniform prior over the box (parameter ranges of Sec. 1)."""
    return Bank(r.uniform(*f0_range, size=count), r.uniform(*tau_range, size=count),
                r.uniform(*n_range, size=count))


# --------------------------------------------------------------------------
# data
# --------------------------------------------------------------------------
def exponential_noise(r: np.random.Generator, shape):
    return r.standard_exponential(size=shape, dtype=np.float32)


def uniform_weights(r: np.random.Generator, n_det: int, n_seg: int, lo=0.5, hi=1.5):
    return r.uniform(lo, hi, size=(n_det, n_seg)).astype(np.float32)


def spindown_frequency(f0, tau, n, T0, t, max_step=2.0):
    """Source frequency from RK4 integration of df/dt = -f^n/((n-1) tau f0^(n-1)).

    t must be sorted ascending; values with t < T0 are returned as NaN.
    """
    t = np.asarray(t, np.float64)
    out = np.full(t.shape, np.nan)
    k = f0 ** (1.0 - n) / ((n - 1.0) * tau)

    def rate(f):
        return -k * f ** n

    f, tc = float(f0), float(T0)
    for j, tj in enumerate(t):
        if tj < T0:
            continue
        span = tj - tc
        steps = max(1, int(math.ceil(span / max_step)))
        h = span / steps
        for _ in range(steps):
            k1 = rate(f)
            k2 = rate(f + 0.5 * h * k1)
            k3 = rate(f + 0.5 * h * k2)
            k4 = rate(f + h * k3)
            f += h * (k1 + 2.0 * k2 + 2.0 * k3 + k4) / 6.0
        tc = tj
        out[j] = f
    return out


def detector_frame_frequency(f_src, det: Detector, nhat, t, h=4.0):
    """Multiply by d/dt of the arrival-time delay r(t).nhat/c (central differences)."""
    t = np.asarray(t, np.float64)
    nhat = np.asarray(nhat, np.float64)
    dp = det.position(t + h) - det.position(t - h)
    rate = (dp @ nhat) / (2.0 * h * C_LIGHT)
    return f_src * (1.0 + rate)


def signal_bins(f_det, f_min, df, n_bin):
    """Bin whose centre f_min + k df is nearest the frequency; -1 when outside."""
    x = (np.asarray(f_det) - f_min) / df
    k = np.where(np.isfinite(x), np.rint(x), -1).astype(np.int64)
    k[(k < 0) | (k >= n_bin)] = -1
    return k


@dataclass
class Injection:
    f0: float
    tau: float
    n: float
    nhat: np.ndarray
    snr: float
    bins: np.ndarray = field(default=None)   # [D][Nseg], -1 = none


def inject(r: np.random.Generator, rho, injection: Injection, detectors, t, T0,
           f_min, df, weights=None):
    """Add one signal to rho in place and return its [D][Nseg] bin track.

    mu_j is proportional to (f_j/f0)^2 (h0 ~ f^2, Eq. 3) and scaled so that the
    expected excess of the weighted sum over its standard deviation is `snr`.
    """
    dd, jj, kk, val = injection_values(r, rho.shape, injection, detectors, t, T0, f_min, df, weights)
    if dd.size:
        rho[dd, jj, kk] = val.astype(rho.dtype)
    return injection.bins


def injection_values(r: np.random.Generator, shape, injection: Injection, detectors, t, T0,
                     f_min, df, weights=None):
    """The (detector, segment, bin) cells of one injected signal and their new
    powers ((x + mu)^2 + y^2)/2, x, y ~ N(0, 1); sets injection.bins."""
    D, n_seg, n_bin = shape
    f_src = spindown_frequency_many([injection.f0], [injection.tau], [injection.n], T0, t)[0]
    bins = np.full((D, n_seg), -1, np.int64)
    fdet = np.full((D, n_seg), np.nan)
    for d, det in enumerate(detectors):
        fd = detector_frame_frequency(f_src, det, injection.nhat, t)
        fdet[d] = fd
        bins[d] = signal_bins(fd, f_min, df, n_bin)
    ok = bins >= 0
    injection.bins = bins
    if not ok.any():
        e = np.zeros(0, np.int64)
        return e, e, e, np.zeros(0)
    w = np.ones((D, n_seg)) if weights is None else np.asarray(weights, np.float64)
    lam_shape = np.where(ok, (fdet / injection.f0) ** 4, 0.0)    # lambda_j ~ f^4
    lam_unit = (w * lam_shape).sum() / math.sqrt((w * w * ok).sum())
    lam0 = injection.snr / lam_unit
    mu = np.sqrt(2.0 * lam0 * lam_shape)
    dd, jj = np.nonzero(ok)
    x = r.normal(size=dd.shape[0])
    y = r.normal(size=dd.shape[0])
    return dd, jj, bins[dd, jj], ((x + mu[dd, jj]) ** 2 + y ** 2) / 2.0


# --------------------------------------------------------------------------
# workload configurations
# --------------------------------------------------------------------------
@dataclass
class Problem:
    rho: np.ndarray            # [D][Nseg][Nbin] float32 or float16
    t_mid: np.ndarray          # [Nseg]
    weights: np.ndarray        # [D][Nseg] float32 or None
    velocity: np.ndarray       # [D][Nseg][3]
    f_min: float
    df: float
    T0: float
    nhat: np.ndarray           # [S][3]
    bank: Bank
    injections: list
    detectors: list
    name: str = ""

    @property
    def shape(self):
        return self.rho.shape


def config_small(seed=20250711, n_det=1, n_seg=256, n_bin=4096, t_sft=32.0,
                 f_min=500.0, n_f0=64, n_tau=16, n_values=(3, 4, 5, 6, 7),
                 n_sky=1, snr=8.0, weights=False, inject_at=None):
    """Plain search, 1 detector, 256 x 4096 spectrogram, 5120-template lattice.

    df = 1/T_SFT; band 500-628 Hz; f0 lattice 560 + m 64/63 Hz, tau geometric
    in [3500, 35000] s, n in {3..7}; one injected track at a lattice point.
    """
    r = rng(seed)
    df = 1.0 / t_sft
    t = segment_times(n_seg, t_sft)
    T0 = t[0] - 0.5 * t_sft
    dets = random_detectors(r, n_det)
    vel = np.stack([d.velocity(t) for d in dets])
    rho = exponential_noise(r, (n_det, n_seg, n_bin))
    w = uniform_weights(r, n_det, n_seg) if weights else None
    f0s = 560.0 + np.arange(n_f0) * (64.0 / 63.0)
    taus = np.geomspace(3500.0, 35000.0, n_tau)
    bank = lattice_bank(f0s, taus, n_values)
    nhat = random_sky(r, n_sky)
    injections = []
    if snr and snr > 0:
        b = int(r.integers(0, len(bank))) if inject_at is None else int(inject_at)
        inj = Injection(float(bank.f0[b]), float(bank.tau[b]), float(bank.n[b]),
                        nhat[int(r.integers(0, n_sky))], snr)
        inject(r, rho, inj, dets, t, T0, f_min, df, w)
        inj.template = b
        injections.append(inj)
    return Problem(rho, t, w, vel, f_min, df, T0, nhat, bank, injections, dets,
                   name="plain-1det-256x4096-lattice5120")


def config_full(seed=20250712, n_det=2, n_seg=10000, n_bin=10000, t_sft=4.0,
                f_min=500.0, n_tmpl=200000, n_sky=1024, n_inj=10, snr=8.0,
                dtype=np.float32, weights=False):
    """Plain search, 2 detectors, 10000 x 10000 spectrogram (500-3000 Hz),
    2e5 uniform-random templates x 1024 Fibonacci sky directions, 10 injections."""
    r = rng(seed)
    df = 1.0 / t_sft
    t = segment_times(n_seg, t_sft)
    T0 = t[0] - 0.5 * t_sft
    dets = random_detectors(r, n_det)
    vel = np.stack([d.velocity(t) for d in dets])
    rho = exponential_noise(r, (n_det, n_seg, n_bin))
    w = uniform_weights(r, n_det, n_seg) if weights else None
    bank = random_bank(r, n_tmpl, f0_range=(f_min, f_min + n_bin * df))
    nhat = fibonacci_sky(n_sky)
    injections = []
    for _ in range(n_inj):
        b = int(r.integers(0, len(bank)))
        inj = Injection(float(bank.f0[b]), float(bank.tau[b]), float(bank.n[b]),
                        nhat[int(r.integers(0, n_sky))], snr)
        inject(r, rho, inj, dets, t, T0, f_min, df, w)
        inj.template = b
        injections.append(inj)
    if dtype != np.float32:
        rho = rho.astype(dtype)
    return Problem(rho, t, w, vel, f_min, df, T0, nhat, bank, injections, dets,
                   name=f"plain-{n_det}det-{n_seg}x{n_bin}-random{n_tmpl}-sky{n_sky}")


def config_batched(seed=20250714, n_events=64, n_seg_range=(2000, 20000), n_bin=10000,
                   sky_range=(256, 4096), n_tmpl=20000, n_det=1, t_sft=4.0, f_min=500.0,
                   dtype=np.float16, snr=8.0, weights=False, device=None):
    """Batched workload: events with uneven spectrograms, each with its own
    epoch, detector(s), signal start T0 (uniform in the first 10 % of its
    span), sky list and one injected track, all against one random bank.

    Returns (events, bank): events are Problems sharing `bank`.  With
    `device` (a torch CUDA device) the noise is drawn on that device by a
    seeded torch generator and rho is a CUDA tensor; otherwise numpy arrays.
    """
    r = rng(seed)
    df = 1.0 / t_sft
    bank = random_bank(r, n_tmpl, f0_range=(f_min, f_min + n_bin * df))
    events = []
    for i in range(n_events):
        n_seg = int(r.integers(n_seg_range[0], n_seg_range[1] + 1))
        t = segment_times(n_seg, t_sft, t_start=GPS_EPOCH0 + float(r.uniform(0.0, 3.0e7)))
        T0 = float(t[0] - 0.5 * t_sft + r.uniform(0.0, 0.1) * n_seg * t_sft)
        dets = random_detectors(r, n_det)
        vel = np.stack([d.velocity(t) for d in dets])
        n_sky = int(r.integers(sky_range[0], sky_range[1] + 1))
        nhat = random_sky(r, n_sky)
        w = uniform_weights(r, n_det, n_seg) if weights else None
        b = int(r.integers(0, n_tmpl))
        inj = Injection(float(bank.f0[b]), float(bank.tau[b]), float(bank.n[b]),
                        nhat[int(r.integers(0, n_sky))], snr)
        inj.template = b
        shape = (n_det, n_seg, n_bin)
        if device is None:
            rho = exponential_noise(r, shape)
            inject(r, rho, inj, dets, t, T0, f_min, df, w)
            if dtype != np.float32:
                rho = rho.astype(dtype)
        else:
            import torch
            g = torch.Generator(device=device)
            g.manual_seed(int(seed) * 1000 + i)
            rho = torch.empty(shape, dtype=torch.float32, device=device).exponential_(generator=g)
            dd, jj, kk, val = injection_values(r, shape, inj, dets, t, T0, f_min, df, w)
            if dd.size:
                idx = tuple(torch.as_tensor(a, device=device) for a in (dd, jj, kk))
                rho[idx] = torch.as_tensor(val, dtype=torch.float32, device=device)
            if dtype == np.float16:
                rho = rho.half()
        events.append(Problem(rho, t, w, vel, f_min, df, T0, nhat, bank, [inj], dets,
                              name=f"event{i}-{n_det}det-{n_seg}x{n_bin}-sky{n_sky}"))
    return events, bank


def spindown_frequency_many(f0, tau, n, T0, t, step=16.0):
    """Source frequency of K sources at the times t: RK4 of the braking law
    df/dt = -f^n/((n-1) tau f0^(n-1)) on a uniform grid of `step` seconds from
    T0, then cubic Hermite interpolation (values and ODE slopes) to t.
    Returns [K][len(t)], NaN before T0."""
    f0, tau, n = (np.asarray(a, np.float64).reshape(-1, 1) for a in (f0, tau, n))
    t = np.asarray(t, np.float64)
    out = np.full((f0.shape[0], t.shape[0]), np.nan)
    ok = t >= T0
    if not ok.any():
        return out
    k = f0 ** (1.0 - n) / ((n - 1.0) * tau)
    G = int(math.ceil((t[ok].max() - T0) / step)) + 1
    fg = np.empty((f0.shape[0], G + 1))
    f = f0[:, 0].copy()
    kk, nn = k[:, 0], n[:, 0]
    fg[:, 0] = f
    for g in range(G):
        k1 = -kk * f ** nn
        k2 = -kk * (f + 0.5 * step * k1) ** nn
        k3 = -kk * (f + 0.5 * step * k2) ** nn
        k4 = -kk * (f + step * k3) ** nn
        f = f + step * (k1 + 2.0 * k2 + 2.0 * k3 + k4) / 6.0
        fg[:, g + 1] = f
    dg = -k * fg ** n
    u = (t[ok] - T0) / step
    i = np.minimum(np.floor(u).astype(np.int64), G - 1)
    s_ = u - i
    h00 = (1 + 2 * s_) * (1 - s_) ** 2
    h10 = s_ * (1 - s_) ** 2
    h01 = s_ * s_ * (3 - 2 * s_)
    h11 = s_ * s_ * (s_ - 1)
    out[:, ok] = (h00 * fg[:, i] + h10 * step * dg[:, i] + h01 * fg[:, i + 1]
                  + h11 * step * dg[:, i + 1])
    return out


def inject_many(r: np.random.Generator, rho, injections, detectors, t, T0, f_min, df, weights=None):
    """inject() for many signals at once: the braking-law frequencies of all
    sources come from one vectorised integration; the cells of each signal
    are then set as inject() does (later signals overwrite shared cells)."""
    if not injections:
        return
    fsrc = spindown_frequency_many([i.f0 for i in injections], [i.tau for i in injections],
                                   [i.n for i in injections], T0, t)
    D, n_seg, n_bin = rho.shape
    w = np.ones((D, n_seg)) if weights is None else np.asarray(weights, np.float64)
    for i, inj in enumerate(injections):
        bins = np.full((D, n_seg), -1, np.int64)
        fdet = np.full((D, n_seg), np.nan)
        for d, det in enumerate(detectors):
            fd = detector_frame_frequency(fsrc[i], det, inj.nhat, t)
            fdet[d] = fd
            bins[d] = signal_bins(fd, f_min, df, n_bin)
        inj.bins = bins
        ok = bins >= 0
        if not ok.any():
            continue
        lam_shape = np.where(ok, (fdet / inj.f0) ** 4, 0.0)
        lam_unit = (w * lam_shape).sum() / math.sqrt((w * w * ok).sum())
        mu = np.sqrt(2.0 * (inj.snr / lam_unit) * lam_shape)
        dd, jj = np.nonzero(ok)
        x = r.normal(size=dd.shape[0])
        y = r.normal(size=dd.shape[0])
        rho[dd, jj, bins[dd, jj]] = (((x + mu[dd, jj]) ** 2 + y ** 2) / 2.0).astype(rho.dtype)


def training_event(seed, bank, n_det=2, n_seg=10000, n_bin=10000, n_sky=1024, t_sft=4.0,
                   f_min=500.0, n_inj=4, snr_range=(5.0, 12.0), device=None, dtype=np.float32):
    """One event for the learned triage: exponential noise (drawn on `device`
    by a seeded torch generator when given), `n_inj` injected tracks with
    templates drawn from `bank`, skies drawn from the event's Fibonacci sky
    and SNR uniform in snr_range.  Each injection records .template and .sky."""
    r = rng(seed)
    df = 1.0 / t_sft
    t = segment_times(n_seg, t_sft, t_start=GPS_EPOCH0 + float(r.uniform(0.0, 3.0e7)))
    T0 = float(t[0] - 0.5 * t_sft)
    dets = random_detectors(r, n_det)
    vel = np.stack([d.velocity(t) for d in dets])
    nhat = fibonacci_sky(n_sky)
    tb = r.integers(0, len(bank), n_inj)
    sk = r.integers(0, n_sky, n_inj)
    snr = r.uniform(snr_range[0], snr_range[1], n_inj)
    fsrc = spindown_frequency_many(bank.f0[tb], bank.tau[tb], bank.n[tb], T0, t)
    shape = (n_det, n_seg, n_bin)
    injections, cells = [], []
    for i in range(n_inj):
        inj = Injection(float(bank.f0[tb[i]]), float(bank.tau[tb[i]]), float(bank.n[tb[i]]),
                        nhat[sk[i]], float(snr[i]))
        inj.template, inj.sky = int(tb[i]), int(sk[i])
        bins = np.full((n_det, n_seg), -1, np.int64)
        fdet = np.full((n_det, n_seg), np.nan)
        for d, det in enumerate(dets):
            fd = detector_frame_frequency(fsrc[i], det, inj.nhat, t)
            fdet[d] = fd
            bins[d] = signal_bins(fd, f_min, df, n_bin)
        inj.bins = bins
        ok = bins >= 0
        if ok.any():
            lam_shape = np.where(ok, (fdet / inj.f0) ** 4, 0.0)
            lam_unit = lam_shape.sum() / math.sqrt(ok.sum())
            mu = np.sqrt(2.0 * (inj.snr / lam_unit) * lam_shape)
            dd, jj = np.nonzero(ok)
            x = r.normal(size=dd.shape[0])
            y = r.normal(size=dd.shape[0])
            cells.append((dd, jj, bins[dd, jj], ((x + mu[dd, jj]) ** 2 + y ** 2) / 2.0))
        injections.append(inj)
    if device is None:
        rho = exponential_noise(r, shape)
        for dd, jj, kk, val in cells:
            rho[dd, jj, kk] = val.astype(np.float32)
        if dtype != np.float32:
            rho = rho.astype(dtype)
    else:
        import torch
        g = torch.Generator(device=device)
        g.manual_seed(int(seed) % (2 ** 62))
        rho = torch.empty(shape, dtype=torch.float32, device=device).exponential_(generator=g)
        for dd, jj, kk, val in cells:
            idx = tuple(torch.as_tensor(a, device=device) for a in (dd, jj, kk))
            rho[idx] = torch.as_tensor(val, dtype=torch.float32, device=device)
        if dtype == np.float16:
            rho = rho.half()
    return Problem(rho, t, None, vel, f_min, df, T0, nhat, bank, injections, dets,
                   name=f"training-{n_det}det-{n_seg}x{n_bin}-sky{n_sky}")
