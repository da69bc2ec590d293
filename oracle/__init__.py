"""Plain FP64 CPU oracle for the tCW template track statistic.

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with
the CUDA library in ``paper_2507_07816_gb300``; neither imports the other.

The arithmetic lives in ``tcw_oracle.c`` (plain loops, FP64, one ``pow`` per
lookup, see the header of that file for the equations and readings).  This
module compiles it with gcc and exposes it through ctypes, plus a few plain
numpy helpers for the parts that are not arithmetic of the search itself.

Functions and the passage each follows:
  track_frequency       Eq. 1
  doppler_frequency     Eq. 2
  bin_index             nearest-centre bin of the track (Sec. 2)
  search_stats          weighted track sum S, W1, W2 (Sec. 2) and Psi (Eq. 4)
  topk                  per-sky top-k by (Psi desc, index asc)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "tcw_oracle.c")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            d, i, i64, p = ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
            lib.oracle_track_frequency.restype = d
            lib.oracle_track_frequency.argtypes = [d, d, d, d, d]
            lib.oracle_doppler_frequency.restype = d
            lib.oracle_doppler_frequency.argtypes = [d, p, p]
            lib.oracle_bin_coordinate.restype = d
            lib.oracle_bin_coordinate.argtypes = [d, d, d]
            lib.oracle_bin_index.restype = i64
            lib.oracle_bin_index.argtypes = [d, d, d]
            lib.oracle_critical_ratio.restype = d
            lib.oracle_critical_ratio.argtypes = [d, d, d]
            lib.oracle_search_stats.restype = None
            lib.oracle_search_stats.argtypes = [
                p, i, i, i, d, d, p, p, p, p, i, p, p, p, i, d, p, i64,
                p, p, p, p, i]
            lib.oracle_search_stats_ext.restype = None
            lib.oracle_search_stats_ext.argtypes = [
                p, i, i, i, d, d, p, p, p, p, i, p, p, p, i, d, i, i, d, i, p, i64,
                p, p, p, p, i]
            lib.oracle_track_coordinates.restype = None
            lib.oracle_track_coordinates.argtypes = [
                i, i, d, d, p, p, p, p, p, p, d, p, i64, p]
            lib.oracle_topk.restype = None
            lib.oracle_topk.argtypes = [p, i64, i64, i64, p, p]
            lib.oracle_philox4x64_10.restype = None
            lib.oracle_philox4x64_10.argtypes = [p, p, p]
            lib.oracle_bank_templates.restype = None
            lib.oracle_bank_templates.argtypes = [i, i64, i64, i64, p, p, ctypes.c_uint64, i64, i64,
                                                  p, p, p]
            lib.oracle_max_threads.restype = i
            lib.oracle_max_threads.argtypes = []
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def track_frequency(f0, tau, n, T0, t) -> float:
    """Eq. 1 at one time."""
    return float(_load().oracle_track_frequency(f0, tau, n, T0, t))


def doppler_frequency(f, v, nhat) -> float:
    """Eq. 2 for one velocity (m/s) and one unit sky vector."""
    v = _c(v, np.float64)
    nhat = _c(nhat, np.float64)
    return float(_load().oracle_doppler_frequency(f, _ptr(v), _ptr(nhat)))


def bin_coordinate(fhat, f_min, df) -> float:
    return float(_load().oracle_bin_coordinate(fhat, f_min, df))


def bin_index(fhat, f_min, df) -> int:
    return int(_load().oracle_bin_index(fhat, f_min, df))


def critical_ratio(S, W1, W2) -> float:
    return float(_load().oracle_critical_ratio(S, W1, W2))


def search_stats(rho, f_min, df, t_mid, weights, velocity, nhat, f0, tau, n, T0,
                 pairs=None, nthreads=0, amp_power=0, rho_th=None, track_bins=1):
    """S, W1, W2, Psi for every (sky, template) pair.

    rho [D][Nseg][Nbin] float32 (float16 input is widened exactly);
    t_mid [Nseg]; weights [D][Nseg] or None; velocity [D][Nseg][3] (m/s);
    nhat [S][3]; f0/tau/n [B]; pairs [P][2] of (sky, template) or None for the
    full [S][B] grid.  amp_power > 0 multiplies every weight by
    (f(t_j)/f0)^amp_power, the template's own amplitude evolution (Eq. 3 gives
    4 for a power statistic).  rho_th (a float > 0) selects the number count
    instead of the power: nu = 1 where rho > rho_th, Psi with mean q*W1 and
    variance q(1-q)*W2, q = exp(-rho_th).  track_bins = 2 sums the two bins
    whose centres bracket the track (floor(x), floor(x) + 1, both in band),
    doubling the mean and variance of Eq. 4.  Returns four float64 arrays
    shaped [P] or [S][B].
    """
    rho = _c(np.asarray(rho).astype(np.float32, copy=False), np.float32)
    D, Nseg, Nbin = rho.shape
    t_mid = _c(t_mid, np.float64)
    weights = _c(weights, np.float32)
    velocity = _c(velocity, np.float64)
    nhat = _c(nhat, np.float64).reshape(-1, 3)
    f0, tau, n = (_c(a, np.float64) for a in (f0, tau, n))
    assert t_mid.shape == (Nseg,)
    assert velocity.shape == (D, Nseg, 3)
    assert weights is None or weights.shape == (D, Nseg)
    S_, B = nhat.shape[0], f0.shape[0]
    if pairs is None:
        shape, P, pp = (S_, B), 0, None
    else:
        pp = _c(pairs, np.int64).reshape(-1, 2)
        assert (pp[:, 0] >= 0).all() and (pp[:, 0] < S_).all()
        assert (pp[:, 1] >= 0).all() and (pp[:, 1] < B).all()
        shape, P = (pp.shape[0],), pp.shape[0]
    outs = [np.empty(shape, np.float64) for _ in range(4)]
    assert int(amp_power) >= 0
    assert rho_th is None or float(rho_th) > 0
    assert track_bins in (1, 2)
    _load().oracle_search_stats_ext(
        _ptr(rho), D, Nseg, Nbin, float(f_min), float(df), _ptr(t_mid),
        _ptr(weights), _ptr(velocity), _ptr(nhat), S_, _ptr(f0), _ptr(tau),
        _ptr(n), B, float(T0), int(amp_power), 0 if rho_th is None else 1,
        0.0 if rho_th is None else float(rho_th), int(track_bins), _ptr(pp), P, *(_ptr(o) for o in outs),
        int(nthreads))
    return tuple(outs)


def track_coordinates(D, f_min, df, t_mid, velocity, nhat, f0, tau, n, T0, pairs):
    """Bin coordinate x = (fhat - f_min)/df per (pair, detector, segment)."""
    t_mid = _c(t_mid, np.float64)
    Nseg = t_mid.shape[0]
    velocity = _c(velocity, np.float64)
    assert velocity.shape == (D, Nseg, 3)
    nhat = _c(nhat, np.float64).reshape(-1, 3)
    f0, tau, n = (_c(a, np.float64) for a in (f0, tau, n))
    pp = _c(pairs, np.int64).reshape(-1, 2)
    assert (pp[:, 0] < nhat.shape[0]).all() and (pp[:, 1] < f0.shape[0]).all()
    out = np.empty((pp.shape[0], D, Nseg), np.float64)
    _load().oracle_track_coordinates(
        D, Nseg, float(f_min), float(df), _ptr(t_mid), _ptr(velocity),
        _ptr(nhat), _ptr(f0), _ptr(tau), _ptr(n), float(T0), _ptr(pp),
        pp.shape[0], _ptr(out))
    return out


def topk(psi, k):
    """Per-row top-k of psi [rows][B] by (Psi desc, index asc)."""
    psi = _c(psi, np.float64)
    if psi.ndim == 1:
        psi = psi[None, :]
    rows, B = psi.shape
    assert 0 < k <= B
    idx = np.empty((rows, k), np.int64)
    val = np.empty((rows, k), np.float64)
    _load().oracle_topk(_ptr(psi), rows, B, k, _ptr(idx), _ptr(val))
    return idx, val


def philox4x64_10(counter, key):
    """Philox4x64-10 block (Salmon et al., SC 2011): four uint64 outputs."""
    c = np.ascontiguousarray(np.asarray(counter, np.uint64).reshape(4))
    k = np.ascontiguousarray(np.asarray(key, np.uint64).reshape(2))
    out = np.empty(4, np.uint64)
    _load().oracle_philox4x64_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def bank_templates(kind, first, count, lo, hi, n_f0=1, n_tau=1, n_n=1, seed=0):
    """Templates [first, first + count) of a lattice (kind 0) or uniform random
    (kind 1) bank over the box lo..hi = (f0, tau, n); three float64 arrays."""
    lo = np.ascontiguousarray(np.asarray(lo, np.float64).reshape(3))
    hi = np.ascontiguousarray(np.asarray(hi, np.float64).reshape(3))
    outs = [np.empty(int(count), np.float64) for _ in range(3)]
    _load().oracle_bank_templates(int(kind), int(n_f0), int(n_tau), int(n_n), _ptr(lo), _ptr(hi),
                                  int(seed), int(first), int(count), *(_ptr(o) for o in outs))
    return tuple(outs)
