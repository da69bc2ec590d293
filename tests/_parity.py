"""Comparison helpers shared by the GPU parity tests.

Tolerances (statistics within 1e-5 relative, indices bit-exact):
  S   |S_gpu - S_ora| <= 1e-5 * sum|w rho| (= S_ora, every term is >= 0) + 1e-6
  W1  |W1_gpu - W1_ora| <= 1e-5 * W1_ora + 1e-6, same for W2
  Psi |Psi_gpu - Psi_ora| <= 1e-5 * S_ora / sqrt(W2_ora) + 1e-5   (Psi is near 0
      in noise, so a relative bound on it is meaningless)
  bins equal wherever the oracle's coordinate is farther than 2^-30 from a tie.
"""
import numpy as np

import oracle

REL = 1e-5
TIE = 2.0 ** -30


def oracle_stats(p, pairs=None, rho=None, nthreads=0, amp_power=0):
    return oracle.search_stats(p.rho if rho is None else rho, p.f_min, p.df, p.t_mid, p.weights,
                               p.velocity, p.nhat, p.bank.f0, p.bank.tau, p.bank.n, p.T0,
                               pairs=pairs, nthreads=nthreads, amp_power=amp_power)


def assert_stats_close(gpu, ora, where=""):
    gS, gW1, gW2, gP = (np.asarray(x, np.float64) for x in gpu)
    oS, oW1, oW2, oP = ora
    assert np.all(np.abs(gS - oS) <= REL * np.abs(oS) + 1e-6), f"S {where}: {np.max(np.abs(gS - oS) / (np.abs(oS) + 1e-12))}"
    assert np.all(np.abs(gW1 - oW1) <= REL * np.abs(oW1) + 1e-6), f"W1 {where}"
    assert np.all(np.abs(gW2 - oW2) <= REL * np.abs(oW2) + 1e-6), f"W2 {where}"
    fin = np.isfinite(oP)
    assert np.array_equal(fin, np.isfinite(gP)), f"Psi finiteness {where}"
    assert np.all(gP[~fin] == oP[~fin]), f"Psi -inf {where}"
    tol = REL * np.abs(oS[fin]) / np.sqrt(oW2[fin]) + 1e-5
    err = np.abs(gP[fin] - oP[fin])
    assert np.all(err <= tol), f"Psi {where}: max err {err.max()} tol {tol[np.argmax(err - tol)]}"


def oracle_bins(p, pairs):
    """Oracle bin index per (pair, det, seg) and a mask of lookups outside the tie band."""
    x = oracle.track_coordinates(p.rho.shape[0], p.f_min, p.df, p.t_mid, p.velocity, p.nhat,
                                 p.bank.f0, p.bank.tau, p.bank.n, p.T0, pairs)
    k = np.where(np.isfinite(x), np.floor(x + 0.5), -1).astype(np.int64)
    k[(k < 0) | (k >= p.rho.shape[2])] = -1
    fr = x - np.floor(x)
    exact = ~np.isfinite(x) | (np.abs(fr - 0.5) > TIE)
    return k, exact


def assert_topk_consistent(psi_full, idx, val, k):
    """GPU top-k equals an exact sort of the GPU's own Psi rows (bit-exact)."""
    ref_idx, ref_val = oracle.topk(psi_full.astype(np.float64), k)
    np.testing.assert_array_equal(idx, ref_idx)
    np.testing.assert_array_equal(val.astype(np.float64), ref_val)


def assert_topk_matches_oracle(idx, val, ora_psi, ora_S, ora_W2, k):
    """Index sets agree with the oracle's top-k except for entries whose oracle
    Psi lies within tolerance of the k-th value; returned Psi matches the oracle."""
    o_idx, o_val = oracle.topk(ora_psi, k)
    for r in range(idx.shape[0]):
        tol = REL * np.abs(ora_S[r]) / np.sqrt(np.maximum(ora_W2[r], 1e-30)) + 1e-5
        kth = o_val[r, -1]
        g = set(idx[r].tolist())
        o = set(o_idx[r].tolist())
        for b in g ^ o:
            assert abs(ora_psi[r, b] - kth) <= 2 * tol[b], (r, b, ora_psi[r, b], kth)
        fin = np.isfinite(ora_psi[r, idx[r]])
        err = np.abs(val[r][fin] - ora_psi[r, idx[r]][fin])
        assert np.all(err <= tol[idx[r]][fin]), (r, err.max())
