"""GPU parity of two-bin lookups (TCW_OPT_TRACK_BINS = 2) against the FP64
oracle: each lookup sums the bins floor(x) and floor(x) + 1 that bracket the
track (both in band), and Eq. 4 takes 2 W1 and 2 W2.

Checked element by element and on the top-k for the group kernel (every
sky-chunk width, band edges, T0 inside the data, FP32 and FP16 maps, with the
number count and the amplitude weight), the per-lookup kernel, the recorded
lower bins (bit-exact outside the tie band), the batched graph path and a
generated bank.  Tolerances as in tests/_parity.py, with Psi's bound taken
for the doubled mean and variance.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2507_07816_gb300 as tcw
import tcw_synth as syn
from _parity import REL, TIE, assert_topk_consistent
from test_gpu_batched import make_batch
from test_gpu_parity import multi_problem

pytestmark = pytest.mark.gpu


def oracle_two(p, rho=None, **kw):
    return oracle.search_stats(p.rho if rho is None else rho, p.f_min, p.df, p.t_mid, p.weights, p.velocity,
                               p.nhat, p.bank.f0, p.bank.tau, p.bank.n, p.T0, track_bins=2, **kw)


def assert_close(gpu, ora, mean=1.0, var=1.0, where=""):
    """mean, var: <s> and sigma^2 per unit weight of one bin (power: 1, 1;
    count: q, q(1 - q)); two bins double both."""
    gS, gW1, gW2, gP = (np.asarray(x, np.float64) for x in gpu)
    oS, oW1, oW2, oP = ora
    assert np.all(np.abs(gS - oS) <= REL * oS + 1e-6), f"S {where}"
    assert np.all(np.abs(gW1 - oW1) <= REL * oW1 + 1e-6), f"W1 {where}"
    assert np.all(np.abs(gW2 - oW2) <= REL * oW2 + 1e-6), f"W2 {where}"
    fin = np.isfinite(oP)
    assert np.array_equal(fin, np.isfinite(gP)), f"Psi finiteness {where}"
    tol = (REL * (oS[fin] + 2 * mean * oW1[fin]) / np.sqrt(2 * var * oW2[fin])
           + REL * np.abs(oP[fin]) + 1e-5)
    err = np.abs(gP[fin] - oP[fin])
    assert np.all(err <= tol), f"Psi {where}: max err {err.max()}"


def run_two(p, kernel=tcw.KERNEL_AUTO, lanes=0, amp=0, rho_th=None, k=10):
    s = tcw.Search(0)
    s.set_option(tcw.OPT_KERNEL, kernel)
    s.set_option(tcw.OPT_KEEP_STATS, 1)
    s.set_option(tcw.OPT_SKY_LANES, lanes)
    s.set_option(tcw.OPT_AMPLITUDE_POWER, amp)
    s.set_option(tcw.OPT_TRACK_BINS, 2)
    if rho_th is not None:
        s.set_statistic(tcw.STAT_NUMBER_COUNT, rho_th)
    s.load_problem(p)
    val, idx = s.search(k)
    return s, val, idx, s.statistics()


def check(p, rho_for_oracle=None, amp=0, rho_th=None, k=10, **kw):
    s, val, idx, st = run_two(p, amp=amp, rho_th=rho_th, k=k, **kw)
    stat = {} if rho_th is None else {"rho_th": rho_th}
    ora = oracle_two(p, rho=rho_for_oracle, amp_power=amp, **stat)
    q = 1.0 if rho_th is None else math.exp(-rho_th)
    mean, var = (1.0, 1.0) if rho_th is None else (q, q * (1 - q))
    assert_close((st["S"], st["W1"], st["W2"], st["psi"]), ora, mean, var, where="two-bin")
    assert_topk_consistent(st["psi"], idx, val, k)
    return s, val, idx, ora


def topk_matches(idx, val, ora, k, mean=1.0, var=1.0):
    """Top-k sets equal the oracle's except within tolerance of the k-th value."""
    oS, oW1, oW2, oP = ora
    o_idx, o_val = oracle.topk(oP, k)
    for r in range(idx.shape[0]):
        tol = (REL * (oS[r] + 2 * mean * oW1[r]) / np.sqrt(np.maximum(2 * var * oW2[r], 1e-300))
               + REL * np.abs(np.where(np.isfinite(oP[r]), oP[r], 0)) + 1e-5)
        kth = o_val[r, k - 1]
        sure = set(o_idx[r][o_val[r] > kth + 2 * tol.max()].tolist())
        assert sure <= set(idx[r].tolist()), r
        fin = np.isfinite(val[r])
        assert np.all(np.abs(val[r][fin] - oP[r, idx[r][fin]]) <= tol[idx[r][fin]]), r


@pytest.mark.parametrize("lanes", [16, 32, 64])
def test_group_kernel_two_bins(lanes):
    p = multi_problem(seed=131, n_sky=300, n_tmpl=300, n_seg=90)
    s, val, idx, ora = check(p, kernel=tcw.KERNEL_GROUP, lanes=lanes)
    assert s.info().kernel == tcw.KERNEL_GROUP and s.info().general_path_lanes > 0
    topk_matches(idx, val, ora, 10)
    s.close()


def test_T0_inside_fp16_count_and_amplitude():
    check(multi_problem(seed=132, t0_shift=30), kernel=tcw.KERNEL_GROUP)
    p = multi_problem(seed=133, dtype=np.float16)
    check(p, rho_for_oracle=p.rho.astype(np.float32), kernel=tcw.KERNEL_GROUP)
    p = multi_problem(seed=134, n_det=1, dtype=np.float16)
    check(p, rho_for_oracle=p.rho.astype(np.float32), rho_th=1.6, kernel=tcw.KERNEL_GROUP)
    check(multi_problem(seed=135), amp=4, rho_th=1.0, kernel=tcw.KERNEL_GROUP)


def test_lookup_kernel_two_bins():
    p = multi_problem(seed=136, n_tmpl=200)
    s, _, _, _ = check(p, kernel=tcw.KERNEL_LOOKUP, amp=4)
    assert s.info().kernel == tcw.KERNEL_LOOKUP
    s.close()


@pytest.mark.parametrize("kernel", [tcw.KERNEL_GROUP, tcw.KERNEL_LOOKUP])
def test_recorded_lower_bins(kernel):
    p = multi_problem(seed=137, n_tmpl=150, n_sky=40)
    s, _, _, _ = run_two(p, kernel=kernel)
    bins = s.track_bins()
    r = syn.rng(8)
    pairs = np.stack([r.integers(0, p.nhat.shape[0], 2000), r.integers(0, len(p.bank), 2000)], 1)
    x = oracle.track_coordinates(p.rho.shape[0], p.f_min, p.df, p.t_mid, p.velocity, p.nhat,
                                 p.bank.f0, p.bank.tau, p.bank.n, p.T0, pairs)
    k = np.where(np.isfinite(x), np.floor(x), -1).astype(np.int64)
    k[(k < 0) | (k + 1 >= p.rho.shape[2])] = -1
    fr = x - np.floor(x)
    exact = ~np.isfinite(x) | ((fr > TIE) & (fr < 1 - TIE))
    got = bins[pairs[:, 0], pairs[:, 1]]
    assert np.array_equal(got[exact], k[exact])
    s.close()


def test_batched_and_generated_two_bins():
    events, bank = make_batch(138, 2, np.float16, True, [33, 150, 7])
    s = tcw.Search(0)
    s.set_option(tcw.OPT_TRACK_BINS, 2)
    s.define_bank(bank.f0, bank.tau, bank.n, 0.0)
    s.load_events(events, events[0].f_min, events[0].df)
    val, idx = s.search_batched(10)
    row = 0
    for e in events:
        S = e.nhat.shape[0]
        ora = oracle.search_stats(np.asarray(e.rho, np.float32), e.f_min, e.df, e.t_mid, e.weights, e.velocity,
                                  e.nhat, bank.f0, bank.tau, bank.n, e.T0, track_bins=2)
        topk_matches(idx[row:row + S], val[row:row + S], ora, 10)
        row += S
    s.close()
    # generated bank, streamed in chunks
    p = multi_problem(seed=139, n_sky=30, n_seg=60, n_tmpl=8)
    lo = (p.f_min - 3, 3500.0, 3.0)
    hi = (p.f_min + p.rho.shape[2] * p.df + 3, 35000.0, 7.0)
    sp = tcw.bank_spec(tcw.BANK_RANDOM, lo, hi, n_tmpl=1500, seed=4)
    s = tcw.Search(0)
    s.set_option(tcw.OPT_TRACK_BINS, 2)
    s.set_option(tcw.OPT_GEN_CHUNK, 512)
    s.load_spectrogram(p.rho, p.f_min, p.df, p.t_mid, p.weights)
    s.load_velocity(p.velocity)
    s.define_sky(p.nhat)
    val, idx = s.search_generated(sp, p.T0, 12)
    f0, tau, n = oracle.bank_templates(1, 0, 1500, lo, hi, seed=4)
    ora = oracle.search_stats(p.rho, p.f_min, p.df, p.t_mid, p.weights, p.velocity, p.nhat, f0, tau, n, p.T0,
                              track_bins=2)
    topk_matches(idx, val, ora, 12)
    s.close()


def test_option_range():
    s = tcw.Search(0)
    for bad in (0, 3, -1):
        with pytest.raises(tcw.TcwError):
            s.set_option(tcw.OPT_TRACK_BINS, bad)
    s.close()
