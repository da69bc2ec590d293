"""GPU parity of the number-count statistic against the FP64 oracle.

With tcw_set_statistic(TCW_STAT_NUMBER_COUNT, rho_th) the search sums
nu = [rho > rho_th] (decided in double on both sides, so bit-identical) and
Eq. 4 takes the Bernoulli mean q W1 and variance q(1-q) W2, q = exp(-rho_th).
Checked element by element (S, W1, W2, Psi) and on the top-k for the group
kernel (every sky-chunk width, band edges, T0 inside the data, FP16 maps whose
counts are staged as fp32), the per-lookup kernel, the amplitude weight,
threshold and statistic changes on one context, the batched graph path, and
the full-size workload on sampled pairs.

Tolerances: S, W1, W2 within 1e-5 relative (+1e-6); Psi within
1e-5 (S + q W1)/sqrt(q(1-q) W2) + 1e-5 |Psi| + 1e-5, the error of an fp32 sum
of terms of those sizes.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2507_07816_gb300 as tcw
import tcw_synth as syn
from _parity import REL, assert_topk_consistent, assert_topk_matches_oracle, oracle_stats
from test_gpu_batched import make_batch
from test_gpu_parity import multi_problem

pytestmark = pytest.mark.gpu

TH = 1.6


def assert_count_close(gpu, ora, rho_th, where=""):
    gS, gW1, gW2, gP = (np.asarray(x, np.float64) for x in gpu)
    oS, oW1, oW2, oP = ora
    assert np.all(np.abs(gS - oS) <= REL * oS + 1e-6), f"S {where}"
    assert np.all(np.abs(gW1 - oW1) <= REL * oW1 + 1e-6), f"W1 {where}"
    assert np.all(np.abs(gW2 - oW2) <= REL * oW2 + 1e-6), f"W2 {where}"
    fin = np.isfinite(oP)
    assert np.array_equal(fin, np.isfinite(gP)), f"Psi finiteness {where}"
    q = math.exp(-rho_th)
    tol = (REL * (oS[fin] + q * oW1[fin]) / np.sqrt(q * (1 - q) * oW2[fin])
           + REL * np.abs(oP[fin]) + 1e-5)
    err = np.abs(gP[fin] - oP[fin])
    assert np.all(err <= tol), f"Psi {where}: max err {err.max()}"


def assert_count_topk(idx, val, ora, rho_th, k):
    """Index sets equal the oracle's top-k except where the oracle's Psi lies
    within tolerance of the k-th value; returned Psi values match the oracle."""
    oS, oW1, oW2, oP = ora
    q = math.exp(-rho_th)
    o_idx, o_val = oracle.topk(oP, k)
    for r in range(idx.shape[0]):
        tol_r = (REL * (oS[r] + q * oW1[r]) / np.sqrt(np.maximum(q * (1 - q) * oW2[r], 1e-300))
                 + REL * np.abs(np.where(np.isfinite(oP[r]), oP[r], 0)) + 1e-5)
        kth = o_val[r, k - 1]
        sure = set(o_idx[r][o_val[r] > kth + 2 * tol_r.max()].tolist())
        got = set(idx[r].tolist())
        assert sure <= got, (r, sorted(sure - got))
        fin = np.isfinite(val[r])
        sel = idx[r][fin]
        assert np.all(np.abs(val[r][fin] - oP[r, sel]) <= tol_r[sel]), r


def run_count(p, rho_th=TH, kernel=tcw.KERNEL_AUTO, lanes=0, amp=0, k=10):
    s = tcw.Search(0)
    s.set_option(tcw.OPT_KERNEL, kernel)
    s.set_option(tcw.OPT_KEEP_STATS, 1)
    s.set_option(tcw.OPT_SKY_LANES, lanes)
    s.set_option(tcw.OPT_AMPLITUDE_POWER, amp)
    s.set_statistic(tcw.STAT_NUMBER_COUNT, rho_th)
    s.load_problem(p)
    val, idx = s.search(k)
    return s, val, idx, s.statistics()


def check(p, rho_th=TH, rho_for_oracle=None, k=10, amp=0, **kw):
    s, val, idx, st = run_count(p, rho_th, k=k, amp=amp, **kw)
    ora = oracle.search_stats(p.rho if rho_for_oracle is None else rho_for_oracle, p.f_min, p.df,
                              p.t_mid, p.weights, p.velocity, p.nhat, p.bank.f0, p.bank.tau,
                              p.bank.n, p.T0, amp_power=amp, rho_th=rho_th)
    assert_count_close((st["S"], st["W1"], st["W2"], st["psi"]), ora, rho_th, where=f"th {rho_th}")
    assert_topk_consistent(st["psi"], idx, val, k)
    assert_count_topk(idx, val, ora, rho_th, k)
    return s, ora


@pytest.mark.parametrize("lanes", [16, 32, 64])
def test_group_kernel_number_count(lanes):
    p = multi_problem(seed=101, n_sky=300, n_tmpl=300, n_seg=90)
    s, ora = check(p, kernel=tcw.KERNEL_GROUP, lanes=lanes)
    info = s.info()
    assert info.kernel == tcw.KERNEL_GROUP and info.general_path_lanes > 0
    # S counts exceedances: a weighted sum of 0/1, at most W1
    assert np.all(ora[0] <= ora[1] + 1e-9)
    s.close()


def test_T0_inside_unit_weights_and_amplitude():
    check(multi_problem(seed=102, t0_shift=35), kernel=tcw.KERNEL_GROUP)
    check(multi_problem(seed=103, weights=False), rho_th=0.7, kernel=tcw.KERNEL_GROUP)
    check(multi_problem(seed=104), amp=4, kernel=tcw.KERNEL_GROUP)


def test_fp16_map_counts_from_half_powers():
    p = multi_problem(seed=105, n_det=1, dtype=np.float16)
    check(p, rho_for_oracle=p.rho.astype(np.float32), kernel=tcw.KERNEL_GROUP)
    p = multi_problem(seed=106, dtype=np.float16)
    check(p, rho_th=2.25, rho_for_oracle=p.rho.astype(np.float32), kernel=tcw.KERNEL_GROUP)


def test_lookup_kernel_number_count():
    p = multi_problem(seed=107, n_tmpl=200)
    s, _ = check(p, kernel=tcw.KERNEL_LOOKUP, amp=4)
    assert s.info().kernel == tcw.KERNEL_LOOKUP


def test_threshold_and_statistic_changes_on_one_context():
    p = multi_problem(seed=108, n_tmpl=150, n_sky=40)
    s, val, idx, st = run_count(p, TH, kernel=tcw.KERNEL_GROUP)
    for th in (2.5, 0.25):
        s.set_statistic(tcw.STAT_NUMBER_COUNT, th)      # the bit map is rebuilt
        s.search(10)
        st = s.statistics()
        ora = oracle.search_stats(p.rho, p.f_min, p.df, p.t_mid, p.weights, p.velocity, p.nhat,
                                  p.bank.f0, p.bank.tau, p.bank.n, p.T0, rho_th=th)
        assert_count_close((st["S"], st["W1"], st["W2"], st["psi"]), ora, th, where=f"th {th}")
    # a new spectrogram on the same context: the bit map follows it
    p2 = multi_problem(seed=109, n_tmpl=150, n_sky=40)
    s.load_problem(p2)
    s.search(10)
    st = s.statistics()
    ora = oracle.search_stats(p2.rho, p2.f_min, p2.df, p2.t_mid, p2.weights, p2.velocity, p2.nhat,
                              p2.bank.f0, p2.bank.tau, p2.bank.n, p2.T0, rho_th=0.25)
    assert_count_close((st["S"], st["W1"], st["W2"], st["psi"]), ora, 0.25, where="reloaded")
    s.set_statistic(tcw.STAT_POWER)
    s.search(10)
    st = s.statistics()
    o = oracle_stats(p2)
    assert np.allclose(st["S"], o[0], rtol=REL, atol=1e-6)
    s.close()


def test_invalid_statistic_arguments():
    s = tcw.Search(0)
    for stat, th in ((tcw.STAT_NUMBER_COUNT, 0.0), (tcw.STAT_NUMBER_COUNT, -1.0),
                     (tcw.STAT_NUMBER_COUNT, float("nan")), (tcw.STAT_NUMBER_COUNT, float("inf")),
                     (7, 1.0)):
        with pytest.raises(tcw.TcwError):
            s.set_statistic(stat, th)
    s.set_statistic(tcw.STAT_POWER)
    s.close()


@pytest.mark.parametrize("dtype", [np.float16, np.float32])
def test_batched_number_count(dtype):
    events, bank = make_batch(110, 2 if dtype == np.float32 else 1, dtype, dtype == np.float32,
                              [33, 150, 7])
    k = 10
    s = tcw.Search(0)
    s.set_statistic(tcw.STAT_NUMBER_COUNT, TH)
    s.define_bank(bank.f0, bank.tau, bank.n, 0.0)
    s.load_events(events, events[0].f_min, events[0].df)
    for stat in ("count", "power", "count"):
        if stat == "power":
            s.set_statistic(tcw.STAT_POWER)
        else:
            s.set_statistic(tcw.STAT_NUMBER_COUNT, TH)
        val, idx = s.search_batched(k)
        row = 0
        for e in events:
            S = e.nhat.shape[0]
            rho = np.asarray(e.rho, np.float32)
            if stat == "count":
                ora = oracle.search_stats(rho, e.f_min, e.df, e.t_mid, e.weights, e.velocity, e.nhat,
                                          bank.f0, bank.tau, bank.n, e.T0, rho_th=TH)
                assert_count_topk(idx[row:row + S], val[row:row + S], ora, TH, k)
            else:
                ora = oracle.search_stats(rho, e.f_min, e.df, e.t_mid, e.weights, e.velocity, e.nhat,
                                          bank.f0, bank.tau, bank.n, e.T0)
                assert_topk_matches_oracle(idx[row:row + S], val[row:row + S], ora[3], ora[0], ora[2], k)
            row += S
    s.close()


def test_full_size_workload_sampled_pairs():
    """2 detectors x 10^4 x 10^4, 2e5 templates x 1024 skies, number count at
    rho_th = 1.6; oracle on sampled pairs and the injected templates."""
    p = syn.config_full()
    s, val, idx, st = run_count(p, TH, k=100)
    assert s.info().kernel == tcw.KERNEL_GROUP
    r = syn.rng(17)
    n = 400
    pairs = np.stack([r.integers(0, p.nhat.shape[0], n), r.integers(0, len(p.bank), n)], 1)
    extra = [(int(np.argmin(np.linalg.norm(p.nhat - inj.nhat, axis=1))), inj.template)
             for inj in p.injections]
    pairs = np.concatenate([pairs, np.array(extra)], 0)
    ora = oracle.search_stats(p.rho, p.f_min, p.df, p.t_mid, p.weights, p.velocity, p.nhat,
                              p.bank.f0, p.bank.tau, p.bank.n, p.T0, pairs=pairs, rho_th=TH)
    gpu = tuple(st[key][pairs[:, 0], pairs[:, 1]] for key in ("S", "W1", "W2", "psi"))
    assert_count_close(gpu, ora, TH, where="full-size sample")
    for sky in r.integers(0, p.nhat.shape[0], 4):
        assert_topk_consistent(st["psi"][sky:sky + 1], idx[sky:sky + 1], val[sky:sky + 1], 100)
    # the count also finds most injections at their own template and sky
    assert int(np.sum(ora[3][n:] > 4.0)) >= len(extra) // 2
    s.close()
