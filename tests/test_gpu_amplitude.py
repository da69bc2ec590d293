"""GPU parity of the amplitude-weighted statistic against the FP64 oracle.

With TCW_OPT_AMPLITUDE_POWER = p every lookup's weight w_{d,j} becomes
w_{d,j} (f(t_j)/f0)^p, the template's own amplitude evolution (Eq. 3: h0 ~ f^2,
so p = 4 for power).  Checked element by element (S, W1, W2, Psi) and on the
top-k for the group kernel (every sky-chunk width, FP32 and FP16 maps, unit
and per-segment weights, band edges, T0 inside the data), the per-lookup
kernel, the recorded-bins variant and the batched graph path (the triaged
search's exhaustive part is checked in test_gpu_triage.py).
"""
import numpy as np
import pytest

import oracle
import paper_2507_07816_gb300 as tcw
import tcw_synth as syn
from _parity import (assert_stats_close, assert_topk_consistent, assert_topk_matches_oracle,
                     oracle_bins, oracle_stats)
from test_gpu_batched import make_batch, run_batched
from test_gpu_parity import multi_problem

pytestmark = pytest.mark.gpu


def run_amp(p, amp, kernel=tcw.KERNEL_AUTO, lanes=0, k=10):
    s = tcw.Search(0)
    s.set_option(tcw.OPT_KERNEL, kernel)
    s.set_option(tcw.OPT_KEEP_STATS, 1)
    s.set_option(tcw.OPT_SKY_LANES, lanes)
    s.set_option(tcw.OPT_AMPLITUDE_POWER, amp)
    s.load_problem(p)
    val, idx = s.search(k)
    st = s.statistics()
    return s, val, idx, st


def check(p, amp, rho_for_oracle=None, k=10, **kw):
    s, val, idx, st = run_amp(p, amp, k=k, **kw)
    ora = oracle_stats(p, rho=rho_for_oracle, amp_power=amp)
    assert_stats_close((st["S"], st["W1"], st["W2"], st["psi"]), ora, where=f"amp {amp}")
    assert_topk_consistent(st["psi"], idx, val, k)
    assert_topk_matches_oracle(idx, val, ora[3], ora[0], ora[2], k)
    return s, ora


@pytest.mark.parametrize("lanes", [16, 32, 64])
def test_group_kernel_amplitude_power_4(lanes):
    p = multi_problem(seed=91, n_sky=300, n_tmpl=300, n_seg=90)
    s, ora = check(p, 4, kernel=tcw.KERNEL_GROUP, lanes=lanes)
    assert s.info().kernel == tcw.KERNEL_GROUP
    assert s.info().general_path_lanes > 0          # band-edge entries took the amplitude too
    plain = oracle_stats(p)
    assert np.all(ora[1] <= plain[1] + 1e-9)         # the weight decays with the track
    s.close()


def test_other_powers_and_unit_weights():
    p = multi_problem(seed=92, weights=False)
    check(p, 4, kernel=tcw.KERNEL_GROUP)
    p = multi_problem(seed=93, t0_shift=30)
    for amp in (1, 2, 8):
        check(p, amp, kernel=tcw.KERNEL_GROUP)


def test_fp16_map_and_one_detector():
    p = multi_problem(seed=94, n_det=1, dtype=np.float16)
    check(p, 4, rho_for_oracle=p.rho.astype(np.float32), kernel=tcw.KERNEL_GROUP)


def test_lookup_kernel():
    p = multi_problem(seed=95, n_tmpl=200)
    s, _ = check(p, 4, kernel=tcw.KERNEL_LOOKUP)
    assert s.info().kernel == tcw.KERNEL_LOOKUP


def test_recorded_bins_and_switching_back():
    p = multi_problem(seed=96, n_tmpl=150, n_sky=40)
    s, val, idx, st = run_amp(p, 4, kernel=tcw.KERNEL_GROUP)
    bins = s.track_bins()
    r = syn.rng(7)
    pairs = np.stack([r.integers(0, p.nhat.shape[0], 2000), r.integers(0, len(p.bank), 2000)], 1)
    ok, exact = oracle_bins(p, pairs)
    got = bins[pairs[:, 0], pairs[:, 1]]
    assert np.array_equal(got[exact], ok[exact])    # the weight never moves a track
    # amplitude off again on the same context: the plain statistic
    s.set_option(tcw.OPT_AMPLITUDE_POWER, 0)
    s.search(10)
    st0 = s.statistics()
    assert_stats_close((st0["S"], st0["W1"], st0["W2"], st0["psi"]), oracle_stats(p), where="amp 0")
    s.close()


def test_option_range():
    s = tcw.Search(0)
    for bad in (-1, 9, 100):
        with pytest.raises(tcw.TcwError):
            s.set_option(tcw.OPT_AMPLITUDE_POWER, bad)
    s.set_option(tcw.OPT_AMPLITUDE_POWER, 0)
    s.close()


def test_batched_graph_path():
    events, bank = make_batch(97, 2, np.float32, True, [33, 140, 9])
    k = 10
    s, val, idx = run_batched(events, bank, k, options=[(tcw.OPT_AMPLITUDE_POWER, 4)])
    row = 0
    for e in events:
        S = e.nhat.shape[0]
        oS, oW1, oW2, oP = oracle.search_stats(np.asarray(e.rho, np.float64), e.f_min, e.df, e.t_mid,
                                               e.weights, e.velocity, e.nhat, bank.f0, bank.tau,
                                               bank.n, e.T0, amp_power=4)
        assert_topk_matches_oracle(idx[row:row + S], val[row:row + S], oP, oS, oW2, k)
        row += S
    # the captured graph is re-recorded when the power changes
    s.set_option(tcw.OPT_AMPLITUDE_POWER, 0)
    val0, idx0 = s.search_batched(k)
    row = 0
    for e in events:
        S = e.nhat.shape[0]
        oS, oW1, oW2, oP = oracle.search_stats(np.asarray(e.rho, np.float64), e.f_min, e.df, e.t_mid,
                                               e.weights, e.velocity, e.nhat, bank.f0, bank.tau,
                                               bank.n, e.T0)
        assert_topk_matches_oracle(idx0[row:row + S], val0[row:row + S], oP, oS, oW2, k)
        row += S
    s.close()
