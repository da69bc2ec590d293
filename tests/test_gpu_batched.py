"""GPU parity of the batched search (many events, one persistent launch per
wave, replayed as a CUDA graph, shapes from the autotuner) against the FP64
oracle, event by event, through the C ABI.

The batches mix uneven segment counts (several 32-segment tiles and ragged
tails), per-event T0 inside the data, a sky list longer than one 1024-sky
chunk, a bank that crosses both band edges, FP16 and FP32 maps, one and two
detectors, unit and non-unit weights.
"""
import numpy as np
import pytest

import oracle
import paper_2507_07816_gb300 as tcw
import tcw_synth as syn
from _parity import REL, assert_topk_matches_oracle

pytestmark = pytest.mark.gpu


def make_batch(seed, n_det, dtype, weights, sky_sizes, n_tmpl=120, n_bin=800):
    events, _ = syn.config_batched(seed=seed, n_events=len(sky_sizes), n_seg_range=(33, 150),
                                   n_bin=n_bin, sky_range=(10, 40), n_tmpl=8, n_det=n_det,
                                   dtype=dtype, weights=weights, snr=12.0)
    r = syn.rng(seed + 1)
    f_min, df = events[0].f_min, events[0].df
    bank = syn.random_bank(r, n_tmpl, f0_range=(f_min - 5.0, f_min + n_bin * df + 5.0),
                           tau_range=(3500.0, 35000.0))
    # the injected templates join the bank so that the signals are present
    inj = [e.injections[0] for e in events]
    bank = syn.Bank(np.concatenate([bank.f0, [i.f0 for i in inj]]),
                    np.concatenate([bank.tau, [i.tau for i in inj]]),
                    np.concatenate([bank.n, [i.n for i in inj]]))
    out = []
    for e, S in zip(events, sky_sizes):
        nhat = syn.random_sky(r, S)
        nhat[0] = e.injections[0].nhat
        e.nhat = nhat
        e.bank = bank
        out.append(e)
    return out, bank


def oracle_event(e, bank):
    rho = np.asarray(e.rho, np.float64)
    return oracle.search_stats(rho, e.f_min, e.df, e.t_mid, e.weights, e.velocity, e.nhat,
                               bank.f0, bank.tau, bank.n, e.T0)


def run_batched(events, bank, k, options=()):
    s = tcw.Search(0)
    for opt, val in options:
        s.set_option(opt, val)
    s.define_bank(bank.f0, bank.tau, bank.n, 0.0)
    s.load_events(events, events[0].f_min, events[0].df)
    val, idx = s.search_batched(k)
    return s, val, idx


def check_against_oracle(events, bank, val, idx, k):
    row = 0
    for e in events:
        S = e.nhat.shape[0]
        oS, oW1, oW2, oP = oracle_event(e, bank)
        assert_topk_matches_oracle(idx[row:row + S], val[row:row + S], oP, oS, oW2, k)
        row += S
    assert row == idx.shape[0]


def test_batched_f16_one_detector_autotuned():
    events, bank = make_batch(71, 1, np.float16, False, [37, 1100, 5, 260, 64])
    k = 12
    s, val, idx = run_batched(events, bank, k)
    check_against_oracle(events, bank, val, idx, k)
    info = s.batch_info()
    assert info["n_events"] == len(events)
    assert info["autotuned"] == 1 and info["n_candidates"] >= 3
    assert info["waves"] == 1
    assert info["graph_kernels"] >= 2 * len(events) + 1
    assert info["lookups"] == sum(e.nhat.shape[0] * len(bank) * e.rho.shape[1] for e in events)
    tune = s.tune_results()
    assert len(tune) == info["n_candidates"]
    assert all(r > 0 for _, _, r in tune)
    assert (info["bank_chunk"], info["tile_segments"]) in [(b, t) for b, t, _ in tune]
    # the injected signal of each event is its sky 0's best template
    row = 0
    for i, e in enumerate(events):
        b = len(bank) - len(events) + i
        assert b in idx[row, :3].tolist() or e.injections[0].bins.max() < 0
        row += e.nhat.shape[0]
    s.close()


def test_batched_f32_two_detectors_weighted_fixed_shape():
    events, bank = make_batch(72, 2, np.float32, True, [90, 17, 300, 1])
    k = 7
    s, val, idx = run_batched(events, bank, k,
                              options=[(tcw.OPT_AUTOTUNE, 0), (tcw.OPT_BANK_CHUNK, 4),
                                       (tcw.OPT_TILE_SEGMENTS, 16)])
    check_against_oracle(events, bank, val, idx, k)
    info = s.batch_info()
    assert info["autotuned"] == 0 and info["bank_chunk"] == 4 and info["tile_segments"] == 16
    s.close()


def test_batched_replay_waves_and_shapes_agree():
    events, bank = make_batch(73, 1, np.float32, False, [200, 45, 1030])
    k = 9
    s, val, idx = run_batched(events, bank, k, options=[(tcw.OPT_AUTOTUNE, 0), (tcw.OPT_SKY_LANES, 64)])
    # a replay of the recorded graph is bit-identical
    val2, idx2 = s.search_batched(k)
    np.testing.assert_array_equal(val, val2)
    np.testing.assert_array_equal(idx, idx2)
    # the same batch split into one wave per event: same arithmetic per pair
    s.set_option(tcw.OPT_BATCH_MEMORY, 1 << 20)
    val3, idx3 = s.search_batched(k)
    assert s.batch_info()["waves"] == len(events)
    np.testing.assert_array_equal(val, val3)
    np.testing.assert_array_equal(idx, idx3)
    # another work-item and tile shape: Psi within the parity tolerance
    s.set_option(tcw.OPT_BATCH_MEMORY, 1 << 34)
    s.set_option(tcw.OPT_BANK_CHUNK, 64)
    s.set_option(tcw.OPT_TILE_SEGMENTS, 64)
    val4, idx4 = s.search_batched(k)
    check_against_oracle(events, bank, val4, idx4, k)
    np.testing.assert_allclose(val4, val, rtol=0, atol=REL * 50 + 1e-5)
    s.close()


def test_batched_errors():
    events, bank = make_batch(74, 1, np.float32, False, [20, 30])
    s = tcw.Search(0)
    s.define_bank(bank.f0, bank.tau, bank.n, 0.0)
    s.batch_sky = [20]
    with pytest.raises(tcw.TcwError) as e:
        s.search_batched(3)
    assert e.value.status == -4    # no events loaded
    bad = events[1].nhat.copy()
    bad[2] *= 1.001
    events[1].nhat = bad
    with pytest.raises(tcw.TcwError) as e:
        s.load_events(events, events[0].f_min, events[0].df)
    assert e.value.status == -1 and "event 1" in str(e.value)
    s.close()
