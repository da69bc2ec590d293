"""The seeded input generator: a batch of injections made at once equals the
same injections made one by one (the density study relies on the vectorised
path), and injected power sits on the signal's bins."""
import numpy as np

import tcw_synth as syn


def _setup(seed):
    r = syn.rng(seed)
    n_seg, n_bin, t_sft = 300, 4096, 8.0
    t = syn.segment_times(n_seg, t_sft)
    T0 = t[0] - 4.0
    dets = syn.random_detectors(r, 2)
    sky = syn.random_sky(r, 3)
    injs = [syn.Injection(f0, tau, n, sky[i], snr)
            for i, (f0, tau, n, snr) in enumerate([(900.0, 1e4, 5.0, 8.0), (905.5, 3500.0, 3.0, 12.0),
                                                   (950.0, 35000.0, 7.0, 6.0)])]
    return t, T0, dets, injs, (2, n_seg, n_bin)


def test_inject_many_equals_inject_one_by_one():
    t, T0, dets, injs, shape = _setup(5)
    w = syn.uniform_weights(syn.rng(6), 2, shape[1])
    a = syn.exponential_noise(syn.rng(7), shape)
    b = a.copy()
    ra, rb = syn.rng(8), syn.rng(8)
    syn.inject_many(ra, a, injs, dets, t, T0, 800.0, 1 / 8, w)
    for inj in injs:
        syn.inject(rb, b, inj, dets, t, T0, 800.0, 1 / 8, w)
    np.testing.assert_allclose(a, b, rtol=1e-6, atol=1e-6)


def test_injected_power_sits_on_the_track():
    t, T0, dets, injs, shape = _setup(9)
    rho = np.zeros(shape, np.float32)
    syn.inject_many(syn.rng(10), rho, injs[:1], dets, t, T0, 800.0, 1 / 8)
    bins = injs[0].bins
    on = np.zeros(shape, bool)
    for d in range(shape[0]):
        ok = bins[d] >= 0
        on[d, np.nonzero(ok)[0], bins[d][ok]] = True
    assert np.all(rho[~on] == 0)              # nothing off the track
    assert rho[on].mean() > 1.0               # excess power on it (mean 1 + mu^2/2)
