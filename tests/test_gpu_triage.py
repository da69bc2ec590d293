"""GPU parity of the learned sky triage against the FP64 oracle
(oracle/triage.py), through the C ABI: the coarse pass and its histogram
features, the bf16 MLP forward and backward passes, BCE and Adam; then a
short training run on method-generated injections that must beat the
untrained network, and the triaged search whose searched rows must equal
the exhaustive search's rows."""
import numpy as np
import pytest

import oracle
from oracle import triage as OT
import paper_2507_07816_gb300 as tcw
from paper_2507_07816_gb300 import triage as TR
import tcw_synth as syn
from _parity import REL

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
DEV = "cuda:0"
COARSE_TIE = 1e-6   # bins: the coarse pass decides bins in fp32 around an FP64 split


def small_event(seed, n_det=2, n_seg=150, n_bin=1200, n_sky=120, n_tmpl=96, n_inj=3, snr=(12.0, 16.0),
                t_sft=4.0, dtype=np.float32):
    r = syn.rng(seed)
    f_min = 500.0
    bank = syn.random_bank(r, n_tmpl, f0_range=(f_min - 3, f_min + n_bin / t_sft + 3),
                           tau_range=(3500.0, 35000.0))
    ev = syn.training_event(seed, bank, n_det=n_det, n_seg=n_seg, n_bin=n_bin, n_sky=n_sky,
                            n_inj=n_inj, snr_range=snr, t_sft=t_sft, dtype=dtype)
    return ev, bank


# 15 patches (sweep form, representatives' factors in order), 120 patches (sweep
# form; neighbouring skies' factors cross, so many (detector, segment) pairs take
# every representative's own bin) and 200 patches (the per-(template, patch) kernel)
# (the 1100-segment event splits every template's segments into 4 ranges); one
# detector; an FP16 map (the oracle reads the same half values widened); 32 s
# segments (F = f/df up to 25 600: the representatives' bins of a lookup span up
# to 5 bins, so lookups take more steps than the straight-line ones, and the
# guessed representative is off by more than one more often)
@pytest.mark.parametrize("P_SIZE,N_SKY,N_SEG,SWEEP,PARTS,N_DET,DTYPE,T_SFT",
                         [(8, 120, 150, 1, 1, 2, np.float32, 4.0), (1, 120, 150, 1, 1, 2, np.float32, 4.0),
                          (1, 200, 150, 0, 0, 2, np.float32, 4.0), (8, 120, 1100, 1, 4, 2, np.float32, 4.0),
                          (8, 120, 150, 1, 1, 1, np.float32, 4.0), (8, 120, 150, 1, 1, 2, np.float16, 4.0),
                          (8, 120, 150, 1, 1, 2, np.float32, 32.0), (3, 120, 150, 1, 1, 2, np.float32, 32.0)])
def test_coarse_features_match_oracle(P_SIZE, N_SKY, N_SEG, SWEEP, PARTS, N_DET, DTYPE, T_SFT):
    n_bin = 1200 if T_SFT == 4.0 else 9600
    ev, bank = small_event(81, n_inj=2, n_sky=N_SKY, n_seg=N_SEG, n_det=N_DET, dtype=DTYPE, t_sft=T_SFT,
                           n_bin=n_bin)
    _check_coarse(ev, bank, P_SIZE, SWEEP, PARTS)


def test_coarse_pass_with_segments_before_T0_matches_oracle():
    """T0 inside the observation (Eq. 1 starts there; earlier segments add
    nothing): the 64-segment tiles wholly before T0 take no anchor, the tile
    holding T0 is anchored at T0 itself (its middle lies before T0), and the
    second segment range starts its anchor chain with pow on a later tile."""
    ev, bank = small_event(85, n_inj=1, n_seg=600)
    ev.T0 = float(ev.t_mid[230] + 1.0)
    _check_coarse(ev, bank, 8, 1, 2)


def _check_coarse(ev, bank, P_SIZE, SWEEP, PARTS):
    LO, HI = -4.0, 12.0
    s = tcw.Search(0)
    TR.load_event(s, ev, bank)
    feat, psi = s.triage_features(P_SIZE, LO, HI, with_psi=True)
    info = s.triage_info()
    assert (info["coarse_kernel"], info["coarse_parts"]) == (SWEEP, PARTS)
    ora = OT.coarse_psi(ev.rho, ev.f_min, ev.df, ev.t_mid, ev.weights, ev.velocity, ev.nhat,
                        bank.f0, bank.tau, bank.n, ev.T0, P_SIZE)
    # pairs with a lookup within COARSE_TIE of a rounding tie may differ
    order = OT.sky_order(ev.velocity, ev.nhat)
    reps = [order[r] for _, _, r in OT.patches(len(order), P_SIZE)]
    pairs = np.array([(pi, b) for pi in range(len(reps)) for b in range(len(bank))])
    x = oracle.track_coordinates(ev.rho.shape[0], ev.f_min, ev.df, ev.t_mid, ev.velocity,
                                 ev.nhat[reps], bank.f0, bank.tau, bank.n, ev.T0, pairs)
    fr = x - np.floor(x)
    near = (np.isfinite(x) & (np.abs(fr - 0.5) <= COARSE_TIE)).any(axis=(1, 2)).reshape(len(reps), len(bank))
    assert near.mean() < 0.05
    S_, _, W2, _ = oracle.search_stats(ev.rho, ev.f_min, ev.df, ev.t_mid, ev.weights, ev.velocity,
                                       ev.nhat[reps], bank.f0, bank.tau, bank.n, ev.T0)
    fin = np.isfinite(ora)
    np.testing.assert_array_equal(np.isfinite(psi), fin)
    tol = REL * np.abs(S_) / np.sqrt(np.maximum(W2, 1e-30)) + 1e-5
    ok = fin & ~near
    err = np.abs(psi.astype(np.float64)[ok] - ora[ok])
    assert np.all(err <= tol[ok]), err.max()
    # histogram counts: equal to the oracle's up to pairs near a tie or a bin edge
    counts_o, _ = OT.histogram_features(ora, LO, HI)
    counts_g = np.rint(np.expm1(feat.astype(np.float64))).astype(np.int64)
    scale = (ora - LO) / (HI - LO) * 128
    edge = fin & (np.abs(scale - np.rint(scale)) < 1e-3)
    slack = (near | edge).sum(axis=1)
    assert np.all(np.abs(counts_g - counts_o).sum(axis=1) <= 2 * slack)
    assert np.all(counts_g.sum(axis=1) == len(bank))
    s.close()


def test_coarse_pass_on_every_third_segment_matches_oracle():
    """TCW_OPT_TRIAGE_STRIDE = 3: the coarse Psi equals the oracle's Psi at
    the patch representatives computed on segments 0, 3, 6, ... (the
    representatives come from the full search's sky order)."""
    ev, bank = small_event(87, n_inj=2, n_seg=151)
    LO, HI, PS, ST = -4.0, 12.0, 8, 3
    s = tcw.Search(0)
    s.set_option(tcw.OPT_TRIAGE_STRIDE, ST)
    TR.load_event(s, ev, bank)
    feat, psi = s.triage_features(PS, LO, HI, with_psi=True)
    assert s.triage_info()["lookups_coarse"] == psi.shape[0] * len(bank) * 2 * (-(-151 // ST))
    order = OT.sky_order(ev.velocity, ev.nhat)
    reps = [order[r] for _, _, r in OT.patches(len(order), PS)]
    sl = slice(None, None, ST)
    w = None if ev.weights is None else ev.weights[:, sl]
    S_, _, W2, ora = oracle.search_stats(ev.rho[:, sl], ev.f_min, ev.df, ev.t_mid[sl], w, ev.velocity[:, sl],
                                         ev.nhat[reps], bank.f0, bank.tau, bank.n, ev.T0)
    pairs = np.array([(pi, b) for pi in range(len(reps)) for b in range(len(bank))])
    x = oracle.track_coordinates(2, ev.f_min, ev.df, ev.t_mid[sl], ev.velocity[:, sl], ev.nhat[reps],
                                 bank.f0, bank.tau, bank.n, ev.T0, pairs)
    fr = x - np.floor(x)
    near = (np.isfinite(x) & (np.abs(fr - 0.5) <= COARSE_TIE)).any(axis=(1, 2)).reshape(len(reps), len(bank))
    fin = np.isfinite(ora)
    np.testing.assert_array_equal(np.isfinite(psi), fin)
    tol = REL * np.abs(S_) / np.sqrt(np.maximum(W2, 1e-30)) + 1e-5
    ok = fin & ~near
    assert ok.mean() > 0.9
    err = np.abs(psi.astype(np.float64)[ok] - ora[ok])
    assert np.all(err <= tol[ok]), err.max()
    with pytest.raises(tcw.TcwError):
        s.set_option(tcw.OPT_TRIAGE_STRIDE, 0)
    s.close()


def test_mlp_forward_backward_bce_adam_match_oracle():
    r = np.random.default_rng(82)
    theta = (r.normal(size=OT.N_PARAMS) * 0.1).astype(np.float32)
    X = np.abs(r.normal(size=(300, 128))).astype(np.float32)
    lab = (r.random(300) < 0.2).astype(np.float32)
    mlp = tcw.Mlp(theta, device=DEV)
    Xt = torch.as_tensor(X, device=DEV)
    H1, H2, y = mlp.forward(Xt)
    oH1, oH2, oy = OT.mlp_forward(theta.astype(np.float64), X)
    np.testing.assert_allclose(y.cpu().numpy(), oy, rtol=1e-4, atol=1e-4 * np.abs(oy).max())
    np.testing.assert_allclose(H2.cpu().numpy(), oH2, rtol=1e-4, atol=1e-4 * np.abs(oH2).max())
    loss, dy = mlp.bce(y, torch.as_tensor(lab, device=DEV), 3.0)
    oloss, ody = OT.bce_with_logits(oy, lab, pw=3.0)
    assert abs(loss.item() - oloss) <= 1e-4 * abs(oloss)
    np.testing.assert_allclose(dy.cpu().numpy(), ody, rtol=1e-3, atol=1e-7)
    grad = mlp.backward(Xt, H1, H2, dy).cpu().numpy().astype(np.float64)
    ograd = OT.mlp_backward(theta.astype(np.float64), X, oH1, oH2, ody)
    for name, sl in _slices().items():
        g, o = grad[sl], ograd[sl]
        assert np.max(np.abs(g - o)) <= 1e-3 * np.abs(o).max() + 1e-9, name
    # one Adam step from zero moments, then the bf16 weights follow theta
    mlp.adam(torch.as_tensor(ograd.astype(np.float32), device=DEV), lr=1e-3)
    oth, _, _ = OT.adam_step(theta.astype(np.float64), 0.0, 0.0, ograd.astype(np.float32).astype(np.float64),
                             1, lr=1e-3)
    th = mlp.parameters().astype(np.float64)
    np.testing.assert_allclose(th, oth, rtol=0, atol=2e-6)
    wb = mlp.wbf.cpu().numpy().view(np.uint16).astype(np.uint32) << 16
    w_gpu = wb.view(np.float32).astype(np.float64)
    w_ora = np.concatenate([OT.bf16_round(th[sl]) for sl in
                            (_slices()["W1"], _slices()["W2"], _slices()["w3"])])
    np.testing.assert_array_equal(w_gpu, w_ora)


def _slices():
    out, off = {}, 0
    for name, shape in OT.SIZES:
        n = int(np.prod(shape))
        out[name] = slice(off, off + n)
        off += n
    return out


def test_training_beats_the_untrained_network():
    # T_SFT = 32 s at 500-800 Hz: the sky's Doppler range spans about +-2 bins,
    # so patches of 16 of 256 skies are a quarter bin apart and separable
    r = syn.rng(83)
    bank = syn.random_bank(r, 64, f0_range=(540.0, 760.0), tau_range=(3500.0, 35000.0))

    def make(i):
        return syn.training_event(1000 + i, bank, n_det=1, n_seg=120, n_bin=9600, n_sky=256,
                                  t_sft=32.0, n_inj=2, snr_range=(10.0, 14.0))

    X, y, sizes = TR.collect(make, 32, bank, patch_size=16)
    Xv, yv, sizes_v = TR.collect(lambda i: make(500 + i), 16, bank, patch_size=16)
    assert y.sum().item() > 40
    untrained = tcw.Mlp(seed=3, device=DEV)
    mlp, losses = TR.train(X, y, steps=400, batch=256, lr=2e-3, seed=3, log_every=50)
    assert losses[-1][1] < 0.7 * losses[0][1], losses
    r_tr = TR.recall_at(mlp, Xv, yv, sizes_v, 0.25)
    r_un = TR.recall_at(untrained, Xv, yv, sizes_v, 0.25)
    assert r_tr >= 0.5 and r_tr > r_un + 0.2, (r_tr, r_un)


@pytest.mark.parametrize("amp,count", [(0, False), (4, False), (0, True)])
def test_triaged_search_rows_equal_exhaustive_rows(amp, count):
    ev, bank = small_event(84, n_sky=200, n_inj=2, snr=(14.0, 16.0), n_bin=9600, t_sft=32.0)
    # hand-set network: score = sum of the log-counts of the 28 highest histogram bins
    theta = np.zeros(OT.N_PARAMS, np.float32)
    p = OT.unpack(theta)
    p["W1"][100:, 0] = 1.0
    p["W2"][0, 0] = 1.0
    p["w3"][0] = 1.0
    mlp = tcw.Mlp(theta, device=DEV)
    s = tcw.Search(0)
    s.set_option(tcw.OPT_TRIAGE_SPREAD, 0)
    s.set_option(tcw.OPT_AMPLITUDE_POWER, amp)     # the exhaustive part takes the weighting
    if count:                                      # and the statistic too
        s.set_statistic(tcw.STAT_NUMBER_COUNT, 1.6)
    TR.load_event(s, ev, bank)
    k = 8
    pf, xf = s.search(k)
    pt, xt, searched = s.search_triaged(mlp, 16, -4.0, 12.0, 0.25, k)
    info = s.triage_info()
    assert info["n_selected"] == int(np.ceil(0.25 * info["n_patch"]))
    assert searched.sum() == info["skies_searched"] > 0
    rows = searched.astype(bool)
    np.testing.assert_array_equal(xt[rows], xf[rows])
    np.testing.assert_array_equal(pt[rows], pf[rows])
    assert np.all(xt[~rows] == -1) and np.all(np.isneginf(pt[~rows]))
    for inj in ev.injections:
        assert searched[inj.sky] == 1
    # with suppression the chosen patches are more than `spread` positions apart
    s.set_option(tcw.OPT_TRIAGE_SPREAD, 2)
    _, _, searched = s.search_triaged(mlp, 16, -4.0, 12.0, 0.2, k)   # 3 of 13 patches always fit
    pos = TR.sorted_positions(s)
    chosen = sorted({int(pos[i]) // 16 for i in np.nonzero(searched)[0]})
    assert len(chosen) == s.triage_info()["n_selected"] == 3
    assert all(b - a > 2 for a, b in zip(chosen, chosen[1:])), chosen
    s.close()


def test_triage_rank_matches_forward_of_features_and_drives_the_triaged_search():
    """tcw_triage_rank: the scores equal tcw_mlp_forward on tcw_triage_features'
    output, the patch order is argsort(-score) with ties by patch index, the
    sky order lists the patches' Doppler-sorted skies in that order, and a
    triaged search with spread 0 searches exactly the first ceil(frac P)
    patches of it."""
    ev, bank = small_event(86, n_sky=200, n_inj=2, snr=(14.0, 16.0), n_bin=9600, t_sft=32.0)
    r = np.random.default_rng(86)
    mlp = tcw.Mlp((r.normal(size=OT.N_PARAMS) * 0.05).astype(np.float32), device=DEV)
    s = tcw.Search(0)
    s.set_option(tcw.OPT_TRIAGE_SPREAD, 0)
    TR.load_event(s, ev, bank)
    PS, LO, HI = 16, -4.0, 12.0
    score, order, skies = s.triage_rank(mlp, PS, LO, HI)
    feat = s.triage_features(PS, LO, HI)
    _, _, y = mlp.forward(torch.as_tensor(feat, device=DEV))
    np.testing.assert_array_equal(score, y.cpu().numpy())
    P = len(score)
    assert P == -(-ev.nhat.shape[0] // PS)
    expect = np.array(sorted(range(P), key=lambda i: (-float(score[i]), i)), np.int32)
    np.testing.assert_array_equal(order, expect)
    sorted_sky = s.sky_order()
    np.testing.assert_array_equal(skies, np.concatenate([sorted_sky[i * PS:(i + 1) * PS] for i in order]))
    assert sorted(skies.tolist()) == list(range(ev.nhat.shape[0]))
    for frac in (0.25, 0.5):
        m = int(np.ceil(frac * P))
        _, _, searched = s.search_triaged(mlp, PS, LO, HI, frac, 4)
        first = np.concatenate([sorted_sky[i * PS:(i + 1) * PS] for i in order[:m]])
        np.testing.assert_array_equal(np.sort(np.nonzero(searched)[0]), np.sort(first))
    with pytest.raises(tcw.TcwError):
        s.triage_rank(mlp, 0, LO, HI)
    s.close()


def test_parameter_regions_search_a_template_subset():
    """TCW_OPT_TRIAGE_TEMPLATES: each chosen patch keeps its best templates by
    coarse Psi; the returned entries are exhaustive-search values of those
    (sky, template) pairs, and the injections are still found."""
    ev, bank = small_event(84, n_sky=200, n_inj=2, snr=(14.0, 16.0), n_bin=9600, t_sft=32.0)
    theta = np.zeros(OT.N_PARAMS, np.float32)
    p = OT.unpack(theta)
    p["W1"][100:, 0] = 1.0
    p["W2"][0, 0] = 1.0
    p["w3"][0] = 1.0
    mlp = tcw.Mlp(theta, device=DEV)
    s = tcw.Search(0)
    s.set_option(tcw.OPT_TRIAGE_SPREAD, 0)
    s.set_option(tcw.OPT_KEEP_STATS, 1)
    TR.load_event(s, ev, bank)
    k = 8
    s.search(k)
    full = s.statistics(("psi",))["psi"]
    s.set_option(tcw.OPT_TRIAGE_TEMPLATES, 100)        # 10 % of the bank per chosen patch
    pt, xt, searched = s.search_triaged(mlp, 16, -4.0, 12.0, 0.25, k)
    info = s.triage_info()
    n_sel = info["n_selected"]
    assert 0 < info["templates_searched"] <= n_sel * int(np.ceil(0.1 * len(bank.f0)))
    assert info["lookups_searched"] == info["skies_searched"] * info["templates_searched"] * ev.rho.shape[0] * ev.rho.shape[1]
    rows = np.nonzero(searched)[0]
    assert len(set(xt[rows].ravel().tolist()) - {-1}) <= info["templates_searched"]
    for r in rows:
        got = pt[r][xt[r] >= 0]
        ref = full[r, xt[r][xt[r] >= 0]]
        assert np.all(np.abs(got - ref) <= 1e-5 * np.abs(ref) + 1e-4)
        assert np.all(np.diff(got) <= 0)
    # the union of the chosen patches' best templates, recomputed from the coarse
    # Psi in the library's sorted-bank order (f0, ties by caller index), ties in Psi
    # broken by that order
    _, cpsi = s.triage_features(16, -4.0, 12.0, with_psi=True)
    pos = TR.sorted_positions(s)
    chosen = sorted({int(pos[i]) // 16 for i in rows})
    order = np.argsort(bank.f0, kind="stable")                  # sorted index -> caller index
    M = int(np.ceil(100 * len(bank.f0) / 1000))
    union = set()
    for pch in chosen:
        v = cpsi[pch][order]
        top = np.lexsort((np.arange(len(order)), -v))[:M]       # Psi desc, sorted index asc
        union |= set(order[top].tolist())
    assert len(union) == info["templates_searched"]
    assert set(xt[rows].ravel().tolist()) - {-1} <= union
    # the injections sit at chosen patches and their templates are kept
    for inj in ev.injections:
        near = np.nonzero(np.abs(pos - pos[inj.sky]) <= 16)[0]
        assert np.any(xt[near] == inj.template)
    s.set_option(tcw.OPT_TRIAGE_TEMPLATES, 1000)
    s.close()



def _batch(seeds, n_segs, n_skies, n_bin=1200, n_tmpl=96, n_det=2, dtype=np.float32):
    r = syn.rng(seeds[0] + 7)
    f_min, t_sft = 500.0, 4.0
    bank = syn.random_bank(r, n_tmpl, f0_range=(f_min - 3, f_min + n_bin / t_sft + 3),
                           tau_range=(3500.0, 35000.0))
    evs = [syn.training_event(sd, bank, n_det=n_det, n_seg=ns, n_bin=n_bin, n_sky=S, n_inj=2,
                              snr_range=(12.0, 16.0), t_sft=t_sft, dtype=dtype)
           for sd, ns, S in zip(seeds, n_segs, n_skies)]
    return evs, bank


def _hand_network():
    # score = sum of the log-counts of the 28 highest histogram bins
    theta = np.zeros(OT.N_PARAMS, np.float32)
    p = OT.unpack(theta)
    p["W1"][100:, 0] = 1.0
    p["W2"][0, 0] = 1.0
    p["w3"][0] = 1.0
    return tcw.Mlp(theta, device=DEV)


@pytest.mark.parametrize("amp,count", [(0, False), (4, False), (0, True)])
def test_batched_triaged_rows_equal_exhaustive_batched_rows(amp, count):
    """tcw_search_batched_triaged with every template: each event's chosen
    patches (ceil(frac * n_patch) of them) are searched in one launch and
    their rows equal tcw_search_batched's rows (the amplitude weighting and the
    number count apply to both); the other rows are empty.  Bit for bit with
    unit weights and counts; with amplitude weights the chosen sky subset's
    chunk width, and with it the segments per ring stage, differs from the
    full batch's, so the per-template weight sums are added in another order:
    Psi within 2 ulp."""
    evs, bank = _batch([91, 92, 93], [150, 90, 200], [120, 208, 64])
    mlp = _hand_network()
    s = tcw.Search(0)
    s.set_option(tcw.OPT_AMPLITUDE_POWER, amp)
    if count:
        s.set_statistic(tcw.STAT_NUMBER_COUNT, 1.6)
    s.define_bank(bank.f0, bank.tau, bank.n, 0.0)
    s.load_events(evs, evs[0].f_min, evs[0].df)
    k = 6
    vx, ix = s.search_batched(k)
    pt, it, searched = s.search_batched_triaged(mlp, 16, -4.0, 12.0, 0.3, k)
    rows = searched.astype(bool)
    info = s.triage_info()
    P = [-(-e.nhat.shape[0] // 16) for e in evs]
    assert info["n_patch"] == sum(P)
    assert info["n_selected"] == sum(int(np.ceil(0.3 * p)) for p in P)
    assert info["skies_searched"] == rows.sum() and 0 < rows.sum() < rows.shape[0]
    assert info["lookups_full"] == sum(e.nhat.shape[0] * len(bank) * 2 * e.rho.shape[1] for e in evs)
    assert info["templates_searched"] == len(evs) * len(bank)
    if amp == 0:
        np.testing.assert_array_equal(it[rows], ix[rows])
        np.testing.assert_array_equal(pt[rows], vx[rows])
    else:
        np.testing.assert_array_max_ulp(pt[rows], vx[rows], maxulp=2)
        assert (it[rows] == ix[rows]).mean() > 0.99
    assert np.all(it[~rows] == -1) and np.all(np.isneginf(pt[~rows]))
    # every event has whole patches searched
    row = 0
    for e, p in zip(evs, P):
        S = e.nhat.shape[0]
        assert rows[row:row + S].sum() >= 16 * int(np.ceil(0.3 * p)) - 15
        row += S
    # patch_size 0: 32 patches of ceil(n_sky / 32) skies per event
    pt0, it0, searched0 = s.search_batched_triaged(mlp, 0, -4.0, 12.0, 0.3, k)
    assert s.triage_info()["n_patch"] == sum(-(-e.nhat.shape[0] // -(-e.nhat.shape[0] // 32)) for e in evs)
    r0 = searched0.astype(bool)
    assert r0.any()
    # 4-sky patches do not keep the full search's 16-sky groups, so the rows agree
    # within the parity tolerance rather than bit for bit
    np.testing.assert_allclose(pt0[r0], vx[r0], rtol=1e-5, atol=1e-5)
    assert (it0[r0][:, 0] == ix[r0][:, 0]).mean() > 0.95
    with pytest.raises(tcw.TcwError):
        s.search_batched_triaged(mlp, -1, -4.0, 12.0, 0.3, k)
    s.close()


@pytest.mark.parametrize("n_det,dtype", [(1, np.float32), (2, np.float16)])
def test_batched_triaged_one_detector_and_fp16_rows_equal_exhaustive_batched_rows(n_det, dtype):
    """tcw_search_batched_triaged on one-detector events and on FP16 maps (the
    coarse pass reads the half values, the group kernel's FP16 instance searches
    the chosen skies): with every template the searched rows equal
    tcw_search_batched's rows bit for bit."""
    evs, bank = _batch([96, 97], [130, 170], [100, 150], n_det=n_det, dtype=dtype)
    mlp = _hand_network()
    s = tcw.Search(0)
    s.define_bank(bank.f0, bank.tau, bank.n, 0.0)
    s.load_events(evs, evs[0].f_min, evs[0].df)
    k = 5
    vx, ix = s.search_batched(k)
    pt, it, searched = s.search_batched_triaged(mlp, 16, -4.0, 12.0, 0.3, k)
    rows = searched.astype(bool)
    assert 0 < rows.sum() < rows.shape[0]
    assert s.triage_info()["coarse_kernel"] == 1
    np.testing.assert_array_equal(it[rows], ix[rows])
    np.testing.assert_array_equal(pt[rows], vx[rows])
    assert np.all(it[~rows] == -1) and np.all(np.isneginf(pt[~rows]))
    s.close()


def test_batched_triaged_regions_match_the_single_event_triaged_search():
    """With TCW_OPT_TRIAGE_TEMPLATES < 1000 every event searches its chosen
    skies over the union of its patches' best templates: the same skies and
    rows (within the parity tolerance) as tcw_search_triaged on that event
    alone."""
    evs, bank = _batch([94, 95], [120, 160], [96, 150], n_tmpl=200)
    mlp = _hand_network()
    k, tpm, frac = 5, 100, 0.35      # 20 templates per chosen patch (>= k)
    s = tcw.Search(0)
    s.set_option(tcw.OPT_TRIAGE_TEMPLATES, tpm)
    s.define_bank(bank.f0, bank.tau, bank.n, 0.0)
    s.load_events(evs, evs[0].f_min, evs[0].df)
    pt, it, searched = s.search_batched_triaged(mlp, 16, -4.0, 12.0, frac, k)
    assert s.triage_info()["templates_searched"] < len(evs) * len(bank)
    row = 0
    for e in evs:
        S = e.nhat.shape[0]
        s1 = tcw.Search(0)
        s1.set_option(tcw.OPT_TRIAGE_TEMPLATES, tpm)
        s1.set_option(tcw.OPT_KEEP_STATS, 1)
        TR.load_event(s1, e, bank)
        p1, i1, sr1 = s1.search_triaged(mlp, 16, -4.0, 12.0, frac, k)
        np.testing.assert_array_equal(searched[row:row + S], sr1)
        r = sr1.astype(bool)
        np.testing.assert_allclose(pt[row:row + S][r], p1[r], rtol=1e-5, atol=1e-5)
        same = (it[row:row + S][r] == i1[r]).mean()
        assert same > 0.99, same
        row += S
        s1.close()
    s.close()
