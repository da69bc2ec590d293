"""Learned sky triage: training data, GPU training, and the judged evaluation.

The paper searches every sky direction (Sec. 2, Eq. 4).  The triage ranks
sky patches (runs of Doppler-sorted skies) by a small network applied to a
coarse pass, then searches only the best-ranked patches exhaustively.  This
module drives the library's kernels only:

  patch features   tcw_triage_features (coarse pass + histogram), on device
  network          Mlp: tcw_mlp_forward / backward / bce / adam, on device
  triaged search   tcw_search_triaged
  judge            the exhaustive tcw_search of every sky, with the detection
                   threshold of Sec. 3: Psi above the largest Psi of
                   noise-only searches with the same bank

Events come from a caller-supplied ``make_event(i)`` returning an object with
rho, t_mid, weights, velocity, f_min, df, T0, nhat and ``injections`` (each
with ``template`` and ``sky`` indices); the bank is fixed per run.
"""
from __future__ import annotations

import time

import numpy as np

from .tcw import Mlp, Search

PATCH_SIZE = 32
PSI_LO, PSI_HI = -4.0, 12.0
# Sky resolution of the statistic: skies whose Doppler factors differ by a
# small fraction of a bin see the same track bins for most segments, so a
# signal is found at every sky of its Doppler neighbourhood.  Labels mark the
# patches within LABEL_RADIUS patches of an injected sky; the judge accepts
# the injected template at any sky within JUDGE_RADIUS Doppler-sorted skies.
LABEL_RADIUS = 1
JUDGE_RADIUS = 64
# Operating point of the triaged search: the best FRAC of the patches are
# searched, each over its best TEMPLATES_PERMILLE per mille of the bank by
# coarse Psi (TCW_OPT_TRIAGE_TEMPLATES); the union of those templates is
# searched at every chosen sky.
FRAC = 0.35
TEMPLATES_PERMILLE = 12
# The coarse pass runs on every STRIDE-th segment (TCW_OPT_TRIAGE_STRIDE).
# Every segment: with a stride of 2 the coarse Psi of an injection loses a
# factor sqrt(2) and falls into the noise of the other patches' maxima.
STRIDE = 1


def load_event(search, ev, bank, define_bank=True):
    search.load_spectrogram(ev.rho, ev.f_min, ev.df, ev.t_mid, ev.weights)
    search.load_velocity(ev.velocity)
    if define_bank:
        search.define_bank(bank.f0, bank.tau, bank.n, ev.T0)
    search.define_sky(ev.nhat)


def sorted_positions(search):
    """Position of every sky in the search's Doppler-sorted order."""
    order = search.sky_order()
    pos = np.empty_like(order)
    pos[order] = np.arange(order.shape[0])
    return pos


def patch_labels(search, ev, patch_size=PATCH_SIZE, radius=LABEL_RADIUS):
    """1 for the patches within `radius` patches of an injected sky, else 0."""
    pos = sorted_positions(search)
    P = -(-pos.shape[0] // patch_size)
    lab = np.zeros(P, np.float32)
    for inj in ev.injections:
        p = pos[inj.sky] // patch_size
        lab[max(0, p - radius):min(P, p + radius + 1)] = 1.0
    return lab


def collect(make_event, n_events, bank, patch_size=PATCH_SIZE, lo=PSI_LO, hi=PSI_HI, device="cuda:0",
            stride=STRIDE):
    """Features [N][128] and labels [N] (CUDA tensors) of n_events events, and
    the number of patches of each event."""
    import torch
    from .tcw import OPT_TRIAGE_STRIDE
    s = Search(0)
    s.set_option(OPT_TRIAGE_STRIDE, stride)
    feats, labs, sizes = [], [], []
    for i in range(n_events):
        ev = make_event(i)
        load_event(s, ev, bank)
        lab = patch_labels(s, ev, patch_size)
        out = torch.empty((lab.shape[0], 128), dtype=torch.float32, device=device)
        s.triage_features_device(patch_size, lo, hi, out)
        feats.append(out)
        labs.append(torch.as_tensor(lab, device=device))
        sizes.append(lab.shape[0])
    s.close()
    return torch.cat(feats), torch.cat(labs), sizes


def train(X, y, steps=2000, batch=4096, lr=1e-3, seed=0, pos_weight=None, mlp=None, log_every=0):
    """Adam on the mean BCE with logits; returns (mlp, losses)."""
    import torch
    n = X.shape[0]
    if pos_weight is None:
        pos = float(y.sum().item())
        pos_weight = max(1.0, (n - pos) / max(pos, 1.0))
    mlp = mlp or Mlp(seed=seed, device=X.device)
    g = torch.Generator(device="cpu").manual_seed(seed)
    losses = []
    for it in range(steps):
        idx = torch.randint(0, n, (min(batch, n),), generator=g).to(X.device)
        xb, yb = X[idx].contiguous(), y[idx].contiguous()
        H1, H2, out = mlp.forward(xb)
        loss, dy = mlp.bce(out, yb, pos_weight)
        grad = mlp.backward(xb, H1, H2, dy)
        mlp.adam(grad, lr=lr)
        if log_every and (it % log_every == 0 or it == steps - 1):
            losses.append((it, float(loss.item())))
    return mlp, losses


def recall_at(mlp, X, y, sizes, frac):
    """Fraction of positive patches that rank within the top ceil(frac * P)
    patches of their own event (ties by patch index, as the search ranks)."""
    _, _, s = mlp.forward(X)
    s = s.detach().cpu().numpy()
    lab = y.detach().cpu().numpy() > 0.5
    hit = tot = 0
    off = 0
    for P in sizes:
        sc, lb = s[off:off + P], lab[off:off + P]
        m = max(1, int(np.ceil(frac * P - 1e-9)))
        top = np.argsort(-sc, kind="stable")[:m]
        hit += int(lb[top].sum())
        tot += int(lb.sum())
        off += P
    return hit / max(tot, 1)


def noise_threshold(make_noise_event, n_events, bank):
    """Detection threshold of Sec. 3: the largest Psi over every sky and
    template of exhaustive searches of n_events noise-only events with the
    same bank (so at most one detection per n_events noise searches)."""
    s = Search(0)
    top = -np.inf
    for i in range(n_events):
        load_event(s, make_noise_event(i), bank)
        psi, _ = s.search(1)
        top = max(top, float(np.max(psi)))
    s.close()
    return top


def judge(ev, psi, idx, pos, psi_det, k_det=10, radius=JUDGE_RADIUS):
    """Injections found: the injected template within the first k_det entries,
    with Psi > psi_det (the noise-only maximum), of some sky within `radius`
    Doppler-sorted positions (pos) of the injected sky."""
    found = []
    for inj in ev.injections:
        near = np.nonzero(np.abs(pos - pos[inj.sky]) <= radius)[0]
        rows_i, rows_p = idx[near, :k_det], psi[near, :k_det]
        hit = (rows_i == inj.template) & (rows_p > psi_det)
        found.append(bool(hit.any()))
    return found


def evaluate(mlp, make_event, n_events, bank, psi_det, frac=FRAC, k=100, patch_size=PATCH_SIZE, lo=PSI_LO,
             hi=PSI_HI, k_det=10, templates_permille=TEMPLATES_PERMILLE, stride=STRIDE):
    """Judge the triaged search against the exhaustive one on fresh events
    (psi_det: the detection threshold, see noise_threshold).
    templates_permille < 1000 also restricts each chosen patch to its best
    templates by coarse Psi (TCW_OPT_TRIAGE_TEMPLATES)."""
    from .tcw import OPT_TRIAGE_STRIDE, OPT_TRIAGE_TEMPLATES
    s = Search(0)
    s.set_option(OPT_TRIAGE_TEMPLATES, templates_permille)
    s.set_option(OPT_TRIAGE_STRIDE, stride)
    full_found = tri_found = 0
    missed = 0
    t_full = t_tri = 0.0
    sums_full = sums_tri = 0
    for i in range(n_events):
        ev = make_event(i)
        load_event(s, ev, bank)
        t0 = time.perf_counter()
        pf, xf = s.search(k)
        t1 = time.perf_counter()
        pt, xt, searched = s.search_triaged(mlp, patch_size, lo, hi, frac, k)
        t2 = time.perf_counter()
        info = s.triage_info()
        pos = sorted_positions(s)
        t_full += t1 - t0
        t_tri += t2 - t1
        sums_full += info["lookups_full"]
        sums_tri += info["lookups_coarse"] + info["lookups_searched"]
        ff = judge(ev, pf, xf, pos, psi_det, k_det)
        tf = judge(ev, pt, xt, pos, psi_det, k_det)
        full_found += sum(ff)
        tri_found += sum(tf)
        missed += sum(a and not b for a, b in zip(ff, tf))
    s.close()
    return {"events": n_events, "detected_full": full_found, "detected_triaged": tri_found,
            "missed": missed, "loss": missed / max(full_found, 1), "time_full_s": t_full,
            "time_triaged_s": t_tri, "speedup": t_full / max(t_tri, 1e-12),
            "sums_full": sums_full, "sums_executed_triaged": sums_tri, "frac": frac,
            "patch_size": patch_size, "templates_permille": templates_permille, "stride": stride,
            "psi_det": psi_det}
