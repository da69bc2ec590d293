"""tcw_search_noalloc: the search for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc -- their device memory belongs to their
own arena or caching allocator, or they cannot accept the device-wide
synchronisation that cudaMalloc/cudaFree imply.  tcw_search_noalloc serves
them from a fixed 64 MiB array inside the library.  These tests call it
through the C ABI on caller-owned device buffers -- twice in a row on two
different problems (the second call reuses the array the first one left
behind), one sky with a large bank, an FP16 map, inputs that take the
per-lookup kernel -- and check each result against the regular tcw_search
within the tolerances of the parity tests; oversized problems and a
capturing stream are refused.  They live in a file that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

import paper_2507_07816_gb300 as tcw
import tcw_synth as syn
from _parity import REL

pytestmark = pytest.mark.gpu


def _problem(seed, n_det, n_seg, n_bin, n_tmpl, n_sky, t_sft=4.0, f_min=500.0, dtype=np.float32):
    r = syn.rng(seed)
    df = 1.0 / t_sft
    t = syn.segment_times(n_seg, t_sft)
    T0 = t[0] - 0.5 * t_sft
    dets = syn.random_detectors(r, n_det)
    vel = np.stack([d.velocity(t) for d in dets])
    rho = syn.exponential_noise(r, (n_det, n_seg, n_bin))
    w = syn.uniform_weights(r, n_det, n_seg)
    bank = syn.random_bank(r, n_tmpl, f0_range=(f_min, f_min + n_bin * df))
    nhat = syn.random_sky(r, n_sky)
    inj = syn.Injection(float(bank.f0[1]), float(bank.tau[1]), float(bank.n[1]), nhat[0], 10.0)
    syn.inject(r, rho, inj, dets, t, T0, f_min, df, w)
    if dtype != np.float32:
        rho = rho.astype(dtype)
    return syn.Problem(rho, t, w, vel, f_min, df, T0, nhat, bank, [inj], dets, name=f"noalloc{seed}")


def _reference(p, k, kernel=None):
    s = tcw.Search(0)
    s.set_option(tcw.OPT_KEEP_STATS, 1)
    s.load_problem(p)
    val, idx = s.search(k)
    st = s.statistics(("S", "W2", "psi"))
    if kernel is not None:
        assert s.info().kernel == kernel
    s.close()
    return val, idx, st


def _call_noalloc(lib, p, k, torch, stream=None):
    dev = torch.device("cuda:0")
    as_t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    half = p.rho.dtype == np.float16
    rho = as_t(p.rho, torch.float16 if half else torch.float32)
    t = as_t(p.t_mid, torch.float64)
    w = as_t(p.weights, torch.float32)
    v = as_t(p.velocity, torch.float64)
    f0, tau, n = (as_t(a, torch.float64) for a in (p.bank.f0, p.bank.tau, p.bank.n))
    nhat = as_t(p.nhat, torch.float64)
    S = p.nhat.shape[0]
    psi = torch.empty((S, k), dtype=torch.float32, device=dev)
    idx = torch.empty((S, k), dtype=torch.int64, device=dev)
    stream = stream or torch.cuda.current_stream(dev)
    P = lambda x: ctypes.c_void_p(x.data_ptr())
    D, Nseg, Nbin = p.rho.shape
    st = lib.tcw_search_noalloc(D, Nseg, Nbin, 1 if half else 0, P(rho), p.f_min, p.df, P(t), P(w), P(v),
                                len(p.bank), P(f0), P(tau), P(n), p.T0, S, P(nhat), k, P(psi),
                                P(idx), ctypes.c_void_p(stream.cuda_stream))
    torch.cuda.synchronize()
    return st, psi.cpu().numpy(), idx.cpu().numpy()


def _assert_matches(val, idx, ref_val, ref_idx, st, k):
    S_, W2, psi = (st[x].astype(np.float64) for x in ("S", "W2", "psi"))
    tol = REL * np.abs(S_) / np.sqrt(np.maximum(W2, 1e-30)) + 1e-5
    for r in range(idx.shape[0]):
        kth = ref_val[r, -1]
        for b in set(idx[r].tolist()) ^ set(ref_idx[r].tolist()):
            assert abs(psi[r, b] - kth) <= 2 * tol[r, b], (r, b)
        err = np.abs(val[r].astype(np.float64) - psi[r, idx[r]])
        assert np.all(err <= tol[r, idx[r]]), (r, err.max())


def _lib():
    lib = tcw.load_library()
    p_, i_, i64, d_ = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    lib.tcw_search_noalloc.argtypes = [i_, i64, i64, i_, p_, d_, d_, p_, p_, p_, i64, p_, p_, p_,
                                       d_, i64, p_, i_, p_, p_, p_]
    lib.tcw_search_noalloc.restype = i_
    return lib


def test_noalloc_matches_regular_search_twice():
    torch = pytest.importorskip("torch")
    lib = _lib()
    a = _problem(41, n_det=2, n_seg=96, n_bin=1500, n_tmpl=200, n_sky=40)
    b = _problem(42, n_det=1, n_seg=70, n_bin=900, n_tmpl=61, n_sky=9)
    ka, kb = 20, 7
    ref_a = _reference(a, ka)
    ref_b = _reference(b, kb)
    st_a, val_a, idx_a = _call_noalloc(lib, a, ka, torch)
    st_b, val_b, idx_b = _call_noalloc(lib, b, kb, torch)
    assert st_a == 0 and st_b == 0, (st_a, st_b)
    _assert_matches(val_a, idx_a, ref_a[0], ref_a[1], ref_a[2], ka)
    _assert_matches(val_b, idx_b, ref_b[0], ref_b[1], ref_b[2], kb)


def test_noalloc_rejects_oversized_problems():
    torch = pytest.importorskip("torch")
    lib = _lib()
    dev = torch.device("cuda:0")
    dummy = torch.zeros(16, dtype=torch.float64, device=dev)
    P = ctypes.c_void_p(dummy.data_ptr())
    # 4096 skies x 200000 templates needs far more than the fixed 64 MiB
    st = lib.tcw_search_noalloc(1, 16, 64, 0, P, 500.0, 0.25, P, None, P, 200000, P, P, P, 0.0,
                                4096, P, 10, P, P, None)
    assert st == -5


def test_noalloc_one_sky_with_a_large_bank():
    """One sky is padded to the narrowest sky chunk (256 skies), as in
    tcw_search, so a 30000-template bank fits the 64 MiB array."""
    torch = pytest.importorskip("torch")
    lib = _lib()
    p = _problem(43, n_det=1, n_seg=64, n_bin=2048, n_tmpl=30000, n_sky=1)
    k = 16
    ref = _reference(p, k)
    st, val, idx = _call_noalloc(lib, p, k, torch)
    assert st == 0, st
    _assert_matches(val, idx, ref[0], ref[1], ref[2], k)


def test_noalloc_fp16_map_and_the_per_lookup_path():
    """An FP16 map, and inputs outside the group kernel's exactness conditions
    (T_SFT = 32 s at 1 kHz: Doppler shifts above 2.9 bins), where the regular
    search and this entry point both take the per-lookup FP64 kernel."""
    torch = pytest.importorskip("torch")
    lib = _lib()
    a = _problem(44, n_det=2, n_seg=80, n_bin=1200, n_tmpl=150, n_sky=50, dtype=np.float16)
    b = _problem(45, n_det=1, n_seg=48, n_bin=3200, n_tmpl=40, n_sky=20, t_sft=32.0, f_min=1000.0)
    for p, k, kern in ((a, 10, tcw.KERNEL_GROUP), (b, 5, tcw.KERNEL_LOOKUP)):
        ref = _reference(p, k, kern)
        st, val, idx = _call_noalloc(lib, p, k, torch)
        assert st == 0, st
        _assert_matches(val, idx, ref[0], ref[1], ref[2], k)


def test_noalloc_refuses_a_capturing_stream():
    """The call synchronises its stream, so it returns TCW_ERR_STATE (-4)
    while that stream is being captured into a CUDA graph."""
    torch = pytest.importorskip("torch")
    lib = _lib()
    dummy = torch.zeros(64, dtype=torch.float64, device=torch.device("cuda:0"))
    P = ctypes.c_void_p(dummy.data_ptr())
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        st = lib.tcw_search_noalloc(1, 32, 600, 0, P, 500.0, 0.25, P, None, P, 20, P, P, P, 0.0, 5, P, 3,
                                    P, P, ctypes.c_void_p(side.cuda_stream))
    assert st == -4
