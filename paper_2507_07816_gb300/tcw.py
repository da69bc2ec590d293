"""Python binding of the C ABI in ``include/tcw.h`` (argument marshalling only).

Every step of the search runs in the CUDA library ``_build/libtcw.so``; this
module converts numpy arrays (host memory) or CUDA torch tensors (device
memory) into pointers and sizes, and raises ``TcwError`` on a non-zero status.
There is no CPU fallback: without the library every call fails.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

from . import build as _build

OK = 0
HOST, DEVICE = 0, 1
F32, F16 = 0, 1
KERNEL_AUTO, KERNEL_GROUP, KERNEL_LOOKUP = 0, 1, 2
OPT_KERNEL, OPT_KEEP_STATS, OPT_TILE_SEGMENTS, OPT_BANK_CHUNK = 1, 2, 3, 4
OPT_AUTOTUNE, OPT_BATCH_MEMORY, OPT_SKY_LANES, OPT_TRIAGE_SPREAD = 5, 6, 7, 8
OPT_AMPLITUDE_POWER, OPT_GEN_CHUNK, OPT_TRACK_BINS, OPT_TRIAGE_TEMPLATES = 9, 10, 11, 12
OPT_TRIAGE_STRIDE = 13
STAT_POWER, STAT_NUMBER_COUNT = 0, 1

_lock = threading.Lock()
_lib = None


class TcwError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"tcw status {status}: {message}")
        self.status = status


class _Info(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("launches", ctypes.c_int), ("lookups", ctypes.c_int64),
                ("general_path_lanes", ctypes.c_int64), ("doppler_bins_max", ctypes.c_double),
                ("quantum", ctypes.c_double), ("search_ms", ctypes.c_float)]


class _Event(ctypes.Structure):
    _fields_ = [("rho", ctypes.c_void_p), ("t_mid", ctypes.c_void_p), ("weights", ctypes.c_void_p),
                ("velocity", ctypes.c_void_p), ("nhat", ctypes.c_void_p), ("n_seg", ctypes.c_int64),
                ("n_sky", ctypes.c_int64), ("T0", ctypes.c_double)]


class _BankSpec(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("reserved", ctypes.c_int), ("n_f0", ctypes.c_int64),
                ("n_tau", ctypes.c_int64), ("n_n", ctypes.c_int64), ("n_tmpl", ctypes.c_int64),
                ("f0_lo", ctypes.c_double), ("f0_hi", ctypes.c_double), ("tau_lo", ctypes.c_double),
                ("tau_hi", ctypes.c_double), ("n_lo", ctypes.c_double), ("n_hi", ctypes.c_double),
                ("seed", ctypes.c_uint64)]


class _GenInfo(ctypes.Structure):
    _fields_ = [("n_tmpl", ctypes.c_int64), ("chunks", ctypes.c_int64), ("chunk_templates", ctypes.c_int64),
                ("lookups", ctypes.c_int64), ("kernel", ctypes.c_int), ("launches", ctypes.c_int),
                ("search_ms", ctypes.c_float), ("total_ms", ctypes.c_float)]


BANK_LATTICE, BANK_RANDOM = 0, 1


def bank_spec(kind, lo, hi, n_f0=1, n_tau=1, n_n=1, n_tmpl=0, seed=0):
    """A tcw_bank_spec: lattice (n_f0 x n_tau x n_n points) or uniform random
    (n_tmpl templates, Philox key `seed`) over lo..hi = (f0, tau, n)."""
    return _BankSpec(int(kind), 0, int(n_f0), int(n_tau), int(n_n), int(n_tmpl), float(lo[0]), float(hi[0]),
                     float(lo[1]), float(hi[1]), float(lo[2]), float(hi[2]), int(seed))


class _BatchInfo(ctypes.Structure):
    _fields_ = [("n_events", ctypes.c_int), ("waves", ctypes.c_int), ("bank_chunk", ctypes.c_int),
                ("tile_segments", ctypes.c_int), ("autotuned", ctypes.c_int),
                ("n_candidates", ctypes.c_int), ("n_items", ctypes.c_int),
                ("graph_kernels", ctypes.c_int), ("total_sky", ctypes.c_int64),
                ("lookups", ctypes.c_int64), ("general_path_lanes", ctypes.c_int64),
                ("tune_ms", ctypes.c_double), ("best_rate", ctypes.c_double),
                ("default_rate", ctypes.c_double), ("quantum", ctypes.c_double),
                ("search_ms", ctypes.c_float)]


class _TriageInfo(ctypes.Structure):
    _fields_ = [("n_patch", ctypes.c_int), ("n_selected", ctypes.c_int),
                ("skies_searched", ctypes.c_int64), ("lookups_full", ctypes.c_int64),
                ("lookups_coarse", ctypes.c_int64), ("lookups_searched", ctypes.c_int64),
                ("coarse_ms", ctypes.c_float), ("mlp_ms", ctypes.c_float),
                ("search_ms", ctypes.c_float), ("templates_searched", ctypes.c_int64),
                ("coarse_kernel", ctypes.c_int), ("coarse_parts", ctypes.c_int)]


MLP_PARAMS, MLP_WEIGHTS = 99073, 98560


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """Load the CUDA library, compiling it first when it is missing or stale."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise TcwError(-100, f"CUDA library not built: {path}")
        lib = ctypes.CDLL(path)
        p, i, i64, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        sig = {
            "tcw_create": [ctypes.POINTER(p), i, p],
            "tcw_destroy": [p],
            "tcw_set_option": [p, i, i64],
            "tcw_set_statistic": [p, i, d],
            "tcw_load_spectrogram": [p, i, i64, i64, i, p, i, d, d, p, p],
            "tcw_load_velocity": [p, p, i],
            "tcw_define_bank": [p, i64, p, p, p, d, i],
            "tcw_define_sky": [p, i64, p, i],
            "tcw_search": [p, i, p, p, i],
            "tcw_get_statistics": [p, p, p, p, p, i],
            "tcw_track_bins": [p, p, i],
            "tcw_get_info": [p, ctypes.POINTER(_Info)],
            "tcw_load_events": [p, i, i64, i, d, d, ctypes.POINTER(_Event), i, i],
            "tcw_search_batched": [p, i, p, p, i],
            "tcw_get_batch_info": [p, ctypes.POINTER(_BatchInfo)],
            "tcw_get_tune_results": [p, i, p, p, p, p],
            "tcw_mlp_pack": [p, p, p],
            "tcw_mlp_forward": [p, p, p, i64, p, p, p, p],
            "tcw_mlp_backward": [p, p, i64, p, p, p, p, p, p],
            "tcw_mlp_bce": [p, p, i64, ctypes.c_float, p, p, p],
            "tcw_mlp_adam": [p, p, p, p, i64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                             ctypes.c_float, p, p],
            "tcw_triage_features": [p, i, ctypes.c_float, ctypes.c_float, p, p, i],
            "tcw_triage_rank": [p, p, p, i, ctypes.c_float, ctypes.c_float, p, p, p, i],
            "tcw_search_triaged": [p, p, p, i, ctypes.c_float, ctypes.c_float, ctypes.c_float, i,
                                   p, p, p, i],
            "tcw_search_batched_triaged": [p, p, p, i, ctypes.c_float, ctypes.c_float, ctypes.c_float, i,
                                           p, p, p, i],
            "tcw_get_triage_info": [p, ctypes.POINTER(_TriageInfo)],
            "tcw_sky_order": [p, p],
            "tcw_bank_size": [ctypes.POINTER(_BankSpec), ctypes.POINTER(i64)],
            "tcw_generate_bank": [p, ctypes.POINTER(_BankSpec), i64, i64, p, p, p, i],
            "tcw_search_generated": [p, ctypes.POINTER(_BankSpec), d, i, p, p, i],
            "tcw_generate_bank_at": [p, ctypes.POINTER(_BankSpec), p, i64, p, p, p, i],
            "tcw_get_generated_info": [p, ctypes.POINTER(_GenInfo)],
            "tcw_probe_read_bandwidth": [i64, i, i, ctypes.POINTER(d)],
            "tcw_probe_fma_rate": [i, i, i, ctypes.POINTER(d)],
        }
        for name, args in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = i
        lib.tcw_status_string.argtypes = [i]
        lib.tcw_status_string.restype = ctypes.c_char_p
        lib.tcw_last_error.argtypes = [p]
        lib.tcw_last_error.restype = ctypes.c_char_p
        _lib = lib
        return lib


def probe_read_bandwidth(nbytes, passes=50, reps=5):
    """Read bandwidth (GB/s) of a streaming kernel over an nbytes device buffer."""
    lib = load_library()
    out = ctypes.c_double()
    st = lib.tcw_probe_read_bandwidth(int(nbytes), int(passes), int(reps), ctypes.byref(out))
    if st != OK:
        raise TcwError(st, "tcw_probe_read_bandwidth: " + lib.tcw_status_string(st).decode())
    return out.value


def probe_fma_rate(fp64, iters=4096, reps=5):
    """Fused multiply-add rate (TFLOP/s) in double (fp64) or float."""
    lib = load_library()
    out = ctypes.c_double()
    st = lib.tcw_probe_fma_rate(1 if fp64 else 0, int(iters), int(reps), ctypes.byref(out))
    if st != OK:
        raise TcwError(st, "tcw_probe_fma_rate: " + lib.tcw_status_string(st).decode())
    return out.value


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _arg(a, dtype):
    """(pointer, flags, keepalive) for a numpy array or a CUDA torch tensor."""
    if a is None:
        return None, HOST, None
    if _is_torch(a):
        if not a.is_cuda:
            a = a.detach().cpu().numpy()
        else:
            import torch
            tdt = {np.float32: torch.float32, np.float64: torch.float64, np.float16: torch.float16,
                   np.int64: torch.int64, np.int32: torch.int32}[np.dtype(dtype).type]
            if a.dtype != tdt:
                raise TypeError(f"expected {tdt}, got {a.dtype}")
            a = a.contiguous()
            return ctypes.c_void_p(a.data_ptr()), DEVICE, a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data_as(ctypes.c_void_p), HOST, arr


@dataclass
class Info:
    kernel: int
    launches: int
    lookups: int
    general_path_lanes: int
    doppler_bins_max: float
    quantum: float
    search_ms: float


class Search:
    """One search context (``tcw_ctx``) on one CUDA device and stream."""

    def __init__(self, device: int = 0, stream=None):
        self._lib = load_library()
        self._h = ctypes.c_void_p()
        st = None if stream is None else ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))
        self._check(self._lib.tcw_create(ctypes.byref(self._h), int(device), st), ctx=False)
        self.n_sky = self.n_tmpl = self.n_det = self.n_seg = self.n_bin = 0

    def _check(self, status, ctx=True):
        if status != OK:
            msg = self._lib.tcw_status_string(status).decode()
            if ctx and self._h:
                msg += ": " + self._lib.tcw_last_error(self._h).decode()
            raise TcwError(status, msg)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.tcw_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_option(self, option: int, value: int):
        self._check(self._lib.tcw_set_option(self._h, option, int(value)))

    def set_statistic(self, statistic: int, rho_th: float = 0.0):
        """STAT_POWER (default) or STAT_NUMBER_COUNT with threshold rho_th > 0."""
        self._check(self._lib.tcw_set_statistic(self._h, int(statistic), float(rho_th)))

    def load_spectrogram(self, rho, f_min, df, t_mid, weights=None):
        dt = np.float16 if str(getattr(rho, "dtype", "")).endswith("float16") else np.float32
        D, Nseg, Nbin = rho.shape
        rp, rf, keep = _arg(rho, dt)
        t = np.ascontiguousarray(np.asarray(t_mid, np.float64))
        w = None if weights is None else np.ascontiguousarray(np.asarray(weights, np.float32))
        if w is not None and w.shape != (D, Nseg):
            raise ValueError("weights must be [n_det][n_seg]")
        if t.shape != (Nseg,):
            raise ValueError("t_mid must be [n_seg]")
        self._check(self._lib.tcw_load_spectrogram(
            self._h, int(D), int(Nseg), int(Nbin), F16 if dt == np.float16 else F32, rp, rf,
            float(f_min), float(df), t.ctypes.data_as(ctypes.c_void_p),
            None if w is None else w.ctypes.data_as(ctypes.c_void_p)))
        self.n_det, self.n_seg, self.n_bin = int(D), int(Nseg), int(Nbin)

    def load_velocity(self, v):
        if tuple(v.shape) != (self.n_det, self.n_seg, 3):
            raise ValueError("velocity must be [n_det][n_seg][3]")
        p, f, keep = _arg(v, np.float64)
        self._check(self._lib.tcw_load_velocity(self._h, p, f))

    def define_bank(self, f0, tau, n, T0):
        a = [_arg(x, np.float64) for x in (f0, tau, n)]
        if not (len(f0) == len(tau) == len(n)):
            raise ValueError("bank arrays differ in length")
        if len({x[1] for x in a}) != 1:
            raise ValueError("bank arrays must all be on the host or all on the device")
        self._check(self._lib.tcw_define_bank(self._h, int(len(f0)), a[0][0], a[1][0], a[2][0],
                                              float(T0), a[0][1]))
        self.n_tmpl = int(len(f0))

    def define_sky(self, nhat):
        p, f, keep = _arg(nhat, np.float64)
        self._check(self._lib.tcw_define_sky(self._h, int(nhat.shape[0]), p, f))
        self.n_sky = int(nhat.shape[0])

    def search(self, k, psi_out=None, idx_out=None):
        """Top-k per sky: returns (psi [S][k] float32, idx [S][k] int64).

        With torch CUDA tensors as outputs the results stay on the device."""
        if psi_out is None:
            psi_out = np.empty((self.n_sky, k), np.float32)
            idx_out = np.empty((self.n_sky, k), np.int64)
        pp, pf, _ = _arg(psi_out, np.float32)
        ip, iff, _ = _arg(idx_out, np.int64)
        if pf != iff:
            raise ValueError("outputs must both be host or both device")
        if pf == HOST and (not isinstance(psi_out, np.ndarray) or psi_out.dtype != np.float32
                           or not psi_out.flags.c_contiguous):
            raise TypeError("host outputs must be C-contiguous numpy arrays")
        self._check(self._lib.tcw_search(self._h, int(k), pp, ip, pf))
        return psi_out, idx_out

    def statistics(self, which=("S", "W1", "W2", "psi")):
        outs = {w: np.empty((self.n_sky, self.n_tmpl), np.float32) for w in which}
        ptr = {w: (outs[w].ctypes.data_as(ctypes.c_void_p) if w in outs else None)
               for w in ("S", "W1", "W2", "psi")}
        self._check(self._lib.tcw_get_statistics(self._h, ptr["S"], ptr["W1"], ptr["W2"],
                                                 ptr["psi"], HOST))
        return outs

    def track_bins(self):
        out = np.empty((self.n_sky, self.n_tmpl, self.n_det, self.n_seg), np.int32)
        self._check(self._lib.tcw_track_bins(self._h, out.ctypes.data_as(ctypes.c_void_p), HOST))
        return out

    def info(self) -> Info:
        i = _Info()
        self._check(self._lib.tcw_get_info(self._h, ctypes.byref(i)))
        return Info(i.kernel, i.launches, i.lookups, i.general_path_lanes, i.doppler_bins_max,
                    i.quantum, i.search_ms)

    def load_problem(self, prob):
        """Load an object with rho, f_min, df, t_mid, weights, velocity, bank, T0, nhat."""
        self.load_spectrogram(prob.rho, prob.f_min, prob.df, prob.t_mid, prob.weights)
        self.load_velocity(prob.velocity)
        self.define_bank(prob.bank.f0, prob.bank.tau, prob.bank.n, prob.T0)
        self.define_sky(prob.nhat)

    # ---------------------------------------------------------------- batched
    def load_events(self, events, f_min, df):
        """Load a batch of events for ``search_batched``.

        ``events``: sequence of objects with ``rho`` [D][n_seg][n_bin] (float32
        or float16; all events the same dtype, D and n_bin), ``t_mid``,
        ``weights`` (or None), ``velocity`` [D][n_seg][3], ``nhat`` [n_sky][3]
        and ``T0``.  All arrays on the host (numpy) or all on the device (CUDA
        torch tensors)."""
        evs = list(events)
        if not evs:
            raise ValueError("no events")
        dt = np.float16 if str(getattr(evs[0].rho, "dtype", "")).endswith("float16") else np.float32
        D, _, Nbin = evs[0].rho.shape
        arr = (_Event * len(evs))()
        keep = []
        flags = set()
        for i, e in enumerate(evs):
            if e.rho.shape[0] != D or e.rho.shape[2] != Nbin:
                raise ValueError("events differ in n_det or n_bin")
            n_seg, n_sky = int(e.rho.shape[1]), int(e.nhat.shape[0])
            small = [e.t_mid, e.weights, e.velocity, e.nhat]
            if _is_torch(e.rho) and e.rho.is_cuda:
                # a device map takes its small arrays along to the same device
                import torch
                small = [None if a is None or (_is_torch(a) and a.is_cuda) else
                         torch.as_tensor(np.ascontiguousarray(a, dtype=t), device=e.rho.device)
                         for a, t in zip(small, (np.float64, np.float32, np.float64, np.float64))]
                small = [a if a is not None else b for a, b in
                         zip(small, [e.t_mid, e.weights, e.velocity, e.nhat])]
            parts = [_arg(e.rho, dt), _arg(small[0], np.float64),
                     _arg(small[1], np.float32), _arg(small[2], np.float64),
                     _arg(small[3], np.float64)]
            for (ptr, fl, k), a in zip(parts, (e.rho, *small)):
                if a is not None:
                    flags.add(fl)
                keep.append(k)
            arr[i] = _Event(parts[0][0], parts[1][0], parts[2][0], parts[3][0], parts[4][0], n_seg,
                            n_sky, float(e.T0))
        if len(flags) != 1:
            raise ValueError("event arrays must all be on the host or all on the device")
        self._check(self._lib.tcw_load_events(self._h, int(D), int(Nbin), F16 if dt == np.float16 else F32,
                                              float(f_min), float(df), arr, len(evs), flags.pop()))
        self.batch_sky = [int(e.nhat.shape[0]) for e in evs]

    def search_batched(self, k, psi_out=None, idx_out=None):
        """Top-k per sky of every event: (psi [total_sky][k], idx [total_sky][k]),
        events in order, each event's skies in the caller's order."""
        total = sum(self.batch_sky)
        if psi_out is None:
            psi_out = np.empty((total, k), np.float32)
            idx_out = np.empty((total, k), np.int64)
        pp, pf, _ = _arg(psi_out, np.float32)
        ip, iff, _ = _arg(idx_out, np.int64)
        if pf != iff:
            raise ValueError("outputs must both be host or both device")
        if pf == HOST and (not isinstance(psi_out, np.ndarray) or not psi_out.flags.c_contiguous):
            raise TypeError("host outputs must be C-contiguous numpy arrays")
        self._check(self._lib.tcw_search_batched(self._h, int(k), pp, ip, pf))
        return psi_out, idx_out

    def batch_info(self) -> dict:
        i = _BatchInfo()
        self._check(self._lib.tcw_get_batch_info(self._h, ctypes.byref(i)))
        return {name: getattr(i, name) for name, _ in _BatchInfo._fields_}

    def tune_results(self):
        """Autotuner measurements: list of (bank_chunk, tile_segments, sums/s)."""
        n = ctypes.c_int()
        self._check(self._lib.tcw_get_tune_results(self._h, 0, None, None, None, ctypes.byref(n)))
        m = n.value
        bc = (ctypes.c_int * max(m, 1))()
        ts = (ctypes.c_int * max(m, 1))()
        rt = (ctypes.c_double * max(m, 1))()
        self._check(self._lib.tcw_get_tune_results(self._h, m, bc, ts, rt, ctypes.byref(n)))
        return [(bc[i], ts[i], rt[i]) for i in range(m)]

    # ---------------------------------------------------------------- triage
    def triage_features(self, patch_size, psi_lo, psi_hi, with_psi=False):
        """Coarse-pass features [n_patch][128] (and Psi [n_patch][n_tmpl]) as numpy."""
        P = -(-self.n_sky // int(patch_size))
        feat = np.empty((P, 128), np.float32)
        psi = np.empty((P, self.n_tmpl), np.float32) if with_psi else None
        self._check(self._lib.tcw_triage_features(
            self._h, int(patch_size), float(psi_lo), float(psi_hi),
            feat.ctypes.data_as(ctypes.c_void_p),
            None if psi is None else psi.ctypes.data_as(ctypes.c_void_p), HOST))
        return (feat, psi) if with_psi else feat

    def triage_features_device(self, patch_size, psi_lo, psi_hi, out):
        """Coarse-pass features into a CUDA float32 tensor out [n_patch][128]."""
        self._check(self._lib.tcw_triage_features(
            self._h, int(patch_size), float(psi_lo), float(psi_hi), ctypes.c_void_p(out.data_ptr()),
            None, DEVICE))
        return out

    def triage_rank(self, mlp, patch_size, psi_lo, psi_hi):
        """Network scores [n_patch], patch order [n_patch] and ranked sky order
        [n_sky] (caller indices) as numpy."""
        P = -(-self.n_sky // max(int(patch_size), 1))   # the library rejects patch_size < 1
        score = np.empty(P, np.float32)
        order = np.empty(P, np.int32)
        skies = np.empty(self.n_sky, np.int32)
        self._check(self._lib.tcw_triage_rank(
            self._h, ctypes.c_void_p(mlp.wbf.data_ptr()), ctypes.c_void_p(mlp.theta.data_ptr()),
            int(patch_size), float(psi_lo), float(psi_hi), score.ctypes.data_as(ctypes.c_void_p),
            order.ctypes.data_as(ctypes.c_void_p), skies.ctypes.data_as(ctypes.c_void_p), HOST))
        return score, order, skies

    def search_triaged(self, mlp, patch_size, psi_lo, psi_hi, frac, k):
        """Triaged search: (psi [S][k], idx [S][k], searched [S]) as numpy."""
        psi = np.empty((self.n_sky, k), np.float32)
        idx = np.empty((self.n_sky, k), np.int64)
        searched = np.empty(self.n_sky, np.int32)
        self._check(self._lib.tcw_search_triaged(
            self._h, ctypes.c_void_p(mlp.wbf.data_ptr()), ctypes.c_void_p(mlp.theta.data_ptr()),
            int(patch_size), float(psi_lo), float(psi_hi), float(frac), int(k),
            psi.ctypes.data_as(ctypes.c_void_p), idx.ctypes.data_as(ctypes.c_void_p),
            searched.ctypes.data_as(ctypes.c_void_p), HOST))
        return psi, idx, searched

    def search_batched_triaged(self, mlp, patch_size, psi_lo, psi_hi, frac, k):
        """Triaged search of every loaded event: (psi [total_sky][k], idx
        [total_sky][k], searched [total_sky]) as numpy, rows as search_batched.
        patch_size 0: 32 patches per event."""
        total = sum(self.batch_sky)
        psi = np.empty((total, k), np.float32)
        idx = np.empty((total, k), np.int64)
        searched = np.empty(total, np.int32)
        self._check(self._lib.tcw_search_batched_triaged(
            self._h, ctypes.c_void_p(mlp.wbf.data_ptr()), ctypes.c_void_p(mlp.theta.data_ptr()),
            int(patch_size), float(psi_lo), float(psi_hi), float(frac), int(k),
            psi.ctypes.data_as(ctypes.c_void_p), idx.ctypes.data_as(ctypes.c_void_p),
            searched.ctypes.data_as(ctypes.c_void_p), HOST))
        return psi, idx, searched

    # -------------------------------------------------------- generated banks
    def bank_size(self, spec) -> int:
        n = ctypes.c_int64()
        self._check(self._lib.tcw_bank_size(ctypes.byref(spec), ctypes.byref(n)))
        return n.value

    def generate_bank(self, spec, first=0, count=None, out=None):
        """Templates [first, first + count) of `spec`: (f0, tau, n) float64.
        ``out``: three torch CUDA tensors to fill on the device, else numpy."""
        if count is None:
            count = self.bank_size(spec) - first
        if out is None:
            out = tuple(np.empty(int(count), np.float64) for _ in range(3))
        ptrs, flags = [], set()
        for a in out:
            pa, fa, _ = _arg(a, np.float64)
            ptrs.append(pa)
            flags.add(fa)
        if len(flags) != 1:
            raise ValueError("outputs must all be host or all device")
        self._check(self._lib.tcw_generate_bank(self._h, ctypes.byref(spec), int(first), int(count), *ptrs,
                                                flags.pop()))
        return out

    def generate_bank_at(self, spec, idx):
        """Templates of `spec` at the int64 indices `idx` (any shape): (f0, tau, n)
        float64 arrays of that shape."""
        ix = np.ascontiguousarray(np.asarray(idx, np.int64))
        out = tuple(np.empty(ix.shape, np.float64) for _ in range(3))
        self._check(self._lib.tcw_generate_bank_at(self._h, ctypes.byref(spec), ix.ctypes.data_as(ctypes.c_void_p),
                                                   ix.size, *(o.ctypes.data_as(ctypes.c_void_p) for o in out),
                                                   HOST))
        return out

    def search_generated(self, spec, T0, k, psi_out=None, idx_out=None):
        """Top-k per sky over a generated bank: (psi [S][k], idx [S][k] int64 =
        generated template index)."""
        if psi_out is None:
            psi_out = np.empty((self.n_sky, k), np.float32)
            idx_out = np.empty((self.n_sky, k), np.int64)
        pp, pf, _ = _arg(psi_out, np.float32)
        ip, iff, _ = _arg(idx_out, np.int64)
        if pf != iff:
            raise ValueError("outputs must both be host or both device")
        self._check(self._lib.tcw_search_generated(self._h, ctypes.byref(spec), float(T0), int(k), pp, ip, pf))
        return psi_out, idx_out

    def generated_info(self) -> dict:
        i = _GenInfo()
        self._check(self._lib.tcw_get_generated_info(self._h, ctypes.byref(i)))
        return {name: getattr(i, name) for name, _ in _GenInfo._fields_}

    def triage_info(self) -> dict:
        i = _TriageInfo()
        self._check(self._lib.tcw_get_triage_info(self._h, ctypes.byref(i)))
        return {name: getattr(i, name) for name, _ in _TriageInfo._fields_}

    def sky_order(self):
        """Doppler-sorted order of the loaded sky (caller indices)."""
        out = np.empty(self.n_sky, np.int32)
        self._check(self._lib.tcw_sky_order(self._h, out.ctypes.data_as(ctypes.c_void_p)))
        return out


class Mlp:
    """Parameters, bfloat16 weights and Adam moments of the triage network, as
    CUDA tensors, driven through the tcw_mlp_* entry points."""

    def __init__(self, theta=None, seed=0, device="cuda:0"):
        import torch
        self._lib = load_library()
        self.device = torch.device(device)
        if theta is None:
            theta = self.initial(seed)
        theta = np.ascontiguousarray(theta, np.float32)
        if theta.shape != (MLP_PARAMS,):
            raise ValueError(f"theta must have {MLP_PARAMS} entries")
        self.theta = torch.as_tensor(theta, device=self.device).clone()
        self.wbf = torch.empty(MLP_WEIGHTS, dtype=torch.int16, device=self.device)
        self.m = torch.zeros_like(self.theta)
        self.v = torch.zeros_like(self.theta)
        self.step = 0
        self._call("tcw_mlp_pack", self.theta, self.wbf)

    @staticmethod
    def initial(seed):
        """He-normal weights, zero biases (packed layout of include/tcw.h)."""
        r = np.random.default_rng(seed)
        parts = [r.normal(0, np.sqrt(2.0 / 128), 128 * 256), np.zeros(256),
                 r.normal(0, np.sqrt(2.0 / 256), 256 * 256), np.zeros(256),
                 r.normal(0, np.sqrt(1.0 / 256), 256), np.zeros(1)]
        return np.concatenate(parts).astype(np.float32)

    def _stream(self):
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    def _call(self, name, *args):
        conv = []
        for a in args:
            if a is None:
                conv.append(None)
            elif _is_torch(a):
                conv.append(ctypes.c_void_p(a.data_ptr()))
            else:
                conv.append(a)
        st = getattr(self._lib, name)(*conv, self._stream())
        if st != OK:
            raise TcwError(st, f"{name}: " + self._lib.tcw_status_string(st).decode())

    def forward(self, X):
        import torch
        n = X.shape[0]
        H1 = torch.empty((n, 256), dtype=torch.float32, device=self.device)
        H2 = torch.empty((n, 256), dtype=torch.float32, device=self.device)
        y = torch.empty(n, dtype=torch.float32, device=self.device)
        self._call("tcw_mlp_forward", self.wbf, self.theta, X.contiguous(), int(n), H1, H2, y)
        return H1, H2, y

    def backward(self, X, H1, H2, dy):
        import torch
        n = X.shape[0]
        grad = torch.empty_like(self.theta)
        work = torch.empty(2 * n * 256, dtype=torch.float32, device=self.device)
        self._call("tcw_mlp_backward", self.wbf, X.contiguous(), int(n), H1, H2, dy, grad, work)
        return grad

    def bce(self, y, label, pos_weight=1.0):
        import torch
        loss = torch.empty(1, dtype=torch.float32, device=self.device)
        dy = torch.empty_like(y)
        self._call("tcw_mlp_bce", y, label.contiguous(), int(y.shape[0]), ctypes.c_float(pos_weight), loss, dy)
        return loss, dy

    def adam(self, grad, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.step += 1
        self._call("tcw_mlp_adam", self.theta, self.m, self.v, grad, int(self.step), ctypes.c_float(lr),
                   ctypes.c_float(beta1), ctypes.c_float(beta2), ctypes.c_float(eps), self.wbf)

    def parameters(self):
        return self.theta.detach().cpu().numpy()

    def save(self, path):
        np.savez(path, theta=self.parameters())

    @classmethod
    def load(cls, path, device="cuda:0"):
        return cls(np.load(path)["theta"], device=device)
