"""Host-side checks of the generated-bank specification (no GPU needed):
tcw_bank_size validates the spec and counts its templates."""
import ctypes

import pytest

from paper_2507_07816_gb300 import tcw

LO = (500.0, 3500.0, 3.0)
HI = (3000.0, 35000.0, 7.0)


def size(spec):
    lib = tcw.load_library()
    n = ctypes.c_int64()
    st = lib.tcw_bank_size(ctypes.byref(spec), ctypes.byref(n))
    return st, n.value


def test_sizes():
    assert size(tcw.bank_spec(tcw.BANK_LATTICE, LO, HI, n_f0=7, n_tau=5, n_n=3)) == (0, 105)
    assert size(tcw.bank_spec(tcw.BANK_RANDOM, LO, HI, n_tmpl=10**9)) == (0, 10**9)
    assert size(tcw.bank_spec(tcw.BANK_LATTICE, LO, LO, n_f0=1)) == (0, 1)       # a single point


@pytest.mark.parametrize("spec", [
    tcw.bank_spec(tcw.BANK_RANDOM, LO, HI, n_tmpl=0),
    tcw.bank_spec(tcw.BANK_LATTICE, LO, HI, n_f0=0, n_tau=1, n_n=1),
    tcw.bank_spec(tcw.BANK_LATTICE, LO, HI, n_f0=2**31, n_tau=2**31, n_n=2),     # beyond 2^62
    tcw.bank_spec(tcw.BANK_RANDOM, (0.0, 3500.0, 3.0), HI, n_tmpl=5),           # f0 must be > 0
    tcw.bank_spec(tcw.BANK_RANDOM, (500.0, 0.0, 3.0), HI, n_tmpl=5),            # tau must be > 0
    tcw.bank_spec(tcw.BANK_RANDOM, (500.0, 3500.0, 1.0), HI, n_tmpl=5),         # n must be > 1
    tcw.bank_spec(tcw.BANK_RANDOM, (3001.0, 3500.0, 3.0), HI, n_tmpl=5),        # lo > hi
    tcw.bank_spec(tcw.BANK_RANDOM, (float("nan"), 3500.0, 3.0), HI, n_tmpl=5),
    tcw.bank_spec(7, LO, HI, n_tmpl=5),                                          # unknown kind
])
def test_invalid_specs(spec):
    assert size(spec)[0] == -1        # TCW_ERR_INVALID_ARGUMENT
