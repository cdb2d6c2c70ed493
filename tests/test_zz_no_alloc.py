"""The allocation-free pairwise contraction (tn_contract_pair_noalloc).

Callers that cannot allocate device memory (their memory belongs to another
allocator, or their host forbids allocation once it runs) use this entry
point; it must give what tn_contract_pair gives.  Each case runs it twice in a
row on different inputs, because every call reuses the same static scratch
array and must not be affected by what the previous call left there.  Each
result is compared with the FP64 oracle contraction of the same host operands
and with tn_contract_pair.  Collected last so that a run stopping at the first
failure has run every other test.
"""
import ctypes
import math

import numpy as np
import pytest

from oracle import pairwise

pytestmark = pytest.mark.gpu

# element-wise bound on |C - C_ref| as a multiple of sqrt(K) rms(A) rms(B)
PAIR_TOL = {("fp32", 4): 1e-5, ("tf32", 4): 3e-3, ("bf16x3", 4): 5e-5, ("fp16x3", 4): 2e-5,
            ("tf32", 3): 6e-3, ("bf16x3", 3): 1e-4, ("fp16x3", 3): 4e-5}


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2111_01066_gb300 import tn
    torch.cuda.set_device(0)
    return tn, torch


def _operands(torch, rng, batch, a_w, b_w):
    a = ((rng.normal(size=(batch, 2 ** len(a_w))) + 1j * rng.normal(size=(batch, 2 ** len(a_w)))) / 2)
    b = ((rng.normal(size=(batch, 2 ** len(b_w))) + 1j * rng.normal(size=(batch, 2 ** len(b_w)))) / 2)
    a = a.astype(np.complex64)
    b = b.astype(np.complex64)
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    return a, b, dev(a), dev(b)


def _noalloc(tn, ta, a_w, tb, b_w, tc, c_w, batch, prec, cm, torch):
    """The entry point called through the C ABI (ctypes), as a C caller would."""
    lib = tn.load()
    return lib.tn_contract_pair_noalloc(
        ctypes.c_void_p(ta.data_ptr()), tn._i32(a_w), len(a_w), ctypes.c_void_p(tb.data_ptr()), tn._i32(b_w),
        len(b_w), ctypes.c_void_p(tc.data_ptr()), tn._i32(c_w), len(c_w), batch, tn.PREC[prec], cm,
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("prec,cm", [("fp32", 4), ("tf32", 4), ("bf16x3", 4), ("fp16x3", 4),
                                     ("bf16x3", 3), ("fp16x3", 3)])
@pytest.mark.parametrize("shape", [(9, 6, 5), (12, 4, 7), (3, 2, 5), (8, 12, 4)])
def test_noalloc_matches_oracle_and_contract_pair_on_two_calls(env, prec, cm, shape):
    tn, torch = env
    nm, nk, nn = shape
    batch = 2
    rng = np.random.default_rng(sum(shape) + len(prec) + cm)
    wires = list(range(10, 10 + nm + nk + nn))
    m_w, k_w, n_w = wires[:nm], wires[nm:nm + nk], wires[nm + nk:]
    a_w = list(rng.permutation(m_w + k_w))
    b_w = list(rng.permutation(k_w + n_w))
    c_w = list(rng.permutation(m_w + n_w))
    tol = PAIR_TOL[(prec, cm)]
    for call in range(2):
        a, b, ta, tb = _operands(torch, rng, batch, a_w, b_w)
        ref = torch.empty((batch, 2 ** len(c_w)), dtype=torch.complex64, device="cuda")
        tn.contract_pair(ta, a_w, tb, b_w, ref, c_w, batch=batch, precision=prec, complex_mult=cm)
        got = torch.full_like(ref, float("nan"))
        st = _noalloc(tn, ta, a_w, tb, b_w, got, c_w, batch, prec, cm, torch)
        assert st == tn.TN_OK, tn.load().tn_last_error()
        tn.device_sync()     # no bounded wait ran out in either call
        g, r = got.cpu().numpy(), ref.cpu().numpy()
        for i in range(batch):
            want = pairwise.contract_pair(a[i].astype(np.complex128), a_w, b[i].astype(np.complex128), b_w, c_w)
            scale = math.sqrt(2 ** nk) * np.sqrt(np.mean(np.abs(a[i]) ** 2) * np.mean(np.abs(b[i]) ** 2))
            assert np.all(np.isfinite(g[i]))
            assert np.max(np.abs(g[i] - want)) <= tol * scale * 8, f"call {call}: vs oracle"
            assert np.max(np.abs(g[i] - r[i])) <= tol * scale * 8, f"call {call}: vs tn_contract_pair"


def test_noalloc_rejects_scratch_beyond_the_static_array(env):
    tn, torch = env
    # B with k = 2^10, n = 2^12 complex entries: about 64 MiB of B' images > 32 MiB
    a_w = list(range(0, 4)) + list(range(100, 110))
    b_w = list(range(100, 110)) + list(range(200, 212))
    c_w = list(range(0, 4)) + list(range(200, 212))
    ta = torch.zeros(2 ** len(a_w), dtype=torch.complex64, device="cuda")
    tb = torch.zeros(2 ** len(b_w), dtype=torch.complex64, device="cuda")
    tc = torch.zeros(2 ** len(c_w), dtype=torch.complex64, device="cuda")
    st = _noalloc(tn, ta, a_w, tb, b_w, tc, c_w, 1, "bf16x3", 4, torch)
    assert st == tn.TN_ERR_ARG
    assert b"static array" in tn.load().tn_last_error()
