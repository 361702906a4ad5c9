"""GPU tests of the numerics routines behind the reduced-precision snapshots and
the Kahan-compensated imaging sums, through the C ABI self-test entry points
(efwi_selftest_store, efwi_selftest_kahan), against FP64 arithmetic.

Reduced-precision store (checkpoints and stored forward velocities): with
s = max |x| of the snapshot field, x is stored as RNE(x 2^k), s 2^k in
[2^14, 2^15), and read back as y 2^-k.  The power-of-two scalings are exact, so
per element |x^ - x| <= 2^-11 |x| (FP16) or 2^-8 |x| (BF16) wherever x 2^k is a
normal number of the format -- for FP16 every |x| >= s 2^-28 -- and
<= 2^-25 2^-k (half the smallest FP16 subnormal) below that.
"""
import copy
import ctypes as C

import numpy as np
import pytest
import torch

import workloads as W
from common import rounded
from oracle import elastic as E

pytestmark = pytest.mark.gpu
FP16, BF16 = 1, 2


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2305_14130_gb300 import _abi
    return _abi.load()


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


@pytest.fixture(scope="module")
def snapshot():
    """Mid-run state x^300 of the 200x100 single-shot configuration (FP64 oracle)."""
    p = rounded(W.single_shot_200x100())
    a = copy.deepcopy(p.acq)
    a.nt = 301
    sh = E.Shot(a, 0, p.vp[0] if p.vp.ndim == 3 else p.vp, p.vs[0] if p.vs.ndim == 3 else p.vs,
                p.rho[0] if p.rho.ndim == 3 else p.rho)
    _, _, ck = sh.forward(keep_every=300)
    st = ck[300]
    return {k: np.float32(st[k]) for k in ("vx", "vz", "sxx", "szz", "sxz")}


def _roundtrip(lib, store, x32):
    x = torch.tensor(x32.ravel(), device="cuda")
    y = torch.empty_like(x)
    enc = torch.empty(x.numel(), dtype=torch.int16, device="cuda")
    s = torch.empty((), dtype=torch.float32, device="cuda")
    rc = lib.efwi_selftest_store(store, x.numel(), C.c_void_p(x.data_ptr()), C.c_void_p(enc.data_ptr()),
                                 C.c_void_p(y.data_ptr()), C.c_void_p(s.data_ptr()), _stream())
    assert rc == 0, lib.efwi_last_error(None)
    torch.cuda.synchronize()
    return float(s.item()), y.cpu().numpy().astype(np.float64), enc.cpu().numpy()


def _store_exp(s):
    """k with s 2^k in [2^14, 2^15), clamped to [-126, 126] (from the float32 bits of s)."""
    e = int((np.float32(s).view(np.uint32) >> 23) & 0xFF)
    return int(np.clip(141 - e, -126, 126))


def _bf16_rne(v32):
    """Round float32 values to bfloat16 (nearest, ties to even) and back, on the bits."""
    u = v32.astype(np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


@pytest.mark.parametrize("store", [FP16, BF16])
def test_store_error_bound_on_a_mid_run_snapshot(lib, snapshot, store):
    rel = 2.0 ** -11 if store == FP16 else 2.0 ** -8
    worst = {}
    for name, x32 in snapshot.items():
        x = x32.astype(np.float64).ravel()
        s, y, _ = _roundtrip(lib, store, x32)
        assert s == float(np.abs(x32).max()) > 0
        k = _store_exp(s)
        assert 2.0 ** 14 <= s * 2.0 ** k < 2.0 ** 15
        err = np.abs(y - x)
        normal = np.abs(x) * 2.0 ** k >= (2.0 ** -14 if store == FP16 else 2.0 ** -126)
        assert np.all(err[normal] <= rel * np.abs(x[normal])), name
        assert np.all(err[~normal] <= 2.0 ** -25 * 2.0 ** -k), name
        # no flush to zero: every element down to s 2^-28 keeps the format's relative precision
        assert np.all(normal[np.abs(x) >= s * 2.0 ** -28])
        # the rounding is round-to-nearest-even of x 2^k, bit for bit
        v = np.float32(x32.ravel() * np.float32(2.0 ** k))
        ref = (v.astype(np.float16).astype(np.float32) if store == FP16 else _bf16_rne(v)) * np.float32(2.0 ** -k)
        assert np.array_equal(np.float32(y), ref), name
        nz = normal & (x != 0)
        worst[name] = float((err[nz] / np.abs(x[nz])).max() / rel)
    print(f"store {store}: worst per-element error / (unit roundoff x |x|): {worst}")
    # half-ulp rounding reaches close to the bound somewhere in a field of this size
    assert max(worst.values()) > 0.9


@pytest.mark.parametrize("store", [FP16, BF16])
def test_store_edge_cases(lib, store):
    # all zeros: stored and read back exactly, s = 0
    s, y, _ = _roundtrip(lib, store, np.zeros(1000, np.float32))
    assert s == 0.0 and not y.any()
    # magnitudes over 60 binades, both signs, a ragged length
    rng = np.random.default_rng(3)
    x32 = np.float32(rng.choice([-1, 1], 4099) * 2.0 ** rng.uniform(-60, 0, 4099))
    s, y, _ = _roundtrip(lib, store, x32)
    x = x32.astype(np.float64)
    k = _store_exp(s)
    rel = 2.0 ** -11 if store == FP16 else 2.0 ** -8
    normal = np.abs(x) * 2.0 ** k >= (2.0 ** -14 if store == FP16 else 2.0 ** -126)
    assert np.all(np.abs(y - x)[normal] <= rel * np.abs(x[normal]))
    assert np.all(np.abs(y - x)[~normal] <= 2.0 ** -25 * 2.0 ** -k)
    # tiny and huge fields: the power of two is clamped, nothing overflows
    for scale in (1e-36, 1e30):
        s, y, _ = _roundtrip(lib, store, np.float32(np.linspace(-1, 1, 257) * scale))
        assert np.all(np.isfinite(y))
        assert np.abs(y - np.float32(np.linspace(-1, 1, 257) * scale)).max() <= rel * scale


def test_store_fp32_is_a_copy(lib, snapshot):
    x32 = snapshot["sxx"]
    s, y, _ = _roundtrip(lib, 0, x32)
    assert np.array_equal(np.float32(y), x32.ravel())


def test_kahan_fold_against_fp64_sum(lib):
    """The imaging sums' fold: nterms FP32 partial sums added into a total with
    Kahan compensation.  Against the exact (FP64) sum of the same FP32 terms the
    error stays within the classic bound (2u + O(N u^2)) sum |x_i|, u = 2^-24,
    and far below that of plain FP32 accumulation in the same order."""
    n, nterms = 8192, 2000
    rng = np.random.default_rng(5)
    # imaging-like terms: a slowly varying positive part, a signed part and rare spikes
    terms = np.float32(1.0 + 1e-3 * rng.standard_normal((nterms, n))
                       + 0.5 * np.sin(np.arange(nterms) / 37.0)[:, None]
                       + (rng.random((nterms, n)) < 1e-3) * 1e3 * rng.standard_normal((nterms, n)))
    t = torch.tensor(terms, device="cuda")
    tot = torch.empty(n, device="cuda")
    cmp = torch.empty(n, device="cuda")
    rc = lib.efwi_selftest_kahan(n, nterms, C.c_void_p(t.data_ptr()), C.c_void_p(tot.data_ptr()),
                                 C.c_void_p(cmp.data_ptr()), _stream())
    assert rc == 0, lib.efwi_last_error(None)
    torch.cuda.synchronize()
    assert not t.any()                          # terms are consumed
    exact = terms.astype(np.float64).sum(0)
    absum = np.abs(terms.astype(np.float64)).sum(0)
    err = np.abs(tot.cpu().numpy().astype(np.float64) - exact)
    u = 2.0 ** -24
    assert np.all(err <= (2 * u + nterms * u * u) * absum)
    naive = np.zeros(n, np.float32)
    for k in range(nterms):
        naive += terms[k]
    err_naive = np.abs(naive.astype(np.float64) - exact)
    print(f"Kahan fold: max error {err.max():.3e}, plain FP32 sum {err_naive.max():.3e}")
    assert np.linalg.norm(err) * 20 < np.linalg.norm(err_naive)
