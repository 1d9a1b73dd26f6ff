"""vie_apply_noalloc: the FP32 operator for callers that cannot let the
library allocate device memory (its workspace is a fixed device array inside
the library).

Checked through the C ABI:
* on a fresh handle, called before anything else has used the handle's
  operator, it allocates nothing: the handle's device byte count and the
  device's free memory are unchanged across the call;
* its output equals that of vie_apply_device, the allocating entry point, on
  the same inputs, for two calls in a row;
* on a 16^3 grid its output matches the oracle's direct-sum operator;
* grids beyond its fixed scratch and handles it does not cover are refused.

Runs last (file name) so that a failure here comes after every other test."""
import ctypes
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
TOL32 = 2e-5  # FP32 operator tolerance used by the operator parity tests
K0 = 2.0 * math.pi


def _fn(vielib):
    L = vielib.load()
    f = L.vie_apply_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    f.restype = ctypes.c_int
    return L, f


def _eps(n, seed):
    rng = np.random.default_rng(seed)
    return 1.0 + rng.uniform(0.5, 3.0, n) * (rng.uniform(size=n) < 0.4)


def test_noalloc_allocates_nothing_on_a_fresh_handle(vielib):
    import torch
    L, f = _fn(vielib)
    n = (32, 32, 32)
    # a first call on another handle loads the library's kernels and the array
    # (module loading is not an allocation by the entry point)
    with vielib.Handle(n, 1.0 / 64.0, _eps(n, 1), K0) as h0:
        Nb0 = h0.info()["n_body"]
        w0 = torch.zeros(1, 3, Nb0, dtype=torch.complex64, device="cuda")
        y0 = torch.empty_like(w0)
        torch.cuda.synchronize()
        assert f(h0.ptr, w0.data_ptr(), y0.data_ptr(), 1) == 0, L.vie_last_error().decode()
        torch.cuda.synchronize()
    with vielib.Handle(n, 1.0 / 64.0, _eps(n, 2), K0) as hd:
        Nb = hd.info()["n_body"]
        g = torch.Generator(device="cuda").manual_seed(7)
        w = torch.randn(3, 3, Nb, dtype=torch.complex64, device="cuda", generator=g)
        y_na = torch.full_like(w, complex(float("nan"), 0.0))
        y_ref = torch.empty_like(w)
        torch.cuda.synchronize()
        held0 = hd.info()["device_bytes"]
        free0 = torch.cuda.mem_get_info()[0]
        code = f(hd.ptr, w.data_ptr(), y_na.data_ptr(), 3)  # first use of this handle's operator
        assert code == 0, L.vie_last_error().decode()
        torch.cuda.synchronize()
        assert hd.info()["device_bytes"] == held0
        assert torch.cuda.mem_get_info()[0] == free0
        hd.apply_device(w.data_ptr(), y_ref.data_ptr(), 3, vielib.PREC_MIXED)
        torch.cuda.synchronize()
        err = (y_na - y_ref).abs().max().item() / y_ref.abs().max().item()
        assert err <= TOL32, err


@pytest.mark.parametrize("n,R", [((32, 32, 32), 3), ((64, 64, 64), 2)])
def test_noalloc_matches_allocating_entry_point(vielib, n, R):
    import torch
    L, f = _fn(vielib)
    with vielib.Handle(n, 1.0 / 64.0, _eps(n, sum(n)), K0) as hd:
        Nb = hd.info()["n_body"]
        assert all(p in (64, 128) for p in hd.info()["P"])
        for call in range(2):  # two calls in a row, different inputs
            g = torch.Generator(device="cuda").manual_seed(100 + call)
            w = torch.randn(R, 3, Nb, dtype=torch.complex64, device="cuda", generator=g)
            y_ref = torch.empty_like(w)
            y_na = torch.full_like(w, complex(float("nan"), 0.0))
            torch.cuda.synchronize()  # the library runs on its own stream
            code = f(hd.ptr, w.data_ptr(), y_na.data_ptr(), R)
            assert code == 0, L.vie_last_error().decode()
            hd.apply_device(w.data_ptr(), y_ref.data_ptr(), R, vielib.PREC_MIXED)
            torch.cuda.synchronize()
            err = (y_na - y_ref).abs().max().item() / y_ref.abs().max().item()
            assert err <= TOL32, (call, err)


def test_noalloc_matches_oracle_direct_sum(vielib):
    """16^3 grid (padded 32): y = w - chi (K * w) against the oracle's direct
    sum over all sources, element by element."""
    import torch
    from oracle import vie as ovie
    L, f = _fn(vielib)
    n, h = (16, 16, 16), 1.0 / 20.0
    eps = _eps(n, 5)
    chi = ovie.contrast(eps)
    body = chi.reshape(-1) > 0
    rng = np.random.default_rng(11)
    R = 2
    w_full = np.zeros((R, 3) + n, dtype=np.complex128)
    for r in range(R):
        for c in range(3):
            v = rng.standard_normal(n) + 1j * rng.standard_normal(n)
            w_full[r, c] = np.where(chi > 0, v, 0.0)
    w_c = w_full.reshape(R, 3, -1)[:, :, body]  # compact layout, body voxels in C order
    Ktab = ovie.kernel_table(n, h, K0)
    y_or = np.stack([ovie.apply_direct(Ktab, n, chi, w_full[r]) for r in range(R)]).reshape(R, 3, -1)[:, :, body]
    with vielib.Handle(n, h, eps, K0) as hd:
        assert hd.info()["n_body"] == int(body.sum())
        w_h = np.ascontiguousarray(w_c, dtype=np.complex64)  # kept alive until the copy is done
        w = torch.from_numpy(w_h).cuda()
        y = torch.empty_like(w)
        y2 = torch.empty_like(w)
        torch.cuda.synchronize()  # the library runs on its own stream
        assert np.array_equal(w.cpu().numpy(), w_h)
        assert f(hd.ptr, w.data_ptr(), y.data_ptr(), R) == 0, L.vie_last_error().decode()
        hd.apply_device(w.data_ptr(), y2.data_ptr(), R, vielib.PREC_MIXED)
        torch.cuda.synchronize()
        y_na = y.cpu().numpy().astype(np.complex128)
        y_ad = y2.cpu().numpy().astype(np.complex128)
    s = np.abs(y_or).max()
    e_na, e_ad = np.abs(y_na - y_or).max() / s, np.abs(y_ad - y_or).max() / s
    assert e_na <= TOL32 and e_ad <= TOL32, (e_na, e_ad, np.abs(y_na - y_ad).max() / s)


def test_noalloc_rejects_grids_beyond_its_scratch(vielib):
    import torch
    L, f = _fn(vielib)
    n = (128, 128, 128)
    eps = np.ones(n)
    eps[60:70, 60:70, 60:70] = 2.0
    with vielib.Handle(n, 1.0 / 128.0, eps, K0) as hd:
        Nb = hd.info()["n_body"]
        w = torch.zeros(1, 3, Nb, dtype=torch.complex64, device="cuda")
        y = torch.zeros_like(w)
        code = f(hd.ptr, w.data_ptr(), y.data_ptr(), 1)
        assert code == vielib.VIE_EINVAL
        assert b"scratch" in L.vie_last_error()


def test_noalloc_rejects_the_generic_fft_path(vielib):
    import torch
    L, f = _fn(vielib)
    n = (16, 16, 16)
    with vielib.Handle(n, 1.0 / 20.0, _eps(n, 9), K0) as hd:
        hd.set_fft_path(1)
        Nb = hd.info()["n_body"]
        w = torch.zeros(1, 3, Nb, dtype=torch.complex64, device="cuda")
        y = torch.zeros_like(w)
        assert f(hd.ptr, w.data_ptr(), y.data_ptr(), 1) == vielib.VIE_EINVAL
        assert b"generic" in L.vie_last_error()
