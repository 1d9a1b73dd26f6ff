"""vie_apply_noalloc: the FP32 operator for callers that cannot let the
library allocate device memory (its workspace is a fixed device array inside
the library).  Checked through the C ABI against vie_apply_device, the
allocating entry point, on the same inputs, for two calls in a row; and its
size limit.  Runs last (file name) so that a failure here comes after every
other test."""
import ctypes

import numpy as np
import pytest

from paper_2508_16471_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL32 = 2e-5  # FP32 operator tolerance used by the operator parity tests


def _fn(vielib):
    L = vielib.load()
    f = L.vie_apply_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    f.restype = ctypes.c_int
    return L, f


@pytest.mark.parametrize("n,R", [((32, 32, 32), 3), ((64, 64, 64), 2)])
def test_noalloc_matches_allocating_entry_point(vielib, n, R):
    import torch
    L, f = _fn(vielib)
    rng = np.random.default_rng(sum(n))
    eps = 1.0 + rng.uniform(0.5, 3.0, n) * (rng.uniform(size=n) < 0.4)
    with vielib.Handle(n, 1.0 / 64.0, eps, 2.0 * np.pi) as hd:
        Nb = hd.info()["n_body"]
        assert all(p in (64, 128) for p in hd.info()["P"])
        for call in range(2):  # two calls in a row, different inputs
            g = torch.Generator(device="cuda").manual_seed(100 + call)
            w = torch.randn(R, 3, Nb, dtype=torch.complex64, device="cuda", generator=g)
            y_ref = torch.empty_like(w)
            y_na = torch.full_like(w, complex(float("nan"), 0.0))
            hd.apply_device(w.data_ptr(), y_ref.data_ptr(), R, vielib.PREC_MIXED)
            code = f(hd.ptr, w.data_ptr(), y_na.data_ptr(), R)
            assert code == 0, L.vie_last_error().decode()
            torch.cuda.synchronize()
            err = (y_na - y_ref).abs().max().item() / y_ref.abs().max().item()
            assert err <= TOL32, (call, err)


def test_noalloc_rejects_grids_beyond_its_scratch(vielib):
    import torch
    L, f = _fn(vielib)
    n = (128, 128, 128)
    eps = np.ones(n)
    eps[60:70, 60:70, 60:70] = 2.0
    with vielib.Handle(n, 1.0 / 128.0, eps, 2.0 * np.pi) as hd:
        Nb = hd.info()["n_body"]
        w = torch.zeros(1, 3, Nb, dtype=torch.complex64, device="cuda")
        y = torch.zeros_like(w)
        code = f(hd.ptr, w.data_ptr(), y.data_ptr(), 1)
        assert code == vielib.VIE_EINVAL
        assert b"scratch" in L.vie_last_error()
