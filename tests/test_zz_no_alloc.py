"""mfp_rhs_noalloc serves callers that must not allocate device memory after
their set-up (memory handed to their own pool, or loops that cannot take
cudaMalloc's implicit synchronisation).  It must give the same load vector
as mfp_rhs, which stages the forcing parameters in a buffer the library
allocates, within the 1e-12 relative tolerance of the other parity tests.
Two calls in a row with different parameters check that the shared fixed
parameter array is refreshed on every call."""
import ctypes

import numpy as np
import pytest
import torch

from conftest import rel_err
from paper_1611_03029_gb300 import synthetic

pytestmark = pytest.mark.gpu


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@pytest.mark.parametrize("disc,stride", [("cg", 1), ("dg", 2)])
def test_rhs_noalloc_matches_rhs(mfp, disc, stride):
    lib = mfp.lib()
    op = mfp.Poisson(3, 4, 2, 3, disc=disc, mapping="sine", map_param=0.1,
                     n_levels=1)
    n = op.n_dofs()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for seed in (1000, 1001):
        g = np.ascontiguousarray(synthetic.gaussian_terms(seed))
        ref = op.rhs(1, g).cpu().numpy()
        out = torch.full((n * stride,), float("nan"), dtype=torch.float64,
                         device="cuda")
        st = lib.mfp_rhs_noalloc(op._h, 1, _dp(g), g.shape[0],
                                 ctypes.c_void_p(out.data_ptr()), stride, s)
        assert st == mfp.MFP_OK, lib.mfp_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()[::stride]
        assert rel_err(got, ref) <= 1e-12


@pytest.mark.parametrize("disc", ["cg", "dg"])
def test_rhs_noalloc_boundary_data(mfp, disc):
    # f_kind 2 (Dirichlet and Neumann data of a Gaussian sum) on a box with
    # Neumann sides; CG rows are atomic sums, equal up to rounding
    lib = mfp.lib()
    op = mfp.Poisson(3, 2, 2, 2, disc=disc, n_levels=1, neumann_sides=(0, 3),
                     box=(-1.0, 1.0))
    g = np.array([[-0.5, 0.5, 0.25, 0.2, 2.0], [0.5, -0.5, 0.5, 0.3, -1.0]])
    ref = op.rhs(2, g).cpu().numpy()
    out = torch.zeros(op.n_dofs(), dtype=torch.float64, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.mfp_rhs_noalloc(op._h, 2, _dp(g), g.shape[0],
                             ctypes.c_void_p(out.data_ptr()), 1, s)
    assert st == mfp.MFP_OK, lib.mfp_last_error()
    torch.cuda.synchronize()
    assert rel_err(out.cpu().numpy(), ref) <= 1e-14


def test_rhs_noalloc_rejects_too_many_terms(mfp):
    lib = mfp.lib()
    op = mfp.Poisson(2, 2, 2, 1, n_levels=1)
    out = torch.zeros(op.n_dofs(), dtype=torch.float64, device="cuda")
    big = np.zeros((4097, 5))
    big[:, 3] = 0.1
    st = lib.mfp_rhs_noalloc(op._h, 1, _dp(big), 4097,
                             ctypes.c_void_p(out.data_ptr()), 1, None)
    assert st == mfp.MFP_ERR_ARG
    assert b"4096" in lib.mfp_last_error()


@pytest.mark.parametrize("disc", ["cg", "dg"])
def test_rhs_noalloc_takes_no_device_memory(mfp, disc):
    # on a freshly created context: the device's free memory is the same
    # before and after the first two calls (mfp_create did the set-up)
    lib = mfp.lib()
    op = mfp.Poisson(4, 3, 2, 3, disc=disc, n_levels=1)
    out = torch.zeros(op.n_dofs(), dtype=torch.float64, device="cuda")
    g = np.ascontiguousarray(synthetic.gaussian_terms(1002))
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        st = lib.mfp_rhs_noalloc(op._h, 1, _dp(g), g.shape[0],
                                 ctypes.c_void_p(out.data_ptr()), 1, s)
        assert st == mfp.MFP_OK, lib.mfp_last_error()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    ref = op.rhs(1, g).cpu().numpy()
    assert rel_err(out.cpu().numpy(), ref) <= 1e-12
