"""The allocation-free GEMM entry point (kh_gemm_noalloc) against the
scratch-taking one (kh_selftest_gemm): same output within the tolerance the
kernel tests use, on two calls in a row (the static scratch keeps the last
call's contents, so the second call must not depend on it).  Collected
after the kernel and parity tests on purpose; it passes alone in a fresh
process or after the other tests."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-13, "fp32": 3e-6, "tf32x3": 1e-5, "tf32": 4e-3}


@pytest.fixture(scope="module")
def g():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1906_02220_gb300 as pkg
    return pkg


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3"])
def test_noalloc_matches_scratch_entry_point_twice(g, prec):
    import torch
    rng = np.random.default_rng(11)
    # both shapes split K over CTAs (few output tiles, long K) inside the scratch
    for call, (M, N, K) in enumerate([(256, 96, 512), (200, 300, 384)]):
        assert g.lib().kh_selftest_bytes(M, N, K) <= g.lib().kh_gemm_noalloc_max_bytes()
        A = torch.as_tensor(rng.standard_normal((M, K)), device="cuda:0")
        B = torch.as_tensor(rng.standard_normal((K, N)), device="cuda:0")
        ref = g.selftest_gemm(A, B, prec).cpu().numpy()
        out = g.gemm_noalloc(A, B, prec).cpu().numpy()
        scale = np.sqrt(K) * float(A.abs().max()) * float(B.abs().max())
        assert np.abs(out - ref).max() <= TOL[prec] * scale, (call, np.abs(out - ref).max())
        exact = A.cpu().numpy() @ B.cpu().numpy()
        assert np.abs(out - exact).max() <= TOL[prec] * scale


def test_noalloc_rejects_sizes_beyond_the_static_scratch(g):
    import torch
    lib = g.lib()
    limit = lib.kh_gemm_noalloc_max_bytes()
    assert limit == 16 << 20
    n = 4096                                    # needs far more than 16 MiB of scratch
    assert lib.kh_selftest_bytes(n, n, n) > limit
    A = torch.zeros((1, 1), dtype=torch.float64, device="cuda:0")
    st = lib.kh_gemm_noalloc(0, n, n, n, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(A.data_ptr()),
                             ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(0))
    assert st == g.KH_EINVAL
