"""Failure detection through status codes, injected on the host (no GPU
fault, trap or hang): forced non-convergence returns KH_ENOCONV, a NaN
seeded into the site tensor returns KH_ENUMERIC from the sweep that meets it,
and afterwards the same context, given a finite tensor and a fresh
environment, converges to Onsager's free energy again.  Collected after the
other library tests."""
import numpy as np
import pytest

from oracle import exact

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1906_02220_gb300 as pkg
    return pkg


def _t(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda:0")


def _recovers(g, ctx, prec):
    Kh, Kv = 0.3, 0.2
    ctx.ctm_set_tensor(0, _t(exact.ising_peps(Kh, Kv, gauge_seed=7)))
    ctx.ctm_init(0)
    ctx.ctm_sweep(0, 300, 3, 1e-11 if prec == "fp64" else 2e-4)
    assert abs(np.log(ctx.ctm_kappa(0)) - exact.onsager_lnZ(Kh, Kv)) < (1e-9 if prec == "fp64" else 2e-5)


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_forced_non_convergence_is_reported(g, prec):
    ctx = g.Context(2, 16, prec, p_max=2, n_slots=1, svd_cut=1e-12 if prec == "fp64" else 1e-6)
    ctx.ctm_set_tensor(0, _t(exact.ising_peps(0.3, 0.2, gauge_seed=7)))
    with pytest.raises(g.KhError) as e:
        ctx.ctm_sweep(0, 1, 1, 0.0)            # one sweep cannot reach tolerance 0
    assert e.value.status == g.KH_ENOCONV
    _recovers(g, ctx, prec)


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_nan_in_the_site_tensor_is_reported(g, prec):
    ctx = g.Context(2, 16, prec, p_max=2, n_slots=1, svd_cut=1e-12 if prec == "fp64" else 1e-6)
    T = exact.ising_peps(0.3, 0.2, gauge_seed=7)
    T[0, 1, 0, 1, 0] = np.nan
    ctx.ctm_set_tensor(0, _t(T))
    with pytest.raises(g.KhError) as e:
        ctx.ctm_sweep(0, 20, 1, 1e-10)
    assert e.value.status == g.KH_ENUMERIC
    assert "NaN" in str(e.value)
    _recovers(g, ctx, prec)
