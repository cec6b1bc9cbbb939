"""Checkpoint and resume through the C ABI (kh_save / kh_load_config /
kh_load): a context restored from a checkpoint holds bitwise the saved site
tensors, environments, spectra and discarded weights of every slot, and one
more Trotter step with observables from the restored context gives what the
original context gives (up to the order of the FP64 atomic sums of the Gram
matrices).  Collected after the other library tests."""
import numpy as np
import pytest

import kh_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1906_02220_gb300 as pkg
    return pkg


def _step(g, ctx):
    Hs = [g.bond_hamiltonian(gm, 0.0, 1.0) for gm in "xyz"]
    ctx.eefu_trotter_step(0.0, [1.0, 1.0, 1.0], 0.01, ctm_max_sweeps=3, ctm_min_sweeps=3, ctm_tol=-1.0, info=False)
    return ctx.observables(Hs, ctm_max_sweeps=2, ctm_min_sweeps=2, ctm_tol=-1.0)


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_checkpoint_round_trip_and_resume(g, prec, tmp_path):
    import torch
    D, chi = 3, 20            # n = chi D^2 = 180: the subspace projector path, warm subspaces in use
    A0, B0 = kh_inputs.perturbed_product_state(D, seed=4, eps=0.1)
    ctx = g.Context(D, chi, prec, svd_cut=1e-12 if prec == "fp64" else 1e-6)
    ctx.set_state(torch.as_tensor(A0, device="cuda:0"), torch.as_tensor(B0, device="cuda:0"))
    _step(g, ctx)
    path = tmp_path / "state.khck"
    ctx.save(path)
    ctx2 = g.Context.load(path)
    fields = [f for f, _ in ctx.cfg._fields_]
    assert [getattr(ctx2.cfg, f) for f in fields] == [getattr(ctx.cfg, f) for f in fields]
    for a, b in zip(ctx.get_state(), ctx2.get_state()):
        assert torch.equal(a, b)
    for slot in range(ctx.cfg.n_slots):
        for a, b in zip(ctx.ctm_get_env(slot), ctx2.ctm_get_env(slot)):
            assert torch.equal(a, b)
        for d in range(4):
            (sa, ta), (sb, tb) = ctx.ctm_projectors(slot, d), ctx2.ctm_projectors(slot, d)
            assert torch.equal(sa, sb) and ta == tb
    r1, r2 = _step(g, ctx), _step(g, ctx2)
    tol = 1e-9 if prec == "fp64" else 1e-6
    assert abs(r1["E_site"] - r2["E_site"]) <= tol * max(1.0, abs(r1["E_site"]))
    for a, b in zip(ctx.get_state(), ctx2.get_state()):
        assert (a - b).abs().max().item() <= tol


def test_truncated_checkpoint_is_reported(g, tmp_path):
    import torch
    ctx = g.Context(2, 8, "fp64")
    path = tmp_path / "state.khck"
    ctx.save(path)
    data = path.read_bytes()
    path.write_bytes(data[: len(data) // 2])
    with pytest.raises(g.KhError) as e:
        g.Context.load(path)
    assert "truncated" in str(e.value)
    torch.cuda.synchronize()
