"""CPU-side checks of the C-ABI library: it loads, exports every entry point
declared in include/eefu.h, sizes its workspace, and its host-side gate
builders agree with the oracle.  No GPU compute is called here."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_1906_02220_gb300", "libeefu_gb300.so")


@pytest.fixture(scope="module")
def g():
    if not os.path.exists(LIB):
        from paper_1906_02220_gb300 import build
        build.build()
    import paper_1906_02220_gb300 as pkg
    return pkg


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "eefu.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w\s\*]*?\b(\w+)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "defined")))


def test_header_declares_the_binding_list(g):
    assert sorted(g.ABI_FUNCTIONS) == _declared_functions()


def test_library_exports_every_declared_symbol(g):
    import ctypes
    lib = ctypes.CDLL(LIB)
    for name in _declared_functions():
        assert hasattr(lib, name), name
    out = os.popen("nm -D --defined-only %s" % LIB).read()
    for name in _declared_functions():
        assert re.search(r"\bT %s\b" % name, out), name


def test_workspace_sizing(g):
    import ctypes
    c = g.default_config(4, 64, "fp32")
    b32 = g.lib().kh_workspace_bytes(ctypes.byref(c))
    c = g.default_config(4, 64, "fp64")
    b64 = g.lib().kh_workspace_bytes(ctypes.byref(c))
    assert 0 < b32 < b64 < 2 ** 31
    for bad in (dict(D=0), dict(chi=0), dict(D=9), dict(prec=7), dict(n_slots=0)):
        c = g.default_config(2, 8, "fp64")
        for k, v in bad.items():
            setattr(c, k, v)
        assert g.lib().kh_workspace_bytes(ctypes.byref(c)) == 0


@pytest.mark.parametrize("D,chi,prec,ok", [(4, 96, "fp64", True), (4, 97, "fp64", False),
                                            (4, 144, "fp32", True), (4, 145, "tf32x3", False),
                                            (2, 28, "fp64", True), (3, 12, "fp64", True)])
def test_workspace_sizing_at_the_jacobi_limits(g, D, chi, prec, ok):
    """The projector's one-CTA Jacobi takes k = chi + 16 up to 112 (FP64) or
    160 (FP32 family); below n = chi D^2 <= k the dense path takes k = n.
    Larger configurations are rejected (0 bytes), the limits themselves are
    accepted."""
    import ctypes
    c = g.default_config(D, chi, prec)
    b = g.lib().kh_workspace_bytes(ctypes.byref(c))
    assert (b > 0) == ok


@pytest.mark.parametrize("chi,ok", [(144, True), (145, False)])
def test_fp64_projector_option_keeps_the_single_precision_limit(g, chi, ok):
    """With proj_fp64 the projector SVD is the FP32 Jacobi refined in FP64, so
    k = chi + 16 keeps the FP32 solver's bound of 160; the FP64 scratch is
    extra, and only 0 and 1 are accepted."""
    import ctypes
    c = g.default_config(4, chi, "tf32x3", proj_fp64=1)
    b = g.lib().kh_workspace_bytes(ctypes.byref(c))
    assert (b > 0) == ok
    if ok:
        c0 = g.default_config(4, chi, "tf32x3")
        assert b > g.lib().kh_workspace_bytes(ctypes.byref(c0))
    c.proj_fp64 = 2
    assert g.lib().kh_workspace_bytes(ctypes.byref(c)) == 0


@pytest.mark.parametrize("gamma", ["x", "y", "z"])
def test_host_gates_match_oracle(g, gamma):
    from oracle import model
    J, K, hA, hB = 0.37, -1.4, 0.2, -0.6
    bias = (hA, hB) if gamma == "z" else (0.0, 0.0)
    H = g.bond_hamiltonian(gamma, J, K, *bias)
    Ho = model.bond_hamiltonian(gamma, J, K, hA=bias[0], hB=bias[1])
    assert np.abs(H - Ho).max() < 1e-15
    for tau in (0.0, 0.0025, 0.3):
        assert np.abs(g.gate(H, tau) - model.gate(gamma, tau, J, K, hA=bias[0], hB=bias[1])).max() < 1e-14


def test_status_codes_on_bad_arguments_without_gpu(g):
    import ctypes
    assert g.lib().kh_bond_hamiltonian(5, 0.0, 0.0, 0.0, 0.0, None) == g.KH_EINVAL
    assert g.lib().kh_create(None, None, None, 0, None) == g.KH_EINVAL


def test_checkpoint_header_without_gpu(g, tmp_path):
    """kh_load_config is host-only: a missing file, a foreign file and a
    truncated header are rejected; a header (magic + configuration) is read
    back field by field.  kh_save / kh_load reject null arguments before any
    GPU work."""
    import ctypes
    cfg = g.KhConfig()
    assert g.lib().kh_load_config(str(tmp_path / "missing").encode(), ctypes.byref(cfg)) == g.KH_EINVAL
    (tmp_path / "foreign").write_bytes(b"NOTACKPT" + b"\0" * 256)
    assert g.lib().kh_load_config(str(tmp_path / "foreign").encode(), ctypes.byref(cfg)) == g.KH_EINVAL
    (tmp_path / "short").write_bytes(b"KHCKPT01" + b"\0" * 8)
    assert g.lib().kh_load_config(str(tmp_path / "short").encode(), ctypes.byref(cfg)) == g.KH_EINVAL
    c0 = g.default_config(3, 20, "tf32x3", n_slots=6, seed=77)
    (tmp_path / "header").write_bytes(b"KHCKPT01" + bytes(c0))
    assert g.lib().kh_load_config(str(tmp_path / "header").encode(), ctypes.byref(cfg)) == g.KH_OK
    assert bytes(cfg) == bytes(c0)
    assert g.lib().kh_save(None, b"x") == g.KH_EINVAL
    ctx = ctypes.c_void_p()
    assert g.lib().kh_load(ctypes.byref(ctx), str(tmp_path / "missing").encode(), None, 0, None) == g.KH_EINVAL
    assert ctx.value is None


def test_batch_gradient_and_selftest_arguments_without_gpu(g):
    """Host-side validation of the later entry points, before any GPU work:
    the batch call rejects empty or null context lists and null couplings;
    the cost gradient rejects a null context; the layered self-test sizes its
    scratch for TF32, 3xTF32 and BF16 and returns 0 for an unknown pass count."""
    import ctypes
    P = ctypes.c_void_p
    one = (P * 1)(None)
    J = np.zeros(1)
    K = np.zeros(3)
    traj = np.zeros(13)
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    lib = g.lib()
    assert lib.eefu_evolve_batch(ctypes.cast(one, ctypes.POINTER(P)), 1, dp(J), dp(K), None, None, 0.01, 1, 1, 4, 1,
                                 -1.0, 2, 1, -1.0, dp(traj), None) == g.KH_EINVAL
    assert lib.eefu_evolve_batch(None, 0, dp(J), dp(K), None, None, 0.01, 1, 1, 4, 1, -1.0, 2, 1, -1.0, dp(traj),
                                 None) == g.KH_EINVAL
    gate = np.eye(4)
    cost = np.zeros(3)
    assert lib.eefu_cost_gradient(None, 0, dp(gate), None, None, 0, 1, 1e-12, None, None, dp(cost)) == g.KH_EINVAL
    sizes = [lib.kh_selftest_site_layered_bytes(npass, 4, 16, 4096) for npass in (1, 3, 16)]
    assert all(s > 0 for s in sizes)
    # the 3xTF32 operand images carry a low part: more scratch than one TF32 pass
    assert sizes[1] > sizes[0]
    assert lib.kh_selftest_site_layered_bytes(2, 4, 16, 4096) == 0
    assert lib.kh_selftest_site_layered_bytes(3, 9, 16, 4096) == 0


def test_flux_operators_match_the_oracle(g):
    """The library's real-form flux operators (host code) against the oracle's
    complex ones: each position's operator is the oracle's up to a factor i
    (one sigma^y at that composite) or 1, the factors multiply to -1 (two
    sigma^y), so W_p = -(product of the real forms) -- in every mapping."""
    import ctypes
    from oracle import observables
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    for gi, gamma in enumerate("xyz"):
        ops = np.zeros((4, 16, 16))
        assert g.lib().kh_flux_operators(gi, dp(ops)) == g.KH_OK
        ref = observables.flux_operators(gamma)
        phase = 1.0 + 0j
        for f in range(4):
            if np.abs(ref[f].imag).max() > 0:
                assert np.abs(ref[f] - 1j * ops[f]).max() < 1e-15, (gamma, f)
                phase *= 1j
            else:
                assert np.abs(ref[f] - ops[f]).max() < 1e-15, (gamma, f)
        assert abs(phase + 1.0) < 1e-15
    assert g.lib().kh_flux_operators(3, dp(np.zeros(1024))) == g.KH_EINVAL
    assert g.lib().kh_flux_operators(0, None) == g.KH_EINVAL


def test_plaquette_and_flux_arguments_without_gpu(g):
    """ctm_plaquette and ctm_flux reject a null context before any GPU work."""
    import ctypes
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    ops = np.tile(np.eye(16), (4, 1, 1))
    out = np.zeros(2)
    assert g.lib().ctm_plaquette(None, 0, dp(ops), dp(out)) == g.KH_EINVAL
    assert g.lib().ctm_flux(None, 3, 0, dp(out)) == g.KH_EINVAL


@pytest.mark.parametrize("prec", ["tf32x3", "tf32", "bf16"])
@pytest.mark.parametrize("D", [2, 4, 6, 8])
def test_layered_form_sizes_the_workspace(g, prec, D):
    """In the tensor-core precisions the layered site contraction keeps its
    chi^2 D^4 p intermediate on chip: doubling p_max grows the workspace only
    by the slots' site-tensor copies and operand images (O(p D^8) at most),
    while the CUDA-core layered form grows by its p n^2 scratch in each of
    the three lanes (n = chi D^2)."""
    chi = 64
    n2 = (chi * D * D) ** 2
    ws = lambda prec_, p, **kw: g.lib().kh_workspace_bytes(g.default_config(D, chi, prec_, p_max=p, **kw))
    tc_growth = ws(prec, 16) - ws(prec, 8)
    simt_growth = ws("fp32", 16, site_form=1) - ws("fp32", 8, site_form=1)
    assert simt_growth >= 3 * 8 * n2 * 4
    assert 0 <= tc_growth < 0.1 * simt_growth
