"""Python binding of the eeFU GB300 library (argument marshalling only).

Every call forwards to the C ABI declared in include/eefu.h; all arithmetic
of the method runs in the CUDA library.  PyTorch supplies device memory (the
workspace and the caller's tensors) and the stream.  Importing this package
fails loudly if the compiled library is missing: there is no fallback.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libeefu_gb300.so")

KH_OK, KH_EINVAL, KH_ENOMEM, KH_ENOCONV, KH_ENUMERIC, KH_ETIMEOUT, KH_ECUDA = range(7)
STATUS_NAMES = ["KH_OK", "KH_EINVAL", "KH_ENOMEM", "KH_ENOCONV", "KH_ENUMERIC", "KH_ETIMEOUT", "KH_ECUDA"]
PREC = {"fp64": 0, "fp32": 1, "tf32": 2, "tf32x3": 3, "bf16": 4}
GAMMA = {"x": 0, "y": 1, "z": 2}
PROFILE_NAMES = ["half_system_product", "site_layer", "corners", "projector_svd", "absorb", "metric", "als_gauge",
                 "svd_jacobi", "cholqr_orth", "subspace_gemm"]

# every entry point of include/eefu.h (checked by the CPU symbol test)
ABI_FUNCTIONS = [
    "kh_config_defaults", "kh_workspace_bytes", "kh_create", "kh_destroy", "kh_last_error",
    "kh_set_state", "kh_get_state", "ctm_set_tensor", "ctm_build_composite", "ctm_init",
    "ctm_copy_env", "ctm_sweep", "ctm_projectors", "ctm_get_env", "ctm_metric", "ctm_kappa",
    "ctm_expval", "ctm_correlation_length", "ctm_plaquette", "ctm_flux", "eefu_apply_gate", "eefu_cost_gradient", "observables", "kh_version", "kh_bond_hamiltonian", "kh_gate", "kh_flux_operators",
    "eefu_trotter_step", "eefu_evolve", "eefu_evolve_flux", "eefu_evolve_batch", "kh_launch_count", "kh_profile", "kh_selftest_bytes", "kh_selftest_gemm",
    "kh_selftest_symeig", "kh_selftest_svd", "kh_selftest_svd_refined", "kh_selftest_orth", "kh_selftest_fp64_newton",
    "kh_selftest_site_layered_bytes", "kh_selftest_site_layered", "kh_gemm_noalloc",
    "kh_gemm_noalloc_max_bytes", "kh_save", "kh_load_config", "kh_load",
]


class KhConfig(ctypes.Structure):
    _fields_ = [
        ("D", ctypes.c_int), ("chi", ctypes.c_int), ("prec", ctypes.c_int), ("n_slots", ctypes.c_int),
        ("p_max", ctypes.c_int), ("svd_oversample", ctypes.c_int), ("svd_iters_cold", ctypes.c_int),
        ("svd_iters_warm", ctypes.c_int), ("jacobi_max_sweeps", ctypes.c_int), ("svd_cut", ctypes.c_double),
        ("als_tol", ctypes.c_double), ("als_max_iter", ctypes.c_int), ("als_reg", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("proj_fp64", ctypes.c_int), ("site_form", ctypes.c_int),
    ]


class KhError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < 7 else status, msg))
        self.status = status


def load_library(path=LIB_PATH):
    if not os.path.exists(path):
        raise ImportError("eeFU CUDA library not built (%s); run paper_1906_02220_gb300.build.build()" % path)
    lib = ctypes.CDLL(path)
    P, I, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    cfgp = ctypes.POINTER(KhConfig)
    sig = {
        "kh_config_defaults": (None, [cfgp]),
        "kh_workspace_bytes": (S, [cfgp]),
        "kh_create": (I, [ctypes.POINTER(P), cfgp, P, S, P]),
        "kh_destroy": (None, [P]),
        "kh_last_error": (ctypes.c_char_p, [P]),
        "kh_version": (ctypes.c_char_p, []),
        "kh_set_state": (I, [P, P, P]),
        "kh_get_state": (I, [P, P, P]),
        "ctm_set_tensor": (I, [P, I, P, I]),
        "ctm_build_composite": (I, [P, I, I, dp]),
        "ctm_init": (I, [P, I, dp]),
        "ctm_copy_env": (I, [P, I, I]),
        "ctm_sweep": (I, [P, I, I, I, D, ip, dp]),
        "ctm_projectors": (I, [P, I, I, P, dp]),
        "ctm_get_env": (I, [P, I, P, P]),
        "ctm_metric": (I, [P, I, P]),
        "ctm_kappa": (I, [P, I, dp]),
        "ctm_expval": (I, [P, I, dp, I, dp]),
        "ctm_correlation_length": (I, [P, I, I, I, D, dp]),
        "ctm_plaquette": (I, [P, I, dp, dp]),
        "ctm_flux": (I, [P, I, I, dp]),
        "eefu_apply_gate": (I, [P, I, dp, I, I, D, dp]),
        "eefu_cost_gradient": (I, [P, I, dp, P, P, I, I, D, P, P, dp]),
        "observables": (I, [P, dp, D, D, I, I, D, dp]),
        "kh_bond_hamiltonian": (I, [I, D, D, D, D, dp]),
        "kh_gate": (I, [dp, D, dp]),
        "kh_flux_operators": (I, [I, dp]),
        "eefu_trotter_step": (I, [P, D, dp, D, D, D, I, I, D, dp]),
        "eefu_evolve": (I, [P, D, dp, D, D, D, I, I, I, I, D, I, I, D, dp]),
        "eefu_evolve_flux": (I, [P, D, dp, D, D, D, I, I, I, I, D, I, I, D, dp, dp]),
        "eefu_evolve_batch": (I, [ctypes.POINTER(P), I, dp, dp, dp, dp, D, I, I, I, I, D, I, I, D, dp, ip]),
        "kh_launch_count": (ctypes.c_ulonglong, []),
        "kh_profile": (I, [P, I, dp]),
        "kh_selftest_bytes": (S, [I, I, I]),
        "kh_selftest_gemm": (I, [I, I, I, I, P, P, P, P, S, P]),
        "kh_selftest_symeig": (I, [I, I, P, P, P, P, S, P]),
        "kh_selftest_svd": (I, [I, I, P, P, P, P, P, S, P]),
        "kh_selftest_orth": (I, [I, I, I, D, P, P, P, S, P]),
        "kh_selftest_svd_refined": (I, [I, P, P, P, P, P, S, P]),
        "kh_selftest_fp64_newton": (I, [I, P, P, P]),
        "kh_selftest_site_layered_bytes": (S, [I, I, I, ctypes.c_longlong]),
        "kh_selftest_site_layered": (I, [I, I, I, I, I, ctypes.c_longlong, P, P, P, P, S, P]),
        "kh_gemm_noalloc": (I, [I, I, I, I, P, P, P, P]),
        "kh_gemm_noalloc_max_bytes": (S, []),
        "kh_save": (I, [P, ctypes.c_char_p]),
        "kh_load_config": (I, [ctypes.c_char_p, cfgp]),
        "kh_load": (I, [ctypes.POINTER(P), ctypes.c_char_p, P, S, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        _LIB = load_library()
    return _LIB


def selftest_gemm(A, B, prec="fp64"):
    """C = A @ B (FP64 CUDA tensors) through the library's contraction GEMM."""
    import torch
    M, K = A.shape
    N = B.shape[1]
    C = torch.empty((M, N), dtype=torch.float64, device=A.device)
    nb = lib().kh_selftest_bytes(M, N, K)
    scr = torch.empty(nb + 256, dtype=torch.uint8, device=A.device)
    base = (scr.data_ptr() + 255) // 256 * 256
    st = lib().kh_selftest_gemm(PREC[prec], M, N, K, _tptr(A.contiguous()), _tptr(B.contiguous()), _tptr(C),
                                ctypes.c_void_p(base), nb, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != KH_OK:
        raise KhError(st, "kh_selftest_gemm")
    return C


def selftest_symeig(G, prec="fp64"):
    """(evals descending, eigenvectors as columns) of a symmetric FP64 CUDA tensor."""
    import torch
    k = G.shape[0]
    W = torch.empty((k, k), dtype=torch.float64, device=G.device)
    E = torch.empty(k, dtype=torch.float64, device=G.device)
    nb = lib().kh_selftest_bytes(k, k, k)
    scr = torch.empty(nb + 256, dtype=torch.uint8, device=G.device)
    base = (scr.data_ptr() + 255) // 256 * 256
    st = lib().kh_selftest_symeig(PREC[prec], k, _tptr(G.contiguous()), _tptr(W), _tptr(E), ctypes.c_void_p(base), nb,
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != KH_OK:
        raise KhError(st, "kh_selftest_symeig")
    return E, W


def selftest_svd(X, prec="fp64"):
    """(S descending, L, Q) with X Q = L S, by the library's one-sided Jacobi kernel."""
    import torch
    k = X.shape[0]
    S = torch.empty(k, dtype=torch.float64, device=X.device)
    L = torch.empty((k, k), dtype=torch.float64, device=X.device)
    Q = torch.empty((k, k), dtype=torch.float64, device=X.device)
    nb = lib().kh_selftest_bytes(k, k, k)
    scr = torch.empty(nb + 256, dtype=torch.uint8, device=X.device)
    base = (scr.data_ptr() + 255) // 256 * 256
    st = lib().kh_selftest_svd(PREC[prec], k, _tptr(X.contiguous()), _tptr(S), _tptr(L), _tptr(Q),
                               ctypes.c_void_p(base), nb, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != KH_OK:
        raise KhError(st, "kh_selftest_svd")
    return S, L, Q


def selftest_svd_refined(X):
    """(S, L, Q) with X Q = L S: FP32 one-sided Jacobi plus three FP64 Newton
    refinement steps (the FP64-projector option's small SVD)."""
    import torch
    k = X.shape[0]
    S = torch.empty(k, dtype=torch.float64, device=X.device)
    L = torch.empty((k, k), dtype=torch.float64, device=X.device)
    Q = torch.empty((k, k), dtype=torch.float64, device=X.device)
    nb = lib().kh_selftest_bytes(k, k, k)
    scr = torch.empty(nb + 256, dtype=torch.uint8, device=X.device)
    base = (scr.data_ptr() + 255) // 256 * 256
    st = lib().kh_selftest_svd_refined(k, _tptr(X.contiguous()), _tptr(S), _tptr(L), _tptr(Q),
                                       ctypes.c_void_p(base), nb, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != KH_OK:
        raise KhError(st, "kh_selftest_svd_refined")
    return S, L, Q


def selftest_site_layered(T, Y, kind=0, frame=0, npass=3):
    """Layered tensor-core site contraction of one (kind, frame):
    out[b][ok][ob] = sum_p sum_{ik,ib} TL[ik][p][ok] Y[b][ib][ik] TL[ib][p][ob]
    from the FP64 CUDA tensors T (p, D, D, D, D) and Y (nb, D^2, D^2)."""
    import torch
    p, D = T.shape[0], T.shape[1]
    nb = Y.shape[0]
    out = torch.empty((nb, D * D, D * D), dtype=torch.float64, device=Y.device)
    nbytes = lib().kh_selftest_site_layered_bytes(npass, D, p, nb)
    if nbytes == 0:
        raise KhError(KH_EINVAL, "kh_selftest_site_layered_bytes")
    scr = torch.empty(nbytes + 256, dtype=torch.uint8, device=Y.device)
    base = (scr.data_ptr() + 255) // 256 * 256
    st = lib().kh_selftest_site_layered(npass, D, p, kind, frame, nb, _tptr(T.contiguous()), _tptr(Y.contiguous()),
                                        _tptr(out), ctypes.c_void_p(base), nbytes,
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != KH_OK:
        raise KhError(st, "kh_selftest_site_layered")
    return out


def selftest_orth(Y, prec="fp64", cut=1e-12):
    """Orthonormal basis (n x k, dropped directions as zero columns) of the
    columns of the FP64 CUDA tensor Y by the library's ordered CholQR2."""
    import torch
    n, k = Y.shape
    Q = torch.empty((n, k), dtype=torch.float64, device=Y.device)
    nb = lib().kh_selftest_bytes(n, k, k)
    scr = torch.empty(nb + 256, dtype=torch.uint8, device=Y.device)
    base = (scr.data_ptr() + 255) // 256 * 256
    st = lib().kh_selftest_orth(PREC[prec], n, k, float(cut), _tptr(Y.contiguous()), _tptr(Q),
                                ctypes.c_void_p(base), nb, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != KH_OK:
        raise KhError(st, "kh_selftest_orth")
    return Q


def selftest_fp64_newton(x):
    """(1/x, 1/sqrt(x), sqrt(x)) of an FP64 CUDA tensor as the library's FP64
    kernels form them (Newton-Raphson from FP32 estimates)."""
    import torch
    n = x.numel()
    out = torch.empty(3 * n, dtype=torch.float64, device=x.device)
    st = lib().kh_selftest_fp64_newton(n, _tptr(x.contiguous()), _tptr(out),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != KH_OK:
        raise KhError(st, "kh_selftest_fp64_newton")
    o = out.view(n, 3)
    return o[:, 0], o[:, 1], o[:, 2]


def gemm_noalloc(A, B, prec="fp64"):
    """C = A @ B (FP64 CUDA tensors) through kh_gemm_noalloc: no device memory
    is allocated by the library; it uses its static scratch array."""
    import torch
    M, K = A.shape
    N = B.shape[1]
    C = torch.empty((M, N), dtype=torch.float64, device=A.device)
    st = lib().kh_gemm_noalloc(PREC[prec], M, N, K, _tptr(A.contiguous()), _tptr(B.contiguous()), _tptr(C),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != KH_OK:
        raise KhError(st, "kh_gemm_noalloc")
    return C


def launch_count():
    return int(lib().kh_launch_count())


def default_config(D, chi, prec="fp64", **kw):
    c = KhConfig()
    lib().kh_config_defaults(ctypes.byref(c))
    c.D, c.chi, c.prec = D, chi, PREC[prec] if isinstance(prec, str) else int(prec)
    if c.prec != PREC["fp64"]:
        # single-precision paths: the Rayleigh-Ritz SVD is capped (its residual
        # is below the FP32-level accuracy of the contractions well before);
        # singular values below 1e-4 s_1 are dropped (the single-precision
        # subspace iteration does not resolve the spectrum below ~2e-5 s_1),
        # and two subspace iterations per move keep the warm subspace on the
        # moving spectrum (one leaves sweep-to-sweep changes ~1e-5 of s_1)
        c.jacobi_max_sweeps = 8
        c.svd_cut = 1e-4
        c.svd_iters_warm = 2
        if c.prec == PREC["bf16"]:
            # BF16 contractions (8-bit mantissas) leave the projector spectrum
            # noisy at ~1e-3 s_1
            c.svd_cut = 1e-3
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def bond_hamiltonian(gamma, J, K_gamma, hA=0.0, hB=0.0):
    """4x4 H^gamma built by the library (host FP64)."""
    H = np.zeros(16)
    h, hp = _dptr(H)
    st = lib().kh_bond_hamiltonian(GAMMA.get(gamma, gamma), J, K_gamma, hA, hB, hp)
    if st != KH_OK:
        raise KhError(st, "kh_bond_hamiltonian")
    return h.reshape(4, 4)


def gate(H, tau):
    """exp(-tau H) built by the library (host FP64)."""
    Hc, hp = _dptr(np.asarray(H).reshape(16))
    g = np.zeros(16)
    gg, gp = _dptr(g)
    st = lib().kh_gate(hp, tau, gp)
    if st != KH_OK:
        raise KhError(st, "kh_gate")
    return gg.reshape(4, 4)


def _dptr(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _tptr(t):
    """Device pointer of a contiguous float64 CUDA tensor."""
    import torch
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """One eeFU context: owns a device workspace (torch uint8 tensor) and a
    stream; wraps every ABI call of include/eefu.h."""

    def __init__(self, D, chi, prec="fp64", device="cuda:0", stream=None, **cfg_kw):
        import torch
        self.torch = torch
        self.cfg = default_config(D, chi, prec, **cfg_kw)
        self.D, self.chi = D, chi
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        aligned, nbytes = self._workspace()
        self._ctx = ctypes.c_void_p()
        st = lib().kh_create(ctypes.byref(self._ctx), ctypes.byref(self.cfg), ctypes.c_void_p(aligned),
                             nbytes, ctypes.c_void_p(self.stream.cuda_stream))
        if st != KH_OK:
            raise KhError(st, "kh_create failed")

    def _workspace(self):
        """Allocate the caller-owned device workspace for self.cfg (256-byte
        aligned); returns its aligned address and size."""
        nbytes = lib().kh_workspace_bytes(ctypes.byref(self.cfg))
        if nbytes == 0:
            raise KhError(KH_EINVAL, "invalid configuration")
        self.workspace = self.torch.empty(nbytes + 256, dtype=self.torch.uint8, device=self.device)
        return (self.workspace.data_ptr() + 255) // 256 * 256, nbytes

    @classmethod
    def load(cls, path, device="cuda:0", stream=None):
        """A context restored from a checkpoint written by save(): same
        configuration, state, environments and warm subspaces."""
        import torch
        cfg = KhConfig()
        st = lib().kh_load_config(os.fsencode(path), ctypes.byref(cfg))
        if st != KH_OK:
            raise KhError(st, "not a readable checkpoint: %s" % path)
        self = cls.__new__(cls)
        self.torch = torch
        self.cfg = cfg
        self.D, self.chi = cfg.D, cfg.chi
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        aligned, nbytes = self._workspace()
        self._ctx = ctypes.c_void_p()
        st = lib().kh_load(ctypes.byref(self._ctx), os.fsencode(path), ctypes.c_void_p(aligned), nbytes,
                           ctypes.c_void_p(self.stream.cuda_stream))
        if st != KH_OK:
            msg = lib().kh_last_error(self._ctx).decode() if self._ctx.value else "kh_load failed"
            self.close()
            raise KhError(st, msg)
        return self

    def save(self, path):
        """Write the context's persistent state to a checkpoint file."""
        self._check(lib().kh_save(self._ctx, os.fsencode(path)))

    def _check(self, st):
        if st != KH_OK:
            raise KhError(st, lib().kh_last_error(self._ctx).decode())

    def close(self):
        if getattr(self, "_ctx", None) and self._ctx.value:
            lib().kh_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- instrumentation
    def profile_start(self):
        self._check(lib().kh_profile(self._ctx, 1, None))

    def profile_stop(self):
        out = np.zeros(3 * len(PROFILE_NAMES))
        o, op = _dptr(out)
        self._check(lib().kh_profile(self._ctx, 0, op))
        return {nm: dict(launches=int(o[3 * k]), ms=o[3 * k + 1], flops=o[3 * k + 2])
                for k, nm in enumerate(PROFILE_NAMES)}

    # ---- state
    def set_state(self, A, B):
        self._check(lib().kh_set_state(self._ctx, _tptr(A), _tptr(B)))

    def get_state(self):
        t = self.torch
        A = t.empty((2, 2, self.D, self.D, self.D), dtype=t.float64, device=self.device)
        B = t.empty_like(A)
        self._check(lib().kh_get_state(self._ctx, _tptr(A), _tptr(B)))
        return A, B

    # ---- CTMRG
    def ctm_set_tensor(self, slot, T):
        self._check(lib().ctm_set_tensor(self._ctx, slot, _tptr(T), int(T.shape[0])))

    def ctm_build_composite(self, slot, gamma, gate=None):
        if gate is None:
            self._check(lib().ctm_build_composite(self._ctx, slot, GAMMA.get(gamma, gamma), None))
        else:
            g, gp = _dptr(gate)
            self._check(lib().ctm_build_composite(self._ctx, slot, GAMMA.get(gamma, gamma), gp))

    def ctm_init(self, slot, edge=None):
        if edge is None:
            self._check(lib().ctm_init(self._ctx, slot, None))
        else:
            e, ep = _dptr(edge)
            self._check(lib().ctm_init(self._ctx, slot, ep))

    def ctm_copy_env(self, dst, src):
        self._check(lib().ctm_copy_env(self._ctx, dst, src))

    def ctm_sweep(self, slot, max_sweeps, min_sweeps=1, tol=-1.0, allow_noconv=False):
        done = ctypes.c_int(0)
        delta = ctypes.c_double(0.0)
        st = lib().ctm_sweep(self._ctx, slot, max_sweeps, min_sweeps, tol, ctypes.byref(done), ctypes.byref(delta))
        if not (allow_noconv and st == KH_ENOCONV):
            self._check(st)
        return done.value, delta.value

    def ctm_projectors(self, slot, direction):
        t = self.torch
        spec = t.empty(self.chi, dtype=t.float64, device=self.device)
        tr = ctypes.c_double(0.0)
        self._check(lib().ctm_projectors(self._ctx, slot, direction, _tptr(spec), ctypes.byref(tr)))
        return spec, tr.value

    def ctm_get_env(self, slot):
        t = self.torch
        C = t.empty((4, self.chi, self.chi), dtype=t.float64, device=self.device)
        E = t.empty((4, self.chi, self.D, self.D, self.chi), dtype=t.float64, device=self.device)
        self._check(lib().ctm_get_env(self._ctx, slot, _tptr(C), _tptr(E)))
        return C, E

    def ctm_metric(self, slot):
        t = self.torch
        n = self.D ** 4
        N = t.empty((n, n), dtype=t.float64, device=self.device)
        self._check(lib().ctm_metric(self._ctx, slot, _tptr(N)))
        return N

    def ctm_kappa(self, slot):
        k = ctypes.c_double(0.0)
        self._check(lib().ctm_kappa(self._ctx, slot, ctypes.byref(k)))
        return k.value

    def ctm_expval(self, slot, ops):
        ops = np.ascontiguousarray(ops, dtype=np.float64)
        if ops.ndim == 2:
            ops = ops[None]
        o, op = _dptr(ops)
        vals = np.zeros(ops.shape[0])
        v, vp = _dptr(vals)
        self._check(lib().ctm_expval(self._ctx, slot, op, ops.shape[0], vp))
        return v

    # ---- eeFU
    def ctm_correlation_length(self, slot, direction=0, max_iter=400, tol=1e-6):
        """(xi, |l2|/|l1|, iterations) of slot's channel transfer matrix."""
        out = np.zeros(3)
        o, op = _dptr(out)
        self._check(lib().ctm_correlation_length(self._ctx, slot, direction, max_iter, tol, op))
        return float(o[0]), float(o[1]), int(o[2])

    def ctm_plaquette(self, slot, ops):
        """(<O_ul O_ur O_dr O_dl>, plain cluster) for four p x p operators on
        a 2 x 2 plaquette of slot's lattice (upper-left first, clockwise)."""
        ops = np.ascontiguousarray(ops, dtype=np.float64)
        o, op = _dptr(ops)
        out = np.zeros(2)
        r, rp = _dptr(out)
        self._check(lib().ctm_plaquette(self._ctx, slot, op, rp))
        return float(r[0]), float(r[1])

    def flux(self, gamma, slot=None):
        """<W_p> from the gamma composite's environment; slot defaults to the
        observables' slot of that mapping (3 + gamma)."""
        g = GAMMA.get(gamma, gamma)
        out = np.zeros(2)
        r, rp = _dptr(out)
        self._check(lib().ctm_flux(self._ctx, 3 + g if slot is None else slot, g, rp))
        return float(r[0])

    def eefu_apply_gate(self, gamma, gate, ctm_max_sweeps=100, ctm_min_sweeps=1, ctm_tol=1e-12, info=True):
        g, gp = _dptr(gate)
        if info:
            out = np.zeros(4)
            o, op = _dptr(out)
            self._check(lib().eefu_apply_gate(self._ctx, GAMMA.get(gamma, gamma), gp, ctm_max_sweeps,
                                              ctm_min_sweeps, ctm_tol, op))
            return dict(rel_cost=o[0], ctm_sweeps=int(o[1]), als_iters=int(o[2]), trunc=o[3])
        self._check(lib().eefu_apply_gate(self._ctx, GAMMA.get(gamma, gamma), gp, ctm_max_sweeps, ctm_min_sweeps,
                                          ctm_tol, None))
        return None

    def cost_gradient(self, gamma, gate, A2, B2, ctm_max_sweeps=100, ctm_min_sweeps=1, ctm_tol=1e-12):
        """(gA, gB, d, <T'|N|T'>) of the bond cost d = <T''-T'|N|T''-T'> for the
        gamma-bond update of the current state with the 4 x 4 gate, at the
        trial factors A2 [sA][aA][u][r][k], B2 [sB][aB][d][l][k] (float64 CUDA
        tensors); ctm_max_sweeps = 0 reuses the slot's environment."""
        torch = self.torch
        A2 = A2.contiguous()
        B2 = B2.contiguous()
        gA = torch.empty_like(A2)
        gB = torch.empty_like(B2)
        g, gp = _dptr(np.asarray(gate, dtype=np.float64).reshape(16))
        out = np.zeros(3)
        o, op = _dptr(out)
        self._check(lib().eefu_cost_gradient(self._ctx, GAMMA.get(gamma, gamma), gp, _tptr(A2), _tptr(B2),
                                             ctm_max_sweeps, ctm_min_sweeps, ctm_tol, _tptr(gA), _tptr(gB), op))
        return gA, gB, float(o[0]), float(o[1])

    def eefu_trotter_step(self, J, K_xyz, dbeta, hA=0.0, hB=0.0, ctm_max_sweeps=100, ctm_min_sweeps=1,
                          ctm_tol=1e-12, info=True):
        k, kp = _dptr(np.asarray(K_xyz, dtype=np.float64))
        if info:
            out = np.zeros(4)
            o, op = _dptr(out)
            self._check(lib().eefu_trotter_step(self._ctx, J, kp, hA, hB, dbeta, ctm_max_sweeps, ctm_min_sweeps,
                                                ctm_tol, op))
            return dict(rel_cost=o[0], ctm_sweeps=int(o[1]), als_iters=int(o[2]), trunc=o[3])
        self._check(lib().eefu_trotter_step(self._ctx, J, kp, hA, hB, dbeta, ctm_max_sweeps, ctm_min_sweeps,
                                            ctm_tol, None))
        return None

    TRAJ_KEYS = ["beta", "E_site", "Hx", "Hy", "Hz", "Ax", "Ay", "Az", "Bx", "By", "Bz", "trunc", "C"]

    def evolve(self, J, K_xyz, dbeta, n_steps, measure_every=1, hA=0.0, hB=0.0, ctm_max_sweeps=100,
               ctm_min_sweeps=1, ctm_tol=1e-12, obs_max_sweeps=None, obs_min_sweeps=None, obs_tol=None,
               flux=False):
        """Imaginary-time trajectory: list of dicts (TRAJ_KEYS) per measurement,
        C the specific heat per site (NaN at the ends of the grid); with
        flux=True each row also carries W, the plaquette flux (eefu_evolve_flux)."""
        nm = n_steps // measure_every
        out = np.zeros(max(nm, 1) * len(self.TRAJ_KEYS))
        o, op = _dptr(out)
        K, kp = _dptr(np.asarray(K_xyz, dtype=np.float64))
        args = (self._ctx, J, kp, hA, hB, dbeta, n_steps, measure_every, ctm_max_sweeps, ctm_min_sweeps, ctm_tol,
                obs_max_sweeps or ctm_max_sweeps, obs_min_sweeps or ctm_min_sweeps,
                ctm_tol if obs_tol is None else obs_tol, op)
        if flux:
            w = np.zeros(max(nm, 1))
            w, wp = _dptr(w)
            st = lib().eefu_evolve_flux(*args, wp)
        else:
            st = lib().eefu_evolve(*args)
        self._check(st)
        rows = o.reshape(-1, len(self.TRAJ_KEYS))[:nm]
        res = [dict(zip(self.TRAJ_KEYS, r.tolist())) for r in rows]
        if flux:
            for r, x in zip(res, w[:nm].tolist()):
                r["W"] = x
        return res

    def observables(self, H_xyz, hA=0.0, hB=0.0, ctm_max_sweeps=100, ctm_min_sweeps=1, ctm_tol=1e-12):
        H = np.ascontiguousarray(np.stack([np.asarray(h, dtype=np.float64) for h in H_xyz]))
        h, hp = _dptr(H)
        out = np.zeros(12)
        o, op = _dptr(out)
        self._check(lib().observables(self._ctx, hp, hA, hB, ctm_max_sweeps, ctm_min_sweeps, ctm_tol, op))
        keys = ["E_site", "Hx", "Hy", "Hz", "Ax", "Ay", "Az", "Bx", "By", "Bz", "trunc", "sweeps"]
        return dict(zip(keys, o.tolist()))


def evolve_batch(contexts, J, K_xyz, dbeta, n_steps, measure_every=1, hA=None, hB=None, ctm_max_sweeps=100,
                 ctm_min_sweeps=1, ctm_tol=1e-12, obs_max_sweeps=None, obs_min_sweeps=None, obs_tol=None):
    """Trajectories of several independent problems advanced concurrently
    (eefu_evolve_batch): contexts[i] with couplings J[i], K_xyz[i] (3 values),
    hA[i], hB[i].  Returns one list of TRAJ_KEYS dicts per problem; raises
    KhError with the first failing problem's message."""
    n = len(contexts)
    keys = Context.TRAJ_KEYS
    nm = n_steps // measure_every
    out = np.zeros(n * max(nm, 1) * len(keys))
    o, op = _dptr(out)
    Jv, jp = _dptr(np.asarray(J, dtype=np.float64).reshape(n))
    Kv, kp = _dptr(np.asarray(K_xyz, dtype=np.float64).reshape(n * 3))
    ha, hap = _dptr(np.zeros(n) if hA is None else np.asarray(hA, dtype=np.float64).reshape(n))
    hb, hbp = _dptr(np.zeros(n) if hB is None else np.asarray(hB, dtype=np.float64).reshape(n))
    arr = (ctypes.c_void_p * n)(*[c._ctx.value for c in contexts])
    stat = (ctypes.c_int * n)()
    st = lib().eefu_evolve_batch(ctypes.cast(arr, ctypes.POINTER(ctypes.c_void_p)), n, jp, kp, hap, hbp, dbeta,
                                 n_steps, measure_every, ctm_max_sweeps, ctm_min_sweeps, ctm_tol,
                                 obs_max_sweeps or ctm_max_sweeps, obs_min_sweeps or ctm_min_sweeps,
                                 ctm_tol if obs_tol is None else obs_tol, op, stat)
    if st != KH_OK:
        bad = [i for i in range(n) if stat[i] != KH_OK]
        if not bad:
            raise KhError(st, "eefu_evolve_batch: invalid arguments")
        raise KhError(st, "problem %d: %s" % (bad[0], lib().kh_last_error(contexts[bad[0]]._ctx).decode()))
    rows = o.reshape(n, max(nm, 1), len(keys))[:, :nm]
    return [[dict(zip(keys, r.tolist())) for r in prob] for prob in rows]


_BOND_COST = None


def bond_cost(ctx, gamma, gate, A2, B2, ctm_max_sweeps=0, ctm_min_sweeps=1, ctm_tol=1e-12):
    """The bond cost d(A'', B'') = <T''-T'|N|T''-T'> of ctx's current state
    and gate as a differentiable torch scalar: the forward and backward passes
    are one eefu_cost_gradient call (the hand-written adjoint); by default
    the slot's environment is reused (ctm_max_sweeps = 0), so N is fixed."""
    global _BOND_COST
    import torch
    if _BOND_COST is None:
        class BondCost(torch.autograd.Function):
            @staticmethod
            def forward(fctx, a2, b2, c, gm, gt, mx, mn, tol):
                gA, gB, d, _ = c.cost_gradient(gm, gt, a2.detach(), b2.detach(), mx, mn, tol)
                fctx.save_for_backward(gA, gB)
                return torch.tensor(d, dtype=torch.float64, device=a2.device)

            @staticmethod
            def backward(fctx, go):
                gA, gB = fctx.saved_tensors
                return go * gA, go * gB, None, None, None, None, None, None
        _BOND_COST = BondCost
    return _BOND_COST.apply(A2, B2, ctx, gamma, gate, ctm_max_sweeps, ctm_min_sweeps, ctm_tol)
