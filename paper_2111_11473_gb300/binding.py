"""ctypes binding of the C ABI in include/thc.h (marshalling only)."""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libthc.so")

THC_PREC_FP64 = 0
THC_PREC_MIXED = 1
THC_PREC_FP64_TC = 2

STATUS = {0: "THC_OK", 1: "THC_ERR_ARG", 2: "THC_ERR_CUDA", 3: "THC_ERR_OOM",
          4: "THC_ERR_NUMERIC", 5: "THC_ERR_NOT_CONVERGED", 6: "THC_ERR_TIMEOUT",
          7: "THC_ERR_UNSUPPORTED"}


class ThcConfig(C.Structure):
    _fields_ = [("n_occ", C.c_int), ("n_vir", C.c_int), ("n_p", C.c_int),
                ("n_g", C.c_int), ("n_k", C.c_int), ("precision", C.c_int),
                ("k_slab", C.c_int), ("i_chunk", C.c_int), ("x_block", C.c_int),
                ("workspace_bytes", C.c_size_t), ("lsq_rel_cutoff", C.c_double),
                ("tc_products", C.c_int), ("alg7_route", C.c_int), ("t2sq_route", C.c_int),
                ("x_block6", C.c_int), ("policy", C.c_int * 10), ("shard_index", C.c_int),
                ("shard_count", C.c_int)]


# Steps of a residual (THC_STEP_*) and per-step arithmetic (THC_POL_*).
STEPS = ["dress", "fock", "alg1", "alg2_8", "post", "alg6_gemm", "triangle", "alg6_post",
         "alg7", "energy"]
POLICIES = {"default": 0, "fp64": 1, "fp64tc": 2, "bf16x3": 3, "bf16": 4, "fp32": 5}


class ThcSolveOpts(C.Structure):
    _fields_ = [("r_tol", C.c_double), ("e_tol", C.c_double), ("max_iter", C.c_int),
                ("diis_n", C.c_int), ("use_mlp", C.c_int), ("verbose", C.c_int),
                ("history", C.c_void_p), ("mlp", C.c_void_p), ("record_pairs", C.c_int),
                ("record_seed", C.c_ulonglong), ("resume", C.c_int), ("mlp_accept", C.c_int),
                ("mlp_blocks", C.c_int)]


class ThcReport(C.Structure):
    _fields_ = [("iters", C.c_int), ("mlp_accepted", C.c_int), ("mlp_rejected", C.c_int),
                ("energy", C.c_double), ("r_norm", C.c_double), ("wall_s", C.c_double)]


N_STEPS = 10


class ThcProfile(C.Structure):
    _fields_ = [("ms", C.c_double * N_STEPS), ("flops", C.c_double * N_STEPS),
                ("launches", C.c_longlong * N_STEPS), ("residuals", C.c_longlong),
                ("kernel_launches", C.c_longlong)]


@dataclass
class Report:
    status: str
    iters: int
    energy: float
    r_norm: float
    wall_s: float
    mlp_accepted: int
    mlp_rejected: int


class ThcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status
        self.name = STATUS.get(status, str(status))


_LIB = None
_VP = C.c_void_p
_DP = C.c_void_p   # double* (host or device); passed as raw addresses

_SIGNATURES = {
    "thc_config_default": (C.c_int, [C.POINTER(ThcConfig), C.c_int, C.c_int, C.c_int,
                                     C.c_int, C.c_int]),
    "thc_solve_opts_default": (C.c_int, [C.POINTER(ThcSolveOpts)]),
    "thc_init": (C.c_int, [C.POINTER(ThcConfig), _DP, _DP, _DP, _DP, _DP, _DP, _VP,
                           C.POINTER(_VP)]),
    "thc_load_cholesky": (C.c_int, [_VP, C.c_int, C.c_int, _DP]),
    "thc_init_finish": (C.c_int, [_VP]),
    "thc_residual": (C.c_int, [_VP, _DP, _DP, _DP, _DP, _DP]),
    "thc_energy": (C.c_int, [_VP, _DP, _DP, _DP]),
    "thc_mp2_density": (C.c_int, [_VP, _DP, _DP, _DP]),
    "thc_solve": (C.c_int, [_VP, C.POINTER(ThcSolveOpts), _DP, _DP, C.POINTER(ThcReport)]),
    "thc_solve_state_size": (C.c_int, [_VP, C.POINTER(C.c_size_t)]),
    "thc_solve_state_save": (C.c_int, [_VP, _VP, C.c_size_t]),
    "thc_solve_state_load": (C.c_int, [_VP, _VP, C.c_size_t]),
    "thc_profile_enable": (C.c_int, [_VP, C.c_int]),
    "thc_profile_read": (C.c_int, [_VP, C.POINTER(ThcProfile)]),
    "thc_step_name": (C.c_char_p, [C.c_int]),
    "thc_energy_noalloc": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, _DP, _DP, _DP,
                                     _DP, _DP, _VP]),
    "thc_solve_pairs": (C.c_int, [_VP, _DP, _DP, _DP, C.c_longlong,
                                  C.POINTER(C.c_longlong)]),
    "thc_mlp_create": (C.c_int, [C.c_int, C.c_ulonglong, C.c_int, _VP, C.POINTER(_VP)]),
    "thc_mlp_num_params": (C.c_int, [_VP, C.POINTER(C.c_longlong)]),
    "thc_mlp_get_params": (C.c_int, [_VP, _DP]),
    "thc_mlp_set_params": (C.c_int, [_VP, _DP]),
    "thc_mlp_predict": (C.c_int, [_VP, _DP, C.c_longlong, _DP]),
    "thc_mlp_loss_grad": (C.c_int, [_VP, _DP, _DP, _DP, C.c_longlong, C.POINTER(C.c_double),
                                    _DP]),
    "thc_mlp_train": (C.c_int, [_VP, _DP, _DP, _DP, C.c_longlong, C.c_int, C.c_int, C.c_double,
                                C.c_ulonglong, C.POINTER(C.c_double)]),
    "thc_mlp_destroy": (None, [_VP]),
    "thc_selftest_bounded_wait": (C.c_int, [C.c_int, _VP]),
    "thc_selftest_gemm_f64": (C.c_int, [C.c_int, C.c_ulonglong, C.POINTER(C.c_double),
                                        C.POINTER(C.c_int), _VP]),
    "thc_selftest_gemm": (C.c_int, [C.c_int, C.c_ulonglong, C.POINTER(C.c_double),
                                    C.POINTER(C.c_int), _VP]),
    "thc_cp_als": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, _DP, _DP, _DP, _DP, _DP,
                             C.c_int, _DP, _VP]),
    "thc_probe_alu": (C.c_int, [C.c_int, C.POINTER(C.c_double), _VP]),
    "thc_probe_gemm": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                 C.POINTER(C.c_double), _VP]),
    "thc_last_error": (C.c_char_p, [_VP]),
    "thc_destroy": (None, [_VP]),
}


def load_library(path: str = LIB_PATH):
    """Load libthc.so and declare the C ABI.  Raises if it is not built."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def exported_symbols():
    return sorted(_SIGNATURES)


def cp_als(U, eps, y_o, y_v, tau, iters, stream=None):
    """Weighted CP-ALS of the projectors (thc_cp_als).  U: (o*v) x N, eps: N,
    start factors y_o (o x W), y_v (v x W), tau (N x W); returns the updated
    factors (new numpy arrays) and the objective after every sweep."""
    lib = load_library()
    U = np.ascontiguousarray(U, dtype=np.float64)
    eps = np.ascontiguousarray(eps, dtype=np.float64)
    yo = np.array(y_o, dtype=np.float64, order="C", copy=True)
    yv = np.array(y_v, dtype=np.float64, order="C", copy=True)
    t = np.array(tau, dtype=np.float64, order="C", copy=True)
    o, W = yo.shape
    v, N = yv.shape[0], t.shape[0]
    if U.shape != (o * v, N) or eps.shape != (N,) or yv.shape[1] != W or t.shape[1] != W:
        raise ValueError("inconsistent CP-ALS shapes")
    hist = np.zeros(max(1, iters))
    st = 0 if stream is None else int(getattr(stream, "cuda_stream", stream))
    status = lib.thc_cp_als(o, v, N, W, U.ctypes.data, eps.ctypes.data, yo.ctypes.data,
                            yv.ctypes.data, t.ctypes.data, int(iters), hist.ctypes.data, _VP(st))
    if status != 0:
        raise ThcError(status, lib.thc_last_error(None).decode())
    return yo, yv, t, list(hist[:iters])


def selftest_gemm(cases=64, seed=0, stream=None):
    """Randomised tensor-core vs CUDA-core product check; returns
    (status name, max bf16x3 relative difference, failures)."""
    lib = load_library()
    st = 0 if stream is None else int(getattr(stream, "cuda_stream", stream))
    mr = C.c_double(0)
    nf = C.c_int(0)
    status = lib.thc_selftest_gemm(int(cases), int(seed), C.byref(mr), C.byref(nf), _VP(st))
    return STATUS.get(status, "?"), mr.value, nf.value


def selftest_gemm_f64(cases=64, seed=0, stream=None):
    """Randomised float64 tensor-core (integer-slice) vs CUDA-core product
    check; returns (status name, max relative difference, failures)."""
    lib = load_library()
    st = 0 if stream is None else int(getattr(stream, "cuda_stream", stream))
    mr = C.c_double(0)
    nf = C.c_int(0)
    status = lib.thc_selftest_gemm_f64(int(cases), int(seed), C.byref(mr), C.byref(nf), _VP(st))
    return STATUS.get(status, "?"), mr.value, nf.value


def probe_alu(kind: int, stream=None) -> float:
    """Measured FMA throughput in TFLOP/s: kind 0 float64, 1 float32,
    2 packed float32 pairs (thc_probe_alu)."""
    lib = load_library()
    st = 0 if stream is None else int(getattr(stream, "cuda_stream", stream))
    v = C.c_double(0)
    status = lib.thc_probe_alu(int(kind), C.byref(v), _VP(st))
    if status != 0:
        raise ThcError(status, lib.thc_last_error(None).decode())
    return v.value


def probe_gemm(mode: int, M: int, N: int, K: int, iters: int = 10, stream=None) -> float:
    """Milliseconds per tensor-core product (thc_probe_gemm): mode 0 bf16x3
    with cached packs, 1 bf16x3 with the pack, 2 bf16x1, 3 float64 slices."""
    lib = load_library()
    st = 0 if stream is None else int(getattr(stream, "cuda_stream", stream))
    v = C.c_double(0)
    status = lib.thc_probe_gemm(int(mode), int(M), int(N), int(K), int(iters), C.byref(v),
                                _VP(st))
    if status != 0:
        raise ThcError(status, lib.thc_last_error(None).decode())
    return v.value


def selftest_bounded_wait(complete: bool, stream=None) -> str:
    """Run the library's bounded-wait self-test; returns the status name
    (THC_OK if the wait completed, THC_ERR_TIMEOUT if it expired)."""
    lib = load_library()
    st = 0 if stream is None else int(getattr(stream, "cuda_stream", stream))
    return STATUS.get(lib.thc_selftest_bounded_wait(int(bool(complete)), _VP(st)), "?")


def _is_torch(a):
    return hasattr(a, "data_ptr") and hasattr(a, "is_cuda")


class _Arg:
    """A float64 C-contiguous buffer and its address (numpy or torch)."""

    def __init__(self, a, shape, writable=False):
        if _is_torch(a):
            import torch
            if a.dtype != torch.float64:
                raise TypeError("expected a float64 tensor")
            if tuple(a.shape) != tuple(shape):
                raise ValueError(f"expected shape {shape}, got {tuple(a.shape)}")
            if not a.is_contiguous():
                if writable:
                    raise ValueError("output tensor must be contiguous")
                a = a.contiguous()
            self.obj = a
            self.ptr = a.data_ptr()
        else:
            arr = np.asarray(a)
            if arr.shape != tuple(shape):
                raise ValueError(f"expected shape {shape}, got {arr.shape}")
            if writable:
                if arr.dtype != np.float64 or not arr.flags.c_contiguous:
                    raise ValueError("output array must be C-contiguous float64")
            else:
                arr = np.ascontiguousarray(arr, dtype=np.float64)
            self.obj = arr
            self.ptr = arr.ctypes.data


class Context:
    """One THC-RR-CCSD system resident on the GPU (wraps thc_ctx*)."""

    def __init__(self, eps_o, eps_v, Y, L, x, z, precision=THC_PREC_FP64, stream=None,
                 k_slab=0, i_chunk=0, x_block=0, workspace_bytes=0, lsq_rel_cutoff=1e-10,
                 tc_products=3, alg7_route=0, t2sq_route=0, x_block6=0, n_k=None,
                 policy=None, shard=None):
        """L = None (with n_k = K) leaves the Cholesky vectors to
        load_cholesky() and finish_init().  policy: {step name: policy name}
        (STEPS, POLICIES), the per-step arithmetic of thc_config.policy.
        shard: (index, count) makes a context that evaluates one shard of the
        residual (thc_config.shard_index / shard_count)."""
        lib = load_library()
        o, v = len(eps_o), len(eps_v)
        n = o + v
        P = Y.shape[1]
        G = x.shape[1]
        if L is None and n_k is None:
            raise ValueError("n_k is required when L is None")
        K = L.shape[0] if L is not None else int(n_k)
        cfg = ThcConfig()
        st = lib.thc_config_default(C.byref(cfg), o, v, P, G, K)
        if st != 0:
            raise ThcError(st, "bad dimensions")
        cfg.precision = int(precision)
        cfg.k_slab, cfg.i_chunk, cfg.x_block = k_slab, i_chunk, x_block
        cfg.workspace_bytes = workspace_bytes
        cfg.lsq_rel_cutoff = lsq_rel_cutoff
        cfg.tc_products = tc_products
        cfg.alg7_route = alg7_route
        cfg.t2sq_route = t2sq_route
        cfg.x_block6 = x_block6
        for step, name in (policy or {}).items():
            cfg.policy[STEPS.index(step)] = POLICIES[name]
        if shard is not None:
            cfg.shard_index, cfg.shard_count = int(shard[0]), int(shard[1])
        args = [_Arg(eps_o, (o,)), _Arg(eps_v, (v,)), _Arg(Y, (n, P)),
                _Arg(L, (K, n, n)) if L is not None else None,
                _Arg(x, (n, G)), _Arg(z, (G, G))]
        handle = _VP()
        stream_ptr = 0 if stream is None else int(getattr(stream, "cuda_stream", stream))
        st = lib.thc_init(C.byref(cfg), *[a.ptr if a is not None else None for a in args],
                          _VP(stream_ptr), C.byref(handle))
        if st != 0:
            raise ThcError(st, lib.thc_last_error(None).decode())
        self._lib = lib
        self._h = handle
        self.o, self.v, self.P, self.G, self.K = o, v, P, G, K
        self.precision = precision

    def load_cholesky(self, k0, L):
        """Cholesky vectors k0 .. k0 + len(L) - 1 (float64, nk x n x n)."""
        n = self.o + self.v
        nk = L.shape[0]
        a = _Arg(L, (nk, n, n))
        self._check(self._lib.thc_load_cholesky(self._h, int(k0), int(nk), a.ptr))

    def finish_init(self):
        self._check(self._lib.thc_init_finish(self._h))

    def _check(self, st):
        if st != 0:
            raise ThcError(st, self._lib.thc_last_error(self._h).decode())

    def _out(self, like, shape):
        if _is_torch(like):
            import torch
            return torch.empty(shape, dtype=torch.float64, device=like.device)
        return np.empty(shape)

    def residual(self, Zc, t1, out=None, want_energy=True):
        """(sigma^WX, Omega_i^a, E) at (Zc, t1); outputs in the inputs' memory."""
        zc = _Arg(Zc, (self.P, self.P))
        tt = _Arg(t1, (self.o, self.v))
        if out is None:
            out = (self._out(Zc, (self.P, self.P)), self._out(Zc, (self.o, self.v)))
        s = _Arg(out[0], (self.P, self.P), writable=True)
        s1 = _Arg(out[1], (self.o, self.v), writable=True)
        e = C.c_double(0.0)
        eptr = C.addressof(e) if want_energy else None
        self._check(self._lib.thc_residual(self._h, zc.ptr, tt.ptr, s.ptr, s1.ptr, eptr))
        return out[0], out[1], (e.value if want_energy else None)

    def mp2_density(self, Zc, out=None):
        """(D_oo, D_vv) of the amplitudes encoded by Zc (App. II, Eqs. 47-56)."""
        zc = _Arg(Zc, (self.P, self.P))
        if out is None:
            out = (self._out(Zc, (self.o, self.o)), self._out(Zc, (self.v, self.v)))
        a = _Arg(out[0], (self.o, self.o), writable=True)
        b = _Arg(out[1], (self.v, self.v), writable=True)
        self._check(self._lib.thc_mp2_density(self._h, zc.ptr, a.ptr, b.ptr))
        return out[0], out[1]

    def energy(self, Zc, t1):
        zc = _Arg(Zc, (self.P, self.P))
        tt = _Arg(t1, (self.o, self.v))
        e = C.c_double(0.0)
        self._check(self._lib.thc_energy(self._h, zc.ptr, tt.ptr, C.addressof(e)))
        return e.value

    def solve(self, Zc=None, t1=None, r_tol=1e-8, e_tol=0.0, max_iter=100, diis_n=8,
              use_mlp=False, verbose=False, raise_on_failure=True, history=None, mlp=None,
              record_pairs=0, record_seed=0, resume=False, mlp_accept=0, mlp_blocks=3):
        """Run thc_solve; Zc and t1 (numpy, updated in place) start at zero.

        If ``history`` is a list, (energy, |r|, seconds) per iteration is
        appended to it.  ``resume`` continues the stopped solve of this
        context (or the state given to load_solve_state); Zc and t1 are then
        outputs only."""
        if Zc is None:
            Zc = np.zeros((self.P, self.P))
        if t1 is None:
            t1 = np.zeros((self.o, self.v))
        zc = _Arg(Zc, (self.P, self.P), writable=True)
        tt = _Arg(t1, (self.o, self.v), writable=True)
        opts = ThcSolveOpts()
        self._lib.thc_solve_opts_default(C.byref(opts))
        opts.r_tol, opts.e_tol, opts.max_iter = r_tol, e_tol, max_iter
        opts.diis_n, opts.use_mlp, opts.verbose = diis_n, int(use_mlp), int(verbose)
        hbuf = np.zeros((max(1, max_iter), 3))
        opts.history = hbuf.ctypes.data
        opts.mlp = mlp._h.value if mlp is not None else None
        opts.record_pairs, opts.record_seed = int(record_pairs), int(record_seed)
        opts.resume = int(bool(resume))
        opts.mlp_accept = int(mlp_accept)
        opts.mlp_blocks = int(mlp_blocks)
        rep = ThcReport()
        st = self._lib.thc_solve(self._h, C.byref(opts), zc.ptr, tt.ptr, C.byref(rep))
        if history is not None:
            history.extend(tuple(r) for r in hbuf[:rep.iters])
        report = Report(STATUS.get(st, str(st)), rep.iters, rep.energy, rep.r_norm, rep.wall_s,
                        rep.mlp_accepted, rep.mlp_rejected)
        if st != 0 and raise_on_failure:
            self._check(st)
        return Zc, t1, report

    def solve_state(self) -> bytes:
        """Checkpoint of the stopped solve (thc_solve_state_save)."""
        n = C.c_size_t(0)
        self._check(self._lib.thc_solve_state_size(self._h, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        self._check(self._lib.thc_solve_state_save(self._h, C.cast(buf, _VP), n))
        return buf.raw

    def load_solve_state(self, state: bytes):
        """Make a checkpoint of the same system resumable here."""
        buf = C.create_string_buffer(state, len(state))
        self._check(self._lib.thc_solve_state_load(self._h, C.cast(buf, _VP), len(state)))

    def solve_pairs(self):
        """Training pairs (X, j, t) recorded by the last solve, as numpy float32."""
        n = C.c_longlong(0)
        self._check(self._lib.thc_solve_pairs(self._h, None, None, None, 0, C.byref(n)))
        X = np.empty((n.value, 8), np.float32)
        j = np.empty(n.value, np.float32)
        t = np.empty(n.value, np.float32)
        if n.value:
            self._check(self._lib.thc_solve_pairs(self._h, X.ctypes.data, j.ctypes.data,
                                                  t.ctypes.data, n.value, C.byref(n)))
        return X, j, t

    def profile(self, on=True):
        """Switch per-step device timing on (clears counters) or off."""
        self._check(self._lib.thc_profile_enable(self._h, int(on)))

    def profile_read(self):
        """{step name: (ms, flops, launches)} accumulated since profile(True)."""
        p = ThcProfile()
        self._check(self._lib.thc_profile_read(self._h, C.byref(p)))
        out = {}
        for i in range(N_STEPS):
            out[self._lib.thc_step_name(i).decode()] = (p.ms[i], p.flops[i], p.launches[i])
        out["residuals"] = p.residuals
        out["kernel_launches"] = p.kernel_launches
        return out

    def close(self):
        if getattr(self, "_h", None):
            self._lib.thc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Mlp:
    """The learned preconditioner network (wraps thc_mlp*)."""

    def __init__(self, hidden=256, seed=0, bf16=True, stream=None):
        lib = load_library()
        h = _VP()
        stream_ptr = 0 if stream is None else int(getattr(stream, "cuda_stream", stream))
        st = lib.thc_mlp_create(hidden, seed, int(bf16), _VP(stream_ptr), C.byref(h))
        if st != 0:
            raise ThcError(st, lib.thc_last_error(None).decode())
        self._lib = lib
        self._h = h
        self.hidden = hidden
        n = C.c_longlong(0)
        lib.thc_mlp_num_params(h, C.byref(n))
        self.n_params = n.value

    def _check(self, st):
        if st != 0:
            raise ThcError(st, self._lib.thc_last_error(None).decode())

    def get_params(self):
        p = np.empty(self.n_params, np.float32)
        self._check(self._lib.thc_mlp_get_params(self._h, p.ctypes.data))
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        assert p.shape == (self.n_params,)
        self._check(self._lib.thc_mlp_set_params(self._h, p.ctypes.data))

    def predict(self, X):
        X = np.ascontiguousarray(X, np.float32)
        y = np.empty(X.shape[0], np.float32)
        self._check(self._lib.thc_mlp_predict(self._h, X.ctypes.data, X.shape[0], y.ctypes.data))
        return y

    def loss_grad(self, X, j, t):
        X = np.ascontiguousarray(X, np.float32)
        j = np.ascontiguousarray(j, np.float32)
        t = np.ascontiguousarray(t, np.float32)
        g = np.empty(self.n_params, np.float32)
        loss = C.c_double(0)
        self._check(self._lib.thc_mlp_loss_grad(self._h, X.ctypes.data, j.ctypes.data,
                                                t.ctypes.data, X.shape[0], C.byref(loss),
                                                g.ctypes.data))
        return loss.value, g

    def train(self, X, j, t, epochs=10, batch=4096, lr=1e-3, seed=0):
        X = np.ascontiguousarray(X, np.float32)
        j = np.ascontiguousarray(j, np.float32)
        t = np.ascontiguousarray(t, np.float32)
        loss = C.c_double(0)
        self._check(self._lib.thc_mlp_train(self._h, X.ctypes.data, j.ctypes.data, t.ctypes.data,
                                            X.shape[0], epochs, batch, lr, seed, C.byref(loss)))
        return loss.value

    def close(self):
        if getattr(self, "_h", None):
            self._lib.thc_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
