"""GB300 tensor-train SDP interior-point library: Python binding.

Every function here marshals arguments into the C ABI of include/tt_sdp.h;
all arithmetic runs in the CUDA library. Device tensors are torch CUDA
tensors (float64, contiguous); host TT cores are lists of numpy arrays.
Importing the package does not load the library; the first call does, and
fails loudly if it has not been built.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib

FP64, FP32, MIXED_TF32, MIXED_BF16 = 0, 1, 2, 3

__all__ = [
    "FP64", "FP32", "MIXED_TF32", "MIXED_BF16", "TTSDPError", "lib",
    "env_left_step", "env_right_step", "local_apply", "local_matrix",
    "hadamard", "matvec", "inner", "round_tt", "round_sdp", "tt_from_dense", "default_options", "Context", "Batch",
    "make_allocator",
    "launch_count", "contraction_stats", "contraction_stats_reset",
]


class TTSDPError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib_ = _lib.load()
        msg = lib_.tt_sdp_status_string(status).decode()
        detail = lib_.tt_last_error().decode()
        super().__init__(f"{where}: {msg} ({status}) {detail}")
        self.status = status


def lib() -> ctypes.CDLL:
    return _lib.load()


def _check(status: int, where: str):
    if status != 0:
        raise TTSDPError(status, where)


def _ptr(t) -> int:
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "device tensors must be contiguous CUDA tensors"
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _dims(d) -> _lib.ContractDims:
    if isinstance(d, dict):
        return _lib.ContractDims(d["rw"], d["rw2"], d["R"], d["R2"], d["rv"], d["rv2"], d["m"], d["n"])
    return _lib.ContractDims(*d)


# --- contraction kernels (rows a6, a7) ---------------------------------------

def env_left_step(dims, phi, u, op, v, out, precision=FP64, stream=None):
    dm = _dims(dims)
    _check(lib().tt_env_left_step(ctypes.byref(dm), _ptr(phi), _ptr(u), _ptr(op), _ptr(v), _ptr(out), precision,
                                  _stream(stream)), "tt_env_left_step")


def env_right_step(dims, psi, u, op, v, out, precision=FP64, stream=None):
    dm = _dims(dims)
    _check(lib().tt_env_right_step(ctypes.byref(dm), _ptr(psi), _ptr(u), _ptr(op), _ptr(v), _ptr(out), precision,
                                   _stream(stream)), "tt_env_right_step")


def local_apply(dims, phi, op, psi, x, y, precision=FP64, stream=None):
    dm = _dims(dims)
    _check(lib().tt_local_apply(ctypes.byref(dm), _ptr(phi), _ptr(op), _ptr(psi), _ptr(x), _ptr(y), precision,
                                _stream(stream)), "tt_local_apply")


def local_matrix(dims, phi, op, psi, out, precision=FP64, stream=None):
    dm = _dims(dims)
    _check(lib().tt_local_matrix(ctypes.byref(dm), _ptr(phi), _ptr(op), _ptr(psi), _ptr(out), precision,
                                 _stream(stream)), "tt_local_matrix")


# --- TT-level operations (rows a3, a8, a9) ------------------------------------

class DevTT:
    """A TT whose cores live in one flat float64 CUDA tensor."""

    def __init__(self, ranks, m, n, flat):
        self.ranks = [int(r) for r in ranks]
        self.m, self.n = int(m), int(n)
        self.flat = flat

    @property
    def d(self):
        return len(self.ranks) - 1

    @staticmethod
    def from_cores(cores, device="cuda"):
        import torch
        c0 = cores[0]
        m = c0.shape[1]
        n = c0.shape[2] if c0.ndim == 4 else 1
        ranks = [c.shape[0] for c in cores] + [cores[-1].shape[-1]]
        flat = np.concatenate([np.ascontiguousarray(c, dtype=np.float64).reshape(-1) for c in cores])
        return DevTT(ranks, m, n, torch.from_numpy(flat).to(device))

    def cores(self):
        flat = self.flat.detach().cpu().numpy()
        out, off = [], 0
        for k in range(self.d):
            shape = (self.ranks[k], self.m, self.n, self.ranks[k + 1]) if self.n > 1 else \
                (self.ranks[k], self.m, self.ranks[k + 1])
            size = int(np.prod(shape))
            out.append(flat[off:off + size].reshape(shape).copy())
            off += size
        return out

    def desc(self):
        self._r = (ctypes.c_int32 * len(self.ranks))(*self.ranks)
        return _lib.TTDesc(self.d, ctypes.cast(self._r, _lib.P_int32), self.m, self.n, _ptr(self.flat))


def _count(ranks, m, n):
    return sum(ranks[k] * m * n * ranks[k + 1] for k in range(len(ranks) - 1))


def hadamard(a: DevTT, b: DevTT, stream=None) -> DevTT:
    import torch
    ranks = [x * y for x, y in zip(a.ranks, b.ranks)]
    out = torch.empty(_count(ranks, a.m, a.n), dtype=torch.float64, device=a.flat.device)
    da, db = a.desc(), b.desc()
    _check(lib().tt_hadamard(ctypes.byref(da), ctypes.byref(db), _ptr(out), _stream(stream)), "tt_hadamard")
    return DevTT(ranks, a.m, a.n, out)


def matvec(op: DevTT, v: DevTT, stream=None) -> DevTT:
    import torch
    ranks = [x * y for x, y in zip(op.ranks, v.ranks)]
    out = torch.empty(_count(ranks, op.m, 1), dtype=torch.float64, device=op.flat.device)
    da, db = op.desc(), v.desc()
    _check(lib().tt_matvec(ctypes.byref(da), ctypes.byref(db), _ptr(out), _stream(stream)), "tt_matvec")
    return DevTT(ranks, op.m, 1, out)


def inner(a: DevTT, b: DevTT, stream=None) -> float:
    res = ctypes.c_double(0.0)
    da, db = a.desc(), b.desc()
    _check(lib().tt_inner(ctypes.byref(da), ctypes.byref(db), ctypes.byref(res), _stream(stream)), "tt_inner")
    return res.value


def min_gen_eig(M: DevTT, dM: DevTT, rank: int = 4, sweeps: int = 4, two_site: bool = True, seed: int = 1234,
                stream=None) -> float:
    """min over TT vectors e of <e, dM e>/<e, M e> (tt_min_gen_eig): the step-length eigenproblem."""
    lam = ctypes.c_double(0.0)
    a, b = M.desc(), dM.desc()
    _check(lib().tt_min_gen_eig(ctypes.byref(a), ctypes.byref(b), int(rank), int(sweeps), int(bool(two_site)),
                                int(seed), ctypes.byref(lam), _stream(stream)), "tt_min_gen_eig")
    return lam.value


def round_tt(a: DevTT, delta: float, cap: int = 0, stream=None):
    """TT rounding of the vector view of `a`; returns (DevTT, zeta)."""
    import torch
    v = DevTT(a.ranks, a.m * a.n, 1, a.flat)
    out = torch.empty(a.flat.numel(), dtype=torch.float64, device=a.flat.device)
    ranks = (ctypes.c_int32 * (a.d + 1))()
    zeta = ctypes.c_double(0.0)
    dv = v.desc()
    _check(lib().tt_round(ctypes.byref(dv), float(delta), int(cap), ranks, _ptr(out), out.numel(),
                          ctypes.byref(zeta), FP64, _stream(stream)), "tt_round")
    rr = list(ranks)
    return DevTT(rr, a.m, a.n, out[:_count(rr, a.m * a.n, 1)].clone()), zeta.value


def tt_from_dense(dense, eps_rel=1e-13, cap=0, stream=None):
    """TT-matrix cores (host numpy, r x n x n x r') of a dense n^d x n^d device matrix (row a1)."""
    import torch
    assert dense.is_cuda and dense.dtype == torch.float64
    N = dense.shape[0]
    d = int(round(np.log2(N)))
    assert 2 ** d == N and dense.shape == (N, N)
    ranks = (ctypes.c_int32 * (d + 1))()
    cnt = ctypes.c_size_t(0)
    dense = dense.contiguous()
    _check(lib().tt_from_dense(_ptr(dense), d, 2, float(eps_rel), int(cap), ranks, None, ctypes.byref(cnt),
                               _stream(stream)), "tt_from_dense")
    buf = np.empty(cnt.value, dtype=np.float64)
    _check(lib().tt_from_dense(_ptr(dense), d, 2, float(eps_rel), int(cap), ranks, buf.ctypes.data_as(ctypes.c_void_p),
                               ctypes.byref(cnt), _stream(stream)), "tt_from_dense")
    r = list(ranks)
    out, off = [], 0
    for k in range(d):
        size = r[k] * 4 * r[k + 1]
        out.append(buf[off:off + size].reshape(r[k], 2, 2, r[k + 1]).copy())
        off += size
    return out


# --- the solver (rows a1-a5, a10-a12) ----------------------------------------

def default_options(**kw) -> _lib.Options:
    o = _lib.Options()
    lib().tt_sdp_default_options(ctypes.byref(o))
    names = {f for f, _ in _lib.Options._fields_}
    for k, v in kw.items():
        if k not in names:
            raise TypeError(f"unknown option {k!r}")
        setattr(o, k, v)
    return o


class _HostTT:
    """Host cores packed for a tt_desc (kept alive with the descriptor)."""

    def __init__(self, cores, m, n):
        self.flat = np.ascontiguousarray(np.concatenate([np.asarray(c, dtype=np.float64).reshape(-1) for c in cores]))
        ranks = [c.shape[0] for c in cores] + [cores[-1].shape[-1]]
        self.r = (ctypes.c_int32 * len(ranks))(*ranks)
        self.desc = _lib.TTDesc(len(cores), ctypes.cast(self.r, _lib.P_int32), m, n,
                                self.flat.ctypes.data_as(ctypes.c_void_p))


def _problem(parts: dict):
    """tt_sdp_problem from host cores: C (r, 2, 2, r'), A_eq and K_y (r, 4, 4, r'),
    B_eq (r, 4, r'), optional A_ineq, B_ineq, K_t, ones_t, ineq_sign, q, lam0, lam0_ineq."""
    keep = []

    def desc(name, m, n):
        cores = parts.get(name)
        if cores is None:
            return _lib.TTDesc(0, None, m, n, None)
        h = _HostTT(cores, m, n)
        keep.append(h)
        return h.desc

    pr = _lib.Problem(desc("C", 2, 2), desc("A_eq", 4, 4), desc("B_eq", 4, 1), desc("K_y", 4, 4),
                      desc("A_ineq", 4, 4), desc("B_ineq", 4, 1), desc("K_t", 4, 4), desc("ones_t", 2, 2),
                      int(parts.get("ineq_sign", 1)), int(parts.get("q", 0)), float(parts.get("lam0", 1.0)),
                      float(parts.get("lam0_ineq", 1e-3)))
    return pr, keep


def make_allocator(alloc, free, user=None):
    """A tt_allocator from two Python callables alloc(nbytes, stream) -> int pointer
    and free(ptr, stream). Keep the returned object alive while contexts use it."""
    a = _lib.Allocator(_lib.ALLOC_FN(lambda n, st, u: alloc(int(n), st) or None),
                       _lib.FREE_FN(lambda ptr, st, u: free(ptr, st)), user)
    return a


def round_sdp(cores, tol, cap=0, psd_shift=0, stream=None):
    """tt_sdp_round on host cores (r, m, n, r') or (r, m, r'): TT rounding plus
    the spectral shift (0 none, 1 zeta I, 2 zeta (J - I)). Returns (cores, zeta)."""
    c0 = np.asarray(cores[0])
    mat = c0.ndim == 4
    m = c0.shape[1]
    n = c0.shape[2] if mat else 1
    h = _HostTT(cores, m, n)
    d = len(cores)
    ranks = (ctypes.c_int32 * (d + 1))()
    out = _lib.TTDesc(d, ctypes.cast(ranks, _lib.P_int32), m, n, None)
    zeta = ctypes.c_double(0.0)
    _check(lib().tt_sdp_round(ctypes.byref(h.desc), float(tol), int(cap), int(psd_shift), ctypes.byref(out),
                              ctypes.byref(zeta), _stream(stream)), "tt_sdp_round")
    r = list(ranks)
    buf = np.empty(_count(r, m, n), dtype=np.float64)
    out.cores = buf.ctypes.data_as(ctypes.c_void_p)
    _check(lib().tt_sdp_round(ctypes.byref(h.desc), float(tol), int(cap), int(psd_shift), ctypes.byref(out),
                              ctypes.byref(zeta), _stream(stream)), "tt_sdp_round")
    assert list(ranks) == r
    res, off = [], 0
    for k in range(d):
        shape = (r[k], m, n, r[k + 1]) if mat else (r[k], m, r[k + 1])
        size = int(np.prod(shape))
        res.append(buf[off:off + size].reshape(shape).copy())
        off += size
    return res, zeta.value


class Context:
    """One SDP in TT form with its iterates on the device (tt_sdp_ctx)."""

    def __init__(self, handle, keep):
        self._h = handle
        self._keep = keep

    @staticmethod
    def create(parts: dict, options=None, allocator=None, stream=None):
        """tt_sdp_create from host cores (see _problem); allocator from make_allocator or None."""
        pr, keep = _problem(parts)
        o = options or default_options()
        h = ctypes.c_void_p()
        _check(lib().tt_sdp_create(ctypes.byref(pr), ctypes.byref(o),
                                   ctypes.byref(allocator) if allocator is not None else None, _stream(stream),
                                   ctypes.byref(h)), "tt_sdp_create")
        return Context(h, keep + [allocator])

    @staticmethod
    def maxcut(weight_cores, options=None, stream=None):
        w = _HostTT(weight_cores, 2, 2)
        o = options or default_options()
        h = ctypes.c_void_p()
        _check(lib().tt_sdp_create_maxcut(ctypes.byref(w.desc), ctypes.byref(o), _stream(stream), ctypes.byref(h)),
               "tt_sdp_create_maxcut")
        return Context(h, [w])

    @staticmethod
    def theta(adj_cores, options=None, stream=None):
        a = _HostTT(adj_cores, 2, 2)
        o = options or default_options()
        h = ctypes.c_void_p()
        _check(lib().tt_sdp_create_theta(ctypes.byref(a.desc), ctypes.byref(o), _stream(stream), ctypes.byref(h)),
               "tt_sdp_create_theta")
        return Context(h, [a])

    @staticmethod
    def cc(c_plus_cores, c_minus_cores, adj_cores, options=None, stream=None):
        p, m, a = _HostTT(c_plus_cores, 2, 2), _HostTT(c_minus_cores, 2, 2), _HostTT(adj_cores, 2, 2)
        o = options or default_options()
        h = ctypes.c_void_p()
        _check(lib().tt_sdp_create_cc(ctypes.byref(p.desc), ctypes.byref(m.desc), ctypes.byref(a.desc),
                                      ctypes.byref(o), _stream(stream), ctypes.byref(h)), "tt_sdp_create_cc")
        return Context(h, [p, m, a])

    def newton_step(self) -> dict:
        info = _lib.IterInfo()
        _check(lib().tt_sdp_newton_step(self._h, ctypes.byref(info)), "tt_sdp_newton_step")
        return {f: getattr(info, f) for f, _ in _lib.IterInfo._fields_}

    def redo_update(self, alpha_p: float = -1.0, alpha_d: float = -1.0):
        """tt_sdp_redo_update: redo the last update with other step lengths (negative keeps one)."""
        _check(lib().tt_sdp_redo_update(self._h, float(alpha_p), float(alpha_d)), "tt_sdp_redo_update")

    def solve(self) -> dict:
        res = _lib.Result()
        st = lib().tt_sdp_solve(self._h, ctypes.byref(res))
        out = {f: getattr(res, f) for f, _ in _lib.Result._fields_}
        if st not in (0, 7):
            _check(st, "tt_sdp_solve")
        return out

    def ranks(self, which: int):
        """Bond ranks (d + 1 ints) of X (0), Y (1), T (2), Z (3) or the AMEn frame (4)."""
        d = lib().tt_sdp_order(self._h)
        ranks = (ctypes.c_int32 * (d + 1))()
        cnt = ctypes.c_size_t(0)
        _check(lib().tt_sdp_get_iterate(self._h, which, ranks, None, ctypes.byref(cnt)), "tt_sdp_get_iterate")
        return list(ranks)

    def iterate(self, which: int):
        """Cores (host numpy, r x 2 x 2 x r') of X (0), Y (1), T (2) or Z (3)."""
        d = lib().tt_sdp_order(self._h)
        ranks = (ctypes.c_int32 * (d + 1))()
        cnt = ctypes.c_size_t(0)
        _check(lib().tt_sdp_get_iterate(self._h, which, ranks, None, ctypes.byref(cnt)), "tt_sdp_get_iterate")
        buf = np.empty(cnt.value, dtype=np.float64)
        _check(lib().tt_sdp_get_iterate(self._h, which, ranks, buf.ctypes.data_as(ctypes.c_void_p),
                                        ctypes.byref(cnt)), "tt_sdp_get_iterate")
        r = list(ranks)
        out, off = [], 0
        for k in range(d):
            size = r[k] * 4 * r[k + 1]
            out.append(buf[off:off + size].reshape(r[k], 2, 2, r[k + 1]).copy())
            off += size
        return out

    def set_rank_predictor(self, pred):
        _check(lib().tt_sdp_set_rank_predictor(self._h, pred._h if pred is not None else None),
               "tt_sdp_set_rank_predictor")

    def set_trace(self, on=True):
        _check(lib().tt_sdp_set_trace(self._h, 1 if on else 0), "tt_sdp_set_trace")

    def trace(self):
        n = ctypes.c_size_t(0)
        _check(lib().tt_sdp_get_trace(self._h, None, None, ctypes.byref(n)), "tt_sdp_get_trace")
        X = np.empty((n.value, 10), dtype=np.float32)
        t = np.empty(n.value, dtype=np.float32)
        if n.value:
            _check(lib().tt_sdp_get_trace(self._h, X.ctypes.data, t.ctypes.data, ctypes.byref(n)), "tt_sdp_get_trace")
        return X, t

    def close(self):
        if self._h and not getattr(self, "_borrowed", False):
            lib().tt_sdp_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """n independent SDPs in one batch context (tt_sdp_create_batch)."""

    def __init__(self, parts_list, options=None, allocator=None, stream=None):
        n = len(parts_list)
        probs = (_lib.Problem * n)()
        self._keep = [allocator]
        for i, parts in enumerate(parts_list):
            probs[i], k = _problem(parts)
            self._keep += k
        o = options or default_options()
        self._h = ctypes.c_void_p()
        _check(lib().tt_sdp_create_batch(n, probs, ctypes.byref(o),
                                         ctypes.byref(allocator) if allocator is not None else None,
                                         _stream(stream), ctypes.byref(self._h)), "tt_sdp_create_batch")

    def __len__(self):
        return int(lib().tt_sdp_batch_size(self._h))

    def solve(self):
        n = len(self)
        res = (_lib.Result * n)()
        st = lib().tt_sdp_solve(self._h, res)
        if st not in (0, 7):
            _check(st, "tt_sdp_solve")
        return [{f: getattr(r, f) for f, _ in _lib.Result._fields_} for r in res]

    def member(self, i: int) -> Context:
        """Instance i as a borrowed Context (do not close it; the batch owns it)."""
        h = lib().tt_sdp_batch_member(self._h, int(i))
        if not h:
            raise IndexError(i)
        c = Context(ctypes.c_void_p(h), [self])
        c._borrowed = True
        return c

    def close(self):
        if self._h:
            lib().tt_sdp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_batch(contexts, workers=8):
    """Solve independent contexts concurrently (tt_sdp_solve_batch); returns one result dict each."""
    n = len(contexts)
    handles = (ctypes.c_void_p * n)(*[c._h for c in contexts])
    res = (_lib.Result * n)()
    st = lib().tt_sdp_solve_batch(n, handles, workers, res)
    if st not in (0, 7):
        _check(st, "tt_sdp_solve_batch")
    return [{f: getattr(r, f) for f, _ in _lib.Result._fields_} for r in res]


class RankPredictor:
    """The learned per-bond rank predictor (tt_rankpred); arrays are host numpy float32."""

    def __init__(self, seed: int = 0):
        self._h = ctypes.c_void_p()
        _check(lib().tt_rankpred_create(seed, ctypes.byref(self._h)), "tt_rankpred_create")
        self.nparam = int(lib().tt_rankpred_param_count())

    @staticmethod
    def _f32(a):
        return np.ascontiguousarray(a, dtype=np.float32)

    def params(self):
        out = np.empty(self.nparam, dtype=np.float32)
        _check(lib().tt_rankpred_get_params(self._h, out.ctypes.data), "tt_rankpred_get_params")
        return out

    def set_params(self, p):
        p = self._f32(p)
        _check(lib().tt_rankpred_set_params(self._h, p.ctypes.data), "tt_rankpred_set_params")

    def grad(self, X, t):
        X, t = self._f32(X), self._f32(t)
        g = np.empty(self.nparam, dtype=np.float32)
        loss = ctypes.c_float(0.0)
        _check(lib().tt_rankpred_grad(self._h, X.ctypes.data, t.ctypes.data, len(t), g.ctypes.data,
                                      ctypes.byref(loss)), "tt_rankpred_grad")
        return loss.value, g

    def train(self, X, t, epochs=200, batch=256, lr=1e-3, seed=0):
        X, t = self._f32(X), self._f32(t)
        loss = ctypes.c_float(0.0)
        _check(lib().tt_rankpred_train(self._h, X.ctypes.data, t.ctypes.data, len(t), epochs, batch, lr, seed,
                                       ctypes.byref(loss)), "tt_rankpred_train")
        return loss.value

    def predict(self, X):
        X = self._f32(X)
        y = np.empty(X.shape[0], dtype=np.float32)
        _check(lib().tt_rankpred_predict(self._h, X.ctypes.data, X.shape[0], y.ctypes.data), "tt_rankpred_predict")
        return y

    def __del__(self):
        try:
            if self._h:
                lib().tt_rankpred_destroy(self._h)
        except Exception:
            pass


def launch_count() -> int:
    return int(lib().tt_launch_count())


def contraction_stats():
    f, s = ctypes.c_double(0.0), ctypes.c_double(0.0)
    lib().tt_contraction_stats(ctypes.byref(f), ctypes.byref(s))
    return f.value, s.value


def tc_stats():
    """(flops, seconds, launches) of the tensor-core GEMM launches since the last reset."""
    f, s, n = ctypes.c_double(0.0), ctypes.c_double(0.0), ctypes.c_uint64(0)
    lib().tt_tc_stats(ctypes.byref(f), ctypes.byref(s), ctypes.byref(n))
    return f.value, s.value, n.value


def contraction_stats_reset():
    lib().tt_contraction_stats_reset()


def profile_report() -> dict:
    """Per-phase seconds collected when TTSDP_PROFILE=1 is set."""
    buf = ctypes.create_string_buffer(1 << 16)
    lib().tt_profile_report(buf, len(buf))
    out = {}
    for ln in buf.value.decode().splitlines():
        k, v = ln.split()
        out[k] = float(v)
    return out


def gemm64_stats():
    """(flops, seconds, launches) of the FP64 strided GEMM launches since the last reset."""
    f, s, n = ctypes.c_double(0.0), ctypes.c_double(0.0), ctypes.c_uint64(0)
    lib().tt_gemm64_stats(ctypes.byref(f), ctypes.byref(s), ctypes.byref(n))
    return f.value, s.value, n.value


def lu_stats():
    """(flops, seconds, systems) of the dense local LU solves since the last reset."""
    f, s, n = ctypes.c_double(0.0), ctypes.c_double(0.0), ctypes.c_uint64(0)
    lib().tt_lu_stats(ctypes.byref(f), ctypes.byref(s), ctypes.byref(n))
    return f.value, s.value, n.value


def lu_solve(K, b, precision=FP64, stream=None) -> float:
    """tt_lu_solve: b (device, float64) <- K^{-1} b for a device K (n x n, float64,
    row-major, kept); returns the FP64 relative residual."""
    n = int(K.shape[0])
    assert K.shape == (n, n) and b.numel() == n
    res = ctypes.c_double(0.0)
    _check(lib().tt_lu_solve(n, _ptr(K), _ptr(b), int(precision), ctypes.byref(res), _stream(stream)),
           "tt_lu_solve")
    return res.value


def kkt_solve(K, b, n_lz: int, precision=FP64, stream=None) -> float:
    """tt_kkt_solve: b (device, float64) <- K^{-1} b for a reduced projected
    system K (n x n, float64, row-major, kept) whose last n_lz rows and first
    n_lz columns hold the positive definite L_Z block, by block elimination;
    returns the FP64 relative residual."""
    n = int(K.shape[0])
    assert K.shape == (n, n) and b.numel() == n
    res = ctypes.c_double(0.0)
    _check(lib().tt_kkt_solve(n, int(n_lz), _ptr(K), _ptr(b), int(precision), ctypes.byref(res),
                              _stream(stream)), "tt_kkt_solve")
    return res.value


def kkt_stats(reset: bool = False, not_pd: bool = False):
    """(block-elimination solves, of them with FP32 factors, LU fallbacks)
    since the last reset, and with not_pd=True also the Cholesky
    factorisations that met a non-positive pivot of L_Z."""
    a, h, f, z = ctypes.c_uint64(0), ctypes.c_uint64(0), ctypes.c_uint64(0), ctypes.c_uint64(0)
    lib().tt_kkt_stats(ctypes.byref(a), ctypes.byref(h), ctypes.byref(f), ctypes.byref(z), int(bool(reset)))
    return (a.value, h.value, f.value, z.value) if not_pd else (a.value, h.value, f.value)
