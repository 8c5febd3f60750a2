"""GB300-native factorization-based DPP sampler (arXiv:1905.00165).

Thin torch-facing wrappers over the C ABI in ``include/dpp.h``. torch provides
device memory and streams; the sampler itself runs in the library's sm_103a
kernels. Functions here only marshal arguments (column-major views, workspace
buffers, the current stream).
"""
from __future__ import annotations

from typing import Optional

from . import _lib
from ._lib import (DPP_C128, DPP_OP_LOGPROB_BACKWARD, DPP_OP_SAMPLE_HERMITIAN,
                   DPP_OP_SAMPLE_LU, DPP_PREC_3XTF32, DPP_PREC_BF16X6, DPP_PREC_FP64, DPP_R64,
                   DPPError, PRECISIONS, decode_result, load, workspace_size)

__all__ = ["sample_hermitian", "sample_hermitian_static", "sample_lu", "greedy_hermitian",
           "greedy_lu", "sample_batched", "BatchedSampler", "autotune",
           "lensemble_to_marginal", "sample_elementary",
           "logprob_backward", "uniforms", "Sample", "DPPLogProb", "DPPError", "load",
           "workspace_size", "draw_schedule", "tuning_knobs"]


def _torch():
    import torch
    return torch


def _dtype_code(t) -> int:
    torch = _torch()
    if t.dtype == torch.float64:
        return DPP_R64
    if t.dtype == torch.complex128:
        return DPP_C128
    raise TypeError(f"K must be float64 or complex128, got {t.dtype}")


def colmajor(K):
    """(tensor, ld): a tensor whose storage holds K column-major."""
    n = K.shape[0]
    if K.dim() != 2 or K.shape[1] != n:
        raise ValueError("K must be square")
    if n == 0:
        return K.contiguous(), 1
    if K.stride(0) == 1 and K.stride(1) >= n:
        return K, K.stride(1)
    return K.t().contiguous().t(), n


def empty_colmajor(n: int, dtype, device):
    """An n x n tensor with column-major storage (ld = n)."""
    torch = _torch()
    return torch.empty((n, n), dtype=dtype, device=device).t()


def _stream(device):
    torch = _torch()
    return torch.cuda.current_stream(device).cuda_stream


class Sample:
    """Device-resident outcome of one draw. ``result()`` synchronises."""

    def __init__(self, keep, pivots, factor, raw):
        self.keep = keep
        self.pivots = pivots
        self.factor = factor
        self.raw = raw
        self._res = None

    def result(self) -> dict:
        if self._res is None:
            self._res = decode_result(bytes(self.raw.cpu().numpy().tobytes()))
        return self._res

    @property
    def logp(self) -> float:
        return self.result()["logp"]

    @property
    def status(self) -> int:
        return self.result()["status"]


def _sample(hermitian: bool, K, seed: int, instance: int, precision: str, uniforms,
            factor: bool, workspace, out_keep=None):
    torch = _torch()
    L = load()
    if not K.is_cuda:
        raise ValueError("K must be a CUDA tensor")
    prec = PRECISIONS[precision]
    dt = _dtype_code(K)
    Kc, ld = colmajor(K)
    n = K.shape[0]
    dev = K.device
    keep = out_keep if out_keep is not None else torch.empty(n, dtype=torch.uint8, device=dev)
    npiv = 2 * n if (not hermitian and dt == DPP_C128) else n
    piv = torch.empty(max(npiv, 1), dtype=torch.float64, device=dev)
    fac = None
    if factor:
        # factor_out shares K's leading dimension: use ld = n for both
        if ld != n and n:
            Kc, ld = Kc.t().contiguous().t(), n
        fac = empty_colmajor(n, K.dtype, dev)
    raw = torch.zeros(_lib.RESULT_BYTES, dtype=torch.uint8, device=dev)
    op = DPP_OP_SAMPLE_HERMITIAN if hermitian else DPP_OP_SAMPLE_LU
    need = workspace_size(op, n, dt, prec, 1 if hermitian else 0)
    if need == 0:
        raise DPPError(_lib.DPP_ERR_UNSUPPORTED, f"unsupported: dtype={K.dtype} precision={precision}")
    ws = workspace if workspace is not None else torch.empty(need, dtype=torch.uint8, device=dev)
    if uniforms is not None:
        uniforms = uniforms.to(device=dev, dtype=torch.float64).contiguous()
        assert uniforms.numel() == n
    f = L.dpp_sample_hermitian if hermitian else L.dpp_sample_lu
    st = f(Kc.data_ptr() if n else None, n, ld, dt, prec, seed, instance,
           None if uniforms is None else uniforms.data_ptr(), keep.data_ptr() if n else None,
           None if fac is None else fac.data_ptr(), piv.data_ptr(), raw.data_ptr(),
           ws.data_ptr(), ws.numel(), _stream(dev))
    _lib.check(st)
    return Sample(keep, piv[:npiv], fac, raw)


def _greedy(hermitian: bool, K, precision: str, factor: bool, workspace):
    torch = _torch()
    L = load()
    if not K.is_cuda:
        raise ValueError("K must be a CUDA tensor")
    prec = PRECISIONS[precision]
    dt = _dtype_code(K)
    Kc, ld = colmajor(K)
    n = K.shape[0]
    dev = K.device
    keep = torch.empty(max(n, 1), dtype=torch.uint8, device=dev)
    npiv = 2 * n if (not hermitian and dt == DPP_C128) else n
    piv = torch.empty(max(npiv, 1), dtype=torch.float64, device=dev)
    fac = None
    if factor:
        if ld != n and n:
            Kc, ld = Kc.t().contiguous().t(), n
        fac = empty_colmajor(n, K.dtype, dev)
    raw = torch.zeros(_lib.RESULT_BYTES, dtype=torch.uint8, device=dev)
    op = _lib.DPP_OP_GREEDY_HERMITIAN if hermitian else _lib.DPP_OP_GREEDY_LU
    need = workspace_size(op, n, dt, prec, 1 if hermitian else 0)
    if need == 0:
        raise DPPError(_lib.DPP_ERR_UNSUPPORTED, f"unsupported: dtype={K.dtype} precision={precision}")
    ws = workspace if workspace is not None else torch.empty(need, dtype=torch.uint8, device=dev)
    f = L.dpp_greedy_hermitian if hermitian else L.dpp_greedy_lu
    st = f(Kc.data_ptr() if n else None, n, ld, dt, prec, keep.data_ptr() if n else None,
           None if fac is None else fac.data_ptr(), piv.data_ptr(), raw.data_ptr(),
           ws.data_ptr(), ws.numel(), _stream(dev))
    _lib.check(st)
    return Sample(keep[:n], piv[:npiv], fac, raw)


def greedy_hermitian(K, precision: str = "fp64", factor: bool = False, workspace=None) -> Sample:
    """Greedy maximum-likelihood set for Hermitian K: keep j iff d_j > 1/2."""
    return _greedy(True, K, precision, factor, workspace)


def greedy_lu(K, precision: str = "fp64", factor: bool = False, workspace=None) -> Sample:
    """Greedy maximum-likelihood set for general K (LU form)."""
    return _greedy(False, K, precision, factor, workspace)


def sample_hermitian(K, seed: int = 0, instance: int = 0, precision: str = "fp64",
                     uniforms=None, factor: bool = False, workspace=None) -> Sample:
    """Draw Y ~ DPP(K) for Hermitian K (LDL^H form; lower triangle read)."""
    return _sample(True, K, seed, instance, precision, uniforms, factor, workspace)


def sample_hermitian_static(K, factor, keep, pivots, raw, seed: int = 0, instance: int = 0,
                            uniforms=None) -> Sample:
    """FP64 Hermitian draw through dpp_sample_hermitian_static, which uses no
    workspace and allocates no device memory. Every output is caller-owned:
    ``factor`` (column-major n x n, may be K itself), ``keep`` (n uint8),
    ``pivots`` (n float64) and ``raw`` (RESULT_BYTES uint8)."""
    L = load()
    dt = _dtype_code(K)
    n = K.shape[0]
    if n and (K.stride(0) != 1 or factor.stride(0) != 1 or factor.stride(1) != K.stride(1)):
        raise ValueError("K and factor must be column-major with the same leading dimension")
    ld = K.stride(1) if n else 1
    st = L.dpp_sample_hermitian_static(
        K.data_ptr() if n else None, n, ld, dt, seed, instance,
        None if uniforms is None else uniforms.data_ptr(), keep.data_ptr() if n else None,
        factor.data_ptr() if n else None, pivots.data_ptr(), raw.data_ptr(), _stream(K.device))
    _lib.check(st)
    return Sample(keep, pivots[:n], factor, raw)


def sample_lu(K, seed: int = 0, instance: int = 0, precision: str = "fp64",
              uniforms=None, factor: bool = False, workspace=None) -> Sample:
    """Draw Y ~ DPP(K) for general K (LU form of Algorithm 1)."""
    return _sample(False, K, seed, instance, precision, uniforms, factor, workspace)


class BatchedSampler:
    """Reusable device state for repeated batched draws over a fixed list of
    real symmetric kernels (device pointer tables, outputs, workspace)."""

    def __init__(self, Ks, instance=None, want_pivots: bool = False, uniforms=None):
        torch = _torch()
        L = load()
        self.L = L
        self.Ks = []
        ns, lds = [], []
        for K in Ks:
            if K.dtype != torch.float64 or not K.is_cuda:
                raise TypeError("batched kernels must be float64 CUDA tensors")
            Kc, ld = colmajor(K)
            self.Ks.append(Kc)
            ns.append(K.shape[0])
            lds.append(ld)
        dev = Ks[0].device if Ks else torch.device("cuda")
        self.device = dev
        self.batch = len(Ks)
        self.n_max = max(ns) if ns else 0
        self.n = torch.tensor(ns, dtype=torch.int64, device=dev)
        self.ld = torch.tensor(lds, dtype=torch.int64, device=dev)
        self.kptr = torch.tensor([k.data_ptr() for k in self.Ks], dtype=torch.int64, device=dev)
        self.keep = [torch.empty(max(m, 1), dtype=torch.uint8, device=dev) for m in ns]
        self.keep_ptr = torch.tensor([k.data_ptr() for k in self.keep], dtype=torch.int64, device=dev)
        self.pivots = None
        self.piv_ptr = None
        if want_pivots:
            self.pivots = [torch.empty(max(m, 1), dtype=torch.float64, device=dev) for m in ns]
            self.piv_ptr = torch.tensor([p.data_ptr() for p in self.pivots], dtype=torch.int64, device=dev)
        self.u = None
        self.u_ptr = None
        if uniforms is not None:
            self.u = [uu.to(device=dev, dtype=torch.float64).contiguous() for uu in uniforms]
            self.u_ptr = torch.tensor([uu.data_ptr() for uu in self.u], dtype=torch.int64, device=dev)
        self.inst = None
        if instance is not None:
            self.inst = torch.tensor(list(instance), dtype=torch.int64, device=dev)
        self.raw = torch.zeros(max(self.batch, 1) * _lib.RESULT_BYTES, dtype=torch.uint8, device=dev)
        need = int(L.dpp_batched_workspace_size(self.batch, self.n_max, _lib.DPP_PREC_FP32))
        if need == 0:
            raise DPPError(_lib.DPP_ERR_UNSUPPORTED, "batched workspace query failed")
        self.ws = torch.empty(need, dtype=torch.uint8, device=dev)

    def draw(self, seed: int = 0) -> None:
        """Enqueue one draw of every instance on the current stream."""
        st = self.L.dpp_sample_batched(
            self.batch, self.n.data_ptr(), self.kptr.data_ptr(), self.ld.data_ptr(), self.n_max,
            _lib.DPP_PREC_FP32, seed, None if self.inst is None else self.inst.data_ptr(),
            self.keep_ptr.data_ptr(), None if self.u_ptr is None else self.u_ptr.data_ptr(),
            None if self.piv_ptr is None else self.piv_ptr.data_ptr(), self.raw.data_ptr(),
            self.ws.data_ptr(), self.ws.numel(), _stream(self.device))
        _lib.check(st)

    def autotune(self, draws: int = 4, seed: int = 0) -> dict:
        """Time this batch's draws with 128- and 256-thread CTAs
        (dpp_autotune_batched) and keep the faster in the library's tuning
        table for this batch's key (n_max bucket). Returns the entry."""
        import ctypes
        e = _lib.TuneEntry()
        _lib.check(self.L.dpp_autotune_batched(
            self.batch, self.n.data_ptr(), self.kptr.data_ptr(), self.ld.data_ptr(), self.n_max,
            seed, self.keep_ptr.data_ptr(), self.raw.data_ptr(), self.ws.data_ptr(),
            self.ws.numel(), draws, ctypes.byref(e), _stream(self.device)))
        return e.as_dict()

    def logprob_backward(self, grad_logp=None, count=None, precision: str = "fp64"):
        """dK_i = g_i (K_i - 1_{Y_i^c})^{-T} for the first ``count`` instances
        (default: all) and their last draw (one persistent launch over every
        instance; ``precision`` "fp64" or "fp32" arithmetic, FP64 dK)."""
        if precision not in ("fp64", "fp32"):
            raise ValueError("precision must be 'fp64' or 'fp32'")
        import ctypes
        import numpy as np
        torch = _torch()
        dev = self.device
        B = self.batch if count is None else min(int(count), self.batch)
        ns = [int(K.shape[0]) for K in self.Ks[:B]]
        if grad_logp is None:
            g = torch.ones(max(B, 1), dtype=torch.float64, device=dev)
        else:
            g = torch.as_tensor(grad_logp, dtype=torch.float64, device=dev).reshape(B).contiguous()
        dKs = [empty_colmajor(m, torch.float64, dev) for m in ns]
        n_h = np.asarray(ns, dtype=np.int64)
        ld_h = np.asarray([K.stride(1) if m else 1 for K, m in zip(self.Ks[:B], ns)], dtype=np.int64)
        ldd_h = np.asarray([d.stride(1) if m else 1 for d, m in zip(dKs, ns)], dtype=np.int64)
        P = ctypes.c_void_p * max(B, 1)
        kp = P(*[K.data_ptr() for K in self.Ks[:B]])
        kk = P(*[k.data_ptr() for k in self.keep[:B]])
        gp = P(*[g.data_ptr() + 8 * i for i in range(B)])
        dp = P(*[d.data_ptr() for d in dKs])
        # the one-launch form: a descriptor per instance and n_max^2 scratch per CTA
        need = self.L.dpp_logprob_backward_batched_workspace(B, max(ns) if ns else 0)
        ws = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)
        fn = (self.L.dpp_logprob_backward_batched if precision == "fp64"
              else self.L.dpp_logprob_backward_batched_fp32)
        st = fn(
            B, n_h.ctypes.data, ctypes.cast(kp, ctypes.c_void_p), ld_h.ctypes.data,
            ctypes.cast(kk, ctypes.c_void_p), ctypes.cast(gp, ctypes.c_void_p),
            ctypes.cast(dp, ctypes.c_void_p), ldd_h.ctypes.data, ws.data_ptr(), ws.numel(),
            _stream(dev))
        _lib.check(st)
        return dKs

    def results(self):
        raw = self.raw.cpu().numpy().tobytes()
        return [decode_result(raw[i * _lib.RESULT_BYTES:(i + 1) * _lib.RESULT_BYTES])
                for i in range(self.batch)]


def sample_batched(Ks, seed: int = 0, instance=None, want_pivots: bool = False, uniforms=None):
    """One persistent-launch draw for each kernel in ``Ks``; returns the sampler
    (``.keep[i]``, ``.pivots[i]``, ``.results()``)."""
    b = BatchedSampler(Ks, instance=instance, want_pivots=want_pivots, uniforms=uniforms)
    b.draw(seed)
    return b


class ElementarySample:
    """Device-resident outcome of one elementary draw. ``result()`` synchronises."""

    def __init__(self, sample, keep, chol, raw):
        self.sample = sample
        self.keep = keep
        self.chol = chol
        self.raw = raw

    def result(self) -> dict:
        return decode_result(bytes(self.raw.cpu().numpy().tobytes()))


def sample_elementary(K, k: int, seed: int = 0, instance: int = 0, uniforms=None,
                      chol: bool = False, workspace=None) -> ElementarySample:
    """Algorithm 2: a sample of DPP(K) for a real symmetric projection K of rank k."""
    torch = _torch()
    L = load()
    if not K.is_cuda or K.dtype != torch.float64:
        raise TypeError("K must be a float64 CUDA tensor")
    Kc, ld = colmajor(K)
    n = K.shape[0]
    dev = K.device
    sample = torch.empty(max(k, 1), dtype=torch.int64, device=dev)
    keep = torch.empty(max(n, 1), dtype=torch.uint8, device=dev)
    ch = empty_colmajor(max(k, 1), torch.float64, dev) if chol else None
    raw = torch.zeros(_lib.RESULT_BYTES, dtype=torch.uint8, device=dev)
    need = int(L.dpp_elementary_workspace_size(n, k))
    if need == 0:
        raise DPPError(_lib.DPP_ERR_INVALID_ARG, "bad n or k")
    ws = workspace if workspace is not None else torch.empty(need, dtype=torch.uint8, device=dev)
    if uniforms is not None:
        uniforms = uniforms.to(device=dev, dtype=torch.float64).contiguous()
    _lib.check(L.dpp_sample_elementary(
        Kc.data_ptr() if n else None, n, ld, k, seed, instance,
        None if uniforms is None else uniforms.data_ptr(), sample.data_ptr(), keep.data_ptr(),
        None if ch is None else ch.data_ptr(), raw.data_ptr(), ws.data_ptr(), ws.numel(),
        _stream(dev)))
    return ElementarySample(sample[:k], keep[:n], ch, raw)


def lensemble_to_marginal(Ls):
    """K_i = L_i (L_i + I)^{-1} for a list of real symmetric PSD L_i (FP64 CUDA
    tensors, n_i <= 4096), in one persistent launch (see
    dpp_lensemble_to_marginal_batched). Returns the K_i (column-major)."""
    import ctypes
    import numpy as np
    torch = _torch()
    L = load()
    B = len(Ls)
    if B == 0:
        return []
    Lc = [colmajor(x)[0] for x in Ls]
    for x in Ls:
        if x.dtype != torch.float64 or not x.is_cuda:
            raise TypeError("L-ensemble kernels must be float64 CUDA tensors")
    ns = [int(x.shape[0]) for x in Ls]
    dev = Ls[0].device
    Ks = [empty_colmajor(m, torch.float64, dev) for m in ns]
    n_h = np.asarray(ns, dtype=np.int64)
    ld_h = np.asarray([x.stride(1) if m else 1 for x, m in zip(Lc, ns)], dtype=np.int64)
    ldk_h = np.asarray([k.stride(1) if m else 1 for k, m in zip(Ks, ns)], dtype=np.int64)
    P = ctypes.c_void_p * B
    lp = P(*[x.data_ptr() for x in Lc])
    kp = P(*[k.data_ptr() for k in Ks])
    need = L.dpp_logprob_backward_batched_workspace(B, max(ns))
    ws = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)
    _lib.check(L.dpp_lensemble_to_marginal_batched(
        B, n_h.ctypes.data, ctypes.cast(lp, ctypes.c_void_p), ld_h.ctypes.data,
        ctypes.cast(kp, ctypes.c_void_p), ldk_h.ctypes.data, ws.data_ptr(), ws.numel(),
        _stream(dev)))
    return Ks


def autotune(K, hermitian: bool = True, precision: str = "3xtf32", max_streams: int = 4,
             draws: int = 8) -> dict:
    """Time the candidate launch configurations of a draw on K (see
    dpp_autotune) and keep the fastest in the library's tuning table, which
    every later call with the same key uses. Returns the chosen entry."""
    import ctypes
    torch = _torch()
    L = load()
    dt = _dtype_code(K)
    Kc, ld = colmajor(K)
    n = K.shape[0]
    op = DPP_OP_SAMPLE_HERMITIAN if hermitian else DPP_OP_SAMPLE_LU
    prec = PRECISIONS[precision]
    need = int(L.dpp_autotune_workspace_size(op, n, dt, prec, max_streams))
    if need == 0:
        raise DPPError(_lib.DPP_ERR_UNSUPPORTED, "autotune: unsupported configuration")
    ws = torch.empty(need, dtype=torch.uint8, device=K.device)
    e = _lib.TuneEntry()
    _lib.check(L.dpp_autotune(op, Kc.data_ptr(), n, ld, dt, prec, max_streams, draws,
                              ws.data_ptr(), need, ctypes.byref(e), _stream(K.device)))
    return e.as_dict()


def draw_schedule(count: int, streams: int, sms: int, cap: int) -> list:
    """Stream and per-launch CTA cap of each of `count` independent draws run
    concurrently on `streams` streams (draw s on stream s mod streams).

    Full rounds of `streams` draws keep `cap` (the tuned share of the `sms`
    SMs; 0 = one CTA per SM). A last, partial round of m < streams draws
    would leave streams - m shares idle, so its draws take max(cap, sms // m)
    CTAs each. Returns [(stream, cap), ...]; pure host arithmetic."""
    if count < 0 or streams < 1 or sms < 1 or cap < 0:
        raise ValueError("draw_schedule: count >= 0, streams >= 1, sms >= 1, cap >= 0")
    full = (count // streams) * streams
    m = count - full
    tail_cap = cap
    if m and cap:
        share = sms // m
        tail_cap = 0 if share >= sms else max(cap, share)
    return [(s % streams, cap if s < full else tail_cap) for s in range(count)]


class tuning_knobs:
    """Context manager: the given DPP_TUNE_* knobs for the calls made inside
    it, the previous values restored on exit. With `entry` (a tuning-table
    entry as returned by _lib.tune_lookup) the table is switched off and the
    entry's outer block, panel pipeline, update variant and CTA cap are set
    explicitly, `max_ctas` (if given) replacing its cap. The knobs are the
    library's process-wide settings, read when a call is enqueued: a context
    changes them for every thread of the process while it is open."""

    def __init__(self, entry=None, max_ctas=None, **knobs):
        self.want = {}
        if entry is not None:
            self.want[_lib.DPP_TUNE_USE_CACHE] = 0
            if entry["outer_block"] >= 32:
                self.want[_lib.DPP_TUNE_OUTER_BLOCK] = entry["outer_block"]
            self.want[_lib.DPP_TUNE_PANEL_PIPELINE] = entry["panel_pipeline"]
            self.want[_lib.DPP_TUNE_UPDATE_VARIANT] = entry["update_variant"]
            self.want[_lib.DPP_TUNE_MAX_CTAS] = entry["max_ctas"]
        if max_ctas is not None:
            self.want[_lib.DPP_TUNE_MAX_CTAS] = max_ctas
        for k, v in knobs.items():
            self.want[getattr(_lib, "DPP_TUNE_" + k.upper())] = v
        self.old = {}

    def __enter__(self):
        for k, v in self.want.items():
            self.old[k] = _lib.get_tuning(k)
            _lib.set_tuning(k, v)
        return self

    def __exit__(self, *exc):
        for k, v in reversed(list(self.old.items())):
            _lib.set_tuning(k, v)
        return False


def uniforms(seed: int, instance: int, n: int, device="cuda"):
    """The Philox uniforms u_0..u_{n-1} the samplers draw for (seed, instance)."""
    torch = _torch()
    out = torch.empty(max(n, 1), dtype=torch.float64, device=device)
    _lib.check(load().dpp_uniforms(seed, instance, n, out.data_ptr(), _stream(out.device)))
    return out[:n]


def logprob_backward(K, keep, grad_logp=None, hermitian: bool = True, workspace=None):
    """dK = g (K - 1_{Y^c})^{-H} (the adjoint of log P(Y) with Y fixed)."""
    torch = _torch()
    L = load()
    dt = _dtype_code(K)
    Kc, ld = colmajor(K)
    n = K.shape[0]
    dev = K.device
    g = grad_logp if grad_logp is not None else torch.ones((), dtype=torch.float64, device=dev)
    g = g.to(device=dev, dtype=torch.float64).reshape(1).contiguous()
    dK = empty_colmajor(n, K.dtype, dev)
    ldd = dK.stride(1) if n else 1
    need = workspace_size(DPP_OP_LOGPROB_BACKWARD, n, dt, DPP_PREC_FP64, 1 if hermitian else 0)
    if need == 0:
        raise DPPError(_lib.DPP_ERR_UNSUPPORTED, "unsupported backward configuration")
    ws = workspace if workspace is not None else torch.empty(need, dtype=torch.uint8, device=dev)
    keep = keep.to(device=dev, dtype=torch.uint8).contiguous()
    st = L.dpp_logprob_backward(Kc.data_ptr() if n else None, n, ld, dt, DPP_PREC_FP64,
                                1 if hermitian else 0, keep.data_ptr() if n else None,
                                g.data_ptr(), dK.data_ptr() if n else None, ldd,
                                ws.data_ptr(), ws.numel(), _stream(dev))
    _lib.check(st)
    return dK


def _make_autograd():
    torch = _torch()

    class _DPPLogProb(torch.autograd.Function):
        """log P(Y) = log|det(K - 1_{Y^c})| for a fixed sample Y.

        forward: the factorization with the decisions forced to ``keep``
        (the sampler's own kernels, uniforms that force each decision).
        backward: dK = g (K - 1_{Y^c})^{-H} from the library's adjoint, with
        the factors recomputed rather than stored.
        """

        @staticmethod
        def forward(ctx, K, keep, hermitian: bool = True):
            u = torch.where(keep.to(torch.bool), torch.tensor(-1e300, dtype=torch.float64, device=K.device),
                            torch.tensor(1e300, dtype=torch.float64, device=K.device))
            s = _sample(hermitian, K.detach(), 0, 0, "fp64", u, False, None)
            ctx.save_for_backward(K.detach(), keep)
            ctx.hermitian = hermitian
            raw = s.raw
            logp = raw[16:24].view(torch.float64).reshape(())
            return logp.clone()

        @staticmethod
        def backward(ctx, g):
            K, keep = ctx.saved_tensors
            dK = logprob_backward(K, keep, g.detach(), hermitian=ctx.hermitian)
            return dK, None, None

    return _DPPLogProb


DPPLogProb = _make_autograd()
