"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every function include/dpp.h declares, and rejects bad arguments before
enqueueing anything."""
import ctypes
import os
import re

import pytest

import paper_1905_00165_gb300 as dpp
from paper_1905_00165_gb300 import _lib
from paper_1905_00165_gb300 import build as cuda_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    cuda_build.build()
    return dpp.load()


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "dpp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dpp_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("dpp_sample_hermitian", "dpp_sample_lu", "dpp_logprob_backward",
                     "dpp_workspace_size", "dpp_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(L):
    for name in _declared_functions():
        assert hasattr(L, name), name


def test_abi_version(L):
    assert L.dpp_abi_version() == 1


def test_workspace_sizes(L):
    for op in (0, 1):
        for dt in (0, 1):
            assert dpp.workspace_size(op, 1000, dt, 0, 1) > 1000 * 1000 * 8
    assert dpp.workspace_size(0, 0, 0, 0, 1) > 0
    assert dpp.workspace_size(0, 100, 7, 0, 1) == 0  # unknown dtype
    assert dpp.workspace_size(9, 100, 0, 0, 1) == 0  # unknown op
    # mixed LU: its FP32 copy of K is full square (planar for complex)
    assert dpp.workspace_size(1, 100, 0, 1, 0) > 100 * 100 * 4
    assert dpp.workspace_size(1, 100, 0, 2, 0) == dpp.workspace_size(1, 100, 0, 1, 0)
    assert dpp.workspace_size(1, 100, 1, 1, 0) > 100 * 100 * 8
    # complex mixed Hermitian: planar FP32 copy (8 B per element)
    assert dpp.workspace_size(0, 100, 1, 2, 1) > 100 * 100 * 8


def _call(L, K=None, n=4, ld=4, dtype=0, prec=0, keep=None, res=None, ws=None, wsb=0):
    return L.dpp_sample_hermitian(K, n, ld, dtype, prec, 0, 0, None, keep, None, None, res, ws, wsb, None)


def test_invalid_arguments_rejected_on_host(L):
    fake = 4096  # never dereferenced: validation fails first
    assert _call(L, n=-1) == _lib.DPP_ERR_INVALID_ARG
    assert "n must be" in dpp._lib.last_error()
    assert _call(L, K=fake, n=4, ld=3, keep=fake, res=fake) == _lib.DPP_ERR_INVALID_ARG
    assert _call(L, K=fake, n=4, ld=4, dtype=5, keep=fake, res=fake) == _lib.DPP_ERR_INVALID_ARG
    assert _call(L, K=None, n=4, keep=fake, res=fake) == _lib.DPP_ERR_INVALID_ARG
    assert _call(L, K=fake, n=4, keep=fake, res=None) == _lib.DPP_ERR_INVALID_ARG
    assert _call(L, K=fake + 4, n=4, keep=fake, res=fake) == _lib.DPP_ERR_INVALID_ARG  # misaligned
    # workspace: missing, misaligned, too small
    assert _call(L, K=fake, n=4, keep=fake, res=fake) == _lib.DPP_ERR_WORKSPACE
    assert _call(L, K=fake, n=4, keep=fake, res=fake, ws=fake + 8, wsb=1 << 20) == _lib.DPP_ERR_WORKSPACE
    assert _call(L, K=fake, n=4, keep=fake, res=fake, ws=fake, wsb=16) == _lib.DPP_ERR_WORKSPACE
    # unsupported precision (FP32 is the batched entry's only)
    assert _call(L, K=fake, n=4, dtype=1, prec=3, keep=fake, res=fake, ws=fake, wsb=1 << 30) == \
        _lib.DPP_ERR_UNSUPPORTED
    assert L.dpp_uniforms(0, 0, -1, None, None) == _lib.DPP_ERR_INVALID_ARG


def test_static_entry_limits_checked_on_host(L):
    """The allocation-free entry point rejects orders whose scratch would not
    fit its fixed array, and a missing factor buffer, before any CUDA call."""
    hdr = open(os.path.join(ROOT, "include", "dpp.h")).read()
    macros = {name: int(v) << int(sh or 0) for name, v, sh in
              re.findall(r"#define (DPP_STATIC_\w+) \(?(\d+)u?(?: << (\d+))?", hdr)}
    assert macros["DPP_STATIC_SCRATCH_BYTES"] == _lib.DPP_STATIC_SCRATCH_BYTES
    assert macros["DPP_STATIC_MAX_N_R64"] == _lib.DPP_STATIC_MAX_N_R64
    assert macros["DPP_STATIC_MAX_N_C128"] == _lib.DPP_STATIC_MAX_N_C128
    fake = 4096  # never dereferenced: validation fails first
    f = L.dpp_sample_hermitian_static
    for dt, nmax in [(_lib.DPP_R64, _lib.DPP_STATIC_MAX_N_R64),
                     (_lib.DPP_C128, _lib.DPP_STATIC_MAX_N_C128)]:
        # the largest accepted order fills the array; one more does not fit
        esz = 16 if dt == _lib.DPP_C128 else 8
        a256 = lambda b: (b + 255) // 256 * 256
        need = lambda n: a256(esz * n * 32) + a256(16 * n) + 512
        assert need(nmax) <= _lib.DPP_STATIC_SCRATCH_BYTES < need(nmax + 1)
        n = nmax + 1
        assert f(fake, n, n, dt, 0, 0, None, fake, fake, None, fake, None) == _lib.DPP_ERR_WORKSPACE
        assert "limit" in _lib.last_error()
    assert f(fake, 4, 4, _lib.DPP_R64, 0, 0, None, fake, None, None, fake, None) == \
        _lib.DPP_ERR_INVALID_ARG
    assert f(fake, 4, 3, _lib.DPP_R64, 0, 0, None, fake, fake, None, fake, None) == \
        _lib.DPP_ERR_INVALID_ARG


def test_batched_adjoint_workspace_query(L):
    """The one-launch batched adjoint's workspace: descriptors per instance plus
    at least one CTA's n_max^2 scratch; grows with the batch and n_max."""
    L.dpp_logprob_backward_batched_workspace.argtypes = [ctypes.c_int32, ctypes.c_int64]
    L.dpp_logprob_backward_batched_workspace.restype = ctypes.c_size_t
    a = L.dpp_logprob_backward_batched_workspace(10, 300)
    assert a >= 8 * 320 * 320
    assert L.dpp_logprob_backward_batched_workspace(1000, 300) > a
    assert L.dpp_logprob_backward_batched_workspace(10, 600) > a
    assert L.dpp_logprob_backward_batched_workspace(-1, 300) == 0


def test_tuning_keys_validated_on_host(L):
    """Every tuning key round-trips through set/get and rejects out-of-range
    values (no CUDA call involved)."""
    cases = [
        (_lib.DPP_TUNE_TAU_SAFETY, [8.0, 4.0], [0.0, -1.0]),
        (_lib.DPP_TUNE_OUTER_BLOCK, [256, 64], [48, 512, 0]),
        (_lib.DPP_TUNE_UPDATE_KERNEL, [0, 1], [2]),
        (_lib.DPP_TUNE_MAX_CTAS, [0, 8, 38], [4, 5000]),
        (_lib.DPP_TUNE_PANEL_PIPELINE, [0, 1, 2, 3], [4, -1]),
        (_lib.DPP_TUNE_WAIT_NS, [2e9, 1e6], [1e4, 1e11, -1.0]),
        (_lib.DPP_TUNE_FAULT_WITHHOLD, [1, 0], [2, -1]),
        (_lib.DPP_TUNE_USE_CACHE, [0, 1], [2, -1]),
        (_lib.DPP_TUNE_UPDATE_VARIANT, [0, 1, 2, 3], [4, -1, 0.5]),
        (_lib.DPP_TUNE_PANEL_CTAS, [0, 8, 16], [4, 5000, 9.5]),
        (_lib.DPP_TUNE_BATCHED_THREADS, [256, 128], [0, 64, 200]),
    ]
    for key, good, bad in cases:
        old = _lib.get_tuning(key)
        try:
            for v in good:
                _lib.set_tuning(key, v)
                assert _lib.get_tuning(key) == v
            for v in bad:
                assert L.dpp_set_tuning(key, float(v)) == _lib.DPP_ERR_INVALID_ARG
                assert _lib.get_tuning(key) == good[-1]
        finally:
            _lib.set_tuning(key, old)
    assert L.dpp_set_tuning(99, 1.0) == _lib.DPP_ERR_INVALID_ARG


def test_mixed_workspace_sizes_per_form():
    """Mixed precision: real Hermitian (either panel pipeline), complex
    Hermitian (planar copy, 8 B per element), real LU (full square) and
    complex LU (planar full square) have workspaces."""
    n = 1000
    herm = dpp.workspace_size(0, n, _lib.DPP_R64, _lib.DPP_PREC_3XTF32, 1)
    cplx = dpp.workspace_size(0, n, _lib.DPP_C128, _lib.DPP_PREC_3XTF32, 1)
    lu = dpp.workspace_size(1, n, _lib.DPP_R64, _lib.DPP_PREC_BF16X6, 0)
    cxlu = dpp.workspace_size(1, n, _lib.DPP_C128, _lib.DPP_PREC_BF16X6, 0)
    assert herm >= 4 * n * n and lu >= 4 * n * n and cplx >= 8 * n * n and cxlu >= 8 * n * n
    assert cxlu == dpp.workspace_size(1, n, _lib.DPP_C128, _lib.DPP_PREC_3XTF32, 0)


def test_greedy_workspace_and_arguments(L):
    """The greedy entry points need the sampler's workspace plus n doubles of
    thresholds, and reject bad arguments on the host."""
    for op_s, op_g, herm in ((0, 3, 1), (1, 4, 0)):
        for prec in (0, 1, 2):
            ws = dpp.workspace_size(op_s, 1000, 0, prec, herm)
            assert dpp.workspace_size(op_g, 1000, 0, prec, herm) == ws + 8000 + 192
    cx = dpp.workspace_size(1, 100, 1, 1, 0)
    assert dpp.workspace_size(4, 100, 1, 1, 0) == cx + 800 + 224  # complex mixed LU
    fake = 4096
    f = L.dpp_greedy_hermitian
    assert f(fake, -1, 4, 0, 0, fake, None, None, fake, fake, 1 << 20, None) == _lib.DPP_ERR_INVALID_ARG
    assert f(fake, 4, 4, 0, 0, fake, None, None, fake, fake, 16, None) == _lib.DPP_ERR_WORKSPACE
    need = dpp.workspace_size(3, 4, 0, 1, 1)
    # mixed in place is refused before anything is enqueued
    assert f(fake, 4, 4, 0, 1, fake, fake, None, fake, fake, need, None) == _lib.DPP_ERR_INVALID_ARG


def test_tune_cache_round_trip(L, tmp_path):
    """The autotuner's table: a JSON file loads, saves back with the same
    entries, merges by key, and malformed or out-of-range files are refused
    (host only: no device is needed to read or write the table)."""
    import json
    entries = [
        {"gpu": "NVIDIA GB300", "sms": 152, "op": 0, "dtype": 0, "precision": 1,
         "n_bucket": 14, "n": 16384, "outer_block": 256, "panel_pipeline": 1,
         "max_ctas": 38, "streams": 4, "samples_per_s": 47.5, "candidates": 12,
         "update_variant": 2},
        {"gpu": "NVIDIA GB300", "sms": 152, "op": 1, "dtype": 0, "precision": 2,
         "n_bucket": 13, "n": 8192, "outer_block": 128, "panel_pipeline": 0,
         "max_ctas": 0, "streams": 1, "samples_per_s": 80.25, "candidates": 6,
         "update_variant": 0},
        {"gpu": "NVIDIA GB300", "sms": 152, "op": 5, "dtype": 0, "precision": 3,
         "n_bucket": 10, "n": 1024, "outer_block": 0, "panel_pipeline": 0,
         "max_ctas": 0, "streams": 1, "samples_per_s": 46089.5, "candidates": 2,
         "update_variant": 0, "batched_threads": 128},
    ]
    for e in entries:
        e.setdefault("batched_threads", 0)
    src = tmp_path / "in.json"
    src.write_text(json.dumps({"version": 1, "entries": entries}))
    _lib.tune_clear()
    try:
        _lib.tune_load(str(src))
        out = tmp_path / "out.json"
        _lib.tune_save(str(out))
        got = json.loads(out.read_text())["entries"]
        assert got == entries
        # an entry with the same key replaces the old one
        upd = dict(entries[0], outer_block=128, samples_per_s=50.0)
        src.write_text(json.dumps({"version": 1, "entries": [upd]}))
        _lib.tune_load(str(src))
        _lib.tune_save(str(out))
        got = json.loads(out.read_text())["entries"]
        assert len(got) == 3 and got[0]["outer_block"] == 128 and got[1:] == entries[1:]
        # refused: malformed, out of range, missing
        bad = tmp_path / "bad.json"
        bad.write_text('{"entries": [{"gpu": "x", "sms": }]}')
        assert L.dpp_tune_load(str(bad).encode()) == _lib.DPP_ERR_INVALID_ARG
        bad.write_text(json.dumps({"entries": [dict(entries[0], outer_block=100)]}))
        assert L.dpp_tune_load(str(bad).encode()) == _lib.DPP_ERR_INVALID_ARG
        bad.write_text(json.dumps({"entries": [dict(entries[2], batched_threads=64)]}))
        assert L.dpp_tune_load(str(bad).encode()) == _lib.DPP_ERR_INVALID_ARG
        bad.write_text(json.dumps({"entries": [dict(entries[0], batched_threads=128)]}))
        assert L.dpp_tune_load(str(bad).encode()) == _lib.DPP_ERR_INVALID_ARG
        assert L.dpp_tune_load(str(tmp_path / "none.json").encode()) == _lib.DPP_ERR_INVALID_ARG
        _lib.tune_save(str(out))
        assert len(json.loads(out.read_text())["entries"]) == 3
    finally:
        _lib.tune_clear()


def test_autotune_batched_rejects_bad_arguments_on_host(L):
    """dpp_autotune_batched refuses a bad draw count or an empty batch before
    any device work."""
    fake = 4096
    f = L.dpp_autotune_batched
    assert f(4, fake, fake, fake, 64, 0, fake, fake, fake, 1 << 20, 0, None, None) == _lib.DPP_ERR_INVALID_ARG
    assert f(4, fake, fake, fake, 64, 0, fake, fake, fake, 1 << 20, 5000, None, None) == _lib.DPP_ERR_INVALID_ARG
    assert f(0, fake, fake, fake, 64, 0, fake, fake, fake, 1 << 20, 2, None, None) == _lib.DPP_ERR_INVALID_ARG


def test_autotune_rejects_bad_arguments_on_host(L):
    fake = 4096
    f = L.dpp_autotune
    need = L.dpp_autotune_workspace_size(0, 1000, 0, 1, 2)
    assert need > 2 * dpp.workspace_size(0, 1000, 0, 1, 1)
    assert L.dpp_autotune_workspace_size(2, 1000, 0, 1, 2) == 0  # not a sampler
    assert L.dpp_autotune_workspace_size(0, 1000, 0, 1, 9) == 0  # too many streams
    assert f(2, fake, 100, 100, 0, 1, 2, 4, fake, need, None, None) == _lib.DPP_ERR_INVALID_ARG
    assert f(0, fake, 100, 50, 0, 1, 2, 4, fake, need, None, None) == _lib.DPP_ERR_INVALID_ARG
    assert f(0, fake, 100, 100, 0, 1, 0, 4, fake, need, None, None) == _lib.DPP_ERR_INVALID_ARG
    assert f(0, fake, 100, 100, 0, 1, 2, 0, fake, need, None, None) == _lib.DPP_ERR_INVALID_ARG
    assert f(0, fake, 1000, 1000, 0, 1, 2, 4, fake, 1024, None, None) == _lib.DPP_ERR_WORKSPACE
    # complex LU in a mixed precision is tunable too: a too small workspace is refused
    assert L.dpp_autotune_workspace_size(1, 100, 1, 1, 2) > 2 * dpp.workspace_size(1, 100, 1, 1, 0)
    assert f(1, fake, 100, 100, 1, 1, 2, 4, fake, 1024, None, None) == _lib.DPP_ERR_WORKSPACE


def test_elementary_arguments_checked_on_host(L):
    fake = 4096
    f = L.dpp_sample_elementary
    need = L.dpp_elementary_workspace_size(100, 10)
    assert need >= 8 * 100 * 10
    assert L.dpp_elementary_workspace_size(100, 101) == 0
    assert L.dpp_elementary_workspace_size(-1, 0) == 0
    assert f(fake, 100, 100, 101, 0, 0, None, fake, None, None, fake, fake, need, None) == \
        _lib.DPP_ERR_INVALID_ARG  # k > n
    assert f(fake, 100, 99, 10, 0, 0, None, fake, None, None, fake, fake, need, None) == \
        _lib.DPP_ERR_INVALID_ARG  # ld < n
    assert f(fake, 100, 100, 10, 0, 0, None, None, None, None, fake, fake, need, None) == \
        _lib.DPP_ERR_INVALID_ARG  # no sample buffer
    assert f(fake, 100, 100, 10, 0, 0, None, fake, None, None, fake, fake, 64, None) == \
        _lib.DPP_ERR_WORKSPACE


def test_draw_schedule_fills_the_last_round():
    """Concurrent draws: full rounds keep the tuned cap; a partial last round
    of m draws takes sms // m CTAs per launch (never fewer than the tuned
    cap, 0 = one per SM when one draw is left); streams stay round-robin."""
    plan = dpp.draw_schedule(20, 8, 152, 19)
    assert [j for j, _ in plan] == [s % 8 for s in range(20)]
    assert [c for _, c in plan] == [19] * 16 + [38] * 4
    assert dpp.draw_schedule(40, 8, 152, 19) == [(s % 8, 19) for s in range(40)]
    assert dpp.draw_schedule(17, 8, 152, 19)[-1] == (0, 0)
    assert [c for _, c in dpp.draw_schedule(5, 8, 152, 19)] == [30] * 5
    assert [c for _, c in dpp.draw_schedule(7, 4, 152, 38)][4:] == [50] * 3
    # untuned (cap 0: one CTA per SM) and single-stream schedules are unchanged
    assert dpp.draw_schedule(3, 1, 152, 0) == [(0, 0)] * 3
    assert dpp.draw_schedule(5, 4, 152, 0) == [(s % 4, 0) for s in range(5)]
    # a tail share below the tuned cap keeps the cap
    assert dpp.draw_schedule(62, 32, 152, 8)[-1] == (29, 8)
    assert dpp.draw_schedule(0, 8, 152, 19) == []
    # every round's launches fit the SMs: sum of caps over a round <= sms
    for count, streams, cap in ((20, 8, 19), (23, 6, 25), (9, 4, 38), (3, 8, 19)):
        plan = dpp.draw_schedule(count, streams, 152, cap)
        for r0 in range(0, count, streams):
            assert sum(c for _, c in plan[r0:r0 + streams]) <= 152
    with pytest.raises(ValueError):
        dpp.draw_schedule(4, 0, 152, 19)


def test_tuning_knobs_set_and_restore(L):
    """The knob context sets a tuning entry's knobs explicitly (table off) and
    restores every previous value on exit, also after an exception."""
    keys = (_lib.DPP_TUNE_USE_CACHE, _lib.DPP_TUNE_OUTER_BLOCK, _lib.DPP_TUNE_PANEL_PIPELINE,
            _lib.DPP_TUNE_UPDATE_VARIANT, _lib.DPP_TUNE_MAX_CTAS)
    before = [_lib.get_tuning(k) for k in keys]
    entry = {"outer_block": 128, "panel_pipeline": 3, "update_variant": 1, "max_ctas": 19}
    with dpp.tuning_knobs(entry=entry, max_ctas=38):
        assert [_lib.get_tuning(k) for k in keys] == [0, 128, 3, 1, 38]
    assert [_lib.get_tuning(k) for k in keys] == before
    with pytest.raises(RuntimeError):
        with dpp.tuning_knobs(max_ctas=24, panel_pipeline=2):
            assert _lib.get_tuning(_lib.DPP_TUNE_MAX_CTAS) == 24
            assert _lib.get_tuning(_lib.DPP_TUNE_PANEL_PIPELINE) == 2
            raise RuntimeError("inside")
    assert [_lib.get_tuning(k) for k in keys] == before
