#!/usr/bin/env python
"""Benchmark of the factorization-based DPP sampler on GB300.

Headline: DPP samples/s for a dense real Hermitian marginal kernel of order
n = 16384, K = Q diag(lam) Q^T, Q Haar-orthogonal (seed 0), lam ~ Beta(1/2,1/2).
One step = one complete draw (every panel decision, panel solve and trailing
Schur update) with Philox seed = step index. Inputs are resident in HBM before
the timed region; the 2 GiB FP64 kernel (plus the 1 GiB FP32 working copy of
the mixed path) exceeds the 129 MB L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank draws its own samples (independent seeds; no
collective on the data path) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

FP64_NOMINAL_TFLOPS = 1.25  # GB300 FP64 (nominal, per GPU)
TF32_PER_BF16 = 1.1 / 2.25  # nominal dense TF32 : BF16 ratio


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=None)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=16384)
    p.add_argument("--kind", default="beta", choices=["beta", "uniform", "projection"])
    p.add_argument("--precision", default="auto", choices=["auto", "fp64", "3xtf32", "bf16x6"])
    p.add_argument("--update", default="tc", choices=["tc", "simt"],
                   help="mixed path trailing update: tcgen05 3xTF32 or SIMT FP32")
    p.add_argument("--gen", default="gpu", choices=["gpu", "cpu"],
                   help="where the input kernel's Haar factor is computed")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--e2e-buffers", type=int, default=0,
                   help="device buffers of K in the end-to-end ring (0: streams + 2)")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-fp64-ref", action="store_true")
    p.add_argument("--no-batched", action="store_true")
    p.add_argument("--streams", type=int, default=0,
                   help="draws in flight on this many streams, each launch capped at "
                        "SMs / streams CTAs (0: the autotuner's choice)")
    p.add_argument("--suite-only", default="",
                   help="with --suite: comma-separated subset of C1,C2,C3,C4,E,A")
    p.add_argument("--suite-cpu", action="store_true",
                   help="the oracle, as it stands, timed on the host cores at each "
                        "configuration of --suite (its own size, a bounded sample)")
    p.add_argument("--suite", action="store_true",
                   help="one JSON line per workload of the paper-shaped configurations "
                        "(FP64 n=512; n=4096 real/complex, projection/Beta; spanning trees of "
                        "the 64x64 grid; LU n=8192; batched L-ensembles)")
    p.add_argument("--batch", type=int, default=4096,
                   help="L-ensembles in the batched measurement (n ~ U{64..1024})")
    p.add_argument("--pipeline", type=int, default=-1,
                   help="with --case: DPP_TUNE_PANEL_PIPELINE for the draws (-1: default)")
    p.add_argument("--update-variant", type=int, default=-1,
                   help="with --case: DPP_TUNE_UPDATE_VARIANT for the draws (-1: default)")
    p.add_argument("--host-inputs", action="store_true",
                   help="with --case herm/cplx: build the kernel with numpy on the host")
    p.add_argument("--case", default="",
                   choices=["", "herm", "lu", "cplx", "aztec", "batched", "adjoint"],
                   help="run one path alone (a small loop for profiling): mixed Hermitian, "
                        "mixed LU, mixed complex Hermitian, mixed complex LU on an Aztec "
                        "diamond, batched sampler or batched adjoint")
    return p.parse_args()


def tc_traffic_per_launch(n: int, split: str = "3xtf32", kb: int = 256):
    """Mean DRAM bytes of one 3xTF32 k_update_tc launch of an order-n draw:
    bytes per m^2 from the one-launch ncu capture summarised in profiles/
    (n = 8192), times the mean m^2 over the draw's launches (m = n - kb,
    n - 2 kb, ...). None once dpp_tc.cu has changed since that capture."""
    import hashlib
    try:
        src = os.path.join(ROOT, "paper_1905_00165_gb300", "csrc", "dpp_tc.cu")
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        vals = {}
        name = f"k_update_tc_{split}_traffic_n8192.txt"
        with open(os.path.join(ROOT, "profiles", name)) as f:
            for ln in f:
                if ": " in ln:  # keys may hold a colon themselves ("sha256[:16]")
                    k, v = ln.split(": ", 1)
                    vals[k.strip()] = v.strip()
        if vals.get("dpp_tc.cu sha256[:16]") != h:
            return None
        per_m2 = float(vals["dram bytes per m^2"])
        ms = [n - kb * k for k in range(1, (n + kb - 1) // kb) if n - kb * k > 0]
        return per_m2 * sum(m * m for m in ms) / max(1, len(ms))
    except Exception:
        return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def bench_batched(dpp, _lib, dev, batch: int, draws: int, seed: int = 0):
    """Batched L-ensembles: `batch` kernels K_i = L_i (L_i + I)^{-1} of orders
    n_i ~ U{64..1024}, one persistent launch draws every instance once (FP32
    factor, FP64 pivots and recompute). samples/s = instances drawn per second."""
    import torch
    import workloads as W
    # L-ensemble kernels L_i = Phi_i Phi_i^T, converted on the device to their
    # marginal kernels K_i = L_i (L_i + I)^{-1} by the library (one launch)
    Ls = W.lensemble_L_batch_torch(batch, seed=seed, device=str(dev))
    torch.cuda.synchronize()
    stream0 = torch.cuda.current_stream(dev)
    c0 = torch.cuda.Event(enable_timing=True)
    c1 = torch.cuda.Event(enable_timing=True)
    c0.record(stream0)
    Ks = dpp.lensemble_to_marginal(Ls)
    c1.record(stream0)
    torch.cuda.synchronize()
    ms_conv = c0.elapsed_time(c1)
    del Ls
    sizes = [int(K.shape[0]) for K in Ks]
    b = dpp.BatchedSampler(Ks)
    stream = torch.cuda.current_stream(dev)
    for w in range(2):
        b.draw(10**6 + w)
    torch.cuda.synchronize()
    _lib.profile_start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for d in range(draws):
        b.draw(d)
    e1.record(stream)
    torch.cuda.synchronize()
    prof = _lib.profile_stop()
    ms = e0.elapsed_time(e1) / draws
    res = b.results()
    flops = sum(m ** 3 / 3.0 for m in sizes)
    bad = sum(1 for r in res if r["status"] & (_lib.DPP_RES_TIMEOUT | _lib.DPP_RES_NONFINITE))
    # adjoint dK_i = (K_i - 1_{Y_i^c})^{-T} of every instance's last draw (FP64)
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    n_adj = batch
    # untimed first call: the output buffers and the workspace come from the
    # caching allocator afterwards
    del_first = b.logprob_backward(count=n_adj)
    torch.cuda.synchronize()
    del del_first
    a0.record(stream)
    dKs = b.logprob_backward(count=n_adj)
    a1.record(stream)
    torch.cuda.synchronize()
    ms_adj = a0.elapsed_time(a1)
    del dKs
    # the same in FP32 arithmetic (dpp_logprob_backward_batched_fp32)
    first32 = b.logprob_backward(count=n_adj, precision="fp32")
    torch.cuda.synchronize()
    del first32
    a0.record(stream)
    dKs = b.logprob_backward(count=n_adj, precision="fp32")
    a1.record(stream)
    torch.cuda.synchronize()
    ms_adj32 = a0.elapsed_time(a1)
    del dKs
    return {"metric": f"batched L-ensemble samples/s ({batch} kernels, n~U{{64..1024}})",
            "value": batch / (ms / 1e3), "unit": "samples/s", "ms_per_draw": ms,
            "draws": draws, "tflops_algorithmic": flops / (ms / 1e3) / 1e12,
            "n_total": sum(sizes), "launches_per_draw":
                sum(v["launches"] for v in prof.values()) / draws,
            "borderline_last_draw": sum(r["n_borderline"] for r in res),
            "failed_instances": bad,
            "conversion": {"instances_per_s": batch / (ms_conv / 1e3), "ms": ms_conv,
                           "what": "K_i = L_i (L_i + I)^{-1} from L_i = Phi_i Phi_i^T, FP64, "
                                   "one persistent launch (dpp_lensemble_to_marginal_batched)"},
            "adjoint": {"instances_per_s": n_adj / (ms_adj / 1e3), "ms": ms_adj,
                        "instances": n_adj, "precision": "fp64",
                        "note": "dK_i = (K_i - 1_{Y_i^c})^{-T}: forced-decision FP64 "
                                "refactorization and triangular inverses, one library call",
                        "fp32": {"instances_per_s": n_adj / (ms_adj32 / 1e3), "ms": ms_adj32,
                                 "note": "the same steps in FP32 arithmetic, FP64 dK "
                                         "(dpp_logprob_backward_batched_fp32)"}},
            "config": {"workload": "lensemble_batch", "batch": batch, "nmin": 64, "nmax": 1024,
                       "features": 64, "quality": "LogUniform(0.1, 10)", "precision": "fp32"}}


def run_suite(args):
    """Every paper-shaped workload on one GPU: samples/s, algorithmic TFLOP/s and
    the fraction of the peak of the pipe the dominant kernel runs on."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1905_00165_gb300 as dpp
    from paper_1905_00165_gb300 import _lib
    import workloads as W
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    peaks = measured_peaks()
    bf16 = peaks.get("bf16_tflops", 1888.3)
    stream = torch.cuda.current_stream(dev)

    def timed(fn, draws, warm=2):
        for w in range(warm):
            fn(10**6 + w)
        torch.cuda.synchronize()
        _lib.profile_start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for d in range(draws):
            fn(d)
        e1.record(stream)
        torch.cuda.synchronize()
        prof = _lib.profile_stop()
        return e0.elapsed_time(e1) / draws, prof

    def line(name, cfg, prec, ms, flops, prof, extra=None):
        tf = flops / (ms / 1e3) / 1e12
        if prec == "fp64":
            peak, pipe = FP64_NOMINAL_TFLOPS, "fp64 nominal"
        else:
            peak, pipe = bf16 / 6.0, "bf16 measured / 6 products"
        upd = prof.get("update_tc") or prof.get("update_fp64")
        d = {"suite": name, "config": cfg, "precision": prec, "samples_per_s": 1e3 / ms,
             "ms_per_draw": ms, "tflops_algorithmic": tf,
             "frac_of_peak": tf / peak, "peak": peak, "peak_source": pipe,
             "update_share": (upd["total_ms"] / max(1e-9, sum(v["total_ms"] for v in prof.values()))
                              if upd else None)}
        if extra:
            d.update(extra)
        print(json.dumps(d), flush=True)

    def hermitian(Kd, n, prec_name, dt=0):
        prec = dpp.PRECISIONS[prec_name]
        need = dpp.workspace_size(0, n, dt, prec, 1)
        ws = torch.empty(need, dtype=torch.uint8, device=dev)
        keep = torch.empty(n, dtype=torch.uint8, device=dev)
        raw = torch.zeros(_lib.RESULT_BYTES, dtype=torch.uint8, device=dev)
        L = dpp.load()

        def fn(seed):
            _lib.check(L.dpp_sample_hermitian(Kd.data_ptr(), n, n, dt, prec, seed, 0, None,
                                              keep.data_ptr(), None, None, raw.data_ptr(),
                                              ws.data_ptr(), need, stream.cuda_stream))
        return fn, keep, raw

    only = {c.strip() for c in args.suite_only.split(",") if c.strip()}

    def want(c):
        return not only or c in only

    # C1: FP64, n = 512, 256 draws with seeds 0..255
    def suite_c1():
        n = 512
        Kd = torch.from_numpy(W.hermitian_kernel(n, seed=0, kind="uniform")).to(dev).contiguous()
        fn, keep, raw = hermitian(Kd, n, "fp64")
        ms, prof = timed(fn, 256)
        line("C1", {"n": n, "kernel": "Haar, lam~U(0,1)", "draws": 256}, "fp64", ms, n ** 3 / 3, prof)
        b = dpp.BatchedSampler([Kd] * 256, instance=list(range(256)))
        ms_b, prof_b = timed(lambda s: b.draw(s), 5)
        print(json.dumps({"suite": "C1-batched", "config": {"n": n, "instances": 256},
                          "precision": "fp32+f64 pivots", "samples_per_s": 256e3 / ms_b,
                          "ms_per_launch": ms_b}), flush=True)
        del b, Kd

    # C2: n = 4096 and 16384; real and complex; projection (rank n/4) and
    # Beta(1/2, 1/2) spectra; FP64 and mixed
    def suite_c2():
        for n in (4096, 16384):
            for dt, cplx in ((0, False), (1, True)):
                for kind in ("projection", "beta"):
                    Kd = W.hermitian_kernel(n, seed=0, kind=kind, complex_=cplx, device=str(dev),
                                            return_torch=True)
                    Kd = Kd.t().contiguous().t() if cplx else Kd.contiguous()
                    flops = (4 if cplx else 1) * n ** 3 / 3
                    big = n >= 16384
                    runs = (("fp64", 1 if big else 2, 1), ("bf16x6", 8 if big else 16, 2),
                            ("3xtf32", 8 if big else 16, 2))
                    for prec_name, draws, warm in runs:
                        fn, keep, raw = hermitian(Kd, n, prec_name, dt=dt)
                        ms, prof = timed(fn, draws, warm=warm)
                        res = _lib.decode_result(bytes(raw.cpu().numpy().tobytes()))
                        extra = {"last_draw_kept": res["n_kept"],
                                 "last_draw_borderline": res["n_borderline"],
                                 "last_draw_status": res["status"]}
                        if kind == "projection":
                            extra["rank"] = n // 4
                        line("C2", {"n": n, "kind": kind, "dtype": "c128" if cplx else "f64"},
                             prec_name, ms, flops, prof, extra)
                        del fn, keep, raw
                        torch.cuda.empty_cache()
                    del Kd
                    torch.cuda.empty_cache()

    # C3: uniform spanning trees of the 64 x 64 grid (n = 8064, rank 4095)
    def suite_c3():
        d = 64
        from oracle import oracle as O
        K, edges, V = W.ust_grid_kernel(d, device=str(dev))
        n = K.shape[0]
        Kd = torch.from_numpy(K).to(dev).contiguous()
        ref = -W.grid_spanning_tree_log_count(d)
        for prec_name, draws in (("bf16x6", 64), ("fp64", 2)):
            fn, keep, raw = hermitian(Kd, n, prec_name)
            ms, prof = timed(fn, draws, warm=1)
            k = keep.cpu().numpy().astype(bool)
            res = _lib.decode_result(bytes(raw.cpu().numpy().tobytes()))
            line("C3", {"grid": d, "n": n, "rank": V - 1}, prec_name, ms, n ** 3 / 3, prof,
                 {"last_draw_spanning_tree": bool(O.is_spanning_tree(edges[k], V)),
                  "last_draw_logp": res["logp"], "logp_expected": ref})
        del Kd

    # C4: real LU n = 8192, K = D^{-1} S D: FP64 and mixed (BF16x6 / 3xTF32)
    def suite_c4():
        n = 8192
        K, S = W.lu_similarity_kernel(n, seed=0, device=str(dev))
        Kd = torch.from_numpy(np.ascontiguousarray(K.T)).to(dev)  # column-major storage
        L = dpp.load()
        cfg4 = {"n": n, "kind": "D^-1 S D, lam~U(0,1), D lognormal(0,0.5)"}

        def lu_fn(prec_name, st):
            prec = dpp.PRECISIONS[prec_name]
            need = dpp.workspace_size(1, n, 0, prec, 0)
            ws = torch.empty(need, dtype=torch.uint8, device=dev)
            keep = torch.empty(n, dtype=torch.uint8, device=dev)
            raw = torch.zeros(_lib.RESULT_BYTES, dtype=torch.uint8, device=dev)

            def fn(seed):
                _lib.check(L.dpp_sample_lu(Kd.data_ptr(), n, n, 0, prec, seed, 0, None,
                                           keep.data_ptr(), None, None, raw.data_ptr(),
                                           ws.data_ptr(), need, st.cuda_stream))
            return fn, raw

        for prec_name, draws in (("fp64", 2), ("bf16x6", 32), ("3xtf32", 16)):
            fn, raw = lu_fn(prec_name, stream)
            ms, prof = timed(fn, draws, warm=1)
            res = _lib.decode_result(bytes(raw.cpu().numpy().tobytes()))
            line("C4", cfg4, prec_name, ms, 2 * n ** 3 / 3, prof,
                 {"last_draw_kept": res["n_kept"], "last_draw_borderline": res["n_borderline"],
                  "last_draw_status": res["status"]})
        # several mixed draws in flight, each launch on a quarter of the SMs
        nst = 4
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        old_cap = _lib.get_tuning(_lib.DPP_TUNE_MAX_CTAS)
        _lib.set_tuning(_lib.DPP_TUNE_MAX_CTAS, max(8, sms // nst))
        try:
            streams = [torch.cuda.Stream(dev) for _ in range(nst)]
            fns = [lu_fn("bf16x6", st)[0] for st in streams]
            draws = 32
            for i, f in enumerate(fns):
                f(10**6 + i)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for d in range(draws):
                fns[d % nst](d)
            torch.cuda.synchronize()
            ms = (time.perf_counter() - t0) * 1e3 / draws
        finally:
            _lib.set_tuning(_lib.DPP_TUNE_MAX_CTAS, old_cap)
        line("C4", dict(cfg4, streams=nst), "bf16x6", ms, 2 * n ** 3 / 3, {},
             {"timing": "wall clock over all streams, after a device synchronize"})

    # E: the elementary sampler (Algorithm 2) on projection kernels: the
    # paper's n = 5000 ranks 10 / 100 / 500, and the rank-n/4 projections of
    # the Hermitian configuration (n = 4096 and 16384)
    def suite_e():
        L = dpp.load()
        for n, k in ((5000, 10), (5000, 100), (5000, 500), (4096, 1024), (16384, 4096)):
            Kd = W.hermitian_kernel(n, seed=0, kind="projection", rank=k, device=str(dev),
                                    return_torch=True).contiguous()
            need = int(L.dpp_elementary_workspace_size(n, k))
            ws = torch.empty(need, dtype=torch.uint8, device=dev)
            sample = torch.empty(k, dtype=torch.int64, device=dev)
            raw = torch.zeros(_lib.RESULT_BYTES, dtype=torch.uint8, device=dev)

            def fn(seed, Kd=Kd, n=n, k=k, ws=ws, sample=sample, raw=raw, need=need):
                _lib.check(L.dpp_sample_elementary(Kd.data_ptr(), n, n, k, seed, 0, None,
                                                   sample.data_ptr(), None, None, raw.data_ptr(),
                                                   ws.data_ptr(), need, stream.cuda_stream))
            draws = 8 if n * k * k < 5e10 else 2
            ms, prof = timed(fn, draws, warm=1)
            res = _lib.decode_result(bytes(raw.cpu().numpy().tobytes()))
            tf = n * k * k / (ms / 1e3) / 1e12
            print(json.dumps({"suite": "E", "config": {"n": n, "rank": k, "kernel": "projection"},
                              "precision": "fp64", "samples_per_s": 1e3 / ms, "ms_per_draw": ms,
                              "tflops_algorithmic": tf, "flops_convention": "n k^2 (multiply-adds x 2 / 2)",
                              "last_draw_kept": res["n_kept"], "last_draw_status": res["status"]}),
                  flush=True)
            del Kd, ws
            torch.cuda.empty_cache()

    # A: uniform domino tilings of the Aztec diamond (complex non-Hermitian
    # Kenyon kernel, n = 4 d^2 edges), the paper's complex LU workload
    def suite_a():
        L = dpp.load()
        for d in (30, 50):
            Kd, edges, nb = W.aztec_kernel(d, device=str(dev), return_torch=True)
            n = Kd.shape[0]
            lt = W.aztec_log_tilings(d)
            cfg = {"aztec_order": d, "n": n, "kernel": "Kenyon over the Kasteleyn matrix"}
            for prec_name, draws in (("fp64", 1 if d >= 50 else 2), ("3xtf32", 8), ("bf16x6", 8)):
                prec = dpp.PRECISIONS[prec_name]
                need = dpp.workspace_size(1, n, 1, prec, 0)
                ws = torch.empty(need, dtype=torch.uint8, device=dev)
                keep = torch.empty(n, dtype=torch.uint8, device=dev)
                raw = torch.zeros(_lib.RESULT_BYTES, dtype=torch.uint8, device=dev)

                def fn(seed, ws=ws, keep=keep, raw=raw, need=need, prec=prec, n=n):
                    _lib.check(L.dpp_sample_lu(Kd.data_ptr(), n, n, 1, prec, seed, 0, None,
                                               keep.data_ptr(), None, None, raw.data_ptr(),
                                               ws.data_ptr(), need, stream.cuda_stream))
                ms, prof = timed(fn, draws, warm=1)
                res = _lib.decode_result(bytes(raw.cpu().numpy().tobytes()))
                line("A", cfg, prec_name, ms, 8 * n ** 3 / 3, prof,
                     {"last_draw_is_tiling": bool(W.is_perfect_matching(
                         edges, keep.cpu().numpy(), nb)),
                      "last_draw_logp_err": res["logp"] + lt,
                      "last_draw_borderline": res["n_borderline"],
                      "last_draw_status": res["status"]})
                del ws
                torch.cuda.empty_cache()
            # several mixed draws in flight, each launch on a quarter of the SMs
            nst = 4
            sms = torch.cuda.get_device_properties(dev).multi_processor_count
            old_cap = _lib.get_tuning(_lib.DPP_TUNE_MAX_CTAS)
            _lib.set_tuning(_lib.DPP_TUNE_MAX_CTAS, max(8, sms // nst))
            try:
                prec = dpp.PRECISIONS["3xtf32"]
                need = dpp.workspace_size(1, n, 1, prec, 0)
                streams = [torch.cuda.Stream(dev) for _ in range(nst)]
                bufs = [(torch.empty(need, dtype=torch.uint8, device=dev),
                         torch.empty(n, dtype=torch.uint8, device=dev),
                         torch.zeros(_lib.RESULT_BYTES, dtype=torch.uint8, device=dev))
                        for _ in range(nst)]

                def fs(seed, i):
                    ws, keep, raw = bufs[i]
                    _lib.check(L.dpp_sample_lu(Kd.data_ptr(), n, n, 1, prec, seed, 0, None,
                                               keep.data_ptr(), None, None, raw.data_ptr(),
                                               ws.data_ptr(), need, streams[i].cuda_stream))
                for i in range(nst):
                    fs(10**6 + i, i)
                torch.cuda.synchronize()
                draws = 16
                t0 = time.perf_counter()
                for dd in range(draws):
                    fs(dd, dd % nst)
                torch.cuda.synchronize()
                ms = (time.perf_counter() - t0) * 1e3 / draws
            finally:
                _lib.set_tuning(_lib.DPP_TUNE_MAX_CTAS, old_cap)
            line("A", dict(cfg, streams=nst), "3xtf32", ms, 8 * n ** 3 / 3, {},
                 {"timing": "wall clock over all streams, after a device synchronize"})
            del bufs, Kd
            torch.cuda.empty_cache()

    if want("A"):
        suite_a()
    if want("E"):
        suite_e()
    if want("C1"):
        suite_c1()
    if want("C2"):
        suite_c2()
    if want("C3"):
        suite_c3()
    if want("C4"):
        suite_c4()
    return 0


def run_case(args):
    """One path alone: `--warmup` then `--steps` draws of the chosen form at
    order --n (the batched forms: --batch L-ensembles), one JSON line with the
    mean time per draw. Used to profile one kernel family on a small case."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1905_00165_gb300 as dpp
    from paper_1905_00165_gb300 import _lib
    import workloads as W
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    n = args.n
    prec = "3xtf32" if args.precision == "auto" else args.precision
    steps = args.steps if args.steps is not None else 4
    if args.update_variant >= 0:
        _lib.set_tuning(_lib.DPP_TUNE_UPDATE_VARIANT, args.update_variant)
    if args.pipeline >= 0:
        _lib.set_tuning(_lib.DPP_TUNE_PANEL_PIPELINE, args.pipeline)
    if args.case in ("batched", "adjoint"):
        Ks = W.lensemble_batch_torch(args.batch, seed=0, device=str(dev))
        b = dpp.BatchedSampler(Ks)
        b.draw(10**6)
        if args.case == "batched":
            fn = b.draw
        else:
            fn = lambda s: b.logprob_backward()
    else:
        if args.case == "lu":
            K, _ = W.lu_similarity_kernel(n, seed=0, device=str(dev))
            Kd = torch.from_numpy(np.ascontiguousarray(K.T)).to(dev).t()
            fn = lambda s: dpp.sample_lu(Kd, seed=s, precision=prec)
        elif args.case == "aztec":
            # the Aztec diamond whose edge count 4 d^2 is closest to --n
            # (built on the host: under a profiler torch's device linear algebra
            # may be unavailable)
            d = max(1, int(round((n / 4) ** 0.5)))
            K, _, _ = W.aztec_kernel(d)
            Kd = torch.from_numpy(np.ascontiguousarray(K.T)).to(dev).t()
            n = Kd.shape[0]
            fn = lambda s: dpp.sample_lu(Kd, seed=s, precision=prec)
        elif args.host_inputs:
            # numpy on the host (under a profiler torch's device linear algebra may
            # be unavailable)
            K = W.hermitian_kernel(n, seed=0, kind=args.kind, complex_=args.case == "cplx")
            Kd = torch.from_numpy(np.ascontiguousarray(K.T)).to(dev).t()
            fn = lambda s: dpp.sample_hermitian(Kd, seed=s, precision=prec)
        else:
            Kd = W.hermitian_kernel(n, seed=0, kind=args.kind, complex_=args.case == "cplx",
                                    device=str(dev), return_torch=True)
            Kd = Kd.t().contiguous().t()
            fn = lambda s: dpp.sample_hermitian(Kd, seed=s, precision=prec)
    for w in range(args.warmup):
        fn(10**6 + w)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for s in range(steps):
        fn(s)
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps({"case": args.case, "n": n, "precision": prec, "steps": steps,
                      "ms_per_draw": e0.elapsed_time(e1) / steps}))
    return 0


def replica_seed_base(rank: int) -> int:
    """Philox seed of a rank's first draw: ranks draw disjoint seed ranges
    (independent replicas; no collective on the data path)."""
    return rank * 1000003


def job_time_ms(ms_local: float, ws_n: int, device=None) -> float:
    """The job's time: the maximum over ranks of each rank's timed region."""
    if ws_n <= 1:
        return ms_local
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms_local], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: int, ws_n: int, ms: float) -> float:
    """Whole-job throughput: every rank's units over the job's time."""
    return ws_n * units_per_rank / (ms / 1e3)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def oracle_full_draw(K_host, seed: int):
    """One oracle draw (Algorithm 1, LDL^H form, FP64, as it stands) on the
    full kernel with the Philox uniforms of `seed`, timed on the host cores."""
    from oracle import oracle as O
    O.build()
    n = K_host.shape[0]
    u = O.uniforms(seed, 0, n)
    t0 = time.perf_counter()
    ref = O.sample_ldl(K_host, u)
    dt = time.perf_counter() - t0
    return ref, u, dt, O.num_threads()


def err_vs_oracle(keep, pivots, res, ref, u, gap=1e-9):
    """Decision agreement, pivot and log P error of one GPU draw against the
    oracle's draw with the same uniforms. Decisions are compared up to the
    first pivot whose uniform lies within `gap` of the oracle's pivot (there
    rounding order may decide either way)."""
    import numpy as np
    n = len(ref.keep)
    piv_o = np.asarray(ref.pivots, dtype=np.float64)
    pre = np.where(ref.keep == 1, piv_o, piv_o + 1.0)
    close = np.flatnonzero(np.abs(u - pre) <= gap)
    j0 = int(close[0]) if len(close) else n
    agree = np.asarray(keep[:j0]) == ref.keep[:j0]
    first_diff = int(np.flatnonzero(~agree)[0]) if not agree.all() else None
    jp = j0 if first_diff is None else first_diff
    perr = float(np.max(np.abs(np.asarray(pivots[:jp]) - piv_o[:jp]))) if jp else 0.0
    return {"decisions_compared": j0, "decisions_equal": bool(agree.all()),
            "first_mismatch": first_diff, "borderline_draw": j0 < n,
            "logp_gpu": res["logp"], "logp_oracle": ref.logp,
            "logp_rel_err": abs(res["logp"] - ref.logp) / max(1.0, abs(ref.logp)),
            "max_pivot_abs_err": perr, "gpu_recomputed_pivots": res["n_borderline"],
            "n_kept_gpu": res["n_kept"], "n_kept_oracle": int(ref.keep.sum())}


def run_suite_cpu(args):
    """The CPU oracle at the paper-shaped configurations, each at its own size:
    the same synthetic kernels as --suite, one JSON line per configuration with
    the oracle's rate on the host cores, timed over a bounded sample (whole
    draws; for the batched L-ensembles the first instances of the batch, each
    converted L -> K and drawn). Configurations whose single draw takes more
    than a few minutes on the host are left to the headline's own measurement
    (n = 16384) or reported as skipped."""
    import numpy as np
    import workloads as W
    from oracle import oracle as O
    O.build()
    dev = None
    try:
        import torch
        if torch.cuda.is_available():
            dev = "cuda:0"
    except Exception:
        dev = None
    cores = O.num_threads()
    O.sample_ldl(np.eye(64) * 0.5, O.uniforms(10**6, 0, 64))  # starts the threads

    def emit(name, cfg, rate, unit, sample):
        print(json.dumps({"suite": name, "impl": "oracle", "config": cfg, "value": rate,
                          "unit": unit, "cores": cores, "sample": sample}), flush=True)

    def draws(fn, count, budget_s):
        times = []
        for s in range(count):
            t0 = time.perf_counter()
            fn(s)
            times.append(time.perf_counter() - t0)
            if sum(times) > budget_s:
                break
        return len(times), sum(times)

    # C1: n = 512 (Haar, lam ~ U(0, 1)), LDL^T form
    K = W.hermitian_kernel(512, seed=0, kind="uniform")
    c, t = draws(lambda s: O.sample_ldl(K, O.uniforms(s, 0, 512)), 256, 20.0)
    emit("C1", {"n": 512, "kernel": "Haar, lam~U(0,1)"}, c / t, "samples/s",
         f"{c} draws, seeds 0..{c - 1}: {t:.2f} s")
    # C2: n = 4096, real and complex, projection and Beta spectra
    for cplx in (False, True):
        for kind in ("projection", "beta"):
            K = W.hermitian_kernel(4096, seed=0, kind=kind, complex_=cplx, device=dev)
            K = np.asarray(K)
            c, t = draws(lambda s: O.sample_ldl(K, O.uniforms(s, 0, 4096)), 4, 20.0)
            emit("C2", {"n": 4096, "kind": kind, "dtype": "c128" if cplx else "f64"}, c / t,
                 "samples/s", f"{c} complete draw(s): {t:.1f} s")
    # C3: uniform spanning trees of the 64 x 64 grid (n = 8064)
    K, edges, V = W.ust_grid_kernel(64, device=dev)
    c, t = draws(lambda s: O.sample_ldl(K, O.uniforms(s, 0, K.shape[0])), 1, 0.0)
    emit("C3", {"grid": 64, "n": int(K.shape[0])}, c / t, "samples/s",
         f"{c} complete draw: {t:.1f} s")
    # C4: real LU, n = 8192, K = D^{-1} S D
    K, _ = W.lu_similarity_kernel(8192, seed=0, device=dev)
    c, t = draws(lambda s: O.sample_lu(K, O.uniforms(s, 0, 8192)), 1, 0.0)
    emit("C4", {"n": 8192, "kind": "D^-1 S D"}, c / t, "samples/s",
         f"{c} complete draw: {t:.1f} s")
    # C5: L-ensembles n ~ U{64..1024}: conversion K = L (L + I)^{-1} and a draw,
    # instance by instance over the first instances of the 4096-instance batch
    sizes = W.lensemble_sizes(4096, 0)
    t_all, done = 0.0, 0
    for i, m in enumerate(sizes):
        Lm = W.lensemble_L(int(m), 1 + i)
        t0 = time.perf_counter()
        Km = np.linalg.solve((Lm + np.eye(int(m))).T, Lm.T).T
        O.sample_ldl(0.5 * (Km + Km.T), O.uniforms(i, 0, int(m)))
        t_all += time.perf_counter() - t0
        done += 1
        if t_all > 20.0:
            break
    emit("C5", {"batch": 4096, "nmin": 64, "nmax": 1024, "instances_timed": done,
                "mean_n_timed": float(np.mean(sizes[:done]))}, done / t_all, "instances/s",
         f"the first {done} instances: numpy conversion and an oracle draw each, {t_all:.1f} s")
    # E: Algorithm 2 on projections of rank 10 / 100 / 500, n = 5000
    for k in (10, 100, 500):
        K = np.asarray(W.hermitian_kernel(5000, seed=0, kind="projection", rank=k, device=dev))
        c, t = draws(lambda s: O.sample_elementary(K, k, O.uniforms(s, 0, 5000)), 8, 10.0)
        emit("E", {"n": 5000, "rank": k}, c / t, "samples/s", f"{c} draws: {t:.2f} s")
    # A: Aztec diamond of order 30 (n = 3600), complex LU
    K, _, _ = W.aztec_kernel(30, device=dev)
    K = np.asarray(K)
    c, t = draws(lambda s: O.sample_lu(K, O.uniforms(s, 0, K.shape[0])), 2, 15.0)
    emit("A", {"aztec_order": 30, "n": int(K.shape[0])}, c / t, "samples/s",
         f"{c} complete draw(s): {t:.1f} s")
    return 0


def run_reference(args):
    """The oracle arm: the plain FP64 CPU oracle, as it stands, timed on the
    host cores on the full n x n kernel of the headline workload. Each step is
    one complete oracle draw; as many steps are run as fit in about two and a
    half minutes (at least one), and `steps` reports that number."""
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    import numpy as np
    import workloads as W
    from oracle import oracle as O
    O.build()
    n = args.n
    t_gen = time.perf_counter()
    dev = None
    try:
        import torch
        if torch.cuda.is_available():
            dev = f"cuda:{local}"
    except Exception:
        dev = None
    # the same kernel as the GPU arm (Haar factor computed on the device when
    # there is one; the oracle itself runs on the host cores only)
    K = W.hermitian_kernel(n, seed=0, kind=args.kind, device=dev)
    K = np.ascontiguousarray(K)
    t_gen = time.perf_counter() - t_gen
    # warm-up: one draw on a 1024 x 1024 block starts the OpenMP threads
    O.sample_ldl(K[:1024, :1024], O.uniforms(10**6, 0, 1024))
    requested = args.steps if args.steps is not None else 1
    budget_s = 150.0
    times = []
    t_all = time.perf_counter()
    for s in range(max(1, requested)):
        t0 = time.perf_counter()
        O.sample_ldl(K, O.uniforms(s, 0, n))
        times.append(time.perf_counter() - t0)
        elapsed = time.perf_counter() - t_all
        if elapsed + times[-1] > budget_s:
            break
    total = sum(times)
    steps = len(times)
    value = steps / total
    line = {
        "impl": "reference", "metric": f"DPP samples/s, dense Hermitian n={n}",
        "value": value, "unit": "samples/s", "n_gpus": args.gpus, "steps": steps,
        "steps_requested": requested, "warmup": 0, "ms_per_step": total / steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"hermitian_real_{args.kind}_n{n}", "n": n,
                   "kernel": f"Q diag(lam) Q^T, Haar Q (seed 0), lam~{args.kind}",
                   "seeds": "Philox seed = step index",
                   "l2_policy": "inputs larger than L2 (2 GiB FP64 K), no flush"},
        "cpu_baseline": {"value": value, "unit": "samples/s", "cores": O.num_threads(),
                         "kind": "oracle",
                         "sample": (f"{steps} complete oracle draw(s) of the n={n} kernel "
                                    f"({', '.join(f'{t:.1f}' for t in times)} s each); "
                                    "warm-up: one draw on a 1024 x 1024 block; the step count "
                                    "is capped so the arm ends in about 2.5 min")},
        "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "input_generation_s": t_gen,
    }
    print(json.dumps(line))
    return 0


def measure_dense_peaks(dev):
    """Dense TF32 and FP64 matmul throughput on this GPU (torch.matmul, CUDA
    events, best of several): the denominators for the FP64 path and a
    measured-TF32 fraction beside the nominal-ratio one."""
    import torch
    out = {}
    for name, dt, n, reps in (("tf32", torch.float32, 8192, 6), ("fp64", torch.float64, 4096, 3)):
        old = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = name == "tf32"
        try:
            a = torch.randn(n, n, device=dev, dtype=dt)
            b = torch.randn(n, n, device=dev, dtype=dt)
            c = a @ b
            torch.cuda.synchronize()
            best = None
            for _ in range(reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                c = a @ b
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                best = ms if best is None else min(best, ms)
            out[f"{name}_tflops"] = 2.0 * n ** 3 / (best / 1e3) / 1e12
            del a, b, c
        finally:
            torch.backends.cuda.matmul.allow_tf32 = old
    out["how"] = "torch.matmul: TF32 8192^3 best of 6, FP64 4096^3 best of 3 (2 n^3 flops)"
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.suite_cpu:
        return run_suite_cpu(args)
    if args.suite:
        return run_suite(args)
    if args.case:
        return run_case(args)
    import numpy as np
    import torch

    ws_n, rank, local = dist_env()
    if ws_n > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__
    __graft_entry__.build()
    import paper_1905_00165_gb300 as dpp
    from paper_1905_00165_gb300 import _lib
    import workloads as W

    L = dpp.load()
    n = args.n
    prec_name = args.precision
    cache = os.path.join(ROOT, "paper_1905_00165_gb300", "tune_gb300.json")
    if os.path.exists(cache):
        _lib.tune_load(cache)
    if prec_name == "auto":
        # the operand split (3xTF32 or BF16x6, both FP32-accurate) whose tuned
        # configuration drew faster on this GPU; 3xTF32 without a tuning entry
        best = None
        for cand in ("3xtf32", "bf16x6"):
            e = _lib.tune_lookup(0, n, 0, dpp.PRECISIONS[cand])
            if e is not None and (best is None or e["samples_per_s"] > best[1]):
                best = (cand, e["samples_per_s"])
        prec_name = best[0] if best else "3xtf32"
    prec = dpp.PRECISIONS[prec_name]
    _lib.set_tuning(_lib.DPP_TUNE_UPDATE_KERNEL, 0 if args.update == "tc" else 1)
    steps = args.steps if args.steps is not None else (40 if prec_name != "fp64" else 4)
    warmup = max(args.warmup, 3)

    # ---- inputs (resident before timing) --------------------------------
    t_gen = time.perf_counter()
    if args.gen == "gpu":
        Kd = W.hermitian_kernel(n, seed=0, kind=args.kind, device=str(dev), return_torch=True)
    else:
        Kd = torch.from_numpy(W.hermitian_kernel(n, seed=0, kind=args.kind)).to(dev)
    Kd = Kd.contiguous()  # symmetric: row-major storage == column-major K
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    need = dpp.workspace_size(0, n, 0, prec, 1)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    tuning = None
    if args.streams > 0:
        # an explicit stream count: the knobs decide, not the tuning table
        nst = args.streams
        _lib.set_tuning(_lib.DPP_TUNE_USE_CACHE, 0)
        if nst > 1:
            _lib.set_tuning(_lib.DPP_TUNE_MAX_CTAS, max(8, sms // nst))
    else:
        # the autotuner's entry for this GPU and key (the committed table, or a
        # tuning run on this kernel now); the library applies its outer block,
        # panel pipeline and CTA cap to every draw below
        tuning = _lib.tune_lookup(0, n, 0, prec)
        source = "tuning table"
        if tuning is None:
            tuning = dpp.autotune(Kd, hermitian=True, precision=prec_name, max_streams=8, draws=16)
            source = "autotuned in this run"
        tuning["source"] = source
        nst = int(tuning["streams"])
    wsbs = [torch.empty(need, dtype=torch.uint8, device=dev) for _ in range(nst)]
    keeps = [torch.empty(n, dtype=torch.uint8, device=dev) for _ in range(nst)]
    pivs = [torch.empty(n, dtype=torch.float64, device=dev) for _ in range(nst)]
    raws = [torch.zeros(_lib.RESULT_BYTES, dtype=torch.uint8, device=dev) for _ in range(nst)]
    wsb, keep, piv, raw = wsbs[0], keeps[0], pivs[0], raws[0]
    stream = torch.cuda.current_stream(dev)
    side = [stream] if nst == 1 else [torch.cuda.Stream(dev) for _ in range(nst)]

    def draw(seed, Kptr=None, si=None):
        j = 0 if si is None else si
        stv = stream if si is None else side[j]
        st = L.dpp_sample_hermitian(Kptr or Kd.data_ptr(), n, n, 0, prec, seed, 0, None,
                                    keeps[j].data_ptr(), None, pivs[j].data_ptr(),
                                    raws[j].data_ptr(), wsbs[j].data_ptr(), need,
                                    stv.cuda_stream)
        _lib.check(st)

    base_seed = replica_seed_base(rank)
    for w in range(warmup):
        draw(base_seed + 900000 + w)
    torch.cuda.synchronize()

    # draws are dealt round-robin to the streams; a last, partial round of m
    # draws takes sms // m CTAs per launch instead of the tuned share, so that
    # its launches still cover the GPU (dpp.draw_schedule)
    if tuning is not None:
        cap0 = int(tuning["max_ctas"])
    else:
        cap0 = int(_lib.get_tuning(_lib.DPP_TUNE_MAX_CTAS))

    def run_schedule(count, one):
        plan = dpp.draw_schedule(count, nst, sms, cap0)
        s = 0
        while s < count:
            cap, e = plan[s][1], s
            while e < count and plan[e][1] == cap:
                e += 1
            if cap == cap0:
                for t in range(s, e):
                    one(t, plan[t][0])
            else:
                with dpp.tuning_knobs(entry=tuning, max_ctas=cap):
                    for t in range(s, e):
                        one(t, plan[t][0])
            s = e
        return plan

    def describe(plan):
        caps = [c for _, c in plan]
        tail = [c for c in caps if c != cap0]
        out = f"{len(caps) - len(tail)} draws at {cap0} CTAs per launch"
        if tail:
            out += f", last {len(tail)} at {tail[0]}"
        return out

    # ---- timed region ----------------------------------------------------
    if ws_n > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    _lib.profile_start()
    l0 = _lib.launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for sv in side:
        if sv is not stream:
            sv.wait_event(ev0)
    plan = run_schedule(steps, lambda s, j: draw(base_seed + s, si=j))
    for sv in side:
        if sv is not stream:
            done = torch.cuda.Event()
            done.record(sv)
            stream.wait_event(done)
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = _lib.launch_count() - l0
    prof = _lib.profile_stop()
    clk = clocks.stop()
    ms = job_time_ms(ev0.elapsed_time(ev1), ws_n, dev)
    if ws_n > 1:
        torch.distributed.barrier()
    res = _lib.decode_result(bytes(raw.cpu().numpy().tobytes()))
    value = job_rate(steps, ws_n, ms)
    algo_flops = n ** 3 / 3.0
    # the last timed draw on the first stream, kept for the oracle comparison
    s_par = max(s for s in range(steps) if s % nst == 0)
    seed_par = base_seed + s_par
    par_keep = keeps[0].cpu().numpy().copy()
    par_piv = pivs[0].cpu().numpy().copy()
    par_res = res
    dense = measure_dense_peaks(dev)

    # ---- roofline of the dominant kernel -----------------------------------
    peaks = measured_peaks()
    dom = max((k for k in prof if k != "panel_decide_solve" or len(prof) == 1),
              key=lambda k: prof[k]["total_ms"], default=None)
    roof = None
    if dom is not None:
        st = prof[dom]
        avg_ms = st["total_ms"] / max(1, st["launches"])
        per_launch_flops = st["flops"] / max(1, st["launches"])
        if dom == "update_fp64":
            ach = per_launch_flops / (avg_ms / 1e3) / 1e12
            f64 = dense["fp64_tflops"]
            roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": f64,
                    "unit": "TFLOP/s", "frac": ach / f64, "traffic": None,
                    "peak_source": "FP64 torch.matmul measured in this run",
                    "frac_of_nominal_1.25": ach / FP64_NOMINAL_TFLOPS}
        elif dom == "update_tc" and prec_name == "3xtf32":
            tf32 = peaks.get("bf16_tflops", 1888.3) * TF32_PER_BF16
            ach = per_launch_flops / (avg_ms / 1e3) / 1e12
            roof = {"kernel": dom, "bound": "tensor", "achieved": ach, "peak": tf32 / 3.0,
                    "unit": "TFLOP/s", "frac": ach / (tf32 / 3.0),
                    "traffic": tc_traffic_per_launch(n, "3xtf32", int(tuning["outer_block"]) if tuning else 256),
                    "traffic_source": "ncu one launch at n = 8192, scaled by m^2 (profiles/)",
                    "executed_tensor_frac": 3.0 * ach / tf32,
                    "peak_source": "measured bf16 x nominal tf32/bf16 (2.25:1.1), / 3 products",
                    "measured_tf32_tflops": dense["tf32_tflops"],
                    "frac_of_measured_tf32_div3": ach / (dense["tf32_tflops"] / 3.0)}
        elif dom == "update_tc":
            bf16 = peaks.get("bf16_tflops", 1888.3)
            ach = per_launch_flops / (avg_ms / 1e3) / 1e12
            roof = {"kernel": dom, "bound": "tensor", "achieved": ach, "peak": bf16 / 6.0,
                    "unit": "TFLOP/s", "frac": ach / (bf16 / 6.0),
                    "traffic": tc_traffic_per_launch(n, "bf16x6", int(tuning["outer_block"]) if tuning else 256),
                    "traffic_source": "ncu one launch at n = 8192, scaled by m^2 (profiles/)",
                    "executed_tensor_frac": 6.0 * ach / bf16,
                    "peak_source": "MEASURED_PEAKS bf16_tflops (burst), / 6 products"}
        else:
            gbs = st["bytes"] / max(1, st["launches"]) / (avg_ms / 1e3) / 1e9
            hbm = peaks.get("hbm_gbs", 6787.6)
            roof = {"kernel": dom, "bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                    "frac": gbs / hbm, "traffic": None, "peak_source": "MEASURED_PEAKS hbm_gbs"}
        roof["launches_per_step"] = st["launches"] / steps
        roof["avg_launch_ms"] = avg_ms
        cap = (int(tuning["max_ctas"]) if tuning is not None
               else (max(8, sms // nst) if nst > 1 else 0))
        if cap and cap < sms:
            # each launch holds at most `cap` CTAs (one per SM), and the
            # streams' launches overlap: the fraction of that SM share
            share = cap / sms
            roof["ctas_per_launch_share"] = share
            roof["frac_of_sm_share"] = roof["frac"] / share
    kernels = {k: {"launches": v["launches"], "total_ms": round(v["total_ms"], 3),
                   "share": v["total_ms"] / max(1e-9, sum(x["total_ms"] for x in prof.values()))}
               for k, v in prof.items()}
    # The same kernel on all SMs: inside the timed region each launch holds one
    # stream's CTA share and overlaps the other streams' launches. One more draw
    # alone after it, with the table's settings but no CTA cap, gives the
    # per-launch rate of the full GPU (a side measurement, outside the timed
    # region; `roofline` itself stays the timed region's).
    if roof is not None and dom == "update_tc" and rank == 0 and tuning is not None:
        keys = (_lib.DPP_TUNE_USE_CACHE, _lib.DPP_TUNE_MAX_CTAS, _lib.DPP_TUNE_OUTER_BLOCK,
                _lib.DPP_TUNE_PANEL_PIPELINE, _lib.DPP_TUNE_UPDATE_VARIANT)
        saved = {k: _lib.get_tuning(k) for k in keys}
        try:
            _lib.set_tuning(_lib.DPP_TUNE_USE_CACHE, 0)
            _lib.set_tuning(_lib.DPP_TUNE_MAX_CTAS, 0)
            _lib.set_tuning(_lib.DPP_TUNE_OUTER_BLOCK, int(tuning["outer_block"]))
            _lib.set_tuning(_lib.DPP_TUNE_PANEL_PIPELINE, int(tuning["panel_pipeline"]))
            _lib.set_tuning(_lib.DPP_TUNE_UPDATE_VARIANT, int(tuning["update_variant"]))
            draw(base_seed + 800000)
            torch.cuda.synchronize()
            _lib.profile_start()
            draw(base_seed + 800001)
            torch.cuda.synchronize()
            p1 = _lib.profile_stop().get("update_tc")
        finally:
            for k, v in saved.items():
                _lib.set_tuning(k, v)
        if p1 and p1["launches"]:
            a1 = p1["flops"] / p1["launches"] / (p1["total_ms"] / p1["launches"] / 1e3) / 1e12
            roof["full_gpu"] = {"achieved": a1, "frac": a1 / roof["peak"],
                                "avg_launch_ms": p1["total_ms"] / p1["launches"],
                                "how": "one draw alone after the timed region, launches on all SMs"}

    # ---- FP64 GPU path at the same n (for the mixed/FP64 ratio) -------------
    fp64_ref = None
    if prec_name != "fp64" and not args.no_fp64_ref and rank == 0:
        need64 = dpp.workspace_size(0, n, 0, 0, 1)
        ws64 = torch.empty(need64, dtype=torch.uint8, device=dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = L.dpp_sample_hermitian(Kd.data_ptr(), n, n, 0, 0, base_seed, 0, None, keep.data_ptr(),
                                    None, piv.data_ptr(), raw.data_ptr(), ws64.data_ptr(), need64,
                                    stream.cuda_stream)
        _lib.check(st)
        e1.record(stream)
        torch.cuda.synchronize()
        t64 = e0.elapsed_time(e1) / 1e3
        fp64_ref = {"samples_per_s": 1.0 / t64, "tflops": algo_flops / t64 / 1e12,
                    "frac_of_measured_fp64": algo_flops / t64 / 1e12 / dense["fp64_tflops"],
                    "draws": 1, "speedup_mixed_over_fp64": value / ws_n * t64}
        del ws64

    # ---- end to end through the public API with host buffers ----------------
    e2e = None
    if not args.no_e2e:
        # each step: K from pinned host memory to the device, one draw through
        # the C ABI, keep mask and result back to pinned host memory. Steps
        # are dealt to the same streams as above; the copies run on their own
        # stream into a ring of nst + 1 device buffers, events order reuse.
        # host and device copies with the same strides, so that each H2D is a
        # straight memcpy of the storage; it is cut into two ranges on two copy
        # streams (two copy engines)
        Kh = torch.empty_strided(Kd.shape, Kd.stride(), dtype=torch.float64, pin_memory=True)
        Kh.copy_(Kd)
        nbuf = args.e2e_buffers if args.e2e_buffers > 0 else nst + 2
        Kin = [torch.empty_strided(Kd.shape, Kd.stride(), dtype=torch.float64, device=dev)
               for _ in range(nbuf)]

        def flat(t):  # the dense storage, in memory order
            return (t.t() if t.stride(0) == 1 and t.stride(1) != 1 else t).reshape(-1)
        Khf = flat(Kh)
        Kinf = [flat(k) for k in Kin]
        assert Khf.data_ptr() == Kh.data_ptr() and all(
            f.data_ptr() == k.data_ptr() for f, k in zip(Kinf, Kin))
        ncopy = 2
        cuts = [n * n * i // ncopy for i in range(ncopy + 1)]
        # the host link alone: one K-sized pinned H2D copy, timed twice (best)
        h2d_ms = []
        for _ in range(2):
            b0 = torch.cuda.Event(enable_timing=True)
            b1 = torch.cuda.Event(enable_timing=True)
            b0.record(stream)
            with torch.cuda.stream(stream):
                Kinf[0].copy_(Khf, non_blocking=True)
            b1.record(stream)
            torch.cuda.synchronize()
            h2d_ms.append(b0.elapsed_time(b1))
        h2d_gbs = 8 * n * n / (min(h2d_ms) / 1e3) / 1e9
        keep_h = [torch.empty(n, dtype=torch.uint8, pin_memory=True) for _ in range(nst)]
        raw_h = [torch.empty(_lib.RESULT_BYTES, dtype=torch.uint8, pin_memory=True)
                 for _ in range(nst)]
        # as many steps as the timed region, so that the pipeline of copies and
        # draws in flight fills as it does there
        e2e_steps = steps
        copy_streams = [torch.cuda.Stream(dev) for _ in range(ncopy)]
        copied = [[torch.cuda.Event() for _ in range(ncopy)] for _ in range(nbuf)]
        consumed = [torch.cuda.Event() for _ in range(nbuf)]
        torch.cuda.synchronize()
        if ws_n > 1:
            torch.distributed.barrier()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for cs in copy_streams:
            cs.wait_event(a0)
        for sv in side:
            if sv is not stream:
                sv.wait_event(a0)

        def stage(s):
            b = s % nbuf
            for c, cs in enumerate(copy_streams):
                with torch.cuda.stream(cs):
                    if s >= nbuf:
                        cs.wait_event(consumed[b])
                    Kinf[b][cuts[c]:cuts[c + 1]].copy_(Khf[cuts[c]:cuts[c + 1]],
                                                        non_blocking=True)
                    copied[b][c].record(cs)

        for s0 in range(min(nbuf, e2e_steps)):
            stage(s0)
        def e2e_step(s, j):
            b = s % nbuf
            sv = side[j]
            for ev in copied[b]:
                sv.wait_event(ev)
            draw(base_seed + 500000 + s, Kptr=Kin[b].data_ptr(), si=j)
            consumed[b].record(sv)
            with torch.cuda.stream(sv):
                keep_h[j].copy_(keeps[j], non_blocking=True)
                raw_h[j].copy_(raws[j], non_blocking=True)
            if s + nbuf < e2e_steps:
                stage(s + nbuf)

        run_schedule(e2e_steps, e2e_step)
        for sv in side:
            if sv is not stream:
                done = torch.cuda.Event()
                done.record(sv)
                stream.wait_event(done)
        a1.record(stream)
        torch.cuda.synchronize()
        e_ms = job_time_ms(a0.elapsed_time(a1), ws_n, dev)
        e2e = {"value": job_rate(e2e_steps, ws_n, e_ms), "unit": "samples/s",
               "h2d_bytes_per_step": 8 * n * n, "d2h_bytes_per_step": n + _lib.RESULT_BYTES,
               "steps": e2e_steps,
               "h2d_alone_gbs": h2d_gbs,
               "h2d_bound_samples_per_s": h2d_gbs * 1e9 / (8 * n * n),
               "overlap": (f"H2D (pinned host copy with the device buffer's layout, "
                           f"{ncopy} ranges on {ncopy} copy streams) into {nbuf} rotating "
                           f"buffers; draws on {nst} streams")}
        del Kh, Kin

    batched = None
    if rank == 0 and not args.no_batched:
        del wsb
        torch.cuda.empty_cache()
        batched = bench_batched(dpp, _lib, dev, args.batch, draws=5)

    cpu = None
    err = None
    if rank == 0 and ws_n == 1 and not args.no_cpu:
        # one complete oracle draw of the same kernel with the uniforms of the
        # kept timed draw: the CPU baseline and that draw's error in one
        ref, u_par, t_or, cores = oracle_full_draw(Kd.cpu().numpy(), seed_par)
        cpu = {"value": 1.0 / t_or, "unit": "samples/s", "cores": cores, "kind": "oracle",
               "sample": (f"one complete oracle draw of the n={n} kernel (seed {seed_par}) "
                          f"on the host cores: {t_or:.1f} s")}
        err = dict(err_vs_oracle(par_keep, par_piv, par_res, ref, u_par), seed=seed_par,
                   draw=f"timed draw {s_par} (stream 0) of the bench configuration")
        del ref

    if rank == 0:
        line = {
            "metric": f"DPP samples/s, dense Hermitian n={n}",
            "value": value, "unit": "samples/s", "n_gpus": ws_n, "steps": steps,
            "warmup": warmup, "ms_per_step": ms / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec_name == "fp64" else f"{prec_name}+f64",
            "data": "synthetic",
            "config": {"workload": f"hermitian_real_{args.kind}_n{n}", "n": n,
                       "precision": prec_name,
                       "update_kernel": args.update if prec_name != "fp64" else "simt_fp64",
                       "kernel": f"Q diag(lam) Q^T, Haar Q (seed 0), lam~{args.kind}",
                       "seeds": f"Philox seed = step index (+ rank offset)",
                       "l2_policy": "inputs larger than L2 (2 GiB FP64 K), no flush",
                       "parallelism": f"replicas x{ws_n}",
                       "streams": nst, "schedule": describe(plan), "tuning": tuning},
            "tflops_algorithmic": value * algo_flops / 1e12,
            "roofline": roof,
            "err_vs_oracle": err,
            "kernels": kernels,
            "fp64_gpu_path": fp64_ref,
            "dense_peaks_measured": dense,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "batched": batched,
            "gpu_launches": launches,
            "clocks": clk,
            "last_draw": {"status": res["status"], "n_kept": res["n_kept"],
                          "n_borderline": res["n_borderline"], "logp": res["logp"]},
            "input_generation_s": t_gen,
        }
        print(json.dumps(line))
    if ws_n > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
