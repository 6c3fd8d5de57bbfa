#!/usr/bin/env python
"""Encrypted SpMV benchmark (one JSON line on stdout).

Workload (default): the 27-point stencil on a 16 x 32 x 32 grid (16,384 rows,
406,456 non-zeros), values uniform in [-1, 1] in fixed point (2^15), under
BGV with N = 2^15, 8 ciphertext primes + 2 special primes, dnum = 4.  One
step is one full encrypted SpMV: the cloud lines of Algorithm 1 (HE-Mult with
relinearisation per chunk) and Aggregation (Algorithm 4), from device-resident
encrypted inputs to the device-resident encrypted result.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs its own independent SpMV instance (weak
scaling, no collective on the data path); rank 0 prints the line.
--impl reference times the CPU oracle on the host cores instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "encrypted SpMV/s and nnz/s at N=2^15, batched vs plain; p50/p99 latency"
CONFIGS = {
    "c3": "27-point stencil 16x32x32 (16384 rows, 406456 nnz), fixed point 2^15; "
          "BGV N=2^15, 8+2 primes of 50 bits, dnum 4, t=1099512938497",
    "c1": "512x512, 2621 nnz uniform, integers [-15,15]; BGV N=2^12, 3+1 primes, dnum 3, t=65537",
    "c2": "4096x4096, 16777 nnz, power-law column counts, integers [-127,127]; "
          "BGV N=2^14, 5+1 primes, dnum 5, t=17006593",
    "c4": "64 square matrices, n log-U[256,8192], density log-U[5e-4,2e-2], integers [-15,15]; "
          "BGV N=2^14, 5+1 primes, dnum 5, t=1146881; batched evaluation vs plain calls",
}
# ALU roofline of a 64-bit modular product: a Shoup product needs 10 32x32-bit
# partial products (3 + 3 for two low halves, 4 for a high half), all on the
# heavy multiply pipe, which completes 32 of them per clock per SM (half of the
# SM's 128 FP32 lanes); times the SM count (device properties) and the maximum
# SM clock (MEASURED_PEAKS.json).  (A microbenchmark of independent Shoup
# chains reaches 1.01 T/s with that pipe 94% busy.)
IMAD_PER_SM_CLK = 32
IMAD_PER_MULMOD = 10
FALLBACK_SM_MAX_MHZ = 2070.0   # the GB300's maximum SM clock, when no measured file exists
KS_SOURCES = ["paper_2603_04742_gb300/csrc/ks.cu", "paper_2603_04742_gb300/csrc/ntt_core.cuh",
              "paper_2603_04742_gb300/csrc/modarith.cuh", "paper_2603_04742_gb300/csrc/persist.h"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c3", choices=sorted(CONFIGS) + ["c5", "sweep", "rot"])
    ap.add_argument("--persistent", action="store_true",
                    help="one persistent launch per evaluation (no autotuning)")
    ap.add_argument("--tuning", default=None,
                    help="a fixed schedule instead of autotuning (c3..c5 and rot): mult_batch,rot_batch,ntt_split,rows_tma,"
                         "persistent,streams (e.g. 14,0,0,0,0,2)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="c3: skip the batched, serving, rotation and boundary-call blocks")
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="serving block of the default run: Poisson requests")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default schedule")
    ap.add_argument("--scheme", default="bgv", choices=["bgv", "bfv", "ckks"],
                    help="bgv (default), bfv (the paper's scheme, exact HE-Mult) or ckks "
                         "(float64 values at scale 2^40, no fixed point)")
    ap.add_argument("--instances", type=int, default=64, help="c4: SpMVs per batched step")
    ap.add_argument("--pool", type=int, default=32, help="c5: distinct instances")
    ap.add_argument("--requests", type=int, default=10000, help="c5: Poisson requests")
    ap.add_argument("--sat-requests", type=int, default=1000, help="c5: closed-loop requests")
    ap.add_argument("--serial-requests", type=int, default=1000, help="c5: serial-server requests")
    ap.add_argument("--slots", type=int, default=3, help="c5: concurrent evaluations")
    ap.add_argument("--max-batch", type=int, default=16, help="c5: requests per evaluation")
    return ap.parse_args()


def load_workload(name):
    from paper_2603_04742_gb300 import synth
    A, x = synth.workload(name)
    if A.vals.dtype.kind == "f":
        A.vals = synth.quantize(A.vals)
        x = synth.quantize(x)
    return A, x, synth.RING[name]


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in KS_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def measured_traffic(kernel, config):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or
    None when the kernel sources changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "kernel_traffic_%s.md" % config)
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    src = [ln for ln in lines if ln.startswith("source hash:")]
    if not src or src[0].split(":", 1)[1].strip() != kernel_source_hash():
        return None
    for ln in lines:
        cells = [c.strip() for c in ln.strip().strip("|").split("|")]
        if len(cells) >= 4 and cells[0] == kernel:
            try:
                return float(cells[1]) + float(cells[2])
            except ValueError:
                return None
    return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0}, "fallback"


def alu_peak():
    """(mulmod/s, description): SMs x heavy-IMAD/clk x max SM clock / IMADs
    per Shoup product."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    peaks, kind = measured_peaks()
    mhz = peaks.get("sm_max_mhz")
    src = "%s sm_max_mhz" % kind
    if not mhz:
        mhz, src = FALLBACK_SM_MAX_MHZ, "nominal maximum clock"
    rate = sms * IMAD_PER_SM_CLK * float(mhz) * 1e6 / IMAD_PER_MULMOD
    return rate, ("derived: %d SMs (device properties) x %d heavy-IMAD/clk x %.0f MHz (%s) / %d per "
                  "Shoup mulmod" % (sms, IMAD_PER_SM_CLK, float(mhz), src, IMAD_PER_MULMOD))


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.device = device
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
            return
        # the timed region starts once the sampler has written its first row
        t0 = time.time()
        while time.time() - t0 < 5 and self.p.poll() is None:
            if os.path.getsize(self.f.name) > 0:
                break
            time.sleep(0.02)

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# a 64 x 64 -> 128-bit word product of the BFV multi-word arithmetic takes 4
# of the 10 heavy-pipe partial products of a Shoup product
WORD_PRODUCT_MULMODS = 0.4


def bfv_basis(logn, L, t, q):
    """Auxiliary basis size and multi-word widths of the BFV HE-Mult (the
    library's rule: B > 2 t N Q in primes of q's size; words for Q and B
    with room for a sign and sums)."""
    import math
    lq = sum(math.log2(v) for v in q[:L])
    need = math.log2(t) + logn + 2 + lq
    lb = math.log2(q[-1])
    nB = int(math.ceil(need / lb))
    wq = int(math.ceil((lq + 2) / 64)) + 1
    wb = int(math.ceil((nB * lb + 2) / 64)) + 1
    return nB, wq, wb


def kernel_model(name, ring, n_ks, n_chunks, n_parts, n_rot, bfv=None):
    """Algorithmic work of one step in kernel `name`: (mulmods, bytes).

    n_ks = key switches per step (relinearisations + elementary rotations).
    Mulmods count every modular product (NTT butterflies, base conversions,
    key products, masks); bytes count one read of every input and one write
    of every output of the kernel (a key is read once per step).  bfv =
    (nB, wq, wb) adds the BFV HE-Mult kernels: its NTTs, the exact extension
    and scale-and-round (Shoup products, plus word products of the
    multi-word sums at WORD_PRODUCT_MULMODS each)."""
    logn, L, K, dnum = ring[:4]
    N = 1 << logn
    LK = L + K
    alpha = -(-L // dnum)
    n1 = logn // 2 if logn > 10 else 0
    n2 = logn - n1
    w = 8 * N  # bytes per limb
    h = N // 2
    ext = dnum * LK - L          # limbs raised by ModUp (each digit's own limbs excluded)
    m = {
        # fused key switch (one launch of each per step and batch group)
        "k_ks_intt_rows": (n_ks * (L + 2 * K) * h * n2, n_ks * (L + 2 * K) * 2 * w),
        # ModUp: the digit's inverse column pass, base conversion, forward column pass
        "k_ks_modup_cols": (n_ks * (L * (h * n1 + N) + ext * (h * n1 + alpha * N)),
                            n_ks * (L + ext) * w),
        "k_ks_rows_fwd": (n_ks * ext * h * n2, n_ks * ext * 2 * w),
        # key product with the output addend (times P) on the Q primes
        "k_ks_mac": (n_ks * 2 * (dnum * LK + L) * N,
                     n_ks * (ext + L + 2 * L + 2 * LK) * w + 2 * dnum * LK * w),
        # ModDown: the P limbs' inverse column pass, conversion, forward column pass
        "k_ks_moddown_cols": (n_ks * 2 * (K * (h * n1 + N) + L * (h * n1 + K * N)),
                              n_ks * 2 * (K + L) * w),
        "k_ks_rows_final": (n_ks * 2 * L * (h * n2 + N), n_ks * 2 * L * 3 * w),
        # ciphertext arithmetic
        "k_tensor": (n_chunks * 4 * L * N, n_chunks * 7 * L * w),
        "k_mask_acc": (n_chunks * 2 * L * N, n_chunks * 2 * L * w + n_parts * 2 * L * w),
        "k_copy_strided": (0, n_ks * 2 * L * w),
        "k_permute": (0, n_ks * 2 * 2 * L * w),
        "k_add": (0, n_rot * 3 * 2 * L * w),
        # unfused key switch (small rings)
        "k_modup": (n_ks * dnum * alpha * (1 + LK - alpha) * N,
                    n_ks * (L + dnum * (LK - alpha)) * w),
        "k_inner": (n_ks * 2 * dnum * LK * N, n_ks * (dnum * LK + 2 * LK) * w + 2 * dnum * LK * w),
        "k_moddown_delta": (n_ks * 2 * (K + K * L + L) * N, n_ks * 2 * (K + L) * w),
        "k_moddown_final": (n_ks * 2 * L * N, n_ks * 2 * L * 3 * w),
    }
    if bfv:
        nB, wq, wb = bfv
        n = n_chunks
        wp = WORD_PRODUCT_MULMODS
        inv = 4 * n * L + 3 * n * (L + nB)     # limb transforms: a, b over Q; d over Q u B
        fwd = 4 * n * nB + 3 * n * L           # a, b over B; the result over Q
        m.update({
            "k_intt_rows": (inv * h * n2, inv * 2 * w),
            "k_intt_cols": (inv * (h * n1 + N), inv * 2 * w),
            "k_fntt_rows": (fwd * h * n2, fwd * 2 * w),
            "k_fntt_cols": (fwd * h * n1, fwd * 2 * w),
            "k_bfv_extend": (4 * n * N * (L + nB * (wq + 1) + wp * L * wq),
                             4 * n * (L + nB) * w),
            "k_bfv_tensor": (n * (L + nB) * N * 4, n * (4 * L + 4 * nB + 3 * (L + nB)) * w),
            "k_bfv_scale": (3 * n * N * (2 * L + nB * (3 + wq + 1) + L * (wb + 1)
                                         + wp * (L * wq + nB * wb)),
                            3 * n * (2 * L + nB) * w),
        })
    if name == "k_ks_persist":   # the whole evaluation in one launch
        parts = ["k_ks_intt_rows", "k_ks_modup_cols", "k_ks_rows_fwd", "k_ks_mac", "k_ks_moddown_cols",
                 "k_ks_rows_final", "k_mask_acc"]
        return (sum(m[k][0] for k in parts), sum(m[k][1] for k in parts))
    return m.get(name, (0, 0))


class OracleSample:
    """The oracle's cloud evaluation (HE-Mult + relinearisation, totalSum,
    mask, accumulate) on the first `sample_chunks` chunks of partition 0;
    keys and ciphertexts are prepared once, outside the timing."""

    def __init__(self, A, x, ring, sample_chunks, seed=1):
        from oracle import spmv as S
        from oracle.bgv import Oracle
        from oracle.params import Params
        logn, L, K, dnum, t = ring
        self.S = S
        self.orc = Oracle(Params(log2n=logn, L=L, K=K, dnum=dnum, t=t))
        plan = S.SpmvPlan(A.rows, A.cols, A.rowptr, A.colidx, A.vals, self.orc.p.slots)
        self.n_total = len(plan.chunks)
        self.chunks = plan.parts[0].chunks[:sample_chunks]
        gels = set()
        for ch in self.chunks:
            for k in S.rotation_steps(ch.c, ch.h):
                gels.update(self.orc.rotation_elements(k))
        self.orc.keygen(seed, sorted(gels))
        reorg = S.reorg_vector(x, self.chunks)
        self.ca = [self.orc.encrypt(self.orc.encode(ch.values), 2, k)
                   for k, ch in enumerate(self.chunks)]
        self.cx = [self.orc.encrypt(self.orc.encode(v), 3, k) for k, v in enumerate(reorg)]

    def run(self):
        t0 = time.perf_counter()
        self.S.cloud(self.orc, self.chunks, self.ca, self.cx)
        return time.perf_counter() - t0


def _allcores_worker(w, nw, A, x, ring, seeds, inbox, out):
    """Worker w of nw: the oracle's cloud evaluation (HE-Mult with
    relinearisation, totalSum, mask product, partial sum per partition) of
    chunks w, w + nw, ...; keys and encryptions are made first, then each
    token from `inbox` starts one evaluation (None ends the worker), whose
    end time (the system's monotonic clock) is reported with the partial
    sums."""
    from oracle import spmv as S
    from oracle.bgv import Oracle
    from oracle.params import Params
    logn, L, K, dnum, t = ring
    orc = Oracle(Params(log2n=logn, L=L, K=K, dnum=dnum, t=t))
    plan = S.SpmvPlan(A.rows, A.cols, A.rowptr, A.colidx, A.vals, orc.p.slots)
    chunks = plan.chunks
    part_of = [p for p, part in enumerate(plan.parts) for _ in part.chunks]
    sel = [i for i in range(len(chunks)) if i % nw == w]
    gels = set()
    for i in sel:
        for k in S.rotation_steps(chunks[i].c, chunks[i].h):
            gels.update(orc.rotation_elements(k))
    orc.keygen(seeds[0], sorted(gels))
    reorg = S.reorg_vector(x, chunks)   # the same encryptions as encrypt_matrix / encrypt_vector
    work = [(part_of[i], chunks[i], orc.encrypt(orc.encode(chunks[i].values), seeds[1], i),
             orc.encrypt(orc.encode(reorg[i]), seeds[2], i)) for i in sel]
    out.put(("ready", w, None))
    while True:
        tok = inbox.get()
        if tok is None:
            return
        sums = {}
        for p, ch, a, b in work:   # Algorithm 1 (HE-Mult), Algorithm 4 (totalSum, mask)
            v = S.total_sum(orc, orc.mult(a, b), ch.h, ch.c)
            v = orc.cmult(v, S.mask_ntt(orc, ch.h))
            sums[p] = orc.add(sums[p], v) if p in sums else v
        out.put(("done", time.perf_counter(), {p: v.tobytes() for p, v in sums.items()} if tok else None))


def _collect(out, procs, n, kind, limit_s):
    got = []
    t0 = time.time()
    while len(got) < n:
        try:
            m = out.get(timeout=1.0)
        except Exception:
            if not all(p.is_alive() or p.exitcode == 0 for p in procs) or time.time() - t0 > limit_s:
                raise RuntimeError("all-core oracle worker failed")
            continue
        if m[0] == kind:
            got.append(m)
    return got


def oracle_allcores(A, x, ring, seeds, cores=None, steps=1, limit_s=900, budget_s=None):
    """The oracle's cloud evaluation of a whole SpMV on every host core:
    one spawned process per core, chunks dealt round robin, partial sums
    added per partition.  Runs `steps` evaluations (fewer once `budget_s`
    seconds of them have run).  Returns (seconds of each evaluation, from
    its start signal to its last worker's end; cores; result ciphertexts
    [n_parts][2][L][N] of the last evaluation)."""
    import multiprocessing as mp
    from oracle import spmv as S
    from oracle.bgv import Oracle
    from oracle.params import Params
    logn, L, K, dnum, t = ring
    cores = cores or os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    inboxes = [ctx.Queue() for _ in range(cores)]
    procs = [ctx.Process(target=_allcores_worker, args=(w, cores, A, x, ring, seeds, inboxes[w], out),
                         daemon=True) for w in range(cores)]
    times, done = [], None
    try:
        for p in procs:
            p.start()
        _collect(out, procs, cores, "ready", limit_s)
        for k in range(steps):
            last = k + 1 == steps or (budget_s is not None and sum(times) > budget_s)
            t0 = time.perf_counter()
            for q in inboxes:
                q.put(bool(last))
            done = _collect(out, procs, cores, "done", limit_s)
            times.append(max(m[1] for m in done) - t0)
            if last:
                break
    finally:
        for q in inboxes:
            q.put(None)
        for p in procs:
            p.join(timeout=5)
            if p.is_alive():
                p.terminate()
    orc = Oracle(Params(log2n=logn, L=L, K=K, dnum=dnum, t=t))
    n_parts = len(S.SpmvPlan(A.rows, A.cols, A.rowptr, A.colidx, A.vals, orc.p.slots).parts)
    res = [np.zeros((2, L, 1 << logn), dtype=np.uint64) for _ in range(n_parts)]
    for m in done:
        for p, b in m[2].items():
            res[p] = orc.add(res[p], np.frombuffer(b, dtype=np.uint64).reshape(2, L, 1 << logn))
    return times, cores, res


REFERENCE_SECONDS = 150.0


def run_reference(args):
    """The oracle as the reference arm, on every host core: each step is the
    oracle's cloud evaluation of the whole SpMV (every chunk; one spawned
    process per core, chunks dealt round robin, keys and encryptions made
    before the first step), timed from its start signal to the last worker's
    end; past REFERENCE_SECONDS of steps the remaining ones are not run (the
    line says how many ran).  The result is decrypted and compared with A.x."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import spmv as S
    from oracle.bgv import Oracle
    from oracle.params import Params
    A, x, ring = load_workload(args.config)
    seeds = (1, 2, 3)
    times, cores, res = oracle_allcores(A, x, ring, seeds, steps=args.warmup + args.steps,
                                        budget_s=REFERENCE_SECONDS)
    timed = times[args.warmup:] or times[-1:]
    per = sum(timed) / len(timed)
    value = 1.0 / per
    logn, L, K, dnum, t = ring
    orc = Oracle(Params(log2n=logn, L=L, K=K, dnum=dnum, t=t))
    orc.keygen(seeds[0], [])
    plan = S.SpmvPlan(A.rows, A.cols, A.rowptr, A.colidx, A.vals, orc.p.slots)
    correct = list(S.decrypt_result(orc, plan, res)) == list(A.matvec(x))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "SpMV/s",
            "n_gpus": args.gpus, "steps": len(timed), "steps_requested": args.steps,
            "warmup": min(args.warmup, len(times) - len(timed)),
            "ms_per_step": per * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": CONFIGS[args.config]},
            "nnz_per_s": value * A.nnz, "correct": bool(correct),
            "cpu_baseline": {"value": value, "unit": "SpMV/s", "cores": cores, "kind": "oracle",
                             "sample": "each step: the oracle's cloud evaluation of the whole SpMV "
                                       "(all %d chunks: HE-Mult, relinearisation, totalSum, mask, "
                                       "add) on %d spawned processes, one per core" % (len(plan.chunks), cores)},
            "e2e": {"value": value, "unit": "SpMV/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def time_steps(fn, stream, steps, barrier):
    """Device time per step (ms) of `steps` calls of fn, CUDA events on the
    launch stream, barrier + synchronize on both sides."""
    import torch
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    return e0.elapsed_time(e1) / steps


def per_step_ms(fn, stream, n):
    """Device time of each of n consecutive steps (one event between steps)."""
    import torch
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(n + 1)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    for i in range(n):
        fn()
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    return [ev[i].elapsed_time(ev[i + 1]) for i in range(n)]


def roofline(ctx, prof, steps, ring, n_ks, n_chunks, n_parts, n_rot, config="c3", bfv=None):
    peaks, peak_kind = measured_peaks()
    kernels = {}
    total_ms = sum(v[1] for v in prof.values())
    for name, (cnt, kms) in prof.items():
        mm, by = kernel_model(name, ring, n_ks, n_chunks, n_parts, n_rot, bfv)
        kernels[name] = {"launches_per_step": cnt / steps, "ms_per_step": kms / steps,
                         "share": kms / total_ms if total_ms else 0.0,
                         "mulmods_per_step": mm, "bytes_per_step": by}
    top = max(kernels, key=lambda k: kernels[k]["ms_per_step"])
    kt = kernels[top]
    launch_ms = kt["ms_per_step"] / kt["launches_per_step"]
    mm_launch = kt["mulmods_per_step"] / kt["launches_per_step"]
    by_launch = kt["bytes_per_step"] / kt["launches_per_step"]
    alu_rate, alu_src = alu_peak()   # mulmod/s
    hbm_peak = peaks["hbm_gbs"] * 1e9
    t_alu, t_hbm = mm_launch / alu_rate, by_launch / hbm_peak
    if t_alu >= t_hbm:
        ach = mm_launch / (launch_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": alu_rate / 1e12, "unit": "Tmulmod/s",
                "frac": ach / (alu_rate / 1e12), "kernel": top,
                "traffic": measured_traffic(top, config), "peak_source": alu_src}
    else:
        ach = by_launch / (launch_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"], "traffic": measured_traffic(top, config),
                "kernel": top,
                "peak_source": "%s hbm_gbs" % peak_kind}
    roof["algorithmic_per_launch"] = {"mulmods": mm_launch, "bytes": by_launch}
    step_mm = sum(v["mulmods_per_step"] for v in kernels.values())
    roof["whole_step"] = {"mulmods": step_mm, "alu_frac_at_profiled_time":
                          step_mm / (total_ms / steps * 1e-3) / alu_rate if total_ms else None}
    roof["mulmod_rate_measured_T"] = ctx.mulmod_rate(0) / 1e12
    roof["timing"] = ("average launch time of %s over a second pass of the timed steps with "
                      "CUDA events around each kernel on the launch stream (one compute stream)" % top)
    return kernels, roof


def boundary_block(ctx, inst, stream, reps=5):
    """The client-side boundary calls around one SpMV of the workload (the
    paper's Table 1 times Encrypt and Decrypt per ciphertext): CSR -> CSSC,
    partitions and chunks on the host (hespmv_encode_cssc); encryption of
    the matrix chunks and of the reorganised vector (hespmv_encrypt);
    decryption of the result with the row map undone (hespmv_decrypt).
    Median wall time of `reps` synchronised calls each."""
    import torch
    from paper_2603_04742_gb300 import binding as B
    A, x = inst

    def med(fn):
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = fn()
            torch.cuda.synchronize()
            ts.append((time.perf_counter() - t0) * 1e3)
        return float(np.median(ts)), r
    t_cssc, m = med(lambda: ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals))
    t_ea, ca = med(lambda: ctx.encrypt(m, B.HESPMV_MATRIX, seed=2))
    t_ex, cx = med(lambda: ctx.encrypt(m, B.HESPMV_VECTOR, x=x, seed=3))
    y = ctx.spmv(m, ca, cx, stream=stream)
    t_dec, out = med(lambda: ctx.decrypt(m, y))
    return {"encode_cssc_ms": t_cssc, "encrypt_matrix_ms": t_ea, "encrypt_vector_ms": t_ex,
            "decrypt_ms": t_dec, "ciphertexts_per_operand": m.n_chunks, "result_ciphertexts": m.n_parts,
            "encrypt_ms_per_ciphertext": (t_ea + t_ex) / (2 * m.n_chunks),
            "decrypt_ms_per_ciphertext": t_dec / m.n_parts,
            "correct": bool(list(out) == list(A.matvec(x))),
            "timing": "median of %d calls, wall clock, device synchronised before and after" % reps}


def batched_block(args, stream, persistent=True):
    """The batched workload (64 uneven SpMVs at N = 2^14): one batched
    evaluation per step under the autotuned schedule, against 64 plain
    hespmv_spmv calls per step and against the persistent form (one launch
    per step); the three give identical ciphertexts, which decrypt to A.x."""
    import torch
    from paper_2603_04742_gb300 import binding as B
    from paper_2603_04742_gb300 import synth
    from paper_2603_04742_gb300.api import Context
    insts = synth.workload("c4", count=args.instances)
    logn, L, K, dnum, t = synth.RING["c4"]
    ctx = Context(logn, L, K, dnum, t)
    ms = [ctx.encode_cssc(a.rows, a.cols, a.rowptr, a.colidx, a.vals) for a, _ in insts]
    ctx.keygen(1, sorted({s for m in ms for s in m.rotation_steps()}))
    As = [ctx.encrypt(m, B.HESPMV_MATRIX, seed=2 + i) for i, m in enumerate(ms)]
    Xs = [ctx.encrypt(m, B.HESPMV_VECTOR, x=xx, seed=3 + i) for i, (m, (_, xx)) in enumerate(zip(ms, insts))]
    t0 = time.perf_counter()
    tune = ctx.autotune(ms, As, Xs, reps=2)
    tune["seconds"] = time.perf_counter() - t0
    steps = max(3, min(args.steps, 20))
    ys = ctx.spmv_batched(ms, As, Xs)
    torch.cuda.synchronize()
    correct = all(list(ctx.decrypt(m, y)) == list(a.matvec(xx)) for m, y, (a, xx) in zip(ms, ys, insts))
    ref = [y.download() for y in ys]

    def batched():
        ctx.spmv_batched(ms, As, Xs, ys, stream=stream)
    for _ in range(3):
        batched()
    ms_b = time_steps(batched, stream, steps, lambda: None)
    ctx.profile_enable(True)
    time_steps(batched, stream, 1, lambda: None)
    launches = sum(v[0] for v in ctx.profile_read().values())
    ctx.profile_enable(False)
    yp = [ctx.spmv(m, a, xx) for m, a, xx in zip(ms, As, Xs)]

    def plain():
        for m, a, xx, y in zip(ms, As, Xs, yp):
            ctx.spmv(m, a, xx, y=y, stream=stream)
    for _ in range(3):
        plain()
    ms_p = time_steps(plain, stream, steps, lambda: None)
    same = all(np.array_equal(y.download(), r) for y, r in zip(yp, ref))
    n = len(insts)
    nnz = sum(a.nnz for a, _ in insts)
    out = {"workload": CONFIGS["c4"], "instances": n, "steps": steps, "nnz": nnz,
           "chunks": sum(m.n_chunks for m in ms), "rotations": sum(m.n_rot for m in ms),
           "keyswitches": sum(m.n_chunks + m.n_keyswitch for m in ms),
           "value": n * 1000.0 / ms_b, "unit": "SpMV/s", "ms_per_step": ms_b,
           "nnz_per_s": nnz * 1000.0 / ms_b, "schedule": tune["best"], "gpu_launches_per_step": launches,
           "correct": bool(correct),
           "plain": {"value": n * 1000.0 / ms_p, "unit": "SpMV/s", "ms_per_step": ms_p,
                     "form": "%d hespmv_spmv calls per step" % n},
           "batched_vs_plain": ms_p / ms_b, "autotune": tune}
    if persistent:
        cur = ctx.get_tuning()
        ctx.set_tuning(16, 0, 0, 0, 1)
        yq = ctx.spmv_batched(ms, As, Xs)

        def pers():
            ctx.spmv_batched(ms, As, Xs, yq, stream=stream)
        for _ in range(3):
            pers()
        ms_q = time_steps(pers, stream, steps, lambda: None)
        same = same and all(np.array_equal(y.download(), r) for y, r in zip(yq, ref))
        out["persistent"] = {"value": n * 1000.0 / ms_q, "unit": "SpMV/s", "ms_per_step": ms_q,
                             "gpu_launches_per_step": 1,
                             "form": "hespmv_spmv_batched with tuning.persistent = 1: one launch per "
                                     "step, HE-Mult groups of 16"}
        ctx.set_tuning(cur["mult_batch"], cur["rot_batch"], cur["ntt_split"], cur["rows_tma"],
                       cur["persistent"], cur["persist_blocks"], cur["streams"])
    out["identical_results"] = bool(same)
    ctx.device_status()
    del ctx, As, Xs, ys, yp
    if persistent:   # the key holder's choices: digits of the key switch, rotation keys
        from paper_2603_04742_gb300.api import tune_keyswitch
        cand = tune_keyswitch(synth.RING["c4"], insts, reps=3)
        out["keyswitch_tuning"] = {
            "candidates": cand,
            "note": "each candidate has its own keys and ciphertexts (decryptions equal); dnum values "
                    "with alpha > K are not offered; 'pow2' is the paper's policy and the value above"}
    return out


def rotation_block(args, stream):
    """A rotation-bearing SpMV at N = 2^15 (the Figure 8 sweep point with
    2^18 non-zeros: 16384 x 16384 uniform positions, power-of-two keys):
    time per SpMV, its kernels and the roofline of the top one."""
    import torch
    from paper_2603_04742_gb300 import binding as B
    from paper_2603_04742_gb300 import synth
    from paper_2603_04742_gb300.api import Context
    ring = synth.RING["c5"]
    logn, L, K, dnum, t = ring
    ctx = Context(logn, L, K, dnum, t)
    g = np.random.default_rng(108)
    A = synth.uniform_positions(g, 16384, 16384, 1 << 18, -15, 15)
    x = g.integers(-15, 16, size=16384, dtype=np.int64)
    m = ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals, max_abs_x=15)
    ctx.keygen(1, m.rotation_steps())
    ca = ctx.encrypt(m, B.HESPMV_MATRIX, seed=18)
    cx = ctx.encrypt(m, B.HESPMV_VECTOR, x=x, seed=118)
    y = ctx.spmv(m, ca, cx)
    torch.cuda.synchronize()
    ref = y.download()
    t0 = time.perf_counter()
    default_ms = time_steps(lambda: ctx.spmv(m, ca, cx, y=y, stream=stream), stream, 10, lambda: None)
    if args.config == "rot" and args.tuning:  # a fixed schedule (profiling runs)
        v = [int(x) for x in args.tuning.split(",")]
        ctx.set_tuning(v[0], v[1], v[2], v[3], v[4], 0, v[5])
        tune = {"fixed": ctx.get_tuning()}
    else:
        tune = ctx.autotune([m], [ca], [cx], reps=3)
    tune["seconds"] = time.perf_counter() - t0
    tune["default_schedule_ms"] = default_ms
    ctx.spmv(m, ca, cx, y=y, stream=stream)
    torch.cuda.synchronize()
    correct = list(ctx.decrypt(m, y)) == list(A.matvec(x)) and np.array_equal(y.download(), ref)

    def step():
        ctx.spmv(m, ca, cx, y=y, stream=stream)
    for _ in range(3):
        step()
    steps = max(10, min(args.steps, 50))
    ms_step = time_steps(step, stream, steps, lambda: None)
    tun = ctx.get_tuning()   # kernels profiled one stream at a time (as in the headline)
    ctx.set_tuning(tun["mult_batch"], tun["rot_batch"], tun["ntt_split"], tun["rows_tma"],
                   tun["persistent"], tun["persist_blocks"], 1)
    step()
    ctx.profile_enable(True)
    time_steps(step, stream, steps, lambda: None)
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    n_ks = m.n_chunks + m.n_keyswitch
    kernels, roof = roofline(ctx, prof, steps, ring, n_ks, m.n_chunks, m.n_parts, m.n_rot, "rot")
    return {"workload": "16384x16384, 2^18 non-zeros at uniform positions, integers [-15,15]; BGV "
                        "N=2^15, 8+2 primes, dnum 4, t=1179649, power-of-two Galois keys",
            "value": 1000.0 / ms_step, "unit": "SpMV/s", "ms_per_step": ms_step, "steps": steps,
            "nnz_per_s": A.nnz * 1000.0 / ms_step, "chunks": m.n_chunks, "rotations": m.n_rot,
            "keyswitches": n_ks, "correct": bool(correct), "roofline": roof, "kernels": kernels,
            "gpu_launches_per_step": sum(v[0] for v in prof.values()) / steps, "autotune": tune}


def serving_measure(args, requests, sat_requests, serial_requests):
    """c5: Poisson arrivals of SpMV requests drawn from a pool of distinct
    pre-encrypted instances, served with continuous batching at 0.7 x the
    saturated throughput; compared with a serial server (one request at a
    time) on the same arrival process."""
    import torch

    from paper_2603_04742_gb300 import binding as B
    from paper_2603_04742_gb300 import synth
    from paper_2603_04742_gb300.api import Context, Server

    pool = synth.workload("c5", pool=args.pool)
    ring = synth.RING["c5"]
    logn, L, K, dnum, t = ring
    ctx = Context(logn, L, K, dnum, t)
    ms = [ctx.encode_cssc(a.rows, a.cols, a.rowptr, a.colidx, a.vals) for a, _ in pool]
    ctx.keygen(1, sorted({s for m in ms for s in m.rotation_steps()}))
    As = [ctx.encrypt(m, B.HESPMV_MATRIX, seed=2 + i) for i, m in enumerate(ms)]
    Xs = [ctx.encrypt(m, B.HESPMV_VECTOR, x=x, seed=500 + i) for i, (m, (_, x)) in enumerate(zip(ms, pool))]
    ys = [ctx.spmv(m, a, x) for m, a, x in zip(ms, As, Xs)]
    torch.cuda.synchronize()
    correct = all(list(ctx.decrypt(m, y)) == list(a.matvec(x)) for m, y, (a, x) in zip(ms, ys, pool))
    rng = np.random.default_rng(105)
    budget = args.slots * (6 << 30)

    def serve(n_req, rate, slots, max_batch):
        srv = Server(ctx, slots=slots, mem_budget_bytes=budget, max_batch=max_batch)
        picks = rng.integers(0, len(pool), n_req)
        gaps = rng.exponential(1.0 / rate, n_req) if rate else np.zeros(n_req)
        arrive = np.cumsum(gaps)
        t0 = time.perf_counter()
        tickets, sub = [], []
        for k in range(n_req):
            while True:
                dt = arrive[k] - (time.perf_counter() - t0)
                if dt <= 0:
                    break
                if dt > 1e-3:
                    time.sleep(dt - 5e-4)
            i = int(picks[k])
            sub.append(time.perf_counter() - t0)
            tickets.append(srv.submit(ms[i], As[i], Xs[i]))
        while srv.stats()["completed"] < n_req:
            time.sleep(1e-3)
        st = srv.stats()
        lat = np.array([srv.poll(tk)[1] for tk in tickets], dtype=np.float64) / 1e6  # ms
        srv.stop(60000)
        end = max(s_ + l_ / 1e3 for s_, l_ in zip(sub, lat))
        nnz = sum(pool[int(i)][0].nnz for i in picks)
        return {"requests": n_req, "throughput": n_req / end, "nnz_per_s": nnz / end,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()), "batches": st["batches"],
                "max_inflight": st["max_inflight"], "slots": slots, "max_batch": max_batch}

    sat = serve(sat_requests, None, args.slots, args.max_batch)
    rate = 0.7 * sat["throughput"]
    cont = serve(requests, rate, args.slots, args.max_batch)
    serial = serve(serial_requests, rate, 1, 1)
    return {"workload": "Poisson arrivals at %.1f req/s (0.7 x saturated), requests drawn from %d "
                        "distinct pre-encrypted instances (n log-U[512,16384], density "
                        "log-U[5e-4,1e-2]), N=2^15, 8+2 primes, dnum 4, t=1179649" % (rate, len(pool)),
            "pool_chunks": sum(m.n_chunks for m in ms), "rate": rate,
            "correct": bool(correct), "latency_ms": {"p50": cont["p50_ms"], "p99": cont["p99_ms"]},
            "value": cont["throughput"], "unit": "SpMV/s", "nnz_per_s": cont["nnz_per_s"],
            "continuous_batching": cont, "saturated": sat, "serial": serial}


def run_serving(args):
    if int(os.environ.get("RANK", "0")) != 0:
        return 0
    r = serving_measure(args, args.requests, args.sat_requests, args.serial_requests)
    line = {"metric": METRIC, "value": r["value"], "unit": "SpMV/s", "n_gpus": 1,
            "steps": args.requests, "warmup": 0, "ms_per_step": 1e3 / r["value"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": {"workload": "c5 serving: " + r["workload"],
                                            "pool_chunks": r["pool_chunks"]},
            "correct": r["correct"], "latency_ms": r["latency_ms"], "nnz_per_s": r["nnz_per_s"],
            "continuous_batching": r["continuous_batching"], "saturated": r["saturated"],
            "serial": r["serial"]}
    print(json.dumps(line), flush=True)
    return 0


def run_sweep(args):
    """Runtime vs nnz at N = 2^15 (the paper's Figure 8 reports a log-log
    slope near 1 for its CPU implementation): uniform random 16384 x 16384
    integer matrices with nnz from 2^10 to 2^22."""
    import torch

    from paper_2603_04742_gb300 import binding as B
    from paper_2603_04742_gb300 import synth
    from paper_2603_04742_gb300.api import Context

    if int(os.environ.get("RANK", "0")) != 0:
        return 0
    logn, L, K, dnum, t = synth.RING["c5"]
    ctx = Context(logn, L, K, dnum, t)
    ctx.keygen(1)   # every power-of-two rotation key
    stream = torch.cuda.current_stream()
    g = np.random.default_rng(108)
    pts = []
    for e in range(10, 23, 2):
        nnz = 1 << e
        A = synth.uniform_positions(g, 16384, 16384, nnz, -15, 15)
        x = g.integers(-15, 16, size=16384, dtype=np.int64)
        m = ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals, max_abs_x=15)
        ca = ctx.encrypt(m, B.HESPMV_MATRIX, seed=e)
        cx = ctx.encrypt(m, B.HESPMV_VECTOR, x=x, seed=100 + e)
        y = ctx.spmv(m, ca, cx)
        torch.cuda.synchronize()
        ok = list(ctx.decrypt(m, y)) == list(A.matvec(x))

        def step():
            ctx.spmv(m, ca, cx, y=y, stream=stream)
        ctx.set_tuning(0, 0, 0, 0)
        for _ in range(3):
            step()
        ms = time_steps(step, stream, args.steps, lambda: None)
        tuned = ctx.autotune([m], [ca], [cx], reps=3)["best"]
        for _ in range(3):
            step()
        ms_tuned = time_steps(step, stream, args.steps, lambda: None)
        ok = ok and list(ctx.decrypt(m, y)) == list(A.matvec(x))
        ctx.set_tuning(0, 0, 0, 0)
        pa = ctx.encode_matrix_plain(m)
        yp = ctx.spmv_ptmatrix(m, pa, cx)
        torch.cuda.synchronize()
        ok_p = list(ctx.decrypt(m, yp)) == list(A.matvec(x))

        def step_p():
            ctx.spmv_ptmatrix(m, pa, cx, y=yp, stream=stream)
        for _ in range(3):
            step_p()
        ms_p = time_steps(step_p, stream, args.steps, lambda: None)
        pts.append({"nnz": A.nnz, "chunks": m.n_chunks, "rotations": m.n_rot,
                    "keyswitches": m.n_chunks + m.n_keyswitch, "ms": ms, "ms_tuned": ms_tuned,
                    "schedule": tuned, "correct": bool(ok),
                    "ms_plain_matrix": ms_p, "correct_plain_matrix": bool(ok_p)})
        del ca, cx, y, m, pa, yp
    lx = np.log([p_["nnz"] for p_ in pts])
    ly = np.log([p_["ms"] for p_ in pts])
    slope_all = float(np.polyfit(lx, ly, 1)[0])
    big = [i for i, p_ in enumerate(pts) if p_["nnz"] >= 1 << 16]
    slope_big = float(np.polyfit(lx[big], ly[big], 1)[0])
    line = {"metric": "runtime vs nnz (Figure 8 sweep)", "unit": "ms per SpMV",
            "config": {"workload": "uniform random 16384x16384 integer matrices, nnz 2^10..2^22; "
                                   "BGV N=2^15, 8+2 primes, dnum 4, t=1179649, power-of-two keys"},
            "points": pts, "loglog_slope_all": slope_all, "loglog_slope_nnz_ge_2^16": slope_big}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.config == "sweep":
        return run_sweep(args)
    if args.config == "rot":
        if int(os.environ.get("RANK", "0")) != 0:
            return 0
        import torch
        r = rotation_block(args, torch.cuda.current_stream())
        r.update({"metric": "encrypted SpMV/s (rotation-bearing SpMV at N=2^15)", "higher_is_better": True})
        print(json.dumps(r), flush=True)
        return 0
    if args.config == "c5":
        return run_serving(args)
    import torch
    import torch.distributed as dist

    from paper_2603_04742_gb300 import binding as B
    from paper_2603_04742_gb300 import synth
    from paper_2603_04742_gb300.api import Context

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            dist.barrier()

    from paper_2603_04742_gb300.dist import max_over_ranks as _max

    def max_over_ranks(v):
        return _max(v, dev)

    stream = torch.cuda.current_stream()
    batched = args.config == "c4"
    if batched:
        insts = synth.workload("c4", count=args.instances)
        ring = synth.RING["c4"]
    elif args.scheme == "ckks":
        A, x = synth.workload(args.config)        # float64 values as generated
        if A.vals.dtype.kind != "f":
            g = np.random.default_rng(7)
            A.vals = g.uniform(-1, 1, A.nnz)
            x = g.uniform(-1, 1, A.cols)
        ring = synth.RING[args.config]
        insts = [(A, x)]
    else:
        A, x, ring = load_workload(args.config)
        insts = [(A, x)]
    logn, L, K, dnum, t = ring
    ct_words = 2 * L * (1 << logn)
    ckks = args.scheme == "ckks"
    ctx = Context(logn, L, K, dnum, 0 if ckks else t, device=local, scheme=args.scheme)
    ms = [ctx.encode_cssc(a.rows, a.cols, a.rowptr, a.colidx, a.vals) for a, _ in insts]
    ctx.keygen(1 + rank, sorted({s for m in ms for s in m.rotation_steps()}))
    if ckks:
        As = [ctx.encrypt_real(m, B.HESPMV_MATRIX, a.vals, seed=2 + 1000 * rank + i)
              for i, (m, (a, _)) in enumerate(zip(ms, insts))]
        Xs = [ctx.encrypt_real(m, B.HESPMV_VECTOR, xx, seed=3 + 1000 * rank + i)
              for i, (m, (_, xx)) in enumerate(zip(ms, insts))]
    else:
        As = [ctx.encrypt(m, B.HESPMV_MATRIX, seed=2 + 1000 * rank + i) for i, m in enumerate(ms)]
        Xs = [ctx.encrypt(m, B.HESPMV_VECTOR, x=xx, seed=3 + 1000 * rank + i)
              for i, (m, (_, xx)) in enumerate(zip(ms, insts))]
    # schedule autotuning (batch sizes, NTT split; results are unchanged)
    tune = None
    if args.persistent:
        ctx.set_tuning(0, 0, 0, 0, 1)
    elif args.tuning:
        v = [int(x) for x in args.tuning.split(",")]
        ctx.set_tuning(v[0], v[1], v[2], v[3], v[4], 0, v[5])
        tune = {"fixed": ctx.get_tuning()}
    elif not args.no_autotune:
        t0 = time.perf_counter()
        tune = ctx.autotune(ms, As, Xs, reps=3)
        tune["seconds"] = time.perf_counter() - t0
    if batched:
        ys = ctx.spmv_batched(ms, As, Xs)

        def step():
            ctx.spmv_batched(ms, As, Xs, ys, stream=stream)
    else:
        ys = [ctx.spmv(ms[0], As[0], Xs[0])]

        def step():
            ctx.spmv(ms[0], As[0], Xs[0], y=ys[0], stream=stream)
    torch.cuda.synchronize()
    if ckks:   # 1e-3 relative in the max norm
        correct = all(np.max(np.abs(ctx.decrypt_real(m, y) - a.matvec(xx)))
                      <= 1e-3 * max(1.0, np.max(np.abs(a.matvec(xx))))
                      for m, y, (a, xx) in zip(ms, ys, insts))
    else:
        correct = all(list(ctx.decrypt(m, y)) == list(a.matvec(xx))
                      for m, y, (a, xx) in zip(ms, ys, insts))
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    clocks = Clocks(local)
    clocks.start()
    ms_step = max_over_ranks(time_steps(step, stream, args.steps, barrier))
    clk = clocks.stop()
    # a sustained pass of the same step (about 2 s) with its own clock samples
    clocks_sus = Clocks(local)
    clocks_sus.start()
    n_sus = max(1, int(2000.0 / max(ms_step, 1e-3)))
    ms_sus = time_steps(step, stream, n_sus, lambda: None)
    clk_sus = clocks_sus.stop()
    if clk_sus:
        clk_sus.update({"steps": n_sus, "ms_per_step": ms_sus})
    n_spmv = len(insts)
    nnz = sum(a.nnz for a, _ in insts)
    value = world * n_spmv * 1000.0 / ms_step
    # step-time distribution (a separate pass, >= 50 steps)
    dist_ms = np.asarray(per_step_ms(step, stream, max(50, args.steps)))
    step_ms = {"median": float(np.median(dist_ms)), "p99": float(np.percentile(dist_ms, 99)),
               "runs": int(dist_ms.size)}

    # per-kernel device times (second pass, kernels one by one); a schedule
    # with two compute streams is profiled on one (the same groups), so that
    # each kernel's time is its own and not shared with a concurrent one
    tun = ctx.get_tuning()
    if tun["streams"] == 2:
        ctx.set_tuning(tun["mult_batch"], tun["rot_batch"], tun["ntt_split"], tun["rows_tma"],
                       tun["persistent"], tun["persist_blocks"], 1)
        step()
    ctx.profile_enable(True)
    ms_profiled = time_steps(step, stream, args.steps, lambda: None)
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    if tun["streams"] == 2:
        ctx.set_tuning(tun["mult_batch"], tun["rot_batch"], tun["ntt_split"], tun["rows_tma"],
                       tun["persistent"], tun["persist_blocks"], 2)

    extra = {}
    if batched:
        # the same instances as plain evaluations, one call each
        yp = [ctx.spmv(m, a, xx) for m, a, xx in zip(ms, As, Xs)]
        torch.cuda.synchronize()

        def plain():
            for m, a, xx, y in zip(ms, As, Xs, yp):
                ctx.spmv(m, a, xx, y=y, stream=stream)
        for _ in range(max(3, args.warmup)):
            plain()
        ms_plain = max_over_ranks(time_steps(plain, stream, args.steps, barrier))
        same = all(np.array_equal(y.download(), z.download()) for y, z in zip(ys, yp))
        extra["plain"] = {"value": world * n_spmv * 1000.0 / ms_plain, "unit": "SpMV/s",
                          "ms_per_step": ms_plain, "identical_results": bool(same),
                          "form": "%d hespmv_spmv calls per step" % n_spmv}
        extra["batched_vs_plain"] = ms_plain / ms_step

    # e2e through the C ABI from pinned host buffers (single-matrix workloads)
    e2e = None
    if not args.no_e2e and not batched:
        m, ca, cx, y = ms[0], As[0], Xs[0], ys[0]
        hA = torch.empty(m.n_chunks * ct_words, dtype=torch.int64, pin_memory=True)
        hX = torch.empty(m.n_chunks * ct_words, dtype=torch.int64, pin_memory=True)
        hY = torch.empty(m.n_parts * ct_words, dtype=torch.int64, pin_memory=True)
        hA.numpy()[:] = ca.download().reshape(-1).view(np.int64)
        hX.numpy()[:] = cx.download().reshape(-1).view(np.int64)
        nA, nX, nY = (hA.numpy().view(np.uint64), hX.numpy().view(np.uint64),
                      hY.numpy().view(np.uint64))
        for _ in range(2):
            ctx.spmv_host(m, nA, nX, nY, stream=stream)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ctx.spmv_host(m, nA, nX, nY, stream=stream)
        dt_u64 = max_over_ranks(time.perf_counter() - t0)
        assert np.array_equal(nY.reshape(y.download().shape), y.download())
        # the packed wire form: W-bit residues uploaded, unpacked per upload
        # group on the device, result packed on the device
        pw, wbits = ctx.ct_packed_words()
        pA = torch.empty(m.n_chunks * pw, dtype=torch.int64, pin_memory=True)
        pX = torch.empty(m.n_chunks * pw, dtype=torch.int64, pin_memory=True)
        pY = torch.empty(m.n_parts * pw, dtype=torch.int64, pin_memory=True)
        pA.numpy()[:] = ctx.ct_pack(ca.download()).reshape(-1).view(np.int64)
        pX.numpy()[:] = ctx.ct_pack(cx.download()).reshape(-1).view(np.int64)
        qA, qX, qY = (pA.numpy().view(np.uint64), pX.numpy().view(np.uint64),
                      pY.numpy().view(np.uint64))
        for _ in range(2):
            ctx.spmv_host_packed(m, qA, qX, qY, stream=stream)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ctx.spmv_host_packed(m, qA, qX, qY, stream=stream)
        dt_sync = max_over_ranks(time.perf_counter() - t0)
        assert np.array_equal(ctx.ct_unpack(qY).reshape(y.download().shape), y.download())
        # pipelined: each step's upload overlaps the previous step's compute
        # (three staging slots); every step still uploads its inputs and
        # downloads its result
        qY[:] = 0
        for _ in range(3):
            ctx.spmv_host_packed_async(m, qA, qX, qY, stream=stream)
        stream.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ctx.spmv_host_packed_async(m, qA, qX, qY, stream=stream)
        stream.synchronize()
        dt = max_over_ranks(time.perf_counter() - t0)
        ctx.device_status()
        assert np.array_equal(ctx.ct_unpack(qY).reshape(y.download().shape), y.download())
        e2e = {"value": world * args.steps / dt, "unit": "SpMV/s",
               "h2d_bytes_per_step": 2 * m.n_chunks * pw * 8,
               "d2h_bytes_per_step": m.n_parts * pw * 8,
               "form": "hespmv_spmv_host_packed_async: %d calls back to back, each uploading its "
                       "inputs and downloading its result, from page-locked host buffers "
                       "(%d-bit residues); one synchronisation at the end" % (args.steps, wbits),
               "sync_form": {"value": world * args.steps / dt_sync, "unit": "SpMV/s",
                             "form": "hespmv_spmv_host_packed, synchronous per call"},
               "u64_form": {"value": world * args.steps / dt_u64, "unit": "SpMV/s",
                            "h2d_bytes_per_step": 2 * m.n_chunks * ct_words * 8,
                            "d2h_bytes_per_step": m.n_parts * ct_words * 8,
                            "form": "hespmv_spmv_host (64-bit words), synchronous per call"}}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    n_chunks = sum(m.n_chunks for m in ms)
    n_ks = n_chunks + sum(m.n_keyswitch for m in ms)
    bfv = None
    if args.scheme == "bfv":
        logn, L = ring[0], ring[1]
        bfv = bfv_basis(logn, L, ring[4], ctx.moduli()[0])
    kernels, roof = roofline(ctx, prof, args.steps, ring, n_ks, n_chunks,
                             sum(m.n_parts for m in ms), sum(m.n_rot for m in ms), args.config, bfv)
    # the committed DRAM counters are for the BGV kernels of this workload
    if args.scheme != "bgv":
        roof["traffic"] = None
    # the whole SpMV: every kernel's algorithmic mulmods over the timed step
    alu_rate, _ = alu_peak()
    roof["whole_step"]["alu_frac"] = roof["whole_step"]["mulmods"] / (ms_step * 1e-3) / alu_rate

    cpu = None
    if not args.no_cpu_baseline and args.scheme == "bgv":
        A0, x0 = insts[0]
        sample = 8 if args.config in ("c3",) else 10 ** 9
        smp = OracleSample(A0, x0, ring, sample)
        dt, n_total = smp.run(), smp.n_total
        n_s = len(smp.chunks)
        per_spmv = dt * n_total / n_s
        if batched:   # scale instance 0 to the whole batch by chunk count
            per_spmv *= n_chunks / max(1, ms[0].n_chunks) / n_spmv
        v = 1.0 / per_spmv
        cpu = {"value": v, "unit": "SpMV/s", "cores": 1, "kind": "oracle",
               "sample": "oracle cloud evaluation of %d of %d chunks of instance 0 (%.1f s), "
                         "scaled to one SpMV%s" % (n_s, n_total, dt,
                                                   " of the batch by chunk count" if batched else "")}
        if args.config == "c3":
            # every host core: the whole SpMV, one process per core; its result
            # ciphertext is compared with the GPU's
            try:
                dts, cores, res = oracle_allcores(A0, x0, ring, (1 + rank, 2 + 1000 * rank, 3 + 1000 * rank))
                dta = dts[-1]
                gy = ys[0].download()
                cpu["all_cores"] = {"value": 1.0 / dta, "unit": "SpMV/s", "cores": cores, "kind": "oracle",
                                    "seconds": dta, "nproc": os.cpu_count(),
                                    "matches_gpu": bool(all(np.array_equal(gy[p], r) for p, r in enumerate(res))),
                                    "sample": "the whole SpMV (all %d chunks), chunks dealt round robin to "
                                              "one spawned process per core, keys and encryptions made "
                                              "before the timed region" % n_total}
            except Exception as e:   # reported, not fatal: the baseline is context
                cpu["all_cores"] = {"error": str(e)[:200]}

    workload = CONFIGS[args.config]
    if args.scheme == "bfv":
        workload = workload.replace("BGV", "BFV (exact HE-Mult)")
    elif args.scheme == "ckks":
        workload = workload.replace("fixed point 2^15; ", "float64 values; ").replace(
            "BGV", "CKKS scale 2^40, masks 2^30").split(", t=")[0]
    cfg = {"workload": workload, "scheme": args.scheme, "instances": n_spmv, "chunks": n_chunks,
           "partitions": sum(m.n_parts for m in ms), "rotations": sum(m.n_rot for m in ms),
           "keyswitches": n_ks,
           "l2": "inputs %.0f MB per step > 129 MB L2 (no flush)" % (2 * n_chunks * ct_words * 8 / 1e6),
           "form": "hespmv_spmv_batched, one graph replay per step" if batched
                   else "hespmv_spmv, one graph replay per step",
           "parallelism": "independent SpMVs per GPU"}
    line = {
        "metric": METRIC, "value": value, "unit": "SpMV/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic", "config": cfg,
        "nnz_per_s": value * nnz / n_spmv,
        "step_ms": step_ms,
        "hbm_bytes": int(ctx.device_bytes()),
        "correct": bool(correct),
        "e2e": e2e,
        "gpu_launches": int(sum(v[0] for v in prof.values())),
        "graph_launches": args.steps,
        "ms_per_step_kernels_one_by_one": ms_profiled,
        "roofline": roof,
        "cpu_baseline": cpu,
        "clocks": clk,
        "kernels": kernels,
    }
    line["autotune"] = tune
    line["clocks_sustained"] = clk_sus
    line.update(extra)
    if args.config == "c3" and args.scheme == "bgv" and not args.no_extra:
        # the rest of the metric: batched vs plain, serving latency, rotations
        # at N = 2^15, and the client-side boundary calls
        blocks = (("boundary_calls", lambda: boundary_block(ctx, insts[0], stream)),
                  ("batched", lambda: batched_block(args, stream)),
                  ("serving", lambda: serving_measure(args, args.serve_requests, 400, 300)),
                  ("rotations", lambda: rotation_block(args, stream)))
        for name, fn in blocks:
            t0 = time.perf_counter()
            try:
                line[name] = fn()
            except Exception as e:   # reported in the line; the headline stands
                line[name] = {"error": "%s: %s" % (type(e).__name__, str(e)[:300])}
            line[name]["seconds"] = time.perf_counter() - t0
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
