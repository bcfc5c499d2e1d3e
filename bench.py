"""Encrypted-inference benchmark: RNS-CKKS evaluation of the fall-detection networks on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload small|large|toy]
                    [--impl hear|reference] [--no-batched] [--no-cpu-baseline]

One step = one pass of the whole hot path (every layer of the encrypted network) over one
batch of ciphertexts already resident in HBM:
  * small (default, the quoted configuration): N = 2^14, 60 + 7x40-bit ciphertext primes,
    one 60-bit special prime, one clip of 16x128 features per ciphertext, FC 2048->128 ->
    x^2 -> FC 128->2, batch 1 (one request);
  * large: N = 2^15, 60 + 14x40-bit primes, two 60-bit special primes, 256 clips packed
    8 per ciphertext (32 ciphertexts in one batch), FC 2048->512 -> x^2 -> FC 512->128 ->
    x^2 -> FC 128->2.
Unless --no-batched, the JSON line also carries the batched large network as "batched".
Rank 0 prints one JSON line.  Under torchrun every rank evaluates its own replica (no
collective on the data path; weak scaling) and the slowest rank's time is reported.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "encrypted inferences/s & p50/p99 latency (N=2^14/2^15), batched vs plain on GB300"
# the serving configuration: Poisson request rates, counted seconds and warm-up per rate
C5_RATES = [10.0, 30.0, 100.0, 300.0, 1000.0, 2000.0]
C5_SECONDS = 60.0
C5_WARMUP = 5.0
UNIT = "inferences/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="small", choices=["small", "large", "toy"])
    ap.add_argument("--impl", default="hear", choices=["hear", "reference"])
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--clips", type=int, default=None, help="clips in the batch (default: the workload's)")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--rates", default="100,1000,2000", help="request rates (req/s) of the served sweep")
    ap.add_argument("--served-seconds", type=float, default=4.0, help="counted seconds per served rate")
    ap.add_argument("--served-warmup", type=float, default=1.0, help="uncounted warm-up seconds per served rate")
    ap.add_argument("--c5", action="store_true",
                    help="the serving configuration in full: Poisson rates 10-2000 req/s, 60 s each after a 5 s "
                         "warm-up, small network and the 70/30 mix (about 13 minutes)")
    ap.add_argument("--no-cnn", action="store_true", help="skip the CNN sections (Table 1 layers, 1D-CNN-64)")
    ap.add_argument("--no-min-level", action="store_true", help="skip the minimal-start-level variant")
    ap.add_argument("--mix-rates", default="100,300,1000", help="request rates (req/s) of the mixed sweep")
    ap.add_argument("--conv-rows", default="all", help="Table 1 rows to time: all | comma-separated indices")
    ap.add_argument("--no-simd", action="store_true", help="skip the slot-batched (one clip per slot) rows")
    ap.add_argument("--no-fc-tune", action="store_true",
                    help="evaluate every network in the default FC form instead of the tuned one")
    ap.add_argument("--fc-form", default=None,
                    help="pin the headline network's FC form as 'n1,hoist[,sums]' (e.g. 32,1,1) instead of tuning it "
                         "(profiles pin the form the timed run chose, as HEAR_NTT_TABLE pins the NTT table)")
    ap.add_argument("--sections-out", default="bench_out/sections.json",
                    help="file for the full result (every section); the last stdout line is the short headline")
    ap.add_argument("--simd-rows", default="all",
                    help="slot-batched rows: all | comma-separated indices into small@top, small@level3, large@top")
    return ap.parse_args()


def describe(w):
    nets = {"toy": "FC 64->16 -> x^2 -> FC 16->2 (collapsed)", "small": "FC 2048->128 -> x^2 -> FC 128->2",
            "large": "FC 2048->512 -> x^2 -> FC 512->128 -> x^2 -> FC 128->2"}
    qb = "%d+%dx%d" % (w.q_bits[0], len(w.q_bits) - 1, w.q_bits[1])
    return ("%s: RNS-CKKS N=2^%d, q=%s bits, p=%s bits, scale 2^40, %s, %d clip(s) of %d features, "
            "%d clips per ciphertext, %d ciphertext(s) per batch" %
            (w.name, w.log_n, qb, "+".join(map(str, w.p_bits)), nets[w.name], w.n_clips, w.clip_dim,
             min(w.clips_per_ct, w.n_clips), w.n_ct))


def describe_short(w):
    nets = {"toy": "FC 64->16->x^2->FC 16->2", "small": "FC 2048->128->x^2->FC 128->2",
            "large": "FC 2048->512->x^2->FC 512->128->x^2->FC 128->2"}
    return "%s: N=2^%d, q=%d+%dx%d, p=%s bits, %s, %d clip(s) in %d ciphertext(s)" % (
        w.name, w.log_n, w.q_bits[0], len(w.q_bits) - 1, w.q_bits[1], "+".join(map(str, w.p_bits)), nets[w.name],
        w.n_clips, w.n_ct)


# ------------------------------------------------------------------ distributed plumbing
class Dist:
    """Rank plumbing for torchrun: one replica per GPU, a barrier around the timed region and
    the max over ranks of the measured times.  NCCL on GPUs; gloo when no GPU is visible
    (or HEAR_DIST_BACKEND=gloo), which is how the host logic is tested on CPU."""

    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        self.device = "cpu"
        if self.world > 1:
            import torch
            import torch.distributed as dist
            backend = os.environ.get("HEAR_DIST_BACKEND") or ("nccl" if torch.cuda.is_available() else "gloo")
            if backend == "nccl":
                torch.cuda.set_device(self.local)
                dist.init_process_group("nccl", device_id=torch.device("cuda", self.local))
                self.device = "cuda"
            else:
                dist.init_process_group("gloo")
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x):
        if not self.pg:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device=self.device)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


def replica_value(world, steps, clips_per_step, max_ms):
    """whole-job throughput of `world` replicas: all ranks' clips over the slowest rank's
    time for `steps` steps (weak scaling)"""
    return world * steps * clips_per_step / (max_ms / 1e3)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.th.join(timeout=2)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if len(r) > 5 + i and r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ------------------------------------------------------------------ peaks
def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# Integer-pipe roofline of the NTT.  Peak: 152 SMs x 4 sub-partitions x 32 lanes, one
# 32-bit integer instruction per lane per cycle, at the 2070 MHz maximum SM clock.
# Algorithmic work: a lazy (Harvey) butterfly with a Shoup product by a precomputed
# twiddle counts 30 32-bit integer operations (the multiply-high of two 64-bit words:
# 4 partial products x 2 words + 4 carries = 12; two 64-bit multiply-lows: 2 x 4 = 8;
# the correction, add and subtract of 64-bit words: 10).
ALU_PEAK_TOPS = 152 * 4 * 32 * 2.070e9 / 1e12
OPS_PER_BUTTERFLY = 30
# Multiply-pipe roofline of the slot-batched matrix product: each 32 x 32 -> 64-bit partial
# product is one warp instruction of the integer multiply (FMA-heavy) pipe holding it 4 cycles
# (ncu on the kernel: 2.47e9 such instructions for 2.42e9 partial products, 3.99 pipe cycles
# each), i.e. 8 lanes per cycle per sub-partition: 152 SMs x 4 x 8 lanes x 2.07 GHz.
MAD_WIDE_PEAK_TOPS = 152 * 4 * 8 * 2.070e9 / 1e12


def ntt_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in ("ntt.cu", "modarith.cuh"):
        with open(os.path.join(ROOT, "paper_2104_09164_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def committed_traffic(workload):
    """DRAM bytes per forward-NTT call from the committed ncu summary of this workload, if
    it was taken on the current NTT source"""
    import re
    path = os.path.join(ROOT, "profiles", "ntt_fwd_%s.md" % workload)
    try:
        txt = open(path).read()
    except OSError:
        return None
    m_src = re.search(r"source_sha256_16:\s*([0-9a-f]{16})", txt)
    m_tr = re.search(r"dram_bytes_per_call:\s*([0-9.e+]+)", txt)
    if not m_src or not m_tr or m_src.group(1) != ntt_source_hash():
        return None
    return float(m_tr.group(1))


def roofline(stages, psteps, log_n, workload, bfly_peak=None):
    """the forward NTT against its measured butterfly ceiling (bfly_peak: butterflies/s of
    hear_dbg_bfly_peak on this context), with the HBM fraction and the derived integer-op
    fraction beside it"""
    hbm, how = peaks()
    fwd = stages.get("ntt_fwd")
    name = max(stages.items(), key=lambda kv: kv[1][1])[0]
    if not fwd:
        return {"bound": "hbm", "kernel": name, "achieved": None, "peak": hbm, "unit": "GB/s", "frac": None,
                "traffic": None}
    calls, ms, byts = fwd
    calls_per_step = calls / 2 / psteps            # two pass kernels per forward NTT
    n = 1 << log_n
    limbs = byts / (16.0 * n)
    butterflies = limbs * (n // 2) * log_n
    alu = OPS_PER_BUTTERFLY * butterflies / (ms / 1e3) / 1e12
    gbs = byts / (ms / 1e3) / 1e9
    total = sum(v[1] for v in stages.values())
    bps = butterflies / (ms / 1e3) / 1e9
    peak = bfly_peak / 1e9 if bfly_peak else None
    return {"bound": "alu", "kernel": "ntt_fwd (forward NTT, pass A + pass B kernels)", "achieved": bps,
            "peak": peak, "unit": "G butterflies/s", "frac": bps / peak if peak else None,
            "peak_kind": "measured: hear_dbg_bfly_peak, the forward butterfly on register-resident radix-16 units "
                         "over the context's primes",
            "derived_alu_tintops": alu, "derived_alu_peak_tintops": ALU_PEAK_TOPS,
            "derived_alu_frac": alu / ALU_PEAK_TOPS,
            "traffic": committed_traffic(workload) if calls else None,
            "algorithmic_bytes_per_call": byts / calls * 2 if calls else None,
            "calls_per_step": calls_per_step, "avg_call_us": ms * 1e3 / (calls / 2),
            "hbm_achieved_gbs": gbs, "hbm_peak_gbs": hbm, "hbm_peak_kind": how, "hbm_frac": gbs / hbm,
            "stage_share": ms / total, "dominant_stage": name}


def ks_roofline(stages, psteps):
    """the key-switch inner product (every k_ks_inner launch form) against the HBM copy
    peak: algorithmic bytes (each stored key byte, each extended digit and each output
    residue once) over the stage time"""
    hbm, how = peaks()
    ks = [v for k, v in stages.items() if k.startswith("k_ks_inner")]
    if not ks:
        return None
    calls = sum(v[0] for v in ks)
    ms = sum(v[1] for v in ks)
    byts = sum(v[2] for v in ks)
    if ms <= 0:
        return None
    gbs = byts / (ms / 1e3) / 1e9
    total = sum(v[1] for v in stages.values())
    return {"bound": "hbm", "kernel": "k_ks_inner (key-switch inner product)",
            "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm, "peak_kind": how,
            "algorithmic_bytes_per_call": byts / calls, "calls_per_step": calls / psteps,
            "avg_call_us": ms * 1e3 / calls, "stage_share": ms / total}


# ------------------------------------------------------------------ oracle CPU timing
def oracle_sample(w, steps_keys, min_seconds=10.0, max_evals=40):
    """Time the CPU oracle (as it stands) evaluating whole ciphertexts of the workload: at
    least min_seconds of evaluations (a bounded sample, at most max_evals of them).
    Returns (inferences/s, cores, description)."""
    from oracle import oracle as O
    o = O.Oracle(w.log_n, w.q_bits, w.p_bits, w.sigma)
    cores = O.lib().or_set_threads(0)
    z, k = O.pack_clips(w.ct_clips(0), w.slots)
    keys = o.keygen(301, [O.galois_for_step(s, o.n) for s in steps_keys])
    ct = o.encrypt(keys.pk, z, 401, 0, 2.0 ** w.log2_scale)
    clips = min(w.clips_per_ct, w.n_clips)
    t0 = time.perf_counter()
    n = 0
    while True:
        o.evaluate(w.layers, ct, k, keys)
        n += 1
        el = time.perf_counter() - t0
        if el >= min_seconds or n >= max_evals:
            break
    return n * clips / el, cores, "%d whole ciphertext evaluation(s) of %d clip(s) each, %.1f s" % (n, clips, el)


# ------------------------------------------------------------------ GPU arm
class Setup:
    def __init__(self, H, w, stream, device, level=None, fc_n1=None, hoist_moddown=False, tune=False,
                 hoist_sums=False):
        """level: evaluate from ciphertexts dropped to this level (None = the top level);
        fc_n1 / hoist_moddown / hoist_sums: the FC evaluation form (hear_model_opts); tune: pick
        the form by timing the candidates at this batch size first (autotune.tune_fc)"""
        self.H, self.w = H, w
        self.ctx = H.hear_context_create(w.log_n, w.q_bits, w.p_bits, w.log2_scale, w.sigma, device)
        report = None
        if tune:
            # launch forms of the key-switch inner product / BSGS inner sums per batch bucket
            H.hear_ks_tune(self.ctx, 32, 3)
        self.ks_table = H.hear_ks_get_table(self.ctx)
        if tune:
            from paper_2104_09164_gb300.autotune import tune_fc
            (fc_n1, hoist_moddown, hoist_sums), report = tune_fc(H, self.ctx, w.layers, w.clip_dim, w.n_ct,
                                                                 w.slots, level, stream=stream)
        self.fc_form = {"fc_n1": fc_n1, "hoist_moddown": hoist_moddown, "hoist_sums": hoist_sums, "tuned": report}
        self.model = H.hear_model_create(self.ctx, w.layers, w.clip_dim, level, fc_n1=fc_n1,
                                         hoist_moddown=hoist_moddown, hoist_sums=hoist_sums)
        self.steps = H.hear_model_rotations(self.model)
        self.sk, self.pk, self.evk = H.hear_keygen(self.ctx, 301, self.steps)
        self.cts = [H.hear_encrypt_clips(self.ctx, self.pk, w.ct_clips(i), 401, i, stream) for i in range(w.n_ct)]
        if level is not None:
            top = self.cts
            self.cts = [H.hear_ciphertext_drop_level(c, level, stream) for c in top]
            for c in top:
                H.hear_ciphertext_destroy(c)
        self.clips_per_step = w.n_clips

    def step(self, stream):
        outs = self.H.hear_evaluate(self.model, self.evk, self.cts, stream)
        return outs

    def close(self):
        H = self.H
        for c in self.cts:
            H.hear_ciphertext_destroy(c)
        H.hear_model_destroy(self.model)
        H.hear_eval_keys_destroy(self.evk)
        H.hear_public_key_destroy(self.pk)
        H.hear_secret_key_destroy(self.sk)
        H.hear_context_destroy(self.ctx)


def run_gpu(S, steps, warmup, dist, torch, stream, sampler_device):
    H = S.H
    for _ in range(warmup):
        for o in S.step(stream):
            H.hear_ciphertext_destroy(o)
    torch.cuda.synchronize()
    dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    launches0 = H.hear_launch_count()
    with ClockSampler(sampler_device) as clk:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("hear_timed")   # ncu --nvtx-include "hear_timed/" selects these steps
        t_start.record(stream)
        for i in range(steps):
            ev[i][0].record(stream)
            outs = S.step(stream)
            ev[i][1].record(stream)
            for o in outs:
                H.hear_ciphertext_destroy(o)
        t_end.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    launches = H.hear_launch_count() - launches0
    dist.barrier()
    torch.cuda.synchronize()
    total_ms = t_start.elapsed_time(t_end)
    lat = sorted(a.elapsed_time(b) for a, b in ev)
    return total_ms, lat, launches, clk.summary()


def profile_stages(S, stream, torch, steps=2):
    H = S.H
    H.hear_profile_begin(S.ctx)
    for _ in range(steps):
        for o in S.step(stream):
            H.hear_ciphertext_destroy(o)
    torch.cuda.synchronize()
    return H.hear_profile_end(S.ctx), steps


def run_e2e(S, steps, warmup, torch, stream):
    """through hear_evaluate_host: H2D of the coefficient-domain inputs from pinned host
    memory, evaluation, D2H of the result ciphertexts -- every step"""
    H, w = S.H, S.w
    words = np.concatenate([H.hear_ciphertext_export(c).reshape(-1) for c in S.cts])
    pin_in = torch.empty(words.size, dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)
    pin_in[:] = words
    out0, lv, sc = H.hear_evaluate_host(S.model, S.evk, pin_in, len(S.cts), 2.0 ** w.log2_scale, None, stream)
    pin_out = torch.empty(out0.size, dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)
    for _ in range(warmup):
        H.hear_evaluate_host(S.model, S.evk, pin_in, len(S.cts), 2.0 ** w.log2_scale, pin_out, stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        H.hear_evaluate_host(S.model, S.evk, pin_in, len(S.cts), 2.0 ** w.log2_scale, pin_out, stream)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    return el, pin_in.nbytes, pin_out.nbytes


class Served:
    """one continuous-batching server over a Setup, with every batch-size graph captured;
    requests cycle through `n_distinct` different encrypted clips (distinct ciphertexts)"""

    def __init__(self, H, S, max_batch, n_slots, budget, n_distinct=8, stream=None):
        self.H, self.S = H, S
        w = S.w
        self.k = min(w.clips_per_ct, w.slots // w.clip_dim)
        self.scale = 2.0 ** w.log2_scale
        rng = np.random.default_rng(611)
        self.words = []
        for i in range(n_distinct):
            x = np.clip(rng.normal(0.0, 1.0, (self.k, w.clip_dim)), -1.0, 1.0)
            ct = H.hear_encrypt_clips(S.ctx, S.pk, x, 901, i, stream)
            self.words.append(H.hear_ciphertext_export(ct).reshape(-1))
            H.hear_ciphertext_destroy(ct)
        self.bufs = {}
        self.next = 0
        self.out_words = H.hear_evaluate_host(S.model, S.evk, self.words[0], 1, self.scale)[0].size
        self.srv = H.hear_server_create(S.model, S.evk, max_batch=max_batch, n_slots=n_slots,
                                        hbm_budget_bytes=budget)
        # capture the graph of every power-of-two batch size on every slot first
        ids = []
        for rep in range(2 * n_slots):
            b = max_batch
            while b >= 1:
                ids.append((H.hear_server_submit(self.srv, self.request(b), b, b * self.k, self.scale), b))
                b //= 2
                if len(ids) % 4 == 0:
                    self.drain_all(ids)
                    ids = []
        self.drain_all(ids)

    def request(self, n_ct):
        """words of a request of n_ct ciphertexts: consecutive distinct ciphertexts, the
        start rotating from request to request (buffers built once per (size, start))"""
        key = (n_ct, self.next)
        self.next = (self.next + 1) % len(self.words)
        buf = self.bufs.get(key)
        if buf is None:
            buf = self.bufs[key] = np.concatenate([self.words[(key[1] + i) % len(self.words)] for i in range(n_ct)])
        return buf

    def drain_all(self, ids):
        for rid, b in ids:
            self.H.hear_server_wait(self.srv, rid, b * self.out_words, timeout_ms=600000)

    def submit(self, n_clips):
        """-> (request id or None if the server refused it as busy, n_ct)"""
        n_ct = (n_clips + self.k - 1) // self.k
        try:
            return self.H.hear_server_submit(self.srv, self.request(n_ct), n_ct, n_clips, self.scale), n_ct
        except self.H.HearError as e:
            if e.code == self.H.HEAR_E_BUSY:
                return None, n_ct
            raise

    def poll(self, rid, n_ct):
        return self.H.hear_server_poll(self.srv, rid, n_ct * self.out_words) is not None

    def close(self):
        self.H.hear_server_destroy(self.srv)


def poisson_sweep(servers, mix, rates, seconds, seed, warmup=1.0):
    """Poisson requests of 1-8 clips (uniform) at each rate for warmup + seconds; each
    request goes to server i with probability mix[i].  Requests submitted during the first
    `warmup` seconds are served but not counted.  Per rate: offered and served inferences/s
    (clips of the counted requests over the time from the end of the warm-up to the last
    counted result), client-side p50/p99 latency (submit -> result read back), and the
    requests the server refused as busy (load shedding under overload)."""
    rng = np.random.default_rng(seed)
    out = []
    for lam in rates:
        t0 = time.perf_counter()
        t_count = t0 + warmup
        t_next = t0
        pend = [{} for _ in servers]     # per server, in submission order
        lat = [[] for _ in servers]
        clips = [0 for _ in servers]
        refused = [0 for _ in servers]
        offered = 0
        t_last = t_count

        def drain(window=32):
            nonlocal t_last
            # requests finish roughly in submission order: poll the oldest `window` per server
            for si, q in enumerate(pend):
                for rid in list(q)[:window]:
                    n_ct, n_clips, ts = q[rid]
                    if servers[si].poll(rid, n_ct):
                        now = time.perf_counter()
                        if ts >= t_count:
                            lat[si].append((now - ts) * 1e3)
                            clips[si] += n_clips
                            t_last = max(t_last, now)
                        del q[rid]
        while True:
            now = time.perf_counter()
            if now - t0 >= warmup + seconds:
                break
            while t_next <= now:
                n_clips = int(rng.integers(1, 9))
                si = int(rng.choice(len(servers), p=mix))
                ts = time.perf_counter()
                rid, n_ct = servers[si].submit(n_clips)
                if ts >= t_count:
                    offered += n_clips
                if rid is None:
                    refused[si] += ts >= t_count
                else:
                    pend[si][rid] = (n_ct, n_clips, ts)
                t_next += rng.exponential(1.0 / lam)
            drain()
            time.sleep(0.0002)
        while any(pend):
            drain()
            time.sleep(0.0002)
        span = max(t_last - t_count, 1e-9)
        row = {"rate_req_s": lam, "seconds": seconds, "warmup_s": warmup, "offered_inferences_s": offered / seconds,
               "inferences_s": sum(clips) / span, "per_net": []}
        for si, sv in enumerate(servers):
            l = sorted(lat[si])
            row["per_net"].append({"net": sv.S.w.name, "inferences_s": clips[si] / span, "requests": len(l),
                                   "refused_busy": refused[si],
                                   "p50_ms": l[len(l) // 2] if l else None,
                                   "p99_ms": l[min(len(l) - 1, int(0.99 * len(l)))] if l else None})
        if len(servers) == 1:
            row.update({k: row["per_net"][0][k] for k in ("requests", "refused_busy", "p50_ms", "p99_ms")})
            del row["per_net"]
        out.append(row)
    return out


def run_served(H, S, rates, seconds=4.0, warmup=1.0, max_batch=32, n_slots=3, seed=601, stream=None):
    """Poisson request stream against the continuous-batching server: each request carries
    1-8 clips (uniform) of the small network (4 clips per ciphertext -> 1 or 2 ciphertexts);
    returns per-rate throughput and p50/p99 latency (submit -> result read back)."""
    sv = Served(H, S, max_batch, n_slots, 96 << 30, stream=stream)
    try:
        return poisson_sweep([sv], [1.0], rates, seconds, seed, warmup)
    finally:
        sv.close()


def run_served_mix(H, stream, device, rates, seconds=4.0, warmup=1.0, seed=602, tune=True):
    """70% small / 30% large requests from one Poisson stream, each network served by its
    own continuous-batching server (own context, keys resident in HBM, HBM budget for the
    ciphertexts in flight); both servers' batches share the GPU."""
    from paper_2104_09164_gb300.workloads import make_workload
    Ss = Setup(H, make_workload("small"), stream, device, tune=tune)
    Sl = Setup(H, make_workload("large", 8), stream, device, tune=tune)
    servers = []
    try:
        servers.append(Served(H, Ss, 32, 2, 48 << 30, stream=stream))
        servers.append(Served(H, Sl, 8, 2, 96 << 30, stream=stream))
        return poisson_sweep(servers, [0.7, 0.3], rates, seconds, seed, warmup)
    finally:
        for sv in servers:
            sv.close()
        Ss.close()
        Sl.close()


# ------------------------------------------------------------------ skeleton CNN sections
# The paper's homomorphic convolution microbenchmark (Table 1; Xeon Platinum 8268, 16
# threads, SEAL 3.4, mean of 608 test samples): ordinary convolution ms, fast convolution
# pre / conv / post / total ms, speedup.  Context only: a different machine and library.
PAPER_TABLE1_MS = [
    (409, 65, 283, 42, 390, 1.1), (422, 49, 156, 37, 242, 1.7),
    (794, 68, 560, 47, 674, 1.2), (1416, 47, 408, 59, 514, 2.8),
    (985, 70, 550, 74, 694, 1.4), (1145, 47, 288, 50, 385, 3.0),
    (2173, 75, 856, 79, 1010, 2.2), (4251, 49, 507, 104, 660, 6.4),
]


def _time_range(H, m, evk, op0, op1, cts, n_samples, torch, stream, iters):
    """device time of operations [op0, op1) on resident inputs (CUDA events on `stream`)"""
    for o in H.hear_cnn_evaluate(m, evk, op0, op1, cts, n_samples, stream):
        H.hear_ciphertext_destroy(o)
    times = []
    for _ in range(iters):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        outs = H.hear_cnn_evaluate(m, evk, op0, op1, cts, n_samples, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        for o in outs:
            H.hear_ciphertext_destroy(o)
    times.sort()
    return times[len(times) // 2]


def simd_mad_lanes(primes, layers, level, n):
    """algorithmic multiply-pipe work of the slot-batched matrix products in mad.wide.u32
    lane operations: per FC row, input and residue the three Karatsuba partial products of two
    pieces (one mad.wide.u32 each below 2^42; a multiply-low / multiply-high pair, the same
    pipe time, for the 60-bit primes)"""
    total = 0.0
    for layer in layers:
        if layer[0] == "square":
            level -= 1
            continue
        if layer[0] == "fc":
            M, K = layer[1].shape
            used = 1
        else:
            M, K = 2 * layer[1].shape[0] * layer[2].shape[0], layer[1].shape[1]
            used = 2
        cost = 3 * (level + 1)
        total += float(M) * K * 2 * n * cost
        level -= used
    return total


SIMD_ROWS = (("small", 8192, 0), ("small", 8192, 3), ("large", 16384, 0))


def run_simd(H, torch, stream, device, plain_value, rows=SIMD_ROWS, steps=3, warmup=1):
    """slot-batched evaluation: one clip per slot, one ciphertext per feature; one step = the
    whole network over a full batch of clips resident in HBM (FC layers as scalar matrix
    products on the integer multiply-add pipe, no rotations)"""
    from paper_2104_09164_gb300.workloads import make_workload
    out = []
    for name, n_clips, level in rows:
        w = make_workload(name, n_clips)
        ctx = H.hear_context_create(w.log_n, w.q_bits, w.p_bits, w.log2_scale, w.sigma, device)
        m = H.hear_simd_model_create(ctx, w.layers, level)
        d_in, d_out, lin, lout = H.hear_simd_model_info(m)
        sk, pk, evk = H.hear_keygen(ctx, 301, [])
        t0 = time.perf_counter()
        b = H.hear_simd_encrypt(ctx, pk, w.clips, 401, level, stream=stream)
        torch.cuda.synchronize()
        enc_s = time.perf_counter() - t0
        for _ in range(warmup):
            H.hear_simd_batch_destroy(H.hear_simd_evaluate(m, evk, b, stream))
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        launches0 = H.hear_launch_count()
        with ClockSampler(device) as clk:
            ta, tb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ta.record(stream)
            for i in range(steps):
                ev[i][0].record(stream)
                y = H.hear_simd_evaluate(m, evk, b, stream)
                ev[i][1].record(stream)
                H.hear_simd_batch_destroy(y)
            tb.record(stream)
            torch.cuda.synchronize()
        launches = H.hear_launch_count() - launches0
        total_ms = ta.elapsed_time(tb)
        lat = sorted(x.elapsed_time(y) for x, y in ev)
        H.hear_profile_begin(ctx)
        y = H.hear_simd_evaluate(m, evk, b, stream)
        torch.cuda.synchronize()
        prof = H.hear_profile_end(ctx)
        logits = H.hear_simd_decrypt(ctx, sk, y, n_clips)
        err = float(np.max(np.abs(logits - w.fp64_forward(w.clips))))
        H.hear_simd_batch_destroy(y)
        gemm_ms = prof.get("k_simd_fc", (0, 0.0, 0.0))[1]
        lanes = simd_mad_lanes(H.hear_context_primes(ctx), w.layers, lin, 1 << w.log_n)
        probe = H.hear_dbg_imad_peak(ctx, 0) / 1e12
        peak = MAD_WIDE_PEAK_TOPS
        achieved = lanes / (gemm_ms / 1e3) / 1e12 if gemm_ms else None
        # end to end: coefficient-domain inputs from pinned host memory, result read back
        words = H.hear_simd_batch_export(b).reshape(-1)
        pin_in = torch.empty(words.size, dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)
        pin_in[:] = words
        del words
        scale = H.hear_simd_batch_info(b)[2]
        o0 = H.hear_simd_evaluate_host(m, evk, pin_in, scale, None, stream)[0]
        pin_out = torch.empty(o0.size, dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)
        torch.cuda.synchronize()
        e2e_times = []   # median of single steps: the host link's rate varies from step to step
        for _ in range(5):
            t0 = time.perf_counter()
            H.hear_simd_evaluate_host(m, evk, pin_in, scale, pin_out, stream)
            torch.cuda.synchronize()
            e2e_times.append(time.perf_counter() - t0)
        e2e_s = sorted(e2e_times)[2]
        v = steps * n_clips / (total_ms / 1e3)
        out.append({"workload": describe(w).split(",")[0] + ", FC/x^2 network of the plain path, %d clips one per "
                                "slot, %d input ciphertexts (one per feature), input level %d" % (n_clips, d_in, lin),
                    "value": v, "unit": UNIT, "ms_per_step": total_ms / steps, "steps": steps,
                    "p50_ms": lat[len(lat) // 2], "gpu_launches": launches, "clocks": clk.summary(),
                    "vs_plain": v / plain_value if plain_value else None,
                    "max_abs_err_vs_fp64": err, "encrypt_s": enc_s,
                    "e2e": {"value": n_clips / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(pin_in.nbytes),
                            "d2h_bytes_per_step": int(pin_out.nbytes)},
                    "roofline": {"bound": "alu", "kernel": "k_simd_fc (scalar matrix product, mad.wide.u32)",
                                 "achieved": achieved, "peak": peak, "unit": "T mad.wide.u32 lane-ops/s",
                                 "frac": achieved / peak if achieved else None, "traffic": None,
                                 "peak_kind": "derived: 152 SMs x 32 lanes/clk x 2.07 GHz (each partial product "
                                              "holds the multiply pipe 4 cycles per warp instruction, ncu)",
                                 "probe_tops": probe},
                    "stages_ms_per_step": {k: v_[1] for k, v_ in sorted(prof.items(), key=lambda kv: -kv[1][1])[:6]}})
        del pin_in, pin_out
        H.hear_simd_batch_destroy(b)
        H.hear_simd_model_destroy(m)
        H.hear_eval_keys_destroy(evk)
        H.hear_public_key_destroy(pk)
        H.hear_secret_key_destroy(sk)
        H.hear_context_destroy(ctx)
    return out


def run_ragged(H, torch, stream, device, tune=True, n_req=64, seed=603, steps=3):
    """ragged mixed batch: n_req requests of U{1..32} clips, 70 % for the small network
    (N = 2^14, 4 clips per ciphertext) and 30 % for the large one (N = 2^15, 8 per ciphertext),
    both networks evaluated by ONE CUDA-graph launch (hear_multi) against the same two
    evaluations launched one after the other"""
    from paper_2104_09164_gb300.workloads import make_workload
    rng = np.random.default_rng(seed)
    clips = rng.integers(1, 33, n_req)
    small = rng.random(n_req) < 0.7
    n_s, n_l = int(clips[small].sum()), int(clips[~small].sum())
    Ss = Setup(H, make_workload("small", n_s), stream, device, tune=tune)
    Sl = Setup(H, make_workload("large", n_l), stream, device, tune=tune)
    mu = H.hear_multi_create([Ss.model, Sl.model], [Ss.evk, Sl.evk], [len(Ss.cts), len(Sl.cts)],
                             [2.0 ** 40, 2.0 ** 40])
    try:
        cts = Ss.cts + Sl.cts

        def one():
            for o in H.hear_multi_evaluate(mu, cts, stream):
                H.hear_ciphertext_destroy(o)

        def two():
            for S in (Ss, Sl):
                for o in H.hear_evaluate(S.model, S.evk, S.cts, stream):
                    H.hear_ciphertext_destroy(o)

        res = {}
        for name, fn in (("one_launch", one), ("two_launches", two)):
            fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            res[name] = e0.elapsed_time(e1) / steps
        return {"workload": "%d requests of 1-32 clips: %d small-network clips (%d ciphertexts, N=2^14) and %d "
                            "large-network clips (%d ciphertexts, N=2^15)" % (n_req, n_s, len(Ss.cts), n_l, len(Sl.cts)),
                "value": (n_s + n_l) / (res["one_launch"] / 1e3), "unit": UNIT, "ms_per_step": res["one_launch"],
                "two_launches_ms": res["two_launches"], "steps": steps,
                "fc_form": {"small": {k: v for k, v in Ss.fc_form.items() if k != "tuned"},
                            "large": {k: v for k, v in Sl.fc_form.items() if k != "tuned"}}}
    finally:
        H.hear_multi_destroy(mu)
        Ss.close()
        Sl.close()


def run_conv_table(H, torch, stream, device, rows, iters=5):
    from paper_2104_09164_gb300.workloads import CONV_BENCH_PARAMS, TABLE1_LAYERS, conv_bench_layer
    log_n, qb, pb = CONV_BENCH_PARAMS
    ctx = H.hear_context_create(log_n, qb, pb, 40.0, 3.2, device)
    out = []
    for idx in rows:
        row = {"network": TABLE1_LAYERS[idx][0], "layer": TABLE1_LAYERS[idx][1]}
        for fast in (False, True):
            spec, xs = conv_bench_layer(idx, fast)
            t0 = time.perf_counter()
            m = H.hear_cnn_create(ctx, spec)
            build_s = time.perf_counter() - t0
            ops = H.hear_cnn_ops(m)
            sk, pk, evk = H.hear_keygen(ctx, 301, H.hear_cnn_rotations(m))
            cts = [H.hear_encrypt(ctx, pk, xs[0][i], 2.0 ** 40, 401, i, stream) for i in range(xs.shape[1])]
            if not fast:
                ms = _time_range(H, m, evk, 0, 1, cts, 1, torch, stream, iters)
                row.update({"n_in": ops[0]["n_in"], "n_out": ops[0]["n_out"], "ordinary_ms": ms,
                            "ordinary_keyswitch": ops[0]["n_keyswitch"], "ordinary_build_s": build_s})
            else:
                # chain the stages once to get each stage's resident input
                packed = H.hear_cnn_evaluate(m, evk, 0, 1, cts, 1, stream)
                conv = H.hear_cnn_evaluate(m, evk, 1, 2, packed, 1, stream)
                pre = _time_range(H, m, evk, 0, 1, cts, 1, torch, stream, iters)
                mid = _time_range(H, m, evk, 1, 2, packed, 1, torch, stream, iters)
                post = _time_range(H, m, evk, 2, 3, conv, 1, torch, stream, iters)
                whole = _time_range(H, m, evk, 0, 3, cts, 1, torch, stream, iters)
                row.update({"n_P": ops[0]["n_in"] // ops[0]["n_out"], "pre_ms": pre, "conv_ms": mid,
                            "post_ms": post, "fast_total_ms": whole, "fast_build_s": build_s,
                            "fast_keyswitch": sum(o["n_keyswitch"] for o in ops)})
                for h in packed + conv:
                    H.hear_ciphertext_destroy(h)
            for h in cts:
                H.hear_ciphertext_destroy(h)
            H.hear_eval_keys_destroy(evk)
            H.hear_public_key_destroy(pk)
            H.hear_secret_key_destroy(sk)
            H.hear_cnn_destroy(m)
        row["speedup"] = row["ordinary_ms"] / row["fast_total_ms"]
        p = PAPER_TABLE1_MS[idx]
        row["paper_cpu_ms"] = {"ordinary": p[0], "pre": p[1], "conv": p[2], "post": p[3], "total": p[4],
                               "speedup": p[5]}
        out.append(row)
    H.hear_context_destroy(ctx)
    return out


def run_cnn(H, torch, stream, device, batches=(1, 16), iters=5):
    """the paper-shaped 1D-CNN-64 (2 x 32 x 15 inputs, N = 2^15): whole encrypted network"""
    from paper_2104_09164_gb300.workloads import cnn_spec, make_cnn
    from paper_2104_09164_gb300.autotune import tune_cnn
    net = make_cnn("cnn1d64", n_samples=max(batches))
    spec = cnn_spec(net)     # as trained: the library collapses it
    ctx = H.hear_context_create(net.log_n, net.q_bits, net.p_bits, net.log2_scale, net.sigma, device)
    t0 = time.perf_counter()
    strategies, tune_report = tune_cnn(H, ctx, spec, net.slots, len(net.q_bits) - 1, iters=3, stream=stream)
    tune_s = time.perf_counter() - t0
    # default strategies (hybrid, n1 = min(4, block shifts)) for comparison
    md = H.hear_cnn_create(ctx, spec)
    m = H.hear_cnn_create(ctx, spec, strategies)
    ops = H.hear_cnn_ops(m)
    steps = sorted(set(H.hear_cnn_rotations(m)) | set(H.hear_cnn_rotations(md)))
    sk, pk, evk = H.hear_keygen(ctx, 301, steps)
    cts = [H.hear_cnn_encrypt(ctx, pk, m, clip, 401, s, stream)[0] for s, clip in enumerate(net.clips)]
    default_ms = _time_range(H, md, evk, 0, len(ops), cts[:1], 1, torch, stream, iters)
    H.hear_cnn_destroy(md)
    res = {"workload": "1D-CNN-64 (conv 2->64->128->256, 3 taps, quadratic activations, average / global "
                       "pooling, FC 256->2; fast convolution in conv2 / conv3), 2x32x15 synthetic skeleton "
                       "clips, RNS-CKKS N=2^15, q=60+14x40 bits, p=60+60 bits",
           "ops": len(ops), "keyswitch_per_sample": sum(o["n_keyswitch"] for o in ops),
           "strategies": {"tuned": [r["best"] for r in tune_report], "tune_s": tune_s, "layers": tune_report,
                          "default_batch1_ms": default_ms},
           "batches": []}
    for b in batches:
        H.hear_profile_begin(ctx)
        for o in H.hear_cnn_evaluate(m, evk, 0, len(ops), cts[:b], b, stream):
            H.hear_ciphertext_destroy(o)
        torch.cuda.synchronize()
        st = H.hear_profile_end(ctx)
        ms = _time_range(H, m, evk, 0, len(ops), cts[:b], b, torch, stream, iters)
        res["batches"].append({"samples": b, "ms": ms, "inferences_s": b / (ms / 1e3),
                               "stages_ms": {k: v[1] for k, v in sorted(st.items(), key=lambda kv: -kv[1][1])[:6]}})
    for h in cts:
        H.hear_ciphertext_destroy(h)
    H.hear_eval_keys_destroy(evk)
    H.hear_public_key_destroy(pk)
    H.hear_secret_key_destroy(sk)
    H.hear_cnn_destroy(m)
    H.hear_context_destroy(ctx)
    return res


def main_gpu(a):
    import torch
    dist = Dist()
    device = dist.local if dist.world > 1 else 0
    torch.cuda.set_device(device)
    from paper_2104_09164_gb300.build import build
    build()
    from paper_2104_09164_gb300 import hear as H
    from paper_2104_09164_gb300.workloads import make_workload
    stream = torch.cuda.Stream(device=device)
    w = make_workload(a.workload, a.clips)
    if a.fc_form:
        f = [int(x) for x in a.fc_form.split(",")] + [0]
        S = Setup(H, w, stream, device, fc_n1=f[0], hoist_moddown=bool(f[1]), hoist_sums=bool(f[2]))
    else:
        S = Setup(H, w, stream, device, tune=not a.no_fc_tune)
    total_ms, lat, launches, clocks = run_gpu(S, a.steps, a.warmup, dist, torch, stream, device)
    total_ms = dist.max(total_ms)
    value = replica_value(dist.world, a.steps, S.clips_per_step, total_ms)
    stages, psteps = profile_stages(S, stream, torch)
    e2e_s, bi, bo = run_e2e(S, max(3, a.steps // 2), 1, torch, stream)
    e2e_value = replica_value(dist.world, max(3, a.steps // 2), S.clips_per_step, dist.max(e2e_s) * 1e3)
    result = None
    if dist.rank == 0:
        ntt = {k: v for k, v in stages.items() if k.startswith("ntt")}
        nl_ntt = sum(v[0] for v in ntt.values())
        ms_ntt = sum(v[1] for v in ntt.values())
        by_ntt = sum(v[2] for v in ntt.values())
        total_stage_ms = sum(v[1] for v in stages.values())
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": total_ms / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": describe(w), "workload_short": describe_short(w),
                       "parallelism": "replicas" if dist.world > 1 else "single",
                       "l2": "no flush: the per-step working set (switching keys %.0f MB plus plaintext "
                             "diagonals) is larger than the 129 MB L2" % _key_mb(w, len(S.steps))},
            "p50_ms": lat[len(lat) // 2], "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo},
            "roofline": roofline(stages, psteps, w.log_n, w.name if a.clips is None else w.name + "_%d" % a.clips,
                                 H.hear_dbg_bfly_peak(S.ctx)),
            "roofline_keyswitch": ks_roofline(stages, psteps),
            "ntt": {"achieved_gbs": by_ntt / (ms_ntt / 1e3) / 1e9 if ms_ntt else None,
                    "launches_per_step": nl_ntt / psteps, "share": ms_ntt / total_stage_ms},
            "stages_ms_per_step": {k: v[1] / psteps for k, v in sorted(stages.items(), key=lambda kv: -kv[1][1])},
            # algorithmic bytes / stage time (each residue a stage must read or write, once)
            "stages_algorithmic_gbs": {k: v[2] / (v[1] / 1e3) / 1e9 for k, v in stages.items() if v[1] > 0},
            "stages_launches_per_step": {k: v[0] / psteps for k, v in stages.items()},
            "clocks": clocks, "gpu_launches": launches,
        }
        # the NTT launch-variant table this run used (pin it with HEAR_NTT_TABLE to profile
        # the same kernels)
        result["config"]["ntt_table"] = H.hear_ntt_get_table(S.ctx)
        # the FC evaluation form (baby steps, hoisted ModDown) and how it was chosen
        result["config"]["fc_form"] = S.fc_form
        # the key-switch / inner-sum launch forms (pin with HEAR_KS_TABLE to profile them)
        result["config"]["ks_table"] = S.ks_table
        # kernels captured with programmatic dependent launch so far (HEAR_PDL=0: none)
        result["config"]["pdl_launches_captured"] = H.hear_pdl_launch_count()
    serving = result is not None and not a.no_served and a.workload == "small" and a.clips is None and dist.world == 1
    if serving:
        if a.c5:
            rates, mix_rates, secs, warm = C5_RATES, C5_RATES, C5_SECONDS, C5_WARMUP
        else:
            rates = [float(x) for x in a.rates.split(",")]
            mix_rates = [float(x) for x in a.mix_rates.split(",")]
            secs, warm = a.served_seconds, a.served_warmup
        key = "served_c5" if a.c5 else "served"
        result[key] = {"workload": "small network, Poisson arrivals, 1-8 clips per request (8 distinct encrypted "
                                   "clips cycled), continuous batching (max 32 ciphertexts, 3 batches in flight)",
                       "note": "latency = client submit -> result read back (host); %g s per rate after a %g s "
                               "warm-up that is not counted" % (secs, warm),
                       "sweep": run_served(H, S, rates, secs, warm, stream=stream)}
        result[key + "_mix" if a.c5 else "served_mix"] = {
            "workload": "70% small (N=2^14) / 30% large (N=2^15) requests of 1-8 clips from one Poisson "
                        "stream; one continuous-batching server per network (max batch 32 / 8 "
                        "ciphertexts, 2 batches in flight each), both on one GPU",
            "note": "latency = client submit -> result read back (host), per rate and network",
            "sweep": run_served_mix(H, stream, device, mix_rates, secs, warm, tune=not a.no_fc_tune)}
    if not a.no_batched and a.workload == "small" and a.clips is None:
        S.close()
        wl = make_workload("large")
        SL = Setup(H, wl, stream, device, tune=not a.no_fc_tune)
        bsteps = max(3, a.steps // 4)
        tms, blat, bl, bclk = run_gpu(SL, bsteps, 2, dist, torch, stream, device)
        tms = dist.max(tms)
        bst, bps = profile_stages(SL, stream, torch, 1)
        if result is not None:
            result["batched"] = {"workload": describe(wl), "value": replica_value(dist.world, bsteps, SL.clips_per_step, tms),
                                 "unit": UNIT, "ms_per_step": tms / bsteps, "steps": bsteps,
                                 "p50_ms": blat[len(blat) // 2], "gpu_launches": bl, "clocks": bclk,
                                 "fc_form": SL.fc_form, "ks_table": SL.ks_table,
                                 "stages_ms_per_step": {k: v[1] / bps for k, v in
                                                        sorted(bst.items(), key=lambda kv: -kv[1][1])[:8]},
                                 # algorithmic bytes / stage time (HBM roofline of each stage)
                                 "stages_algorithmic_gbs": {k: v[2] / (v[1] / 1e3) / 1e9 for k, v in
                                                            sorted(bst.items(), key=lambda kv: -kv[1][1])[:8]
                                                            if v[1] > 0}}
            result["batched"]["vs_plain"] = result["batched"]["value"] / result["value"]
        SL.close()
    else:
        S.close()
    if result is not None and not a.no_batched and a.workload == "small" and a.clips is None and dist.world == 1:
        # the same small network batched: clips packed 4 per ciphertext, many ciphertexts per
        # launch (one CUDA-graph replay per step), against the plain one-clip-per-launch path
        rows = []
        # the FC form tuned for each batch size, and the default form at 512 clips
        for n_clips, tune in ((128, True), (512, True), (512, False)):
            wb = make_workload("small", n_clips)
            SB = Setup(H, wb, stream, device, tune=tune and not a.no_fc_tune)
            bsteps = 5
            tms, blat, bl, bclk = run_gpu(SB, bsteps, 2, dist, torch, stream, device)
            v = bsteps * SB.clips_per_step / (tms / 1e3)
            rows.append({"clips": n_clips, "ciphertexts": wb.n_ct, "fc_n1": SB.fc_form["fc_n1"],
                         "ks_table": SB.ks_table,
                         "hoist_moddown": SB.fc_form["hoist_moddown"], "fc_tuned": SB.fc_form["tuned"] is not None,
                         "value": v, "unit": UNIT,
                         "ms_per_step": tms / bsteps, "p50_ms": blat[len(blat) // 2], "gpu_launches": bl,
                         "clocks": bclk, "vs_plain": v / result["value"]})
            SB.close()
        result["batched_small"] = {"workload": "small network (as the plain path), batches of 128 / 512 clips "
                                               "in 32 / 128 ciphertexts per launch, FC form tuned per batch "
                                               "size; last row: the default FC form", "rows": rows}
    if result is not None and not a.no_min_level and a.workload == "small" and a.clips is None and dist.world == 1:
        # minimal start level: inputs dropped to the depth of the network (3 of 7 levels for
        # the small network, 5 of 14 for the large one); the same networks and parameters
        ms = {}
        for name, level, steps in (("small", 3, a.steps), ("large", 5, max(3, a.steps // 4))):
            wl = make_workload(name)
            SM = Setup(H, wl, stream, device, level, tune=not a.no_fc_tune)
            tms, mlat, ml, mclk = run_gpu(SM, steps, 2, dist, torch, stream, device)
            ms[name] = {"workload": describe(wl), "start_level": level, "fc_form": SM.fc_form,
                        "ks_table": SM.ks_table,
                        "value": steps * SM.clips_per_step / (tms / 1e3), "unit": UNIT,
                        "ms_per_step": tms / steps, "p50_ms": mlat[len(mlat) // 2],
                        "p99_ms": mlat[min(len(mlat) - 1, int(0.99 * len(mlat)))], "gpu_launches": ml,
                        "clocks": mclk}
            SM.close()
        result["min_start_level"] = ms
    if result is not None and not a.no_batched and a.workload == "small" and a.clips is None and dist.world == 1:
        result["ragged_mix"] = run_ragged(H, torch, stream, device, tune=not a.no_fc_tune)
    if result is not None and not a.no_simd and a.workload == "small" and a.clips is None and dist.world == 1:
        result["batched_simd"] = {
            "note": "slot-batched form: the batch's clips one per slot, FC layers as plaintext-scalar "
                    "matrix products over the per-feature ciphertexts (no rotations); same parameters, "
                    "networks and accuracy bound; value = clips / step time",
            "rows": run_simd(H, torch, stream, device, result["value"],
                             SIMD_ROWS if a.simd_rows == "all" else
                             [SIMD_ROWS[int(i)] for i in a.simd_rows.split(",")])}
    if result is not None and not a.no_cnn and dist.world == 1:
        rows = list(range(8)) if a.conv_rows == "all" else [int(x) for x in a.conv_rows.split(",")]
        result["conv_table1"] = {
            "note": "Table 1 layers at N=2^14 (q=60+7x40, p=60), inputs at the top level, one sample, "
                    "synthetic weights, median device ms of 5 runs; paper_cpu_ms = the paper's Xeon/SEAL "
                    "numbers (context, other hardware)",
            "rows": run_conv_table(H, torch, stream, device, rows)}
        result["cnn"] = run_cnn(H, torch, stream, device)
    if result is not None and not a.no_cpu_baseline and dist.world == 1:
        v, cores, desc = oracle_sample(w, H_steps_for(w))
        result["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}
    if result is not None:
        path = write_sections(result, a.sections_out)
        print(json.dumps(headline(result, path), separators=(",", ":")), flush=True)
    dist.close()


def _r(x, nd=4):
    """x rounded to nd significant digits (None stays None)"""
    if x is None:
        return None
    return float("%.*g" % (nd, x))


def write_sections(result, path):
    """the full result (served sweeps, per-stage tables, CNN rows, ...) as one JSON file;
    returns its path relative to the repository (None if it could not be written)"""
    if not path:
        return None
    full = path if os.path.isabs(path) else os.path.join(ROOT, path)
    try:
        os.makedirs(os.path.dirname(full), exist_ok=True)
        with open(full, "w") as f:
            json.dump(result, f, indent=1)
    except OSError:
        return None
    return os.path.relpath(full, ROOT)


def headline(result, sections_path):
    """the one short JSON line bench.py prints last: the metric on the quoted workload,
    its end-to-end form, the dominant kernel's roofline, the CPU baseline, the clocks and
    one number per section (the whole sections are in the file `sections_path`)"""
    keep = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
            "scaling", "vs_baseline", "dtype", "data", "p50_ms", "p99_ms", "gpu_launches")
    h = {k: result[k] for k in keep if k in result}
    for k in ("value", "ms_per_step", "p50_ms", "p99_ms"):
        h[k] = _r(h.get(k), 6)
    cfg = result["config"]
    ff = cfg["fc_form"]
    h["config"] = {"workload": cfg.get("workload_short", cfg["workload"]), "parallelism": cfg["parallelism"],
                   "l2": "no flush: working set > L2",
                   "fc_form": "n1=%s%s%s" % (ff.get("fc_n1"), " hoist_moddown" if ff.get("hoist_moddown") else "",
                                             " hoist_sums" if ff.get("hoist_sums") else ""),
                   "sections": sections_path}
    e = result["e2e"]
    h["e2e"] = {"value": _r(e["value"], 6), "unit": e["unit"], "h2d_bytes_per_step": e["h2d_bytes_per_step"],
                "d2h_bytes_per_step": e["d2h_bytes_per_step"]}
    rf = result["roofline"]
    h["roofline"] = {k: (_r(rf.get(k)) if isinstance(rf.get(k), float) else rf.get(k))
                     for k in ("bound", "achieved", "peak", "unit", "frac", "traffic", "hbm_peak_gbs", "hbm_frac",
                               "derived_alu_frac") if k in rf}
    h["roofline"]["kernel"] = "ntt_fwd"
    h["roofline"]["peak_kind"] = "measured bfly probe" if rf.get("peak") else None
    if result.get("roofline_keyswitch"):
        kr = result["roofline_keyswitch"]
        h["roofline_keyswitch"] = {k: (_r(kr[k]) if isinstance(kr[k], float) else kr[k])
                                   for k in ("bound", "achieved", "peak", "unit", "frac")}
    if "cpu_baseline" in result:
        cb = result["cpu_baseline"]
        h["cpu_baseline"] = {"value": _r(cb["value"]), "unit": cb["unit"], "cores": cb["cores"], "kind": cb["kind"],
                             "sample": cb["sample"]}
    ck = result["clocks"]
    h["clocks"] = {"sm_mhz": ck.get("sm_mhz"), "sm_max_mhz": ck.get("sm_max_mhz"), "reasons": ck.get("reasons")}
    s = {}
    if "batched" in result:
        b = result["batched"]
        s["batched_large"] = {"value": _r(b["value"]), "vs_plain": _r(b["vs_plain"], 3)}
    if "batched_small" in result:
        best = max(result["batched_small"]["rows"], key=lambda r: r["value"])
        s["batched_small"] = {"clips": best["clips"], "value": _r(best["value"]), "vs_plain": _r(best["vs_plain"], 3)}
    for key in ("served", "served_c5"):
        if key in result:
            rows = result[key]["sweep"]
            top = max(rows, key=lambda r: r["inferences_s"])
            s[key] = {"rate_req_s": top["rate_req_s"], "value": _r(top["inferences_s"]),
                      "vs_plain": _r(top["inferences_s"] / result["value"], 3), "p99_ms": _r(top.get("p99_ms"))}
    for key in ("served_mix", "served_c5_mix"):
        if key in result:
            rows = result[key]["sweep"]
            top = max(rows, key=lambda r: r["inferences_s"])
            s[key] = {"rate_req_s": top["rate_req_s"], "value": _r(top["inferences_s"])}
    if "ragged_mix" in result:
        s["ragged_mix"] = {"value": _r(result["ragged_mix"]["value"])}
    if "min_start_level" in result:
        s["min_start_level"] = {k: _r(v["value"]) for k, v in result["min_start_level"].items()}
    if "batched_simd" in result:
        r = result["batched_simd"]["rows"][0]
        s["batched_simd"] = {"value": _r(r["value"]), "vs_plain": _r(r["vs_plain"], 3),
                             "frac": _r(r["roofline"]["frac"], 3)}
    if "cnn" in result:
        s["cnn1d64_batch1_ms"] = _r(result["cnn"]["batches"][0]["ms"])
    if "conv_table1" in result:
        s["conv_table1_max_speedup"] = _r(max(r["speedup"] for r in result["conv_table1"]["rows"]), 3)
    h["summary"] = s
    return h


def _key_mb(w, n_rot):
    n = 1 << w.log_n
    nq, npp = len(w.q_bits), len(w.p_bits)
    dnum = (nq + npp - 1) // npp
    return (n_rot + 1) * dnum * 2 * (nq + npp) * n * 8 / 1e6


def H_steps_for(w):
    from oracle import oracle as O
    k = w.slots // w.clip_dim
    return O.rotation_steps(w.layers, w.clip_dim, k)


def main_reference(a):
    """The oracle on the host cores, same metric and workload, each step one whole
    ciphertext of the workload (bounded sample)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2104_09164_gb300.workloads import make_workload
    from oracle import oracle as O
    w = make_workload(a.workload)
    o = O.Oracle(w.log_n, w.q_bits, w.p_bits, w.sigma)
    cores = O.lib().or_set_threads(0)
    z, k = O.pack_clips(w.ct_clips(0), w.slots)
    steps = O.rotation_steps(w.layers, w.clip_dim, k)
    keys = o.keygen(301, [O.galois_for_step(s, o.n) for s in steps])
    ct = o.encrypt(keys.pk, z, 401, 0, 2.0 ** w.log2_scale)
    clips = min(w.clips_per_ct, w.n_clips)
    for _ in range(a.warmup):
        o.evaluate(w.layers, ct, k, keys)
    lat = []
    t0 = time.perf_counter()
    for _ in range(a.steps):
        t1 = time.perf_counter()
        o.evaluate(w.layers, ct, k, keys)
        lat.append((time.perf_counter() - t1) * 1e3)
    el = time.perf_counter() - t0
    value = a.steps * clips / el
    lat.sort()
    desc = "one ciphertext (%d clip(s)) of the %s workload per step" % (clips, w.name)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": el * 1e3 / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": describe(w)}, "p50_ms": lat[len(lat) // 2],
        "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


if __name__ == "__main__":
    args = parse()
    if args.impl == "reference":
        main_reference(args)
    else:
        main_gpu(args)
