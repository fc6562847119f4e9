"""RowSel benchmark on GB300: queries/s vs batch, DB GB/s, per-path comparison.

One step = one batched RowSel (all of its work: every limb, slot, client and
column) over device-resident synthetic inputs through the C ABI
(gpir_rowsel_batch). Prints ONE JSON line (rank 0). The default workload is
the large database: N=4096, 2 limbs, D0=1024 x D1=128 (4 GiB in NTT form),
128 clients.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                  [--path auto|cudacore|imma|tc] [--impl gpir|reference]
  python bench.py --case rowsel|coltor|expand|pir [--batch B --d0 D0 --d1 D1
                  --n N --limbs L --path P --variant V --reps R ...]

--case runs one seeded synthetic problem of any shape: a fixed launch sequence
for profilers (ncu -k <kernel> -s <skip> -c <count>) and a quick timing.

With N > 1 (torchrun) every rank runs an independent replica of the workload
(RowSel needs no exchange between replicas); value = all ranks' queries / the
slowest rank's time.
"""

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402
from paper_2604_04696_gb300 import sizes  # noqa: E402

METRIC = "RowSel queries/s vs batch; DB GB/s; INT8-TC path vs plain path, bit-exact"
PATH_IDS = {"auto": 0, "cudacore": 1, "imma": 2, "tc": 4}
PATH_NAMES = {1: "cudacore", 2: "imma", 4: "tc"}
# Integer multiply-add lanes per SM (IMAD.WIDE.U32 issues at the full IMAD rate,
# measured 17.7e12/s on 152 SMs) and the recipe's maximum SM clock.
IMAD_PER_SM_CLK = 64
SM_MAX_MHZ = 2070.0
N_SMS = 152


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return {"hbm_gbs": float(p["hbm_gbs"]), "bf16_tflops": float(p["bf16_tflops"]),
                "bf16_tflops_sustained": float(p.get("bf16_tflops_sustained", p["bf16_tflops"])),
                "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


def workload_shape(name, batch=None):
    c = synth.config_shapes(name)
    B = batch if batch is not None else c["B"]
    if not isinstance(B, int):
        B = 32
    return dict(N=c["N"], L=c["L"], D0=c["D0"], D1=c["D1"], B=B, seed=c["seed"], primes=list(c["primes"]))


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline leg and --impl reference)
# ---------------------------------------------------------------------------

def _sample_slots(w, n_slots, seed):
    rng = np.random.default_rng(seed)
    return [(int(rng.integers(0, w["L"])), int(rng.integers(0, w["N"]))) for _ in range(n_slots)]


def _oracle_worker(w, slots):
    """Generate the inputs of `slots` (untimed), then run the oracle on them;
    returns (start, end) wall-clock stamps of the oracle part."""
    import oracle
    ct = synth.ct_slots(w["seed"], w["B"], w["D0"], w["L"], w["N"], w["primes"], slots)
    db = synth.db_slots(w["seed"], w["D0"], w["D1"], w["L"], w["N"], w["primes"], slots)
    t0 = time.time()
    for k, (l, _t) in enumerate(slots):
        oracle.rowsel(ct[:, :, :, None, k:k + 1], db[:, :, None, k:k + 1], [w["primes"][l]])
    return t0, time.time()


def host_cpu():
    """(usable cores, CPU model) of this host."""
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as fh:
                for line in fh:
                    if line.lower().startswith(("model name", "cpu part")):
                        model = line.split(":", 1)[1].strip()
                        break
        except Exception:
            model = "unknown"
    return cores, model


class OraclePool:
    """The oracle, as it stands, run over slot subsets on every host core: one
    spawned process per core (spawned, never forked from a CUDA process).
    time(w, slots) returns the wall time of the parallel oracle section."""

    def __init__(self, cores):
        import multiprocessing as mp
        self.cores = cores
        self.pool = mp.get_context("spawn").Pool(cores) if cores > 1 else None

    def time(self, w, slots):
        if self.pool is None:
            t0, t1 = _oracle_worker(w, slots)
            return t1 - t0
        chunks = [slots[k::self.cores] for k in range(self.cores)]
        chunks = [c for c in chunks if c]
        stamps = self.pool.starmap(_oracle_worker, [(w, c) for c in chunks])
        return max(e for _s, e in stamps) - min(s for s, _e in stamps)

    def close(self):
        if self.pool is not None:
            self.pool.close()
            self.pool.join()


def oracle_baseline(w, seconds_target=15.0):
    """cpu_baseline: the oracle on all host cores over a bounded slot sample
    (about `seconds_target` of wall time), plus a 1-core figure; both
    extrapolated from the sample to the whole batch (every limb and slot)."""
    cores, model = host_cpu()
    t_one = OraclePool(1).time(w, _sample_slots(w, 1, 3))
    total = w["L"] * w["N"]
    n1 = int(max(1, min(total, 0.4 * seconds_target / max(t_one, 1e-6))))
    dt1 = OraclePool(1).time(w, _sample_slots(w, n1, 5))
    pool = OraclePool(cores)
    try:
        n = int(max(cores, min(total, cores * seconds_target / max(t_one, 1e-6))))
        dt = pool.time(w, _sample_slots(w, n, 7))
    finally:
        pool.close()
    return {"value": w["B"] / (dt * total / n), "unit": "queries/s", "cores": cores, "kind": "oracle",
            "sample": "%d of %d (limb, slot) points on %d processes in %.1f s wall, extrapolated to the whole "
                      "batch" % (n, total, cores, dt),
            "one_core": {"value": w["B"] / (dt1 * total / n1), "unit": "queries/s",
                         "sample": "%d points in %.1f s on 1 core, extrapolated" % (n1, dt1)},
            "nproc": os.cpu_count(), "cpu_model": model}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = workload_shape(args.workload, args.batch)
    total_slots = w["L"] * w["N"]
    cores, model = host_cpu()
    t1 = OraclePool(1).time(w, _sample_slots(w, 1, 3))
    # per step: a slot sample sized so warm-up + steps stay within ~2.5 minutes of wall time
    per_step_budget = 150.0 / max(1, args.steps + args.warmup)
    n = int(max(cores, min(total_slots, cores * per_step_budget / max(t1, 1e-6))))
    pool = OraclePool(cores)
    try:
        for k in range(args.warmup):
            pool.time(w, _sample_slots(w, n, 1 + k))
        times = [pool.time(w, _sample_slots(w, n, 100 + s)) for s in range(args.steps)]
    finally:
        pool.close()
    step = statistics.mean(times)
    qps = w["B"] / (step * total_slots / n)
    sample = ("%d of %d (limb, slot) points per step on %d processes (one per host core), extrapolated to the whole "
              "batch" % (n, total_slots, cores))
    line = {
        "impl": "reference", "metric": METRIC, "value": qps, "unit": "queries/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step * 1e3 * total_slots / n,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64 (numpy)",
        "data": "synthetic", "config": cfg_dict(args.workload, w, "oracle", None),
        "cpu_baseline": {"value": qps, "unit": "queries/s", "cores": cores, "kind": "oracle", "sample": sample,
                         "nproc": os.cpu_count(), "cpu_model": model},
        "e2e": {"value": qps, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def cfg_dict(workload, w, path_name, variant):
    alg = sizes.rowsel_algorithmic_bytes(w["B"], w["D0"], w["D1"], w["N"], w["L"])
    return {"workload": workload, "N": w["N"], "limbs": w["L"], "D0": w["D0"], "D1": w["D1"],
            "batch": w["B"], "primes": w["primes"], "path": path_name, "variant": variant,
            "db_bytes": sizes.db_bytes(w["D0"], w["D1"], w["N"], w["L"]),
            "l2": "inputs larger than L2 (%.2f GB moved per step vs 129 MB L2); no flush" % (alg / 1e9)}


# ---------------------------------------------------------------------------
# GPU side
# ---------------------------------------------------------------------------

class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower().startswith("active"):
                        reasons.add(nm)
            except Exception:
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# kernel name -> (path id, source file, exact digit products per modular MAC)
KERNELS = {"rowsel_cc": (1, "rowsel_cc.cu", 1), "rowsel_imma": (2, "rowsel_imma.cu", 16),
           "tc_gemm": (4, "rowsel_tc.cu", 16), "tc_ingest": (4, "rowsel_tc.cu", 16),
           "tc_fused": (4, "rowsel_tc.cu", 16), "tc_cluster": (4, "rowsel_tc.cu", 16),
           "tc_tmem": (4, "rowsel_tmem.cu", 12), "tc_tmem_pair": (4, "rowsel_tmem.cu", 12)}
# tensor-core path variants that run the tensor-memory kernel (the variant
# table in rowsel_tc.cu): 12 digit products per modular MAC, the others 16
TMEM_VARIANT_IDS = (8, 9, 10, 11)


def path_products(path, variant):
    return 12 if path == 4 and variant in TMEM_VARIANT_IDS else 16


def kernel_src_hash(kernel):
    f = KERNELS[kernel][1]
    with open(os.path.join(ROOT, "paper_2604_04696_gb300", "csrc", f), "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def recorded_traffic(kernel, workload, batch):
    """DRAM bytes per launch from a committed ncu capture, or None when absent or
    when the kernel source changed since it was taken."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            t = json.load(fh)
    except Exception:
        return None
    e = t.get("%s/%s/B%d" % (kernel, workload, batch))
    if not e or e.get("src_sha") != kernel_src_hash(kernel):
        return None
    return e.get("dram_bytes_per_launch")


def kernel_roofline(name, w, ms, peaks, workload):
    """Roofline of one kernel: its algorithmic work per launch over its own
    average launch time (CUDA events on its launch stream)."""
    alg = sizes.rowsel_algorithmic_bytes(w["B"], w["D0"], w["D1"], w["N"], w["L"])
    macs = sizes.rowsel_modmacs(w["B"], w["D0"], w["D1"], w["N"], w["L"])
    s = ms / 1e3
    path_id, _, products = KERNELS[name]
    traffic = recorded_traffic(name, workload, w["B"])
    if name == "tc_ingest":
        b = sizes.query_ct_bytes(w["B"], w["D0"], w["N"], w["L"])
        a = b / s / 1e9
        return {"kernel": name, "bound": "hbm", "achieved": a, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": a / peaks["hbm_gbs"], "traffic": traffic,
                "note": "selection-ciphertext bytes (read once) per launch vs %s copy BW" % peaks["source"]}
    r = roofline(path_id, w, ms, peaks, workload, products)
    r["kernel"] = name
    r["traffic"] = traffic
    return r


def roofline(path_id, w, ms, peaks, workload, products=16):
    """Roofline of a RowSel step on one path. `products` is the number of exact
    fp16 digit products the tensor-core kernel spends per modular MAC (16 for
    the base-256 kernels, 12 for the tensor-memory kernel's 4 x 3 centred
    digits)."""
    alg = sizes.rowsel_algorithmic_bytes(w["B"], w["D0"], w["D1"], w["N"], w["L"])
    macs = sizes.rowsel_modmacs(w["B"], w["D0"], w["D1"], w["N"], w["L"])
    s = ms / 1e3
    t_hbm = alg / (peaks["hbm_gbs"] * 1e9)
    traffic = None
    if path_id == 4:
        flops = 2.0 * products * macs     # exact fp16 digit products per modular MAC
        t_c = flops / (peaks["bf16_tflops"] * 1e12)
        if t_c >= t_hbm:
            a = flops / s / 1e12
            return {"bound": "tensor", "achieved": a, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                    "frac": a / peaks["bf16_tflops"], "traffic": traffic,
                    "note": "fp16 digit-product flops (%d per modular MAC) vs %s cuBLAS bf16 burst "
                            "(fp16 and bf16 share one nominal dense rate)" % (products, peaks["source"])}
    elif path_id == 2:
        ops = 2.0 * 16 * macs         # 16 u8 x u8 products per modular MAC
        imma_peak = 151.0             # TOPS, measured mma.sync m16n8k32 u8 on this GB300 pool
        t_c = ops / (imma_peak * 1e12)
        if t_c >= t_hbm:
            a = ops / s / 1e12
            return {"bound": "tensor", "achieved": a, "peak": imma_peak, "unit": "TOPS",
                    "frac": a / imma_peak, "traffic": traffic,
                    "note": "u8 products (16 per modular MAC) vs measured mma.sync IMMA peak"}
    else:
        alu_peak = N_SMS * IMAD_PER_SM_CLK * SM_MAX_MHZ * 1e6
        t_c = macs / alu_peak
        if t_c >= t_hbm:
            a = macs / s / 1e12
            return {"bound": "alu", "achieved": a, "peak": alu_peak / 1e12, "unit": "T IMAD.WIDE/s",
                    "frac": a * 1e12 / alu_peak, "traffic": traffic,
                    "note": "one IMAD.WIDE.U32 per modular MAC; peak = 152 SMs x 64 lanes x 2070 MHz"}
    a = alg / s / 1e9
    return {"bound": "hbm", "achieved": a, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": a / peaks["hbm_gbs"],
            "traffic": traffic, "note": "algorithmic bytes (DB + cts read once, outputs written once) vs %s copy BW"
            % peaks["source"]}


class GpuWorkload:
    """One RowSel workload on this GPU: the database made resident and one
    batch of selection ciphertexts, all drawn on the device. With `shard` (a
    SlotShard) only that rank's slots are kept: the full tensors are drawn,
    sliced to the shard's compact [..., L, T] layout and dropped, so every rank
    holds exactly the values of the unsharded workload at its slots."""

    def __init__(self, g, torch, w, path_mask, shard=None):
        self.g, self.torch, self.w, self.shard = g, torch, w, shard
        N, L, D0, D1, B = w["N"], w["L"], w["D0"], w["D1"], w["B"]
        T = shard.T if shard else N
        self.T = T
        gen = g.gpir_params_create(N, w["primes"])              # the full ring: generator limb mapping
        self.params = g.gpir_params_create(T, w["primes"]) if shard else gen
        self.stream = torch.cuda.current_stream()
        db = torch.empty(D0 * D1 * L * N, dtype=torch.int32, device="cuda")
        g.gpir_fill_uniform(db, db.numel(), 0, w["seed"], synth.TAG_DB, gen, N, self.stream)
        if shard:
            db = shard.take(db.view(D0, D1, L, N))
        self.h = g.gpir_db_upload(self.params, D0, D1, db, True, path_mask, self.stream)
        del db
        ct = torch.empty(B * D0 * 2 * L * N, dtype=torch.int32, device="cuda")
        g.gpir_fill_uniform(ct, ct.numel(), 0, w["seed"], synth.TAG_CT, gen, N, self.stream)
        self.ct = shard.take(ct.view(B, D0, 2, L, N)).view(-1) if shard else ct
        del ct
        self.out = torch.empty(B * D1 * 2 * L * T, dtype=torch.int32, device="cuda")
        if shard:
            g.gpir_params_destroy(gen)
        torch.cuda.synchronize()
        torch.cuda.empty_cache()

    def step(self, path):
        self.g.gpir_rowsel_batch(self.h, self.w["B"], self.ct, self.out, path, self.stream)

    def time_steps(self, path, steps, warmup, barrier=None, clocks=None):
        torch = self.torch
        for _ in range(warmup):
            self.step(path)
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
        if barrier:
            barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(self.stream)
        for _ in range(steps):
            self.step(path)
        e1.record(self.stream)
        torch.cuda.synchronize()
        if barrier:
            barrier()
        clk = clocks.stop() if clocks else None
        self.g.gpir_sync(self.stream, 60000)
        return e0.elapsed_time(e1) / steps, clk

    def check_sample(self, n_slots=3):
        """Bit-exact check of a few sampled (limb, slot) points of this GPU's
        slots against the oracle."""
        import oracle
        w = self.w
        t0 = self.shard.t0 if self.shard else 0
        rng = np.random.default_rng(5)
        local = [(int(rng.integers(0, w["L"])), int(rng.integers(0, self.T))) for _ in range(n_slots)]
        slots = [(l, t0 + t) for l, t in local]
        ct = synth.ct_slots(w["seed"], w["B"], w["D0"], w["L"], w["N"], w["primes"], slots)
        db = synth.db_slots(w["seed"], w["D0"], w["D1"], w["L"], w["N"], w["primes"], slots)
        out = self.out.view(w["B"], w["D1"], 2, w["L"], self.T)
        for k, (l, t) in enumerate(local):
            want = oracle.rowsel(ct[:, :, :, None, k:k + 1], db[:, :, None, k:k + 1], [w["primes"][l]])[..., 0, 0]
            got = out[:, :, :, l, t].contiguous().cpu().numpy().view(np.uint32)
            if not np.array_equal(got, want):
                return False
        return True

    def e2e(self, path, steps, warmup):
        """Same metric through gpir_rowsel_batch_host: pinned host ct in, host out back,
        copies inside the timed region."""
        torch, g, w = self.torch, self.g, self.w
        ct_h = torch.empty(self.ct.numel(), dtype=torch.int32, pin_memory=True)
        ct_h.copy_(self.ct)
        out_h = torch.empty(self.out.numel(), dtype=torch.int32, pin_memory=True)
        for _ in range(warmup):
            g.gpir_rowsel_batch_host(self.h, w["B"], ct_h, out_h, path, self.stream)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(self.stream)
        for _ in range(steps):
            g.gpir_rowsel_batch_host(self.h, w["B"], ct_h, out_h, path, self.stream)
        e1.record(self.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        return ms, ct_h.numel() * 4, out_h.numel() * 4

    def kernel_times(self, path, steps):
        """Average device time per kernel of one step, from the library's
        CUDA-event trace on the launch stream."""
        g = self.g
        g.gpir_trace_enable(True)
        for _ in range(steps):
            self.step(path)
        recs = g.gpir_trace_read()
        g.gpir_trace_enable(False)
        tot = {}
        for name, ms in recs:
            tot.setdefault(name, []).append(ms)
        return {k: sum(v) / len(v) for k, v in tot.items()}, {k: len(v) // steps for k, v in tot.items()}

    def close(self):
        self.g.gpir_db_free(self.h)
        self.g.gpir_params_destroy(self.params)


def run_coltor(g, torch, B=32, D1=64, steps=10, warmup=3):
    """ColTor (the column tournament after RowSel) on the 32-client workload's
    RowSel output shape: B clients x D1 ciphertexts, N=4096, 2 limbs, one
    RGSW ciphertext per stage. Inputs are uniform residues drawn on the device
    (the arithmetic does not depend on their values). Roofline: the modular
    products of the NTT butterflies and the RGSW multiply-accumulate, each at
    least 3 IMAD (28-bit Shoup / Barrett), against 152 SMs x 64 IMAD lanes x
    2.07 GHz / 3."""
    c = synth.config_shapes("c2_rowsel")
    N, L, primes = c["N"], c["L"], list(c["primes"])
    params = g.gpir_params_create(N, primes)
    ell = g.gpir_coltor_gadget_digits(params)
    stages = D1.bit_length() - 1
    ct = torch.empty(B * D1 * 2 * L * N, dtype=torch.int32, device="cuda")
    rgsw = torch.empty(B * stages * 2 * ell * 2 * L * N, dtype=torch.int32, device="cuda")
    out = torch.empty(B * 2 * L * N, dtype=torch.int32, device="cuda")
    g.gpir_fill_uniform(ct, ct.numel(), 0, 9, synth.TAG_COLTOR, params, N)
    g.gpir_fill_uniform(rgsw, rgsw.numel(), 0, 9, synth.TAG_RGSW, params, N)
    st = torch.cuda.current_stream()
    for _ in range(warmup):
        g.gpir_coltor(params, B, D1, ct, rgsw, out, st.cuda_stream)
    st.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        g.gpir_coltor(params, B, D1, ct, rgsw, out, st.cuda_stream)
    e1.record(st)
    st.synchronize()
    g.gpir_sync(None, 60000)
    ms = e0.elapsed_time(e1) / steps
    g.gpir_params_destroy(params)
    logn = N.bit_length() - 1
    nodes = B * (D1 - 1)
    products = nodes * ((2 * L + 2 * ell * L) * (N // 2) * logn + 4 * ell * L * N)
    peak = 152 * 64 * 2.07e9 / 3 / 1e12
    achieved = products / (ms / 1e3) / 1e12
    ct_bytes = 2 * L * N * 4
    alg_bytes = ct_bytes * (B * D1 + B * stages * 2 * ell + B)
    return {"workload": "ColTor after the 32-client RowSel: %d clients x %d ciphertexts, N=%d, %d limbs, ell=%d, "
                        "%d stages" % (B, D1, N, L, ell, stages),
            "ms": ms, "queries_s": B / (ms / 1e3),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T modmul/s",
                         "frac": achieved / peak,
                         "note": "NTT butterflies + RGSW products (%.3g per step), 3 IMAD each, vs 152x64x2.07GHz/3; "
                                 "HBM: %.0f MB algorithmic, %.3f ms at the measured copy bandwidth"
                                 % (products, alg_bytes / 1e6, alg_bytes / 6652.3e9 * 1e3)}}


def run_expand(g, torch, B=32, D0=256, D1=64, steps=10, warmup=3):
    """ExpandQuery (the query-expansion tree before RowSel) on the 32-client
    workload: each client's query expands into D0 + log2(D1) ell ciphertexts
    (the RowSel selection vector plus the RGSW material of ColTor), J =
    ceil(log2 of that) stages, N=4096, 2 limbs, one evaluation key per stage.
    Inputs are uniform residues drawn on the device. Roofline as ColTor's: the
    modular products of the NTTs and of the key multiply-accumulate."""
    c = synth.config_shapes("c2_rowsel")
    N, L, primes = c["N"], c["L"], list(c["primes"])
    params = g.gpir_params_create(N, primes)
    ell = g.gpir_coltor_gadget_digits(params)
    n_out = D0 + (D1.bit_length() - 1) * ell
    J = (n_out - 1).bit_length()
    query = torch.empty(B * 2 * L * N, dtype=torch.int32, device="cuda")
    evk = torch.empty(B * J * ell * 2 * L * N, dtype=torch.int32, device="cuda")
    out = torch.empty(B * n_out * 2 * L * N, dtype=torch.int32, device="cuda")
    g.gpir_fill_uniform(query, query.numel(), 0, 9, synth.TAG_QUERY, params, N)
    g.gpir_fill_uniform(evk, evk.numel(), 0, 9, synth.TAG_EVK, params, N)
    st = torch.cuda.current_stream()
    for _ in range(warmup):
        g.gpir_expand_query(params, B, J, n_out, query, evk, out, st.cuda_stream)
    st.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        g.gpir_expand_query(params, B, J, n_out, query, evk, out, st.cuda_stream)
    e1.record(st)
    st.synchronize()
    g.gpir_sync(None, 60000)
    ms = e0.elapsed_time(e1) / steps
    g.gpir_params_destroy(params)
    logn = N.bit_length() - 1
    nodes = B * sum(min(1 << j, n_out) for j in range(J))
    products = nodes * ((L + ell * L) * (N // 2) * logn + 2 * ell * L * N + 2 * L * N)
    peak = 152 * 64 * 2.07e9 / 3 / 1e12
    achieved = products / (ms / 1e3) / 1e12
    ct_bytes = 2 * L * N * 4
    alg_bytes = ct_bytes * (B + B * J * ell + B * n_out)
    return {"workload": "ExpandQuery before the 32-client RowSel: %d clients, %d outputs each (%d + %d x %d), "
                        "%d stages, N=%d, %d limbs" % (B, n_out, D0, D1.bit_length() - 1, ell, J, N, L),
            "ms": ms, "queries_s": B / (ms / 1e3),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T modmul/s",
                         "frac": achieved / peak,
                         "note": "NTT butterflies + key products + X^-2^j products (%.3g per step), 3 IMAD each, "
                                 "vs 152x64x2.07GHz/3; HBM: %.0f MB algorithmic, %.3f ms at the measured copy "
                                 "bandwidth" % (products, alg_bytes / 1e6, alg_bytes / 6652.3e9 * 1e3)}}


def run_pir_pipeline(g, torch, steps=5, warmup=3):
    """The whole server step on the 32-client workload through gpir_pir_batch:
    ExpandQuery (J = 8 stages, 256 selection ciphertexts per client), RowSel
    against the resident 512 MiB DB (tensor-core path), ColTor over the 64
    results. Inputs are uniform residues drawn on the device; per-phase device
    times come from the library's launch trace."""
    eng = GpuWorkload(g, torch, workload_shape("c2_rowsel"), 4)
    w, params, N, L = eng.w, eng.params, eng.w["N"], eng.w["L"]
    B, D0, D1 = w["B"], w["D0"], w["D1"]
    ell = g.gpir_coltor_gadget_digits(params)
    J = (D0 - 1).bit_length()
    stages = D1.bit_length() - 1
    ctw = 2 * L * N
    query = torch.empty(B * ctw, dtype=torch.int32, device="cuda")
    evk = torch.empty(B * J * ell * ctw, dtype=torch.int32, device="cuda")
    rgsw = torch.empty(B * stages * 2 * ell * ctw, dtype=torch.int32, device="cuda")
    sel = torch.empty(B * D0 * ctw, dtype=torch.int32, device="cuda")
    rows = torch.empty(B * D1 * ctw, dtype=torch.int32, device="cuda")
    out = torch.empty(B * ctw, dtype=torch.int32, device="cuda")
    g.gpir_fill_uniform(query, query.numel(), 0, 9, synth.TAG_QUERY, params, N)
    g.gpir_fill_uniform(evk, evk.numel(), 0, 9, synth.TAG_EVK, params, N)
    g.gpir_fill_uniform(rgsw, rgsw.numel(), 0, 9, synth.TAG_RGSW, params, N)
    st = torch.cuda.current_stream()
    call = lambda: g.gpir_pir_batch(eng.h, B, J, query, evk, rgsw, sel, rows, out, 4, st.cuda_stream)
    for _ in range(warmup):
        call()
    st.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        call()
    e1.record(st)
    st.synchronize()
    g.gpir_sync(None, 60000)
    ms = e0.elapsed_time(e1) / steps
    g.gpir_trace_enable(True)
    g.gpir_trace_read()
    call()
    st.synchronize()
    recs = g.gpir_trace_read()
    g.gpir_trace_enable(False)
    phase = {"expand_query": 0.0, "rowsel": 0.0, "coltor": 0.0}
    for name, t in recs:
        key = "expand_query" if name.startswith("expand") else ("coltor" if name.startswith("coltor") else "rowsel")
        phase[key] += t
    eng.close()
    return {"workload": "one server step, 32 clients: ExpandQuery (%d stages, %d selection cts) -> RowSel "
                        "(%dx%d DB, tensor core) -> ColTor (%d stages), N=%d, %d limbs" % (J, D0, D0, D1, stages, N, L),
            "ms": ms, "queries_s": B / (ms / 1e3), "phase_ms": {k: round(v, 4) for k, v in phase.items()}}


def run_serving(g, torch, rates=(200, 500, 1000, 2000), seconds=1.5, seed=4, repeats=3):
    """The serving workload: three resident DBs (N=4096, 2 limbs; 256x64,
    512x64, 1024x128), Poisson arrivals at each rate, every query a toy-RLWE
    one-hot selection drawn from a per-DB pool; p50/p99 latency and queries/s,
    each the median of `repeats` runs (every run listed)."""
    from paper_2604_04696_gb300.server import Request, ResidentDb, Server, poisson_arrivals
    from synth.device import toy_rlwe_query
    import gc
    gc.collect()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()   # the earlier sections' cached buffers go back before the DBs are made resident
    c = synth.config_shapes("c5_serving")
    N, L, primes = c["N"], c["L"], list(c["primes"])
    params = g.gpir_params_create(N, primes)
    dbs, pools = [], []
    rng = np.random.default_rng(seed)
    for k, (D0, D1) in enumerate(c["dbs"]):
        db = torch.empty(D0 * D1 * L * N, dtype=torch.int32, device="cuda")
        g.gpir_fill_uniform(db, db.numel(), 0, seed * 10 + k, synth.TAG_DB, params, N)
        h = g.gpir_db_upload(params, D0, D1, db, True, 0)
        del db
        dbs.append(ResidentDb(h, D0, D1, N, L))
        pool = []
        for qi in range(4):
            ct, _ = toy_rlwe_query(g.gpir_fill_uniform, params, D0, L, N, primes, int(rng.integers(0, D0)),
                                   seed * 100 + k * 10 + qi)
            pool.append(ct.cpu().pin_memory())
            del ct
        pools.append(pool)
    torch.cuda.synchronize()
    srv = Server(dbs, mem_budget_bytes=16 << 30, max_batch=32, n_streams=3)
    # warm-up: one short burst (autotune-free path; sizes the per-stream workspaces)
    warm = [Request(i, i % 3, pools[i % 3][0], 0.0) for i in range(3 * 32 * 3)]
    srv.run(warm)
    out = []
    for rate in rates:
        reps = []
        for rep in range(repeats):
            n = max(50, int(rate * seconds))
            arr = poisson_arrivals(float(rate), n, seed=seed + rate + 1000 * rep)
            reqs = []
            for i, t in enumerate(arr):
                d = int(rng.integers(0, 3))
                reqs.append(Request(i, d, pools[d][int(rng.integers(0, 4))], float(t)))
            reps.append(srv.run(reqs))
        med = lambda k: float(np.median([r[k] for r in reps]))
        out.append({"offered_qps": rate, "queries_s": med("queries_s"), "p50_ms": med("p50_ms"),
                    "p99_ms": med("p99_ms"), "mean_batch": med("mean_batch"),
                    "requests": int(sum(r["requests"] for r in reps)), "rejected": int(sum(r["rejected"] for r in reps)),
                    "repeats": [{"p50_ms": round(r["p50_ms"], 3), "p99_ms": round(r["p99_ms"], 3),
                                 "queries_s": round(r["queries_s"], 1)} for r in reps]})
    for d in dbs:
        g.gpir_db_free(d.h)
    g.gpir_params_destroy(params)
    return out


def run_case(a):
    """One seeded synthetic problem through the C ABI: a fixed launch sequence
    for profilers and a quick CUDA-event timing. Inputs are drawn on the device
    with gpir_fill_uniform. rowsel: two fill kernels (DB, ciphertexts), the
    upload's range check and packing kernels, then `reps` warm-up launches and
    `reps` timed ones; the trees and the server step likewise."""
    import torch
    from paper_2604_04696_gb300 import _build
    _build.build()
    from paper_2604_04696_gb300 import gpir as g
    B, D0, D1, N, L = (a.batch or 32), a.d0, a.d1, a.n, a.limbs
    params = g.gpir_params_create(N, list(synth.PRIMES_28[:L]))
    ell = g.gpir_coltor_gadget_digits(params)
    ctw = 2 * L * N
    dev = lambda n: torch.empty(n, dtype=torch.int32, device="cuda")
    h = None
    if a.case in ("rowsel", "pir"):
        path = PATH_IDS[a.path] if a.path != "auto" else 4
        db = dev(D0 * D1 * L * N)
        g.gpir_fill_uniform(db, db.numel(), 0, 1, synth.TAG_DB, params, N)
        h = g.gpir_db_upload(params, D0, D1, db, True, path if a.case == "rowsel" else g.GPIR_PATH_TC)
        del db
        torch.cuda.empty_cache()
    if a.case == "rowsel":
        ct = dev(B * D0 * ctw)
        g.gpir_fill_uniform(ct, ct.numel(), 0, 1, synth.TAG_CT, params, N)
        out = dev(B * D1 * ctw)
        if a.variant >= 0:
            g.gpir_set_variant(h, B, path, a.variant)
        step = lambda: g.gpir_rowsel_batch(h, B, ct, out, path)
        what = "rowsel %s B=%d D0=%d D1=%d N=%d L=%d" % (PATH_NAMES[path], B, D0, D1, N, L)
    elif a.case == "coltor":
        stages = D1.bit_length() - 1
        ct = dev(B * D1 * ctw)
        rgsw = dev(B * stages * 2 * ell * ctw)
        out = dev(B * ctw)
        g.gpir_fill_uniform(ct, ct.numel(), 0, 9, synth.TAG_COLTOR, params, N)
        g.gpir_fill_uniform(rgsw, rgsw.numel(), 0, 9, synth.TAG_RGSW, params, N)
        step = lambda: g.gpir_coltor(params, B, D1, ct, rgsw, out)
        what = "coltor B=%d D1=%d N=%d L=%d ell=%d (%d stages)" % (B, D1, N, L, ell, stages)
    elif a.case == "expand":
        query = dev(B * ctw)
        evk = dev(B * a.stages * ell * ctw)
        out = dev(B * a.n_out * ctw)
        g.gpir_fill_uniform(query, query.numel(), 0, 9, synth.TAG_QUERY, params, N)
        g.gpir_fill_uniform(evk, evk.numel(), 0, 9, synth.TAG_EVK, params, N)
        step = lambda: g.gpir_expand_query(params, B, a.stages, a.n_out, query, evk, out)
        what = "expand B=%d J=%d n_out=%d N=%d L=%d ell=%d" % (B, a.stages, a.n_out, N, L, ell)
    else:
        J = (D0 - 1).bit_length()
        stages = D1.bit_length() - 1
        query = dev(B * ctw)
        evk = dev(B * J * ell * ctw)
        rgsw = dev(B * stages * 2 * ell * ctw)
        g.gpir_fill_uniform(query, query.numel(), 0, 9, synth.TAG_QUERY, params, N)
        g.gpir_fill_uniform(evk, evk.numel(), 0, 9, synth.TAG_EVK, params, N)
        g.gpir_fill_uniform(rgsw, rgsw.numel(), 0, 9, synth.TAG_RGSW, params, N)
        sel, rows, out = dev(B * D0 * ctw), dev(B * D1 * ctw), dev(B * ctw)
        step = lambda: g.gpir_pir_batch(h, B, J, query, evk, rgsw, sel, rows, out, g.GPIR_PATH_TC)
        what = "pir step B=%d D0=%d D1=%d N=%d L=%d (J=%d, %d ColTor stages)" % (B, D0, D1, N, L, J, stages)
    for _ in range(a.reps):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.reps):
        step()
    e1.record()
    torch.cuda.synchronize()
    g.gpir_sync(None, 60000)
    extra = ""
    if a.case == "rowsel":
        extra = " (variant %d)" % g.gpir_selected_variant(h, B, path)
    print("%s%s: %.4f ms per call" % (what, extra, e0.elapsed_time(e1) / a.reps), flush=True)
    if h is not None:
        g.gpir_db_free(h)
    g.gpir_params_destroy(params)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gpir", choices=["gpir", "reference"])
    ap.add_argument("--workload", default="c4_large", choices=["c1_plain", "c2_rowsel", "c4_large", "c3_sweep"])
    ap.add_argument("--batch", type=int, default=None)
    ap.add_argument("--path", default="auto", choices=list(PATH_IDS))
    ap.add_argument("--no-extras", action="store_true", help="skip the sweep, trees, serving and pipeline sections")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--case", choices=["rowsel", "coltor", "expand", "pir"], default=None,
                    help="run one synthetic problem (profiling / quick timing) and exit")
    ap.add_argument("--d0", type=int, default=256)
    ap.add_argument("--d1", type=int, default=64)
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--limbs", type=int, default=2)
    ap.add_argument("--variant", type=int, default=-1, help="--case rowsel: tile variant (-1: library default)")
    ap.add_argument("--stages", type=int, default=9, help="--case expand: expansion stages J")
    ap.add_argument("--n-out", type=int, default=274, help="--case expand: outputs kept per client")
    ap.add_argument("--reps", type=int, default=3, help="--case: warm-up and timed launches")
    args = ap.parse_args()
    if args.case:
        return run_case(args)
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    barrier = None
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        barrier = lambda: dist.barrier(device_ids=[local])

    from paper_2604_04696_gb300 import _build
    _build.build()
    from paper_2604_04696_gb300 import gpir as g

    peaks = load_peaks()
    w = workload_shape(args.workload, args.batch)
    built = [p for p in (1, 2, 4) if g.gpir_num_variants(p) > 0]
    mask = 0
    for p in built:
        mask |= p
    # N > 1: each rank keeps and computes its slot shard of the one workload
    # (RowSel is independent per NTT point: no exchange while it runs)
    sh = None
    if world > 1:
        from paper_2604_04696_gb300.shard import SlotShard
        sh = SlotShard(w["N"], world, rank)
    wl = GpuWorkload(g, torch, w, mask, shard=sh)
    w_rank = dict(w, N=wl.T)      # this GPU's share, for its kernels' rooflines

    # choose the path: requested, else the fastest built path after autotuning each
    per_path = {}
    for p in built:
        v = g.gpir_autotune(wl.h, w["B"], wl.ct, wl.out, p, wl.stream)
        ms, _ = wl.time_steps(p, max(3, min(args.steps, 10)), 2)
        per_path[p] = {"variant": v, "ms": ms}
    if args.path != "auto":
        path = PATH_IDS[args.path]
    else:
        path = min(per_path, key=lambda p: per_path[p]["ms"])
    variant = per_path[path]["variant"]

    clocks = Clocks(local)
    ms, clk = wl.time_steps(path, args.steps, args.warmup, barrier=barrier, clocks=clocks)
    exact = wl.check_sample() if rank == 0 else None
    ktimes, kcount = wl.kernel_times(path, max(3, min(args.steps, 10)))
    dom = max(ktimes, key=lambda k: ktimes[k] * kcount[k])
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    qps = w["B"] / (ms / 1e3)      # the whole batch, all ranks together
    e2e_ms, h2d, d2h = wl.e2e(path, max(3, args.steps // 2), 2)
    if world > 1:
        t = torch.tensor([e2e_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())
        h2d, d2h = h2d * world, d2h * world
    e2e_val = w["B"] / (e2e_ms / 1e3)

    db_bytes = sizes.db_bytes(w["D0"], w["D1"], w["N"], w["L"])
    alg = sizes.rowsel_algorithmic_bytes(w["B"], w["D0"], w["D1"], w["N"], w["L"])
    line = {
        "metric": METRIC, "value": qps, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "strong" if world > 1 else "weak",
        "vs_baseline": None, "dtype": {1: "u32 (u64 accumulate)", 2: "u8 (s32 accumulate)",
                                       4: "fp16 digits (fp32 exact accumulate)"}[path],
        "data": "synthetic",
        "config": dict(cfg_dict(args.workload, w, PATH_NAMES[path], variant),
                       parallelism=("slot shards: %d ranks x %d slots per limb, no collective in the step"
                                    % (world, wl.T)) if world > 1 else "one GPU"),
        "db_gbs": db_bytes / (ms / 1e3) / 1e9, "alg_gbs": alg / (ms / 1e3) / 1e9,
        "bit_exact_sample": exact,
        # the dominant kernel's roofline: from the untraced step when the step is
        # that one launch, else from its traced per-launch time
        "roofline": kernel_roofline(dom, w_rank, ms if (len(kcount) == 1 and kcount[dom] == 1) else ktimes[dom],
                                    peaks, args.workload),
        "step_roofline": roofline(path, w_rank, ms, peaks, args.workload, KERNELS[dom][2]),
        "kernels": {k: {"ms": v, "launches_per_step": kcount[k], "share": v * kcount[k] / sum(
            ktimes[x] * kcount[x] for x in ktimes)} for k, v in ktimes.items()},
        "e2e": {"value": e2e_val, "unit": "queries/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": args.steps * sum(kcount.values()),
        "clocks": clk,
        "paths": {PATH_NAMES[p]: {"ms": v["ms"], "queries_s": w["B"] / (v["ms"] / 1e3), "variant": v["variant"]}
                  for p, v in per_path.items()},
    }
    wl.close()
    if not args.no_extras and rank == 0:
        # queries/s vs batch on the same DB shape (best path), one line item per batch
        if True:
            sweep = []
            for b in (1, 8, 32, 128, 256):
                # per batch: autotuned path and tile, captured once into a CUDA
                # graph (gpir_graph_create), timed as graph replays
                ws = workload_shape("c3_sweep", b)
                wk = GpuWorkload(g, torch, ws, mask)
                g.gpir_autotune(wk.h, b, wk.ct, wk.out, 0, wk.stream)     # fastest path and tile for b
                chosen = g.gpir_selected_path(wk.h, b)
                gs = torch.cuda.Stream()
                graph = g.gpir_graph_create([(wk.h, b, wk.ct, wk.out)], chosen, gs)
                for _ in range(3):
                    g.gpir_graph_launch(graph, gs)
                gs.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(gs)
                for _ in range(10):
                    g.gpir_graph_launch(graph, gs)
                e1.record(gs)
                gs.synchronize()
                g.gpir_sync(gs, 60000)
                mss = e0.elapsed_time(e1) / 10
                g.gpir_graph_destroy(graph)
                vb = g.gpir_selected_variant(wk.h, b, chosen)
                sweep.append({"batch": b, "path": PATH_NAMES.get(chosen, str(chosen)), "variant": vb, "ms": mss,
                              "queries_s": b / (mss / 1e3), "timed": "CUDA-graph replays",
                              "roofline_frac": roofline(chosen, ws, mss, peaks, "c3_sweep",
                                                        path_products(chosen, vb))["frac"]})
                wk.close()
            line["sweep"] = sweep
        line["pir_pipeline"] = run_pir_pipeline(g, torch)
        line["expand_query"] = run_expand(g, torch)
        line["coltor"] = run_coltor(g, torch)
        line["serving"] = {"workload": "c5_serving: 3 resident DBs 256x64 / 512x64 / 1024x128, N=4096, 2 limbs, "
                                       "Poisson arrivals, toy-RLWE one-hot queries, 3 streams, max batch 32",
                           "rates": run_serving(g, torch)}
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_baseline(w, seconds_target=15.0)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
