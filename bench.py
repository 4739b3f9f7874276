#!/usr/bin/env python
"""Benchmark of the Clifford circuit-cutting hot path on GB300s.

Workload (default, the largest single-GPU configuration): 500 qubits, depth-30
random Clifford brickwork, 16 T gates in four 2-wire non-Clifford regions, 8
wire cuts -> a 500-wire Clifford body (1000 x 1001-bit tableau, 20736
variants) and four statevector leaves; 2^14 Philox shots per Clifford
variant; 16-qubit marginal from the contraction over the 4^8 cut terms.
One step = one pass of the whole path: body evolution, outcome spaces,
sampling folded into the contraction operand, statevectors, fold,
contraction.

value   Clifford variant-shots/s, plan resident on the device, one CUDA-graph
        replay of the evaluation + one of the recombination per step, L2
        flushed between steps (outside the step events); the FP32
        contraction (the precision gated at 1e-5 against the FP64 oracle).
e2e     the same metric through the public C ABI from host buffers: plan build
        (host compile + upload), evaluation, recombination, read-back to host
        memory, every step; steps are served by eight host worker threads, one
        step at a time each, on their own contexts and streams.
plain   the plain GPU form in the same run: per-variant simulation of every
        variant's whole circuit, stream launches, FP32, no tuning.
bf16    the same steps with the contraction in BF16 on the tensor cores.
stitched
        the same circuits in the Clifford-specific stitching mode (exact: no
        shots, each hub operand row in closed form, vanishing rows skipped).
ml      the same sampled steps with the maximum-likelihood correction of the
        Clifford fragment models between evaluation and contraction (or the
        reason it does not apply: a fragment with more than 6 cut slots).

With --gpus N (torchrun, or N spawned ranks when started plainly) every rank
runs its own batch of the workload (other Philox seeds; other circuits for
many-circuit workloads): independent problems, no data-path collective,
weak scaling; the step time is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Clifford variant-shots/s and circuits/s end-to-end; % of HBM/tensor roofline"
UNIT = "variant-shots/s"
SEED = (0x9E3779B9, 0x7F4A7C15)
N_SM = 152


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def workloads_for(name, rank=0):
    """The batch of circuits one step of one rank processes."""
    import workloads as W
    if name == "config1":
        return [W.config1()]
    if name == "config2":
        return [W.config2()]
    if name == "config3":
        return [W.config3()]
    if name == "config4":
        return W.config4(256, seed_offset=rank)
    if name == "config4x16":          # 16 circuits of the same population (profiling captures)
        return W.config4(16, seed_offset=rank)
    # the paper's own benchmark shapes (Sec. VI-B, 5000 shots per sampled
    # distribution as in Sec. VI-A); cut sets are searched by the library
    if name == "hwea300":
        return [W.hwea(300, rounds=5, n_t=1, n_z=8, shots=5000, seed=W.SEED_BASE + 6 + 1000 * rank)]
    if name == "hwea300x64":
        return [W.hwea(300, rounds=5, n_t=1, n_z=8, shots=5000, seed=W.SEED_BASE + 600 + i + 1000 * rank)
                for i in range(64)]
    if name == "skqaoa26":
        return [W.sk_qaoa(26, rounds=1, n_t=1, n_z=8, shots=5000, seed=W.SEED_BASE + 7 + 1000 * rank)]
    raise SystemExit(f"unknown workload {name}")


def with_cuts(ws, ctx=None):
    """Copies of the circuits with searched cut sets filled in (a host-only
    plan when no context is given); explicit cut sets are kept."""
    import dataclasses
    if all(x.cuts is not None for x in ws):
        return ws
    from paper_2303_10788_gb300 import ccs
    ctx = ctx or ccs.ccs_create(-1)
    plan = ccs.ccs_build_fragments(ctx, ws)
    return [x if x.cuts is not None else dataclasses.replace(x, cuts=ccs.ccs_plan_cuts(ctx, plan, i))
            for i, x in enumerate(ws)]


def describe(ws):
    w = ws[0]
    if len(ws) == 1:
        return (f"{w.name}: {w.circuit.n_qubits} qubits, {len(w.circuit.gates)} gates, {w.circuit.n_t} T, "
                f"{len(w.cuts)} cuts, {w.shots} shots/Clifford variant, {len(w.marginal)}-qubit marginal, "
                f"{len(w.zstrings)} Z-strings")
    nq = [x.circuit.n_qubits for x in ws]
    return (f"{w.name.split('_')[0]}: {len(ws)} circuits of {min(nq)}-{max(nq)} qubits, "
            f"{min(len(x.cuts) for x in ws)}-{max(len(x.cuts) for x in ws)} cuts, {w.shots} shots/Clifford "
            f"variant, {len(w.marginal)}-qubit marginal each, one plan and one launch sequence per step")


# --- clocks during the timed region ------------------------------------------

class Clocks:
    """SM clock and throttle reasons sampled during the timed region: NVML
    (read-only queries, every 2 ms on a thread) when the driver's library
    loads, else nvidia-smi."""

    _BITS = {"hw_slowdown": 0x8, "hw_thermal_slowdown": 0x40, "sw_thermal_slowdown": 0x20, "sw_power_cap": 0x4}

    def __init__(self, index):
        self.sm, self.mx, self.reasons, self.p = [], 0.0, set(), None
        self.stop_ev = threading.Event()
        self.nv = self._nvml(index)
        if self.nv is not None:
            self.t = threading.Thread(target=self._poll, daemon=True)
            self.t.start()
        else:
            self._smi(index)

    def _nvml(self, index):
        import ctypes as C
        try:
            nv = C.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() != 0:
                return None
            h = C.c_void_p()
            if nv.nvmlDeviceGetHandleByIndex_v2(C.c_uint(index), C.byref(h)) != 0:
                return None
            mx = C.c_uint()
            if nv.nvmlDeviceGetMaxClockInfo(h, 1, C.byref(mx)) == 0:       # NVML_CLOCK_SM
                self.mx = float(mx.value)
            self.h = h
            self.reason_fn = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                getattr(nv, "nvmlDeviceGetCurrentClocksThrottleReasons")
            return nv
        except Exception:
            return None

    def _poll(self):
        import ctypes as C
        mhz, rs = C.c_uint(), C.c_ulonglong()
        while True:
            if self.nv.nvmlDeviceGetClockInfo(self.h, 1, C.byref(mhz)) == 0:
                self.sm.append(float(mhz.value))
            if self.reason_fn(self.h, C.byref(rs)) == 0:
                for n, b in self._BITS.items():
                    if rs.value & b:
                        self.reasons.add(n)
            if self.stop_ev.wait(0.002):
                return

    def _smi(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "10"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.nv is not None:
            self.stop_ev.set()
            self.t.join(2)
            src = "nvml"
        elif self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(5)
            except Exception:
                self.p.kill()
            self.f.flush()
            names = list(self._BITS)
            for l in open(self.f.name).read().splitlines():
                r = l.split(",")
                try:
                    self.sm.append(float(r[1])); self.mx = max(self.mx, float(r[2]))
                    for n, v in zip(names, r[5:9]):
                        if v.strip() == "Active":
                            self.reasons.add(n)
                except Exception:
                    pass
            os.unlink(self.f.name)
            src = "nvidia-smi"
        else:
            return None
        if not self.sm:
            return None
        return {"sm_mhz": statistics.median(self.sm), "sm_max_mhz": self.mx, "reasons": sorted(self.reasons),
                "samples": len(self.sm), "source": src}


# --- the CPU oracle ------------------------------------------------------------

def host_cores(cap=32):
    """Cores this process may run on (its affinity mask, else the CPU count),
    at most `cap` (bounds the oracle runs' length on very wide hosts)."""
    try:
        n = len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        n = os.cpu_count() or 1
    return max(1, min(cap, n))


def _oracle_chunk(args):
    """Worker of the threaded baseline (a spawned process): the oracle on a
    list of body variants."""
    w, body, vs = args
    from oracle.pipeline import evaluate_workload
    evaluate_workload(w, mode="sampled", seed_lo=SEED[0], seed_hi=SEED[1], keep_tableaus=False,
                      variants_only={body: vs})
    return len(vs)


def oracle_threaded(w, n_variants, body, per_variant_s, budget_s=10.0):
    """The same oracle over all host cores, threaded over variants as
    separate processes (spawned, so no CUDA state is inherited): each process
    evaluates its own body variants; only the parallel part is timed."""
    import multiprocessing as mp
    procs = host_cores()
    k = max(1, int(budget_s / 2 / max(per_variant_s, 1e-3)))
    chunks = [[(p * k + i) * 97 % n_variants for i in range(k)] for p in range(procs)]
    with mp.get_context("spawn").Pool(procs) as pool:
        pool.map(_oracle_chunk, [(w, body, [0])] * procs, chunksize=1)   # start-up and imports, untimed
        t0 = time.perf_counter()
        done = sum(pool.map(_oracle_chunk, [(w, body, c) for c in chunks], chunksize=1))
        dt = time.perf_counter() - t0
    return {"value": done * w.shots / dt, "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": f"{procs} processes x {k} body variants x {w.shots} shots of the first circuit, {dt:.1f} s "
                      f"(Clifford body variants only: no statevector variants, fold or recombination)"}


def oracle_baseline(ws, budget_s=20.0, threaded=True, threaded_budget_s=10.0):
    """The CPU oracle on a bounded sample of the workload: whole circuits when
    one fits the budget, else a sample of Clifford variants of the first one;
    single-threaded, and (``threaded``) over all host cores beside it."""
    from oracle.pipeline import evaluate_workload
    from oracle.cutting import fragment_circuit
    w = ws[0]
    frags, _ = fragment_circuit(w.circuit, w.cuts, w.marginal)
    ncl = sum(f.n_variants for f in frags if f.clifford)
    body = max(range(len(frags)), key=lambda i: frags[i].n if frags[i].clifford else -1)
    if ncl <= 400:
        t0 = time.perf_counter()
        evaluate_workload(w, mode="sampled", seed_lo=SEED[0], seed_hi=SEED[1], keep_tableaus=False)
        dt = time.perf_counter() - t0
        out = {"value": ncl * w.shots / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"one full circuit of the workload ({ncl} Clifford variants x {w.shots} shots, "
                         f"all statevector variants, fold and recombination), {dt:.1f} s single-threaded",
               "circuits_per_s": 1.0 / dt}
        per_variant = dt / max(1, ncl)
    else:
        vs, t_tot = [], 0.0
        while t_tot < budget_s and len(vs) < frags[body].n_variants:
            v = len(vs) * 97 % frags[body].n_variants
            t0 = time.perf_counter()
            evaluate_workload(w, mode="sampled", seed_lo=SEED[0], seed_hi=SEED[1], keep_tableaus=False,
                              variants_only={body: [v]})
            t_tot += time.perf_counter() - t0
            vs.append(v)
        out = {"value": len(vs) * w.shots / t_tot, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{len(vs)} body variants x {w.shots} shots of the first circuit ({t_tot:.1f} s "
                         f"single-threaded; a whole circuit has {ncl} Clifford variants; Clifford body "
                         f"variants only: no statevector variants, fold or recombination)"}
        per_variant = t_tot / len(vs)
    if threaded and frags[body].clifford:
        try:
            out["threaded"] = oracle_threaded(w, frags[body].n_variants, body, per_variant, threaded_budget_s)
        except Exception as e:      # the extra figure must not cost the bench line
            out["threaded"] = {"unavailable": f"{type(e).__name__}: {e}"[:200]}
    return out


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle, timed on all host cores (rank 0 only):
    one spawned process per core, each evaluating its own sample of body
    variants every step (sized so a step takes a few seconds); one process
    in this one when no pool can start."""
    if rank != 0:
        return
    import multiprocessing as mp
    from oracle.pipeline import evaluate_workload
    from oracle.cutting import fragment_circuit
    ws = with_cuts(workloads_for(args.workload))
    w = ws[0]
    frags, _ = fragment_circuit(w.circuit, w.cuts, w.marginal)
    body = max(range(len(frags)), key=lambda i: frags[i].n if frags[i].clifford else -1)
    nv = frags[body].n_variants
    t0 = time.perf_counter()      # one variant, to size the per-step sample
    evaluate_workload(w, mode="sampled", seed_lo=SEED[0], seed_hi=SEED[1], variants_only={body: [0]},
                      keep_tableaus=False)
    per_v = time.perf_counter() - t0
    nsamp = max(1, min(8, int(2.5 / max(per_v, 1e-3))))
    procs = host_cores()
    chunks = [[(p * nsamp + i) * 97 % nv for i in range(nsamp)] for p in range(procs)]
    pool = None
    try:
        pool = mp.get_context("spawn").Pool(procs)
        pool.map(_oracle_chunk, [(w, body, [0])] * procs, chunksize=1)   # start-up and imports, untimed
    except Exception:
        if pool is not None:
            pool.terminate()
        pool, procs, chunks = None, 1, chunks[:1]

    def step():
        if pool is not None:
            pool.map(_oracle_chunk, [(w, body, c) for c in chunks], chunksize=1)
        else:
            evaluate_workload(w, mode="sampled", seed_lo=SEED[0], seed_hi=SEED[1],
                              variants_only={body: chunks[0]}, keep_tableaus=False)

    try:
        for _ in range(args.warmup):
            step()
        times = []
        for _ in range(args.steps):
            t0 = time.perf_counter(); step(); times.append(time.perf_counter() - t0)
    finally:
        if pool is not None:
            pool.close()
            pool.join()
    tot = sum(times)
    units = procs * nsamp * w.shots * args.steps
    val = units / tot
    line = {"metric": METRIC, "value": val, "unit": UNIT, "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8/f64",
            "data": "synthetic",
            "config": {"workload": describe(ws), "parallelism": f"CPU oracle, {procs} host processes",
                       "scope": "Clifford body variants only (tableau, outcome space, shots); "
                                "no statevector variants, fold or recombination"},
            "cpu_baseline": {"kind": "oracle", "cores": procs, "value": val, "unit": UNIT,
                             "sample": f"per step: {procs} processes x {nsamp} body variants x {w.shots} shots "
                                       f"(Clifford body variants only)"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --- rooflines -----------------------------------------------------------------

def _ncu_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu
    summary (profiles/dram_traffic.md), or None when none is recorded or the
    kernel's source changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    for m in re.finditer(r"^\|\s*(\w+)\s*\|\s*(\w+)\s*\|\s*([0-9.]+)\s*\|\s*([0-9.]+)\s*\|\s*(\S+)\s*\|\s*([0-9a-f]{16})\s*\|",
                         text, re.M):
        k, wl, rd, wr, src, sha = m.groups()
        if k == kernel and wl == workload:
            try:
                now = hashlib.sha256(open(os.path.join(ROOT, src), "rb").read()).hexdigest()[:16]
            except OSError:
                return None
            return (float(rd) + float(wr)) * 1e6 if now == sha else None
    return None


E2E_WORKERS = 8     # host threads serving end-to-end steps, one step at a time each


def stage_kernel(st, precision, tuning=None, ws=None, prob_infos=None):
    """The kernel that stands for a stage (its longest launch): the hub
    sampler the autotuner picked (byte or 16-bit counters); the contraction
    of wide hub operands (the first-leaf streaming GEMM, or tcgen05 in BF16)
    or of small stars (leaf by leaf); the body kernel for the Clifford stage."""
    if st == "sample":
        return "sample_hub_kernel" if (tuning or {}).get("hub_counters") == "16-bit" else "sample_hub8_kernel"
    if st == "recombine":
        wide = False
        for x, infos in zip(ws or [], prob_infos or []):
            k = len(x.cuts or [])
            hubs = [i for i in infos if i["n_slots"] == k]
            wide = wide or any((4 ** k) << i["n_marg"] >= 1 << 24 for i in hubs)
        if not wide:
            return "contract_kernel"
        return "gemm_bf16_tc_kernel" if precision == "bf16" else "gemm_fact_bulk_kernel"
    if st == "clifford":
        return "clifford_kernel" if (tuning or {}).get("variant_path") else "body_kernel"
    return None


def stage_rooflines(stage, ws, prob_infos, pk, pk_kind, precision, workload, tuning=None):
    """Roofline of every stage: algorithmic work per launch / live duration.

    Peaks: lane ops = SMs x 128 lanes x max SM clock (one 32-bit op per lane
    per clock, the issue limit); FP32 = SMs x 128 FMA x 2 x clock; shared
    memory = SMs x 128 B x clock; HBM = the measured copy bandwidth.

    clifford    smem: the body evolved once per Clifford fragment, each fused
                two-qubit op reading and writing its 4 columns of 2n bits
                (2n bytes per op); per variant the screen's elimination of
                (n_meas + n_qout + n_qin) vectors of n_meas bits (4 bytes each,
                read and written per pivot)
    sample      alu: per shot a 1/(4 s) share of one Philox4x32-10 call (10
                rounds of 2 wide multiplies and 2 three-way XORs = 40 lane
                ops; s = 4, 2, 1 shots per output word at |A| <= 8, 16, above),
                1 op for its field, 3 per table lookup (L = 1, 2, 3) and 3 for
                the counter increment; per hub variant and output o, 2^qout
                counter reads and one store per operand row of the variant
                (2^(Z-basis outputs)), averaged over the variants
    statevector alu: a fused 4x4 complex op costs 32 FP32 flops per amplitude
    recombine   hbm: the hub operand read once at its stored width (2 B per
                element as int16 count sums of a sampled Clifford hub or in
                BF16, else 4 B),
                the Kronecker operand R (K x N x 4 B) and the split-K partials
                written and read once
    fold, operands
                hbm: variant data read once and fragment tensors written once
    """
    clk = pk.get("sm_max_mhz", 2070.0) * 1e6
    lanes = N_SM * 128 * clk
    out = {}
    for st, ms in stage.items():
        t = ms * 1e-3
        if t <= 0:
            continue
        if st == "clifford":
            by = 0
            for x, infos in zip(ws, prob_infos):
                for i in infos:
                    if i["clifford"]:
                        by += i["n_ops"] * 2 * i["n_wires"]
                        by += i["n_variants"] * (i["n_meas"] + i["n_qout"] + i["n_qin"]) * i["n_meas"] * 8
            out[st] = {"bound": "smem", "achieved": by / t / 1e9, "peak": N_SM * 128 * clk / 1e9, "unit": "GB/s",
                       "peak_source": f"derived: {N_SM} SMs x 128 B x {clk/1e6:.0f} MHz"}
        elif st == "sample":
            ops = 0.0
            for x, infos in zip(ws, prob_infos):
                for i in infos:
                    if not i["clifford"]:
                        continue
                    per_word = 4 if i["n_meas"] <= 8 else 2 if i["n_meas"] <= 16 else 1
                    lookups = 1 if i["n_meas"] <= 8 else 2 if i["n_meas"] <= 16 else 3
                    ops += i["n_variants"] * x.shots * (40 / (4 * per_word) + 1 + 3 * lookups + 3)
                    if i["n_slots"] == len(x.cuts):   # hub of the star: the operand rows
                        rows = (4 ** i["n_qin"]) * (4 ** i["n_qout"]) / max(1, i["n_variants"])
                        ops += i["n_variants"] * (1 << i["n_marg"]) * ((1 << i["n_qout"]) + rows)
            out[st] = {"bound": "alu", "achieved": ops / t / 1e12, "peak": lanes / 1e12, "unit": "T lane-op/s",
                       "peak_source": f"derived: {N_SM} SMs x 128 lanes x {clk/1e6:.0f} MHz"}
        elif st == "statevector":
            fl = sum(i["n_variants"] * i["n_ops"] * 32 * (1 << i["n_wires"])
                     for infos in prob_infos for i in infos if not i["clifford"])
            out[st] = {"bound": "alu", "achieved": fl / t / 1e12, "peak": N_SM * 256 * clk / 1e12,
                       "unit": "TFLOP/s", "peak_source": f"derived: {N_SM} SMs x 128 FP32 FMA x 2 x {clk/1e6:.0f} MHz"}
        else:
            by = 0
            for x, infos in zip(ws, prob_infos):
                k = len(x.cuts)
                if st == "recombine":
                    hubs = [i for i in infos if i["n_slots"] == k]
                    M = 1 << max([i["n_marg"] for i in hubs] or [0])
                    N = (1 << len(x.marginal)) // M
                    # a Clifford hub sampled with at most 32767 shots stores its
                    # operand as exact int16 count sums: 2 B per element read
                    i16 = bool(hubs) and hubs[0]["clifford"] and x.shots <= 32767
                    by += (4 ** k) * M * (2 if (precision == "bf16" or i16) else 4) + (4 ** k) * N * 4
                else:
                    for i in infos:
                        hub = i["n_slots"] == k
                        if st == "fold" and not (hub and i["clifford"]):
                            by += i["n_variants"] * 4 * (1 << i["n_meas"]) + 4 * (1 << i["n_marg"]) * 4 ** i["n_slots"]
                        if st == "operands" and not hub:
                            by += 8 * (1 << i["n_marg"]) * 4 ** i["n_slots"]
            out[st] = {"bound": "hbm", "achieved": by / t / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s",
                       "peak_source": pk_kind}
        out[st]["frac"] = out[st]["achieved"] / out[st]["peak"]
        kern = stage_kernel(st, precision, tuning, ws, prob_infos)
        out[st]["traffic"] = _ncu_traffic(kern, workload) if kern else None
        out[st]["ms"] = ms
    return out


# --- our arm -------------------------------------------------------------------

def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2303_10788_gb300 import ccs
    from paper_2303_10788_gb300.sharding import max_over_ranks
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    ws_in = workloads_for(args.workload, rank)      # cuts None: searched inside ccs_build_fragments
    seed = (SEED[0] + rank, SEED[1])
    ctx = ccs.ccs_create(local_rank)
    plan = ccs.ccs_build_fragments(ctx, ws_in)
    ws = with_cuts(ws_in, ctx)
    w = ws[0]
    prob_infos = [[ccs.ccs_fragment_info_get(ctx, plan, pi, f) for f in range(ccs.ccs_plan_counts(ctx, plan, pi)[0])]
                  for pi in range(len(ws))]
    infos = [i for pi in prob_infos for i in pi]
    n_cliff_var = sum(i["n_variants"] for i in infos if i["clifford"])
    units_per_step = n_cliff_var * w.shots
    marg = torch.zeros(sum(1 << len(x.marginal) for x in ws), dtype=torch.float64, device="cuda")
    zexp = torch.zeros(max(1, sum(len(x.zstrings) for x in ws)), dtype=torch.float64, device="cuda")
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")      # > 129 MB L2
    if args.plain:
        args.precision = "fp32"
    prec = ccs.CCS_BF16 if args.precision == "bf16" else ccs.CCS_FP32
    pvb = bool(args.per_variant_body or args.plain)
    graph = not args.plain
    tune = not args.no_autotune and not args.plain
    ev = dict(mode=ccs.CCS_SAMPLED, shots=w.shots, seed_lo=seed[0], seed_hi=seed[1], per_variant_body=pvb)
    res = ccs.ccs_eval_variants(ctx, plan, use_graph=graph, autotune=tune, **ev)
    tuning = ccs.ccs_get_tuning(ctx, res)

    def step(p=prec):
        ccs.ccs_eval_variants(ctx, plan, use_graph=graph, res=res, **ev)
        ccs.ccs_recombine(ctx, plan, res, precision=p, marginal_out=marg, zexp_out=zexp, use_graph=graph)

    def timed(fn, steps):
        """CUDA-event time of `steps` calls of fn, L2 flushed before each."""
        stream = torch.cuda.current_stream()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            flush.zero_()
            evs[i][0].record(stream)
            fn()
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs) / 1e3

    for _ in range(max(3, args.warmup)):
        step()
    barrier()
    clk = Clocks(local_rank)
    launches0 = ccs.ccs_launch_count()
    torch.cuda.nvtx.range_push("timed_steps")    # profilers can select the timed launches by this range
    t_local = timed(step, args.steps)
    torch.cuda.nvtx.range_pop()
    barrier()
    launches = ccs.ccs_launch_count() - launches0
    clocks = clk.stop()
    t_tot = max_over_ranks(t_local, dist, device="cuda")
    value = units_per_step * args.steps * world / t_tot

    # --- per-stage kernel times (profiled pass, same work, no graph) ----------
    ccs.ccs_set_profiling(ctx, True)
    acc = {}
    for _ in range(args.steps):
        flush.zero_()
        ccs.ccs_eval_variants(ctx, plan, res=res, **ev)
        ccs.ccs_recombine(ctx, plan, res, precision=prec, marginal_out=marg, zexp_out=zexp)
        for k, v in ccs.ccs_get_stage_times(ctx).items():
            acc.setdefault(k, []).append(v)
    ccs.ccs_set_profiling(ctx, False)
    stage = {k: statistics.mean(v) for k, v in acc.items()}
    dom = max(stage, key=stage.get)

    # --- end to end through the C ABI from host buffers ------------------------
    # the host inputs are the C-ABI problem structs, marshalled once (with
    # the cut search inside the timed build where the workload has no cut
    # set).  Every step builds and uploads its plan, evaluates, recombines
    # and reads the result back to pinned host memory.  Steps are served by
    # E2E_WORKERS host threads, the way a serving frontend takes requests:
    # each worker runs one step at a time start to finish on its own context
    # and stream, so host work overlaps across steps and the device work of
    # different steps may overlap too.  The contexts use the library's own
    # stream-ordered pool (the C ABI default): an allocator that calls back
    # into Python would serialise the workers on the interpreter lock.
    import threading
    from concurrent.futures import ThreadPoolExecutor
    packed = ccs.pack_problems(ws_in)
    tls, ctxs = threading.local(), []
    nm = sum(1 << len(x.marginal) for x in ws)
    nzs = max(1, sum(len(x.zstrings) for x in ws))

    def e2e_step(_=None):
        if not hasattr(tls, "ctx"):
            tls.stream = torch.cuda.Stream(local_rank)
            torch.cuda.set_stream(tls.stream)
            tls.ctx = ccs.ccs_create(local_rank, torch_allocator=False)
            ctxs.append(tls.ctx)
            tls.dev = (torch.empty(nm, dtype=torch.float64, device="cuda"),
                       torch.empty(nzs, dtype=torch.float64, device="cuda"))
            tls.host = (torch.empty(nm, dtype=torch.float64, pin_memory=True),
                        torch.empty(nzs, dtype=torch.float64, pin_memory=True))
            tls.done = torch.cuda.Event()
        tls.keep = None                                  # the previous step's plan and result
        p2 = ccs.ccs_build_fragments(tls.ctx, packed)
        r2 = ccs.ccs_eval_variants(tls.ctx, p2, autotune=tune, **ev)
        ccs.ccs_recombine(tls.ctx, p2, r2, precision=prec, marginal_out=tls.dev[0], zexp_out=tls.dev[1])
        tls.host[0].copy_(tls.dev[0], non_blocking=True)
        tls.host[1].copy_(tls.dev[1], non_blocking=True)
        tls.done.record(tls.stream)
        tls.done.synchronize()                           # the step's result is in host memory
        tls.keep = (p2, r2)

    with ThreadPoolExecutor(E2E_WORKERS) as ex:
        gate = threading.Barrier(E2E_WORKERS)

        def on_every_worker(fn):
            def once():
                gate.wait()
                fn()
            for f in [ex.submit(once) for _ in range(E2E_WORKERS)]:
                f.result()

        on_every_worker(e2e_step)          # contexts, buffers and autotuned shapes, outside the clock
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        list(ex.map(e2e_step, range(args.steps)))
        e2e_local = (time.perf_counter() - t0) / args.steps

        def drop():
            tls.keep = None
        on_every_worker(drop)              # plans and results go on their own threads
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(e2e_local, dist, device="cuda")
    h2d = sum(24 * len(x.circuit.gates) + 8 * len(x.cuts or []) + 4 * len(x.marginal) +
              4 * sum(len(z) + 1 for z in x.zstrings) for x in ws)
    d2h = 8 * sum((1 << len(x.marginal)) + len(x.zstrings) for x in ws)

    pk, pk_kind = peaks()
    tune_info = {"hub_counters": "8-bit" if tuning[3] < 0 else "16-bit", "variant_path": bool(tuning[4])}
    roofs = stage_rooflines(stage, ws, prob_infos, pk, pk_kind, args.precision, args.workload, tune_info)
    roof = dict(roofs[dom], stage=dom, kernel=stage_kernel(dom, args.precision, tune_info, ws, prob_infos))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64/" + args.precision, "data": "synthetic",
            "config": {"workload": describe(ws) + ("; cut sets searched by ccs_build_fragments"
                                                   if any(x.cuts is None for x in ws_in) else ""),
                       "variant_shots_per_step": units_per_step,
                       "l2": "flushed between steps (512 MB write, outside the step events)",
                       "parallelism": (f"{world} ranks, each its own batch (other Philox seeds"
                                       f"{', other circuits' if len(ws) > 1 else ''}); no collective"),
                       "launch": ("plain: per-variant simulation, stream launches" if args.plain else
                                  "two CUDA-graph replays per step (evaluation, recombination)"),
                       "recombination": args.precision + (" (tcgen05 where eligible)" if args.precision == "bf16" else
                                                          " (CUDA-core FMA, FP64 across splits)"),
                       "tuning": {"threads": tuning[0], "words_per_op": tuning[1], "shots_per_cta": tuning[2],
                                  "hub_threads": abs(tuning[3]),
                                  "hub_counters": "8-bit" if tuning[3] < 0 else "16-bit",
                                  "path": "per-variant simulation" if tuning[4] else "shared bodies + screen",
                                  "autotuned": tune}},
            "circuits_per_s": world * len(ws) * args.steps / t_tot,
            "stage_ms": stage, "roofline": roof, "stage_roofline": roofs,
            "e2e": {"value": units_per_step * world / e2e_s, "unit": UNIT, "circuits_per_s": world * len(ws) / e2e_s,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "pipeline": f"{E2E_WORKERS} host worker threads, each serving one step at a time "
                                "(build, upload, evaluation, recombination, read-back to pinned host "
                                "memory) on its own context and stream; contexts on the library's "
                                "stream-ordered pool"},
            "gpu_launches": launches, "clocks": clocks}

    # --- the same run's other forms: BF16 tensor-core contraction, plain GPU form
    if not args.plain and not args.no_extras:
        k2 = max(3, min(args.steps, 10))
        if prec == ccs.CCS_FP32:
            for _ in range(2):
                step(ccs.CCS_BF16)
            t16 = max_over_ranks(timed(lambda: step(ccs.CCS_BF16), k2), dist, device="cuda")
            line["bf16"] = {"value": units_per_step * k2 * world / t16, "ms_per_step": 1e3 * t16 / k2,
                            "circuits_per_s": world * len(ws) * k2 / t16,
                            "recombination": "bf16 operands, tcgen05 where eligible, FP32 accumulation"}
        # Clifford-specific stitching (no shots: the hub operand in closed form,
        # vanishing rows skipped); the same circuits, exact results
        ev_s = dict(mode=ccs.CCS_STITCH, per_variant_body=False)
        res_s = ccs.ccs_eval_variants(ctx, plan, use_graph=True, **ev_s)

        def stitch_step():
            ccs.ccs_eval_variants(ctx, plan, use_graph=True, res=res_s, **ev_s)
            ccs.ccs_recombine(ctx, plan, res_s, precision=ccs.CCS_FP32, marginal_out=marg, zexp_out=zexp,
                              use_graph=True)

        for _ in range(2):
            stitch_step()
        ts = max_over_ranks(timed(stitch_step, k2), dist, device="cuda")
        line["stitched"] = {"ms_per_step": 1e3 * ts / k2, "circuits_per_s": world * len(ws) * k2 / ts,
                            "variants_per_s": n_cliff_var * k2 * world / ts,
                            "mode": "Clifford-specific stitching (exact; no shots; zero Pauli rows skipped)"}
        del res_s
        # maximum-likelihood correction of the sampled fragment models (Sec. V-C)
        # between evaluation and contraction, on the same result
        wide = max(i["n_slots"] for i in infos if i["clifford"]) if n_cliff_var else 0
        if wide > 6:
            line["ml"] = {"unsupported": f"a Clifford fragment with {wide} cut slots (the correction takes <= 6)"}
        elif n_cliff_var:
            def ml_step():
                ccs.ccs_eval_variants(ctx, plan, use_graph=graph, res=res, **ev)
                ccs.ccs_ml_correct(ctx, plan, res)
                ccs.ccs_recombine(ctx, plan, res, precision=ccs.CCS_FP32, marginal_out=marg, zexp_out=zexp,
                                  use_graph=graph)

            for _ in range(2):
                ml_step()
            tm = max_over_ranks(timed(ml_step, k2), dist, device="cuda")
            line["ml"] = {"ms_per_step": 1e3 * tm / k2, "circuits_per_s": world * len(ws) * k2 / tm,
                          "value": units_per_step * k2 * world / tm,
                          "form": "sampled evaluation, maximum-likelihood correction of the Clifford fragment "
                                  "models, FP32 contraction"}
        ev_p = dict(ev, per_variant_body=True)
        res_p = ccs.ccs_eval_variants(ctx, plan, **ev_p)

        def plain_step():
            ccs.ccs_eval_variants(ctx, plan, res=res_p, **ev_p)
            ccs.ccs_recombine(ctx, plan, res_p, precision=ccs.CCS_FP32, marginal_out=marg, zexp_out=zexp)

        kp = max(2, min(args.steps, 5))
        plain_step()
        tp = max_over_ranks(timed(plain_step, kp), dist, device="cuda")
        line["plain"] = {"value": units_per_step * kp * world / tp, "ms_per_step": 1e3 * tp / kp,
                         "circuits_per_s": world * len(ws) * kp / tp,
                         "form": "per-variant simulation of each variant's whole circuit, stream launches, "
                                 "FP32 contraction, default launch shapes"}
        del res_p
    if rank == 0 and world == 1 and not args.no_cpu_baseline:   # the oracle baseline at N = 1 only
        line["cpu_baseline"] = oracle_baseline(ws)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def _spawned(local_rank, world, port, argv):
    os.environ.update(RANK=str(local_rank), LOCAL_RANK=str(local_rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.argv = [sys.argv[0]] + argv
    main()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="config3")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the BF16 and plain-form figures")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16"],
                    help="operands of the 4^k contraction (bf16 uses the tcgen05 GEMM where it applies)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
    ap.add_argument("--per-variant-body", action="store_true",
                    help="simulate every variant's whole circuit (no shared fragment body)")
    ap.add_argument("--plain", action="store_true",
                    help="the plain GPU form: per-variant simulation, no CUDA graph, FP32, no autotuning")
    args = ap.parse_args()
    if "WORLD_SIZE" not in os.environ and args.gpus > 1:
        # started without a launcher: one spawned rank per GPU
        import torch.multiprocessing as mp
        port = 29400 + os.getpid() % 1000
        mp.start_processes(_spawned, args=(args.gpus, port, sys.argv[1:]), nprocs=args.gpus, start_method="spawn")
        return
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
