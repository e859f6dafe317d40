"""Benchmark: sigma = H c Slater-Condon pairs per second on GB300.

One step is one sigma = H c over the whole selected determinant space (every kernel of
the hot path: diagonal term, double-excitation and single-excitation kernels), with the
integrals, determinant tables and c resident in HBM.  Default workload: 30 spatial
orbitals, 10 alpha + 10 beta electrons, 2,000,000 selected determinants (HF + all singles
and doubles + seeded random triples/quadruples), Cholesky rank 120, FP64, one vector.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload sel_30o|sel_64s|fci_8o]
                    [--nvec V] [--impl gb300|reference]

Beside the headline step, the default run times the side sections: the 8-root Davidson
solvers (FP64 against FP32-refined), the density matrices and autograd energy, the 64
batched instances, ENPT2, and one sigma on the 1,000,000-determinant 64-spinor complex
space (`spinor`), each with its own figures.

Under torchrun (N > 1) the ranks share the sigma of one space: each holds the whole
determinant list and the integrals, computes a contiguous range of rows balanced by the
rows' connection counts, and one NCCL all-gather of the row slices ends the step (the
paper's Sec. 3.1 split: static data replicated, results merged).  Strong scaling: the
value is the space's pairs per step / the slowest rank's time per step.
`--impl reference` times the CPU oracle (the only reference implementation: the paper
ships no code) on a bounded sample of rows of the same workload.
"""
from __future__ import annotations

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

from paper_2501_18185_gb300 import workloads as W  # noqa: E402

METRIC = "sigma Slater-Condon pairs/sec"
UNIT = "pairs/s"
GOLDEN = os.path.join(ROOT, "tests", "golden", "pair_counts.json")
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0


def make_workload(name: str, nvec: int, M: int | None = None):
    if name == "sel_30o":
        return W.selected_30o(nvec=nvec) if M is None else W.selected_30o(M=M, nvec=nvec)
    if name == "sel_64s":
        return W.selected_spinor_64(nvec=nvec) if M is None else W.selected_spinor_64(M=M, nvec=nvec)
    if name == "fci_8o":
        return W.fci_small_8o()
    raise SystemExit(f"unknown workload {name}")


def golden_pairs(w):
    try:
        return json.load(open(GOLDEN)).get(w.name, {}).get("pairs")
    except (OSError, ValueError):
        return None


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """The largest x over the ranks of the process group (a job lasts as long as its
    slowest rank); x itself without a group."""
    if dist is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(pairs_per_step: int, steps: int, world: int, total_ms: float) -> float:
    """Whole-job pairs/s when every rank runs its own replica of `pairs_per_step` pairs per
    step (weak scaling), timed by the slowest rank's total."""
    return world * pairs_per_step * steps / (total_ms / 1e3)


def split_throughput(pairs_per_step: int, steps: int, total_ms: float) -> float:
    """Whole-job pairs/s when the ranks share one sigma of `pairs_per_step` pairs per step
    (row split, strong scaling), timed by the slowest rank's total."""
    return pairs_per_step * steps / (total_ms / 1e3)


def measured_peaks() -> dict:
    """The measured copy-bandwidth and GEMM peaks of MEASURED_PEAKS.json ({} when the file is absent)."""
    try:
        return json.load(open(PEAKS))
    except (OSError, ValueError):
        return {}


def hbm_peak():
    try:
        return float(json.load(open(PEAKS))["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return FALLBACK_HBM_GBS, "fallback"


_PIPE_PEAKS = {}


def pipe_peaks(device: int) -> dict:
    """Measured FMA rates of the FP64 and FP32 pipes of this GPU (sci_peak_fma: 8 CTAs of
    256 threads per SM, 8 independent FMA chains per thread, CUDA events), once per
    process; with the SM clock seen right after the timed launch (nvidia-smi)."""
    if device in _PIPE_PEAKS:
        return _PIPE_PEAKS[device]
    from paper_2501_18185_gb300 import sci

    f64 = max(sci.sci_peak_fma(device, sci.SCI_PREC_F64, 2500) for _ in range(3))
    f32 = max(sci.sci_peak_fma(device, sci.SCI_PREC_F32_STORE_F64_ACC, 160000) for _ in range(3))
    mhz = None
    try:
        out = subprocess.run(["nvidia-smi", f"--id={device}", "--query-gpu=clocks.sm", "--format=csv,noheader,nounits"],
                             capture_output=True, text=True, timeout=20).stdout.strip()
        mhz = float(out.splitlines()[0])
    except (OSError, ValueError, IndexError, subprocess.SubprocessError):
        pass
    _PIPE_PEAKS[device] = {"fp64_fma_per_s": f64, "fp32_fma_per_s": f32, "sm_mhz_after": mhz,
                           "how": "sci_peak_fma: best of 3 timed launches (8 CTAs x 256 threads per SM, "
                                  "8 independent FMA chains per thread)"}
    return _PIPE_PEAKS[device]


def profile_figures(key: str) -> dict:
    """Per-launch DRAM and L2 bytes of the doubles kernel for a workload, from the ncu
    summaries in profiles/traffic.json ({} if absent)."""
    try:
        d = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    except (OSError, ValueError):
        return {}
    return {"dram": d.get(key), "l2": d.get("l2:" + key), "l2_note": d.get("_l2_note")}


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.3)

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_model() -> str:
    """The host CPU as /proc/cpuinfo names it (model name, or the Arm implementer and part
    numbers when there is no model name)."""
    try:
        info = open("/proc/cpuinfo").read().splitlines()
    except OSError:
        return "unknown"
    for key in ("model name", "Model name"):
        for ln in info:
            if ln.startswith(key):
                return ln.split(":", 1)[1].strip()
    fields = {}
    for ln in info:
        if ":" in ln:
            k, v = (x.strip() for x in ln.split(":", 1))
            fields.setdefault(k, v)
    if "CPU implementer" in fields:
        return f"implementer {fields['CPU implementer']} part {fields.get('CPU part', '?')}"
    return "unknown"


def cpu_baseline(w, budget_s: float = 12.0, seed: int = 0, one_thread_s: float = 5.0):
    """Time the CPU oracle, as it stands, on a bounded random sample of rows: on all the
    host's cores (the reported value) and on one thread (`one_thread`)."""
    import oracle
    from oracle import Oracle

    o = Oracle.from_workload(w)
    rng = np.random.default_rng(seed)
    cores = len(os.sched_getaffinity(0))

    def sample(threads, budget):
        oracle.set_threads(threads)
        try:
            rows = np.sort(rng.choice(w.M, min(w.M, 100), replace=False))
            t = time.perf_counter()
            o.sigma_rows(rows, w.c)
            per_row = (time.perf_counter() - t) / len(rows)
            n = int(min(w.M, max(100, budget / max(per_row, 1e-9))))
            rows = np.sort(rng.choice(w.M, n, replace=False))
            t = time.perf_counter()
            o.sigma_rows(rows, w.c)
            dt = time.perf_counter() - t
        finally:
            oracle.set_threads(0)
        pairs = sum(len(o.connections(int(r))[0]) for r in rows)
        return pairs / dt, f"{n} random rows of {w.M} ({pairs} pairs, {dt:.1f} s, OpenMP {threads} threads)"

    v, smp = sample(cores, budget_s)
    v1, smp1 = sample(1, one_thread_s)
    return {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": smp, "cpu": cpu_model(),
            "one_thread": {"value": v1, "unit": UNIT, "cores": 1, "sample": smp1}}


def kato_temple(energies, residuals, nroots, target=1e-8, floor=1e-12):
    """From the Ritz values e_j of a reference run (at least nroots + 1 of them) and their
    residual norms r_j: for each of the first nroots, the Kato-Temple gap
        delta_k = min_{j != k} (|e_k - e_j| - r_j)   (clamped below at `floor`),
    a lower bound on the distance from e_k to the rest of the exact spectrum (each exact
    eigenvalue lies within r_j of some e_j), the bounds r_k^2 / delta_k on |E_k - exact|,
    and the residual sqrt(target * min delta) that bounds every root's error by `target`."""
    e = np.asarray(energies, dtype=np.float64)
    r = np.asarray(residuals, dtype=np.float64)
    assert len(r) == len(e) and len(e) > nroots
    gaps = np.array([max(floor, min(abs(e[k] - e[j]) - r[j] for j in range(len(e)) if j != k))
                     for k in range(nroots)])
    return gaps, r[:nroots] ** 2 / gaps, float(np.sqrt(target * gaps.min()))


def davidson_bench(H, w, nroots=8, tol=1e-6):
    """Time to the lowest `nroots` energies: plain FP64 Davidson against the FP32-storage
    block Davidson with FP64 refinement (its residual estimates in paired FP32, and in
    FP64 beside it; with paired-FP32 block kernels throughout; and plain Davidson on the
    FP64-accurate paired-FP32 sigma).
    E_ref is a tight FP64 run (residual 1e-8) with one extra root, so that each energy's
    Kato-Temple bound r^2 / gap is reported; every energy's error against it is reported.
    Both solvers run at residual `tol` and again at the residual sqrt(1e-8 * min gap),
    which by the same bound puts every energy within 1e-8 Eh of the exact one.  Wall-clock seconds, each solver timed after
    one untimed warm-up sigma; the sigma time of each precision at `nroots` vectors is
    reported beside them (CUDA events, mean of 5)."""
    import torch

    from paper_2501_18185_gb300 import sci
    from paper_2501_18185_gb300.davidson import davidson, davidson_mixed

    diag = H.diagonal()

    def hi(X):
        return H.sigma(X.contiguous())

    def lo(X):
        return H.sigma(X.to(torch.float32).contiguous(), prec=sci.SCI_PREC_F32_STORE_F64_ACC)

    def ds(X):
        return H.sigma(X.contiguous(), prec=sci.SCI_PREC_F64_DS)

    probe = torch.zeros((H.M, nroots), dtype=torch.float64, device=H.device)
    sig_ms = {}
    for name, f in (("fp64", hi), ("fp32_storage", lo), ("ds", ds)):
        f(probe)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(5):
            f(probe)
        e1.record()
        torch.cuda.synchronize()
        sig_ms[name] = e0.elapsed_time(e1) / 5
    # one root more than asked, so that every reference energy has a gap on both sides
    ref = davidson(hi, diag, nroots=nroots + 1, tol=1e-8, max_iter=1000)
    e_all = ref.energies.cpu().numpy()
    r_all = ref.residual_norms.cpu().numpy()
    e_ref = e_all[:nroots]
    # Kato-Temple: |E_k - exact| <= r_k^2 / gap_k; the residual that guarantees 1e-8 Eh
    # for every root is sqrt(1e-8 * min gap)
    gaps, bounds, tol_1e8 = kato_temple(e_all, r_all, nroots)
    out = {"nroots": nroots, "residual_tol": tol, "ref_residual": 1e-8, "ref_converged": bool(ref.converged),
           "E_ref": [float(x) for x in e_ref], "ref_error_bound_Eh": float(bounds.max()),
           "min_gap_Eh": float(gaps.min()), "residual_tol_for_1e-8_Eh": tol_1e8, f"sigma_ms_nvec{nroots}": sig_ms}
    for name, run in (("fp64", lambda: davidson(hi, diag, nroots=nroots, tol=tol, max_iter=600)),
                      ("fp32_refined", lambda: davidson_mixed(lo, hi, diag, nroots=nroots, tol=tol, max_iter=600)),
                      ("fp32_refined_f64_estimates", lambda: davidson_mixed(lo, hi, diag, nroots=nroots, tol=tol,
                                                                            max_iter=600, est_arith="f64")),
                      ("fp32_refined_dsblock", lambda: davidson_mixed(lo, hi, diag, nroots=nroots, tol=tol,
                                                                      max_iter=600, arith="ds")),
                      ("ds", lambda: davidson(ds, diag, nroots=nroots, tol=tol, max_iter=600)),
                      ("fp64_at_1e-8_Eh", lambda: davidson(hi, diag, nroots=nroots, tol=tol_1e8, max_iter=600)),
                      ("fp32_refined_at_1e-8_Eh", lambda: davidson_mixed(lo, hi, diag, nroots=nroots, tol=tol_1e8,
                                                                         max_iter=600))):
        torch.cuda.synchronize()
        t = time.perf_counter()
        res = run()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        err = np.abs(res.energies.cpu().numpy() - e_ref)
        out[name] = {"seconds": dt, "converged": bool(res.converged), "iterations": res.iterations,
                     "sigma_calls": res.sigma_calls, "max_abs_err_Eh": float(err.max()),
                     "errors_Eh": [float(x) for x in err]}
        if name.startswith("fp32_refined"):
            out[name]["sigma_calls_fp32"] = res.sigma_calls_lo
            out[name]["sigma_calls_fp64"] = res.sigma_calls_hi
    out["speedup_fp32_refined_vs_fp64"] = out["fp64"]["seconds"] / out["fp32_refined"]["seconds"]
    out["speedup_fp32_refined_vs_fp64_at_1e-8_Eh"] = (out["fp64_at_1e-8_Eh"]["seconds"]
                                                       / out["fp32_refined_at_1e-8_Eh"]["seconds"])
    return out


def rdm_bench(H, w, nvec=4, reps=3):
    """Density matrices and the autograd energy on the bench space with `nvec` vectors
    (seeded normal coefficients, normalised; the cost does not depend on the values):
    CUDA-event milliseconds of sci_rdm12 without and with the 2-RDM, and of one forward +
    backward of the Rayleigh-quotient energy with respect to h, the Cholesky factors and
    C (mean of `reps` after one warm-up)."""
    import torch

    from paper_2501_18185_gb300.autograd import rayleigh_energy

    g = torch.Generator(device="cpu").manual_seed(5)
    C = torch.randn((H.M, nvec), generator=g, dtype=torch.float64).to(H.device)
    C /= torch.linalg.vector_norm(C, dim=0)
    h = torch.from_numpy(w.ints.h.copy()).to(H.device)
    L = torch.from_numpy(w.ints.chol.copy()).to(H.device)

    def ev_ms(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    def fwd_bwd():
        hh, LL, CC = h.clone().requires_grad_(True), L.clone().requires_grad_(True), C.clone().requires_grad_(True)
        rayleigh_energy(hh, LL, CC, H).sum().backward()

    out = {"nvec": nvec, "norb": H.norb,
           "rdm1_ms": ev_ms(lambda: H.rdm12(C, rdm2=False)),
           "rdm12_ms": ev_ms(lambda: H.rdm12(C)),
           "energy_forward_backward_ms": ev_ms(fwd_bwd)}
    # the energy path re-uploaded the same integrals: leave the context as it was
    H.set_integrals(w.mode, w.ints.h, chol=w.ints.chol)
    return out


def blockvec_bench(M=2_000_000, k=96, a=8, reps=5):
    """The tall-skinny products of the 8-root Davidson at its largest shapes (k = 96
    search vectors, blocks of a = 8, M rows): CUDA-event milliseconds (L2 flushed before
    each launch) of sci_bv_gemm_tn (P = [V T]^T T over k + a columns) and sci_bv_gemm_nn
    (the residual R = W Y - V (Y theta) with the preconditioner epilogue), FP64 and paired
    FP32.  Roofline: the FP64 policy is bound by the FP64 pipe, whose peak is derived as
    2 FMA per clock per SM x SMs x the maximum SM clock; the paired policy is reported
    against the same FP64-equivalent work."""
    import torch

    from paper_2501_18185_gb300 import sci

    dev = torch.device("cuda", torch.cuda.current_device())
    g = torch.Generator(device="cpu").manual_seed(9)
    V = torch.randn((M, k + a), generator=g, dtype=torch.float64).to(dev)
    W = torch.randn((M, k), generator=g, dtype=torch.float64).to(dev)
    Y = torch.randn((k, a), generator=g, dtype=torch.float64).to(dev)
    th = torch.linspace(-3, -1, a, dtype=torch.float64).to(dev)
    Yt = (-(Y * th[None, :])).contiguous()
    d = torch.randn(M, generator=g, dtype=torch.float64).to(dev)
    P = torch.empty((k + a, a), dtype=torch.float64, device=dev)
    R = torch.empty((M, a), dtype=torch.float64, device=dev)
    cs = torch.zeros(a, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 8, dtype=torch.float64, device=dev)
    ctx = sci.sci_create(dev.index, torch.cuda.current_stream().cuda_stream)
    stream = torch.cuda.current_stream()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks = measured_peaks()
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    fp64_peak = 2 * 2 * sms * mhz * 1e6 / 1e12   # TFLOP/s

    def ev_ms(fn):
        fn()
        out = []
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            out.append(e0.elapsed_time(e1))
        return statistics.median(out)

    res = {"M": M, "k": k, "a": a, "fp64_peak_tflops": fp64_peak,
           "peak_source": f"derived: 2 FP64 FMA/clk/SM x {sms} SMs x {mhz:.0f} MHz"}
    flops_tn, flops_nn = 2.0 * M * (k + a) * a, 2.0 * M * 2 * k * a
    for name, prec in (("f64", sci.SCI_PREC_F64), ("ds", sci.SCI_PREC_F64_DS)):
        t_tn = ev_ms(lambda: sci.sci_bv_gemm_tn(ctx, M, k + a, a, V, k + a, V[:, k:], k + a, P, prec))
        t_nn = ev_ms(lambda: sci.sci_bv_gemm_nn(ctx, M, a, W, k, k, Y, V, k + a, k, Yt, 0.0, R, a, d, th, cs, prec))
        res[name] = {"tn_ms": t_tn, "nn_ms": t_nn,
                     "tn_GBps": M * (k + a) * 8 / t_tn / 1e6, "nn_GBps": (M * 2 * k * 8 + M * a * 16) / t_nn / 1e6}
        if name == "f64":   # FP64 FMAs on the FP64 pipe: a fraction of that pipe's peak
            res[name].update({"tn_tflops": flops_tn / t_tn / 1e9, "nn_tflops": flops_nn / t_nn / 1e9,
                              "tn_frac_fp64_peak": flops_tn / t_tn / 1e9 / fp64_peak,
                              "nn_frac_fp64_peak": flops_nn / t_nn / 1e9 / fp64_peak})
        else:               # paired FP32 on the FP32 pipes: FP64-equivalent rate, no FP64-pipe fraction
            res[name].update({"tn_fp64_equiv_tflops": flops_tn / t_tn / 1e9,
                              "nn_fp64_equiv_tflops": flops_nn / t_nn / 1e9})
    VT = V[:, :k + a]
    res["cublas_f64_tn_ms"] = ev_ms(lambda: VT.T @ V[:, k:])
    sci.sci_destroy(ctx)
    return res


def pt2_bench(sizes=(60_000, 200_000, 1_000_000, 2_000_000), table_gb=16.0):
    """Epstein-Nesbet PT2 of the ground state on spaces of the bench recipe: (E0, c) from
    the FP64 block Davidson (residual 1e-6), then exact sci_enpt2 (no screening).  Wall
    seconds of sci_enpt2 (synchronous), batches, distinct determinants of W summed, the
    generated contributions (M x excitations per determinant) and E2[Q]."""
    import torch

    from paper_2501_18185_gb300 import sci
    from paper_2501_18185_gb300 import workloads as W

    out = []
    for M in sizes:
        w = W.selected_30o(M=M)
        H = sci.Hamiltonian.from_workload(w)
        from paper_2501_18185_gb300.davidson import davidson

        r = davidson(lambda X: H.sigma(X.contiguous()), H.diagonal(), nroots=1, tol=1e-6, max_iter=400)
        c = r.vectors.contiguous()
        E0 = [float(r.energies[0])]
        torch.cuda.synchronize()
        t = time.perf_counter()
        e2w, e2p, e2q, st = H.enpt2(c, E0, table_bytes=int(table_gb * (1 << 30)))
        dt = time.perf_counter() - t
        # the same with screening (eps = 1e-7): classes skipped by the bounds of their
        # elements, single contributions below eps dropped
        torch.cuda.synchronize()
        t = time.perf_counter()
        s2w, s2p, s2q, sst = H.enpt2(c, E0, eps=1e-7, table_bytes=int(table_gb * (1 << 30)))
        dts = time.perf_counter() - t
        screened = {"eps": 1e-7, "seconds": dts, "E2_Q": float(s2q[0]), "distinct_W": sst["distinct_W"],
                    "batches": sst["batches"]}
        n, na, nb = w.n, w.n_alpha, w.n_beta
        ua, ub = n - na, n - nb
        per = na * ua + nb * ub + na * (na - 1) // 2 * (ua * (ua - 1) // 2) + nb * (nb - 1) // 2 * (ub * (ub - 1) // 2) \
            + na * ua * nb * ub
        out.append({"M": M, "seconds": dt, "davidson_converged": bool(r.converged), "E0": E0[0],
                    "E0_plus_E2": E0[0] + float(e2q[0]), "E2_Q": float(e2q[0]), "E2_W": float(e2w[0]),
                    "E2_P": float(e2p[0]), "generated": M * per, "generated_per_s": M * per / dt, **st,
                    "screened": screened})
        del H
        torch.cuda.empty_cache()
    return out


def pt2_spinor_bench(M=200_000, table_gb=16.0):
    """Epstein-Nesbet PT2 in complex spinor mode (the 4C workloads of the paper's Sec. 4) on
    a space of the 64-spinor recipe: c is the recipe's complex vector (|c| = exp(-level),
    random phases), normalised, and E0 its Rayleigh quotient c^+ H c; exact sci_enpt2 (no
    screening), wall seconds (synchronous), batches, distinct W and the generated count
    (M x (N (n - N) + C(N,2) C(n - N, 2)))."""
    import torch

    from paper_2501_18185_gb300 import sci

    w = W.selected_spinor_64(M=M)
    H = sci.Hamiltonian.from_workload(w)
    c = torch.from_numpy(np.ascontiguousarray(w.c)).cuda()
    c = c / torch.linalg.vector_norm(c)
    E0 = [float((c.conj() * H.sigma(c)).sum().real)]
    H.enpt2(c, E0, table_bytes=1 << 28)   # warm-up: loads the kernels
    torch.cuda.synchronize()
    t = time.perf_counter()
    e2w, e2p, e2q, st = H.enpt2(c, E0, table_bytes=int(table_gb * (1 << 30)))
    dt = time.perf_counter() - t
    n, N = w.n, w.n_alpha
    per = N * (n - N) + N * (N - 1) // 2 * ((n - N) * (n - N - 1) // 2)
    out = {"workload": w.name, "M": M, "seconds": dt, "E0": E0[0], "E2_Q": float(e2q[0]), "E2_W": float(e2w[0]),
           "E2_P": float(e2p[0]), "generated": M * per, "generated_per_s": M * per / dt, **st}
    del H
    torch.cuda.empty_cache()
    return out


def batch_bench(reps=10):
    """The 64 heterogeneous full-CI instances in one persistent launch: setup, autotuner
    time and choices, and CUDA-event milliseconds per batched sigma (L2 flushed before
    each timed launch) for the graph-captured AUTO plan, the all-TILE and all-WARP plans,
    and the 64 instances' own sci_sigma calls one after another."""
    import torch

    from paper_2501_18185_gb300 import sci
    from paper_2501_18185_gb300 import workloads as W

    t = time.perf_counter()
    ws = W.batch_instances()
    hams = [sci.Hamiltonian.from_workload(w) for w in ws]
    setup_s = time.perf_counter() - t
    C = torch.from_numpy(np.concatenate([w.c[:, 0] for w in ws])).cuda()
    S = torch.empty_like(C)
    flush = torch.empty(256 * 1024 * 1024 // 8, dtype=torch.float64, device=C.device)
    stream = torch.cuda.current_stream()

    def ev_ms(fn):
        fn()
        out = []
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            out.append(e0.elapsed_time(e1))
        return statistics.median(out)

    B = sci.Batch(hams)
    res = {"instances": len(ws), "M_total": B.M, "setup_s": round(setup_s, 3)}
    for name, sch in (("tile", sci.SCI_SCHED_TILE), ("warp", sci.SCI_SCHED_WARP)):
        B.plan(sch)
        res[f"ms_all_{name}"] = ev_ms(lambda: B.sigma(C, out=S))
    t = time.perf_counter()
    B.plan(sci.SCI_SCHED_AUTO, C, S)
    res["autotune_s"] = round(time.perf_counter() - t, 3)
    B.capture(C, S)
    res["ms_auto_graph"] = ev_ms(B.replay)
    res["ms_instances_one_by_one"] = ev_ms(
        lambda: [H.sigma(C[o:o + H.M], out=S[o:o + H.M].view(-1, 1)) for H, o in zip(hams, B.offsets)])
    it = B.items()
    res.update({"pairs": it["pairs"], "work_items": it["items"], "persistent_ctas": it["ctas"],
                "pairs_per_s_auto_graph": it["pairs"] / (res["ms_auto_graph"] / 1e3),
                "schedules": {k: sum(1 for i in range(len(ws)) if B.info(i)["schedule"] == k) for k in ("tile", "warp")},
                "l2": "flushed before each timed launch (256 MB write)"})
    res["ground_states"] = batch_ground_states(ws, hams)
    return res


def batch_ground_states(ws, hams, tol=1e-8):
    """Lowest eigenpair of all 64 instances: the batched Davidson (one graph-replayed
    batched sigma per iteration; its time includes the batch's autotuned plan and graph
    capture) against the single-instance FP64 Davidson run on each instance in turn, both
    with 32-column spaces and restarts keeping 4 vectors (wall seconds, synchronised)."""
    import torch

    from paper_2501_18185_gb300 import sci
    from paper_2501_18185_gb300.batch_davidson import davidson_batched
    from paper_2501_18185_gb300.davidson import davidson

    # untimed warm-up of both solvers on the two smallest instances: the first use of
    # each kernel in a process loads its code (seconds on a fresh machine)
    small = sorted(hams, key=lambda H: H.M)[:2]
    davidson_batched(sci.Batch(small), tol=1e-6, max_iter=20)
    davidson(lambda Y: small[0].sigma(Y.contiguous()), small[0].diagonal(), nroots=1, tol=1e-6, max_iter=20,
             max_space=32, keep=4)
    B = sci.Batch(hams)
    torch.cuda.synchronize()
    t = time.perf_counter()
    r = davidson_batched(B, tol=tol, max_iter=400)
    torch.cuda.synchronize()
    batched_s = time.perf_counter() - t
    t = time.perf_counter()
    E1, conv1, calls1 = [], 0, 0
    for H in hams:
        one = davidson(lambda Y, H=H: H.sigma(Y.contiguous()), H.diagonal(), nroots=1, tol=tol, max_space=32,
                       keep=4)
        E1.append(float(one.energies[0]))
        conv1 += bool(one.converged)
        calls1 += one.sigma_calls
    torch.cuda.synchronize()
    one_s = time.perf_counter() - t
    return {"batched_s": round(batched_s, 3), "one_by_one_s": round(one_s, 3),
            "batched_iterations": r.iterations, "batched_sigma_launches": r.sigma_launches,
            "batched_converged": int(r.converged.sum()), "one_by_one_converged": conv1,
            "one_by_one_sigma_calls": calls1, "tol": tol,
            "max_abs_diff_Eh": float(np.abs(np.asarray(E1) - r.energies).max())}


def spinor_bench(device, steps=10, warmup=3):
    """The relativistic workload: 64 spinors, 14 electrons, 1,000,000 selected
    determinants, complex128 (HF, singles, doubles and seeded random triples; 80 complex
    Hermitian Cholesky vectors).  One sigma on one vector in FP64 and in paired FP32,
    each timed as the main bench (CUDA events, L2 flushed between steps, per-kernel
    events), with the doubles kernel's algorithmic-byte fraction of HBM (32 B per double
    pair), its useful FP64 FMAs (4 per complex double pair) against the measured FP64
    pipe rate, and the CPU oracle on sampled rows of the same space."""
    import torch

    from paper_2501_18185_gb300 import sci

    dev = torch.device("cuda", device)
    w = W.selected_spinor_64()
    t = time.perf_counter()
    H = sci.Hamiltonian.from_workload(w, device=device)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t
    info = H.info()
    gp = golden_pairs(w)
    if gp is not None and gp != info["pairs"]:
        raise SystemExit(f"spinor pair count {info['pairs']} differs from the oracle's {gp}")
    C = torch.from_numpy(np.ascontiguousarray(w.c)).to(dev)
    S = torch.empty_like(C)
    flush = torch.empty(256 * 1024 * 1024 // 8, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    peak, peak_kind = hbm_peak()
    pp = pipe_peaks(device)
    sci.sci_profile(H.ctx, True)
    out = {"workload": w.name, "M": w.M, "pairs_per_step": info["pairs"], "pairs_doubles": info["pairs_doubles"],
           "setup_s": round(setup_s, 3), "l2": "flushed between timed steps (256 MB write)"}
    for name, prec in (("f64", sci.SCI_PREC_F64), ("ds", sci.SCI_PREC_F64_DS)):
        for _ in range(warmup):
            H.sigma(C, out=S, prec=prec)
        ms, kern = [], []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            H.sigma(C, out=S, prec=prec)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            kern.append(sci.sci_kernel_times(H.ctx))
        m = statistics.mean(ms)
        dbl = statistics.mean(k[1] for k in kern)
        achieved = info["pairs_doubles"] * 32 / (dbl / 1e3) / 1e9
        out[name] = {"ms_per_step": m, "pairs_per_s": info["pairs"] / (m / 1e3),
                     "kernel_ms": {"init": statistics.mean(k[0] for k in kern), "doubles": dbl,
                                   "singles": statistics.mean(k[2] for k in kern)},
                     "doubles_alg_GBps": achieved, "doubles_alg_frac_hbm": achieved / peak}
        if name == "f64":
            fma = 4.0 * info["pairs_doubles"] / (dbl / 1e3)
            out[name]["fp64_pipe"] = {"useful_fma_per_s": fma, "peak_fma_per_s": pp["fp64_fma_per_s"],
                                      "frac": fma / pp["fp64_fma_per_s"]}
    sci.sci_profile(H.ctx, False)
    H.sync_status()
    out["hbm_peak"] = {"GBps": peak, "source": peak_kind}
    out["cpu_baseline"] = cpu_baseline(w, budget_s=8.0, one_thread_s=3.0)
    del H
    torch.cuda.empty_cache()
    return out


def two_word_bench(H, w, device, steps=10, warmup=3, M=2_000_000):
    """Occupation strings of more than 64 spin-orbitals (two or three 64-bit words per
    key).  (1) The bench space given as [M, 2] and [M, 3] keys with zero upper words: the
    same pairs through the multi-word set-up and singles code, against the one-word sigma
    of `H`.  (2) A selected space of 40 spatial orbitals (80 spin-orbitals, 8 alpha + 8
    beta electrons: HF, all singles and doubles, seeded random triples up to M) and (3) one
    of 70 spatial orbitals (140 spin-orbitals, 4 + 4 electrons, three words): FP64 sigma on
    one vector, CUDA-event milliseconds (L2 flushed), the doubles kernel's algorithmic-byte
    fraction of HBM and useful FMAs against the measured FP64 pipe rate, and the oracle
    on sampled rows.  (4) ENPT2 on a 200k cut of the 80 spin-orbital recipe."""
    import torch

    from paper_2501_18185_gb300 import sci

    dev = torch.device("cuda", device)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 8, dtype=torch.float64, device=dev)

    def timed(Hx, C, prec=sci.SCI_PREC_F64):
        S = torch.empty_like(C)
        for _ in range(warmup):
            Hx.sigma(C, out=S, prec=prec)
        sci.sci_profile(Hx.ctx, True)
        ms, kern = [], []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            Hx.sigma(C, out=S, prec=prec)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            kern.append(sci.sci_kernel_times(Hx.ctx))
        sci.sci_profile(Hx.ctx, False)
        Hx.sync_status()
        return S, statistics.mean(ms), {"init": statistics.mean(k[0] for k in kern),
                                        "doubles": statistics.mean(k[1] for k in kern),
                                        "singles": statistics.mean(k[2] for k in kern)}

    out = {}
    C = torch.from_numpy(np.ascontiguousarray(w.c)).to(dev)
    S1, ms1, k1 = timed(H, C)
    keys2 = np.zeros((w.M, 2), dtype=np.uint64)
    keys2[:, 0] = w.keys
    t = time.perf_counter()
    H2 = sci.Hamiltonian(device, stream)
    H2.set_integrals(w.mode, w.ints.h, chol=w.ints.chol)
    H2.set_determinants(keys2, w.n_alpha, w.n_beta)
    torch.cuda.synchronize()
    setup2 = time.perf_counter() - t
    if H2.count_pairs() != H.count_pairs():
        raise SystemExit("two-word pair count differs from the one-word count")
    S2, ms2, k2 = timed(H2, C)
    rel = float(torch.linalg.norm(S2 - S1) / torch.linalg.norm(S1))
    out["same_space_two_words"] = {"workload": w.name, "one_word_ms": ms1, "two_word_ms": ms2,
                                   "one_word_kernel_ms": k1, "two_word_kernel_ms": k2,
                                   "two_word_setup_s": round(setup2, 3), "rel_diff": rel}
    del H2, S2
    torch.cuda.empty_cache()
    keys3 = np.zeros((w.M, 3), dtype=np.uint64)
    keys3[:, 0] = w.keys
    t = time.perf_counter()
    H2 = sci.Hamiltonian(device, stream)
    H2.set_integrals(w.mode, w.ints.h, chol=w.ints.chol)
    H2.set_determinants(keys3, w.n_alpha, w.n_beta)
    torch.cuda.synchronize()
    setup3w = time.perf_counter() - t
    if H2.count_pairs() != H.count_pairs():
        raise SystemExit("three-word pair count differs from the one-word count")
    S3, ms3w, k3w = timed(H2, C)
    out["same_space_three_words"] = {"workload": w.name, "one_word_ms": ms1, "three_word_ms": ms3w,
                                     "three_word_kernel_ms": k3w, "three_word_setup_s": round(setup3w, 3),
                                     "rel_diff": float(torch.linalg.norm(S3 - S1) / torch.linalg.norm(S1))}
    del H2, S1, S3, C
    torch.cuda.empty_cache()

    w2 = W.selected_two_word(n=40, na=8, nb=8, M=M)
    t = time.perf_counter()
    H3 = sci.Hamiltonian.from_workload(w2, device=device)
    torch.cuda.synchronize()
    setup3 = time.perf_counter() - t
    info = H3.info()
    C = torch.from_numpy(np.ascontiguousarray(w2.c)).to(dev)
    _, ms3, k3 = timed(H3, C)
    peak, peak_kind = hbm_peak()
    pp = pipe_peaks(device)
    achieved = info["pairs_doubles"] * 16 / (k3["doubles"] / 1e3) / 1e9
    fma = info["pairs_doubles"] / (k3["doubles"] / 1e3)
    out["selected_80so"] = {"workload": w2.name, "M": w2.M, "pairs_per_step": info["pairs"],
                            "pairs_doubles": info["pairs_doubles"], "setup_s": round(setup3, 3),
                            "ms_per_step": ms3, "pairs_per_s": info["pairs"] / (ms3 / 1e3), "kernel_ms": k3,
                            "doubles_alg_GBps": achieved, "doubles_alg_frac_hbm": achieved / peak,
                            "fp64_pipe_frac": fma / pp["fp64_fma_per_s"],
                            "l2": "flushed between timed steps (256 MB write)",
                            "cpu_baseline": cpu_baseline(w2, budget_s=6.0, one_thread_s=2.0)}
    del H3, C
    torch.cuda.empty_cache()
    # three words: 70 spatial orbitals (140 spin-orbitals; alpha across words 0/1, beta
    # across words 1/2), 4 alpha + 4 beta electrons, the same recipe
    w3 = W.selected_three_word(n=70, na=4, nb=4, M=M)
    t = time.perf_counter()
    H3 = sci.Hamiltonian.from_workload(w3, device=device)
    torch.cuda.synchronize()
    setup3 = time.perf_counter() - t
    info = H3.info()
    C = torch.from_numpy(np.ascontiguousarray(w3.c)).to(dev)
    _, ms3, k3 = timed(H3, C)
    achieved = info["pairs_doubles"] * 16 / (k3["doubles"] / 1e3) / 1e9
    fma = info["pairs_doubles"] / (k3["doubles"] / 1e3)
    out["selected_140so"] = {"workload": w3.name, "M": w3.M, "pairs_per_step": info["pairs"],
                             "pairs_doubles": info["pairs_doubles"], "setup_s": round(setup3, 3),
                             "ms_per_step": ms3, "pairs_per_s": info["pairs"] / (ms3 / 1e3), "kernel_ms": k3,
                             "doubles_alg_GBps": achieved, "doubles_alg_frac_hbm": achieved / peak,
                             "fp64_pipe_frac": fma / pp["fp64_fma_per_s"],
                             "l2": "flushed between timed steps (256 MB write)",
                             "cpu_baseline": cpu_baseline(w3, budget_s=6.0, one_thread_s=2.0)}
    del H3, C
    torch.cuda.empty_cache()
    # three-word spinors: 136 complex spinors (the size of the paper's 4C spaces), 14
    # electrons, 1M determinants, FP64 and paired FP32; and ENPT2 of a 6-electron 150k space
    # (oracle not timed: its dense complex integrals would take 5.5 GB)
    w5 = W.selected_spinor_words(n=136, N=14, M=M // 2)
    t = time.perf_counter()
    H5 = sci.Hamiltonian.from_workload(w5, device=device)
    torch.cuda.synchronize()
    setup5 = time.perf_counter() - t
    info = H5.info()
    C = torch.from_numpy(np.ascontiguousarray(w5.c)).to(dev)
    _, ms5, k5 = timed(H5, C)
    _, ms5d, k5d = timed(H5, C, sci.SCI_PREC_F64_DS)
    fma = 4 * info["pairs_doubles"] / (k5["doubles"] / 1e3)   # a complex product is 4 FMAs
    out["selected_136s"] = {"workload": w5.name, "M": w5.M, "pairs_per_step": info["pairs"],
                            "pairs_doubles": info["pairs_doubles"], "max_bucket": info["max_bucket"],
                            "setup_s": round(setup5, 3), "f64": {"ms_per_step": ms5, "pairs_per_s": info["pairs"] / (ms5 / 1e3),
                                                               "kernel_ms": k5, "fp64_pipe_frac": fma / pp["fp64_fma_per_s"]},
                            "ds": {"ms_per_step": ms5d, "pairs_per_s": info["pairs"] / (ms5d / 1e3), "kernel_ms": k5d},
                            "l2": "flushed between timed steps (256 MB write)"}
    del H5, C
    torch.cuda.empty_cache()
    w6 = W.selected_spinor_words(n=136, N=6, M=150_000)
    H6 = sci.Hamiltonian.from_workload(w6, device=device)
    c = torch.from_numpy(np.ascontiguousarray(w6.c)).to(dev)
    c = c / torch.linalg.vector_norm(c)
    E0 = [float((c.conj() * H6.sigma(c)).sum().real)]
    torch.cuda.synchronize()
    t = time.perf_counter()
    e2w, e2p, e2q, st = H6.enpt2(c, E0, table_bytes=16 << 30)
    sec = time.perf_counter() - t
    out["pt2_136s"] = {"workload": w6.name, "M": w6.M, "seconds": sec, "E0": E0[0], "E2_Q": float(e2q[0]),
                       "batches": st["batches"], "distinct_W": st["distinct_W"],
                       "generate_us": st["generate_us"], "evaluate_us": st["evaluate_us"]}
    del H6, c
    torch.cuda.empty_cache()
    # ENPT2 of a 150k space of the 140 spin-orbital recipe (three words, spin-orbital mode)
    w7 = W.selected_three_word(n=70, na=4, nb=4, M=150_000)
    H7 = sci.Hamiltonian.from_workload(w7, device=device)
    c = torch.from_numpy(np.ascontiguousarray(w7.c)).to(dev)
    c = c / torch.linalg.vector_norm(c)
    E0 = [float((c * H7.sigma(c)).sum())]
    torch.cuda.synchronize()
    t = time.perf_counter()
    e2w, e2p, e2q, st = H7.enpt2(c, E0, table_bytes=16 << 30)
    sec = time.perf_counter() - t
    out["pt2_140so"] = {"workload": w7.name, "M": w7.M, "seconds": sec, "E0": E0[0], "E2_Q": float(e2q[0]),
                        "batches": st["batches"], "distinct_W": st["distinct_W"],
                        "generate_us": st["generate_us"], "evaluate_us": st["evaluate_us"]}
    del H7, c
    torch.cuda.empty_cache()
    # ENPT2 on a 200k-determinant space of the same recipe (128-bit table keys), one
    # normalised vector with its Rayleigh quotient as E0
    w4 = W.selected_two_word(n=40, na=8, nb=8, M=200_000)
    H4 = sci.Hamiltonian.from_workload(w4, device=device)
    c = torch.from_numpy(np.ascontiguousarray(w4.c)).to(dev)
    c = c / torch.linalg.vector_norm(c)
    E0 = [float((c * H4.sigma(c)).sum())]
    torch.cuda.synchronize()
    t = time.perf_counter()
    e2w, e2p, e2q, st = H4.enpt2(c, E0, table_bytes=16 << 30)
    sec = time.perf_counter() - t
    out["pt2_80so"] = {"workload": w4.name, "M": w4.M, "seconds": sec, "E0": E0[0], "E2_Q": float(e2q[0]),
                       "batches": st["batches"], "distinct_W": st["distinct_W"],
                       "generate_us": st["generate_us"], "evaluate_us": st["evaluate_us"]}
    del H4, c
    torch.cuda.empty_cache()
    return out


def deterministic_bench(H, w, steps=10):
    """sigma with deterministic accumulation (sci_set_deterministic: row sums stored per
    bucket entry, then summed per row in a fixed order) against the default FP64 atomics,
    on the bench workload's vector: CUDA-event milliseconds per step (L2 flushed), the four
    kernel times, the set-up seconds and device bytes of the mode, and whether two calls
    agree bit for bit."""
    import torch

    from paper_2501_18185_gb300 import sci

    dev = H.device
    stream = torch.cuda.current_stream(dev)
    C = torch.from_numpy(np.ascontiguousarray(w.c)).to(dev)
    S = torch.empty_like(C)
    flush = torch.empty(256 * 1024 * 1024 // 8, dtype=torch.float64, device=dev)

    def timed():
        H.sigma(C, out=S)
        ms, kern = [], []
        sci.sci_profile(H.ctx, True)
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            H.sigma(C, out=S)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            kern.append(sci.sci_kernel_times(H.ctx, 4))
        sci.sci_profile(H.ctx, False)
        return statistics.median(ms), [statistics.median(k[i] for k in kern) for i in range(4)]

    atomic_ms, atomic_k = timed()
    a1 = H.sigma(C).clone()
    a2 = H.sigma(C)
    b0 = H.info()["device_bytes"]
    t = time.perf_counter()
    H.set_deterministic(C.shape[1])
    setup = time.perf_counter() - t
    det_bytes = H.info()["device_bytes"] - b0
    det_ms, det_k = timed()
    d1 = H.sigma(C).clone()
    d2 = H.sigma(C)
    H.set_deterministic(0)
    H.sync_status()
    rel = float(torch.linalg.vector_norm(d1 - a1) / torch.linalg.vector_norm(a1))
    return {"atomic_ms": atomic_ms, "atomic_kernel_ms": atomic_k, "deterministic_ms": det_ms,
            "deterministic_kernel_ms": {"init": det_k[0], "doubles": det_k[1], "singles": det_k[2],
                                        "row_sums": det_k[3]},
            "setup_s": round(setup, 3), "device_bytes": det_bytes,
            "atomic_repeat_bitwise_equal": bool(torch.equal(a1, a2)),
            "deterministic_repeat_bitwise_equal": bool(torch.equal(d1, d2)),
            "rel_diff_deterministic_vs_atomic": rel}


def rowsplit_bench(H, parts=(2, 4, 8), steps=5):
    """The row split of the bench space, each rank timed alone on this GPU: for K ranks,
    the K ranges balanced by connection count + C(N, 2) per row, then for each range its
    set-up (range tables), its device bytes, its pairs and its sigma time (CUDA events, L2
    flushed, median of `steps` after one warm-up).  A K-GPU step takes the slowest rank's
    sigma plus one all-gather of sigma's M x 8 bytes; `speedup_vs_full` is the full
    sigma's time over the slowest rank's (the all-gather left out: not measurable on one
    GPU)."""
    import math

    import torch

    from paper_2501_18185_gb300 import partition as PT

    dev = H.device
    stream = torch.cuda.current_stream(dev)
    C = torch.ones((H.M, 1), dtype=torch.float64, device=dev) / math.sqrt(max(H.M, 1))
    S = torch.empty_like(C)
    flush = torch.empty(256 * 1024 * 1024 // 8, dtype=torch.float64, device=dev)

    def med_ms():
        H.sigma(C, out=S)
        out = []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            H.sigma(C, out=S)
            e1.record(stream)
            e1.synchronize()
            out.append(e0.elapsed_time(e1))
        return statistics.median(out)

    H.set_row_range(0, H.M)
    full_ms = med_ms()
    base_bytes = H.info()["device_bytes"]
    cost = H.row_costs().cpu().numpy()
    over = math.comb(H.n_electrons, 2)
    res = {"full_ms": full_ms, "row_weight": f"connected determinants + C(N,2) = {over}", "parts": {}}
    weights = PT.row_weights(cost, over)

    def time_ranges(ranges):
        ranks = []
        for b, e in ranges:
            t = time.perf_counter()
            H.set_row_range(b, e)
            setup = time.perf_counter() - t
            inf = H.info()
            ranks.append({"rows": [int(b), int(e)], "pairs": inf["pairs"], "setup_s": round(setup, 3),
                          "range_table_bytes": inf["device_bytes"] - base_bytes, "ms": med_ms()})
        H.set_row_range(0, H.M)
        mx = max(r["ms"] for r in ranks)
        return {"max_ms": mx, "mean_ms": statistics.mean(r["ms"] for r in ranks),
                "speedup_vs_full": full_ms / mx, "ranks": ranks}

    for K in parts:
        first = time_ranges(PT.balanced_ranges(weights, K))
        # one feedback round: the measured times re-cut the ranges (partition.rebalance)
        again = time_ranges(PT.rebalance(weights, [tuple(r["rows"]) for r in first["ranks"]],
                                         [r["ms"] for r in first["ranks"]]))
        res["parts"][str(K)] = {"by_weights": first, "rebalanced": again}
    H.sync_status()
    return res


def run_reference(args, rank, world):
    """--impl reference: the CPU oracle on bounded samples of the same workload."""
    if rank != 0:
        return
    from oracle import Oracle

    w = make_workload(args.workload, args.nvec, args.M)
    o = Oracle.from_workload(w)
    rng = np.random.default_rng(1)
    nrows = args.ref_rows
    samples = [np.sort(rng.choice(w.M, min(nrows, w.M), replace=False)) for _ in range(args.warmup + args.steps)]
    for s in samples[:args.warmup]:
        o.sigma_rows(s, w.c)
    tot_t, tot_p = 0.0, 0
    for s in samples[args.warmup:]:
        t = time.perf_counter()
        o.sigma_rows(s, w.c)
        tot_t += time.perf_counter() - t
        tot_p += sum(len(o.connections(int(r))[0]) for r in s)
    value = tot_p / tot_t
    cores = len(os.sched_getaffinity(0))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64" if not w.ints.complex_ else "c128",
            "data": "synthetic", "config": {"workload": w.name, "nvec": w.c.shape[1], "rows_per_step": int(nrows)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} x {nrows} random rows of {w.M}", "cpu": cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="sel_30o")
    ap.add_argument("--nvec", type=int, default=1)
    ap.add_argument("--M", type=int, default=None, help="smaller space of the same recipe (profiling)")
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--ref-rows", type=int, default=2000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-davidson", action="store_true",
                    help="skip the 8-root Davidson timing and the density-matrix timing")
    ap.add_argument("--pt2-table-gb", type=float, default=16.0,
                    help="hash-table memory of the pt2 section (16 GB: larger tables make the random inserts slower)")
    ap.add_argument("--no-spinor", action="store_true", help="skip the 64-spinor complex workload section")
    ap.add_argument("--only", default=None, choices=["blockvec", "rdm", "batch", "davidson", "pt2", "spinor",
                                                     "rowsplit", "pt2_spinor", "deterministic", "two_word"],
                    help="run one side section alone and print its JSON (profiling runs)")
    ap.add_argument("--prec", default="f64", choices=["f64", "ds", "f32"],
                    help="f64: FP64 FMA path; ds: paired-FP32 products/sums (FP64 tolerance); "
                         "f32: FP32 storage of C and the tables, FP64 accumulation (real mode)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch

    from paper_2501_18185_gb300 import build, sci

    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    build.build()

    if args.only in ("blockvec", "batch", "pt2", "spinor", "pt2_spinor"):
        out = (blockvec_bench(M=args.M or 2_000_000) if args.only == "blockvec" else
               batch_bench() if args.only == "batch" else
               spinor_bench(local) if args.only == "spinor" else
               pt2_spinor_bench(M=args.M or 200_000, table_gb=args.pt2_table_gb) if args.only == "pt2_spinor" else
               pt2_bench(sizes=(args.M,) if args.M else (60_000, 200_000, 1_000_000, 2_000_000),
                         table_gb=args.pt2_table_gb))
        print(json.dumps({args.only: out}), flush=True)
        return
    w = make_workload(args.workload, args.nvec, args.M)
    stream = torch.cuda.current_stream(dev)
    t = time.perf_counter()
    H = sci.Hamiltonian(local, stream)
    H.set_integrals(w.mode, w.ints.h, chol=w.ints.chol)
    H.set_determinants(w.keys, w.n_alpha, w.n_beta)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t
    info = H.info()
    pairs = info["pairs"]
    gp = golden_pairs(w)
    if gp is not None and gp != pairs:
        raise SystemExit(f"pair count {pairs} differs from the oracle's {gp}")
    split = None
    if world > 1:   # row split: this rank's range of rows, merged by one all-gather per step
        from paper_2501_18185_gb300.partition import RowSplitSigma, gather_rows

        t = time.perf_counter()
        split = RowSplitSigma.balanced(H, world, rank)
        torch.cuda.synchronize()
        split_setup_s = time.perf_counter() - t
        # one feedback round: time this rank's sigma, re-cut the ranges from all ranks' times
        Cw = torch.from_numpy(np.ascontiguousarray(w.c)).to(dev)
        Sw = torch.empty_like(Cw)
        H.sigma(Cw, out=Sw)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            H.sigma(Cw, out=Sw)
        e1.record(stream)
        e1.synchronize()
        split.rebalance(e0.elapsed_time(e1) / 3, split.weights)
        del Cw, Sw

    if args.only in ("rdm", "davidson", "rowsplit", "deterministic", "two_word"):
        out = (rdm_bench(H, w) if args.only == "rdm" else davidson_bench(H, w) if args.only == "davidson"
               else rowsplit_bench(H) if args.only == "rowsplit" else two_word_bench(H, w, local)
               if args.only == "two_word" else deterministic_bench(H, w))
        print(json.dumps({args.only: out}), flush=True)
        return
    C64 = torch.from_numpy(np.ascontiguousarray(w.c)).to(dev)
    if args.prec == "f32" and w.ints.complex_:
        raise SystemExit("--prec f32 is a real-mode precision")
    C = C64.float() if args.prec == "f32" else C64
    S = torch.empty_like(C64)
    flush = torch.empty(256 * 1024 * 1024 // 8, dtype=torch.float64, device=dev)  # 256 MB > L2
    nv = C.shape[1]
    prec = {"f64": sci.SCI_PREC_F64, "ds": sci.SCI_PREC_F64_DS, "f32": sci.SCI_PREC_F32_STORE_F64_ACC}[args.prec]
    other = sci.SCI_PREC_F64_DS if args.prec == "f64" else sci.SCI_PREC_F64
    def vec(p):
        return C if p == prec else C64

    def step(p):
        H.sigma(vec(p), out=S, prec=p)
        if split is not None:
            gather_rows(S, split.ranges)

    for _ in range(args.warmup):
        step(prec)
        step(other)
    H.sync_status()
    sci.sci_profile(H.ctx, True)

    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)

    def timed(prec, steps):
        ms_, kern_ = [], []
        for _ in range(steps):
            flush.zero_()                      # evict L2 between timed steps
            ev0.record(stream)
            step(prec)
            ev1.record(stream)
            ev1.synchronize()
            ms_.append(ev0.elapsed_time(ev1))
            kern_.append(sci.sci_kernel_times(H.ctx))
        return ms_, kern_

    step_ms, kern = timed(prec, args.steps)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    # the other precision mode on the same inputs (same protocol, fewer steps)
    o_ms, o_kern = timed(other, max(3, min(args.steps, 5)))
    variant = {"prec": "ds" if other == sci.SCI_PREC_F64_DS else "f64",
               "ms_per_step": statistics.mean(o_ms),
               "value": pairs / (statistics.mean(o_ms) / 1e3),
               "kernel_ms": {"init": statistics.mean(k[0] for k in o_kern),
                             "doubles": statistics.mean(k[1] for k in o_kern),
                             "singles": statistics.mean(k[2] for k in o_kern)}}
    sci.sci_profile(H.ctx, False)
    H.sync_status()

    total_ms = max_over_ranks(sum(step_ms), dist, dev)
    ms = total_ms / args.steps
    value = split_throughput(pairs, args.steps, total_ms)

    # end to end through the public API with host buffers (pinned), copies inside: one
    # process calls sci_sigma_host; with a row split each rank copies C in, computes its
    # rows, the slices are all-gathered and S is copied out
    Ch = torch.from_numpy(np.ascontiguousarray(w.c, dtype=np.float32 if args.prec == "f32" else None)).pin_memory()
    Sh = torch.empty(tuple(C64.shape), dtype=C64.dtype).pin_memory()

    def e2e_step():
        if split is None:
            sci.sci_sigma_host(H.ctx, Ch, Sh, nv, prec)
            return
        vec(prec).copy_(Ch, non_blocking=True)
        step(prec)
        Sh.copy_(S, non_blocking=True)
        torch.cuda.synchronize()

    e2e_step()
    e2e_t = []
    for _ in range(max(3, min(args.steps, 10))):
        flush.zero_()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t = time.perf_counter()
        e2e_step()
        e2e_t.append(time.perf_counter() - t)
    e2e = pairs / (max_over_ranks(statistics.mean(e2e_t) * 1e3, dist, dev) / 1e3)
    nbytes = Ch.numel() * Ch.element_size()
    nbytes_out = Sh.numel() * Sh.element_size()

    # roofline of the dominant kernel (double excitations): algorithmic bytes per launch
    # (with a row split, of this rank's launch: its rows' double pairs)
    if split is not None:
        info = H.info()
    sb = 16 if w.ints.complex_ else (4 if args.prec == "f32" else 8)
    dbl_ms = statistics.mean(k[1] for k in kern)
    sgl_ms = statistics.mean(k[2] for k in kern)
    init_ms = statistics.mean(k[0] for k in kern)
    alg_bytes = info["pairs_doubles"] * (nv * sb + sb)
    peak, peak_kind = hbm_peak()
    achieved = alg_bytes / (dbl_ms / 1e3) / 1e9
    figs = profile_figures(f"{w.name}/nvec{nv}") if args.prec == "f64" else {}
    traffic = figs.get("dram")
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic,
            "measure": "algorithmic-byte equivalent (what an HBM-streaming evaluation of the same pairs "
                       "would move: double pairs x (nvec+1) x scalar bytes) / measured HBM copy peak",
            "dram_GBps": traffic / (dbl_ms / 1e3) / 1e9 if traffic else None,
            "dram_frac": traffic / (dbl_ms / 1e3) / 1e9 / peak if traffic else None,
            "kernel": {"f64": "k_doubles", "ds": "k_doubles_ds", "f32": "k_doubles_f32"}[args.prec],
            "peak_source": peak_kind,
            "algorithmic_bytes_per_launch": alg_bytes,
            "kernel_ms": {"init": init_ms, "doubles": dbl_ms, "singles": sgl_ms}}
    # the resources that bind the doubles kernel: the FP64 pipe (one FMA per double pair
    # and vector, four in complex mode) against its measured rate, and L2 (ncu bytes)
    pp = pipe_peaks(local)
    if args.prec == "f64":
        fma = (4 if w.ints.complex_ else 1) * nv * info["pairs_doubles"] / (dbl_ms / 1e3)
        roof["fp64_pipe"] = {"useful_fma_per_s": fma, "peak_fma_per_s": pp["fp64_fma_per_s"],
                             "frac": fma / pp["fp64_fma_per_s"], "peak_source": pp["how"]}
    if figs.get("l2"):
        roof["l2"] = {"bytes_per_launch": figs["l2"], "GBps": figs["l2"] / (dbl_ms / 1e3) / 1e9,
                      "source": figs.get("l2_note")}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(w)
    dav = None
    rdm = batch = pt2 = rowsplit = determ = two_word = None
    if not args.no_davidson and world == 1 and not w.ints.complex_:
        dav = davidson_bench(H, w)
        dav["blockvec"] = blockvec_bench()
        rdm = rdm_bench(H, w)
        batch = batch_bench()
        pt2 = pt2_bench(sizes=(200_000, 2_000_000))
        pt2.append({"spinor": pt2_spinor_bench()})
        rowsplit = rowsplit_bench(H)
        determ = deterministic_bench(H, w)
        two_word = two_word_bench(H, w, local)
    spinor = None
    if not args.no_spinor and world == 1 and not w.ints.complex_:
        spinor = spinor_bench(local)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None,
            "dtype": "c128" if w.ints.complex_ else {"f64": "f64", "ds": "f64", "f32": "f32-store/f64-acc"}[args.prec],
            "data": "synthetic",
            "config": {"workload": w.name, "M": w.M, "nvec": nv, "pairs_per_step": pairs,
                       "l2": "flushed between timed steps (256 MB write)", "setup_s": round(setup_s, 3),
                       "parallelism": f"rowsplit{world}" if world > 1 else "single",
                       **({"rank0_rows": list(split.ranges[0]), "split_setup_s": round(split_setup_s, 3)}
                          if split is not None else {})},
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes_out},
            "gpu_launches": args.steps * (1 + {"f64": 2, "ds": 4, "f32": 3}[args.prec]
                                          * ((nv + 7) // 8 if not w.ints.complex_ else (nv + 3) // 4)),
            "roofline": roof, "cpu_baseline": cpu, "clocks": clocks, "prec": args.prec,
            "other_prec": variant, "pipe_peaks": pp, "davidson": dav, "rdm": rdm, "batch": batch, "pt2": pt2,
            "spinor": spinor, "rowsplit": rowsplit, "deterministic": determ, "two_word": two_word}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
