"""Benchmark: two-scale PCG solve to 1e-8 and the operator apply at n = 7 on GB300.

Workload (the configuration the headline metric is quoted on): 32^3 hexes of the unit
cube, +-20 % vertex perturbation (seed 1), random renumbering and orientation, order
n = 7 (11,390,625 DOFs), lambda = 1, manufactured u* = sin(pi x) sin(pi y) sin(pi z),
homogeneous Dirichlet boundary. A step is one full two-scale PCG solve (Algorithm 1
with P = P^c + P^f) from u_0 = 0 to ||r|| <= 1e-8 ||b||; value = DOFs solved per
second (all ranks), ms_per_step = the time-to-1e-8. The operator apply (Ax GDOF/s)
is measured alongside with stored and recomputed geometric factors.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

--impl reference times the CPU oracle on a bounded sample of the same workload.
Under torchrun (N > 1) every rank solves its own replica (the path does not shard).
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Ax GDOF/s & PCG time-to-1e-8 (s) at N=7, % HBM roofline; mixed vs FP64"
E_FULL, A_FULL, SEED_FULL, ORDER, LAM = 32, 0.2, 1, 7, 1.0
E_SAMPLE = 8          # CPU-oracle sample: same recipe at 8^3 hexes (185,193 DOFs)
RTOL = 1e-8
WORKLOAD = "unit cube 32^3 hexes, +-20% perturbation seed 1, random numbering/orientation, n=7, lambda=1, Dirichlet"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-config3", action="store_true",
                    help="skip the 48^3-hex precision block of the default line")
    ap.add_argument("--no-config4", action="store_true",
                    help="skip the 24-problem x 4-load batching block of the default line")
    ap.add_argument("--no-config5", action="store_true",
                    help="skip the learned-correction block (training and evaluation) of the default line")
    ap.add_argument("--no-kcycle", action="store_true", help="skip the K-cycle block of the default line")
    ap.add_argument("--no-heat", action="store_true", help="skip the heat-rod block (n = 7) of the default line")
    ap.add_argument("--precision-variant", action="store_true",
                    help="48^3 hexes, +-20%% (seed 2), n=7, lambda=0: FP64 vs mixed time-to-1e-8 and the "
                         "per-result error of the mixed solution")
    ap.add_argument("--batch-variant", action="store_true",
                    help="24 problems (8^3..24^3 hexes, n in 3..8, +-15%%, seed 3), 4 Gaussian loads each: "
                         "one at a time vs sem_solve_many, default vs autotuned tile shapes")
    ap.add_argument("--learned-variant", action="store_true",
                    help="learned correction: train on seeded 16^3-hex n=5 meshes (lambda ~ U[0,10]), then "
                         "plain against flexible PCG with the network on an unseen 32^3-hex n=7 mesh (seed 4)")
    ap.add_argument("--heat-variant", action="store_true",
                    help="heat equation: 70 backward-Euler steps on a 16x16x244-hex rod (moving source, "
                         "kappa 1e-2, dt 0.04), orders 2..7, FP64 and mixed")
    ap.add_argument("--heat-orders", default="2,3,4,5,6,7")
    ap.add_argument("--heat-geom", default="recompute", choices=["recompute", "stored"],
                    help="geometric factors of the heat variant (the paper recomputes them)")
    ap.add_argument("--kcycle-variant", action="store_true",
                    help="coarse solver: the paper's K-cycle (unsmoothed aggregation, flexible PCG) against "
                         "the default three V-cycles on the 32^3 n=7 workload, FP64 and mixed")
    ap.add_argument("--patch-variant", action="store_true",
                    help="P^f patches: face layers only against the full (n+3)^3 box, 32^3 n=7, FP64 and mixed")
    ap.add_argument("--train-meshes", type=int, default=200)
    ap.add_argument("--train-steps", type=int, default=3000)
    ap.add_argument("--solve-case", type=int, default=0, metavar="E",
                    help="only run one SEM_PREC_FP64 solve on an E^3, n=7 mesh inside the NVTX range \"solve\" "
                         "(the launch list of a solve for ncu), then exit")
    ap.add_argument("--solve-prec", default="fp64", choices=["fp64", "fp32"],
                    help="with --solve-case: SEM_PREC_FP64 (default) or the mixed path (fp32)")
    ap.add_argument("--kernel-case", type=int, default=0, metavar="E",
                    help="only run a few operator / preconditioner applies on an E^3, n=7 mesh "
                         "(a small case for ncu captures), then exit")
    ap.add_argument("--kernel-geom", default="stored", choices=["stored", "recompute"],
                    help="with --kernel-case: stored or recomputed geometric factors")
    return ap.parse_args()


# ---------------------------------------------------------------- CPU oracle leg
def _oracle_sample_worker(E, steps, q):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    import numpy as np
    from synth import lattice_hex_mesh, manufactured_s
    from oracle.problem import Problem
    mesh = lattice_hex_mesh(E, A_FULL, SEED_FULL)
    pr = Problem(mesh, ORDER, LAM)
    b = pr.load(manufactured_s(pr.coords, LAM))
    times, iters = [], []
    for _ in range(steps):
        t0 = time.perf_counter()
        u, it, hist = pr.solve(b, rtol=RTOL)
        times.append(time.perf_counter() - t0)
        iters.append(int(it))
    q.put({"G": int(pr.G), "times": times, "iters": iters})


def oracle_sample(E, steps):
    """Runs the oracle in a spawned, single-threaded process (no CUDA state inherited)."""
    import multiprocessing as mp
    env_keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    old = {k: os.environ.get(k) for k in env_keys}
    for k in env_keys:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        q = ctx.Queue()
        p = ctx.Process(target=_oracle_sample_worker, args=(E, steps, q))
        p.start()
        res = q.get()
        p.join()
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return res


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    W, K = args.warmup, args.steps
    res = oracle_sample(E_SAMPLE, W + K)
    t = res["times"][W:]
    G = res["G"]
    per_step = sum(t) / len(t)
    value = G / per_step / 1e9
    sample = ("oracle two-scale PCG to 1e-8 on the same recipe at %d^3 hexes (n=7, lambda=1, %d DOFs, "
              "%d iterations); one full solve per step" % (E_SAMPLE, G, res["iters"][-1]))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GDOF/s",
        "n_gpus": args.gpus, "steps": K, "warmup": W, "ms_per_step": per_step * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample": "%d^3 hexes" % E_SAMPLE},
        "cpu_baseline": {"value": value, "unit": "GDOF/s", "cores": 1, "kind": "oracle", "sample": sample,
                         "cpu": cpu_model()},
        "e2e": {"value": value, "unit": "GDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

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
        self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


class Ranks:
    """Replica bookkeeping under torchrun: one problem per rank, no data-path collective;
    only the timing barrier and the max over ranks use the process group."""

    def __init__(self, backend=None, device=None):
        import torch.distributed as dist
        self.dist = dist
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.device = device
        if self.world > 1 and not dist.is_initialized():
            kw = {"device_id": device} if (backend == "nccl" and device is not None) else {}
            dist.init_process_group(backend, **kw)

    def barrier(self):
        if self.world > 1:
            self.dist.barrier()

    def max(self, v):
        if self.world == 1:
            return float(v)
        import torch
        t = torch.tensor([float(v)], dtype=torch.float64, device=self.device if self.device is not None else "cpu")
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def total_rate(self, units_per_rank, seconds_max):
        """Whole-job throughput: units processed by all ranks / the slowest rank's time."""
        return self.world * units_per_rank / seconds_max

    def close(self):
        if self.world > 1 and self.dist.is_initialized():
            self.dist.destroy_process_group()


def schwarz_flops_paper(n, ne):
    """The paper's O_P count (Sec. 4.2) with an FMA as 2 flops: six unfolded (n+3)^4
    contractions plus 15 (n+3)^3."""
    P = n + 3
    return ne * (12.0 * P ** 4 + 15.0 * P ** 3)


def ax_flops_paper(n, ne):
    """O_R = N_E [12 (n+1)^4 + 18 (n+1)^3] (Sec. 3.1)."""
    p = n + 1
    return ne * (12.0 * p ** 4 + 18.0 * p ** 3)


def schwarz_flops(n, ne):
    """Flops the patch kernel's algorithm executes per launch (FMA = 2, add or multiply = 1):
    per 1D line of P = n+3 nodes, the even/odd folded forward contraction takes 2H + 2HP +
    (P odd) NE and the backward one H (2P + 2) + (P odd) 2 NE, H = P // 2, NE = P - H;
    3 P^2 lines each way, then P^3 scalings by the stored inverse diagonal (which carries the
    patch scale 8/(hx hy hz))."""
    P = n + 3
    H, odd = P // 2, P % 2
    NE = P - H
    fwd = 2 * H + 2 * H * P + odd * NE
    bwd = H * (2 * P + 2) + odd * 2 * NE
    return ne * (3.0 * P * P * (fwd + bwd) + 1.0 * P ** 3)


def ax_flops(n, ne):
    """Flops the operator kernel executes per launch (FMA = 2): per 1D line of p = n+1 nodes
    the folded D contraction takes 2H + H (4H + 2) + (p odd) 3H, H = p // 2, with 6 p^2
    lines (3 gradients, 3 divergences); per node 15 for G grad u, and 4 for the three
    divergence terms and lambda m u (stored lambda m, one FMA)."""
    p = n + 1
    H, odd = p // 2, p % 2
    line = 2 * H + H * (4 * H + 2) + odd * 3 * H
    return ne * (6.0 * p * p * line + 19.0 * p ** 3)


def dw_ops_schwarz(n, ne):
    """FP32-pipe operations (add, multiply or FMA, one each) the double-FP32 patch kernel
    executes per launch, counted from its loops: a pair sum or difference is a TwoSum (6)
    plus 2 adds, a pair product 1 multiply + 3 FMAs, a pair multiply-accumulate 12; per
    1D line of P = n+3 nodes the folded forward contraction takes 2H sums, (P odd) NE
    products and H (NE + H) multiply-accumulates, the backward one H (NE + H) + (P odd) NE
    multiply-accumulates and 2H sums; 3 P^2 lines each way, P^3 products by the diagonal
    and P^3 input splits (2 FP32 operations each; their integer operations are not counted)."""
    P = n + 3
    H, odd = P // 2, P % 2
    NE = P - H
    fwd = 8 * 2 * H + 4 * odd * NE + 12 * H * (NE + H)
    bwd = 12 * H * (NE + H) + 8 * 2 * H + 12 * odd * NE
    return ne * (3.0 * P * P * (fwd + bwd) + 4.0 * P ** 3 + 2.0 * P ** 3)


def dw_ops_ax(n, ne):
    """FP32-pipe operations of the double-FP32 operator kernel per launch (the counts of
    dw_ops_schwarz): per 1D line of p = n+1 nodes, H = p // 2, 2H pair sums for the even/odd
    folding, (p odd) H products by the middle column, 2 H^2 + (p odd) H
    multiply-accumulates and 2H output sums, 6 p^2 lines; per node 3 metric products (a
    product and two multiply-accumulates, 28 each), one pair sum of the divergence, the
    lambda m u term with the last sum (20), one input split (2) and one output join (6)."""
    p = n + 1
    H, odd = p // 2, p % 2
    line = 8 * 2 * H + 4 * odd * H + 12 * (2 * H * H + odd * H) + 8 * 2 * H
    return ne * (6.0 * p * p * line + (84.0 + 8.0 + 20.0 + 2.0 + 6.0) * p ** 3)


def dw_ops_ax_recompute(n, ne):
    """FP32-pipe operations of the double-FP32 operator kernel with the metric recomputed
    (counts as dw_ops_ax: pair product 4, multiply-accumulate 12, pair sum 8, TwoSum 6; sign
    flips and the reciprocal estimate not counted). Lines as dw_ops_ax. Per node: the metric
    products (84), three pair sums of the divergence terms and the lambda m u term (two
    products, 8), the input split (2) and the output join (6), and the metric's per-node part:
    J's first two columns from the line's sums (6 products, 6 multiply-accumulates, 6
    renormalisations), 9 renormalised cofactors (a product, a multiply-accumulate and a TwoSum),
    the determinant (28), one pair division (26), 6 entries of C^T C scaled (32 each) and m
    (4): 580. Per line (p^2 of them): 4 halvings (2), 4 corner products with a halving (6),
    72 multiply-accumulates and 15 renormalisations: 986."""
    p = n + 1
    H, odd = p // 2, p % 2
    line = 8 * 2 * H + 4 * odd * H + 12 * (2 * H * H + odd * H) + 8 * 2 * H
    node_metric = 6 * (4 + 12) + 6 * 6 + 9 * (4 + 12 + 6) + 28 + 26 + 6 * 32 + 4
    line_metric = 4 * 2 + 4 * 6 + 72 * 12 + 15 * 6
    return ne * (6.0 * p * p * line + (84.0 + 3 * 8.0 + 8.0 + 2.0 + 6.0 + node_metric) * p ** 3
                 + line_metric * p * p)


def _cpu_ax_worker(E, nthreads_list, reps, q):
    """The oracle's matrix-free operator at full size: one thread, then element chunks on
    a thread pool (numpy releases the GIL inside its loops), the gather as written."""
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    import numpy as np
    from concurrent.futures import ThreadPoolExecutor
    from synth import lattice_hex_mesh
    from oracle.problem import Problem
    from oracle.operator import matfree_local
    t0 = time.perf_counter()
    pr = Problem(lattice_hex_mesh(E, A_FULL, SEED_FULL), ORDER, LAM, coarse_solver=None, with_schwarz=False)
    t_setup = time.perf_counter() - t0
    x = np.random.default_rng(0).standard_normal(pr.G)
    out = {"G": int(pr.G), "setup_s": t_setup, "threads": {}}
    for nt in nthreads_list:
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            if nt == 1:
                pr.apply_A(x)
            else:
                xf = np.where(pr.mask > 0, 0.0, x)
                ne = pr.l2g.shape[0]
                chunks = np.array_split(np.arange(ne), 4 * nt)

                def work(ix):
                    a, b = ix[0], ix[-1] + 1
                    return matfree_local(xf[pr.l2g[a:b]], pr.Dh, pr.Gf[:, a:b], pr.m_loc[a:b], pr.lam)

                with ThreadPoolExecutor(nt) as ex:
                    r = np.concatenate(list(ex.map(work, chunks)))
                y = np.bincount(pr.l2g.ravel(), weights=r.ravel(), minlength=pr.G)
                y = np.where(pr.mask > 0, x, y)
            ts.append(time.perf_counter() - t0)
        out["threads"][nt] = min(ts)
    q.put(out)


def oracle_ax_full(E, nthreads_list, reps=2):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_cpu_ax_worker, args=(E, nthreads_list, reps, q))
    p.start()
    res = q.get()
    p.join()
    return res


def l2_flush(buf):
    """Flush L2 between timed steps: write a buffer larger than L2, then read it back, so that
    no dirty line of the flush is left for the timed kernels to write back to HBM."""
    buf.zero_()
    buf.sum()


def config4_block(steps, warmup, flush=None):
    """Batching variant: 24 seeded problems (E ~ U{8..24} hexes per direction, n ~ U{3..8},
    +-15 %, lambda = 0, Dirichlet, seed 3) with 4 Gaussian loads each, FP64 two-scale PCG to
    1e-8. One handle per problem: its 4 loads solved one at a time (4 graph launches) against
    one block solve (sem_solve_block, every kernel over the 4 loads; one graph launch)."""
    import numpy as np
    import torch
    from synth import lattice_hex_mesh, gaussian_load
    from paper_1506_05996_gb300 import sem as S
    rng = np.random.default_rng(3)
    specs = [(int(rng.integers(8, 25)), int(rng.integers(3, 9))) for _ in range(24)]
    t0 = time.perf_counter()
    probs = []
    for k, (E, n) in enumerate(specs):
        mesh = lattice_hex_mesh(E, 0.15, 3000 + k)
        pr = S.SemProblem(mesh.xyz, mesh.hex2vert, n, 0.0)
        free = (pr.mask() == 0).double()
        B = torch.stack([torch.as_tensor(gaussian_load(pr.n_dof, 30000 + 4 * k + r), device="cuda") * free
                         for r in range(4)]).contiguous()
        S.sem_autotune(pr.h)
        probs.append((pr, B, torch.empty_like(B)))
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    total = float(sum(4 * pr.n_dof for pr, _, _ in probs))

    def one_at_a_time():
        its = []
        for pr, B, X in probs:
            for r in range(4):
                rc, it, hist, tr = S.sem_solve(pr.h, B[r], X[r], RTOL, 1000, want_history=False)
                its.append(it)
        return its

    def block():
        its = []
        for pr, B, X in probs:
            rc, it, sts, trs = S.sem_solve_block(pr.h, B, X, RTOL, 1000)
            assert rc == 0, sts
            its += it
        return its

    def many_block():
        rc, it, sts = S.sem_solve_many_block([pr.h for pr, _, _ in probs], [B for _, B, _ in probs],
                                             [X for _, _, X in probs], RTOL, 1000)
        assert rc == 0, sts
        return [i for row in it for i in row]

    def timed(fn):
        for _ in range(max(1, warmup)):
            fn()
        best = None
        for _ in range(max(1, steps)):
            if flush is not None:
                l2_flush(flush)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            its = fn()
            e1.record()
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / 1e3
            best = t if best is None or t < best else best
        return best, its

    t_seq, its_seq = timed(one_at_a_time)
    t_blk, its_blk = timed(block)
    t_many, its_many = timed(many_block)
    same = its_seq == its_blk == its_many
    for pr, _, _ in probs:
        pr.close()
    return {"workload": "24 problems: E ~ U{8..24} hexes per direction, n ~ U{3..8}, +-15% perturbation, lambda=0, "
                        "Dirichlet, 4 Gaussian N(0,1) loads each (seed 3); SEM_PREC_FP64 two-scale PCG to 1e-8",
            "problems": [{"E": E, "n": n} for E, n in specs], "solves": 96, "total_dofs_solved": int(total),
            "setup_s": t_setup,
            "one_at_a_time": {"s": t_seq, "solves_per_s": 96 / t_seq, "gdofs_solved": total / t_seq / 1e9},
            "block_k4": {"s": t_blk, "solves_per_s": 96 / t_blk, "gdofs_solved": total / t_blk / 1e9,
                         "speedup": t_seq / t_blk},
            "many_block_k4": {"s": t_many, "solves_per_s": 96 / t_many, "gdofs_solved": total / t_many / 1e9,
                              "speedup": t_seq / t_many,
                              "how": "sem_solve_many_block: the 24 handles' 4-column block solves as the "
                                     "branches of one graph, one launch"},
            "iterations_equal": same,
            "iterations": {"min": int(min(its_blk)), "max": int(max(its_blk)), "mean": float(np.mean(its_blk))},
            "note": "block solves, batched or not, are bit-identical to the single solves (tests/test_gpu_block.py); "
                    "the time of the faster of the timed passes, each pass all 96 solves"}


def run_gpu(args):
    import numpy as np
    import torch
    from synth import lattice_hex_mesh, manufactured_s, manufactured_u
    from paper_1506_05996_gb300 import sem as S

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    ranks = Ranks("nccl", torch.device("cuda", local))
    world, rank = ranks.world, ranks.rank
    barrier, max_over_ranks = ranks.barrier, ranks.max
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # 512 MB > L2

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    hbm_source = "MEASURED_PEAKS.json hbm_gbs (copy)" if "hbm_gbs" in peaks else "fallback 6800 GB/s"

    # ---- arithmetic peaks: the library's FMA loop, with the clock sampled meanwhile
    clk_peak = ClockSampler(local)
    clk_peak.start()
    fp64_tf, _ = S.sem_measure_fma_peak("fp64", 8000)
    fp32_tf, _ = S.sem_measure_fma_peak("fp32", 400000)
    ck = clk_peak.stop()
    meas = {"fp64_tflops": fp64_tf, "fp32_tflops": fp32_tf, "fp32_tops": fp32_tf / 2,
            "sm_mhz_during": ck.get("sm_mhz"), "hbm_gbs": hbm_peak, "hbm_source": hbm_source,
            "how": "sem_measure_fma_peak: 8 chains of dependent FMAs per thread, 2048 threads per SM, "
                   "best of 3 CUDA-event-timed launches; FMA = 2 flops; fp32_tops counts one FP32-pipe "
                   "operation per FMA"}

    def solve_problem(E, a, seed, lam):
        mesh = lattice_hex_mesh(E, a, seed)
        pr = S.SemProblem(mesh.xyz, mesh.hex2vert, ORDER, lam, geom="stored", mixed=True)
        X = pr.dof_coords()
        b = pr.load(torch.as_tensor(manufactured_s(X.cpu().numpy(), lam), device="cuda"))   # b = m_N s
        return mesh, pr, X, b

    mesh, prob, X, b = solve_problem(E_FULL, A_FULL, SEED_FULL, LAM)
    G, NE = prob.n_dof, mesh.n_hex
    x = torch.empty_like(b)
    # tile shapes (elements per CTA) by the library's autotuner, per precision, before any
    # timing; the handle ends in SEM_PREC_FP64
    tiles = {}
    for prec in ("p32", "fp32", "fp64_native", "fp64"):
        prob.set_precision(prec)
        tiles[prec] = list(S.sem_autotune(prob.h))

    def one_solve():
        rc, it, hist, tr = S.sem_solve(prob.h, b, x, RTOL, 1000, want_history=False)
        return rc, it, tr

    def timed_solves(steps, warmup, pre=None, clocks=None):
        for _ in range(warmup):
            one_solve()
        evs, its, trs = [], [], []
        torch.cuda.synchronize()
        if clocks is not None:
            clocks.start()
        barrier()
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        for k in range(steps):
            l2_flush(flush)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rc, it, tr = one_solve()
            e1.record(stream)
            evs.append((e0, e1))
            its.append(it)
            trs.append(tr)
            if rc != 0:
                raise RuntimeError("solve did not converge: rc=%d" % rc)
        torch.cuda.synchronize()
        barrier()
        wall = time.perf_counter() - w0
        t = max_over_ranks(sum(a.elapsed_time(c) for a, c in evs) / 1e3) / steps
        return t, its[-1], trs[-1], wall

    # ---- headline: SEM_PREC_FP64 solves as users run them (one graph launch per solve)
    prob.set_precision("fp64")
    clocks = ClockSampler(local)
    per_step, it64, tr64, t_wall = timed_solves(args.steps, args.warmup, clocks=clocks)
    clk = clocks.stop()
    # a measurement under hardware or thermal slowdown is not kept: it is taken once more (the
    # decision is the max over ranks, so that every rank times the same steps)
    slowed = bool(set(clk.get("reasons") or []) & {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"})
    if max_over_ranks(1.0 if slowed else 0.0) > 0.0:
        first = clk.get("reasons")
        clocks = ClockSampler(local)
        per_step, it64, tr64, t_wall = timed_solves(args.steps, 1, clocks=clocks)
        clk = clocks.stop()
        clk["remeasured_after"] = first
    value = ranks.total_rate(G, per_step) / 1e9

    # ---- the same solves with per-kernel CUDA events (host-driven loop, one event pair per
    # launch), for the kernel breakdown and the dominant kernel's roofline
    S.sem_profile(prob.h, 1)
    t_prof, _, _, _ = timed_solves(args.steps, 0)
    prof = S.sem_profile_read(prob.h)
    S.sem_profile(prob.h, 0)
    launches_per_step = sum(v[0] for v in prof.values()) / args.steps
    kern, (nl, tot) = max(prof.items(), key=lambda kv: kv[1][1])
    avg_ms = tot / nl
    ops = {"schwarz_local": dw_ops_schwarz, "ax_local": dw_ops_ax}.get(kern)
    fp64eq = {"schwarz_local": schwarz_flops, "ax_local": ax_flops}.get(kern)
    # DRAM bytes per launch: one ncu capture of the kernel at 24^3 hexes (13,824 elements, 2
    # per CTA as here; 211,711,488 bytes read + 79,164,416 written), scaled by the element
    # count: the kernel's bytes are per element (pair diagonals, patch table, r, results)
    traffic = {"schwarz_local": (211711488 + 79164416) / 13824 * NE}.get(kern)
    roof = {"kernel": kern + " (double-FP32)", "bound": "alu", "unit": "Tops/s",
            "peak": meas["fp32_tops"],
            "peak_source": "measured FP32 FMA loop (sem_measure_fma_peak), one operation per FMA, at %s MHz"
                           % ck.get("sm_mhz"),
            "achieved": (ops(ORDER, NE) / (avg_ms * 1e-3) / 1e12) if ops else None,
            "ops_per_launch": ops(ORDER, NE) if ops else None,
            "ops_note": "FP32-pipe operations of the pair arithmetic, counted from the kernel's loops "
                        "(TwoSum 6, pair sum 8, pair product 4, multiply-accumulate 12); integer "
                        "operations of the binary64 splits are not counted",
            "fp64_equivalent_tflops": (fp64eq(ORDER, NE) / (avg_ms * 1e-3) / 1e12) if fp64eq else None,
            "fp64_pipe_peak_tflops": fp64_tf,
            "avg_launch_ms": avg_ms, "launches": nl, "traffic": traffic,
            "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch at 24^3 hexes, "
                              "scaled to this mesh by the element count" if traffic else None,
            "share_of_step": tot / (t_prof * args.steps * 1e3)}
    roof["frac"] = (roof["achieved"] / roof["peak"]) if roof["achieved"] else None

    def variant(prec, weighted=False):
        prob.set_precision(prec)
        S.sem_set_weights(prob.h, 1 if weighted else 0)
        t, it, tr, _ = timed_solves(args.steps, args.warmup)
        prob.set_precision("fp64")
        S.sem_set_weights(prob.h, 0)
        return {"time_to_1e-8_s": t, "gdofs_solved": world * G / t / 1e9, "iterations": it,
                "true_rel_res": tr, "speedup_vs_fp64": per_step / t}

    native = variant("fp64_native")
    native["dtype"] = "binary64 everywhere (FP64 pipe)"
    native["fp64_speedup_over_native"] = native["time_to_1e-8_s"] / per_step
    mixed = variant("fp32")
    mixed["dtype"] = ("FP32 operator and patch solves; FP64 vectors, dots, recurrences, coarse solve, "
                      "residual replacement (double-FP32 operator) and final check")
    prob.set_precision("fp32")
    S.sem_set_patch_solver(prob.h, "bf16_tc")
    mixed_tc = variant("fp32")
    S.sem_set_patch_solver(prob.h, "fp32")
    mixed_tc["dtype"] = ("as mixed, with the patch solves in BF16 on the tensor cores (tcgen05, FP32 accumulation) "
                         "and the flexible beta")
    p32 = variant("p32")
    p32["dtype"] = "double-FP32 operator; FP32 patch solves and prolongation sums; FP64 vectors and recurrences"
    weighted = {"fp64": variant("fp64", True), "mixed": variant("fp32", True),
                "note": "not the paper's P^f: W (sum of patch solves) W, w = c^-1/2 per DOF (c patches contain it)"}
    prob.set_precision("fp64")

    # ---- operator apply (Ax GDOF/s) and its HBM roofline
    def time_apply(pr, prec, reps=20):
        f32io = prec == "fp32io"
        pr.set_precision("fp32" if f32io else prec)
        xin = torch.randn(G, dtype=torch.float32 if f32io else torch.float64, device="cuda")
        y = torch.empty_like(xin)
        apply = S.sem_apply_A_f32 if f32io else S.sem_apply_A
        for _ in range(3):
            apply(pr.h, xin, y)
        S.sem_profile(pr.h, 1)
        evs = []
        for _ in range(reps):
            l2_flush(flush)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            apply(pr.h, xin, y)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        pk = S.sem_profile_read(pr.h)
        S.sem_profile(pr.h, 0)
        pr.set_precision("fp64")
        return sorted(a.elapsed_time(c) for a, c in evs)[reps // 2], pk["ax_local"][1] / pk["ax_local"][0]

    ax = {}
    p3 = (ORDER + 1) ** 3
    L = NE * p3
    rec = S.SemProblem(mesh.xyz, mesh.hex2vert, ORDER, LAM, geom="recompute")
    for prec in ("fp32", "fp64_native", "fp64"):
        rec.set_precision(prec)
        S.sem_autotune(rec.h)
    for geom, prec, pr in (("stored", "fp64", prob), ("stored", "fp64_native", prob), ("recompute", "fp64", rec),
                           ("recompute", "fp64_native", rec), ("stored", "fp32", prob), ("recompute", "fp32", rec), ("stored", "bf16", prob),
                           ("stored", "fp32io", prob)):
        ms, kms = time_apply(pr, prec)
        # algorithmic bytes of one apply: x read and y written (G each), the local-to-global
        # index (int32 per local node), stored factors (7 per local node: 8 bytes as binary64
        # or as an FP32 pair, 4 as FP32, 2 as BF16) or the 24 vertex coordinates per element
        fb = {"fp64": 8, "fp64_native": 8, "fp32": 4, "bf16": 2, "fp32io": 4}[prec]
        vb = 4 if prec == "fp32io" else 8
        wb = 8 if prec in ("fp64", "fp64_native") else 4
        geo_bytes = 7 * fb * L if geom == "stored" else 24 * 8 * NE
        alg_bytes = 2 * vb * G + 4 * L + geo_bytes
        # the element kernel alone: x and the mask read once per DOF; l2g and the factors per
        # local node; interior DOFs of y written directly in y's type (Gi of them), the other
        # local results in the local-result type
        Gi = NE * (ORDER - 1) ** 3
        k_bytes = (vb + 1) * G + 4 * L + geo_bytes + vb * Gi + wb * (L - Gi)
        key = geom + ("" if prec == "fp64" else "_" + prec)
        ax[key] = {"gdofs": G / (ms * 1e-3) / 1e9, "ms": ms, "ax_local_ms": kms,
                   "bytes_per_dof": alg_bytes / G, "hbm_gbs": alg_bytes / (ms * 1e-3) / 1e9,
                   "frac_hbm_roofline": alg_bytes / (ms * 1e-3) / 1e9 / hbm_peak,
                   "ax_local_frac_hbm_roofline": k_bytes / (kms * 1e-3) / 1e9 / hbm_peak,
                   "paper_equivalent_tflops_ax_local": ax_flops_paper(ORDER, NE) / (kms * 1e-3) / 1e12}
        if prec == "fp64_native":
            ax[key]["frac_fp64_pipe_peak"] = ax_flops(ORDER, NE) / (kms * 1e-3) / 1e12 / fp64_tf
        if prec == "fp64":
            ax_ops = dw_ops_ax(ORDER, NE) if geom == "stored" else dw_ops_ax_recompute(ORDER, NE)
            ax[key]["frac_fp32_ops_peak"] = ax_ops / (kms * 1e-3) / 1e12 / meas["fp32_tops"]
    ax["note"] = ("bytes count x, mask and y once per DOF; fp64 = double-FP32 kernel (stored: pair factors; "
                  "recompute: the factors recomputed per node in pairs), fp64_native = binary64")
    rec.close()

    # ---- end to end through the public API with host buffers
    b_host = b.cpu().pin_memory()
    x_host = torch.empty(G, dtype=torch.float64).pin_memory()
    n_e2e = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        b_dev = b_host.to("cuda", non_blocking=True)
        S.sem_solve(prob.h, b_dev, x, RTOL, 1000, want_history=False)
        x_host.copy_(x, non_blocking=True)
        torch.cuda.synchronize()
    t_e2e = max_over_ranks((time.perf_counter() - t0) / n_e2e)
    prob.close()

    # ---- precision variant (48^3 hexes, lambda = 0, seed 2): SEM_PREC_FP64 against the mixed
    # path and binary64, errors per result against the binary64 solution
    # the variant blocks describe one GPU: replicas (N > 1) skip them
    config3 = None
    if not args.no_config3 and world == 1:
        mesh3, pr3, X3, b3 = solve_problem(48, 0.2, 2, 0.0)
        G3 = pr3.n_dof
        ustar = torch.as_tensor(manufactured_u(X3.cpu().numpy()), device="cuda")
        free = ~pr3.mask().bool()
        sols, c3 = {}, {}
        for prec in ("fp64_native", "fp64", "fp32"):
            pr3.set_precision(prec)
            S.sem_autotune(pr3.h)
            x3 = torch.empty_like(b3)
            S.sem_solve(pr3.h, b3, x3, RTOL, 1000, want_history=False)
            ts = []
            for _ in range(2):
                l2_flush(flush)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                rc, it, hist, tr = S.sem_solve(pr3.h, b3, x3, RTOL, 1000, want_history=False)
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1) / 1e3)
            sols[prec] = x3
            c3[prec] = {"time_to_1e-8_s": min(ts), "iterations": it, "true_rel_res": tr,
                        "max_err_vs_manufactured": float((x3 - ustar)[free].abs().max())}
        ref = sols["fp64_native"]
        for prec in ("fp64", "fp32"):
            dlt = sols[prec] - ref
            c3[prec]["vs_binary64_solution"] = {"max_rel": float(dlt.abs().max() / ref.abs().max()),
                                                "rel_l2": float(dlt.norm() / ref.norm())}
        c3["mixed_speedup_vs_fp64"] = c3["fp64"]["time_to_1e-8_s"] / c3["fp32"]["time_to_1e-8_s"]
        c3["mixed_speedup_vs_binary64"] = c3["fp64_native"]["time_to_1e-8_s"] / c3["fp32"]["time_to_1e-8_s"]
        c3["fp64_vs_config2_fp64_time_ratio"] = c3["fp64"]["time_to_1e-8_s"] / per_step
        config3 = {"workload": "unit cube 48^3 hexes, +-20% perturbation seed 2, random numbering/orientation, "
                               "n=7, lambda=0, Dirichlet", "n_dof": G3,
                   "note": "errors against the binary64 GPU solution (it matches the oracle to 1e-12 in the "
                           "parity tests); time of the faster of 2 solves after one warm-up", **c3}
        pr3.close()

    config4 = None
    if not args.no_config4 and world == 1:
        config4 = config4_block(max(1, min(args.steps, 3)), 1, flush)
    config5 = None
    if not args.no_config5 and world == 1:
        config5 = learned_block(args, max(1, min(args.steps, 3)))
    kcycle = None
    if not args.no_kcycle and world == 1:
        kcycle = kcycle_block(args)
    heat = None
    if not args.no_heat and world == 1:
        heat = heat_block(args, [7])

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        res = oracle_sample(E_SAMPLE, 3)
        tc = sum(res["times"]) / len(res["times"])
        ncores = os.cpu_count() or 1
        full = oracle_ax_full(E_FULL, [1, ncores])
        t1, tn = full["threads"][1], full["threads"][ncores]
        cpu = {"value": res["G"] / tc / 1e9, "unit": "GDOF/s", "cores": 1, "kind": "oracle",
               "sample": ("oracle two-scale PCG to 1e-8, same recipe at %d^3 hexes (%d DOFs, %d iterations), "
                          "mean of 3 solves, single thread" % (E_SAMPLE, res["G"], res["iters"][-1])),
               "cpu": cpu_model(), "host_cores_available": ncores,
               "ax_full_size": {"workload": "oracle matrix-free A x at the full 32^3, n=7 size (%d DOFs)" % full["G"],
                                "gdofs_1_thread": full["G"] / t1 / 1e9, "s_1_thread": t1,
                                "gdofs_all_cores": full["G"] / tn / 1e9, "s_all_cores": tn, "cores": ncores,
                                "how": "element chunks of the oracle's local apply on a thread pool (numpy "
                                       "releases the GIL), gather as written; best of 2",
                                "gpu_speedup_fp64_stored": ax["stored"]["gdofs"] / (full["G"] / tn / 1e9)}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GDOF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": per_step * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "arith": ("SEM_PREC_FP64: binary64 vectors, dot products, alpha/beta, residual updates and the "
                      "final true-residual check; operator and patch-solve element kernels and the P-sum in "
                      "double-FP32 (pairs of FP32 with error-free transforms, 2^-46 per step); "
                      "fp64_native: binary64 everywhere"),
            "config": {"workload": WORKLOAD, "n_dof": G, "n_hex": NE, "order": ORDER, "lambda": LAM,
                       "rtol": RTOL, "preconditioner": "two-scale (P^c + P^f)", "geometry": "stored",
                       "loop": "one graph launch per solve (device-evaluated while loop)",
                       "l2": "inputs larger than L2 (0.94 GB stored factors) and a 512 MB flush between steps (written, then read back)",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "tiles_epb_ax_sw": tiles},
            "time_to_1e-8_s": per_step, "iterations": it64, "true_rel_res": tr64, "wall_s": t_wall,
            "fp64_native": native, "mixed": mixed, "bf16_precond": mixed_tc, "p32": p32, "weighted": weighted,
            "profiled": {"ms_per_step": t_prof * 1e3,
                         "note": "host-driven loop with a CUDA event pair around every launch",
                         "kernels_ms_per_step": {k: v[1] / args.steps
                                                 for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}},
            "ax": ax, "peaks": meas, "roofline": roof, "config3": config3, "config4": config4, "config5": config5,
            "kcycle": kcycle, "heat": heat,
            "e2e": {"value": world * G / t_e2e / 1e9, "unit": "GDOF/s", "h2d_bytes_per_step": 8 * G,
                    "d2h_bytes_per_step": 8 * G, "s_per_step": t_e2e},
            "gpu_launches": int(round(launches_per_step * args.steps)),
            "gpu_launches_note": "kernels executed per solve (counted in the profiled pass) x steps",
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    ranks.close()


def run_solve_case(E, prec="fp64"):
    """One SEM_PREC_FP64 solve of the headline recipe at E^3 hexes, n = 7, after a warm-up
    solve, inside the NVTX range "solve" (for ncu --nvtx --nvtx-include solve/)."""
    import torch
    from synth import lattice_hex_mesh, manufactured_s
    from paper_1506_05996_gb300 import sem as S
    mesh = lattice_hex_mesh(E, A_FULL, SEED_FULL)
    prob = S.SemProblem(mesh.xyz, mesh.hex2vert, ORDER, LAM, geom="stored", mixed=(prec == "fp32"))
    X = prob.dof_coords()
    b = prob.load(torch.as_tensor(manufactured_s(X.cpu().numpy(), LAM), device="cuda"))
    prob.set_precision(prec)
    S.sem_autotune(prob.h)
    # the eager host loop launches each kernel of an iteration by itself, so ncu lists every
    # launch (the graphs of the other loops are profiled only as wholes)
    S.sem_set_loop(prob.h, S.SEM_LOOP_EAGER)
    x, rc, it, hist, tr = prob.solve(b)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("solve")
    x, rc, it, hist, tr = prob.solve(b)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"solve_case": E, "precision": prec, "n_dof": prob.n_dof, "iterations": it, "true_rel_res": tr}))
    prob.close()


def run_kernel_case(E, geom="stored"):
    """A few applies of each hot kernel (SEM_PREC_FP64's double-FP32 kernels, binary64, FP32)
    on an E^3-hex, n = 7 mesh with stored or recomputed geometric factors, with the
    tile shapes the autotuner picks; the applies sit in the NVTX range "kernels" (for
    ncu --nvtx --nvtx-include kernels/), the tuning launches outside it."""
    import torch
    from synth import lattice_hex_mesh
    from paper_1506_05996_gb300 import sem as S
    mesh = lattice_hex_mesh(E, A_FULL, SEED_FULL)
    prob = S.SemProblem(mesh.xyz, mesh.hex2vert, ORDER, LAM, geom=geom, mixed=True)
    x = torch.randn(prob.n_dof, dtype=torch.float64, device="cuda")
    tiles = {}
    for prec in ("fp32", "fp64_native", "fp64"):
        prob.set_precision(prec)
        tiles[prec] = S.sem_autotune(prob.h)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("kernels")
    for prec in ("fp64", "fp64_native", "fp32"):
        prob.set_precision(prec)
        for _ in range(2):
            prob.apply_A(x)
            prob.apply_P(x, "two-scale")
    S.sem_set_patch_solver(prob.h, "bf16_tc")       # the tensor-core patch solve (FP32 path)
    for _ in range(2):
        prob.apply_P(x, "two-scale")
    S.sem_set_patch_solver(prob.h, "fp32")
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"kernel_case": E, "geom": geom, "n_dof": prob.n_dof, "tiles": tiles}))
    prob.close()


def run_precision_variant(args):
    """Precision variant: 48^3 hexes (38,272,753 DOFs), FP64 against the mixed path."""
    import numpy as np
    import torch
    from synth import lattice_hex_mesh, manufactured_s, manufactured_u
    from paper_1506_05996_gb300 import sem as S
    mesh = lattice_hex_mesh(48, 0.2, 2)
    lam = 0.0
    t0 = time.perf_counter()
    prob = S.SemProblem(mesh.xyz, mesh.hex2vert, ORDER, lam, geom="stored", mixed=True)
    t_setup = time.perf_counter() - t0
    G = prob.n_dof
    X = prob.dof_coords()
    b = (prob.mass() * torch.as_tensor(manufactured_s(X.cpu().numpy(), lam), device="cuda")).contiguous()
    ustar = torch.as_tensor(manufactured_u(X.cpu().numpy()), device="cuda")
    mask = prob.mask().bool()
    out = {}
    sols = {}
    stream = torch.cuda.current_stream()
    for prec in ("fp64", "fp32"):
        prob.set_precision(prec)
        x = torch.empty_like(b)
        for _ in range(max(1, args.warmup)):
            S.sem_solve(prob.h, b, x, RTOL, 1000, want_history=False)
        times, its, trs = [], [], []
        for _ in range(max(1, args.steps)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rc, it, hist, tr = S.sem_solve(prob.h, b, x, RTOL, 1000, want_history=False)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
            its.append(it)
            trs.append(tr)
        sols[prec] = x.clone()
        err_star = float((x - ustar)[~mask].abs().max())
        out[prec] = {"time_to_1e-8_s": sum(times) / len(times), "iterations": its[-1], "true_rel_res": trs[-1],
                     "max_err_vs_manufactured": err_star}
    d = (sols["fp32"] - sols["fp64"])
    out["mixed_vs_fp64"] = {
        "max_abs_diff": float(d.abs().max()),
        "max_rel_diff": float(d.abs().max() / sols["fp64"].abs().max()),
        "rel_l2_diff": float(d.norm() / sols["fp64"].norm()),
        "speedup": out["fp64"]["time_to_1e-8_s"] / out["fp32"]["time_to_1e-8_s"]}
    print(json.dumps({"variant": "precision", "config": {
        "workload": "unit cube 48^3 hexes, +-20% perturbation seed 2, random numbering/orientation, n=7, "
                    "lambda=0, Dirichlet", "n_dof": G, "setup_s": t_setup},
        "note": "the FP64 GPU solution stands in for the oracle at this size (the FP64 path matches the "
                "oracle to 1e-12 in the parity tests, including every DOF of A x at 32^3)", **out}))
    prob.close()


def run_batch_variant(args):
    """Batched variant: 24 seeded problems x 4 loads, solved one at a time and together."""
    import numpy as np
    import torch
    from synth import lattice_hex_mesh, gaussian_load
    from paper_1506_05996_gb300 import sem as S
    rng = np.random.default_rng(3)
    specs = [(int(rng.integers(8, 25)), int(rng.integers(3, 9))) for _ in range(24)]
    t0 = time.perf_counter()
    handles, bs, xs, dofs, keep = [], [], [], [], []
    for k, (E, n) in enumerate(specs):
        mesh = lattice_hex_mesh(E, 0.15, 3000 + k)
        for r in range(4):
            st = torch.cuda.Stream()
            pr = S.SemProblem(mesh.xyz, mesh.hex2vert, n, 0.0, stream=st)
            free = (pr.mask() == 0).double()
            b = (torch.as_tensor(gaussian_load(pr.n_dof, 30000 + 4 * k + r), device="cuda") * free).contiguous()
            handles.append(pr.h)
            bs.append(b)
            xs.append(torch.empty_like(b))
            dofs.append(pr.n_dof)
            keep.append((pr, st))
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0

    def one_at_a_time():
        torch.cuda.synchronize()
        t = time.perf_counter()
        its = []
        for h, b, x in zip(handles, bs, xs):
            rc, it, hist, tr = S.sem_solve(h, b, x, RTOL, 1000, want_history=False)
            its.append(it)
        torch.cuda.synchronize()
        return time.perf_counter() - t, its

    def batched():
        torch.cuda.synchronize()
        t = time.perf_counter()
        rc, its, sts = S.sem_solve_many(handles, bs, xs, RTOL, 1000)
        torch.cuda.synchronize()
        assert rc == 0, (rc, sts)
        return time.perf_counter() - t, its

    for _ in range(max(1, args.warmup)):
        one_at_a_time()
        batched()
    reps = max(1, args.steps)
    t_seq = min(one_at_a_time()[0] for _ in range(reps))
    t_bat, its = min((batched() for _ in range(reps)), key=lambda v: v[0])
    tiles = [S.sem_autotune(h) for h in handles]
    for _ in range(max(1, args.warmup)):
        batched()
    t_tuned, its_t = min((batched() for _ in range(reps)), key=lambda v: v[0])
    total = float(sum(dofs))
    by_order = {}
    for (E, n), tl in zip([s for s in specs for _ in range(4)], tiles):
        by_order.setdefault(n, set()).add(tl)
    print(json.dumps({"variant": "batch", "config": {
        "workload": "24 problems: E ~ U{8..24} hexes per direction, n ~ U{3..8}, +-15% perturbation, lambda=0, "
                    "Dirichlet, 4 Gaussian N(0,1) loads each (seed 3); FP64 two-scale PCG to 1e-8",
        "problems": [{"E": E, "n": n} for E, n in specs], "solves": len(handles), "total_dofs": int(total),
        "setup_s": t_setup},
        "one_at_a_time": {"s": t_seq, "gdofs_solved": total / t_seq / 1e9, "solves_per_s": len(handles) / t_seq},
        "batched": {"s": t_bat, "gdofs_solved": total / t_bat / 1e9, "solves_per_s": len(handles) / t_bat,
                    "speedup": t_seq / t_bat},
        "batched_autotuned": {"s": t_tuned, "gdofs_solved": total / t_tuned / 1e9,
                              "solves_per_s": len(handles) / t_tuned, "speedup": t_seq / t_tuned,
                              "tiles_by_order": {str(k): sorted(list(v)) for k, v in sorted(by_order.items())}},
        "iterations": {"min": int(min(its)), "max": int(max(its)), "mean": float(np.mean(its))}}))
    for pr, st in keep:
        pr.close()


def run_learned_variant(args):
    """Learned correction: GPU training on solver-harvested samples, then plain two-scale PCG
    against flexible PCG with the network (fallback on stall), FP64 and mixed."""
    print(json.dumps(learned_block(args, max(1, args.steps))))


def learned_block(args, steps):
    """The learned-correction block (config 5): returns the result as a dict."""
    import numpy as np
    import torch
    from paper_1506_05996_gb300 import sem as S
    from paper_1506_05996_gb300.learn import harvest, make_problem, timed_solve, train, training_set
    t0 = time.perf_counter()
    problems, samples = training_set(args.train_meshes, 16, 5, seed=0)
    torch.cuda.synchronize()
    t_harvest = time.perf_counter() - t0
    net = S.sem_net_create(5)
    t0 = time.perf_counter()
    losses = train(net, samples, args.train_steps, lr=3e-3, seed=1, loss="angle")
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    for prob, _ in problems:
        prob.close()
    del problems, samples
    prob, b = make_problem(32, 0.2, 4, ORDER, LAM, mixed=True)
    # quality on the unseen mesh: A-angle cosine of z0 = P r and z = z0 + N(s) with the error
    quality = []
    for s_, d_, r_, z0_ in harvest(prob, b, ks=(0, 2, 8, 24)):
        c = torch.empty_like(s_)
        S.sem_net_apply(net, prob.h, s_, c)
        e = d_ + z0_
        E = float(e @ r_)
        cos = lambda z: float(z @ r_) / np.sqrt(float(z @ prob.apply_A(z)) * E)
        quality.append({"cos_P": cos(z0_), "cos_P_plus_N": cos(z0_ + c)})
    out = {}
    for prec in ("fp64", "fp32"):
        prob.set_precision(prec)
        row = {}
        for name, nn in (("plain", None), ("learned", net)):
            its, ts, trs, used = [], [], [], []
            for _ in range(steps):
                it, dt, tr, rc, u = timed_solve(prob, b, nn, rtol=RTOL, maxit=1000, window=8, ratio=0.5, theta=0.25)
                its.append(it)
                ts.append(dt)
                trs.append(tr)
                used.append(u)
            row[name] = {"iterations": its[-1], "time_to_1e-8_s": float(np.median(ts)), "true_rel_res": trs[-1],
                         "iterations_using_network": used[-1] if nn is not None else 0}
        row["time_ratio_learned_over_plain"] = row["learned"]["time_to_1e-8_s"] / row["plain"]["time_to_1e-8_s"]
        row["iteration_gain"] = row["plain"]["iterations"] - row["learned"]["iterations"]
        out[prec] = row
    res = {"variant": "learned", "config": {
        "training": "%d seeded 16^3-hex meshes (+-20%%, seeds 1000..), n=5, lambda ~ U[0,10], manufactured and "
                    "Gaussian loads; samples at PCG iterates k in {0,1,2,4,8,16}; %d Adam steps, angle loss, "
                    "lr 3e-3 cosine" % (args.train_meshes, args.train_steps),
        "evaluation": "unseen 32^3-hex mesh, +-20% perturbation seed 4, n=7, lambda=1, manufactured load; "
                      "flexible PCG z = P r + N(r - A P r), accept if (z0+c).r >= 0.25 z0.r, off when "
                      "||r_k|| >= 0.5 ||r_k-8||",
        "n_dof": prob.n_dof, "params": S.sem_net_num_params()},
        "harvest_s": t_harvest, "train_s": t_train,
        "loss_first_50": float(np.mean(losses[:50])), "loss_last_300": float(np.mean(losses[-300:])),
        "unseen_mesh_angle_cosines": quality, **out}
    S.sem_net_destroy(net)
    prob.close()
    return res


def run_heat_variant(args):
    """The paper's heat-equation experiment (Sec. 5) on a synthetic rod: wall time for 70 steps."""
    print(json.dumps(heat_block(args, [int(v) for v in args.heat_orders.split(",")])))


def heat_block(args, orders):
    """The heat-rod experiment at the given orders; returns the result as a dict."""
    import numpy as np
    import torch
    from synth import lattice_hex_mesh, moving_source
    from paper_1506_05996_gb300 import sem as S
    kappa, dt, q0, rho, cp, steps = 1e-2, 0.04, 1000.0, 7000.0, 0.8, 70
    lam = 1.0 / (kappa * dt)
    mesh = lattice_hex_mesh((16, 16, 244), 0.2, 5, box=(1.0, 1.0, 15.25))
    rows = []
    for n in orders:
        t0 = time.perf_counter()
        prob = S.SemProblem(mesh.xyz, mesh.hex2vert, n, lam, geom=args.heat_geom, neumann=True,
                            mixed=(args.heat_geom == "stored"))
        t_setup = time.perf_counter() - t0
        X = prob.dof_coords().cpu().numpy()
        # the moving source at every step, prepared before the timed loop (input synthesis)
        gs = [torch.as_tensor(moving_source(X, dt * (k + 1), q0=q0) / (rho * cp * kappa), device="cuda")
              for k in range(steps)]
        row = {"n": n, "n_dof": prob.n_dof, "setup_s": t_setup}
        for prec in ("fp64", "fp32"):
            prob.set_precision(prec)
            u = torch.zeros(prob.n_dof, dtype=torch.float64, device="cuda")
            S.sem_heat_step(prob.h, u, gs[0], torch.empty_like(u), RTOL, 1000)   # warm-up (graph capture)
            torch.cuda.synchronize()
            its = []
            t0 = time.perf_counter()
            for k in range(steps):
                rc, it, tr = S.sem_heat_step(prob.h, u, gs[k], u, RTOL, 1000)
                its.append(it)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            row[prec] = {"wall_s_70_steps": wall, "iterations_total": int(sum(its)),
                         "iterations_per_step": [int(min(its)), int(max(its))],
                         "gdof_steps_per_s": prob.n_dof * steps / wall / 1e9,
                         "final_max_u": float(u.abs().max())}
        rows.append(row)
        prob.close()
        del gs
    return {"variant": "heat", "config": {
        "workload": "rod [0,1]x[0,1]x[0,15.25], 16x16x244 = 62,464 hexes, +-20% perturbation seed 5, insulated "
                    "(Neumann) boundary; backward Euler, kappa 1e-2, dt 0.04, c = 1/dt (lambda = 1/(kappa dt) "
                    "= 2500); moving Gaussian source Q = 1000 exp(-|x-c(t)|^2/(2*0.25^2)), c(t) = (0.5, 0.5, "
                    "1 + 2t), rho 7000, c_p 0.8; 70 steps, each to 1e-8 of its right-hand side from the "
                    "previous field; " + ("recomputed" if args.heat_geom == "recompute" else "stored")
                    + " geometric factors",
        "paper": "Table 4: 70 steps on a 62,540-hex rod, CUDA on a GTX 980 in FP32: 13.4 / 14.8 / 32.1 / 53.6 / "
                 "90.3 / 134.9 s for n = 2..7 (context: other hardware, other mesh, tolerance not stated)"},
        "orders": rows}


def run_patch_variant(args):
    """P^f patches with face layers only (default) against the full (n+3)^3 box, headline workload."""
    import numpy as np
    import torch
    from synth import lattice_hex_mesh, manufactured_s
    from paper_1506_05996_gb300 import sem as S
    mesh = lattice_hex_mesh(32, A_FULL, SEED_FULL)
    out = {}
    for patch in ("face", "full"):
        prob = S.SemProblem(mesh.xyz, mesh.hex2vert, ORDER, LAM, geom="stored", mixed=True, patch=patch)
        X = prob.dof_coords()
        b = (prob.mass() * torch.as_tensor(manufactured_s(X.cpu().numpy(), LAM), device="cuda")).contiguous()
        row = {}
        for prec in ("fp64", "fp32"):
            prob.set_precision(prec)
            x = torch.empty_like(b)
            for _ in range(max(1, args.warmup)):
                S.sem_solve(prob.h, b, x, RTOL, 1000, want_history=False)
            ts = []
            for _ in range(max(1, args.steps)):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rc, it, _, tr = S.sem_solve(prob.h, b, x, RTOL, 1000, want_history=False)
                torch.cuda.synchronize()
                ts.append(time.perf_counter() - t0)
            row[prec] = {"iterations": it, "time_to_1e-8_s": float(np.median(ts)), "true_rel_res": tr}
        out[patch] = row
        prob.close()
    print(json.dumps({"variant": "patch", "config": {"workload": WORKLOAD,
                      "face": "box nodes with one index in {-1, n+1} (face layers), others absent",
                      "full": "all (n+3)^3 box nodes (edge and corner layers filled)"}, **out}))


def run_kcycle_variant(args):
    """P_0 as the paper's K-cycle against the default V-cycles, same workload as the headline."""
    print(json.dumps(kcycle_block(args)))


def kcycle_block(args):
    """The K-cycle against the V-cycles on the headline workload; returns the result as a dict."""
    import numpy as np
    import torch
    from synth import lattice_hex_mesh, manufactured_s
    from paper_1506_05996_gb300 import sem as S
    mesh = lattice_hex_mesh(32, A_FULL, SEED_FULL)
    prob = S.SemProblem(mesh.xyz, mesh.hex2vert, ORDER, LAM, geom="stored", mixed=True)
    X = prob.dof_coords()
    b = (prob.mass() * torch.as_tensor(manufactured_s(X.cpu().numpy(), LAM), device="cuda")).contiguous()
    stream = torch.cuda.current_stream()
    out = {}
    for kind in ("vcycle", "kcycle"):
        t0 = time.perf_counter()
        prob.set_coarse_solver(kind)
        t_build = time.perf_counter() - t0
        row = {"amg_build_s": t_build}
        for prec in ("fp64", "fp32"):
            prob.set_precision(prec)
            x = torch.empty_like(b)
            for _ in range(max(1, args.warmup)):
                S.sem_solve(prob.h, b, x, RTOL, 1000, want_history=False)
            ts = []
            for _ in range(max(1, args.steps)):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                rc, it, _, tr = S.sem_solve(prob.h, b, x, RTOL, 1000, want_history=False)
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1) / 1e3)
            S.sem_profile(prob.h, 1)
            S.sem_solve(prob.h, b, x, RTOL, 1000, want_history=False)
            prof = S.sem_profile_read(prob.h)
            S.sem_profile(prob.h, 0)
            amg_ms, amg_launches = prof.get("coarse_amg", (0, 0.0))[1], prof.get("coarse_amg", (0, 0.0))[0]
            row[prec] = {"iterations": it, "time_to_1e-8_s": float(np.median(ts)), "true_rel_res": tr,
                         "coarse_amg_ms_per_application": amg_ms / max(1, it + 1),
                         "coarse_amg_kernels_per_application": amg_launches / max(1, it + 1)}
        out[kind] = row
    prob.set_precision("fp64")
    res = {"variant": "kcycle", "config": {
        "workload": WORKLOAD, "n_dof": prob.n_dof,
        "vcycle": "smoothed aggregation (3 pairwise passes), P_0 = three V(1,1) damped-Jacobi cycles, PCG",
        "kcycle": "unsmoothed aggregation (2 passes), P_0 = one recursive K-cycle with damped Jacobi (Sec. 4.1), "
                  "flexible PCG"}, **out}
    prob.close()
    return res


def main():
    args = parse()
    if args.patch_variant:
        run_patch_variant(args)
    elif args.kcycle_variant:
        run_kcycle_variant(args)
    elif args.heat_variant:
        run_heat_variant(args)
    elif args.learned_variant:
        run_learned_variant(args)
    elif args.batch_variant:
        run_batch_variant(args)
    elif args.precision_variant:
        run_precision_variant(args)
    elif args.kernel_case:
        run_kernel_case(args.kernel_case, args.kernel_geom)
    elif args.solve_case:
        run_solve_case(args.solve_case, args.solve_prec)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
