"""Benchmark of the multi-frequency Laplace-domain BEM operator on one B300.

Workload (the sphere configuration): unit sphere, icosphere with 5,120 flat
triangles (2,562 nodes), steel, K = 64 frequencies of BDF2 CQ with N = 64,
dt = 2e-5 s; collocation at the nodes (Neumann rows); cluster trees with leaf
32, admissibility eta = 2; 3D-ACA tolerance 1e-6.  One step = the whole hot
path for both operators of the Neumann system (single layer V: 2,562 x 5,120
blocks, double layer C + K: 2,562 x 2,562 blocks): entry generation,
near-field blocks, batched 3D-ACA, then the batched apply Y_k = C(s_k) X_k to
seeded N(0, 1) complex vectors of all K frequencies.

Prints one JSON line (see the keys below).  `--impl reference` times the FP64
CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthetic as syn  # noqa: E402

WORKLOAD = dict(workload="sphere-5120-K64", mesh="icosphere level 4, radius 1 m, 5120 triangles, 2562 nodes",
                material="steel rho=7850 E=210GPa nu=0.3", N=64, dt=2e-5, K=64, leaf=32, eta=2.0, eps=1e-6,
                rows="nodes (Neumann)", operators="V (SL) + C+K (DL)")
METRIC = "3D-ACA tensor entries/s"
# k_face DRAM traffic / algorithmic bytes of one launch at this workload's
# size (ncu dram__bytes_read.sum + dram__bytes_write.sum, one pass, launch
# 11 = iteration 10 of the single layer), None until the counters are taken
# on the current kernel
FACE_TRAFFIC_RATIO = 37.38e9 / (11 * 144 * 13117440)
FACE_TRAFFIC_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one bench-size launch (iteration 10 of "
                       "the single layer: 31.91 + 5.47 GB in 16.75 ms against 20.78 GB algorithmic, ratio 1.80), "
                       "times each launch's algorithmic bytes")
UNIT = "block entries/s"


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                if out:
                    self.samples.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if len(s) > 3 + i and "Active" in s[3 + i]
                          and "Not" not in s[3 + i]})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


# ---------------------------------------------------------------------------
# reference arm / CPU baseline: the FP64 oracle on a bounded sample
# ---------------------------------------------------------------------------

_ORACLE_TREES = {}


def _oracle_trees(s):
    """The oracle operators of both layers and their blocks in a seeded order
    (blocks of up to 150,000 tensor entries: a block takes seconds in the
    oracle, the largest would take minutes)."""
    from oracle import bem, pipeline
    xyz, tri = syn.icosphere(4)
    order = []
    for li, kern in enumerate((bem.KERNEL_SL, bem.KERNEL_DL)):
        op = bem.Operator(xyz, tri, syn.STEEL, rows=bem.ROWS_NODES, kernel=kern)
        _, _, blocks = pipeline.trees(op, WORKLOAD["leaf"], WORKLOAD["eta"])
        perm = np.random.default_rng(11 + li).permutation(len(blocks))
        order.append((op, [blocks[i] for i in perm
                           if len(blocks[i].rows.idx) * len(blocks[i].cols.idx) * len(s) <= 150000]))
    return order


def cpu_oracle_sample(budget_s: float = 15.0):
    """Block entries/s of the oracle doing the GPU's work on the bench
    workload: its own cluster and block trees of the sphere for V and C + K
    (node rows, leaf 32, eta 2), then, block by block in a seeded order
    alternating the two layers, the dense tensor of the block at all K
    frequencies and its 3D-ACA with face ACA (Algorithm 1, Eq. (3.12)),
    until the time budget is spent.  The oracle evaluates every entry of a
    block (m n K), which is the count reported."""
    from oracle import aca, bem
    s = bem.freqs_bdf2(WORKLOAD["N"], WORKLOAD["dt"], WORKLOAD["K"])
    eps = WORKLOAD["eps"]
    order = _ORACLE_TREES.get("order")
    if order is None:
        order = _ORACLE_TREES["order"] = _oracle_trees(s)
    t0 = time.perf_counter()
    c0 = time.process_time()
    n = 0
    done = [0, 0]
    sizes = []
    while time.perf_counter() - t0 < budget_s:
        li = (done[0] + done[1]) % 2
        op, blocks = order[li]
        if done[li] >= len(blocks):
            break
        b = blocks[done[li]]
        rows, cols = b.rows.idx, b.cols.idx
        C = op.block(rows, cols, s)
        aca.compress_block(C, rows, cols, b.far, eps, eps / 100.0)
        n += len(rows) * len(cols) * len(s)
        sizes.append((len(rows), len(cols)))
        done[li] += 1
    dt = time.perf_counter() - t0
    cpu = time.process_time() - c0
    return {"value": n / dt, "unit": UNIT, "cores": round(cpu / dt, 2), "kind": "oracle",
            "cores_how": "process CPU time / wall time over the sample (threads actually busy)",
            "host_cpus": os.cpu_count(), "cpu_model": _cpu_model(),
            "sample": (f"{done[0]} single-layer and {done[1]} double-layer blocks of the bench trees (seeded order, "
                       "blocks of at most 150,000 tensor entries), "
                       f"dense tensor at all {len(s)} frequencies + 3D-ACA + face ACA each; {n} block entries, "
                       f"{dt:.1f} s"),
            "same_work": "the bench's compression of both layers, on a sample of its blocks",
            "seconds": dt}


def _cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    steps = []
    for _ in range(args.warmup):
        cpu_oracle_sample(budget_s=2.0)
    for _ in range(args.steps):
        steps.append(cpu_oracle_sample(budget_s=10.0))
    v = float(np.mean([s["value"] for s in steps]))
    step_ms = float(np.mean([s["seconds"] for s in steps])) * 1e3
    cb = dict(steps[-1])
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(WORKLOAD), "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# small case for profiler captures (not a bench line)
# ---------------------------------------------------------------------------

def run_small(level=3):
    import torch
    import paper_2607_15292_b300 as g
    xyz, tri = syn.icosphere(level)
    s = g.freqs_bdf2(WORKLOAD["N"], WORKLOAD["dt"], WORKLOAD["K"])
    ctx = g.Context(eps=WORKLOAD["eps"], leaf=WORKLOAD["leaf"], eta=WORKLOAD["eta"], precision=g.BEM_MIXED)
    ctx.material(*syn.STEEL)
    ctx.freqs(s)
    t = ctx.mesh(xyz, tri).tree(g.BEM_ROWS_NODES, g.BEM_SL)
    op = t.compress()
    X = torch.tensor(syn.complex_normal(1, (len(s), t.n_cols, 3)), dtype=torch.complex64, device="cuda")
    Y = torch.empty((len(s), t.n_rows, 3), dtype=torch.complex64, device="cuda")
    op.apply(X, Y)
    torch.cuda.synchronize()
    st = op.stats()
    print(json.dumps({"case": f"icosphere-{level} single layer, node rows, K=64, MIXED", "face_launches": st.face_launches,
                      "face_alg_bytes": st.face_alg_bytes, "t_face_ms": st.t_face_ms,
                      "t_compress_ms": st.t_compress_ms, "apply_bytes": st.apply_bytes}))


# ---------------------------------------------------------------------------
# multi-mesh workload: one work list over many meshes (not the bench line)
# ---------------------------------------------------------------------------

def run_batch(count, n_max, n_streams):
    """Single layer, node rows, MIXED, of the multi-mesh workload (mesh i of
    synthetic.batch_meshes: N = K, dt = 0.6 h / c1): every operator
    compressed one after the other, then all from one work list on
    n_streams streams; block entries/s of both (dense tensor sizes summed)."""
    import time
    import torch
    import paper_2607_15292_b300 as g
    rho, lam, mu = syn.STEEL
    c1 = float(np.sqrt((lam + 2.0 * mu) / rho))   # P-wave speed, for dt of the recipe

    def trees():
        out = []
        for name, xyz, tri, K in syn.batch_meshes(count, n_max):
            e = np.concatenate([xyz[tri[:, 1]] - xyz[tri[:, 0]], xyz[tri[:, 2]] - xyz[tri[:, 1]]])
            h = float(np.linalg.norm(e, axis=1).mean())
            ctx = g.Context(eps=1e-6, leaf=32, eta=2.0, precision=g.BEM_MIXED)
            ctx.material(*syn.STEEL)
            ctx.freqs(g.freqs_bdf2(K, 0.6 * h / c1, K))
            out.append(ctx.mesh(xyz, tri).tree(g.BEM_ROWS_NODES, g.BEM_SL))
        return out
    warm = trees()[:2]
    g.compress_batch(warm, 2)
    del warm
    ts = trees()
    entries = sum(t.n_rows * t.n_cols * t.mesh.ctx.K for t in ts)
    # one operator at a time, each released before the next (the 32
    # compressed operators of the largest meshes do not fit together)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for t in ts:
        op = t.compress(stream=0)
        del op
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    # the work list in waves that fit the device: an operator's faces and
    # fibres during 3D-ACA take about 144 bytes per block entry and
    # iteration; with up to K / 3 iterations assumed, waves of at most
    # n_streams operators whose estimates sum to half the free memory
    ts = trees()
    ts.sort(key=lambda t: -t.n_rows * t.n_cols * t.mesh.ctx.K)
    budget = 0.5 * torch.cuda.mem_get_info()[0]
    waves, cur, used = [], [], 0.0
    for t in ts:
        est = 144.0 * t.n_rows * t.n_cols * max(1, t.mesh.ctx.K // 3)
        if cur and (len(cur) == n_streams or used + est > budget):
            waves.append(cur)
            cur, used = [], 0.0
        cur.append(t)
        used += est
    waves.append(cur)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for wv in waves:
        ops = g.compress_batch(wv, min(n_streams, len(wv)))
        del ops
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    print(json.dumps({"case": "multi-mesh workload, single layer, node rows, MIXED", "meshes": len(ts),
                      "n_max": n_max, "triangles": int(sum(t.n_cols for t in ts)), "block_entries": int(entries),
                      "sequential_s": t_seq, "batch_s": t_batch, "n_streams": n_streams,
                      "batch_form": f"{len(waves)} waves of at most {n_streams} operators (memory-bounded)",
                      "sequential_entries_per_s": entries / t_seq, "batch_entries_per_s": entries / t_batch}))


# ---------------------------------------------------------------------------
# adjoint workload: box, traction pulse, receiver energy gradient (not the
# bench line)
# ---------------------------------------------------------------------------

def run_adjoint(h, steps):
    """The box adjoint workload of synthetic.BOX_ADJOINT at grid spacing h
    (0.4 m is the full 20,000-triangle size): MIXED compression of V, C + K
    and their four wave-speed derivative operators (node rows), then the
    receiver energy and its gradient in the traction and in c_p, c_s
    (bem_receiver_energy_grad: forward solve, adjoint solve, CQ transforms)
    timed over `steps` calls after one warm-up call; one JSON line."""
    import torch
    import paper_2607_15292_b300 as g
    w = syn.BOX_ADJOINT
    xyz, tri = syn.box(w["lx"], w["ly"], w["lz"], h)
    N, dt = w["N"], w["dt"]
    K = (N + 1) // 2 + 1
    s = g.freqs_bdf2(N, dt, K)
    ctx = g.Context(eps=1e-6, leaf=32, eta=2.0, precision=g.BEM_MIXED)
    ctx.material(*syn.STEEL)
    ctx.freqs(s)
    mesh = ctx.mesh(xyz, tri)
    kinds = (g.BEM_SL, g.BEM_DL, g.BEM_SL_DCP, g.BEM_SL_DCS, g.BEM_DL_DCP, g.BEM_DL_DCS)
    trees = [mesh.tree(g.BEM_ROWS_NODES, k) for k in kinds]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ops = [t.compress() for t in trees]
    torch.cuda.synchronize()
    t_comp = time.perf_counter() - t0
    V, A, dVp, dVs, dAp, dAs = ops
    A.set_precond(1)   # block Jacobi for the forward and adjoint solves
    gt = torch.tensor(syn.box_traction(xyz, tri, N, dt, w["width"], w["t0"], w["tw"]), dtype=torch.float64,
                      device="cuda")
    rec = syn.box_receivers(xyz, w["receivers"])
    args = dict(dV=(dVp, dVs), dA=(dAp, dAs), tol=1e-6, max_iter=500)
    g.receiver_energy_grad(V, A, gt, rec, N, dt, **args)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        J, dg, dc, it = g.receiver_energy_grad(V, A, gt, rec, N, dt, **args)
    torch.cuda.synchronize()
    t_grad = (time.perf_counter() - t0) / steps
    st = [o.stats() for o in ops]
    print(json.dumps({
        "case": "box adjoint workload (receiver energy and its gradient in traction and c_p, c_s)",
        "box": [w["lx"], w["ly"], w["lz"]], "h": h, "triangles": len(tri), "nodes": len(xyz), "N": N, "dt": dt,
        "K": K, "receivers": len(rec), "precision": "MIXED", "eps": 1e-6, "solve_tol": 1e-6,
        "preconditioner": "block Jacobi (3x3 diagonal blocks of C + K)",
        "compress_s_six_operators": t_comp, "gradient_ms": t_grad * 1e3, "steps": steps,
        "J": J, "dJ_dc": dc, "dJ_dg_max": float(dg.abs().max()),
        "iters_forward_max": int(it[:K].max()), "iters_adjoint_max": int(it[K:].max()),
        "stored_gb": [round(x.stored_bytes / 1e9, 3) for x in st],
        "rank_mean": [round(x.rank_mean, 2) for x in st]}))


def run_rkcq(h, steps, N=127):
    """Runge-Kutta CQ (2-stage Radau IIA) of the box single layer at grid
    spacing h (the box of synthetic.BOX_ADJOINT; 0.4 m is 20,000 triangles):
    N + 1 steps of dt = 2 x BOX_ADJOINT's dt over the same time span, the
    half frequency set (K = 2 (floor((N + 1) / 2) + 1) = 130 of the 256:
    conjugate pairs of real data); MIXED compression, then
    bem_rkcq_apply (stage DFT + eigen-mixing, batched apply, unmix, inverse
    DFT) timed over `steps` calls after one warm-up call, beside the
    batched apply alone at the same K; one JSON line."""
    import torch
    import paper_2607_15292_b300 as g
    w = syn.BOX_ADJOINT
    xyz, tri = syn.box(w["lx"], w["ly"], w["lz"], h)
    dt = 2.0 * w["dt"]
    s, _ = g.freqs_radau2(N, dt, half=True)
    ctx = g.Context(eps=1e-6, leaf=32, eta=2.0, precision=g.BEM_MIXED)
    ctx.material(*syn.STEEL)
    ctx.freqs(s)
    mesh = ctx.mesh(xyz, tri)
    tree = mesh.tree(g.BEM_ROWS_NODES, g.BEM_SL)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    V = tree.compress()
    torch.cuda.synchronize()
    t_comp = time.perf_counter() - t0
    gs = torch.tensor(syn.box_traction(xyz, tri, N, dt, w["width"], w["t0"], w["tw"], offsets=(1.0 / 3.0, 1.0)),
                      dtype=torch.float64, device="cuda")
    y = torch.empty((N + 1, 2, tree.n_rows, 3), dtype=torch.float64, device="cuda")
    g.rkcq_apply(V, gs, y, N, dt)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    torch.cuda.synchronize()
    ev[0].record()
    for _ in range(steps):
        g.rkcq_apply(V, gs, y, N, dt)
    ev[1].record()
    X = torch.zeros((len(s), tree.n_cols, 3), dtype=torch.complex64, device="cuda")
    Y = torch.empty((len(s), tree.n_rows, 3), dtype=torch.complex64, device="cuda")
    V.apply(X, Y)
    ev[2].record()
    for _ in range(steps):
        V.apply(X, Y)
    ev[3].record()
    torch.cuda.synchronize()
    t_rk = ev[0].elapsed_time(ev[1]) / steps
    t_ap = ev[2].elapsed_time(ev[3]) / steps
    st = V.stats()
    print(json.dumps({
        "case": "box single layer, RK-CQ with 2-stage Radau IIA (constant steps)",
        "box": [w["lx"], w["ly"], w["lz"]], "h": h, "triangles": len(tri), "nodes": len(xyz), "N": N, "dt": dt,
        "K": len(s), "frequency_set": "half (conjugate pairs)", "precision": "MIXED", "eps": 1e-6,
        "compress_s": t_comp, "rkcq_ms": t_rk,
        "batched_apply_ms": t_ap, "transforms_and_mixing_ms": t_rk - t_ap, "steps": steps,
        "y_max": float(y.abs().max()), "stored_gb": round(st.stored_bytes / 1e9, 3),
        "rank_mean": round(st.rank_mean, 2)}))


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def combine_ranks(ms, units, device):
    """Whole-job figures of independent replicas (one per rank, each with
    its own operators and work): the slowest rank's time and the units of
    all ranks (torch.distributed, initialised by the caller: NCCL on the
    GPUs, gloo in the CPU tests)."""
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(u)
    return float(t.item()), int(round(u.item()))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--small", action="store_true",
                    help="one MIXED compression and batched apply of the icosphere-3 single layer "
                         "(1,280 triangles, K = 64), for profiler captures; prints its statistics")
    ap.add_argument("--small-level", type=int, default=3, metavar="L",
                    help="icosphere level of --small (4: the bench mesh, for a bench-size capture of one kernel)")
    ap.add_argument("--batch", type=int, default=0, metavar="COUNT",
                    help="multi-mesh workload: compress the first COUNT meshes one by one and from one "
                         "work list; prints both rates (not the bench line)")
    ap.add_argument("--batch-nmax", type=int, default=25, help="cap on the grid size n of --batch meshes")
    ap.add_argument("--batch-streams", type=int, default=4)
    ap.add_argument("--adjoint", type=float, default=0.0, metavar="H",
                    help="box adjoint workload at grid spacing H (0.4 = full size): compression of the six "
                         "operators and the receiver-energy gradient; prints its statistics (not the bench line)")
    ap.add_argument("--rkcq", type=float, default=0.0, metavar="H",
                    help="box single layer through Runge-Kutta CQ (2-stage Radau IIA, half set K = 130) at grid spacing "
                         "H (0.4 = full size); prints its statistics (not the bench line)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.small:
        return run_small(args.small_level)
    if args.batch:
        return run_batch(args.batch, args.batch_nmax, args.batch_streams)
    if args.adjoint > 0:
        return run_adjoint(args.adjoint, max(1, args.steps))
    if args.rkcq > 0:
        return run_rkcq(args.rkcq, max(1, args.steps))

    import torch
    import paper_2607_15292_b300 as g

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    # roofline denominators of this GPU's units (FP32, FP64, ex2, TF32 MMA)
    unit_peaks = g.measure_peaks(local)

    xyz, tri = syn.icosphere(4)
    s = g.freqs_bdf2(WORKLOAD["N"], WORKLOAD["dt"], WORKLOAD["K"])
    K = len(s)

    def make(precision):
        ctx = g.Context(eps=WORKLOAD["eps"], leaf=WORKLOAD["leaf"], eta=WORKLOAD["eta"], precision=precision,
                        device=local)
        ctx.material(*syn.STEEL)
        ctx.freqs(s)
        mesh = ctx.mesh(xyz, tri)
        return ctx, mesh, mesh.tree(g.BEM_ROWS_NODES, g.BEM_SL), mesh.tree(g.BEM_ROWS_NODES, g.BEM_DL)

    ctx, mesh, tV, tK = make(g.BEM_MIXED)
    cdt = torch.complex64
    XV = torch.tensor(syn.complex_normal(1, (K, len(tri), 3)), dtype=cdt, device=dev)
    XK = torch.tensor(syn.complex_normal(2, (K, len(xyz), 3)), dtype=cdt, device=dev)
    YV = torch.empty((K, len(xyz), 3), dtype=cdt, device=dev)
    YK = torch.empty((K, len(xyz), 3), dtype=cdt, device=dev)

    def step():
        oV = tV.compress(stream)
        oK = tK.compress(stream)
        oV.apply(XV, YV, g.BEM_APPLY_BATCHED, stream)
        oK.apply(XK, YK, g.BEM_APPLY_BATCHED, stream)
        return oV, oK

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    entries = 0
    entry_ms = 0.0
    face = {"ms": 0.0, "launches": 0, "bytes": 0.0}
    l0 = g.kernel_launches()
    with Clocks(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            oV, oK = step()
            sv, sk = oV.stats(), oK.stats()
            entries += sv.entries_evaluated + sk.entries_evaluated
            entry_ms += sv.t_entries_ms + sk.t_entries_ms
            for st_ in (sv, sk):
                face["ms"] += st_.t_face_ms
                face["launches"] += st_.face_launches
                face["bytes"] += st_.face_alg_bytes
        ev1.record(stream)
        barrier()
    launches = g.kernel_launches() - l0
    ms = ev0.elapsed_time(ev1)
    if world > 1:
        ms, entries = combine_ranks(ms, entries, dev)
    value = entries / (ms / 1e3)

    # apply throughput (algorithmic bytes / time) on the compressed operators:
    # the tensor-core kernel (the MIXED default) and, for comparison, the
    # SIMT kernel on the same operators
    oV, oK = step()
    torch.cuda.synchronize()
    reps = 20

    def time_apply():
        for _ in range(2):
            oV.apply(XV, YV, g.BEM_APPLY_BATCHED, stream)
            oK.apply(XK, YK, g.BEM_APPLY_BATCHED, stream)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(reps):
            oV.apply(XV, YV, g.BEM_APPLY_BATCHED, stream)
            oK.apply(XK, YK, g.BEM_APPLY_BATCHED, stream)
        a1.record(stream)
        torch.cuda.synchronize()
        return a0.elapsed_time(a1) / reps
    for o in (oV, oK):
        o.set_apply_kernel(0)
    apply_ms_simt = time_apply()
    for o in (oV, oK):
        o.set_apply_kernel(1)
    apply_ms = time_apply()
    sv, sk = oV.stats(), oK.stats()
    apply_bytes = sv.apply_bytes + sk.apply_bytes
    apply_gbs = apply_bytes / (apply_ms / 1e3) / 1e9
    apply_tflops = (sv.apply_tensor_flops + sk.apply_tensor_flops) / (apply_ms / 1e3) / 1e12

    extra = {"apply_gbs": apply_gbs, "apply_ms": apply_ms, "apply_kernel": "tcgen05 kind::tf32 (split operands)",
             "apply_ms_simt": apply_ms_simt, "apply_gbs_simt": apply_bytes / (apply_ms_simt / 1e3) / 1e9,
             "apply_tensor_tflops": apply_tflops, "compression_rate_V": sv.compression_rate,
             "compression_rate_K": sk.compression_rate, "rank_mean_V": sv.rank_mean, "rank_mean_K": sk.rank_mean,
             "blocks_V": [sv.n_aca, sv.n_dense, sv.n_rank0], "blocks_K": [sk.n_aca, sk.n_dense, sk.n_rank0],
             "faces_lowrank_V": [sv.n_faces_lowrank, sv.n_faces], "faces_lowrank_K": [sk.n_faces_lowrank, sk.n_faces],
             "face_rank_mean_V": sv.face_rank_mean, "face_rank_mean_K": sk.face_rank_mean,
             "face_aca_ms_V": sv.t_face_aca_ms, "face_aca_ms_K": sk.t_face_aca_ms,
             "compress_ms_V": sv.t_compress_ms, "compress_ms_K": sk.t_compress_ms}

    # end-to-end solve of the Neumann problem of the workload (sphere under
    # uniform pressure): b_k = V(s_k) t, t = -n; (C + K)(s_k) u_k = b_k for all
    # 64 frequencies by the K-batched BiCGstab on the compressed operators
    e1 = xyz[tri[:, 1]] - xyz[tri[:, 0]]
    e2 = xyz[tri[:, 2]] - xyz[tri[:, 0]]
    nrm = np.cross(e1, e2)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    Tload = torch.tensor(np.broadcast_to(-nrm, (K,) + nrm.shape).copy(), dtype=cdt, device=dev)
    Bload = torch.empty((K, len(xyz), 3), dtype=cdt, device=dev)
    Usol = torch.empty_like(Bload)
    torch.cuda.synchronize()
    t0s = time.perf_counter()
    oV.apply(Tload, Bload, g.BEM_APPLY_BATCHED, stream)
    its, rres = oK.solve(Bload, Usol, tol=2e-6, max_iter=300, stream=stream, check=False)
    torch.cuda.synchronize()
    solve_s = time.perf_counter() - t0s
    extra.update({"solve_ms": solve_s * 1e3, "solve_iters_max": int(its.max()), "solve_iters_mean": float(its.mean()),
                  "solve_relres_max": float(rres.max()),
                  "solve": "Neumann sphere under uniform pressure, all 64 frequencies, BiCGstab tol 2e-6, "
                           "right-hand side V t included"})

    # error against the exact operator on sampled rows: the rows of C(s_k)
    # from the library's FP64 entries (parity-checked against the oracle to
    # 1e-10), applied to the same vectors
    rows_sample = np.sort(np.random.default_rng(5).choice(len(xyz), 24, replace=False))
    ctxE = g.Context(eps=WORKLOAD["eps"], precision=g.BEM_FP64, device=local)
    ctxE.material(*syn.STEEL)
    ctxE.freqs(s)
    meshE = ctxE.mesh(xyz, tri)

    def exact_rows(kern, X):
        ncol = len(tri) if kern == g.BEM_SL else len(xyz)
        r_, c_, k_ = np.meshgrid(rows_sample, np.arange(ncol), np.arange(K), indexing="ij")
        req = torch.tensor(np.stack([r_.ravel(), c_.ravel(), k_.ravel()], 1).astype(np.int32), device=dev)
        out = torch.empty((req.shape[0], 3, 3), dtype=torch.complex128, device=dev)
        meshE.entries(g.BEM_ROWS_NODES, kern, req, out, stream)
        C = out.view(len(rows_sample), ncol, K, 3, 3)
        return torch.einsum("ijkab,kjb->kia", C, X.to(torch.complex128))

    def rel(a, b):
        return (torch.linalg.norm(a - b) / torch.linalg.norm(b)).item()

    YV_ex = exact_rows(g.BEM_SL, XV)
    YK_ex = exact_rows(g.BEM_DL, XK)
    oV.apply(XV, YV, g.BEM_APPLY_BATCHED, stream)
    oK.apply(XK, YK, g.BEM_APPLY_BATCHED, stream)
    torch.cuda.synchronize()
    rs = torch.tensor(rows_sample, device=dev)
    extra.update({"mixed_vs_exact_rel_err_V": rel(YV[:, rs].to(torch.complex128), YV_ex),
                  "mixed_vs_exact_rel_err_K": rel(YK[:, rs].to(torch.complex128), YK_ex),
                  "error_sample": "24 seeded node rows x all columns x all 64 frequencies, FP64 entries"})

    # FP64 GPU form: same path in FP64, speedup and error of the mixed apply
    if not args.no_fp64:
        ctx64, mesh64, tV64, tK64 = make(g.BEM_FP64)
        XV64, XK64 = XV.to(torch.complex128), XK.to(torch.complex128)
        YV64 = torch.empty((K, len(xyz), 3), dtype=torch.complex128, device=dev)
        YK64 = torch.empty_like(YV64)
        # warm-up: every FP64 kernel launched once (module load, attributes)
        # on the icosphere-2 mesh, then two timed steps of the workload
        xw, tw = syn.icosphere(2)
        cw = g.Context(eps=WORKLOAD["eps"], leaf=WORKLOAD["leaf"], eta=WORKLOAD["eta"], precision=g.BEM_FP64,
                       device=local)
        cw.material(*syn.STEEL)
        cw.freqs(s)
        mw = cw.mesh(xw, tw)
        for kern, ncol in ((g.BEM_SL, len(tw)), (g.BEM_DL, len(xw))):
            ow = mw.tree(g.BEM_ROWS_NODES, kern).compress(stream)
            ow.apply(torch.zeros((K, ncol, 3), dtype=torch.complex128, device=dev),
                     torch.empty((K, len(xw), 3), dtype=torch.complex128, device=dev), g.BEM_APPLY_BATCHED, stream)
        torch.cuda.synchronize()
        fp64_steps = 2
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        for _ in range(fp64_steps):
            oV64 = tV64.compress(stream)
            oK64 = tK64.compress(stream)
            oV64.apply(XV64, YV64, g.BEM_APPLY_BATCHED, stream)
            oK64.apply(XK64, YK64, g.BEM_APPLY_BATCHED, stream)
        b1.record(stream)
        torch.cuda.synchronize()
        ms64 = b0.elapsed_time(b1) / fp64_steps
        e64 = oV64.stats().entries_evaluated + oK64.stats().entries_evaluated
        s64V, s64K = oV64.stats(), oK64.stats()
        extra.update({"fp64_compression_rate_V": s64V.compression_rate, "fp64_compression_rate_K": s64K.compression_rate,
                      "fp64_faces_lowrank_V": [int(s64V.n_faces_lowrank), int(s64V.n_faces)],
                      "fp64_faces_lowrank_K": [int(s64K.n_faces_lowrank), int(s64K.n_faces)],
                      "fp64_rank_mean_V": s64V.rank_mean, "fp64_rank_mean_K": s64K.rank_mean})
        oV.apply(XV, YV, g.BEM_APPLY_BATCHED, stream)
        oK.apply(XK, YK, g.BEM_APPLY_BATCHED, stream)
        torch.cuda.synchronize()
        errV = (torch.linalg.norm(YV.to(torch.complex128) - YV64) / torch.linalg.norm(YV64)).item()
        errK = (torch.linalg.norm(YK.to(torch.complex128) - YK64) / torch.linalg.norm(YK64)).item()
        extra.update({"fp64_entries_per_s": e64 / (ms64 / 1e3), "fp64_ms_per_step": ms64,
                      "fp64_timing": f"{fp64_steps} steps after an FP64 warm-up on icosphere level 2",
                      "mixed_vs_fp64_speedup": (ms64 / 1e3) / (ms / args.steps / 1e3),
                      "mixed_vs_fp64_rel_err_V": errV, "mixed_vs_fp64_rel_err_K": errK,
                      "fp64_vs_exact_rel_err_V": rel(YV64[:, rs], YV_ex),
                      "fp64_vs_exact_rel_err_K": rel(YK64[:, rs], YK_ex)})
        del oV64, oK64

    # end to end through the public API with host buffers
    XVh = torch.empty(XV.shape, dtype=cdt, pin_memory=True)
    XVh.copy_(XV.cpu())
    XKh = torch.empty(XK.shape, dtype=cdt, pin_memory=True)
    XKh.copy_(XK.cpu())
    YVh = torch.empty(YV.shape, dtype=cdt, pin_memory=True)
    YKh = torch.empty(YK.shape, dtype=cdt, pin_memory=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e_entries = 0
    for _ in range(args.steps):
        c2, m2, tv2, tk2 = make(g.BEM_MIXED)
        XV.copy_(XVh, non_blocking=True)
        XK.copy_(XKh, non_blocking=True)
        o1 = tv2.compress(stream)
        o2 = tk2.compress(stream)
        o1.apply(XV, YV, g.BEM_APPLY_BATCHED, stream)
        o2.apply(XK, YK, g.BEM_APPLY_BATCHED, stream)
        YVh.copy_(YV, non_blocking=True)
        YKh.copy_(YK, non_blocking=True)
        torch.cuda.synchronize()
        e_entries += o1.stats().entries_evaluated + o2.stats().entries_evaluated
    e2e_s = time.perf_counter() - t0
    h2d = (xyz.nbytes + tri.astype(np.int32).nbytes) + XV.numel() * 8 + XK.numel() * 8
    d2h = YV.numel() * 8 + YK.numel() * 8

    peaks = _peaks()
    hbm = peaks.get("hbm_gbs") or 6400.0
    face_gbs = face["bytes"] / (face["ms"] / 1e3) / 1e9 if face["ms"] > 0 else None
    alg_per_launch = face["bytes"] / max(1, face["launches"])
    roofline = {"kernel": "k_face (3D-ACA face: FP32 entries, float-float residual pass and FP32 Gram pass over the "
                          "TMA-staged previous faces), MIXED",
                "bound": "hbm", "achieved": face_gbs, "peak": hbm, "unit": "GB/s",
                "frac": (face_gbs / hbm) if face_gbs else None,
                # DRAM read + write per launch: the ratio to the algorithmic bytes
                # of one bench-size launch (ncu), times the bytes per launch
                "traffic": FACE_TRAFFIC_RATIO * alg_per_launch if FACE_TRAFFIC_RATIO else None,
                "traffic_source": FACE_TRAFFIC_SOURCE if FACE_TRAFFIC_RATIO
                else "not yet captured for this kernel version",
                "launches": face["launches"],
                "avg_launch_ms": face["ms"] / max(1, face["launches"]),
                "algorithmic_bytes_per_launch": face["bytes"] / max(1, face["launches"]),
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6.4 TB/s"}
    # the batched apply on the tensor cores: TF32 work against the measured
    # kind::tf32 rate (bem_measure_peaks on this GPU), bytes against HBM
    tf32_peak = unit_peaks.get("tf32_tflops_n128")
    apply_roof = {"kernel": "k_apply_faces_tc (batched apply, tcgen05 kind::tf32, split operands), MIXED",
                  "bound": "tensor", "achieved": extra["apply_tensor_tflops"], "peak": tf32_peak, "unit": "TFLOP/s",
                  "frac": extra["apply_tensor_tflops"] / tf32_peak if tf32_peak else None,
                  "peak_source": "bem_measure_peaks tcgen05 kind::tf32 M=128 N=128 (of measured)",
                  "hbm_achieved_gbs": apply_gbs, "hbm_frac": apply_gbs / hbm,
                  "work": "24 x rows x columns x K TF32 flops per face (8 per complex multiply-add, 3 split "
                          "products), stored operator + X + Y bytes"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64",
            "dtype_detail": ("MIXED: FP32 entries (near/singular included), float-float 3D-ACA faces/fibres "
                             "during compression, c64 storage and apply; FP64 rigid-body diagonal, fibre step, "
                             "pivots and norms"),
            "data": "synthetic", "config": dict(WORKLOAD, l2="inputs larger than L2 (faces ~GB)"),
            "clocks": clk.summary(),
            "e2e": {"value": e_entries / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": launches, "roofline": roofline, "roofline_apply": apply_roof,
            "unit_peaks": unit_peaks, **extra}
    line["entry_kernels_ms_per_step"] = entry_ms / args.steps
    line["peaks_source"] = "MEASURED_PEAKS.json" if peaks else "fallback"
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_oracle_sample(15.0)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
