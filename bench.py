"""Benchmark of the preconditioned Richardson solve (Algorithm 3) on one GB300.

One step = one complete solve, from u_0 = 0 to the relative residual 1e-6, of
the checkerboard workload: unit square, 128 x 128 mesh (16,641 P1 nodes),
512-triangle sphere (256 even / 768 odd angular functions), Henyey-Greenstein
g = 0.9, sigma_t in {1, 10} on a 4 x 4 checkerboard, sigma_s = 0.99 sigma_t,
one seeded Gaussian source.  Every row of the hot path runs in every
iteration: transport A / A^T, (M^- - K^-)^{-1}, K^+, E_0^{-1} by per-direction
CG, P_1^l, restriction, coarse solve and prolongation.

Prints one JSON line.  value = DOF * iterations / second (DOF = n_R^+ n_S^+
per right-hand side), device-timed with CUDA events over K steps after W
warm-up steps; e2e = the same metric through the C ABI with host buffers
(host->device copy of the nodal source, assembly of q, solve, device->host
copy of u inside the timed region).

--impl reference times the FP64 CPU oracle instead (a bounded sample of the
same workload on the host cores).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("time-to-1e-6 residual & DOF·iter/s, mixed vs FP64 on GB300; "
          "p50/p99 solve latency")
WORKLOAD = dict(workload='checkerboard_128x128_T512_g0.90_c0.99', mesh=128,
                sphere_triangles=512, g=0.9, sigma_s_over_sigma_t=0.99,
                tol=1e-6)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument('--gpus', type=int, default=1)
    ap.add_argument('--steps', type=int, default=3)
    ap.add_argument('--warmup', type=int, default=3)
    ap.add_argument('--impl', default='ours', choices=['ours', 'reference'])
    ap.add_argument('--precision', default='mixed_bf16',
                    choices=['fp64', 'mixed_fp32', 'mixed_bf16'])
    ap.add_argument('--mesh', type=int, default=128,
                    help='mesh size (profiling of smaller cases only)')
    ap.add_argument('--levels', type=int, default=3,
                    help='sphere refinement levels (profiling only)')
    ap.add_argument('--profile-once', action='store_true',
                    help='set up, run one solve and exit (for ncu captures)')
    ap.add_argument('--no-cpu-baseline', action='store_true')
    ap.add_argument('--no-fp64-compare', action='store_true',
                    help='skip the plain-FP64 comparison solve')
    ap.add_argument('--no-serving', action='store_true',
                    help='skip the serving (continuous batching) measurement')
    ap.add_argument('--serve-requests', type=int, default=48)
    ap.add_argument('--serve-sweep', action='store_true',
                    help='also sweep the arrival rate of the serving stream (minutes)')
    ap.add_argument('--batch', action='store_true',
                    help='also time the 64 uneven instances of the batching workload')
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get('RANK', '0'))
    world = int(os.environ.get('WORLD_SIZE', '1'))
    local = int(os.environ.get('LOCAL_RANK', '0'))
    return rank, world, local


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons during a timed region."""
    Q = ('index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,'
         'clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,'
         'clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap')

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ['nvidia-smi', '-i', str(self.index), '--query-gpu=' + self.Q,
                 '--format=csv,noheader,nounits', '-lms', '200'],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ['hw_slowdown', 'hw_thermal_slowdown', 'sw_thermal_slowdown',
                 'sw_power_cap']
        for ln in self.lines:
            f = [x.strip() for x in ln.split(',')]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith('active'):
                    reasons.add(n)
        if not sm:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=['unsampled'])
        return dict(sm_mhz=statistics.median(sm), sm_max_mhz=max(mx),
                    reasons=sorted(reasons), samples=len(sm))


def aggregate(secs, units, world):
    """Whole-job throughput of independent replicas: the slowest rank's time
    (max over ranks) and the units all ranks processed.  Works with the gloo
    (CPU tensors) and NCCL (CUDA tensors) backends."""
    if world <= 1:
        return secs, units
    import torch
    import torch.distributed as dist
    dev = 'cuda' if dist.get_backend() == 'nccl' else 'cpu'
    t = torch.tensor([float(secs)], dtype=torch.float64, device=dev)
    u = torch.tensor([float(units)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def load_peaks():
    path = os.path.join(ROOT, 'MEASURED_PEAKS.json')
    try:
        with open(path) as f:
            return json.load(f), 'measured'
    except OSError:
        return dict(hbm_gbs=6800.0, bf16_tflops=1900.0), 'fallback'


def fp64_peak_tflops(torch):
    """Measured FP64 contraction rate of this GPU: cuBLAS DGEMM through
    torch (best of 5 after warm-up), the denominator for FP64 contractions."""
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device='cuda')
    b = torch.randn(n, n, dtype=torch.float64, device='cuda')
    for _ in range(2):
        torch.matmul(a, b)
    torch.cuda.synchronize()
    best = 1e9
    for _ in range(5):
        e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    return 2.0 * n ** 3 / best / 1e12


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of a
# kernel group as last captured with ncu on the default workload (the summary
# and command are in profiles/); a kernel changed since its capture has no
# entry.  k_e0_pcg_f: mean of two captured launches (the 9th and 10th of the
# solve).
PROFILED_DRAM_BYTES = {'e0_cg_lo': 2.81e9}


def kernel_work(name, d, nrhs, info):
    """Algorithmic work of one launch of a named kernel group: (amount, unit,
    bound).  Contractions count 2 M N K flops.  Memory-bound kernels count
    the bytes they must move once per launch:
      * transport A: read U^+ (FP64), write Z (FP64);
      * A^T + M^+ + R - K^+ gather: read Z, U^+ and U S^+, write Y;
      * E_0 PCG (persistent): per CG iteration the coarsest level's dense
        per-direction inverses (read once per V-cycle) and, per (node, column), the level-0
        CG vector traffic (P read and AP written by the apply; P, R, AP read,
        R and V-cycle input written by the update; R, z read for r.z and
        r.r; z, P read and P written by the direction update: 12 words of
        the CG precision, plus the iterate read and written: 16 B in FP64,
        8 B in the FP32 kernel, which writes FP64 X once at the end) and the
        V-cycle's 17 FP32 array
        passes per level (4^-l of the level-0 size), times the V-cycles of
        the launch (the mean over the solve's launches), each weighted by the
        fraction of direction quads with a column not yet converged: the
        mixed-mode kernel visits only those.  The FP32 kernel forms the stencil coefficients on chip
        (224 B per node per pass, not counted); the FP64 kernel also reads 7
        FP64 coefficients per item;
      * E_c PCG: per iteration the FP64 level-0 blocks (7 d^2 per node) and
        ~12 FP64 vector passes, plus the FP32 V-cycle (7 d^2 + 18 d words
        per node per sweep-equivalent, 4/3 for the coarser levels)."""
    nRp, nRm, nS, nSm = d['nRp'], d['nRm'], d['nSp'], d['nSm']
    if name in ('gemm_mk_eig1', 'gemm_mk_eig2'):
        return 2.0 * nrhs * nRm * nSm * nSm, 'flop', 'fp64'
    if name in ('tc_gemm_mk1', 'tc_gemm_mk2'):
        return 2.0 * nrhs * nRm * nSm * nSm, 'flop', 'tensor'
    if name == 'gemm_kplus':
        return 2.0 * nrhs * nRp * nS * nS, 'flop', 'fp64'
    if name == 'transport_A':
        return 8.0 * nrhs * (nRp * nS + nRm * nSm), 'byte', 'hbm'
    if name == 'apply_even':
        return 8.0 * nrhs * (nRm * nSm + 3 * nRp * nS), 'byte', 'hbm'
    if name in ('e0_cg', 'e0_cg_lo'):
        ts = 8 if name == 'e0_cg' else 4
        cols = nrhs * nS
        cg = nRp * cols * (12 * ts + 2 * ts + (7 * 8 if name == 'e0_cg' else 0))
        vc = sum(nRp / 4 ** l * cols * 4 * 17 for l in range(d['e0_levels']))
        # the coarsest level's dense per-direction inverses, read once per V-cycle
        mc = d['mesh'] >> (d['e0_levels'] - 1)
        vc += ((mc + 1) ** 2) ** 2 * nS * 4
        # V-cycles per launch, each weighted by the fraction of direction
        # quads still active (converged columns are not visited again)
        n = info.get('e0_launches', 0)
        per = info['e0_active_vcycles'] / n if n else max(info.get('e0_iters', 1), 1)
        once = nRp * cols * 16   # B read and X written in FP64, once per launch
        return (cg + vc) * per + once, 'byte', 'hbm'
    if name == 'coarse_cg':
        dp = d['dP']
        cg = nRp * nrhs * (7 * dp * dp + 12 * dp) * 8
        vc = nRp * nrhs * (7 * dp * dp + 18 * dp) * 4 * 6 * 4 / 3
        return (cg + vc) * max(info.get('coarse_iters', 1), 1), 'byte', 'hbm'
    return None


def levels_of(m, max_nodes=300):
    """Multigrid levels the library builds for an m x m mesh (m -> m // 2
    while m >= 4 and the level has more than max_nodes nodes)."""
    lv = 1
    while m >= 4 and (m + 1) ** 2 > max_nodes:
        m //= 2
        lv += 1
    return lv


def run_ours(args):
    import numpy as np
    import torch
    import workloads
    import paper_2102_09038_gb300 as rte

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group('nccl')
    prec = dict(fp64=rte.FP64, mixed_fp32=rte.MIXED_FP32,
                mixed_bf16=rte.MIXED_BF16)[args.precision]
    p = workloads.checkerboard(m=args.mesh, levels=args.levels, g=0.9, ratio=0.99,
                               seed=rank)
    solver = rte.Solver(p, precision=prec)
    setup_ms = {k: round(v, 1) for k, v in solver.setup_times().items()}
    qn = torch.tensor(p.q_nodal, dtype=torch.float64, device='cuda')
    q = solver.rhs(qn)
    u = solver.even(p.nrhs)
    stream = solver.stream
    dofs = p.dofs * p.nrhs

    def step():
        u.zero_()
        _, info = solver.solve(q, u=u, tol=p.tol)
        if info['status'] != 0:
            raise RuntimeError('solve failed: %s' % info)
        return info

    if args.profile_once:
        info = step()
        torch.cuda.synchronize()
        print(json.dumps(dict(profile_once=True, iterations=info['iterations'],
                              rel_residual=info['rel_residual'])))
        return
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    launches0 = rte.kernel_launches()
    iters = 0
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
        e0.record(stream)
        infos = []
        for _ in range(args.steps):
            infos.append(step())
        e1.record(stream)
        torch.cuda.synchronize()
    launches = rte.kernel_launches() - launches0
    secs = e0.elapsed_time(e1) / 1e3
    iters = sum(i['iterations'] for i in infos)
    secs, total_units = aggregate(secs, dofs * iters, world)
    value = total_units / secs

    # ------------------------------------------------- per-kernel timing
    solver.timing(True)
    last_info = step()
    tim = solver.timing_read()
    solver.timing(False)
    d = dict(nRp=solver.n_nodes, nRm=solver.n_cells, nSp=solver.n_dirs,
             nSm=solver.n_odd)
    top = max(tim.items(), key=lambda kv: kv[1][0])
    peaks, src = load_peaks()
    d['e0_levels'] = levels_of(args.mesh)
    d['mesh'] = args.mesh
    d['dP'] = solver.d_plus
    work = kernel_work(top[0], d, p.nrhs, last_info)
    avg_ms = top[1][0] / max(top[1][1], 1)
    roof = dict(kernel=top[0], bound=None, achieved=None, peak=None, unit=None,
                frac=None, traffic=PROFILED_DRAM_BYTES.get(top[0]), launches=top[1][1],
                avg_ms=avg_ms)
    if work is not None:
        amount, unit, bound = work
        if unit == 'flop' and bound == 'fp64':
            peak = fp64_peak_tflops(torch)
            ach = amount / (avg_ms / 1e3) / 1e12
            roof.update(bound='alu', achieved=ach, peak=peak, unit='TFLOP/s',
                        frac=ach / peak, peak_source='measured cuBLAS FP64 GEMM in this run')
        elif unit == 'flop':
            ach = amount / (avg_ms / 1e3) / 1e12
            peak = peaks['bf16_tflops']
            roof.update(bound='tensor', achieved=ach, peak=peak, unit='TFLOP/s',
                        frac=ach / peak, peak_source=src + ' bf16 burst')
        else:
            ach = amount / (avg_ms / 1e3) / 1e9
            roof.update(bound=bound, achieved=ach, peak=peaks['hbm_gbs'], unit='GB/s',
                        frac=ach / peaks['hbm_gbs'], peak_source=src,
                        algorithmic_bytes=amount)
    share = {k: round(v[0] / sum(x[0] for x in tim.values()), 4)
             for k, v in tim.items()}

    # ------------------------------------------------------------- e2e
    qh = torch.tensor(p.q_nodal, dtype=torch.float64).pin_memory()
    uh = torch.empty((p.nrhs, solver.n_nodes, solver.n_dirs),
                     dtype=torch.float64).pin_memory()
    qd = torch.empty_like(qn)

    def e2e_step():
        qd.copy_(qh, non_blocking=True)
        solver.rhs(qd, out=q)
        u.zero_()
        _, info = solver.solve(q, u=u, tol=p.tol)
        uh.copy_(u, non_blocking=True)
        return info

    e2e_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    it_e2e = 0
    for _ in range(args.steps):
        it_e2e += e2e_step()['iterations']
    torch.cuda.synchronize()
    e2e_secs = time.perf_counter() - t0
    e2e = dict(value=dofs * it_e2e * world / e2e_secs, unit='DOF*iter/s',
               h2d_bytes_per_step=qh.numel() * 8,
               d2h_bytes_per_step=uh.numel() * 8,
               time_to_tol_s=e2e_secs / args.steps)

    fp64 = None
    if not args.no_fp64_compare and args.precision != 'fp64':
        s64 = rte.Solver(p, precision=rte.FP64)
        q64 = s64.rhs(qn)
        u64 = s64.even(p.nrhs)
        _, i64 = s64.solve(q64, u=u64, tol=p.tol)    # warm-up
        u64.zero_()
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(True), torch.cuda.Event(True)
        f0.record(s64.stream)
        _, i64 = s64.solve(q64, u=u64, tol=p.tol)
        f1.record(s64.stream)
        torch.cuda.synchronize()
        t64 = f0.elapsed_time(f1) / 1e3
        fp64 = dict(precision='fp64 (SIMT FP64 GEMMs, inner solves to 1e-12)',
                    time_to_tol_s=t64, iterations=i64['iterations'],
                    value=dofs * i64['iterations'] / t64, unit='DOF*iter/s',
                    mixed_speedup_time_to_tol=t64 / (secs / args.steps))
        s64.close()
    serving = None
    if rank == 0 and world == 1 and not args.no_serving:
        serving = serving_bench(args, torch, rte)
        if args.serve_sweep:
            serving['rate_sweep'] = serving_sweep(args, torch, rte,
                                                  serving['sequential_fp64_solves_per_s'])
    batch = None
    if rank == 0 and world == 1 and args.batch:
        batch = batch_bench(torch, rte)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(p)

    if rank == 0:
        out = dict(metric=METRIC, value=value, unit='DOF*iter/s', n_gpus=world,
                   steps=args.steps, warmup=args.warmup,
                   ms_per_step=secs * 1e3 / args.steps, higher_is_better=True,
                   scaling='weak', vs_baseline=None, dtype=args.precision.replace('mixed_', 'mixed-'),
                   data='synthetic',
                   config=dict(WORKLOAD, nrhs=p.nrhs, dofs=p.dofs,
                               precision=args.precision,
                               p1=('l PCG steps' if args.precision != 'fp64'
                                   else 'P_1^l Richardson steps'),
                               inner_tol=('E_0 0.3, E_c 0.1' if args.precision != 'fp64'
                                          else 'E_0 and E_c 1e-12'),
                               iterations_per_solve=iters / args.steps,
                               time_to_tol_s=secs / args.steps,
                               l2='inputs larger than L2: odd work arrays %d MB'
                                  % (d['nRm'] * d['nSm'] * 8 // 2 ** 20),
                               parallelism='replicas' if world > 1 else 'single'),
                   e2e=e2e, gpu_launches=launches, roofline=roof,
                   kernel_share=share, clocks=clk.summary(), cpu_baseline=cpu,
                   fp64_compare=fp64, serving=serving, setup_ms=setup_ms)
        if batch is not None:
            out['batch'] = batch
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()


def serving_requests(n, seed=0):
    """A seeded stream of solve requests mixing the sizes and parameters of
    the other workloads (plain 32x32/128-triangle problems, uneven instances
    with 32..64 meshes, 128 or 512 triangles, g in [0.3, 0.9], log-uniform
    sigma_t, sigma_s/sigma_t in [0.5, 0.999], 1..4 Gaussian sources)."""
    import numpy as np
    import workloads
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        kind = rng.integers(0, 3)
        if kind == 0:
            p = workloads.plain_fp64()
        else:
            p = workloads.batch_instances(1, seed=int(rng.integers(1 << 30)),
                                          m_range=(32, 64), levels=(2, 3),
                                          nrhs_range=(1, 4))[0]
        out.append(p)
    return out


def serving_bench(args, torch, rte):
    """Continuous batching: requests arrive as a Poisson stream (rate set to
    ~1.5x the measured sequential throughput, so the server must overlap
    them), are admitted by an HBM budget into worker slots, and their
    latencies (submission to completion) give p50/p99.  The same requests
    solved one after another in plain FP64 give the sequential baseline."""
    import numpy as np
    reqs = serving_requests(args.serve_requests, seed=1)
    free, total = torch.cuda.mem_get_info()
    budget = int(free * 0.6)
    opts = dict(precision=rte.MIXED_BF16)
    # sequential FP64 reference on a sample
    sample = reqs[:6]
    t0 = time.perf_counter()
    for p in sample:
        s = rte.Solver(p, max_rhs=p.nrhs)
        q = s.rhs(torch.tensor(p.q_nodal, dtype=torch.float64, device='cuda'))
        s.solve(q, tol=1e-6)
        torch.cuda.synchronize()
        s.close()
    seq_rate = len(sample) / (time.perf_counter() - t0)
    sv = rte.Server(budget, slots=8, **opts)
    # warm-up request
    sv.wait(sv.submit(reqs[0], reqs[0].q_nodal, tol=1e-6))
    rng = np.random.default_rng(2)
    rate = 1.5 * seq_rate
    arrivals = np.cumsum(rng.exponential(1.0 / rate, len(reqs)))
    t0 = time.perf_counter()
    ids = []
    for p, ta in zip(reqs, arrivals):
        delay = ta - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        ids.append(sv.submit(p, p.q_nodal, tol=1e-6))
    lat, iters = [], []
    for rid in ids:
        _, info = sv.wait(rid)
        lat.append(info['latency'])
        iters.append(info['iterations'])
    wall = time.perf_counter() - t0
    sv.close()
    lat = np.array(lat)
    return dict(requests=len(reqs), arrival_rate_per_s=rate, hbm_budget_bytes=budget, slots=8,
                precision='mixed_bf16', p50_latency_s=float(np.percentile(lat, 50)),
                p99_latency_s=float(np.percentile(lat, 99)), solves_per_s=len(reqs) / wall,
                sequential_fp64_solves_per_s=seq_rate,
                sequential_fp64_sample=len(sample), mean_iterations=float(np.mean(iters)))


def serving_sweep(args, torch, rte, seq_rate):
    """The serving stream at several arrival rates (multiples of the
    sequential FP64 rate): p50/p99 latency and served solves/s per rate,
    to show where latency saturates."""
    import numpy as np
    reqs = serving_requests(args.serve_requests, seed=3)
    free, _ = torch.cuda.mem_get_info()
    out = []
    for mult in (0.5, 1.0, 2.0, 4.0, 8.0):
        sv = rte.Server(int(free * 0.6), slots=8, precision=rte.MIXED_BF16)
        sv.wait(sv.submit(reqs[0], reqs[0].q_nodal, tol=1e-6))
        rate = mult * seq_rate
        arrivals = np.cumsum(np.random.default_rng(4).exponential(1.0 / rate, len(reqs)))
        t0 = time.perf_counter()
        ids = []
        for p, ta in zip(reqs, arrivals):
            delay = ta - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            ids.append(sv.submit(p, p.q_nodal, tol=1e-6))
        lat = np.array([sv.wait(rid)[1]['latency'] for rid in ids])
        wall = time.perf_counter() - t0
        sv.close()
        out.append(dict(rate_per_s=rate, rate_over_sequential_fp64=mult,
                        p50_latency_s=float(np.percentile(lat, 50)),
                        p99_latency_s=float(np.percentile(lat, 99)),
                        solves_per_s=len(reqs) / wall))
    return out


def batch_bench(torch, rte):
    """The batching workload: 64 uneven instances (meshes 32..128, 128 or
    512 triangles, 1-8 right-hand sides) submitted at once to the server
    (8 slots, mixed BF16, tol 1e-6); DOF*iter/s summed over all right-hand
    sides, against plain FP64 solves of a sample one after another."""
    import workloads
    insts = workloads.batch_instances(64, seed=0)
    free, _ = torch.cuda.mem_get_info()
    sv = rte.Server(int(free * 0.6), slots=8, precision=rte.MIXED_BF16)
    sv.wait(sv.submit(insts[0], insts[0].q_nodal, tol=1e-6))
    t0 = time.perf_counter()
    ids = [sv.submit(p, p.q_nodal, tol=1e-6) for p in insts]
    work = 0.0
    for p, rid in zip(insts, ids):
        _, info = sv.wait(rid)
        work += (p.m + 1) ** 2 * 4 ** (p.levels + 1) * p.nrhs * info['iterations']
    wall = time.perf_counter() - t0
    sv.close()
    sample = insts[:4]
    swork, t0 = 0.0, time.perf_counter()
    for p in sample:
        s = rte.Solver(p, max_rhs=p.nrhs)
        q = s.rhs(torch.tensor(p.q_nodal, dtype=torch.float64, device='cuda'))
        _, info = s.solve(q, tol=1e-6)
        torch.cuda.synchronize()
        s.close()
        swork += (p.m + 1) ** 2 * 4 ** (p.levels + 1) * p.nrhs * info['iterations']
    swall = time.perf_counter() - t0
    return dict(instances=len(insts), slots=8, precision='mixed_bf16', wall_s=wall,
                value=work / wall, unit='DOF*iter/s',
                sequential_fp64=dict(sample=len(sample), value=swork / swall,
                                     note='setup included, one solve after another'))


def cpu_baseline(p, budget_s=30.0):
    """The FP64 oracle, as it stands, timed on a bounded sample of the same
    workload.  One outer iteration costs (l+1) = 5 applications of E (the
    dominant dense work, timed once at full size) plus l = 4 applications of
    E_0^{-1} (n_S^+ sparse direction solves; 8 directions are timed after
    their factorisation and scaled to all n_S^+).  The coarse solve is left
    out, so the figure is an upper bound on the oracle's throughput."""
    import numpy as np
    import oracle
    t0 = time.perf_counter()
    disc = oracle.Discretisation(p.m, p.levels, p.sigma_t, p.sigma_s, p.g)
    ops = oracle.Operators(disc)
    t_setup = time.perf_counter() - t0
    x = np.random.default_rng(0).standard_normal((disc.nRp, disc.nSp))
    t0 = time.perf_counter()
    ops.apply_E(x)
    t_E = time.perf_counter() - t0
    e0 = ops.e0_blocks()
    ks = list(range(0, disc.nSp, max(1, disc.nSp // 8)))[:8]
    import scipy.sparse.linalg as spla
    for k in ks:
        e0['lu'][k] = spla.splu(e0['blocks'][k])
    t0 = time.perf_counter()
    for k in ks:
        e0['lu'][k].solve(x[:, k])
    t_E0 = (time.perf_counter() - t0) * disc.nSp / len(ks)
    t_iter = 5 * t_E + 4 * t_E0
    return dict(value=disc.nRp * disc.nSp / t_iter, unit='DOF*iter/s',
                cores=os.cpu_count(), kind='oracle',
                sample='1 full-size Apply-E (%.2f s) x5 + 8/%d E_0 direction '
                       'solves scaled x4 (%.2f s); coarse solve excluded; '
                       'assembly %.1f s not counted' % (t_E, disc.nSp, t_E0, t_setup))


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    import workloads
    p = workloads.checkerboard(m=128, levels=3, g=0.9, ratio=0.99, seed=0)
    vals = []
    cb = None
    for _ in range(args.warmup + args.steps):
        cb = cpu_baseline(p)
        vals.append(cb['value'])
    value = statistics.median(vals[args.warmup:]) if args.steps else vals[-1]
    cb['value'] = value
    out = dict(impl='reference', metric=METRIC, value=value, unit='DOF*iter/s',
               n_gpus=world, steps=args.steps, warmup=args.warmup,
               ms_per_step=None, higher_is_better=True, scaling='weak',
               vs_baseline=None, dtype='f64', data='synthetic',
               config=dict(WORKLOAD, precision='fp64'), cpu_baseline=cb,
               e2e=dict(value=value, unit='DOF*iter/s', h2d_bytes_per_step=0,
                        d2h_bytes_per_step=0))
    print(json.dumps(out))


if __name__ == '__main__':
    a = parse()
    if a.impl == 'reference':
        run_reference(a)
    else:
        run_ours(a)
