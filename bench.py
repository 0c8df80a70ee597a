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
    ap.add_argument('--precision', default='fp64',
                    choices=['fp64', 'mixed_fp32', 'mixed_bf16'])
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


def kernel_work(name, d, nrhs):
    """Algorithmic work per launch of a named kernel group: (amount, unit,
    bound).  FP64 GEMMs count 2 M N K flops; HBM-bound kernels count the
    bytes they must read and write once."""
    nRp, nRm, nS, nSm = d['nRp'], d['nRm'], d['nSp'], d['nSm']
    if name in ('gemm_mk_eig1', 'gemm_mk_eig2'):
        return 2.0 * nrhs * nRm * nSm * nSm, 'flop', 'alu'
    if name == 'gemm_kplus':
        return 2.0 * nrhs * nRp * nS * nS, 'flop', 'alu'
    if name == 'transport_A':
        return 8.0 * nrhs * (nRp * nS + nRm * nSm), 'byte', 'hbm'
    if name == 'apply_even':
        return 8.0 * nrhs * (nRm * nSm + 3 * nRp * nS), 'byte', 'hbm'
    return None


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
    p = workloads.checkerboard(m=128, levels=3, g=0.9, ratio=0.99, seed=rank)
    solver = rte.Solver(p, precision=prec)
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
    step()
    tim = solver.timing_read()
    solver.timing(False)
    d = dict(nRp=solver.n_nodes, nRm=solver.n_cells, nSp=solver.n_dirs,
             nSm=solver.n_odd)
    top = max(tim.items(), key=lambda kv: kv[1][0])
    peaks, src = load_peaks()
    roof = None
    work = kernel_work(top[0], d, p.nrhs)
    avg_ms = top[1][0] / max(top[1][1], 1)
    if work is not None:
        amount, unit, bound = work
        if unit == 'flop':
            peak = fp64_peak_tflops(torch)
            ach = amount / (avg_ms / 1e3) / 1e12
            roof = dict(kernel=top[0], bound=bound, achieved=ach, peak=peak,
                        unit='TFLOP/s', frac=ach / peak, traffic=None,
                        peak_source='measured cuBLAS FP64 GEMM in this run')
        else:
            ach = amount / (avg_ms / 1e3) / 1e9
            roof = dict(kernel=top[0], bound=bound, achieved=ach,
                        peak=peaks['hbm_gbs'], unit='GB/s',
                        frac=ach / peaks['hbm_gbs'], traffic=None,
                        peak_source=src)
    else:
        roof = dict(kernel=top[0], bound='hbm', achieved=None, peak=None,
                    unit=None, frac=None, traffic=None)
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

    cpu = None
    if rank == 0 and world == 1:
        cpu = cpu_baseline(p)

    if rank == 0:
        out = dict(metric=METRIC, value=value, unit='DOF*iter/s', n_gpus=world,
                   steps=args.steps, warmup=args.warmup,
                   ms_per_step=secs * 1e3 / args.steps, higher_is_better=True,
                   scaling='weak', vs_baseline=None, dtype=args.precision.replace('mixed_', 'mixed-'),
                   data='synthetic',
                   config=dict(WORKLOAD, nrhs=p.nrhs, dofs=p.dofs,
                               precision=args.precision,
                               iterations_per_solve=iters / args.steps,
                               time_to_tol_s=secs / args.steps,
                               l2='inputs larger than L2: odd work arrays %d MB'
                                  % (d['nRm'] * d['nSm'] * 8 // 2 ** 20),
                               parallelism='replicas' if world > 1 else 'single'),
                   e2e=e2e, gpu_launches=launches, roofline=roof,
                   kernel_share=share, clocks=clk.summary(), cpu_baseline=cpu)
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()


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
