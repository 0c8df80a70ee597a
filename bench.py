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
    ap.add_argument('--serve-requests', type=int, default=64)
    ap.add_argument('--serve-sweep', action='store_true',
                    help='also sweep the arrival rate of the serving stream (minutes)')
    ap.add_argument('--batch', action='store_true',
                    help='also time the 64 uneven instances of the batching workload')
    ap.add_argument('--mk-routes', action='store_true',
                    help='time the eigenbasis and the PCG (Algorithm 1) routes of '
                         '(M^- - K^-)^{-1} on the 128x128 and 96x96 workloads and exit')
    ap.add_argument('--params', action='store_true',
                    help='time to 1e-6 on the benchmark workload (mixed BF16) over the method '
                         'parameters N^+, l and the coarse tolerance, and exit')
    ap.add_argument('--h2', action='store_true',
                    help='time the H^2-compressed S^+ apply against the dense products over '
                         'n_S^+ = 1024 .. 65536 (the paper\'s compression table) and exit')
    ap.add_argument('--h2-rows', type=int, default=2048,
                    help='row vectors of the --h2 study (spatial nodes times right-hand sides)')
    ap.add_argument('--h2-levels', default='4,5,6,7')
    ap.add_argument('--rates', action='store_true',
                    help='print the contraction rates rho and eta of the iteration matrix '
                         'over g, d_N and l (the paper\'s Section 6.2 study) and exit')
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


# DRAM traffic of a timing scope's kernel from an ncu launch list of this
# benchmark's own workload (`bench.py --profile-once`; the summary and the
# command are in profiles/launches_checkerboard_128x128_T512_mixed_bf16.md):
# dram__bytes_read.sum + dram__bytes_write.sum averaged over the kernel's
# launches in one solve, the source file the kernel lives in and that file's
# SHA-256 prefix at the capture.  The bench reports it only for the workload
# it was captured on, and null once the source has changed since.
PROFILED_DRAM = {
    'coarse_cg': dict(source='paper_2102_09038_gb300/csrc/mg.cu', sha='e29a65ac179f3b0b',
                      workload='checkerboard_128x128_T512_g0.90_c0.99',
                      bytes_per_launch=1.829e9, coarse_iters=5,
                      note='ncu launch list, 16 launches of k_ec_pcg<0> in one solve '
                           '(5 CG iterations each)'),
    'e0_direct': dict(source='paper_2102_09038_gb300/csrc/e0_direct.cu', sha='170f9aa09a001022',
                      workload='checkerboard_128x128_T512_g0.90_c0.99',
                      bytes_per_launch=4.736e9,
                      note='ncu launch list, 32 launches of k_e0_direct_tma in one solve'),
}


def source_sha(rel):
    import hashlib
    with open(os.path.join(ROOT, rel), 'rb') as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def e0_units(d, nrhs, info):
    """Work units of one E_0^{-1} launch: (node, column) items times the
    launch's CG iterations, each weighted by the fraction of direction quads
    still active (the mixed-mode kernel visits only those)."""
    n = info.get('e0_launches', 0)
    per = info['e0_active_vcycles'] / n if n else max(info.get('e0_iters', 1), 1)
    return d['nRp'] * nrhs * d['nSp'] * per, per


def split_slices_for(tol, smax=7):
    """Digit slices the library's split FP64 GEMMs use for a solve to `tol`:
    the smallest S >= 3 with S 2^-7S <= tol / 1000, at most the slices set up."""
    for S in range(3, smax):
        if S * 2.0 ** (-7 * S) <= tol / 1000.0:
            return S
    return smax


def kernel_work(name, d, nrhs, info, tol=None):
    """Algorithmic work of one launch of a named kernel group, as the
    per-unit counts of the measurement plan (work per outer iteration of the
    method: flops of the dense contractions, bytes each memory-bound step
    must move at least once): (amount, unit, bound).
      * contractions: 2 M N K flops;
      * split FP64 contractions: the BF16 products of the S(S+1)/2 digit
        slice pairs, 2 M N K each (S as the library takes it from the
        solve's tolerance);
      * transport A: read U^+, write Z (w = 8 B);
      * A^T + M^+ + R - K^+ gather: read Z, U^+ and U S^+, write Y;
      * E_0 direct (the default route): its factor read twice (the forward
        and the backward sweep), 2 n_S^+ (m+1)^3 w bytes (w = 4 FP32, 8
        FP64), plus the FP64 right-hand side read and solution written;
      * E_0 PCG: per CG iteration over all (node, column) items the four CG
        streams x, r, p, Ap read and written once, w 6 N^+ s bytes (w = 4 in
        the FP32 kernel, 8 in FP64), plus the stencil at its minimal size
        (six spatial parts of 7 coefficients per node, the per-direction
        weights being negligible), times the launch's CG iterations (the
        V-cycles, each weighted by the fraction of active direction quads),
        plus the FP64 right-hand side read and solution written once;
      * E_c PCG: per CG iteration w (5 d N^+) of vectors plus the E_c stencil
        as the CG's own apply reads it (7 d^2 N^+), w = 8, times the CG
        iterations."""
    nRp, nRm, nS, nSm = d['nRp'], d['nRm'], d['nSp'], d['nSm']
    if name in ('gemm_mk_eig1', 'gemm_mk_eig2'):
        return 2.0 * nrhs * nRm * nSm * nSm, 'flop', 'fp64'
    if name in ('tc_gemm_mk1', 'tc_gemm_mk2'):
        return 2.0 * nrhs * nRm * nSm * nSm, 'flop', 'tensor'
    if name == 'gemm_kplus':
        return 2.0 * nrhs * nRp * nS * nS, 'flop', 'fp64'
    if name in ('dgemm_split_mk1', 'dgemm_split_mk2', 'dgemm_split_kplus') and tol:
        S = split_slices_for(tol)
        pairs = S * (S + 1) // 2
        if name == 'dgemm_split_kplus':
            return pairs * 2.0 * nrhs * nRp * nS * nS, 'flop', 'tensor'
        return pairs * 2.0 * nrhs * nRm * nSm * nSm, 'flop', 'tensor'
    if name == 'transport_A':
        return 8.0 * nrhs * (nRp * nS + nRm * nSm), 'byte', 'hbm'
    if name == 'apply_even':
        return 8.0 * nrhs * (nRm * nSm + 3 * nRp * nS), 'byte', 'hbm'
    if name in ('e0_cg', 'e0_cg_lo'):
        w = 8 if name == 'e0_cg' else 4
        _, per = e0_units(d, nrhs, info)
        it = w * 6 * nRp * nrhs * nS + 6 * 7 * nRp * w
        return it * per + 16.0 * nRp * nrhs * nS, 'byte', 'hbm'
    if name == 'coarse_cg':
        dp = d['dP']
        it = 8 * (5 * dp * nRp * nrhs + 7 * dp * dp * nRp)
        return it * max(info.get('coarse_iters', 1), 1), 'byte', 'hbm'
    if name in ('e0_direct', 'e0_direct64'):
        w = 8 if name == 'e0_direct64' else 4
        b = d['mesh'] + 1
        return 2.0 * nS * b * b * b * w + 16.0 * nRp * nrhs * nS, 'byte', 'hbm'
    return None


def roofline_of(name, total_ms, launches, d, nrhs, info, peaks, src, fp64_peak, tol=None):
    """Roofline of one timing scope: the algorithmic work of one launch
    (kernel_work) over the scope's mean launch time, against the measured
    peak of its bound; fp64_peak() gives the measured FP64 rate (timed only
    when a scope needs it)."""
    avg_ms = total_ms / max(launches, 1)
    roof = dict(kernel=name, bound=None, achieved=None, peak=None, unit=None, frac=None,
                launches=launches, avg_ms=avg_ms)
    work = kernel_work(name, d, nrhs, info, tol)
    if work is None:
        return roof
    amount, unit, bound = work
    if unit == 'flop' and bound == 'fp64':
        peak = fp64_peak()
        ach = amount / (avg_ms / 1e3) / 1e12
        roof.update(bound='alu', achieved=ach, peak=peak, unit='TFLOP/s',
                    frac=ach / peak, peak_source='measured cuBLAS FP64 GEMM in this run')
    elif unit == 'flop':
        ach = amount / (avg_ms / 1e3) / 1e12
        peak = peaks['bf16_tflops']
        roof.update(bound='tensor', achieved=ach, peak=peak, unit='TFLOP/s',
                    frac=ach / peak, peak_source=src + ' bf16 burst', algorithmic_flops=amount)
    else:
        ach = amount / (avg_ms / 1e3) / 1e9
        roof.update(bound=bound, achieved=ach, peak=peaks['hbm_gbs'], unit='GB/s',
                    frac=ach / peaks['hbm_gbs'], peak_source=src,
                    algorithmic_bytes=amount)
        impl = kernel_impl_bytes(name, d, nrhs, info)
        if impl is not None:
            roof.update(impl_bytes=impl,
                        impl_frac=impl / (avg_ms / 1e3) / 1e9 / peaks['hbm_gbs'])
    return roof


def scope_rooflines(tim, d, nrhs, info, peaks, src, fp64_peak, tol, count=4):
    """The roofline of the largest timing scope and those of the `count`
    largest ({scope: (total ms, launches)} as the library's timing reports
    it), each against its own bound."""
    ranked = sorted(tim.items(), key=lambda kv: -kv[1][0])
    top = ranked[0]
    roof = roofline_of(top[0], top[1][0], top[1][1], d, nrhs, info, peaks, src, fp64_peak, tol)
    rooflines = [roofline_of(k, v[0], v[1], d, nrhs, info, peaks, src, fp64_peak, tol)
                 for k, v in ranked[:count]]
    return roof, rooflines


def kernel_impl_bytes(name, d, nrhs, info):
    """The bytes the E_0 kernels move by their own design, per launch (kept
    beside the algorithmic count): per V-cycle and active (node, column) the
    12 CG-vector passes of the precision w and the iterate read and written,
    the V-cycle's 17 FP32 array passes per level (4^-l of the level-0 size)
    and the coarsest level's dense per-direction inverses, plus the FP64
    right-hand side and solution once."""
    nRp, nS = d['nRp'], d['nSp']
    if name in ('e0_direct', 'e0_direct64'):
        # the factor rows padded to ld (a multiple of 4), read twice per
        # sweep of up to 4 right-hand sides; B read, the forward result
        # written, read and overwritten; four coupling coefficients per item
        w = 8 if name == 'e0_direct64' else 4
        b = d['mesh'] + 1
        ld = (b + 3) // 4 * 4
        sweeps = (nrhs + 3) // 4
        return (2.0 * nS * b * ld * ld * w * sweeps + 32.0 * nRp * nrhs * nS
                + 4 * 8.0 * nRp * nS * sweeps)
    if name not in ('e0_cg', 'e0_cg_lo'):
        return None
    w = 8 if name == 'e0_cg' else 4
    cols = nrhs * nS
    cg = nRp * cols * (12 * w + 2 * w + (7 * 8 if name == 'e0_cg' else 0))
    vc = sum(nRp / 4 ** l * cols * 4 * 17 for l in range(d['e0_levels']))
    mc = d['mesh'] >> (d['e0_levels'] - 1)
    vc += ((mc + 1) ** 2) ** 2 * nS * 4
    _, per = e0_units(d, nrhs, info)
    return (cg + vc) * per + nRp * cols * 16


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
    ranked = sorted(tim.items(), key=lambda kv: -kv[1][0])
    top = ranked[0]
    peaks, src = load_peaks()
    d['e0_levels'] = levels_of(args.mesh)
    d['mesh'] = args.mesh
    d['dP'] = solver.d_plus
    traffic, traffic_note = None, 'no ncu capture of the current kernel source'
    prof = PROFILED_DRAM.get(top[0])
    if prof:
        if source_sha(prof['source']) != prof['sha']:
            traffic_note = 'kernel changed since its ncu capture'
        elif (prof['workload'] != WORKLOAD['workload'] or args.mesh != WORKLOAD['mesh']
              or 8 * 4 ** args.levels != WORKLOAD['sphere_triangles']):
            traffic_note = 'ncu capture taken on another workload'
        elif prof.get('coarse_iters') not in (None, last_info.get('coarse_iters')):
            traffic_note = 'ncu capture taken at another coarse iteration count'
        else:
            traffic = prof['bytes_per_launch']
            traffic_note = prof['note']
    fp64_rate = []

    def fp64_peak():
        if not fp64_rate:
            fp64_rate.append(fp64_peak_tflops(torch))
        return fp64_rate[0]

    roof, rooflines = scope_rooflines(tim, d, p.nrhs, last_info, peaks, src, fp64_peak, p.tol)
    roof.update(traffic=traffic, traffic_source=traffic_note)
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

    arms = None
    if not args.no_fp64_compare and args.precision != 'fp64':
        arms = precision_arms(rte, torch, p, qn, secs / args.steps, iters / args.steps, u, dofs)
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
                               p1=('2 PCG steps' if args.precision != 'fp64'
                                   else 'P_1^l Richardson steps'),
                               inner_tol=('E_0 0.3, E_c 0.3' if args.precision != 'fp64'
                                          else 'E_0 and E_c 1e-12'),
                               iterations_per_solve=iters / args.steps,
                               e0_route=('direct' if 'e0_direct' in tim or 'e0_direct64' in tim
                                         else 'multigrid'),
                               coarse_cg_iterations_last=last_info.get('coarse_iters'),
                               time_to_tol_s=secs / args.steps,
                               l2='inputs larger than L2: odd work arrays %d MB'
                                  % (d['nRm'] * d['nSm'] * 8 // 2 ** 20),
                               parallelism='replicas' if world > 1 else 'single'),
                   e2e=e2e, gpu_launches=launches, roofline=roof, rooflines=rooflines,
                   kernel_share=share, clocks=clk.summary(), cpu_baseline=cpu,
                   serving=serving, setup_ms=setup_ms)
        if arms is not None:
            out.update(arms)
        if batch is not None:
            out['batch'] = batch
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()


# The FP64 arm with the mixed arm's algorithm: P_1 as PCG steps, inner
# tolerances 0.3 (E_0) and 0.1 (E_c), and the FP64 dense contractions on the
# split (FP64-accurate) tensor-core GEMM; only the arithmetic of the inner
# steps differs from the mixed modes.
FP64_MATCHED = dict(precision=0, dgemm=2, p1_route=1, e0_tol=0.3, coarse_tol=0.3)


def timed_solve(solver, q, tol, warm=True):
    """(seconds, info, u) of one solve from u = 0, device-timed with CUDA
    events on the solver's stream (after one untimed solve when warm)."""
    import torch
    u = solver.even(q.shape[0])
    if warm:
        solver.solve(q, u=u, tol=tol)
        u.zero_()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
    e0.record(solver.stream)
    _, info = solver.solve(q, u=u, tol=tol)
    e1.record(solver.stream)
    torch.cuda.synchronize()
    if info['status'] != 0:
        raise RuntimeError('solve failed: %s' % info)
    return e0.elapsed_time(e1) / 1e3, info, u


def precision_arms(rte, torch, p, qn, t_mixed, it_mixed, u_mixed, dofs):
    """The other precisions on the same workload and tolerance, each a full
    solve timed like the headline: FP32 mixed; FP64 with the mixed arm's
    algorithm (so that the ratio to it is the speed-up from precision
    alone); FP64 as the paper states the method (P_1^l, inner solves to
    1e-12, FP64 GEMMs on the FP64 units; the ratio of the two FP64 arms is
    the speed-up from the algorithm's inner tolerances and P_1 route).  The
    error of each solution against an FP64 reference solved to 1e-11 (the
    matched FP64 arm) is reported beside it."""
    ref = rte.Solver(p, **FP64_MATCHED)
    qr = ref.rhs(qn)
    _, iref, uref = timed_solve(ref, qr, 1e-11, warm=False)
    ref.close()
    uref = uref.cpu().numpy()
    import numpy as np

    def err(u):
        return float(np.linalg.norm(u.cpu().numpy() - uref) / np.linalg.norm(uref))

    out = dict(error_vs_fp64=dict(
        reference='FP64 solve (matched algorithm) to relative residual 1e-11',
        reference_residual=iref['rel_residual'], reference_iterations=iref['iterations'],
        tol=p.tol, mixed_bf16=err(u_mixed)))
    arms = {}
    for name, opts in (('mixed_fp32', dict(precision=rte.MIXED_FP32)),
                       ('fp64_matched', FP64_MATCHED),
                       ('fp64_paper', dict(precision=rte.FP64))):
        s = rte.Solver(p, **opts)
        q = s.rhs(qn)
        t, info, u = timed_solve(s, q, p.tol, warm=name != 'fp64_paper')
        out['error_vs_fp64'][name] = err(u)
        arms[name] = dict(time_to_tol_s=t, iterations=info['iterations'],
                          value=dofs * info['iterations'] / t, unit='DOF*iter/s')
        s.close()
    arms['fp64_matched']['note'] = ('P_1 as 2 PCG steps, inner tolerances 0.3 / 0.3, split '
                                    'FP64 tensor-core GEMMs: the mixed arm\'s algorithm in FP64')
    arms['fp64_paper']['note'] = ('P_1^l, inner solves to 1e-12, FP64 GEMMs on the FP64 '
                                  'units: the method as the paper states it')
    out['precision_arms'] = arms
    out['speedup'] = dict(
        precision=arms['fp64_matched']['time_to_tol_s'] / t_mixed,
        algorithm=arms['fp64_paper']['time_to_tol_s'] / arms['fp64_matched']['time_to_tol_s'],
        total_vs_fp64_paper=arms['fp64_paper']['time_to_tol_s'] / t_mixed,
        fp32_vs_bf16=arms['mixed_fp32']['time_to_tol_s'] / t_mixed,
        note='ratios of time to tolerance; precision = FP64 (matched) / mixed BF16')
    return out


def serving_requests(n, seed=0):
    """A seeded stream of solve requests mixing the sizes and parameters of
    the other workloads: the plain 32x32 / 128-triangle problem (g = 0.5);
    the 128x128 / 512-triangle checkerboard (g = 0.9, c = 0.99) with a
    seeded Gaussian source per request; the 96x96 / 2048-triangle
    precision case (g = 0.8 or 0.95, c = 0.999); and uneven instances of
    the batching workload (meshes 32..128, 128 or 512 triangles, g in
    [0.3, 0.9], log-uniform sigma_t, sigma_s / sigma_t in [0.5, 0.999], 1..8
    Gaussian sources)."""
    import numpy as np
    import workloads
    rng = np.random.default_rng(seed)
    out = []
    for kind in rng.choice(4, size=n, p=[0.4, 0.2, 0.1, 0.3]):
        if kind == 0:
            p = workloads.plain_fp64()
        elif kind == 1:
            p = workloads.checkerboard(m=128, levels=3, g=0.9, ratio=0.99,
                                       seed=int(rng.integers(1 << 30)))
        elif kind == 2:
            p = workloads.precision_case(g=float(rng.choice([0.8, 0.95])))
        else:
            p = workloads.batch_instances(1, seed=int(rng.integers(1 << 30)))[0]
        out.append(p)
    return out


def run_stream(rte, reqs, rate, budget, slots, opts, seed):
    """Poisson arrivals at `rate` per second into a fresh server: (latencies,
    iterations, wall seconds, cache hits, misses)."""
    import numpy as np
    sv = rte.Server(budget, slots=slots, **opts)
    arrivals = np.cumsum(np.random.default_rng(seed).exponential(1.0 / rate, len(reqs)))
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
    hits, misses, _ = sv.cache_stats()
    sv.close()
    return np.array(lat), iters, wall, hits, misses


def serving_bench(args, torch, rte):
    """Continuous batching: requests arrive as a Poisson stream, are admitted
    by an HBM budget into 8 worker slots (each request's set-up is skipped
    when the server holds an idle handle of its operator), and their
    latencies (submission to completion) give p50/p99.  Baseline: the
    same requests one after another in FP64 with the same algorithm (the
    matched FP64 arm: no server, no cache, every request set up), on a
    sample bounded to about 30 s."""
    import numpy as np
    reqs = serving_requests(args.serve_requests, seed=1)
    free, total = torch.cuda.mem_get_info()
    budget = int(free * 0.6)
    opts = dict(precision=rte.MIXED_BF16)
    n_seq, t_seq = 0, 0.0
    t0 = time.perf_counter()
    for p in reqs:
        s = rte.Solver(p, max_rhs=p.nrhs, **FP64_MATCHED)
        q = s.rhs(torch.tensor(p.q_nodal, dtype=torch.float64, device='cuda'))
        s.solve(q, tol=1e-6)
        torch.cuda.synchronize()
        s.close()
        n_seq += 1
        t_seq = time.perf_counter() - t0
        if t_seq > 30.0:
            break
    seq_rate = n_seq / t_seq
    # warm-up of the server path (first-use initialisation of the libraries)
    run_stream(rte, reqs[:2], 100.0, budget, 8, opts, 0)
    rate = 1.5 * seq_rate
    lat, iters, wall, hits, misses = run_stream(rte, reqs, rate, budget, 8, opts, 2)
    kinds = ['instance' if p.name.startswith('inst') else p.name.split('_')[0] for p in reqs]
    return dict(requests=len(reqs), mix={k: kinds.count(k) for k in sorted(set(kinds))},
                arrival_rate_per_s=rate, hbm_budget_bytes=budget, slots=8,
                precision='mixed_bf16', p50_latency_s=float(np.percentile(lat, 50)),
                p99_latency_s=float(np.percentile(lat, 99)), solves_per_s=len(reqs) / wall,
                operator_cache=dict(hits=hits, misses=misses),
                sequential_fp64_solves_per_s=seq_rate, sequential_fp64_sample=n_seq,
                mean_iterations=float(np.mean(iters)))


def serving_sweep(args, torch, rte, seq_rate):
    """The serving stream at several arrival rates (multiples of the
    sequential FP64 rate): p50/p99 latency and served solves/s per rate,
    to show where latency saturates."""
    import numpy as np
    reqs = serving_requests(args.serve_requests, seed=3)
    free, _ = torch.cuda.mem_get_info()
    out = []
    for mult in (1.0, 2.0, 4.0, 8.0):
        lat, _, wall, hits, misses = run_stream(rte, reqs, mult * seq_rate, int(free * 0.6), 8,
                                                dict(precision=rte.MIXED_BF16), 4)
        out.append(dict(rate_per_s=mult * seq_rate, rate_over_sequential_fp64=mult,
                        p50_latency_s=float(np.percentile(lat, 50)),
                        p99_latency_s=float(np.percentile(lat, 99)),
                        solves_per_s=len(reqs) / wall, cache_hits=hits))
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
        s = rte.Solver(p, max_rhs=p.nrhs, **FP64_MATCHED)
        q = s.rhs(torch.tensor(p.q_nodal, dtype=torch.float64, device='cuda'))
        _, info = s.solve(q, tol=1e-6)
        torch.cuda.synchronize()
        s.close()
        swork += (p.m + 1) ** 2 * 4 ** (p.levels + 1) * p.nrhs * info['iterations']
    swall = time.perf_counter() - t0
    return dict(instances=len(insts), slots=8, precision='mixed_bf16', wall_s=wall,
                value=work / wall, unit='DOF*iter/s',
                sequential_fp64=dict(sample=len(sample), value=swork / swall,
                                     note='matched FP64 arm, setup included, one solve '
                                          'after another'))


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


def mk_routes_study(args):
    """Time to 1e-6 with each route of (M^- - K^-)^{-1}: the full
    eigenbasis (two dense contractions per apply, the default) and the
    paper's Algorithm 1 (PCG with the Lemma's preconditioner to 1e-12, run
    as a device-side graph loop), in the matched FP64 arm (split
    tensor-core GEMMs) and in mixed BF16 (where the PCG route applies to the
    FP64 residual), on the 128 x 128 / 512-triangle checkerboard and the
    96 x 96 / 2048-triangle precision case at g = 0.8."""
    import torch
    import workloads
    import paper_2102_09038_gb300 as rte
    torch.cuda.set_device(0)
    cases = [('checkerboard_128x128_T512', workloads.checkerboard(m=128, levels=3, g=0.9,
                                                                  ratio=0.99, seed=0)),
             ('precision_96x96_T2048_g0.80', workloads.precision_case(g=0.8))]
    out = []
    for name, p in cases:
        qn = torch.tensor(p.q_nodal, dtype=torch.float64, device='cuda')
        for arm, opts in (('fp64_matched', FP64_MATCHED), ('mixed_bf16', dict(precision=2))):
            for route in (rte.MK_EIGEN, rte.MK_PCG):
                s = rte.Solver(p, mk_route=route, **opts)
                t, info, _ = timed_solve(s, s.rhs(qn), p.tol)
                s.close()
                row = dict(case=name, arm=arm, route=('eigenbasis', 'pcg')[route],
                           time_to_tol_s=t, iterations=info['iterations'],
                           mk_iters_last=info['mk_iters'])
                out.append(row)
                print(json.dumps(row), flush=True)
    return out


def params_study(args):
    """Time to 1e-6 in mixed BF16 over the method's parameters: the degree
    N^+ of the subspace correction (d^+ = 1, 6, 15), the steps l of P_1 and
    the tolerance of the coarse CG, on the benchmark workload (128 x 128 mesh,
    512 triangles, g = 0.9, c = 0.99) and, for N^+ = 4, on the 96 x 96 /
    2048-triangle precision cases (g = 0.8 and 0.95, c = 0.999).  Each solve
    from u = 0, CUDA-event timed after one untimed solve; the residual is the
    library's FP64 one."""
    import torch
    import workloads
    import paper_2102_09038_gb300 as rte
    torch.cuda.set_device(0)
    cases = [('checkerboard_128x128_T512',
              workloads.checkerboard(m=args.mesh, levels=args.levels, g=0.9, ratio=0.99, seed=0),
              [(n, l, c) for n in (0, 2, 4) for l in (1, 2, 3, 4, 6) for c in (0.1, 0.3, 0.5)]),
             ('precision_96x96_T2048_g0.80', workloads.precision_case(g=0.8),
              [(4, l, c) for l in (1, 2, 4) for c in (0.1, 0.3)]),
             ('precision_96x96_T2048_g0.95', workloads.precision_case(g=0.95),
              [(4, l, c) for l in (1, 2, 4) for c in (0.1, 0.3)])]
    out = []
    for name, p, grid in cases:
        qn = torch.tensor(p.q_nodal, dtype=torch.float64, device='cuda')
        for n_plus, l, ctol in grid:
            s = rte.Solver(p, precision=rte.MIXED_BF16, n_plus=n_plus, l=l, coarse_tol=ctol,
                           max_iter=400)
            try:
                t, info, _ = timed_solve(s, s.rhs(qn), p.tol)
                row = dict(case=name, n_plus=n_plus, d_plus=s.d_plus, l=l, coarse_tol=ctol,
                           time_to_tol_s=t, iterations=info['iterations'],
                           coarse_iters_last=info['coarse_iters'],
                           rel_residual=info['rel_residual'])
            except RuntimeError as e:
                row = dict(case=name, n_plus=n_plus, l=l, coarse_tol=ctol, failed=str(e)[:100])
            s.close()
            out.append(row)
            print(json.dumps(row), flush=True)
    return out


def h2_study(args):
    """Dense against H^2-compressed S^+ (Section 5.2; the compression table
    of Section 6): for n_S^+ = 4 * 4^levels, g = 0.5 and the paper's
    eta = 1.4, p = 4, the set-up time and device bytes of the H^2 matrices and
    the time of Y = X S^+ for R row vectors (CUDA events on the handle's
    stream, after a warm-up apply; inputs far larger than L2), in FP64 and
    FP32, beside the dense products the solver uses for the same Y: the
    split FP64 tensor-core GEMM and the BF16 tcgen05 GEMM, with a dense S^+ of
    the same size (random values: their time does not depend on them).
    The H^2 apply's flops count every 64 x 64 block product it performs
    (leaf and transfer matrices, couplings, near blocks)."""
    import torch
    import paper_2102_09038_gb300 as rte
    torch.cuda.set_device(0)
    R = args.h2_rows
    fp64_peak = fp64_peak_tflops(torch)
    peaks, _ = load_peaks()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    # FP32 SIMT peak: 128 FP32 lanes per SM, 2 flops per FMA, at the SM clock
    # the run sees (sampled below)
    out = []
    for levels in [int(v) for v in args.h2_levels.split(',')]:
        h = rte.H2Scattering(levels, 0.5, parities=1)
        inf = h.info()
        n = inf['n_plus']
        gen = torch.Generator(device='cuda').manual_seed(levels)
        X = torch.randn((R, n), dtype=torch.float64, device='cuda', generator=gen)
        st = h.stream
        blocks = (2 * inf['leaves'] + 2 * inf['transfers'] + sum(inf['far_blocks'])
                  + inf['near_matrices'])
        flops = 2.0 * R * 64 * 64 * blocks

        def timed(fn, reps=3):
            fn()
            e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
            st.synchronize()
            e0.record(st)
            for _ in range(reps):
                fn()
            e1.record(st)
            e1.synchronize()
            return e0.elapsed_time(e1) / 1e3 / reps

        with Clocks(0) as clk:
            t64 = timed(lambda: h.apply(X, precision=rte.FP64), reps=2)
            t32 = timed(lambda: h.apply(X, precision=rte.MIXED_FP32))
            tbf = timed(lambda: h.apply(X, precision=rte.MIXED_BF16))
        mhz = clk.summary().get('sm_mhz') or 2070.0
        fp32_peak = sms * 128 * 2 * mhz * 1e6 / 1e12
        row = dict(levels=levels, n_plus=n, rows=R, h2_setup_s=inf['setup_ms'] / 1e3,
                   h2_bytes=inf['bytes'], far_blocks=inf['far_blocks'],
                   near_matrices=inf['near_matrices'], block_products=blocks,
                   h2_fp64_s=t64, h2_fp32_s=t32,
                   h2_fp64_tflops=flops / t64 / 1e12, h2_fp64_frac=flops / t64 / 1e12 / fp64_peak,
                   h2_fp32_tflops=flops / t32 / 1e12, h2_fp32_frac=flops / t32 / 1e12 / fp32_peak,
                   h2_bf16_s=tbf, h2_bf16_tflops=flops / tbf / 1e12,
                   h2_bf16_frac=flops / tbf / 1e12 / peaks['bf16_tflops'],
                   fp64_peak_tflops=fp64_peak, fp32_simt_peak_tflops=fp32_peak,
                   dense_bytes_fp64=8 * n * n)
        h.close()
        del X
        torch.cuda.empty_cache()
        # dense products of the same Y = X S (S symmetric: Bt = S)
        try:
            S = torch.randn((n, n), dtype=torch.float64, device='cuda', generator=gen)
            Xd = torch.randn((R, n), dtype=torch.float64, device='cuda', generator=gen)
            row['dense_split_fp64_s'] = timed(lambda: rte.dgemm_split(Xd, S, slices=5), reps=2)
            Sb, Xb = S.to(torch.bfloat16), Xd.to(torch.bfloat16)
            del S, Xd
            row['dense_bf16_s'] = timed(lambda: rte.gemm_lowp(Xb, Sb))
            del Sb, Xb
        except (RuntimeError, rte.RteError) as e:
            row['dense_note'] = str(e).splitlines()[0][:120]
        torch.cuda.empty_cache()
        out.append(row)
        print(json.dumps(row), flush=True)
    return out


def rates_study(args):
    """rho (spectral radius) and eta (energy norm) of Algorithm 3's
    iteration matrix (I - P_G)(I - P_1^l (E - K^+)) by power iteration on the
    library's FP64 operators (rte_rates), over the anisotropy g, the
    subspace dimension d_N (N^+ = 0, 2, 4: d = 1, 6, 15) and the steps l of
    P_1^l: the study of the paper's Section 6.2 (Tables 3-7) on a synthetic
    geometry, since the paper's lattice layout is not reproducible.  The
    geometry: the unit square, 24 x 24 mesh, 4 x 4 checkerboard of
    sigma_t in {1, 10} with sigma_s = 0.999 sigma_t (c = 0.999, the
    paper's strongly scattering regime), 256 even directions."""
    import torch
    import workloads
    import paper_2102_09038_gb300 as rte
    torch.cuda.set_device(0)
    out = []
    for g in (0.1, 0.3, 0.5, 0.7, 0.9):
        p = workloads.checkerboard(m=24, levels=3, g=g, ratio=0.999, blocks=4, seed=0)
        for n_plus in (0, 2, 4):
            for l in (1, 2, 3, 4, 5, 6):
                s = rte.Solver(p, precision=rte.FP64, n_plus=n_plus, l=l,
                               p1_route=rte.P1_RICHARDSON)
                rho, eta, steps = s.rates(maxit=300, tol=1e-7)
                s.close()
                row = dict(g=g, d_N=(n_plus + 1) * (n_plus + 2) // 2, l=l, rho=rho, eta=eta,
                           steps=steps, g_pow_l=g ** l)
                out.append(row)
                print(json.dumps(row), flush=True)
    return out


if __name__ == '__main__':
    a = parse()
    if a.rates:
        rates_study(a)
        sys.exit(0)
    if a.mk_routes:
        mk_routes_study(a)
        sys.exit(0)
    if a.h2:
        h2_study(a)
        sys.exit(0)
    if a.params:
        params_study(a)
        sys.exit(0)
    if a.impl == 'reference':
        run_reference(a)
    else:
        run_ours(a)
