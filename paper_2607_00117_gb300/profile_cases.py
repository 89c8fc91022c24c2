"""Single-kernel cases for profiler captures: each runs one part of the path through the C-ABI on
seeded synthetic inputs, small enough for a multi-pass capture (a few GB on the device at most).

    python -m paper_2607_00117_gb300.profile_cases orbit --grid axisym_2k --potential barred_100k \
        --n-orb 100000 --nsteps 64
        integrate + project a library (the fused orbit kernel, its finalize pass) on one workload's
        grid in another's potential (and pattern speed), without the weight solve
    python -m paper_2607_00117_gb300.profile_cases factor --k 4096 --mode 0
        the active set's preconditioner factorisation (sw_factor_preconditioner) of a shifted,
        Jacobi-scaled passive Gram with near-duplicate column pairs

Each case runs --reps times after one untimed run and prints the CUDA-event time of each run.
"""
import argparse
import json

import numpy as np

from . import inputs


def _passive_gram(K: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    M = 2 * K + 50
    A = np.abs(rng.standard_normal((M, K))) * rng.uniform(0.2, 3.0, K)
    A[:, 1::2] = A[:, 0:K - K % 2:2][:, :A[:, 1::2].shape[1]] + 0.3 * np.abs(rng.standard_normal((M, K // 2)))
    H = A.T @ A
    s = 1.0 / np.sqrt(np.diag(H))
    return ((s[:, None] * H * s[None, :]) + 1e-3 * np.eye(K)).astype(np.float32)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["orbit", "factor"])
    names = sorted(inputs.WORKLOADS.keys() - {"batched_64"})
    ap.add_argument("--grid", default="axisym_2k", choices=names)
    ap.add_argument("--potential", default=None, choices=names, help="default: the grid's workload")
    ap.add_argument("--n-orb", type=int, default=100_000)
    ap.add_argument("--nsteps", type=int, default=64)
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--k", type=int, default=4096)
    ap.add_argument("--mode", type=int, default=0)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--bundle", type=int, default=1, help="orbit case: orbits per column (bundles at bin time)")
    ap.add_argument("--integrator", type=int, default=0, help="orbit case: 0 kick-drift-kick, 1 the adaptive pair")
    ap.add_argument("--drift", action="store_true", help="orbit case: also run the drift-only pass (no binning)")
    ap.add_argument("--ej-every", type=int, default=0, help="orbit case: steps between Jacobi checks (0: default)")
    args = ap.parse_args()

    import torch
    from . import sw
    sw.lib()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    ctx = sw.Context(0, args.prec, stream.cuda_stream)
    times = []
    if args.case == "orbit":
        W = inputs.WORKLOADS[args.grid]
        P = inputs.WORKLOADS[args.potential or args.grid]
        ctx.set_potential(P["potential"])
        ctx.set_option("project_bundle", args.bundle)
        ctx.set_option("integrator", args.integrator)
        if args.ej_every:
            ctx.set_option("ej_every", args.ej_every)
        ics = inputs.disc_ics(inputs.DISC_HALO, args.n_orb, seed=W["seeds"]["ic"])
        ics_d = torch.from_numpy(ics).to(dev)
        for rep in range(args.reps + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if args.drift:
                drift = torch.empty(args.n_orb, dtype=torch.float64, device=dev)
                status = torch.empty(args.n_orb, dtype=torch.uint8, device=dev)
                ctx.integrate_library_device(ics_d, P["omega_p"], W["dt"], args.nsteps, drift, status)
            else:
                ctx.integrate_library_device(ics_d, P["omega_p"], W["dt"], args.nsteps)
            U = ctx.project(dict(W["grid"], gh=0))
            e1.record(stream)
            torch.cuda.synchronize()
            U.free()
            if rep:
                times.append(e0.elapsed_time(e1))
        print(json.dumps({"case": "orbit", "grid": args.grid, "potential": args.potential or args.grid,
                          "n_orb": args.n_orb, "bundle": args.bundle, "integrator": args.integrator,
                          "nsteps": args.nsteps,
                          "rows": inputs.rows_of(dict(W["grid"], gh=0)), "ms": times}))
    else:
        G = _passive_gram(args.k, 7000 + args.k)
        import time
        for rep in range(args.reps + 1):
            t0 = time.perf_counter()
            L, X, info = ctx.factor_preconditioner(G, args.mode)
            if rep:
                times.append(1e3 * (time.perf_counter() - t0))
        print(json.dumps({"case": "factor", "k": args.k, "mode": args.mode, "info": info,
                          "ms_with_copies": times}))


if __name__ == "__main__":
    main()
