"""Time single kernels of the library on a synthetic lattice (also the workload of
the committed ncu captures).

    python kernelbench.py dhop --workload 16^3x32 --variants 2 4
    python kernelbench.py eopair --workload 16^3x32
    python kernelbench.py dots --a 80 --b 8 --n 1572864

``dhop``: the operator-pair kernel shapes (A p, A^+ phat for k slots) through
``Solver.time_kernel``; after the timed runs each listed shape is launched once
more (the launches an ncu capture skips to). ``eopair``: the even-odd (Schur
complement) operator pair A_hat p, A_hat^+ phat on the odd half lattice for k
slots (two stage kernels per pair): one warm-up pair, reps timed, one more.
``dots``: the inner-product matrix
X^H Y of FP32 fields on the tensor cores and on the CUDA cores; the last launch
is one more tensor-core call. ``restart``: eigBiCG on k sources stopped a few
iterations after the first window restart (the m-th iteration launches the
tensor-core restart product that does work). Inputs are seeded synthetic fields.
"""
from __future__ import annotations

import argparse
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python kernelbench.py")
    sub = ap.add_subparsers(dest="what", required=True)
    d = sub.add_parser("dhop")
    d.add_argument("--workload", default="16^3x32")
    d.add_argument("--k", type=int, default=8)
    d.add_argument("--variants", type=int, nargs="+", default=[2, 4])
    d.add_argument("--reps", type=int, default=5)
    d.add_argument("--no-autotune", dest="autotune", action="store_false",
                   help="skip the init autotuner: the only operator launches are the listed shapes' "
                        "(reps timed + 1 each, in order)")
    e = sub.add_parser("eopair")
    e.add_argument("--workload", default="16^3x32")
    e.add_argument("--k", type=int, default=8)
    e.add_argument("--reps", type=int, default=5)
    r = sub.add_parser("restart")
    r.add_argument("--workload", default="16^3x32")
    r.add_argument("--k", type=int, default=2)
    t = sub.add_parser("dots")
    t.add_argument("--a", type=int, default=80)
    t.add_argument("--b", type=int, default=8)
    t.add_argument("--n", type=int, default=12 * 16 ** 3 * 32)
    t.add_argument("--reps", type=int, default=5)
    args = ap.parse_args(argv)

    import numpy as np
    import torch
    from paper_0911_2285_gb300.lqcd import Solver, field_dots
    if args.what == "dhop":
        from seeded_inputs import WORKLOADS, workload_links
        w = WORKLOADS[args.workload]
        with Solver(workload_links(args.workload), w["dims"], w["kappa"], nev=2, m=8, n1=1, tol=1e-10,
                    maxiter=100, precision="mixed", k_max=args.k, autotune=args.autotune) as s:
            V = 1
            for L in w["dims"]:
                V *= L
            alg = V * (4 * 48 + args.k * 4 * 96)
            tag = "autotuned" if args.autotune else "default"
            print(f"{args.workload}: {tag} shape {s.dslash_variant()}, algorithmic bytes {alg}")
            for v in args.variants:
                ms = s.time_kernel(10 + v, args.k, args.reps)
                print(f"  shape {v}: {ms:.4f} ms  {alg / ms / 1e6:.0f} GB/s")
            for v in args.variants:
                s.time_kernel(10 + v, args.k, 1)
    elif args.what == "eopair":
        from seeded_inputs import WORKLOADS, workload_links
        w = WORKLOADS[args.workload]
        with Solver(workload_links(args.workload), w["dims"], w["kappa"], nev=2, m=8, n1=1, tol=1e-10,
                    maxiter=100, precision="mixed", k_max=args.k, evenodd=True) as s:
            V = 1
            for L in w["dims"]:
                V *= L
            # per stage the links once (two-row FP32); per slot, stage 1 reads p, phat and
            # writes the two even-half intermediates, stage 2 reads them and p, phat and
            # writes A_hat p, A_hat^+ phat: ten half-lattice fields
            alg = 2 * V * 4 * 48 + args.k * 10 * (V // 2) * 96
            s.time_kernel(0, args.k, 1)   # first launches load the kernels' module
            ms = s.time_kernel(0, args.k, args.reps)
            print(f"{args.workload}: even-odd operator pair, k={args.k}: {ms:.4f} ms, "
                  f"algorithmic bytes {alg} ({alg / ms / 1e6:.0f} GB/s)")
            s.time_kernel(0, args.k, 1)
    elif args.what == "restart":
        from seeded_inputs import WORKLOADS, workload_links, workload_source
        w = WORKLOADS[args.workload]
        b = np.stack([workload_source(args.workload, i) for i in range(args.k)])
        with Solver(workload_links(args.workload), w["dims"], w["kappa"], nev=w["nev"], m=w["m"], n1=args.k,
                    tol=1e-10, maxiter=w["m"] + 4, precision="mixed", k_max=args.k) as s:
            _, info, _ = s.solve(b, mode="eigbicg", raise_on_fail=False)
            print(f"{args.workload}: eigBiCG window m={w['m']} nev={w['nev']}, {args.k} sources, "
                  f"{info[0]['iters']} iterations, {info[0]['restarts']} restart(s)")
    else:
        g = torch.Generator(device="cuda").manual_seed(5)
        X = torch.randn(args.a, args.n, dtype=torch.complex64, device="cuda", generator=g)
        Y = torch.randn(args.b, args.n, dtype=torch.complex64, device="cuda", generator=g)
        gb = (args.a + args.b) * args.n * 8 / 1e9
        _, t1 = field_dots(X, Y, path=1, reps=args.reps)
        _, t0 = field_dots(X, Y, path=0, reps=args.reps)
        print(f"X^H Y {args.a}x{args.b}, n={args.n}: tensor cores {t1:.4f} ms ({gb / t1 * 1e3:.0f} GB/s), "
              f"CUDA cores {t0:.4f} ms ({gb / t0 * 1e3:.0f} GB/s)")
        field_dots(X, Y, path=1)


if __name__ == "__main__":
    main()
