"""Small, self-contained invocation of the hot path for profilers.

Runs the first RK4 stage of the saturated workload on a d-mode slice:
operator apply (hopf_apply_op) and one rounding (tt_round) at rank 6r, plus
one fused hopf_step when --step is given.  Sized by --d/--n/--r so a capture
stays small (d=4, n=128, r=64 holds about 2.5 GB on the device).

  python -m paper_2403_04946_gb300.profile_case --d 4 --n 128 --r 64 [--mixed [--qr-method doublefloat]] [--profile]

With --surrogate it instead runs the surrogate network alone on seeded
synthetic data (26 -> 256 x 4 -> 14, 4 members): 20 training steps of batch
128 (one captured CUDA graph, replayed) and one 4096-query prediction.

  python -m paper_2403_04946_gb300.profile_case --surrogate
"""
from __future__ import annotations

import argparse
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--d", type=int, default=4)
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--r", type=int, default=64)
    ap.add_argument("--tol", type=float, default=1e-7)
    ap.add_argument("--step", action="store_true")
    ap.add_argument("--mixed", action="store_true", help="HOPF_MIXED precision")
    ap.add_argument("--surrogate", action="store_true", help="the surrogate network only")
    ap.add_argument("--profile", action="store_true", help="print the per-class profile record")
    ap.add_argument("--qr-method", choices=["tensor", "doublefloat"], default="tensor",
                    help="mixed precision QR: tensor-core products (default) or double-float on the FP32 pipe")
    ap.add_argument("--steps", type=int, default=1, help="RK4 steps with --step (the first sets up workspaces)")
    ap.add_argument("--cdf", action="store_true",
                    help="the paper's CDF equation on a saturated state, explicit midpoint steps (--d 20 --n 64 --r 128)")
    args = ap.parse_args()
    from paper_2403_04946_gb300 import binding
    import synthetic

    if args.surrogate:
        return surrogate_case(binding, synthetic)
    if args.cdf:
        return cdf_case(binding, synthetic, args)

    cores, _ = synthetic.saturated_tt_cores(args.d, args.n, args.r, seed=0)
    ctx = binding.Context(d=args.d, n=args.n, nu=0.01, tol=args.tol, rank_cap=args.r, L=12.4,
                          precision=binding.HOPF_MIXED if args.mixed else binding.HOPF_FP64)
    if args.mixed:
        ctx.hopf_set_qr_method(binding.HOPF_QR_TENSOR if args.qr_method == "tensor" else binding.HOPF_QR_DOUBLEFLOAT)
    t = ctx.tt_from_host(cores, max_rank=args.r)
    big = ctx.tt_create(6 * args.r)
    if args.profile:
        ctx.hopf_profile_enable(True)
    t0 = time.time()
    ctx.hopf_apply_op(t, big)
    disc, _ = ctx.tt_round(big, args.tol, args.r)
    print(f"apply+round d={args.d} n={args.n} r={args.r}: {time.time() - t0:.3f} s, "
          f"ranks {ctx.tt_get_ranks(big)}, discarded {disc:.3e}")
    if args.profile:
        print_profile(ctx.hopf_profile_read(reset=True))
    if args.step:
        for s in range(args.steps):
            t0 = time.time()
            ctx.hopf_step(t, 1.2e-5, 1)
            print(f"hopf_step {s}: {time.time() - t0:.3f} s")
            if args.profile:
                print_profile(ctx.hopf_profile_read(reset=True))
    ctx.tt_free(big)
    ctx.tt_free(t)
    ctx.close()


def cdf_case(binding, synthetic, args):
    """Explicit-midpoint steps of the CDF equation (box [-1.3, 1.3], gamma =
    0.01) on a saturated state with every interior rank at --r."""
    cores, _ = synthetic.saturated_tt_cores(args.d, args.n, args.r, seed=0)
    ctx = binding.Context(d=args.d, n=args.n, nu=0.01, tol=args.tol, rank_cap=args.r,
                          precision=binding.HOPF_MIXED if args.mixed else binding.HOPF_FP64)
    ctx.hopf_set_equation(binding.HOPF_EQ_CDF, 1.3)
    if args.profile:
        ctx.hopf_profile_enable(True)
    t = ctx.tt_from_host(cores, max_rank=args.r)
    for s in range(args.steps):
        t0 = time.time()
        out = ctx.hopf_step_scheme(t, binding.HOPF_MIDPOINT, 1e-4, 1, record=True)
        print(f"CDF midpoint step {s} d={args.d} n={args.n} r={args.r}: {time.time() - t0:.3f} s, "
              f"max ranks per rounding {out['ranks'].max(axis=1).tolist()}")
        if args.profile:
            print_profile(ctx.hopf_profile_read(reset=True))
    ctx.tt_free(t)
    ctx.close()


def print_profile(prof):
    for k, v in prof.items():
        if isinstance(v, dict) and v.get("launches", 0):
            rate = v["flops"] / (v["ms"] / 1e3) / 1e12 if v["ms"] > 0 and v["flops"] > 0 else 0.0
            print(f"  {k:8s} {v['ms']:10.2f} ms  {v['launches']:6d} launches  {rate:8.3f} TFLOP/s")


def surrogate_case(binding, synthetic):
    import numpy as np

    dims, members, iters, batch, ns = [26, 256, 256, 256, 256, 14], 4, 20, 128, 1280
    ctx = binding.Context(d=4, n=8, nu=0.05, tol=1e-10, rank_cap=4, L=3.0)
    net = binding.Mlp(ctx, dims[0], dims[1], len(dims) - 2, dims[-1], members, 4096,
                      synthetic.mlp_init(0, dims, members))
    rng = np.random.default_rng(1)
    X, Y = rng.normal(size=(ns, dims[0])), rng.normal(size=(ns, dims[-1]))
    net.set_data(X, Y)
    t0 = time.time()
    loss = net.train(synthetic.batch_indices(2, iters, members, batch, ns), np.full(iters, 1e-3))
    t1 = time.time()
    net.predict(np.repeat(X, 4, axis=0)[:4096], 1.0)
    t2 = time.time()
    print(f"surrogate: {iters} training steps {t1 - t0:.3f} s (loss {loss[0].mean():.3f} -> "
          f"{loss[-1].mean():.3f}), 4096-query prediction {t2 - t1:.4f} s")
    net.close()
    ctx.close()


if __name__ == "__main__":
    main()
