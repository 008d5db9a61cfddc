"""Run a few T-REXI steps of one configuration, for profiler captures (ncu).

    python -m paper_1812_03431_gb300.profile_case --N 170 --batch 16 --M 256 --layout spectral --steps 2

Inputs are the seeded n^-3 spectra of ``inputs.random_spectral``; for the grid
layout they are synthesised on the device first.  Prints one line with the
output checksum so that a plain run can be checked before a profiled one.
"""
import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--N", type=int, default=170)
    ap.add_argument("--nlat", type=int, default=0)
    ap.add_argument("--nlon", type=int, default=0)
    ap.add_argument("--M", type=int, default=256)
    ap.add_argument("--tau", type=float, default=1200.0)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--layout", default="spectral", choices=["spectral", "grid"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--adjoint", action="store_true")
    ap.add_argument("--tune", action="store_true", help="pick the pole-slot layout by timing, as bench.py does")
    ap.add_argument("--pole-slots", type=int, default=0, help="fixed pole-slot count (0: the plan's default)")
    ap.add_argument("--solver", default="delta", choices=["delta", "phi"])
    ap.add_argument("--solve-arith", default="fp64", choices=["fp64", "fp32x2"])
    ap.add_argument("--layout-shape", type=int, default=-1,
                    help="with --pole-slots: 0 same pole groups for every order, 1 proportional to length; "
                         "2 (3: lean, 4: lean on two-warp CTAs) the fused solve with --pole-slots states per CTA tile")
    ap.add_argument("--pole-groups", type=int, default=0,
                    help="with layout shapes 2 to 4: CTAs per tile's poles (0: the default)")
    args = ap.parse_args()
    import torch

    from paper_1812_03431_gb300 import inputs, rexi
    nlon = args.nlon or 3 * args.N + 3 + (3 * args.N + 3) % 2
    while not rexi._smooth(nlon):
        nlon += 2
    nlat = args.nlat or nlon // 2
    plan = rexi.Plan(args.N, nlat, nlon, M=args.M, tau=args.tau, max_batch=args.batch, layout=args.layout,
                     precision=args.precision, pole_slots=args.pole_slots, solver=args.solver,
                     solve_arith=args.solve_arith)
    if args.layout_shape >= 0 and args.pole_slots > 0:
        plan.set_pole_slots(args.batch, args.pole_slots, args.layout_shape, groups=args.pole_groups)
    slots = plan.tune(args.batch) if args.tune else plan.info()["pole_slots"]
    S = torch.from_numpy(inputs.random_spectral(args.N, args.batch, 3)).cuda()
    x = plan.synthesize(S) if args.layout == "grid" else S
    y = None
    for _ in range(args.steps):
        y = plan.step_adjoint(x) if args.adjoint else plan.step(x)
    torch.cuda.synchronize()
    print("profile_case ok: N=%d nlat=%d nlon=%d batch=%d layout=%s pole_slots=%d checksum=%.12e"
          % (args.N, nlat, nlon, args.batch, args.layout, slots, float(y.abs().sum())))
    plan.close()


if __name__ == "__main__":
    main()
