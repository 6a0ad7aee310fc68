"""Small driver for kernel profiles: one plan, a few imaginary-time steps
(every pass of the step, one cadence with parity projection), then an energy.

    python -m paper_2006_16935_gb300.profile_step --n 256 --precision c64 --steps 2 --tuning 2,2,0

Used as the target of ncu captures of single kernels on a lattice larger than
L2 but small enough for a multi-pass capture.  --tuning y,z,x sets the launch
shapes of the plan's step arithmetic (qfd_set_tuning: y 0..2, z -1..2, x 0..2)
so that a capture sees the variant the autotuner picks at full size.
"""
from __future__ import annotations

import argparse

from . import qfd


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--precision", default="c64", choices=sorted(qfd.PRECISION))
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--parity", type=int, default=1)
    ap.add_argument("--kinetic", type=int, default=2)
    ap.add_argument("--tuning", default="", help="y,z,x launch shapes of the step arithmetic")
    args = ap.parse_args(argv)
    centre = "offgrid" if args.kinetic == 0 else "grid"  # the Dirichlet box of H_K(0) is symmetric off-grid
    with qfd.Plan(args.n, 0.05, 1.0, 5e-4, args.kinetic, precision=args.precision, ortho_every=2,
                  centre=centre) as p:
        p.fill_potential("softcoul", (0.01,))
        if args.tuning:
            y, z, x = (int(v) for v in args.tuning.split(","))
            policy = {"c128": 0, "c64": 1, "df64": 2}[args.precision]
            p.set_tuning(policy, y, z, x)
        p.fill_psi_uniform(0, 3)
        p.set_parity(0, args.parity)
        p.step(0, args.steps)
        e, n2 = p.energy(0)
    print(f"n={args.n} precision={args.precision} steps={args.steps} E={e:.12f} norm2={n2:.6e}")


if __name__ == "__main__":
    main()
