"""One hull of a synthetic workload on cuda:0, for profilers.

    python -m paper_2510_09417_gb300.profile_hull --dist disk --n 20000000 --seed 2

Builds nothing: it loads the in-tree library, runs vq_hull2d once on the
seeded points (library kernel timing on) and prints the hull size and the
partition kernel's counters (launches, points classified and kept, event
time).  Run it under ncu to capture the kernels of exactly one hull.
"""
from __future__ import annotations

import argparse
import os
import sys


def main(argv=None) -> None:
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import torch

    import paper_2510_09417_gb300 as vq
    import synth

    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--dist", default="disk", choices=synth.DISTRIBUTIONS)
    ap.add_argument("--n", type=int, default=20_000_000)
    ap.add_argument("--seed", type=int, default=2)
    args = ap.parse_args(argv)
    vq.load()
    x, y = synth.points(args.dist, args.n, args.seed)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    vq.vq_set_config(profile=1)
    vq.vq_profile_read(reset=True)
    h = vq.vq_hull2d(xd, yd)
    torch.cuda.synchronize()
    p = vq.vq_profile_read(reset=True)
    vq.vq_set_config(profile=0)
    print(f"h {h.shape[0]} k1_launches {p['k1_launches']} read {p['k1_points_read']} "
          f"kept {p['k1_points_kept']} k1_ms {p['k1_ms']:.3f}")


if __name__ == "__main__":
    main()
