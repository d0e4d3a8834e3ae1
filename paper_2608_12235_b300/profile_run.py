"""A bounded window of the benchmark workload for profilers.

    python -m paper_2608_12235_b300.profile_run --what pair|build|iters [--skin-abs 100] [--skin-s 0.02]
        [--densify 6000]

Densifies the lognormal N = 1e6, S = 5e5 packing (mixed precision) outside the
profiled range, then brackets with cudaProfilerStart/Stop either two
iterations launched one by one (`pair`), one neighbour rebuild (`build`), or
100 graph-driven iterations (`iters`), so that `ncu --profile-from-start off`
captures only that window.
"""
from __future__ import annotations

import argparse

import torch

from . import inputs, rcp


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--what", choices=["pair", "build", "iters"], default="pair")
    ap.add_argument("--skin-abs", type=float, default=100.0)
    ap.add_argument("--skin-s", type=float, default=0.02)
    ap.add_argument("--densify", type=int, default=6000)
    ap.add_argument("--precision", type=int, default=rcp.RCP_MIXED)
    a = ap.parse_args()
    D0 = inputs.lognormal(1_000_000, 2.0, 5e5)
    p = rcp.Packing(D0, seed=0, precision=a.precision, skin_abs=a.skin_abs, skin_s=a.skin_s)
    r = p.run(max_iters=a.densify, shrink=False)
    rcp.rcp_build_neighbors(p.h)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    if a.what == "pair":
        rcp.rcp_profile(p.h, 2)
    elif a.what == "build":
        rcp.rcp_build_neighbors(p.h)
    else:
        p.run(max_iters=100, shrink=False)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print(f"window done: iters={r.iters} pairs={r.pairs}")
    p.close()


if __name__ == "__main__":
    main()
