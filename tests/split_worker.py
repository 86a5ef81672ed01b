"""One rank of the split-form GPU test (run as a separate process by test_gpu_split.py).

The rank bundles its share of a graph's edges on cuda:0 and sums the splatted histogram
with the other ranks' through a gloo group on host copies each iteration; it saves its
final polylines and density stacks for the test to compare with one context over all edges.
usage: python split_worker.py <rank> <world> <port> <input.npz> <output.npz>
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def main():
    rank, world, port = int(sys.argv[1]), int(sys.argv[2]), int(sys.argv[3])
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_1504_02687_gb300 as pkg

    d = np.load(sys.argv[4])
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    torch.cuda.set_device(0)
    off, xy, group, weight = d["off"], d["xy"], d["group"], d["weight"]
    E = off.shape[0] - 1
    lo, hi = rank * E // world, (rank + 1) * E // world  # this rank's edges
    part_off = off[lo:hi + 1] - off[lo]
    part_xy = xy[off[lo]:off[hi]]
    p = pkg.default_params(grid_w=int(d["W"]), grid_h=int(d["H"]), radius=int(d["r"]),
                           passes=int(d["k"]), n_fixed=0, n_max=int(d["n_max"]),
                           sum_bits=int(d["sum_bits"]))
    ctx = pkg.bundle_init_polylines(p, part_off, part_xy, group[lo:hi], int(d["G"]),
                                    weight[lo:hi], map5=d["map5"])
    try:
        pkg.bundle_iterate_split(ctx, int(d["iters"]), dist.all_reduce, on_device=False)
        o, x = pkg.bundle_fetch(ctx, pixels=True)
        np.savez(sys.argv[5], off=o, xy=x,
                 hist=pkg.bundle_fetch_density(ctx, pkg.DENSITY_HIST),
                 sums=pkg.bundle_fetch_density(ctx, pkg.DENSITY_SUMS),
                 rho=pkg.bundle_fetch_density(ctx, pkg.DENSITY_RHO))
    finally:
        pkg.bundle_destroy(ctx)
    dist.barrier()
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
