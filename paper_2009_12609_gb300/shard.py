"""Direction sharding of the 3D ALI iteration over several devices.

The directions of one radiation-field simulation are independent (Sect. 2.2:
every direction's rays cross the model on their own, and each cell's SIJ,
ESC and NORM are sums over all of them).  So each rank marches a contiguous
share of the model's direction table into its own accumulators, one sum
all-reduce of the accumulator arrays gives every rank the sums of the whole
simulation, and every rank then solves the rate equations of all cells
(loc_solve): the populations stay the same on all ranks, and the next
iteration starts from them everywhere.

This module is host-side orchestration only: the march, the solve and the
accumulators' layout are the library's (loc_march with a direction range,
loc_radiation_buffers, loc_solve); the all-reduce is torch.distributed's
(NCCL on the device buffers in production).
"""
import numpy as np


def direction_range(n_dir, rank, world):
    """Contiguous share [begin, end) of n_dir directions for `rank` of
    `world`: shares differ by at most one direction and cover every
    direction exactly once."""
    if not (0 <= rank < world) or n_dir < world:
        raise ValueError(f"cannot split {n_dir} directions over {world} ranks (rank {rank})")
    return (rank * n_dir) // world, ((rank + 1) * n_dir) // world


class _DeviceArray:
    """A library-owned device array seen through __cuda_array_interface__,
    so that torch can view it without a copy."""

    def __init__(self, ptr, n, dtype):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": np.dtype(dtype).str,
                                         "data": (int(ptr), False), "version": 2}


def accumulator_tensors(model, precision="fp32"):
    """Zero-copy torch views of the model's accumulators that a ray
    simulation with `precision` writes: {SIJ, ESC} and NORM with their
    compensation words (fp32, fp32plain) or the FP64 ones (fp64acc)."""
    import torch
    bufs = model.radiation_buffers()
    names = ("acc64", "norm64") if precision == "fp64acc" else ("acc", "acc_c", "norm", "norm_c")
    return [torch.as_tensor(_DeviceArray(*bufs[k]), device="cuda") for k in names]


def iterate_sharded(model, n_iter, rank, world, tensors=accumulator_tensors, all_reduce=None,
                    **opts):
    """n_iter ALI iterations of a 3D model with the directions split over
    `world` ranks: march this rank's share, sum every accumulator array over
    the ranks, solve.  Returns the solve reports.  `all_reduce(t)` sums a
    tensor in place over the ranks (default: torch.distributed.all_reduce);
    `tensors(model, precision)` lists the arrays to sum."""
    if all_reduce is None:
        import torch.distributed as dist

        def all_reduce(t):
            dist.all_reduce(t, op=dist.ReduceOp.SUM)
    opts = dict(opts)
    opts.pop("max_iter", None)
    n_dir = model.n_dir()
    rng = direction_range(n_dir, rank, world)
    reports = []
    for _ in range(n_iter):
        model.march(dir_range=rng, **opts)
        for t in tensors(model, opts.get("precision", "fp32")):
            all_reduce(t)
        reports.append(model.solve(**opts))
    return reports
