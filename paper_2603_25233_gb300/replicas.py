"""Independent replicas on several GPUs of one node (one process per GPU).

The solver's problems shard with no exchange (each rank solves its own problems), so the only
collectives are the timing ones: a barrier around the timed region, the maximum of the ranks'
times and the sum of the work they did.  NCCL on GPUs; gloo (CPU tensors) where CUDA is absent,
which is how the multi-rank path is tested on machines without GPUs.
"""
import os


def init():
    """Read RANK / WORLD_SIZE / LOCAL_RANK (torchrun) and join the process group when
    WORLD_SIZE > 1.  Returns (world, rank, local_rank)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if not dist.is_initialized():
            if torch.cuda.is_available():
                torch.cuda.set_device(local)
                dist.init_process_group("nccl")
            else:
                dist.init_process_group("gloo")
    return world, rank, local


def _device():
    import torch
    import torch.distributed as dist
    return "cuda" if dist.get_backend() == "nccl" else "cpu"


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce(x, world, op):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=op)
    return float(t.item())


def reduce_max(x, world):
    import torch.distributed as dist
    return _reduce(x, world, dist.ReduceOp.MAX if world > 1 else None)


def reduce_sum(x, world):
    import torch.distributed as dist
    return _reduce(x, world, dist.ReduceOp.SUM if world > 1 else None)


def aggregate(units_local, seconds_local, world):
    """Whole-job throughput of independent replicas: the work of all ranks over the slowest
    rank's time.  Returns (units per second, max seconds, total units)."""
    t_max = reduce_max(seconds_local, world)
    total = reduce_sum(units_local, world)
    return total / t_max, t_max, total


def finalize(world):
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
