"""Multi-GPU: independent replicas, and output-channel shards of one layer.

Replicas (what the bench measures): each rank runs whole layers on its own
GPU; the only cross-rank traffic is host-side timing aggregation, a barrier
around the timed region and the maximum elapsed time over ranks (so the
whole-job throughput is total work / slowest rank).

Shards of one layer: a layer's output channels are independent (output
ciphertext m*B + b needs all input ciphertexts of block b and only the weights
of channel m), so rank r holds the weights of its contiguous channel range
(channel_shard, hc_weights_preprocess_range) and the one exchange step is a
broadcast of the 2*I*L input polynomial limbs from the rank that received
them into every rank's own device memory (broadcast_inputs); each rank then
writes its own output ciphertexts [m0*B, m1*B), with no reduction.

Launched by torchrun, one process per GPU; the backend is NCCL on GPUs and
gloo on CPU (tests).
"""
import os


def env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend=None):
    """Initialise torch.distributed from the torchrun environment when WORLD_SIZE > 1."""
    rank, world, local = env_rank()
    if world > 1:
        import torch
        import torch.distributed as dist
        if not dist.is_initialized():
            if backend is None:
                backend = "nccl" if torch.cuda.is_available() else "gloo"
            dist.init_process_group(backend=backend)
    return rank, world, local


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def reduce_max(x: float) -> float:
    """Maximum of a host scalar over all ranks (identity when not distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_throughput(units_per_rank: float, world: int, max_seconds: float) -> float:
    """Units processed by all ranks divided by the slowest rank's time."""
    return units_per_rank * world / max_seconds


def channel_shard(M, world, rank):
    """Contiguous output-channel range [m0, m1) of `rank` when M channels are split over
    `world` ranks as evenly as possible (the first M % world ranks take one more)."""
    base, extra = divmod(M, world)
    m0 = rank * base + min(rank, extra)
    return m0, m0 + base + (1 if rank < extra else 0)


def broadcast_inputs(t, src=0):
    """The sharded layer's one exchange: the input ciphertexts (a tensor on this rank's
    device, or on the CPU under gloo) broadcast from `src` into every rank's copy."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.broadcast(t, src=src)
    return t


def shutdown():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.destroy_process_group()
