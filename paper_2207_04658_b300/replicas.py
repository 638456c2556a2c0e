"""Multi-GPU runs: replicas only.

Scenes are independent, so N GPUs run N independent replicas with no collective on the
data path (weak scaling): rank r steps its own copy of the workload (drawn with seed offset
r) or its share of the serving requests, and the only communication is timing: a barrier
before and after the timed region and the maximum of the ranks' times.  One process per
GPU, launched by torchrun (RANK, LOCAL_RANK, WORLD_SIZE, MASTER_ADDR/PORT from the
environment); the backend is NCCL on GPUs and gloo on the CPU (tests).
"""
import os


class Replicas:
    def __init__(self, backend=None):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.backend = backend
        self.dist = None
        self.device = "cpu"
        if self.world > 1:
            import torch.distributed as dist
            self.dist = dist

    def init(self, torch):
        backend = self.backend or ("nccl" if torch.cuda.is_available() else "gloo")
        self.backend = backend
        if backend == "nccl":
            torch.cuda.set_device(self.local)
            self.device = f"cuda:{self.local}"
        if self.dist is not None:
            kw = {"device_id": torch.device("cuda", self.local)} if backend == "nccl" else {}
            self.dist.init_process_group(backend, **kw)

    def seed_offset(self):
        """Rank r's replica draws its scene with seed + r."""
        return self.rank

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def max(self, torch, v):
        """Maximum of a scalar over the ranks (the whole job takes as long as the slowest)."""
        if self.dist is None:
            return float(v)
        t = torch.tensor([float(v)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def sum(self, torch, v):
        if self.dist is None:
            return float(v)
        t = torch.tensor([float(v)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.dist is not None and self.dist.is_initialized():
            self.dist.destroy_process_group()


def job_throughput(units_per_rank, world, max_seconds):
    """Whole-job rate of weak scaling: every rank processes units_per_rank units, the job
    takes the slowest rank's time."""
    return units_per_rank * world / max_seconds


def shard(items, rank, world):
    """Rank r's share of a request stream: every world-th request, starting at r (arrival
    order, so each rank sees the same arrival process thinned by world)."""
    return items[rank::world]
