"""The multi-GPU path is replicas only (scenes are independent): its host logic -- seed
offsets, the barrier and max-over-ranks timing, the whole-job throughput, the sharding of
the serving stream -- on world_size 2 with the gloo backend on the CPU."""
import os
import socket



def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import json
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    from paper_2207_04658_b300 import replicas, scenes
    r = replicas.Replicas(backend="gloo")
    r.init(torch)
    r.barrier()
    res = {"rank": r.rank, "world": r.world, "seed_offset": r.seed_offset(),
           "max": r.max(torch, 1.5 + rank), "sum": r.sum(torch, 10.0 * (rank + 1))}
    reqs = scenes.serving_requests(rate=20.0, duration=3.0, seed=5)
    res["shard"] = [q["t"] for q in replicas.shard(reqs, r.rank, r.world)]
    res["all"] = [q["t"] for q in reqs]
    r.barrier()
    r.close()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump(res, f)


def test_replicas_on_two_gloo_ranks(tmp_path):
    import json
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    res = [json.load(open(tmp_path / f"rank{k}.json")) for k in range(2)]
    assert [r["rank"] for r in res] == [0, 1] and all(r["world"] == 2 for r in res)
    assert [r["seed_offset"] for r in res] == [0, 1]  # independent replicas
    assert all(r["max"] == 2.5 for r in res)  # the slowest rank's time
    assert all(r["sum"] == 30.0 for r in res)
    a, b = res[0]["shard"], res[1]["shard"]
    assert sorted(a + b) == sorted(res[0]["all"]) and not set(a) & set(b)
    assert abs(len(a) - len(b)) <= 1


def test_job_throughput_is_weak_scaling():
    from paper_2207_04658_b300.replicas import job_throughput
    assert job_throughput(8_192_000 * 100, 4, 2.0) == 8_192_000 * 100 * 4 / 2.0
