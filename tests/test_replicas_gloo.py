"""Replica logic over two CPU processes (gloo): sharding covers every problem once,
results gathered from the ranks equal the single-process results, timing takes the
slowest rank, and a rank that fails before the exchange is detected on the host by
the other rank's process-group timeout (no GPU involved)."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, mode, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import oracle as O
    from paper_1901_08393_gb300 import inputs, replicas

    replicas.init("gloo", timeout_s=10.0 if mode == "fail" else 60.0)
    try:
        meshes = [inputs.cube_mesh(n) for n in (1, 2, 3)] + [inputs.tetra_mesh(k) for k in (2, 3)]
        mine = replicas.shard(list(enumerate(meshes)), rank, world)
        if mode == "fail" and rank == 1:
            raise RuntimeError("rank 1 fails before the exchange")
        caps = {k: O.solve_capacity(m.verts, O.canonical(m.verts, m.tris), tol=1e-12)[0] for k, m in mine}
        t = replicas.reduce_max(1.0 + rank)
        n = replicas.reduce_sum(len(mine))
        allcaps = {}
        for d in replicas.gather(caps):
            allcaps.update(d)
        q.put((rank, "ok", t, n, allcaps))
    except Exception as e:  # reported to the parent, never a GPU fault
        q.put((rank, "error", repr(e)))


def _run(mode):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, mode, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=60)
    return sorted(out, key=lambda x: x[0])


def test_shard_covers_everything_once():
    from paper_1901_08393_gb300 import replicas

    items = list(range(11))
    parts = [replicas.shard(items, r, 3) for r in range(3)]
    assert sorted(sum(parts, [])) == items
    assert max(map(len, parts)) - min(map(len, parts)) <= 1


@pytest.mark.slow
def test_two_rank_replicas_match_single_process():
    import oracle as O
    from paper_1901_08393_gb300 import inputs

    out = _run("ok")
    assert [o[1] for o in out] == ["ok", "ok"], out
    meshes = [inputs.cube_mesh(n) for n in (1, 2, 3)] + [inputs.tetra_mesh(k) for k in (2, 3)]
    ref = {k: O.solve_capacity(m.verts, O.canonical(m.verts, m.tris), tol=1e-12)[0] for k, m in enumerate(meshes)}
    for rank, status, t, n, allcaps in out:
        assert t == 2.0 and n == len(meshes)
        assert allcaps == ref


@pytest.mark.slow
def test_failed_rank_is_detected_on_the_host():
    out = _run("fail")
    assert out[1][1] == "error" and "rank 1 fails" in out[1][2]
    assert out[0][1] == "error"  # the surviving rank's collective ended with an error
