"""Host-side logic of bench.py's multi-rank runs on CPU: the cost-balanced
split of the uneven-shell batch over ranks and the max-over-ranks timing,
with two gloo ranks (no GPU)."""

import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_1104_3408_gb300 import inputs


def test_shell_split_is_a_balanced_partition():
    descs = inputs.shell_batch(256, seed=0)
    for ws in (1, 2, 3, 4, 8):
        parts = [bench._shells_for_rank(descs, r, ws) for r in range(ws)]
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(descs)))
        loads = [sum(bench._shell_units(descs[i]) for i in p) for p in parts]
        # greedy longest-first: within one largest shell of each other
        biggest = max(bench._shell_units(d) for d in descs)
        assert max(loads) - min(loads) <= biggest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    r, lr, w, d = bench._dist()
    descs = inputs.shell_batch(16, seed=1)
    mine = bench._shells_for_rank(descs, r, w)
    t = bench._max_over_ranks(10.0 + r, d)
    q.put((r, lr, w, mine, t))
    d.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_share_the_batch_and_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=100) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[2] == 2 for o in out)
    assert sorted(out[0][3] + out[1][3]) == list(range(16))
    assert not set(out[0][3]) & set(out[1][3])
    assert all(o[4] == 11.0 for o in out)


def test_operator_work_is_the_method_count():
    # the roofline's algorithmic work per pt-field per substep is the method's
    # 2 n_r + 16 N + 2 (L + 1) FP64 flops (d_r, d_theta + d_phi, and the
    # filter's DFT, projection and inverse DFT)
    w = dict(inputs.WORKLOADS["ks_33x48x96"], name="ks_33x48x96")
    P = w["n_r"] * w["n_theta"] * w["n_phi"] * w["n_fields"]
    total = sum(bench._op_flops(w, ph) for ph in bench.PAIRS)
    assert total == (2 * 33 + 16 * 48 + 2 * (46 + 1)) * P == 928 * P
    assert set(bench.PAIRS) == set(bench.FAMILIES["k_op_tc"])
