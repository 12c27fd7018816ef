"""World-size-2 runs over gloo on the CPU.

1. The weak-scaling layout: each rank its own instance, the job time is the
   slowest rank's.
2. One problem's N scenarios split across the ranks, in the library's
   partials layout [P1 | P2 | P3 | P4] (saa_partials, include/saa.h): each
   rank takes multirank.scenario_ranges' range, forms that range's partial
   sums (here with the oracle, the CPU stand-in for the rank's GPU, so no
   GPU is involved), multirank.merge_partials adds them with one
   collective, and the estimate finalized from the totals equals the
   single-rank oracle result.  The GPU side of the same exchange (the
   library's saa_partials, saa_partials_merge and saa_finalize_partials) is
   checked in tests/test_gpu_partials.py.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


D, N, K, LAM = 6, 3001, 3, 0.5


def _worker(rank, world, port, root, q):
    import sys
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2404_11631_gb300 import inputs, multirank, saa
        # 1. weak scaling
        inst = multirank.instance_for_rank(rank)
        tmax = multirank.max_time_over_ranks(0.5 + rank)
        # 2. split one instance's N over the ranks and merge the partials
        ins = inputs.instance(D, 0)
        X = inputs.decisions(K, D, 0)
        P = oracle.make_problem(D, N, ins.mu, ins.chol, law=oracle.LAW_MIX, seed=4, lam=LAM)
        a, b = multirank.scenario_ranges(N, world)[rank]
        part = torch.tensor(oracle.partials(P, 32, a, b - a, X, grad=True))
        assert part.numel() == saa.partials_len(D, K, True)
        tot = multirank.merge_partials(part, ordered=False).numpy()
        out = oracle.finalize_partials(N, X, ins.mu, LAM, tot, grad=True)
        q.put((rank, inst, tmax, (a, b), out["f"], out["grad"]))
    finally:
        dist.destroy_process_group()


def test_two_rank_weak_scaling_and_partial_merge():
    import oracle
    from paper_2404_11631_gb300 import inputs
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, root, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort(key=lambda r: r[0])
    assert [r[1] for r in res] == [0, 1]
    assert all(r[2] == 1.5 for r in res)
    assert [r[3] for r in res] == [(0, N // 2), (N // 2, N)]
    ins = inputs.instance(D, 0)
    X = inputs.decisions(K, D, 0)
    P = oracle.make_problem(D, N, ins.mu, ins.chol, law=oracle.LAW_MIX, seed=4)
    ref = oracle.saa(P, 32, X, grad=True)
    for r in res:
        assert np.allclose(r[4], ref["f"], rtol=1e-10, atol=1e-12)
        assert np.allclose(r[5], ref["grad"], rtol=1e-9, atol=1e-11)
    # both ranks hold the same totals, so the same estimate bit for bit
    assert np.array_equal(res[0][4], res[1][4]) and np.array_equal(res[0][5], res[1][5])


def test_scenario_ranges_cover_without_overlap():
    from paper_2404_11631_gb300 import multirank
    for n, w in ((10, 3), (1 << 20, 8), (7, 7), (2, 1)):
        r = multirank.scenario_ranges(n, w)
        assert r[0][0] == 0 and r[-1][1] == n
        assert all(a < b for a, b in r) and all(r[i][1] == r[i + 1][0] for i in range(w - 1))
        assert max(b - a for a, b in r) - min(b - a for a, b in r) <= 1
    with pytest.raises(ValueError):
        multirank.scenario_ranges(3, 4)
