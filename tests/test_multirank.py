"""World-size-2 runs over gloo on the CPU.

1. The weak-scaling layout: each rank its own instance, the job time is the
   slowest rank's.
2. The exchange that splitting one instance's scenarios across ranks needs:
   each rank forms the FP64 partial sums of Eq. 4 over its scenario range
   (here from the oracle's samples, so no GPU is involved), one all-reduce
   merges them, and the finalized f_hat and gradient equal the single-rank
   oracle result.
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


def _worker(rank, world, port, root, q):
    import sys
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2404_11631_gb300 import inputs, multirank
        # 1. weak scaling
        inst = multirank.instance_for_rank(rank)
        tmax = multirank.max_time_over_ranks(0.5 + rank)
        # 2. split one instance's N over the ranks and merge the partials
        d, N, K, lam = 6, 3001, 3, 0.5
        ins = inputs.instance(d, 0)
        X = inputs.decisions(K, d, 0)
        P = oracle.make_problem(d, N, ins.mu, ins.chol, law=oracle.LAW_MIX, seed=4, lam=lam)
        a, b = multirank.scenario_ranges(N, world)[rank]
        z, s, _ = oracle.generate(P, 32, a, b - a)
        A = s[:, None] * z                              # a_i = s_i zhat_i
        Y = X @ ins.chol                                # y_k = C'w_k (rows)
        Q = A @ Y.T                                     # [n, K]
        part = np.concatenate([Q.sum(0), (Q * Q).sum(0), A.sum(0), (A.T @ Q).T.ravel()])
        tot = multirank.merge_partials(torch.tensor(part)).numpy()
        S1, S2, m_t, G = tot[:K], tot[K:2 * K], tot[2 * K:2 * K + d], tot[2 * K + d:].reshape(K, d)
        c = X @ ins.mu
        V = (S2 - S1 * S1 / N) / (N - 1)
        f = lam * V - (c + S1 / N)
        m = m_t / N
        grad = (lam * 2 / (N - 1) * (G - S1[:, None] * m[None, :]) - m[None, :]) @ ins.chol.T - ins.mu[None, :]
        q.put((rank, inst, tmax, f, grad))
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
    res.sort()
    assert [r[1] for r in res] == [0, 1]
    assert all(r[2] == 1.5 for r in res)
    d, N, K = 6, 3001, 3
    ins = inputs.instance(d, 0)
    X = inputs.decisions(K, d, 0)
    P = oracle.make_problem(d, N, ins.mu, ins.chol, law=oracle.LAW_MIX, seed=4)
    ref = oracle.saa(P, 32, X, grad=True)
    for r in res:
        assert np.allclose(r[3], ref["f"], rtol=1e-10, atol=1e-12)
        assert np.allclose(r[4], ref["grad"], rtol=1e-9, atol=1e-11)
