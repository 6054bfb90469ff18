"""Host statistics of energy traces and the combination of independent
replicas (the multi-GPU form of this library), checked with two gloo ranks
on the CPU."""
import math
import os
import socket

import numpy as np

from paper_1909_01589_gb300 import stats


def test_reblock_ar1_error():
    """Blocking recovers the error of the mean of an AR(1) series,
    sigma^2/n (1 + phi)/(1 - phi)."""
    rng = np.random.default_rng(0)
    phi, n = 0.8, 1 << 17
    x = np.empty(n)
    x[0] = 0.0
    eps = rng.normal(size=n) * math.sqrt(1 - phi * phi)
    for t in range(1, n):
        x[t] = phi * x[t - 1] + eps[t]
    err, _ = stats.reblock(x)
    expect = math.sqrt(1.0 / n * (1 + phi) / (1 - phi))
    assert abs(err / expect - 1) < 0.2


def test_energy_estimate_weights():
    e = np.array([1.0, 2.0, 3.0, 4.0])
    w = np.array([1.0, 2.0, 1.0, 1.0])
    assert stats.energy_estimate(e, w, 0) == 2.5
    # L = 1: G_k = wbar_k
    assert abs(stats.energy_estimate(e, w, 1) - (1 + 4 + 3 + 4) / 5.0) < 1e-15
    # L = 2: G = [1, 2, 2, 1]
    assert abs(stats.energy_estimate(e, w, 2) - (1 + 4 + 6 + 4) / 6.0) < 1e-15


def test_combine_replicas_inverse_variance():
    est, err = stats.combine_replicas([1.0, 2.0], [1.0, 1.0])
    assert est == 1.5 and abs(err - 1 / math.sqrt(2)) < 1e-15
    est, err = stats.combine_replicas([1.0, 2.0], [1.0, 2.0])
    assert abs(est - (1.0 + 2.0 / 4) / 1.25) < 1e-15


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rng = np.random.default_rng(100 + rank)
    e = -2.9 + 0.01 * rng.normal(size=512)
    w = 1.0 + 0.01 * rng.normal(size=512)
    comb = stats.gather_and_combine(e, w, L=4)
    thr = stats.reduce_throughput(10.0 + rank, 1000 * (rank + 1))
    dist.destroy_process_group()
    out.put((rank, comb, thr))


def test_replicas_two_gloo_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    # both ranks agree, and agree with the serial combination
    ests, errs = [], []
    for r in range(2):
        rng = np.random.default_rng(100 + r)
        e = -2.9 + 0.01 * rng.normal(size=512)
        w = 1.0 + 0.01 * rng.normal(size=512)
        ests.append(stats.energy_estimate(e, w, 4))
        errs.append(stats.reblock(e)[0])
    expect = stats.combine_replicas(ests, errs)
    for _, comb, thr in res:
        assert np.allclose(comb, expect, rtol=1e-12)
        # throughput: all moves over the slowest rank's time
        assert abs(thr[0] - 3000 / 11e-3) < 1e-6 and thr[1] == 11.0
