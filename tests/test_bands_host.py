"""Frequency-band sharding of the dictionary step: the host protocol on CPU.

Two gloo ranks run bands.band_update with stand-in learners whose exported
rows encode (rank, sample, filter, frequency) in their values, so the test can
check that each band owner folds exactly its rows of every sample, in rank
order, and that every rank projects the same support sums, added in rank
order.  The kernels behind the real calls are tested on the GPU.
"""
import os
import socket

import pytest

from paper_1706_06972_gb300.bands import band_partition, ordered_sum


def test_band_partition_covers_the_rows_once_in_even_runs():
    for N in (64, 128, 256, 288, 512):
        for G in (1, 2, 3, 4, 7):
            bands = band_partition(N, G)
            assert len(bands) == G and bands[0][0] == 0 and bands[-1][1] == N
            for (lo, hi), (lo2, _) in zip(bands, bands[1:]):
                assert hi == lo2
            sizes = [hi - lo for lo, hi in bands]
            assert all(s % 2 == 0 and s > 0 for s in sizes) and max(sizes) - min(sizes) <= 2
    with pytest.raises(ValueError):
        band_partition(8, 5)


def test_ordered_sum_is_the_left_to_right_sum():
    import torch

    parts = [torch.tensor([1e8], dtype=torch.float32), torch.tensor([1.0]), torch.tensor([-1e8])]
    assert float(ordered_sum(parts)) == float((parts[0] + parts[1]) + parts[2])


class FakeLearner:
    """Exports rows whose values name their origin; records what it folds and
    projects."""

    def __init__(self, N, K, M, rank, band, n_local):
        self.N, self.K, self.M, self.rank, self.band, self.n_local = N, K, M, rank, band, n_local
        self.totals = []
        self.dropped = False

    def band_rows(self):
        return self.band

    def band_export(self, lo, hi, n):
        import torch

        NH = self.N // 2 + 1
        fb = (hi - lo) * NH
        s = torch.arange(n).view(n, 1, 1).float()
        k = torch.arange(self.K).view(1, self.K, 1).float()
        p = (lo * NH + torch.arange(fb)).view(1, 1, fb).float()
        Z = torch.complex(self.rank * 1000 + s * 100 + k + 0 * p, p + 0 * s + 0 * k)
        x = torch.complex((self.rank * 1000 + s * 100).view(n, 1) + 0 * p.view(1, fb), p.view(1, fb) + 0 * s.view(n, 1))
        return Z.to(torch.complex64), x.to(torch.complex64)

    def band_fold(self, Z, x):
        self.Z, self.x = Z, x

    def band_dict_step(self):
        import torch

        g = torch.Generator().manual_seed(100 * self.rank + len(self.totals))
        return torch.randn((self.K, self.M, self.M), generator=g) * 10 ** (3 * self.rank)

    def band_project(self, total, last):
        self.totals.append((total.clone(), last))

    def drop_pending(self):
        self.dropped = True


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q, n_locals):
    import torch
    import torch.distributed as dist

    from paper_1706_06972_gb300.bands import TorchComm, band_update

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    N, K, M, Jd = 16, 3, 2, 4
    band = band_partition(N, world)[rank]
    lr = FakeLearner(N, K, M, rank, band, n_locals[rank])
    comm = TorchComm()
    band_update(lr, comm, n_locals[rank], Jd)
    totals = torch.stack([t for t, _ in lr.totals])
    every = comm.all_gather(totals)
    q.put((rank, band, lr.Z.numpy(), lr.x.numpy(), [last for _, last in lr.totals], lr.dropped,
           [e.numpy() for e in every]))
    dist.destroy_process_group()


@pytest.mark.parametrize("n_locals", [(2, 3), (1, 0)])
def test_band_update_exchanges_rows_and_reduces_in_rank_order_gloo_world2(n_locals):
    import numpy as np
    import torch
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q, n_locals)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=180) for _ in procs), key=lambda o: o[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    N, K, M, NH = 16, 3, 2, 9
    for rank, (lo, hi), Z, x, lasts, dropped, every in out:
        # the mini-batch is rank 0's samples, then rank 1's, each restricted to this band
        assert Z.shape == (sum(n_locals), K, (hi - lo) * NH)
        row = 0
        for src in range(2):
            for s in range(n_locals[src]):
                assert np.all(Z[row].real == src * 1000 + s * 100 + np.arange(K)[:, None])
                assert np.all(Z[row].imag == lo * NH + np.arange((hi - lo) * NH)[None, :])
                assert np.all(x[row].real == src * 1000 + s * 100)
                row += 1
        assert lasts == [False, False, False, True] and dropped
        # both ranks projected the same sums, and they are the rank-order sums
        assert np.array_equal(every[0], every[1])
        for t in range(4):
            parts = [torch.randn((K, M, M), generator=torch.Generator().manual_seed(100 * r + t)) * 10 ** (3 * r)
                     for r in range(2)]
            assert np.array_equal(every[rank][t], ordered_sum(parts).numpy())
