"""Frequency-band sharding of the online dictionary step across ranks.

Proposition 1 (Sec. III-B) decouples the D-row systems of eq. (sub_d_sol) per
frequency, so each rank keeps the history A^p, b^p, its factorisation and the
D~-step of one band of frequencies (rows k1 of the half spectrum); only the
V-step of Proposition 2 couples the bands, through the support crop
H(F^-1(D~ + theta^)), a sum over frequencies.  One update of Algorithm 2 then
exchanges the codes' band rows once (all-to-all) and sums K M^2 floats per
dictionary-ADMM iteration (an all-reduce, done here as an all-gather added in
rank order, so that every rank holds the same bits).  The arithmetic runs in
the library's kernels (ocsc_band_*); this module only moves buffers.

Two drivers share the steps: ``band_update`` for one band context per rank
over a communicator (``TorchComm`` wraps torch.distributed), and
``band_update_local`` for several band contexts driven from one process (for
instance on one GPU).
"""
from __future__ import annotations


def band_partition(N: int, G: int):
    """G contiguous ranges [lo, hi) of k1 rows covering 0 .. N once, each with
    an even row count, as equal as possible (G <= N / 2)."""
    if G < 1 or G > N // 2:
        raise ValueError(f"{G} bands do not fit {N} rows in pairs")
    base, extra = divmod(N // 2, G)
    out, lo = [], 0
    for g in range(G):
        n = 2 * (base + (1 if g < extra else 0))
        out.append((lo, lo + n))
        lo += n
    return out


def ordered_sum(parts):
    """parts[0] + parts[1] + ... in that order (the same bits on every rank)."""
    total = parts[0].clone()
    for p in parts[1:]:
        total += p
    return total


class TorchComm:
    """The collectives band_update needs, over torch.distributed.  Tensors
    travel on the backend's device (CUDA for NCCL, the host for gloo) and come
    back on the device they were given on."""

    def __init__(self, group=None):
        import torch.distributed as dist

        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.device = "cuda" if dist.get_backend(group) == "nccl" else "cpu"

    def all_gather(self, x):
        import torch

        xr = (torch.view_as_real(x) if x.is_complex() else x).contiguous().to(self.device)
        out = [torch.empty_like(xr) for _ in range(self.world)]
        self.dist.all_gather(out, xr, group=self.group)
        out = [o.to(x.device) for o in out]
        return [torch.view_as_complex(o) for o in out] if x.is_complex() else out

    def all_to_all(self, send, counts_out, shape_of):
        """send[g] goes to rank g; returns recv[r] from rank r, whose leading
        size is counts_out[r] and trailing shape shape_of(r)."""
        import torch

        dist = self.dist
        home = send[0].device
        send_r = [torch.view_as_real(s).contiguous().to(self.device) for s in send]
        recv_r = [torch.empty((counts_out[r],) + tuple(shape_of(r)) + (2,), device=self.device,
                              dtype=send_r[0].dtype) for r in range(self.world)]
        if dist.get_backend(self.group) == "nccl":
            dist.all_to_all(recv_r, send_r, group=self.group)
        else:  # point-to-point pairs (gloo has no all-to-all)
            ops = []
            for peer in range(self.world):
                if peer == self.rank:
                    recv_r[peer].copy_(send_r[peer])
                    continue
                ops.append(dist.isend(send_r[peer], peer, group=self.group))
                ops.append(dist.irecv(recv_r[peer], peer, group=self.group))
            for op in ops:
                op.wait()
        return [torch.view_as_complex(r.to(home)) for r in recv_r]


def band_update(learner, comm, n_local: int, Jd: int):
    """One dictionary update of a band context (this rank's band: its
    (band_lo, band_hi) must be band_partition(N, world)[rank]) over `comm`.
    n_local: samples this rank coded since the last update (pending).  The
    mini-batch is every rank's samples in rank order."""
    import torch

    bands = band_partition(learner.N, comm.world)
    if tuple(learner.band_rows()) != bands[comm.rank]:
        raise ValueError(f"rank {comm.rank} owns rows {learner.band_rows()}, expected {bands[comm.rank]}")
    counts = [int(c.item()) for c in comm.all_gather(torch.tensor([float(n_local)]))]
    exports = [learner.band_export(lo, hi, n_local) for (lo, hi) in bands]
    lo, hi = bands[comm.rank]
    fb = (hi - lo) * (learner.N // 2 + 1)
    Zs = comm.all_to_all([e[0] for e in exports], counts, lambda r: (learner.K, fb))
    xs = comm.all_to_all([e[1] for e in exports], counts, lambda r: (fb,))
    learner.band_fold(torch.cat(Zs), torch.cat(xs))
    for t in range(Jd):
        part = learner.band_dict_step()
        learner.band_project(ordered_sum(comm.all_gather(part)), last=t == Jd - 1)
    learner.drop_pending()


def band_update_local(learners, n_locals, Jd: int):
    """The same update for G band contexts driven from one process:
    learners[g] owns band_partition(N, G)[g] and has n_locals[g] pending
    samples; the mini-batch is every context's samples in context order."""
    import torch

    G = len(learners)
    bands = band_partition(learners[0].N, G)
    exports = [[lr.band_export(lo, hi, n_locals[r]) for (lo, hi) in bands] for r, lr in enumerate(learners)]
    for g, lr in enumerate(learners):
        if tuple(lr.band_rows()) != bands[g]:
            raise ValueError(f"context {g} owns rows {lr.band_rows()}, expected {bands[g]}")
        lr.band_fold(torch.cat([exports[r][g][0] for r in range(G)]),
                     torch.cat([exports[r][g][1] for r in range(G)]))
    for t in range(Jd):
        total = ordered_sum([lr.band_dict_step() for lr in learners])
        for lr in learners:
            lr.band_project(total, last=t == Jd - 1)
    for lr in learners:
        lr.drop_pending()
