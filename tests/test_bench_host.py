"""Host-side logic of bench.py on CPU: multi-rank aggregation over gloo
(world size 2) and the algorithmic FLOP counts of the factor kernel."""
import os
import socket

import pytest

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(1.5 + rank)   # rank 1 is the slow one
    bench.barrier()
    q.put((rank, t, bench.dist_env()))
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [2.5, 2.5]
    assert out[0][2] == (2, 0, 0) and out[1][2] == (2, 1, 1)


def test_single_process_aggregation_is_identity():
    assert bench.max_over_ranks(3.25) == 3.25


def _count_fold_factor_flops(K):
    """Count the kernel's FP64 operations by walking its loops (8 flops per
    complex multiply-add, 2 per complex-by-real scaling)."""
    f = 0
    for j in range(K):
        f += 2 * (K - j - 1)                 # column scaling by 1/L_jj
        n = K - j - 1
        f += 8 * n * (n + 1) // 2            # trailing update
    f += 8 * K * (K - 1) // 2                # forward substitution of y
    return f


@pytest.mark.parametrize("K", [1, 2, 16, 100])
def test_fold_factor_flop_count(K):
    assert bench.fold_factor_fp64_flops(K, 1) == pytest.approx(_count_fold_factor_flops(K))


def test_fp64_peak_is_derived_from_unit_counts():
    assert bench.FP64_PEAK_TFLOPS == pytest.approx(152 * 2 * 2 * 2.07e9 / 1e12)


def test_fp32_peak_is_derived_from_unit_counts():
    assert bench.FP32_PEAK_TFLOPS == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)


def _count_fold_factor_df_flops(K):
    """Walk the factorisation column by column: every trailing entry of step
    j takes one double-float complex multiply-subtract (4 error-free real
    multiply-accumulates of 1 FMUL + 3 FFMA + 8 FADD = 15 flops), so does
    every row of the right-hand side below j; the column scaling is 32 flops
    per entry; X = L^-1 takes one FP32 complex MAC (8 flops) per entry of the
    forward substitution."""
    f = 0
    for j in range(K):
        n = K - j - 1
        f += 60 * n * (n + 1) // 2           # trailing update, pairs
        f += 60 * n                          # y_i -= L_ij y_j, pairs
        f += 32 * n                          # L_ij = M_ij / L_jj
        f += 8 * n * (j + 1)                 # X_ic -= L_ij X_jc, c <= j
    return f


@pytest.mark.parametrize("K", [1, 2, 16, 100])
def test_fold_factor_df_flop_count(K):
    assert bench.fold_factor_df_flops(K, 1) == pytest.approx(_count_fold_factor_df_flops(K))


@pytest.mark.parametrize("K,B", [(1, 1), (16, 1), (100, 64)])
def test_fold_factor_method_flop_count(K, B):
    """Sec. III-C's work per frequency: complex Cholesky (sum over columns of
    the trailing updates, 8 flops per complex MAC: ~4/3 K^3), the inverse of
    the triangular factor (~4/3 K^3) and the rank-B fold (8 K^2 B)."""
    chol = sum(8 * (K - j - 1) * (K - j) / 2 for j in range(K))
    inv = sum(8 * (K - j - 1) * (K - j) / 2 for j in range(K))
    exact = chol + inv + 8 * K * K * B
    approx = bench.fold_factor_method_flops(K, 1, B)
    assert approx == pytest.approx(8.0 / 3.0 * K ** 3 + 8 * K * K * B)
    if K >= 16:
        assert abs(approx - exact) / exact < 0.1     # the K^3 terms dominate


def test_code_plane_bytes_by_iteration_walk():
    """Walk the Jz iterations of one coding call and count what each must move."""
    K, N, B, Jz = 7, 64, 3, 5
    F, P = N * (N // 2 + 1), N * N
    total = 0
    for t in range(Jz):
        first, last = t == 0, t == Jz - 1
        per = 0
        per += 0 if first else F * 8      # W^ read
        per += 0 if last else F * 8       # W^ written
        per += 0 if first else P * 4      # Gamma read
        per += P * 4                      # Gamma written
        per += F * 8 if last else 0       # Z~ kept for the fold
        per += P * 4 if last else 0       # U written
        total += B * K * per + B * F * 8 + K * F * 8
    assert bench.code_plane_bytes(K, N, B, Jz, True) == total
