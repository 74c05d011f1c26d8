"""The allocation-free entry point ocsc_code_noalloc gives the same codes as
the regular context path.

ocsc_code_noalloc is for callers that cannot allocate device memory while they
run: a plug-in living inside an application that already owns all device
memory through its own allocator, a latency-critical pipeline that must avoid
the device-wide synchronisation cudaMalloc / cudaFree can bring, or a service
that must not fail at run time for lack of memory.  Its scratch is a fixed
array inside the library, shared by every call, so these tests make two calls
in a row on different images and check both against ocsc_code on the same
dictionary, through the C ABI.  Both paths run the same kernels on the same
inputs, so the codes must agree bit for bit.  The cases include the largest
filter counts the array holds (the scratch then ends within a few KB of the
array's end) and an odd K.  The file name keeps it last in collection.
"""
import numpy as np
import pytest

from workloads import make_image, raw_filters

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("K,M,N,side", [(100, 11, 128, 100), (122, 11, 128, 110), (128, 8, 64, 60),
                                        (37, 5, 64, 57)])
def test_noalloc_matches_context_path_on_two_calls_in_a_row(K, M, N, side):
    _need_gpu()
    import paper_1706_06972_gb300 as pkg

    lam, rho, Jz = 1.0, 1.0, 20
    raw = raw_filters(K, M, 21 + K).astype(np.float64)
    D = (raw / np.sqrt(np.sum(raw ** 2, axis=(1, 2), keepdims=True))).astype(np.float32)
    xs = [torch.from_numpy(make_image(side, side, 900 + K + i)).cuda() for i in range(2)]

    learner = pkg.OCSC(K, M, lam, rho, fft_size=N, pad=N - side, Jz=Jz, Jd=2, max_batch=2)
    learner.set_dict(D, normalize=False)
    ref = learner.code(xs)
    learner.sync()
    learner.close()

    Dd = torch.from_numpy(D).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    us = [torch.full((K, N, N), float("nan"), device="cuda") for _ in range(2)]
    torch.cuda.synchronize()
    for i in range(2):
        pkg.ocsc_code_noalloc(xs[i].data_ptr(), side, side, Dd.data_ptr(), K, M, N, lam, rho, Jz,
                              us[i].data_ptr(), stream)
        torch.cuda.synchronize()
        diff = float((us[i] - ref[i]).abs().max())
        print(f"noalloc K={K} N={N} call {i}: max |u - u_ctx| = {diff:.3e}")
        assert bool(torch.isfinite(us[i]).all())
        assert torch.equal(us[i], ref[i])


def test_noalloc_second_call_takes_no_device_memory():
    """Once the first call has loaded the array and the kernels on this device,
    further calls leave the free device memory unchanged."""
    _need_gpu()
    import paper_1706_06972_gb300 as pkg

    K, M, N = 64, 7, 128
    raw = raw_filters(K, M, 5).astype(np.float64)
    D = torch.from_numpy((raw / np.sqrt(np.sum(raw ** 2, axis=(1, 2), keepdims=True))).astype(np.float32)).cuda()
    x = torch.from_numpy(make_image(100, 100, 31)).cuda()
    u = torch.empty((K, N, N), device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    pkg.ocsc_code_noalloc(x.data_ptr(), 100, 100, D.data_ptr(), K, M, N, 1.0, 1.0, 5, u.data_ptr(), stream)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        pkg.ocsc_code_noalloc(x.data_ptr(), 100, 100, D.data_ptr(), K, M, N, 1.0, 1.0, 5, u.data_ptr(), stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_sizes_beyond_its_array():
    _need_gpu()
    import paper_1706_06972_gb300 as pkg

    x = torch.zeros((128, 128), device="cuda")
    D = torch.zeros((128, 3, 3), device="cuda")
    u = torch.zeros((128, 128, 128), device="cuda")
    for K in (123, 128):   # more than 32 MiB of scratch at N = 128
        with pytest.raises(pkg.OCSCError) as e:
            pkg.ocsc_code_noalloc(x.data_ptr(), 128, 128, D.data_ptr(), K, 3, 128, 1.0, 1.0, 5,
                                  u.data_ptr(), torch.cuda.current_stream().cuda_stream)
        assert e.value.status == 6 and "scratch" in str(e.value)
