"""The allocation-free entry point ocsc_code_noalloc gives the same codes as
the regular context path.

ocsc_code_noalloc is for callers that cannot allocate device memory while they
run: a plug-in living inside an application that already owns all device
memory through its own allocator, a latency-critical pipeline that must avoid
the device-wide synchronisation cudaMalloc / cudaFree can bring, or a service
that must not fail at run time for lack of memory.  Its scratch is a fixed
array inside the library, shared by every call, so this test makes two calls in
a row on different images and checks both against ocsc_code on the same
dictionary, through the C ABI.  The file name keeps it last in collection.
"""
import numpy as np
import pytest

from workloads import make_image, raw_filters

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_TOL = 1e-3  # the norm-relative code tolerance of the parity tests


def _rel(a, b):
    a = a.double()
    b = b.double()
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def test_noalloc_matches_context_path_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1706_06972_gb300 as pkg

    K, M, N, lam, rho, Jz = 100, 11, 128, 1.0, 1.0, 50
    raw = raw_filters(K, M, 21).astype(np.float64)
    D = (raw / np.sqrt(np.sum(raw ** 2, axis=(1, 2), keepdims=True))).astype(np.float32)
    xs = [torch.from_numpy(make_image(100, 100, 900 + i)).cuda() for i in range(2)]

    learner = pkg.OCSC(K, M, lam, rho, fft_size=N, pad=10, Jz=Jz, Jd=10, max_batch=2)
    learner.set_dict(D, normalize=False)
    ref = learner.code(xs)
    learner.sync()

    Dd = torch.from_numpy(D).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    for i in range(2):
        u = torch.full((K, N, N), float("nan"), device="cuda")
        pkg.ocsc_code_noalloc(xs[i].data_ptr(), 100, 100, Dd.data_ptr(), K, M, N, lam, rho, Jz,
                              u.data_ptr(), stream)
        torch.cuda.synchronize()
        assert bool(torch.isfinite(u).all())
        assert _rel(u, ref[i]) < REL_TOL
    learner.close()


def test_noalloc_rejects_sizes_beyond_its_array():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1706_06972_gb300 as pkg

    x = torch.zeros((128, 128), device="cuda")
    D = torch.zeros((128, 3, 3), device="cuda")
    u = torch.zeros((128, 128, 128), device="cuda")
    with pytest.raises(pkg.OCSCError) as e:   # K = 128 at N = 128 needs more than 32 MiB
        pkg.ocsc_code_noalloc(x.data_ptr(), 128, 128, D.data_ptr(), 128, 3, 128, 1.0, 1.0, 5,
                              u.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert e.value.status == 6 and "scratch" in str(e.value)
