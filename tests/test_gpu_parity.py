"""Parity of the CUDA path with the FP64 oracle on the same seeded inputs.

All GPU work goes through the C ABI (libocsc.so via the ctypes binding).
Tolerances come from FP32 arithmetic: FFTs of N x N planes carry a relative
error of a few eps32 * log2(N^2) (eps32 = 6e-8), and the ADMM iterates
propagate it through Jz = 50 code iterations and Jd = 10 dictionary
iterations; the dictionary solve adds the FP32 triangular products with the
inverse of the Cholesky factor (factored in double-float, FP32 hi + lo pairs
of ~48 bits; FP64 for K > 128), whose error grows with the condition number of
A + rho I.
The bars below are those of the method statement: relative objective 1e-4 on
the FP32 path, and norm-relative code / dictionary errors 1e-3.
"""
import numpy as np
import pytest

import oracle
from workloads import WORKLOADS, make_image, raw_filters

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OBJ_TOL = 1e-4      # relative objective, FP32 path
REL_TOL = 1e-3      # norm-relative code and dictionary errors


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def rel(a, b):
    a = np.asarray(a)
    a = a.astype(np.complex128) if np.iscomplexobj(a) else a.astype(np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def run_gpu(images, raw, K, M, lam, rho, N, Jz, Jd, batch=1, normalize=True, **opts):
    import paper_1706_06972_gb300 as pkg

    learner = pkg.OCSC(K, M, lam, rho, fft_size=N, Jz=Jz, Jd=Jd, max_batch=batch, **opts)
    learner.set_dict(raw, normalize=normalize)
    codes, dicts = [], []
    for s in range(0, len(images), batch):
        xs = [torch.from_numpy(np.ascontiguousarray(im, np.float32)).cuda() for im in images[s:s + batch]]
        us = learner.code(xs)
        learner.update_dict()
        codes.extend([u.cpu().numpy() for u in us])
        dicts.append(learner.get_dict())
    learner.close()
    return codes, dicts


def run_oracle(images, raw, N, lam, rho, Jz, Jd, batch=1, **flags):
    st = oracle.init_state(np.asarray(raw, np.float64), N, N, lam, rho, **flags)
    codes, dicts, coding_dicts = [], [], []
    for s in range(0, len(images), batch):
        coding_dicts.append(oracle.published_filters(st))
        res = [oracle.code(st, im, Jz) for im in images[s:s + batch]]
        oracle.update_dict(st, res, Jd)
        codes.extend([r.U for r in res])
        dicts.append(oracle.published_filters(st))
    return codes, dicts, coding_dicts


def surrogate_objective(codes, coding_dicts, images, N, lam, batch):
    vals = []
    for i, (U, x) in enumerate(zip(codes, images)):
        D = coding_dicts[i // batch]
        vals.append(oracle.sample_objective(D, U, oracle.pad_to(np.asarray(x, np.float64), N, N), lam))
    return float(np.mean(vals))


# --- FFT building block ------------------------------------------------------

@pytest.mark.parametrize("N", [64, 96, 128, 144, 192, 256, 288, 384, 512, 576])
def test_fft_building_block_matches_numpy(N):
    _need_gpu()
    import paper_1706_06972_gb300 as pkg

    learner = pkg.OCSC(2, 3, 1.0, 1.0, fft_size=N)
    rng = np.random.default_rng(N)
    x = rng.standard_normal((3, N, N)).astype(np.float32)   # odd count: unpaired last plane
    X = learner.fft2_r2c(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = np.fft.rfft2(x.astype(np.float64))
    assert rel(X, ref) < 2e-6
    back = learner.fft2_c2r(torch.from_numpy(ref.astype(np.complex64)).cuda()).cpu().numpy()
    assert rel(back, x) < 2e-6
    learner.close()


# --- one sample, config-1 sizes ----------------------------------------------

def test_single_sample_code_and_update():
    _need_gpu()
    w = WORKLOADS["plain_64_k16"]
    imgs = [w.image(0)]
    raw = w.filters0()
    codes, dicts = run_gpu(imgs, raw, w.K, w.M, w.lam, w.rho, 64, w.Jz, w.Jd, pad=w.pad)
    ocodes, odicts, _ = run_oracle(imgs, raw, 64, w.lam, w.rho, w.Jz, w.Jd)
    assert rel(codes[0], ocodes[0]) < REL_TOL
    assert rel(dicts[0], odicts[0]) < REL_TOL
    norms = np.sqrt(np.sum(dicts[0].astype(np.float64) ** 2, axis=(1, 2)))
    assert np.all(norms <= 1 + 1e-6)


# --- whole online pass, 20 images 64x64, K=16 ----------------------------------

def test_online_pass_plain_64_k16():
    _need_gpu()
    w = WORKLOADS["plain_64_k16"]
    imgs = [w.image(i) for i in range(w.n_images)]
    raw = w.filters0()
    codes, dicts = run_gpu(imgs, raw, w.K, w.M, w.lam, w.rho, 64, w.Jz, w.Jd, pad=w.pad)
    ocodes, odicts, ocd = run_oracle(imgs, raw, 64, w.lam, w.rho, w.Jz, w.Jd)
    for t in range(len(imgs)):
        assert rel(codes[t], ocodes[t]) < REL_TOL, t
        assert rel(dicts[t], odicts[t]) < REL_TOL, t
    gcd = [oracle.normalize_filters(raw)] + dicts[:-1]
    f_gpu = surrogate_objective(codes, gcd, imgs, 64, w.lam, 1)
    f_orc = surrogate_objective(ocodes, ocd, imgs, 64, w.lam, 1)
    assert abs(f_gpu - f_orc) / abs(f_orc) < OBJ_TOL
    xs = [oracle.pad_to(np.asarray(x, np.float64), 64, 64) for x in imgs]
    F_gpu = oracle.objective(dicts[-1], codes, xs, w.lam)
    F_orc = oracle.objective(odicts[-1], ocodes, xs, w.lam)
    assert abs(F_gpu - F_orc) / abs(F_orc) < OBJ_TOL


# --- full size: 100x100 in 128x128, K=100 filters 11x11 (sampled) -------------

def test_plain_100in128_k100_first_samples():
    """The bench workload at its full size: the first two samples and updates
    of the stream, compared with the oracle sample by sample."""
    _need_gpu()
    w = WORKLOADS["plain_100in128_k100"]
    imgs = [w.image(i) for i in range(2)]
    raw = w.filters0()
    codes, dicts = run_gpu(imgs, raw, w.K, w.M, w.lam, w.rho, 128, w.Jz, w.Jd, pad=w.pad)
    ocodes, odicts, ocd = run_oracle(imgs, raw, 128, w.lam, w.rho, w.Jz, w.Jd)
    for t in range(2):
        assert rel(codes[t], ocodes[t]) < REL_TOL, t
        assert rel(dicts[t], odicts[t]) < REL_TOL, t
    gcd = [oracle.normalize_filters(raw)] + dicts[:-1]
    f_gpu = surrogate_objective(codes, gcd, imgs, 128, w.lam, 1)
    f_orc = surrogate_objective(ocodes, ocd, imgs, 128, w.lam, 1)
    assert abs(f_gpu - f_orc) / abs(f_orc) < OBJ_TOL


# --- edge cases ------------------------------------------------------------------

def _small_images(n, h, w, seed):
    return [make_image(h, w, seed + i) for i in range(n)]


@pytest.mark.parametrize("case", [
    dict(K=15, M=5, lam=0.5, rho=1.0, Jz=20, Jd=5, n=3, hw=(64, 64), pad=0),      # odd K
    dict(K=4, M=1, lam=0.2, rho=2.0, Jz=10, Jd=3, n=2, hw=(40, 50), pad=0),       # 1x1 filters, rectangular
    dict(K=8, M=7, lam=0.0, rho=1.0, Jz=15, Jd=4, n=2, hw=(57, 57), pad=6),       # lambda = 0, zero padding
    dict(K=6, M=4, lam=1.0, rho=0.5, Jz=1, Jd=1, n=2, hw=(64, 64), pad=0),        # single iterations
    dict(K=33, M=3, lam=0.3, rho=1.0, Jz=8, Jd=3, n=2, hw=(100, 90), pad=2),      # K > 32, N = 128
    dict(K=7, M=5, lam=0.5, rho=1.0, Jz=12, Jd=4, n=2, hw=(230, 200), pad=10),    # N = 256, odd K
    dict(K=4, M=3, lam=0.5, rho=1.0, Jz=8, Jd=3, n=2, hw=(400, 300), pad=10),     # N = 512
    dict(K=9, M=11, lam=1.0, rho=1.0, Jz=10, Jd=4, n=2, hw=(256, 256), pad=32),   # N = 288 = 2^5 3^2
    dict(K=5, M=5, lam=0.5, rho=1.0, Jz=10, Jd=4, n=2, hw=(80, 70), pad=10),      # N = 96 = 2^5 3
    dict(K=6, M=5, lam=0.5, rho=1.0, Jz=10, Jd=4, n=2, hw=(130, 120), pad=10),    # N = 144 = 2^4 3^2
    dict(K=4, M=5, lam=0.5, rho=1.0, Jz=8, Jd=3, n=2, hw=(180, 175), pad=10),     # N = 192 = 2^6 3
    dict(K=3, M=5, lam=0.5, rho=1.0, Jz=6, Jd=3, n=2, hw=(370, 360), pad=10),     # N = 384 = 2^7 3
    dict(K=2, M=3, lam=0.5, rho=1.0, Jz=5, Jd=2, n=2, hw=(560, 500), pad=10),     # N = 576 = 2^6 3^2
])
def test_edge_cases_match_oracle(case):
    _need_gpu()
    h, wd = case["hw"]
    imgs = _small_images(case["n"], h, wd, 77)
    raw = raw_filters(case["K"], case["M"], 5)
    N = next(n for n in (64, 96, 128, 144, 192, 256, 288, 384, 512, 576) if n >= max(h, wd) + case["pad"])
    codes, dicts = run_gpu(imgs, raw, case["K"], case["M"], case["lam"], case["rho"], N,
                           case["Jz"], case["Jd"], pad=case["pad"])
    ocodes, odicts, _ = run_oracle(imgs, raw, N, case["lam"], case["rho"], case["Jz"], case["Jd"])
    for t in range(case["n"]):
        assert rel(codes[t], ocodes[t]) < REL_TOL, t
        assert rel(dicts[t], odicts[t]) < REL_TOL, t


def test_fold_of_more_samples_than_one_chunk_matches_oracle():
    """A mini-batch of 20 samples: the fold stages pending codes in chunks of
    16, so the running sums cross a chunk boundary before the factorisation."""
    _need_gpu()
    imgs = _small_images(20, 48, 48, 1700)
    raw = raw_filters(12, 5, 1701)
    codes, dicts = run_gpu(imgs, raw, 12, 5, 0.5, 1.0, 64, 8, 4, batch=20, pad=0)
    ocodes, odicts, _ = run_oracle(imgs, raw, 64, 0.5, 1.0, 8, 4, batch=20)
    assert max(rel(codes[t], ocodes[t]) for t in range(20)) < REL_TOL
    assert rel(dicts[0], odicts[0]) < REL_TOL


@pytest.mark.parametrize("K", [1, 3, 5, 127, 128])
def test_factor_panel_edges_match_oracle(K):
    """The per-frequency factorisation works on panels of 4 columns with the
    next panel factored ahead: K = 1 (a single pivot), 3 and 5 (ragged last
    panel; trailing triangles smaller than two panels), 127 and 128 (ragged or
    full last panel at the largest in-shared-memory size).  Two updates."""
    _need_gpu()
    imgs = _small_images(2, 56, 56, 700 + K)
    raw = raw_filters(K, 5, 900 + K)
    codes, dicts = run_gpu(imgs, raw, K, 5, 0.5, 1.0, 64, 8, 4, pad=0)
    ocodes, odicts, _ = run_oracle(imgs, raw, 64, 0.5, 1.0, 8, 4)
    for t in range(2):
        assert rel(codes[t], ocodes[t]) < REL_TOL, t
        assert rel(dicts[t], odicts[t]) < REL_TOL, t


def test_minibatch_fold_matches_oracle():
    _need_gpu()
    imgs = _small_images(6, 64, 64, 200)
    raw = raw_filters(12, 6, 9)
    codes, dicts = run_gpu(imgs, raw, 12, 6, 0.5, 1.0, 64, 20, 6, batch=3, pad=0)
    ocodes, odicts, _ = run_oracle(imgs, raw, 64, 0.5, 1.0, 20, 6, batch=3)
    for t in range(6):
        assert rel(codes[t], ocodes[t]) < REL_TOL
    for u in range(2):
        assert rel(dicts[u], odicts[u]) < REL_TOL


@pytest.mark.parametrize("flags,gflags,lam,rho", [
    (dict(warm_start=False), dict(warm_start=0), 0.5, 1.0),
    (dict(rho_convention="paper"), dict(rho_convention=1), 0.005, 0.01),
])
def test_reading_flags_match_oracle(flags, gflags, lam, rho):
    _need_gpu()
    imgs = _small_images(3, 64, 64, 300)
    raw = raw_filters(10, 5, 11)
    codes, dicts = run_gpu(imgs, raw, 10, 5, lam, rho, 64, 15, 5, pad=0, **gflags)
    ocodes, odicts, _ = run_oracle(imgs, raw, 64, lam, rho, 15, 5, **flags)
    for t in range(3):
        assert rel(codes[t], ocodes[t]) < REL_TOL
        assert rel(dicts[t], odicts[t]) < REL_TOL


def test_deterministic_reruns():
    _need_gpu()
    imgs = _small_images(3, 64, 64, 400)
    raw = raw_filters(16, 8, 13)
    a = run_gpu(imgs, raw, 16, 8, 1.0, 1.0, 64, 10, 4, pad=0)
    b = run_gpu(imgs, raw, 16, 8, 1.0, 1.0, 64, 10, 4, pad=0)
    for x, y in zip(a[0] + a[1], b[0] + b[1]):
        assert np.array_equal(x, y)


# --- host-side error handling (no kernel ever sees a bad argument) -------------

def test_error_statuses():
    _need_gpu()
    import paper_1706_06972_gb300 as pkg

    with pytest.raises(pkg.OCSCError) as e:
        pkg.OCSC(0, 3, 1.0, 1.0)
    assert e.value.status == 6
    with pytest.raises(pkg.OCSCError) as e:
        pkg.OCSC(4, 3, 1.0, 0.0)
    assert e.value.status == 1
    learner = pkg.OCSC(4, 3, 1.0, 1.0, fft_size=64, pad=0, max_batch=1)
    with pytest.raises(pkg.OCSCError) as e:      # 100x100 does not map to N = 64
        learner.code([torch.zeros((100, 100), device="cuda")])
    assert e.value.status == 6
    learner.code([torch.zeros((64, 64), device="cuda")])
    with pytest.raises(pkg.OCSCError) as e:      # pending would exceed max_batch
        learner.code([torch.zeros((64, 64), device="cuda")])
    assert e.value.status == 5
    with pytest.raises(pkg.OCSCError) as e:      # infeasible filters without normalisation
        learner.set_dict(np.full((4, 3, 3), 2.0, np.float32), normalize=False)
    assert e.value.status == 1
    learner.update_dict()
    learner.sync()
    learner.close()


# --- objective kernel and mini-batches ------------------------------------------

@pytest.mark.parametrize("name,N", [("plain_64_k16", 64), ("plain_100in128_k100", 128),
                                    ("batched_mixed_k100", 256), ("batched_mixed_k100", 288),
                                    ("batched_mixed_k100", 512)])
def test_objective_matches_oracle_evaluation(name, N):
    """The GPU objective of eq. (ocsc0) equals the oracle's FP64 evaluation of
    the same dictionary and codes (Parseval on the half spectrum, padding)."""
    _need_gpu()
    import paper_1706_06972_gb300 as pkg

    w = WORKLOADS[name]
    learner = pkg.OCSC(w.K, w.M, w.lam, w.rho, fft_size=N, pad=w.pad, Jz=10, Jd=w.Jd, max_batch=2)
    learner.set_dict(w.filters0(), normalize=True)
    side = N // 2 if N >= 256 else None
    imgs = [w.image(7), w.image(8)] if side is None else [make_image(side, side, 70 + N + i) for i in range(2)]
    xs = [torch.from_numpy(im).cuda() for im in imgs]
    us = learner.code(xs)
    f_gpu = learner.objective(xs, us)
    D = learner.get_dict().astype(np.float64)
    for im, u, fg in zip(imgs, us, f_gpu):
        fo = oracle.sample_objective(D, u.cpu().numpy().astype(np.float64),
                                     oracle.pad_to(np.asarray(im, np.float64), N, N), w.lam)
        assert abs(fg - fo) / abs(fo) < 1e-5
    learner.drop_pending()
    learner.code([xs[0]])     # pending was cleared: room again
    learner.close()


def test_larger_minibatch_matches_oracle():
    _need_gpu()
    imgs = _small_images(16, 64, 64, 500)
    raw = raw_filters(24, 7, 17)
    codes, dicts = run_gpu(imgs, raw, 24, 7, 0.5, 1.0, 64, 20, 6, batch=8, pad=0)
    ocodes, odicts, _ = run_oracle(imgs, raw, 64, 0.5, 1.0, 20, 6, batch=8)
    for t in range(16):
        assert rel(codes[t], ocodes[t]) < REL_TOL
    for u in range(2):
        assert rel(dicts[u], odicts[u]) < REL_TOL


# --- uneven sizes: size classes with the consensus dictionary step --------------

def test_size_classes_match_oracle():
    """Images of two padded sizes in one learner (reading R16): per-class
    histories and duals, V-step on the mean of the class crops; one batch
    leaves the 128 class idle (refactored with its new weight only)."""
    _need_gpu()
    import paper_1706_06972_gb300 as pkg

    K, M, lam, rho, Jz, Jd = 10, 7, 0.5, 1.0, 15, 5
    sides = [[50, 100, 50], [100, 100], [50]]
    raw = raw_filters(K, M, 23)
    learner = pkg.OCSC(K, M, lam, rho, fft_sizes=[64, 128], pad=6, Jz=Jz, Jd=Jd, max_batch=3)
    learner.set_dict(raw, normalize=True)
    st = oracle.init_multi(np.asarray(raw, np.float64), [(64, 64), (128, 128)], lam, rho)
    seed = 900
    for batch in sides:
        imgs = [make_image(s, s + 7 if s == 100 else s, seed + i) for i, s in enumerate(batch)]
        seed += 10
        us = learner.code([torch.from_numpy(im).cuda() for im in imgs])
        learner.update_dict()
        D = learner.get_dict()
        res = {}
        for im, u in zip(imgs, us):
            N = 64 if max(im.shape) + 6 <= 64 else 128
            r = oracle.code_multi(st, im, (N, N), Jz)
            res.setdefault((N, N), []).append(r)
            assert u.shape[-1] == N
            assert rel(u.cpu().numpy(), r.U) < REL_TOL
        oracle.update_dict_multi(st, res, Jd)
        assert rel(D, st.V) < REL_TOL
    learner.close()


# --- checkpoint ------------------------------------------------------------------

def test_checkpoint_resumes_bit_identically():
    """A learner restored from a checkpoint continues exactly like the one that
    saved it (two size classes, so every per-class array is in the state)."""
    _need_gpu()
    import paper_1706_06972_gb300 as pkg

    K, M = 8, 5
    raw = raw_filters(K, M, 61)
    mk = lambda: pkg.OCSC(K, M, 0.5, 1.0, fft_sizes=[64, 128], pad=4, Jz=8, Jd=3, max_batch=2)
    a = mk()
    a.set_dict(raw, normalize=True)
    imgs = [torch.from_numpy(make_image(s, s, 700 + i)).cuda() for i, s in enumerate([50, 90, 40, 100, 60, 70])]
    for s in range(0, 4, 2):
        a.code(imgs[s:s + 2], want_codes=False)
        a.update_dict()
    state = a.get_state()
    b = mk()
    b.set_state(state)
    assert np.array_equal(a.get_dict(), b.get_dict())
    ua = a.code(imgs[4:6])
    a.update_dict()
    ub = b.code(imgs[4:6])
    b.update_dict()
    for x, y in zip(ua, ub):
        assert torch.equal(x, y)
    assert np.array_equal(a.get_dict(), b.get_dict())
    assert a.get_state() == b.get_state()
    a.code(imgs[:1], want_codes=False)
    with pytest.raises(pkg.OCSCError) as e:     # pending samples
        a.get_state()
    assert e.value.status == 5
    c = pkg.OCSC(K, M, 0.5, 1.0, fft_sizes=[64], pad=4, Jz=8, Jd=3, max_batch=2)
    with pytest.raises(pkg.OCSCError) as e:     # another shape
        c.set_state(state)
    assert e.value.status == 1
    for x in (a, b, c):
        x.close()


# --- tensor-core history fold (precision variants) ----------------------------------

class _StateHeader(__import__("ctypes").Structure):
    """Mirror of the checkpoint header (OCSC_MAX_FFT_SIZES = 12 classes)."""
    import ctypes as _c
    _fields_ = [("magic", _c.c_uint32), ("format", _c.c_uint32), ("K", _c.c_int32), ("M", _c.c_int32),
                ("ncls", _c.c_int32), ("N", _c.c_int32 * 12), ("rho_convention", _c.c_int32),
                ("return_feasible", _c.c_int32), ("warm_start", _c.c_int32), ("precision", _c.c_int32),
                ("lam", _c.c_double), ("rho", _c.c_double), ("n_seen", _c.c_int64), ("version", _c.c_uint64),
                ("class_seen", _c.c_int64 * 12)]


def _history_from_state(state, K, M, N, precision):
    """A = A_hi + A_lo of a one-class state as [F, K, K] (lower triangle)."""
    import ctypes

    NH = N // 2 + 1
    F = N * NH
    T = K * (K + 1) // 2
    TS = T + (T & 1)
    off = ctypes.sizeof(_StateHeader) + K * M * M * 4 + 4 * K * F * 8
    A = np.frombuffer(state, np.complex64, F * TS, off).reshape(F, TS).astype(np.complex128)
    off += F * TS * 8
    if precision:
        A = A + np.frombuffer(state, np.complex64, F * TS, off).reshape(F, TS)
    full = np.zeros((F, K, K), np.complex128)
    for j in range(K):
        o = j * (2 * K - j + 1) // 2
        full[:, j:, j] = A[:, o:o + K - j]
    return full


# History tolerances from the operand rounding: FP32 codes carry ~1e-6 of the
# coding path's own error; one BF16 word keeps 8 significant bits (unit
# roundoff 2^-9 = 2e-3 per factor of every product); the split hi + lo keeps
# 16 (the dropped lo*lo term and the rounding of lo are ~2^-16 = 1.5e-5).
@pytest.mark.parametrize("precision,a_tol,d_tol", [(0, 1e-5, 1e-3), (1, 1e-2, 2e-2), (2, 6e-5, 1e-3)])
def test_history_fold_precision_matches_oracle(precision, a_tol, d_tol):
    """Two rank-8 folds: the FP32 path, BF16 tensor-core products (1 term)
    and split-BF16 products (3 terms), each with the history checked against
    the FP64 oracle's A^p entry by entry (lower triangle) and the dictionary
    and objective after each update."""
    _need_gpu()
    import paper_1706_06972_gb300 as pkg

    K, M, N, B, lam, rho, Jz, Jd = 24, 5, 64, 8, 0.5, 1.0, 15, 5
    raw = raw_filters(K, M, 71)
    imgs = [make_image(60, 60, 1200 + i) for i in range(2 * B)]
    lr = pkg.OCSC(K, M, lam, rho, fft_size=N, pad=4, Jz=Jz, Jd=Jd, max_batch=B, precision=precision)
    lr.set_dict(raw, normalize=True)
    st = oracle.init_state(np.asarray(raw, np.float64), N, N, lam, rho)
    NH = N // 2 + 1
    k1, k2 = np.divmod(np.arange(N * NH), NH)
    codes, coding = [], []
    for s in range(0, 2 * B, B):
        coding.append(oracle.published_filters(st))
        us = lr.code([torch.from_numpy(im).cuda() for im in imgs[s:s + B]])
        lr.update_dict()
        D = lr.get_dict()
        res = [oracle.code(st, im, Jz) for im in imgs[s:s + B]]
        oracle.update_dict(st, res, Jd)
        codes.extend(u.cpu().numpy() for u in us)
        A = _history_from_state(lr.get_state(), K, M, N, precision)
        Ao = st.hist.A[k1, k2]
        low = np.tril(np.ones((K, K), bool))
        a_err = np.linalg.norm((A - Ao)[:, low]) / np.linalg.norm(Ao[:, low])
        d_err = rel(D, st.V)
        print(f"precision={precision} update={s // B}: history {a_err:.3e} dictionary {d_err:.3e}")
        assert a_err < a_tol, (precision, a_err)
        assert d_err < d_tol
    fo = surrogate_objective([r.U for r in res], [coding[-1]] * B, imgs[B:], N, lam, B)
    fg = surrogate_objective(codes[B:], [coding[-1]] * B, imgs[B:], N, lam, B)
    print(f"precision={precision}: relative objective {abs(fg - fo) / abs(fo):.3e}")
    assert abs(fg - fo) / abs(fo) < 1e-3
    lr.close()


@pytest.mark.parametrize("K,precision,a_tol,d_tol", [(136, 0, 1e-5, 1e-3), (136, 2, 6e-5, 1e-3),
                                                     (256, 0, 1e-5, 1e-3), (256, 1, 1e-2, 3e-2)])
def test_large_K_factor_matches_oracle(K, precision, a_tol, d_tol):
    """K > 128: blocked FP64 Cholesky through the global workspace, D-step by
    substitution, FP32 or tensor-core fold (two 128-row blocks).  With one
    BF16 word per operand the history bound applies to the first fold only:
    later codes are computed against a dictionary that already differs from
    the oracle's by the BF16 error, and the difference compounds."""
    _need_gpu()
    import paper_1706_06972_gb300 as pkg

    M, N, B, lam, rho, Jz, Jd = 5, 64, 4, 0.5, 1.0, 8, 4
    raw = raw_filters(K, M, 91)
    imgs = [make_image(60, 60, 1400 + i) for i in range(2 * B)]
    lr = pkg.OCSC(K, M, lam, rho, fft_size=N, pad=4, Jz=Jz, Jd=Jd, max_batch=B, precision=precision)
    lr.set_dict(raw, normalize=True)
    st = oracle.init_state(np.asarray(raw, np.float64), N, N, lam, rho)
    NH = N // 2 + 1
    k1, k2 = np.divmod(np.arange(N * NH), NH)
    low = np.tril(np.ones((K, K), bool))
    for s in range(0, 2 * B, B):
        lr.code([torch.from_numpy(im).cuda() for im in imgs[s:s + B]], want_codes=False)
        lr.update_dict()
        D = lr.get_dict()
        oracle.update_dict(st, [oracle.code(st, im, Jz) for im in imgs[s:s + B]], Jd)
        A = _history_from_state(lr.get_state(), K, M, N, precision)
        Ao = st.hist.A[k1, k2]
        a_err = np.linalg.norm((A - Ao)[:, low]) / np.linalg.norm(Ao[:, low])
        d_err = rel(D, st.V)
        print(f"K={K} precision={precision} update={s // B}: history {a_err:.3e} dictionary {d_err:.3e}")
        assert a_err < a_tol or (precision == 1 and s > 0)
        assert d_err < d_tol
    lr.close()


# --- batching machinery: CUDA graphs and the autotuner -----------------------------

def _run_sequence(pkg, graphs, autotune, precision=0):
    K, M = 10, 5
    raw = raw_filters(K, M, 81)
    lr = pkg.OCSC(K, M, 0.5, 1.0, fft_sizes=[64, 256], pad=4, Jz=6, Jd=3, max_batch=2,
                  graphs=graphs, autotune=autotune, precision=precision)
    lr.set_dict(raw, normalize=True)
    codes = []
    for r in range(4):   # the same chunk shapes every pass: captured at the second pass
        xs = [torch.from_numpy(make_image(s, s, 1500 + 10 * r + i)).cuda() for i, s in enumerate([50, 200])]
        us = lr.code(xs)
        lr.update_dict()
        codes.extend(u.cpu().numpy() for u in us)
    D = lr.get_dict()
    counters = lr.counters()
    tun = {N: lr.tuning(N) for N in (64, 256)}
    lr.close()
    return codes, D, counters, tun


def test_graph_replay_matches_direct_launches():
    _need_gpu()
    import paper_1706_06972_gb300 as pkg

    a = _run_sequence(pkg, graphs=0, autotune=0)
    b = _run_sequence(pkg, graphs=1, autotune=0)
    for x, y in zip(a[0], b[0]):
        assert np.array_equal(x, y)
    assert np.array_equal(a[1], b[1])
    assert a[2]["graph_launches"] == 0 and b[2]["graph_launches"] == 6   # 2 classes x rounds 2, 3, 4
    assert a[2]["kernel_launches"] == b[2]["kernel_launches"]


@pytest.mark.parametrize("precision", [0, 1])
def test_autotuned_tiles_do_not_change_results(precision):
    """Every tuned tile shape performs the same operations in the same order."""
    _need_gpu()
    import paper_1706_06972_gb300 as pkg

    a = _run_sequence(pkg, graphs=0, autotune=0, precision=precision)
    b = _run_sequence(pkg, graphs=0, autotune=1, precision=precision)
    for x, y in zip(a[0], b[0]):
        assert np.array_equal(x, y)
    assert np.array_equal(a[1], b[1])
    t = b[3]
    print("tuned tiles:", t)
    assert t[64]["fold_threads"] in (256, 512) and t[256]["fold_threads"] in (256, 512)
    assert t[256]["spat_cb"] in (8, 16) and t[64]["spat_cb"] == 0
    if precision:
        assert t[64]["gram_sc"] in (32, 64, 128)


# --- evaluation of Sec. IV: objective terms, PSNR, relative change, passes ---------

def test_objective_terms_psnr_and_rel_diff_match_oracle():
    _need_gpu()
    import paper_1706_06972_gb300 as pkg

    K, M, N, lam = 8, 5, 64, 0.5
    raw = raw_filters(K, M, 111)
    lr = pkg.OCSC(K, M, lam, 1.0, fft_sizes=[64, 96], pad=4, Jz=12, Jd=3, max_batch=2)
    lr.set_dict(raw, normalize=True)
    imgs = [make_image(s, s, 1600 + i) for i, s in enumerate([60, 80])]
    xs = [torch.from_numpy(im).cuda() for im in imgs]
    us = lr.code(xs)
    r2, l1 = lr.objective_terms(xs, us)
    ps = lr.psnr(xs, us, peak=4.0)
    D = lr.get_dict().astype(np.float64)
    for im, u, a, b, q in zip(imgs, us, r2, l1, ps):
        Nn = u.shape[-1]
        U = u.cpu().numpy().astype(np.float64)
        xp = oracle.pad_to(np.asarray(im, np.float64), Nn, Nn)
        r = oracle.reconstruct(D, U) - xp
        assert abs(a - float(np.sum(r * r))) / float(np.sum(r * r)) < 1e-5
        assert abs(b - float(np.sum(np.abs(U)))) / float(np.sum(np.abs(U))) < 1e-12
        assert abs(q - oracle.psnr(D, U, xp, peak=4.0)) < 1e-4
    v = lr.rel_diff(us[0], 0.75 * us[0])
    assert abs(v - 0.25) < 1e-7
    assert abs(lr.rel_diff(us[0], us[0] * 0 + us[0])) == 0.0
    lr.drop_pending()
    lr.close()


def test_fit_stops_by_the_rule_of_the_paper():
    """Passes over four images until the codes and the dictionary change by
    less than tol between passes (a loose tol so that it stops quickly)."""
    _need_gpu()
    import paper_1706_06972_gb300 as pkg

    K, M = 4, 5
    lr = pkg.OCSC(K, M, 0.5, 1.0, fft_size=64, pad=4, Jz=20, Jd=5, max_batch=2)
    lr.set_dict(raw_filters(K, M, 121), normalize=True)
    xs = [torch.from_numpy(make_image(60, 60, 1700 + i)).cuda() for i in range(4)]
    res = lr.fit(xs, max_passes=40, tol=5e-2, batch=2)
    assert res["stopped"] and res["pass"] >= 1
    assert res["code_change"] < 5e-2 and res["dict_change"] < 5e-2
    order = pkg.filter_order(lr.get_dict())
    assert sorted(order.tolist()) == list(range(K))
    lr.close()


# --- recursion variant of the history (eq. C_update, reading R3) ---------------------

# The printed recursion comes with the printed rho P: C_t = (A_t + (rho P / t) I)^-1,
# and DictOCSC runs with the matching penalty rho / t (reading R23).  (With the
# spatial rho = 1 the ridge starts at 1 against |z|^2 ~ 1e4 and the oracle's own
# FP64 recursion loses its accuracy within ten samples.)  C is double-float on the
# GPU (~48 bits) and FP64 in the oracle; the FP32 codes and b carry the usual
# coding error.
RECURSION_DICT_TOL = REL_TOL

@pytest.mark.parametrize("wname,N,nimg,batch", [("plain_64_k16", 64, 20, 1), ("plain_64_k16", 64, 12, 4),
                                                ("plain_100in128_k100", 128, 2, 1)])
def test_recursion_history_matches_oracle(wname, N, nimg, batch):
    """history = 1: C from the printed Sherman-Morrison recursion (a ridge
    decaying as rho / t), against the oracle's recursion mode sample by sample."""
    _need_gpu()
    w = WORKLOADS[wname]
    imgs = [w.image(i) for i in range(nimg)]
    raw = w.filters0()
    codes, dicts = run_gpu(imgs, raw, w.K, w.M, w.lam, w.rho, N, w.Jz, w.Jd, batch=batch, pad=w.pad, history=1,
                           rho_convention=1)
    ocodes, odicts, ocd = run_oracle(imgs, raw, N, w.lam, w.rho, w.Jz, w.Jd, batch=batch, history="recursion",
                                     rho_convention="paper")
    derr = [rel(dicts[t], odicts[t]) for t in range(len(dicts))]
    cerr = [rel(codes[t], ocodes[t]) for t in range(nimg)]
    gcd = [oracle.normalize_filters(raw)] + dicts[:-1]
    f_gpu = surrogate_objective(codes, gcd, imgs, N, w.lam, batch)
    f_orc = surrogate_objective(ocodes, ocd, imgs, N, w.lam, batch)
    print(f"recursion {wname} B={batch}: dictionary max {max(derr):.2e}, code max {max(cerr):.2e}, "
          f"objective {abs(f_gpu - f_orc) / abs(f_orc):.2e}; per update {[f'{x:.1e}' for x in derr]}")
    assert max(derr) < RECURSION_DICT_TOL and max(cerr) < RECURSION_DICT_TOL
    assert abs(f_gpu - f_orc) / abs(f_orc) < OBJ_TOL


def test_recursion_history_rejects_unsupported_setups():
    _need_gpu()
    import paper_1706_06972_gb300 as pkg

    with pytest.raises(pkg.OCSCError) as e:
        pkg.OCSC(8, 5, 0.5, 1.0, fft_sizes=[64, 128], history=1, rho_convention=1)
    assert e.value.status == 6
    with pytest.raises(pkg.OCSCError) as e:
        pkg.OCSC(8, 5, 0.5, 1.0, fft_size=64, history=1, precision=1, rho_convention=1)
    assert e.value.status == 6
    with pytest.raises(pkg.OCSCError) as e:
        pkg.OCSC(8, 5, 0.5, 1.0, fft_size=64, history=1)
    assert e.value.status == 6
