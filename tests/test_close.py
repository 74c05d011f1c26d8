"""The element-wise comparison used by the GPU parity tests catches localised
defects that a whole-array norm misses (CPU only: the defects are planted in
arrays derived from the oracle, never in the CUDA path)."""
import numpy as np

import oracle
from tests.close import errors
from workloads import make_image, raw_filters


def _codes():
    D = oracle.normalize_filters(raw_filters(16, 5, 3).astype(np.float64))
    x = oracle.pad_to(make_image(56, 56, 4).astype(np.float64), 64, 64)
    return oracle.code_admm(x, oracle.filters_spectrum(D, 64, 64), 0.3, 1.0, 20).U


def test_one_wrong_self_conjugate_row_is_caught():
    U = _codes()
    S = np.fft.fft2(U)
    S[:, 0, :] *= 1.005                      # row k1 = 0 of every filter 0.5 % off
    bad = np.real(np.fft.ifft2(S))
    e = errors(bad, U)
    assert e["norm"] < 5e-3                  # a 1e-3 whole-array bar would pass it ...
    assert e["row"] > 4e-3                   # ... the per-row check does not


def test_one_filter_slightly_off_is_caught():
    U = _codes()
    bad = U.copy()
    bad[3] *= 1.005
    e = errors(bad, U)
    assert e["plane"] > 3e-3 and e["norm"] < 1e-3   # 30x the 1e-4 plane bar


def test_identical_arrays_have_zero_error():
    U = _codes()
    assert all(v == 0.0 for v in errors(U.copy(), U).values())


def test_empty_reference_planes_do_not_inflate_the_ratio():
    U = _codes()
    U[5] = 0.0
    near = U.copy()
    near[5, 10, 10] = 1e-9 * np.max(np.abs(U))   # rounding-size value in an empty plane
    assert errors(near, U)["plane"] < 1e-6
