"""Pins of the FP64 oracle against brute force, closed forms and invariants.

Each test fixes one step of the oracle with something other than the oracle's
own formula: dense spatial-domain solves built from the convolution matrix
T(.) of Sec. III-D eq. (csc2sc), an explicit DFT matrix, textbook FISTA, exact
special cases, and invariants of the method (feasibility, running means).
A plausible slip in the oracle (a dropped 1/P, a missing conjugate, a wrong
sign in the dual update, a transposed history matrix) fails at least one.
"""
import numpy as np
import pytest

import oracle
from tests import brute

RNG = np.random.default_rng(1234)


def _rand_filters(K, M, rng=RNG):
    return oracle.normalize_filters(rng.standard_normal((K, M, M)))


# --- convolution theorem (Sec. II-C) -----------------------------------------

def test_fft_convolution_equals_direct_circular_convolution():
    rng = np.random.default_rng(1)
    for (n1, n2, m) in [(6, 7, 3), (8, 8, 5), (5, 9, 2)]:
        D = rng.standard_normal((2, m, m))
        U = rng.standard_normal((2, n1, n2))
        direct = brute.circ_conv2(D[0], U[0]) + brute.circ_conv2(D[1], U[1])
        np.testing.assert_allclose(oracle.reconstruct(D, U), direct, rtol=0, atol=1e-12)


def test_sample_objective_matches_direct_evaluation():
    rng = np.random.default_rng(2)
    D = rng.standard_normal((3, 3, 3))
    U = rng.standard_normal((3, 8, 8)) * (rng.random((3, 8, 8)) < 0.3)
    x = rng.standard_normal((8, 8))
    r = x - sum(brute.circ_conv2(D[k], U[k]) for k in range(3))
    want = 0.5 * np.sum(r * r) + 0.7 * np.sum(np.abs(U))
    assert abs(oracle.sample_objective(D, U, x, 0.7) - want) < 1e-11 * abs(want)


# --- code Z~-step: closed form vs dense spatial solve ---------------------------

@pytest.mark.parametrize("rho", [1.0, 0.37, 5.0])
def test_code_zstep_equals_dense_spatial_solve(rho):
    """8x8 image, K=2 filters 3x3: the per-frequency rank-one+rho*I solve equals
    the dense normal equations (T^T T + rho I) z = T^T x + rho w in space."""
    rng = np.random.default_rng(3)
    n = 8
    D = rng.standard_normal((2, 3, 3))
    x = rng.standard_normal((n, n))
    W = rng.standard_normal((2, n, n))
    T = np.hstack([brute.conv_matrix(D[k], n, n) for k in range(2)])
    z = np.linalg.solve(T.T @ T + rho * np.eye(2 * n * n), T.T @ x.ravel() + rho * W.ravel())
    Dh = oracle.filters_spectrum(D, n, n)
    Zh = oracle.code_zstep(Dh, oracle.fft2(x), oracle.fft2(W), rho)
    Zs = oracle.ifft2(Zh)
    assert np.max(np.abs(Zs.imag)) < 1e-12
    np.testing.assert_allclose(Zs.real.ravel(), z, rtol=0, atol=1e-11)


def test_code_zstep_non_square_domain():
    rng = np.random.default_rng(31)
    n1, n2 = 6, 10
    D = rng.standard_normal((3, 3, 3))
    x = rng.standard_normal((n1, n2))
    W = rng.standard_normal((3, n1, n2))
    T = np.hstack([brute.conv_matrix(D[k], n1, n2) for k in range(3)])
    z = np.linalg.solve(T.T @ T + 2.0 * np.eye(3 * n1 * n2), T.T @ x.ravel() + 2.0 * W.ravel())
    Zh = oracle.code_zstep(oracle.filters_spectrum(D, n1, n2), oracle.fft2(x), oracle.fft2(W), 2.0)
    np.testing.assert_allclose(oracle.ifft2(Zh).real.ravel(), z, rtol=0, atol=1e-11)


# --- history fold (eqs. A_update, B_update) ----------------------------------

def test_fold_is_running_mean_and_batch_invariant():
    rng = np.random.default_rng(4)
    K, n = 3, 4
    Zs = [rng.standard_normal((K, n, n)) + 1j * rng.standard_normal((K, n, n)) for _ in range(5)]
    xs = [rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) for _ in range(5)]
    h1 = oracle.History.zeros(K, n, n)
    for Z, x in zip(Zs, xs):
        h1 = oracle.fold_history(h1, [Z], [x])
    h2 = oracle.fold_history(oracle.History.zeros(K, n, n), Zs[:2], xs[:2])
    h2 = oracle.fold_history(h2, Zs[2:], xs[2:])
    # direct mean, entry by entry
    A = np.zeros((n, n, K, K), complex)
    b = np.zeros((n, n, K), complex)
    for Z, x in zip(Zs, xs):
        for p1 in range(n):
            for p2 in range(n):
                for i in range(K):
                    b[p1, p2, i] += x[p1, p2] * np.conj(Z[i, p1, p2]) / 5
                    for j in range(K):
                        A[p1, p2, i, j] += np.conj(Z[i, p1, p2]) * Z[j, p1, p2] / 5
    for h in (h1, h2):
        assert h.n == 5
        np.testing.assert_allclose(h.A, A, atol=1e-12)
        np.testing.assert_allclose(h.b, b, atol=1e-12)
    # Hermitian PSD per frequency
    assert np.allclose(h1.A, np.conj(np.swapaxes(h1.A, -1, -2)))
    assert np.min(np.linalg.eigvalsh(h1.A)) > -1e-10


def test_proposition1_per_frequency_form():
    """Prop. 1: the frequency objective of eq. (ocsc) equals the per-frequency
    quadratic form in A^p, b^p plus a constant independent of D~."""
    rng = np.random.default_rng(5)
    K, n, t = 3, 4, 4
    Zs = [rng.standard_normal((K, n, n)) + 1j * rng.standard_normal((K, n, n)) for _ in range(t)]
    xs = [rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) for _ in range(t)]
    h = oracle.fold_history(oracle.History.zeros(K, n, n), Zs, xs)
    P = n * n
    const = sum(np.sum(np.abs(x) ** 2) for x in xs) / (2 * t * P)
    for _ in range(3):
        Dh = rng.standard_normal((K, n, n)) + 1j * rng.standard_normal((K, n, n))
        lhs = sum(np.sum(np.abs(x - np.sum(Dh * Z, axis=0)) ** 2) for Z, x in zip(Zs, xs)) / (2 * t * P)
        d = np.moveaxis(Dh, 0, -1)
        quad = np.einsum("xyi,xyij,xyj->", np.conj(d), h.A, d).real
        lin = np.einsum("xyi,xyi->", np.conj(h.b), d).real
        rhs = (quad - 2 * lin) / (2 * P) + const
        assert abs(lhs - rhs) < 1e-10 * abs(lhs)


# --- D~-step: eq. (sub_d_sol) vs dense spatial solve ----------------------------

def _dense_dict_system(Zsp, xs, n):
    t = len(xs)
    K = Zsp[0].shape[0]
    G = np.zeros((K * n * n, K * n * n))
    r = np.zeros(K * n * n)
    for Z, x in zip(Zsp, xs):
        S = np.hstack([brute.conv_matrix(Z[k], n, n) for k in range(K)])
        G += S.T @ S / t
        r += S.T @ x.ravel() / t
    return G, r


@pytest.mark.parametrize("rho", [1.0, 0.5])
def test_dstep_equals_dense_spatial_solve(rho):
    """One D~-step equals the dense normal equations of
    1/(2t) sum_i ||x_i - sum_k Z_ik (*) d_k||^2 + rho/2 sum_k ||d_k - (v_k - theta_k)||^2
    over full-size real filters d_k."""
    rng = np.random.default_rng(6)
    K, n, M, t = 2, 6, 3, 3
    Zsp = [rng.standard_normal((K, n, n)) for _ in range(t)]
    xs = [rng.standard_normal((n, n)) for _ in range(t)]
    h = oracle.fold_history(oracle.History.zeros(K, n, n),
                            [oracle.fft2(Z) for Z in Zsp], [oracle.fft2(x) for x in xs])
    V = rng.standard_normal((K, M, M)) * 0.3
    theta = rng.standard_normal((K, n, n)) * 0.2
    _, _, Dh = oracle.dict_ocsc(h, V, oracle.fft2(theta), rho, 1)
    G, r = _dense_dict_system(Zsp, xs, n)
    v = oracle.pad_to(V, n, n).ravel()
    d = np.linalg.solve(G + rho * np.eye(K * n * n), r + rho * (v - theta.ravel()))
    Ds = oracle.ifft2(Dh)
    assert np.max(np.abs(Ds.imag)) < 1e-12
    np.testing.assert_allclose(Ds.real.ravel(), d, atol=1e-10)


def test_dstep_paper_rho_convention_is_rho_times_P():
    rng = np.random.default_rng(7)
    K, n, M = 2, 4, 2
    Zs = [oracle.fft2(rng.standard_normal((K, n, n))) for _ in range(2)]
    xs = [oracle.fft2(rng.standard_normal((n, n))) for _ in range(2)]
    h = oracle.fold_history(oracle.History.zeros(K, n, n), Zs, xs)
    V = rng.standard_normal((K, M, M))
    th = oracle.fft2(rng.standard_normal((K, n, n)))
    _, _, Da = oracle.dict_ocsc(h, V, th, 0.01, 1, rho_convention="paper")
    # dense: rho' = rho * P  in the spatial penalty
    Zsp = [oracle.ifft2(Z).real for Z in Zs]
    xsp = [oracle.ifft2(x).real for x in xs]
    G, r = _dense_dict_system(Zsp, xsp, n)
    v = oracle.pad_to(V, n, n).ravel()
    th_s = oracle.ifft2(th).real.ravel()
    rp = 0.01 * n * n
    d = np.linalg.solve(G + rp * np.eye(K * n * n), r + rp * (v - th_s))
    np.testing.assert_allclose(oracle.ifft2(Da).real.ravel(), d, atol=1e-10)


# --- V-step: Proposition 2 ---------------------------------------------------

@pytest.mark.parametrize("scale", [0.05, 3.0])
def test_proposition2_is_constrained_argmin(scale):
    """Prop. 2 equals projected gradient on min ||y~ - F(pad V)||^2, ||V|| <= 1,
    with the DFT as an explicit matrix (no FFT)."""
    rng = np.random.default_rng(8)
    n, M = 6, 3
    y = rng.standard_normal((n, n)) * scale
    yh = oracle.fft2(y)
    # closed form through the oracle's V-step pieces
    V_cf = oracle.project_filters(oracle.crop(oracle.ifft2(yh[None]).real, M))[0]
    # brute force
    Fm = brute.dft_matrix_2d(n, n)
    sup = np.zeros((n, n), bool)
    sup[:M, :M] = True
    Fs = Fm[:, sup.ravel()]
    yv = yh.ravel()
    v = np.zeros(M * M)
    L = 2 * np.linalg.norm(Fs, 2) ** 2
    for _ in range(3000):
        g = 2 * np.real(np.conj(Fs).T @ (Fs @ v - yv))
        v = v - g / L
        nv = np.linalg.norm(v)
        if nv > 1:
            v /= nv
    np.testing.assert_allclose(V_cf.ravel(), v, atol=1e-9)
    assert np.linalg.norm(V_cf) <= 1 + 1e-12


# --- whole code ADMM: convergence, special cases ------------------------------

def test_code_admm_reaches_fista_optimum_and_residuals_vanish():
    rng = np.random.default_rng(9)
    n, K, M, lam = 8, 2, 3, 0.2
    D = _rand_filters(K, M, rng)
    x = rng.standard_normal((n, n))
    T = np.hstack([brute.conv_matrix(D[k], n, n) for k in range(K)])
    z_f = brute.fista_lasso(T, x.ravel(), lam, 20000)
    f_fista = 0.5 * np.sum((x.ravel() - T @ z_f) ** 2) + lam * np.sum(np.abs(z_f))
    res = oracle.code_admm(x, oracle.filters_spectrum(D, n, n), lam, 1.0, 3000)
    f_admm = oracle.sample_objective(D, res.U, x, lam)
    assert abs(f_admm - f_fista) <= 1e-8 * abs(f_fista)
    assert res.primal[-1] < 1e-8 and res.dual[-1] < 1e-8
    assert res.primal[-1] < res.primal[5] and res.max_imag < 1e-12


def test_identity_filter_reduces_to_soft_threshold():
    """K=1, M=1, D=[1]: the code problem is elementwise, U* = S_lam(x)."""
    rng = np.random.default_rng(10)
    x = rng.standard_normal((8, 8)) * 2
    res = oracle.code_admm(x, oracle.filters_spectrum(np.ones((1, 1, 1)), 8, 8), 0.5, 1.0, 200)
    want = np.where(np.abs(x) > 0.5, x - 0.5 * np.sign(x), 0.0)
    np.testing.assert_allclose(res.U[0], want, atol=1e-12)


def test_zero_lambda_identity_filter_reproduces_sample():
    rng = np.random.default_rng(11)
    x = rng.standard_normal((4, 6))
    res = oracle.code_admm(x, oracle.filters_spectrum(np.ones((1, 1, 1)), 4, 6), 0.0, 1.0, 100)
    np.testing.assert_allclose(res.U[0], x, atol=1e-12)


def test_planted_codes_are_recovered():
    """x = sum_k D_k (*) Z_k with known unit-norm filters and sparse Z: coding
    with the true filters recovers the support of Z."""
    rng = np.random.default_rng(12)
    n, K, M = 32, 3, 5
    D = _rand_filters(K, M, rng)
    Z = np.zeros((K, n, n))
    for k in range(K):
        idx = rng.choice(n * n, 6, replace=False)
        Z[k].ravel()[idx] = rng.choice([-1, 1], 6) * rng.uniform(3, 5, 6)
    x = oracle.reconstruct(D, Z)
    res = oracle.code_admm(x, oracle.filters_spectrum(D, n, n), 0.05, 1.0, 400)
    est = np.abs(res.U) > 0.5
    true = Z != 0
    tp = np.sum(est & true)
    f1 = 2 * tp / (np.sum(est) + np.sum(true))
    assert f1 >= 0.95
    np.testing.assert_allclose(res.U[true], Z[true], rtol=0.1)


# --- dictionary ADMM (Algorithm 2) converges to the constrained optimum --------

def test_dictocsc_converges_to_constrained_optimum():
    rng = np.random.default_rng(13)
    K, n, M, t = 2, 6, 2, 3
    Zsp = [rng.standard_normal((K, n, n)) * (rng.random((K, n, n)) < 0.5) for _ in range(t)]
    xs = [rng.standard_normal((n, n)) * 2 for _ in range(t)]
    h = oracle.fold_history(oracle.History.zeros(K, n, n),
                            [oracle.fft2(Z) for Z in Zsp], [oracle.fft2(x) for x in xs])
    V0 = np.zeros((K, M, M))
    V, _, _ = oracle.dict_ocsc(h, V0, np.zeros((K, n, n), complex), 1.0, 4000)
    # projected gradient on min 1/(2t) sum ||x_i - sum_k Z_ik (*) V_k||^2, ||V_k|| <= 1
    sup = np.zeros((n, n), bool)
    sup[:M, :M] = True
    S_list = [np.hstack([brute.conv_matrix(Z[k], n, n)[:, sup.ravel()] for k in range(K)])
              for Z in Zsp]
    G = sum(S.T @ S for S in S_list) / t
    r = sum(S.T @ x.ravel() for S, x in zip(S_list, xs)) / t
    L = np.linalg.norm(G, 2)
    v = np.zeros(K * M * M)
    for _ in range(20000):
        v = v - (G @ v - r) / L
        for k in range(K):
            seg = v[k * M * M:(k + 1) * M * M]
            nv = np.linalg.norm(seg)
            if nv > 1:
                v[k * M * M:(k + 1) * M * M] = seg / nv
    np.testing.assert_allclose(V.reshape(-1), v, atol=1e-6)


# --- Algorithm 3 invariants -----------------------------------------------------

def test_online_loop_feasibility_and_real_iterates():
    rng = np.random.default_rng(14)
    n, K, M = 16, 3, 4
    imgs = [rng.standard_normal((12, 12)) for _ in range(4)]
    raw = rng.standard_normal((K, M, M))
    for batch in (1, 2):
        st, codes = oracle.run(imgs, raw, n, n, 0.3, 1.0, 20, 5, batch=batch)
        assert st.hist.n == 4 and st.updates == 4 // batch
        nrm = np.sqrt(np.sum(st.V ** 2, axis=(1, 2)))
        assert np.all(nrm <= 1 + 1e-12)
        full = oracle.ifft2(st.Dh)
        assert np.max(np.abs(full.imag)) < 1e-12
        assert np.max(np.abs(full.real[:, M:, :])) < 1e-12
        assert np.max(np.abs(full.real[:, :, M:])) < 1e-12
        assert all(c.max_imag < 1e-10 for c in codes)


def test_initial_filters_unit_norm():
    raw = RNG.standard_normal((5, 4, 4)) * 7
    V = oracle.normalize_filters(raw)
    np.testing.assert_allclose(np.sqrt(np.sum(V ** 2, axis=(1, 2))), 1.0, atol=1e-14)
    np.testing.assert_allclose(V * np.linalg.norm(raw[0]), raw * (np.linalg.norm(raw[0]) /
                               np.sqrt(np.sum(raw ** 2, axis=(1, 2), keepdims=True))), atol=1e-12)


def test_filters_recovered_from_known_codes():
    """Images synthesised from planted unit-norm filters and known sparse codes:
    folding the true codes and running DictOCSC recovers the filters."""
    rng = np.random.default_rng(17)
    n, K, M = 24, 2, 4
    Dtrue = _rand_filters(K, M, rng)
    Zs, xs = [], []
    for _ in range(10):
        Z = np.zeros((K, n, n))
        for k in range(K):
            idx = rng.choice(n * n, 8, replace=False)
            Z[k].ravel()[idx] = rng.standard_normal(8) * 3
        Zs.append(Z)
        xs.append(brute.circ_conv2(Dtrue[0], Z[0]) + brute.circ_conv2(Dtrue[1], Z[1]))
    h = oracle.fold_history(oracle.History.zeros(K, n, n),
                            [oracle.fft2(Z) for Z in Zs], [oracle.fft2(x) for x in xs])
    V, _, _ = oracle.dict_ocsc(h, np.zeros((K, M, M)), np.zeros((K, n, n), complex), 1.0, 1000)
    np.testing.assert_allclose(V, Dtrue, atol=1e-7)


def test_learning_reduces_objective_on_planted_dictionary():
    """Online learning from a random D_0 on images synthesised from planted
    filters lowers the objective of held-out samples versus D_0."""
    rng = np.random.default_rng(15)
    n, K, M = 24, 2, 4
    Dtrue = _rand_filters(K, M, rng)

    def sample():
        Z = np.zeros((K, n, n))
        for k in range(K):
            idx = rng.choice(n * n, 8, replace=False)
            Z[k].ravel()[idx] = rng.standard_normal(8) * 3
        return oracle.reconstruct(Dtrue, Z)

    train = [sample() for _ in range(40)]
    test = [sample() for _ in range(3)]
    raw = rng.standard_normal((K, M, M))
    st, _ = oracle.run(train, raw, n, n, 0.1, 1.0, 60, 20, batch=1)

    def test_obj(D):
        Dh = oracle.filters_spectrum(D, n, n)
        Us = [oracle.code_admm(x, Dh, 0.1, 1.0, 200).U for x in test]
        return oracle.objective(D, Us, test, 0.1)

    assert test_obj(st.V) < 0.8 * test_obj(oracle.normalize_filters(raw))


# --- eq. (C_update): the printed Sherman-Morrison recursion --------------------

def test_printed_sherman_morrison_recursion_has_decaying_ridge():
    """Reading R3: the recursion of eq. (C_update) yields (A_t + (rho P / t) I)^-1,
    not the (A_t + rho P I)^-1 that eq. (sub_d_sol) defines; the hot path uses
    the definition (a factorisation), so this pins the reading, not a kernel."""
    rng = np.random.default_rng(16)
    K, rP = 4, 3.0
    zs = [rng.standard_normal(K) + 1j * rng.standard_normal(K) for _ in range(6)]
    C = None
    A = np.zeros((K, K), complex)
    for t, z in enumerate(zs, start=1):
        zc = np.conj(z)[:, None]
        zr = z[None, :]
        if t == 1:
            C = np.eye(K) / rP - (zc @ zr) / (rP * (rP + (zr @ zc)[0, 0]))
        else:
            C = (t / (t - 1)) * (C - (C @ zc @ zr @ C) / ((t - 1) + (zr @ C @ zc)[0, 0]))
        A = (1 - 1 / t) * A + (1 / t) * (zc @ zr)
    decaying = np.linalg.inv(A + (rP / len(zs)) * np.eye(K))
    fixed = np.linalg.inv(A + rP * np.eye(K))
    assert np.max(np.abs(C - decaying)) < 1e-10
    assert np.max(np.abs(C - fixed)) > 1e-2


# --- size classes (reading R16) ---------------------------------------------------

def test_one_class_consensus_equals_dictocsc():
    rng = np.random.default_rng(18)
    K, n, M = 3, 8, 3
    raw = rng.standard_normal((K, M, M))
    imgs = [rng.standard_normal((n, n)) for _ in range(3)]
    single = oracle.init_state(raw, n, n, 0.3, 1.0)
    multi = oracle.init_multi(raw, [(n, n)], 0.3, 1.0)
    for im in imgs:
        rs = oracle.code(single, im, 15)
        rm = oracle.code_multi(multi, im, (n, n), 15)
        np.testing.assert_array_equal(rs.U, rm.U)
        oracle.update_dict(single, [rs], 6)
        oracle.update_dict_multi(multi, {(n, n): [rm]}, 6)
        np.testing.assert_allclose(multi.V, single.V, atol=1e-13)


def test_two_class_consensus_reaches_pooled_constrained_optimum():
    """Two FFT sizes: many consensus iterations reach the minimiser of the
    pooled objective (1/n) sum_i 1/2 ||x_i - sum_k Z_ik (*) V_k||^2 over
    feasible V, each convolution circular on its sample's own grid."""
    rng = np.random.default_rng(19)
    K, M = 2, 2
    sizes = [(5, 5), (6, 6)]
    data = {s: [] for s in sizes}
    for s, cnt in zip(sizes, (2, 3)):
        for _ in range(cnt):
            Z = rng.standard_normal((K,) + s) * (rng.random((K,) + s) < 0.6)
            x = rng.standard_normal(s) * 2
            data[s].append((Z, x))
    st = oracle.init_multi(np.ones((K, M, M)), sizes, 0.1, 1.0)
    for s in sizes:
        c = st.classes[s]
        c.hist = oracle.fold_history(c.hist, [oracle.fft2(Z) for Z, _ in data[s]],
                                     [oracle.fft2(x) for _, x in data[s]])
    st.V = np.zeros((K, M, M))
    V = oracle.dict_ocsc_multi(st, 6000)
    # brute force: projected gradient with dense convolution matrices
    n_tot = sum(len(v) for v in data.values())
    G = np.zeros((K * M * M, K * M * M))
    r = np.zeros(K * M * M)
    for s in sizes:
        sup = np.zeros(s, bool)
        sup[:M, :M] = True
        for Z, x in data[s]:
            S = np.hstack([brute.conv_matrix(Z[k], *s)[:, sup.ravel()] for k in range(K)])
            G += S.T @ S / n_tot
            r += S.T @ x.ravel() / n_tot
    L = np.linalg.norm(G, 2)
    v = np.zeros(K * M * M)
    for _ in range(30000):
        v = v - (G @ v - r) / L
        for k in range(K):
            seg = v[k * M * M:(k + 1) * M * M]
            nv = np.linalg.norm(seg)
            if nv > 1:
                v[k * M * M:(k + 1) * M * M] = seg / nv
    np.testing.assert_allclose(V.reshape(-1), v, atol=1e-6)


# --- evaluation of Sec. IV -------------------------------------------------------

def test_psnr_closed_form():
    """Reconstruction off by a constant c everywhere: ||x_rec - x||^2 = c^2 P, so
    PSNR = 10 log10(peak^2 / c^2) whatever the image."""
    rng = np.random.default_rng(3)
    K, M, n = 3, 3, 16
    D = rng.standard_normal((K, M, M))
    U = rng.standard_normal((K, n, n))
    x_rec = oracle.reconstruct(D, U)
    c = 0.25
    val = oracle.psnr(D, U, x_rec - c, peak=2.0)
    assert abs(val - 10.0 * np.log10(4.0 / c ** 2)) < 1e-9


def test_rel_change_closed_form():
    a = np.arange(1.0, 7.0).reshape(2, 3)
    assert abs(oracle.rel_change(a, 0.9 * a) - 0.1) < 1e-15
    assert oracle.rel_change(a, a) == 0.0
    assert oracle.rel_change(np.zeros(3), np.ones(3)) == float("inf")


def test_filter_order_by_variance():
    """2 x 2 filters: entries 1,2,3,4 have variance 5/3 (mean 2.5, squared
    deviations 2.25 + 0.25 + 0.25 + 2.25 over 3); constant filters 0."""
    D = np.stack([np.array([[1.0, 2.0], [3.0, 4.0]]),
                  np.full((2, 2), 7.0),
                  np.array([[0.0, 0.0], [0.0, 3.0]])])        # mean 0.75, var (3*0.5625+5.0625)/3 = 2.25
    assert list(oracle.filter_order(D)) == [1, 0, 2]


def test_oracle_recursion_mode_equals_decaying_ridge_solve():
    """sm_fold (the recursion variant of the oracle) against the definition it
    reduces to: C_t = (A_t + (r / t) I)^-1 with A_t the running mean, over a
    batch fold of 3 samples after 2 earlier ones; and one DictOCSC step with it
    against the explicit solve."""
    rng = np.random.default_rng(21)
    K, n = 3, 4
    r = 0.7
    Zs = [rng.standard_normal((K, n, n)) + 1j * rng.standard_normal((K, n, n)) for _ in range(5)]
    xs = [rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) for _ in range(5)]
    h = oracle.History.zeros(K, n, n)
    h = oracle.fold_history(h, Zs[:2], xs[:2])
    C = oracle.sm_fold(None, Zs[:2], 0, r)
    h = oracle.fold_history(h, Zs[2:], xs[2:])
    C = oracle.sm_fold(C, Zs[2:], 2, r)
    ref = np.linalg.inv(h.A + (r / 5) * np.eye(K))
    assert np.max(np.abs(C - ref)) < 1e-10
    V = oracle.normalize_filters(rng.standard_normal((K, 2, 2)))
    th = np.zeros((K, n, n), complex)
    _, _, Dh = oracle.dict_ocsc(h, V, th, r, 1, C=C)
    rhs = h.b + r * np.moveaxis(oracle.filters_spectrum(V, n, n), 0, -1)
    d = np.linalg.solve(h.A + (r / 5) * np.eye(K), rhs[..., None])[..., 0]
    assert np.max(np.abs(np.moveaxis(Dh, 0, -1) - d)) < 1e-10


def test_printed_recursion_with_the_fixed_penalty_diverges():
    """Reading R23: with C_t from eq. (C_update) (ridge r / t) but the fixed
    penalty rho on the right of eq. (sub_d_sol), each DictOCSC iteration scales
    the components of D~ in the null space of A_t (t < K samples) by about
    t - 1, so the iteration diverges; with the matching penalty rho / t it is an
    ADMM and stays bounded."""
    rng = np.random.default_rng(23)
    K, n, M, t = 6, 8, 3, 4
    Zs = [rng.standard_normal((K, n, n)) + 1j * rng.standard_normal((K, n, n)) for _ in range(t)]
    xs = [rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) for _ in range(t)]
    h = oracle.fold_history(oracle.History.zeros(K, n, n), Zs, xs)
    C = oracle.sm_fold(None, Zs, 0, 1.0)
    V = oracle.normalize_filters(rng.standard_normal((K, M, M)))
    th = np.zeros((K, n, n), complex)
    grow = []
    for iters in (10, 20):
        _, _, Dh = oracle.dict_ocsc(h, V, th, 1.0, iters, C=C)
        grow.append(np.abs(Dh).max())
    assert grow[1] / grow[0] > (t - 1.5) ** 10           # geometric, ratio ~ t - 1
    for iters in (10, 20):
        _, _, Dh = oracle.dict_ocsc(h, V, th, 1.0 / t, iters, C=C)
        assert np.abs(Dh).max() < 10.0


def test_recursion_mode_update_equals_factorised_admm_at_rho_over_t():
    """Two recursion-mode updates (batches of 2 and 3 samples, paper's rho P)
    against DictOCSC on np.linalg.inv(A_t + (rho P / t) I), the penalty rho / t
    and the scaled dual carried as rho Theta (reading R23)."""
    import types

    rng = np.random.default_rng(24)
    K, n, M, rho, Jd = 4, 6, 3, 0.05, 4
    raw = rng.standard_normal((K, M, M))
    res = [types.SimpleNamespace(Zh=rng.standard_normal((K, n, n)) + 1j * rng.standard_normal((K, n, n)),
                                 xh=rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
           for _ in range(5)]
    st = oracle.init_state(raw, n, n, 0.1, rho, rho_convention="paper", history="recursion")
    h = oracle.History.zeros(K, n, n)
    V, th = oracle.normalize_filters(raw), np.zeros((K, n, n), complex)
    for batch in (res[:2], res[2:]):
        oracle.update_dict(st, batch, Jd)
        nb = h.n
        h = oracle.fold_history(h, [r.Zh for r in batch], [r.xh for r in batch])
        if nb:
            th = th * (h.n / nb)
        V, th, _ = oracle.dict_ocsc(h, V, th, rho / h.n, Jd, rho_convention="paper")
        assert np.max(np.abs(st.V - V)) < 1e-10
        assert np.max(np.abs(st.thetah - th)) < 1e-10 * max(1.0, np.abs(th).max())


# --- the literal branches of Algorithm 2 (readings R6, R7) --------------------------

class _Coded:
    """A coded sample as update_dict takes it (spectra of given spatial codes)."""

    def __init__(self, Z, x):
        self.Zh = oracle.fft2(Z)
        self.xh = oracle.fft2(x)


def _project_rows(a, K, M):
    """alpha_k / max(||alpha_k||, 1) on a flat [K * M * M] vector."""
    out = a.copy()
    for k in range(K):
        seg = out[k * M * M:(k + 1) * M * M]
        out[k * M * M:(k + 1) * M * M] = seg / max(np.linalg.norm(seg), 1.0)
    return out


def _crop_flat(d, K, n, M):
    return d.reshape(K, n, n)[:, :M, :M].reshape(-1)


@pytest.mark.parametrize("rho", [1.0, 0.3])
def test_literal_return_publishes_the_last_dstep(rho):
    """return_feasible=False: Algorithm 2 returns D~_{t,J} and Algorithm 3
    publishes H(F^-1(D~_t)).  From a cold start (warm_start=False) with J = 2
    the D-steps are, by dense spatial solves over full-size filters,
      d1 = (G + rho I)^-1 r,          V1 = Prop. 2 of H(d1),  theta1 = d1 - pad(V1),
      d2 = (G + rho I)^-1 (r + rho (pad(V1) - theta1)),
    so the published filters are H(d2) and the coding spectrum is F(d2)."""
    rng = np.random.default_rng(31)
    K, n, M, t = 2, 6, 3, 3
    Zsp = [rng.standard_normal((K, n, n)) * (rng.random((K, n, n)) < 0.6) for _ in range(t)]
    xs = [rng.standard_normal((n, n)) * 2 for _ in range(t)]
    st = oracle.init_state(rng.standard_normal((K, M, M)), n, n, 0.1, rho, warm_start=False,
                           return_feasible=False)
    # a first update so that the cold start has something to discard
    oracle.update_dict(st, [_Coded(Zsp[0], xs[0])], 3)
    oracle.update_dict(st, [_Coded(Z, x) for Z, x in zip(Zsp[1:], xs[1:])], 2)
    G, r = _dense_dict_system(Zsp, xs, n)          # running mean over all t samples
    A = G + rho * np.eye(K * n * n)
    d1 = np.linalg.solve(A, r)
    v1 = np.zeros(K * n * n)
    v1.reshape(K, n, n)[:, :M, :M] = _project_rows(_crop_flat(d1, K, n, M), K, M).reshape(K, M, M)
    th1 = d1 - v1
    d2 = np.linalg.solve(A, r + rho * (v1 - th1))
    np.testing.assert_allclose(oracle.published_filters(st).reshape(-1), _crop_flat(d2, K, n, M), atol=1e-10)
    np.testing.assert_allclose(st.Dh, oracle.fft2(d2.reshape(K, n, n)), atol=1e-9)
    # the feasible V of the same update is Prop. 2 of H(d2 + theta1)
    np.testing.assert_allclose(st.V.reshape(-1), _project_rows(_crop_flat(d2 + th1, K, n, M), K, M), atol=1e-10)


def test_literal_return_tends_to_the_feasible_filters():
    """At the ADMM fixed point D~ = F(pad V): after many iterations the literal
    return and the feasible V coincide."""
    rng = np.random.default_rng(32)
    K, n, M = 2, 6, 2
    samples = [_Coded(rng.standard_normal((K, n, n)) * (rng.random((K, n, n)) < 0.5),
                      rng.standard_normal((n, n)) * 2) for _ in range(3)]
    st = oracle.init_state(rng.standard_normal((K, M, M)), n, n, 0.1, 1.0, return_feasible=False)
    oracle.update_dict(st, samples, 3000)
    np.testing.assert_allclose(oracle.published_filters(st), st.V, atol=1e-7)
    assert np.max(np.abs(oracle.ifft2(st.Dh).real[:, M:, :])) < 1e-7


def test_cold_start_of_the_multi_class_step_discards_the_previous_state():
    """warm_start=False with size classes (readings R6, R16): with J = 1 every
    class solves from V = 0, theta = 0, so the update gives Prop. 2 of the mean
    over classes of H(d_c), d_c = (w_c G_c + rho I)^-1 w_c r_c by dense spatial
    solves, whatever V and theta the earlier update left."""
    rng = np.random.default_rng(33)
    K, M, rho = 2, 2, 0.7
    sizes = [(5, 5), (6, 6)]
    st = oracle.init_multi(rng.standard_normal((K, M, M)), sizes, 0.1, rho, warm_start=False)
    data = {s: [] for s in sizes}
    first = {s: [] for s in sizes}
    for s, cnt in zip(sizes, (2, 1)):
        for j in range(cnt):
            Z = rng.standard_normal((K,) + s) * (rng.random((K,) + s) < 0.6)
            x = rng.standard_normal(s) * 2
            (first if j == 0 else data)[s].append((Z, x))
    oracle.update_dict_multi(st, {s: [_Coded(Z, x) for Z, x in first[s]] for s in sizes}, 4)
    oracle.update_dict_multi(st, {s: [_Coded(Z, x) for Z, x in data[s]] for s in sizes}, 1)
    n_tot = sum(len(first[s]) + len(data[s]) for s in sizes)
    alpha = np.zeros(K * M * M)
    for s in sizes:
        pairs = first[s] + data[s]
        G, r = _dense_dict_system([Z for Z, _ in pairs], [x for _, x in pairs], s[0])
        w = len(pairs) / n_tot
        d = np.linalg.solve(w * G + rho * np.eye(G.shape[0]), w * r)
        alpha += _crop_flat(d, K, s[0], M) / len(sizes)
    np.testing.assert_allclose(st.V.reshape(-1), _project_rows(alpha, K, M), atol=1e-10)
