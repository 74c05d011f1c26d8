"""Plain FP64 CPU oracle of online convolutional sparse coding (OCSC).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run this module.  The product
path (the CUDA library and its Python binding) never calls it, and this module
imports nothing from the product package.

Everything is float64 / complex128 and uses the FULL N1 x N2 spectrum (no
Hermitian half-spectrum shortcut), numpy's FFT as the DFT primitive and
``numpy.linalg.inv`` as the per-frequency K x K inverse.  The forward DFT F is
unnormalised; F^-1 carries 1/P (P = N1*N2 pixels).  Convolution is circular on
the padded N1 x N2 domain; filters and images sit in the top-left corner.

Steps follow the paper:
  * code subproblem, Sec. II-C.1 eq. (fcsc_code), solved by the scaled-dual
    ADMM template of Sec. II-B eqs. (admm_aux, admm_dual);
  * history matrices A^p, b^p and their running-mean update,
    Sec. III-B eqs. (A_update, B_update);
  * dictionary ADMM DictOCSC, Algorithm 2, with the D-row solve
    eq. (sub_d_sol) and the V projection of Proposition 2;
  * the online loop, Algorithm 3;
  * the online objective, Sec. III eq. (ocsc0).

Readings taken where the paper is silent or inconsistent (each one is listed
with its justification in the design notes of this repository):
  R1  A^p = mean(conj(z) z^T), b^p = mean(x~(p) conj(z)); the D-row system is
      (A^p + rho I) d = b^p + rho (v^ - theta^)  (column-vector form of
      eq. sub_d_sol, derived from |x~(p) - z^T d|^2).
  R2  rho is a spatial-domain penalty for both ADMMs: the code system is
      (conj(d) d^T + rho I) and the D-row system (A + rho I); the paper's
      frequency-domain rho' relates by rho = rho' * P.  ``rho_convention=
      "paper"`` uses A + rho*P*I in the D-row solve as eq. (sub_d_sol) prints.
  R4  a mini-batch of B samples is folded as an exact running mean with
      weights n/(n+B) and 1/(n+B); B = 1 is eq. (A_update) exactly.
  R5  code ADMM starts from U = Gamma = 0, runs a fixed J_z iterations; the
      history uses Z~ from the last Z~-step, the returned code is U.
  R6  warm start: V and theta^ of DictOCSC carry over between updates
      (``warm_start=False`` restarts them at 0 as Algorithm 2 is printed).
  R7  the published dictionary is the feasible V_{t,J} and D~_t = F(V_{t,J})
      (``return_feasible=False`` publishes D~_{t,J} as Algorithm 2 returns).
  R9  filter support is the top-left [0,M) x [0,M) corner.
  R10 D~_0: raw N(0,1) spatial filters, each scaled to unit l2 norm.
  R14 soft-threshold maps |v| <= t to 0.

Parity of a learned dictionary on real images is unpinned (the paper prints
no numeric example); every step here is pinned piecewise by the tests in
``tests/test_oracle_pins.py`` against brute force and closed forms.
"""
from __future__ import annotations

import dataclasses

import numpy as np


# ----------------------------------------------------------------------------
# Domain helpers (Sec. II-C: zero-padding of filters to P, the crop operator H)
# ----------------------------------------------------------------------------

def fft2(a: np.ndarray) -> np.ndarray:
    """Unnormalised 2D DFT over the last two axes (F in Sec. II-C)."""
    return np.fft.fft2(a, axes=(-2, -1))


def ifft2(a: np.ndarray) -> np.ndarray:
    """Inverse 2D DFT with the 1/P factor (F^-1 in Sec. II-C)."""
    return np.fft.ifft2(a, axes=(-2, -1))


def pad_to(a: np.ndarray, n1: int, n2: int) -> np.ndarray:
    """Zero-pad the last two axes at the end to n1 x n2 (top-left placement)."""
    out = np.zeros(a.shape[:-2] + (n1, n2), dtype=np.float64)
    out[..., : a.shape[-2], : a.shape[-1]] = a
    return out


def crop(a: np.ndarray, m: int) -> np.ndarray:
    """The operator H of Sec. II-C: keep the [0,M) x [0,M) support."""
    return np.array(a[..., :m, :m], dtype=np.float64)


def soft_threshold(v: np.ndarray, t: float) -> np.ndarray:
    """Proximal map of t*|.|_1 (the U-step of the code ADMM); ties map to 0."""
    return np.sign(v) * np.maximum(np.abs(v) - t, 0.0)


def normalize_filters(raw: np.ndarray) -> np.ndarray:
    """Reading R10 of Algorithm 3's initialisation: each filter scaled to norm 1."""
    raw = np.asarray(raw, dtype=np.float64)
    nrm = np.sqrt(np.sum(raw * raw, axis=(-2, -1), keepdims=True))
    return raw / nrm


def filters_spectrum(V: np.ndarray, n1: int, n2: int) -> np.ndarray:
    """D~ = F(zero-padded filters), shape [K, n1, n2] complex."""
    return fft2(pad_to(V, n1, n2))


# ----------------------------------------------------------------------------
# Code update: Sec. II-C.1 eq. (fcsc_code) by ADMM (Sec. II-B)
# ----------------------------------------------------------------------------

def code_zstep(Dh: np.ndarray, xh: np.ndarray, Wh: np.ndarray, rho: float) -> np.ndarray:
    """Z~-step of the code ADMM, independently at every frequency p.

    With d = D~(p,:)^T and w^ = F(U - Gamma)(p), the augmented objective of
    eq. (fcsc_code) scaled by P gives  1/2|x~(p) - d^T z|^2 + rho/2 |z - w^|^2,
    whose normal equations are (conj(d) d^T + rho I) z = conj(d) x~(p) + rho w^.
    The matrix is rank one plus rho*I, so Sherman-Morrison gives
    z = (c - conj(d) (d^T c) / (rho + |d|^2)) / rho  with c the right side.
    """
    c = np.conj(Dh) * xh[None] + rho * Wh
    dtc = np.sum(Dh * c, axis=0)
    nd = np.sum(np.abs(Dh) ** 2, axis=0)
    return (c - np.conj(Dh) * (dtc / (rho + nd))[None]) / rho


@dataclasses.dataclass
class CodeResult:
    U: np.ndarray           # [K, n1, n2] sparse code after the last U-step
    Zh: np.ndarray          # [K, n1, n2] Z~ of the last Z~-step (history input)
    xh: np.ndarray          # [n1, n2] spectrum of the padded sample
    primal: list            # ||Z - U|| per iteration
    dual: list              # rho ||U - U_prev|| per iteration
    max_imag: float         # largest |Im F^-1(Z~)| seen (real data => ~0)


def code_admm(x_pad: np.ndarray, Dh: np.ndarray, lam: float, rho: float,
              iters: int) -> CodeResult:
    """Code ADMM for one padded sample (Sec. II-C.1, template eqs. admm_aux/admm_dual).

    Variables: Z~ (frequency codes), U (spatial sparse codes), Gamma (scaled
    dual of U = F^-1(Z~)).  Iteration:
        W^    = F(U - Gamma)
        Z~    = per-frequency solve (code_zstep)
        Z     = F^-1(Z~)
        U     = S_{lam/rho}(Z + Gamma)
        Gamma = Gamma + Z - U
    The penalty rho is on the spatial constraint U = F^-1(Z~) (reading R2).
    """
    x_pad = np.asarray(x_pad, dtype=np.float64)
    n1, n2 = x_pad.shape
    K = Dh.shape[0]
    rho_s = rho
    xh = fft2(x_pad)
    U = np.zeros((K, n1, n2))
    G = np.zeros((K, n1, n2))
    primal, dual = [], []
    max_imag = 0.0
    Zh = np.zeros((K, n1, n2), dtype=np.complex128)
    for _ in range(iters):
        Wh = fft2(U - G)
        Zh = code_zstep(Dh, xh, Wh, rho_s)
        Zc = ifft2(Zh)
        max_imag = max(max_imag, float(np.max(np.abs(Zc.imag))))
        Z = Zc.real
        U_new = soft_threshold(Z + G, lam / rho_s)
        G = G + Z - U_new
        primal.append(float(np.linalg.norm(Z - U_new)))
        dual.append(float(rho_s * np.linalg.norm(U_new - U)))
        U = U_new
    return CodeResult(U=U, Zh=Zh, xh=xh, primal=primal, dual=dual, max_imag=max_imag)


# ----------------------------------------------------------------------------
# History: Sec. III-B, A^p and b^p with eqs. (A_update, B_update)
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class History:
    n: int                  # samples folded so far
    A: np.ndarray           # [n1, n2, K, K]  A^p = mean conj(z) z^T
    b: np.ndarray           # [n1, n2, K]     b^p = mean x~(p) conj(z)

    @staticmethod
    def zeros(K: int, n1: int, n2: int) -> "History":
        return History(0, np.zeros((n1, n2, K, K), np.complex128),
                       np.zeros((n1, n2, K), np.complex128))


def fold_history(h: History, Zh_list, xh_list) -> History:
    """Running-mean fold of a batch of codes (eqs. A_update, B_update; reading R4).

    A^p <- n/(n+B) A^p + 1/(n+B) sum_i conj(z_i) z_i^T
    b^p <- n/(n+B) b^p + 1/(n+B) sum_i x~_i(p) conj(z_i)
    where z_i = Z~_i(p, :)^T.
    """
    B = len(Zh_list)
    n = h.n
    sA = np.zeros_like(h.A)
    sb = np.zeros_like(h.b)
    for Zh, xh in zip(Zh_list, xh_list):
        z = np.moveaxis(Zh, 0, -1)                    # [n1, n2, K]
        sA += np.conj(z)[..., :, None] * z[..., None, :]
        sb += xh[..., None] * np.conj(z)
    A = (n / (n + B)) * h.A + (1.0 / (n + B)) * sA
    b = (n / (n + B)) * h.b + (1.0 / (n + B)) * sb
    return History(n + B, A, b)


# ----------------------------------------------------------------------------
# Dictionary update: Algorithm 2 (DictOCSC), eq. (sub_d_sol), Proposition 2
# ----------------------------------------------------------------------------

def project_filters(alpha: np.ndarray) -> np.ndarray:
    """Proposition 2: V_k = alpha_k / max(||alpha_k||_2, 1)."""
    nrm = np.sqrt(np.sum(alpha * alpha, axis=(-2, -1), keepdims=True))
    return alpha / np.maximum(nrm, 1.0)


@dataclasses.dataclass
class DictState:
    V: np.ndarray           # [K, M, M] spatial filters (feasible)
    thetah: np.ndarray      # [K, n1, n2] scaled dual in the frequency domain
    Dh_last: np.ndarray     # [K, n1, n2] D~_{t,J} of the last update


def sm_fold(C, Zh_list, n: int, r: float):
    """The printed recursion of eq. (C_update) over a batch of codes in order.

    Sample number t = n + 1, n + 2, ...:
      t = 1:  C = I / r - conj(z) z^T / (r (r + z^T conj(z)))
      t > 1:  C = t/(t-1) [C - C conj(z) z^T C / ((t-1) + z^T C conj(z))]
    with z = Z~(p, :)^T at every frequency and r = rho (rho P under the paper's
    convention).  C_t = (A_t + (r / t) I)^-1 (reading R3), the inverse of
    eq. (sub_d_sol) for the penalty rho / t, which DictOCSC then uses (R23).
    Returns C [n1, n2, K, K].
    """
    for i, Zh in enumerate(Zh_list):
        t = n + 1 + i
        z = np.moveaxis(Zh, 0, -1)                        # [n1, n2, K]
        zc = np.conj(z)[..., :, None]                     # conj(z), K x 1
        zr = z[..., None, :]                              # z^T, 1 x K
        if t == 1:
            K = z.shape[-1]
            nz = np.real(zr @ zc)                         # [n1, n2, 1, 1]
            C = np.eye(K) / r - (zc @ zr) / (r * (r + nz))
        else:
            u = C @ zc                                    # C conj(z)
            den = (t - 1) + (zr @ u)
            C = (t / (t - 1)) * (C - (u @ (zr @ C)) / den)
    return C


def dict_ocsc(h: History, V: np.ndarray, thetah: np.ndarray, rho: float, iters: int,
              rho_convention: str = "spatial", C=None):
    """DictOCSC (Algorithm 2) on the current history.

    C^p = (A^p + rho I)^-1 (eq. sub_d_sol; rho*P under the paper's convention).
    For tau = 1..J:
        D~(p,:) = C^p (b^p + rho (V^(p) - theta^(p)))       (eq. sub_d_sol)
        V_k     = Prop. 2 projection of H(F^-1(D~_k + theta^_k))
        theta^  = theta^ + D~ - F(V)
    Returns (V, theta^, D~_{t,J}).  A given C (the recursion of eq. C_update)
    replaces the inverse.
    """
    K, M = V.shape[0], V.shape[-1]
    n1, n2 = h.A.shape[0], h.A.shape[1]
    P = n1 * n2
    r = rho * P if rho_convention == "paper" else rho
    eye = np.eye(K)
    if C is None:
        C = np.linalg.inv(h.A + r * eye)              # [n1, n2, K, K]
    Dh = None
    for _ in range(iters):
        Vh = filters_spectrum(V, n1, n2)              # [K, n1, n2]
        rhs = h.b + r * np.moveaxis(Vh - thetah, 0, -1)
        d = np.einsum("xyij,xyj->xyi", C, rhs)        # [n1, n2, K]
        Dh = np.moveaxis(d, -1, 0)
        alpha = crop(ifft2(Dh + thetah).real, M)
        V = project_filters(alpha)
        thetah = thetah + Dh - filters_spectrum(V, n1, n2)
    return V, thetah, Dh


# ----------------------------------------------------------------------------
# Online loop: Algorithm 3
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class OCSCState:
    K: int
    M: int
    n1: int
    n2: int
    lam: float
    rho: float
    V: np.ndarray
    thetah: np.ndarray
    Dh: np.ndarray          # dictionary spectrum used to code the next sample
    hist: History
    warm_start: bool = True
    return_feasible: bool = True
    rho_convention: str = "spatial"
    updates: int = 0
    history: str = "factor"     # "recursion": C from eq. (C_update) (variant)
    C: np.ndarray = None        # [n1, n2, K, K] when history == "recursion"


def init_state(raw_filters: np.ndarray, n1: int, n2: int, lam: float, rho: float,
               warm_start: bool = True, return_feasible: bool = True,
               rho_convention: str = "spatial", history: str = "factor") -> OCSCState:
    """Algorithm 3 initialisation: D~_0 from Gaussian filters (R10), C = b = 0."""
    V = normalize_filters(raw_filters)
    K, M = V.shape[0], V.shape[-1]
    return OCSCState(K=K, M=M, n1=n1, n2=n2, lam=lam, rho=rho, V=V,
                     thetah=np.zeros((K, n1, n2), np.complex128),
                     Dh=filters_spectrum(V, n1, n2),
                     hist=History.zeros(K, n1, n2), warm_start=warm_start,
                     return_feasible=return_feasible, rho_convention=rho_convention,
                     history=history)


def code(state: OCSCState, image: np.ndarray, iters: int) -> CodeResult:
    """Algorithm 3, FFT and code steps for one sample against the current D~."""
    x_pad = pad_to(np.asarray(image, dtype=np.float64), state.n1, state.n2)
    return code_admm(x_pad, state.Dh, state.lam, state.rho, iters)


def update_dict(state: OCSCState, results, iters: int) -> OCSCState:
    """Algorithm 3, history and dictionary steps for a batch of coded samples."""
    n_before = state.hist.n
    state.hist = fold_history(state.hist, [r.Zh for r in results], [r.xh for r in results])
    C = None
    rho_d = state.rho
    if state.warm_start:
        V0, th0 = state.V, state.thetah
    else:
        V0 = np.zeros_like(state.V)
        th0 = np.zeros_like(state.thetah)
    if state.history == "recursion":
        r = state.rho * state.n1 * state.n2 if state.rho_convention == "paper" else state.rho
        state.C = sm_fold(state.C, [r_.Zh for r_ in results], n_before, r)
        C = state.C
        # Reading R23: C_t = (A_t + (r / t) I)^-1 is the D-row minimiser's
        # inverse for the penalty rho / t, so the ADMM runs with that penalty;
        # the scaled dual keeps the unscaled dual rho Theta across updates.
        t = state.hist.n
        rho_d = state.rho / t
        if n_before > 0:
            th0 = th0 * (t / n_before)
    V, thetah, Dh_last = dict_ocsc(state.hist, V0, th0, rho_d, iters, state.rho_convention, C=C)
    state.V, state.thetah = V, thetah
    state.Dh = filters_spectrum(V, state.n1, state.n2) if state.return_feasible else Dh_last
    state.updates += 1
    return state


def published_filters(state: OCSCState) -> np.ndarray:
    """D_t: V under R7, else H(F^-1(D~_t)) as Algorithm 3's last loop."""
    if state.return_feasible:
        return state.V.copy()
    return crop(ifft2(state.Dh).real, state.M)


def run(images, raw_filters, n1: int, n2: int, lam: float, rho: float, Jz: int, Jd: int,
        batch: int = 1, **flags):
    """Whole Algorithm 3 over ``images`` in mini-batches; returns (state, codes)."""
    st = init_state(raw_filters, n1, n2, lam, rho, **flags)
    codes = []
    for s in range(0, len(images), batch):
        res = [code(st, im, Jz) for im in images[s:s + batch]]
        codes.extend(res)
        update_dict(st, res, Jd)
    return st, codes


# ----------------------------------------------------------------------------
# Objective: Sec. III eq. (ocsc0) for one sample / a set of samples
# ----------------------------------------------------------------------------

def reconstruct(D: np.ndarray, U: np.ndarray) -> np.ndarray:
    """sum_k D_k (*) U_k, circular on U's grid (convolution theorem, Sec. II-C)."""
    n1, n2 = U.shape[-2:]
    return np.real(ifft2(np.sum(filters_spectrum(D, n1, n2) * fft2(U), axis=0)))


def sample_objective(D: np.ndarray, U: np.ndarray, x_pad: np.ndarray, lam: float) -> float:
    """1/2 ||x - sum_k D_k (*) U_k||^2 + lam ||U||_1 for one padded sample."""
    r = np.asarray(x_pad, np.float64) - reconstruct(np.asarray(D, np.float64),
                                                    np.asarray(U, np.float64))
    return 0.5 * float(np.sum(r * r)) + lam * float(np.sum(np.abs(U)))


def objective(D, Us, x_pads, lam: float) -> float:
    """Eq. (ocsc0): mean over samples of sample_objective."""
    vals = [sample_objective(D, U, x, lam) for U, x in zip(Us, x_pads)]
    return float(np.mean(vals))


# ----------------------------------------------------------------------------
# Evaluation of Sec. IV: stopping rule of the online method, test-set PSNR,
# filter order for display.
# ----------------------------------------------------------------------------

def rel_change(new: np.ndarray, old: np.ndarray) -> float:
    """||new - old||_2 / ||new||_2, the relative change of the stopping rule
    (codes Z_t against the previous pass, dictionary D against the previous
    update; both must fall below 1e-3)."""
    new = np.asarray(new, np.float64)
    d = np.linalg.norm(new - np.asarray(old, np.float64))
    n = np.linalg.norm(new)
    return float(d / n) if n > 0 else (0.0 if d == 0 else float("inf"))


def psnr(D: np.ndarray, U: np.ndarray, x_pad: np.ndarray, peak: float = 255.0) -> float:
    """10 log10(peak^2 P / ||x_rec - x||^2), x_rec = sum_k D_k (*) U_k, over the
    padded P = N1 x N2 domain the model is defined on (the paper averages this
    over the test set with peak 255 for 8-bit images)."""
    x_pad = np.asarray(x_pad, np.float64)
    r = reconstruct(np.asarray(D, np.float64), np.asarray(U, np.float64)) - x_pad
    return float(10.0 * np.log10(peak * peak * x_pad.size / float(np.sum(r * r))))


def filter_order(D: np.ndarray) -> np.ndarray:
    """Filter indices in ascending order of their sample variance over the M x M
    entries (unbiased: divided by the entry count minus one), the display order
    of Sec. IV."""
    D = np.asarray(D, np.float64).reshape(len(D), -1)
    mu = D.sum(axis=1) / D.shape[1]
    var = ((D - mu[:, None]) ** 2).sum(axis=1) / (D.shape[1] - 1)
    return np.argsort(var, kind="stable")


# ----------------------------------------------------------------------------
# Uneven image sizes: one spatial dictionary, one frequency grid per size class
# (reading R16; the paper uses a single P).  Each class c keeps its own history
# (A_c, b_c, n_c) and scaled dual theta^_c; with w_c = n_c / n the D-row system
# of class c is (w_c A_c + rho I) d = w_c b_c + rho (v^_c - theta^_c), and the
# V-step projects the mean over the active classes of H(F_c^-1(D~_c + theta^_c))
# (consensus form of Proposition 2: every class penalises its own spatial
# constraint with the same rho).  With one class this is dict_ocsc exactly.
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class SizeClass:
    n1: int
    n2: int
    hist: History
    thetah: np.ndarray          # [K, n1, n2]
    Dh: np.ndarray              # [K, n1, n2] coding spectrum of this class


@dataclasses.dataclass
class MultiState:
    K: int
    M: int
    lam: float
    rho: float
    V: np.ndarray
    classes: dict               # (n1, n2) -> SizeClass
    warm_start: bool = True
    updates: int = 0


def init_multi(raw_filters: np.ndarray, sizes, lam: float, rho: float,
               warm_start: bool = True) -> MultiState:
    V = normalize_filters(raw_filters)
    K = V.shape[0]
    classes = {}
    for (n1, n2) in sizes:
        classes[(n1, n2)] = SizeClass(n1, n2, History.zeros(K, n1, n2),
                                      np.zeros((K, n1, n2), np.complex128),
                                      filters_spectrum(V, n1, n2))
    return MultiState(K=K, M=V.shape[-1], lam=lam, rho=rho, V=V, classes=classes,
                      warm_start=warm_start)


def code_multi(state: MultiState, image: np.ndarray, size, iters: int) -> CodeResult:
    cls = state.classes[size]
    x_pad = pad_to(np.asarray(image, dtype=np.float64), cls.n1, cls.n2)
    return code_admm(x_pad, cls.Dh, state.lam, state.rho, iters)


def dict_ocsc_multi(state: MultiState, iters: int):
    """Consensus DictOCSC over the active size classes (reading R16)."""
    active = [c for c in state.classes.values() if c.hist.n > 0]
    n = sum(c.hist.n for c in active)
    K, M, r = state.K, state.M, state.rho
    eye = np.eye(K)
    Cs = []
    for c in active:
        w = c.hist.n / n
        Cs.append((w, np.linalg.inv(w * c.hist.A + r * eye)))
    V = state.V
    for _ in range(iters):
        ds, alphas = [], []
        for c, (w, C) in zip(active, Cs):
            Vh = filters_spectrum(V, c.n1, c.n2)
            rhs = w * c.hist.b + r * np.moveaxis(Vh - c.thetah, 0, -1)
            d = np.moveaxis(np.einsum("xyij,xyj->xyi", C, rhs), -1, 0)
            ds.append(d)
            alphas.append(crop(ifft2(d + c.thetah).real, M))
        V = project_filters(np.mean(alphas, axis=0))
        for c, d in zip(active, ds):
            c.thetah = c.thetah + d - filters_spectrum(V, c.n1, c.n2)
    return V


def update_dict_multi(state: MultiState, results_by_size: dict, iters: int) -> MultiState:
    """Fold each class's new codes (eqs. A_update, B_update per class) and run
    the consensus DictOCSC; every class then codes against F_c(pad V)."""
    for size, res in results_by_size.items():
        if res:
            c = state.classes[size]
            c.hist = fold_history(c.hist, [r.Zh for r in res], [r.xh for r in res])
    if not state.warm_start:
        state.V = np.zeros_like(state.V)
        for c in state.classes.values():
            c.thetah = np.zeros_like(c.thetah)
    state.V = dict_ocsc_multi(state, iters)
    for c in state.classes.values():
        c.Dh = filters_spectrum(state.V, c.n1, c.n2)
    state.updates += 1
    return state
