"""Pins for the FP64 oracle against what the paper and the mathematics fix.

Nothing here retypes the oracle's own formulas: each check is a closed form, an
invariant, a special case that reduces to a textbook or library routine, a
published known-answer vector, or brute force on tiny inputs.  CPU only.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1911_07434_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def proj(U):
    return U @ U.conj().T


def rand_herm(rng, n, scale=1.0):
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return scale * (A + A.conj().T) / 2


def steering(M, theta_deg, d=0.5):
    m = np.arange(M)[:, None]
    return np.exp(1j * 2 * np.pi * d * m * np.sin(np.deg2rad(np.atleast_1d(theta_deg)))[None, :])


def dft_bin_population(M, bins, powers, sigma2):
    """Population covariance A diag(P) A^H + sigma^2 I with sin(theta_k) = 2 n_k / M,
    which makes the steering columns exactly orthogonal (sum of M-th roots of unity)."""
    s = 2.0 * np.asarray(bins) / M
    theta = np.rad2deg(np.arcsin(s))
    A = steering(M, theta)
    R = A @ np.diag(powers) @ A.conj().T + sigma2 * np.eye(M)
    return R, A, theta


# ---------------------------------------------------------------- Philox ---
def test_philox_known_answers():
    """Random123 known-answer vectors (Salmon et al., SC'11)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert list(out) == v[6:10]


def test_gaussian_test_matrix_statistics():
    """Re and Im of Pi are i.i.d. N(0,1) (Sec. III-B): moments over 40k draws."""
    Pi = oracle.gaussian_test_matrix(seed=7, frame_id=3, M=2000, l=20)
    x = np.concatenate([Pi.real.ravel(), Pi.imag.ravel()])
    assert abs(x.mean()) < 0.02
    assert abs(x.var() - 1.0) < 0.03
    assert abs(np.mean(x ** 4) - 3.0) < 0.15          # Gaussian kurtosis
    assert abs(np.corrcoef(Pi.real.ravel(), Pi.imag.ravel())[0, 1]) < 0.02
    # different frames / seeds give different matrices, same inputs the same one
    assert not np.allclose(Pi[:5], oracle.gaussian_test_matrix(7, 4, 5, 20))
    assert np.array_equal(Pi[:5], oracle.gaussian_test_matrix(7, 3, 5, 20))


def test_sample_indices_properties():
    for M, l in [(10, 1), (10, 10), (64, 13), (512, 24), (7, 6)]:
        I = oracle.sample_indices(11, 5, M, l)
        assert len(set(I.tolist())) == l
        assert np.all(np.diff(I) > 0) and I.min() >= 0 and I.max() < M
    assert np.array_equal(oracle.sample_indices(11, 5, 30, 30), np.arange(30))
    # uniformity: each index appears with frequency l/M over many frames
    cnt = np.zeros(20)
    for f in range(4000):
        cnt[oracle.sample_indices(3, f, 20, 5)] += 1
    assert np.all(np.abs(cnt / 4000 - 5 / 20) < 0.03)


# ------------------------------------------------------------ covariance ---
def test_covariance_worked_example():
    Y, S = [], []
    for line in open(os.path.join(GOLDEN, "covariance_worked_2x2.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        tag, *vals = line.split()
        row = [complex(float(v.split(",")[0]), float(v.split(",")[1])) for v in vals]
        (Y if tag == "Y" else S).append(row)
    R = oracle.covariance(np.array(Y, dtype=np.complex64))
    assert np.array_equal(R, np.array(S))


def test_covariance_rank_one_exact():
    """X = a s^T with small Gaussian integers: R = a a^H * sum|s|^2 / T exactly."""
    rng = np.random.default_rng(0)
    a = rng.integers(-3, 4, 9) + 1j * rng.integers(-3, 4, 9)
    s = rng.integers(-3, 4, 8) + 1j * rng.integers(-3, 4, 8)
    X = np.outer(a, s).astype(np.complex64)
    R = oracle.covariance(X)
    expect = np.outer(a, a.conj()) * (np.sum(s.real ** 2 + s.imag ** 2) / 8)
    assert np.array_equal(R, expect)


def test_covariance_invariants():
    rng = np.random.default_rng(1)
    X = (rng.standard_normal((17, 33)) + 1j * rng.standard_normal((17, 33))).astype(np.complex64)
    R = oracle.covariance(X)
    assert np.allclose(R, R.conj().T, atol=0, rtol=0) or np.max(np.abs(R - R.conj().T)) < 1e-15
    assert np.all(np.abs(np.diag(R).imag) == 0) and np.all(np.diag(R).real >= 0)
    Xd = X.astype(np.complex128)
    assert abs(np.trace(R).real - np.sum(np.abs(Xd) ** 2) / 33) < 1e-12
    # brute force single entries written as explicit sums
    for (i, j) in [(0, 0), (3, 7), (16, 2)]:
        acc = sum(complex(Xd[i, t]) * complex(Xd[j, t]).conjugate() for t in range(33)) / 33
        assert abs(R[i, j] - acc) < 1e-13


# ----------------------------------------------------------------- Jacobi --
def test_jacobi_2x2_closed_form():
    for (a, c, b) in [(2.0, -1.0, 0.5 + 0.7j), (1.0, 1.0, 1j), (3.0, 0.0, 0.0), (-2.0, 5.0, -1.5)]:
        w, V, _ = oracle.eigh_jacobi(np.array([[a, b], [np.conj(b), c]]))
        r = np.sqrt(((a - c) / 2) ** 2 + abs(b) ** 2)
        assert np.allclose(w, [(a + c) / 2 + r, (a + c) / 2 - r], atol=1e-14)


def test_jacobi_diagonal_and_permutation():
    d = np.array([0.5, -3.0, 7.0, 2.0])
    w, V, sweeps = oracle.eigh_jacobi(np.diag(d).astype(complex))
    assert np.array_equal(w, np.sort(d)[::-1]) and sweeps == 0
    assert np.allclose(np.abs(V), np.eye(4)[:, [2, 3, 0, 1]])


def test_jacobi_residual_orthonormality_and_lapack():
    rng = np.random.default_rng(2)
    for n in (3, 13, 40):
        A = rand_herm(rng, n, 3.0)
        w, V, _ = oracle.eigh_jacobi(A)
        nrm = np.linalg.norm(A)
        assert np.linalg.norm(A @ V - V * w) <= 1e-12 * nrm
        assert np.linalg.norm(V.conj().T @ V - np.eye(n)) <= 1e-13
        assert np.all(np.diff(w) <= 0)
        # special case reducing to a library routine: LAPACK's eigenvalues
        assert np.allclose(w, np.sort(np.linalg.eigvalsh(A))[::-1], atol=1e-12 * nrm)


def test_eq4_eigenstructure_population_covariance():
    """Eq. 4: with orthogonal steering columns, eigenvalues are M P_k + sigma^2 (K of them)
    and sigma^2 (M-K of them); the noise subspace is orthogonal to every a(theta_k)."""
    M, bins, P, s2 = 32, [-5, 2, 9], np.array([4.0, 1.0, 0.25]), 0.3
    R, A, theta = dft_bin_population(M, bins, P, s2)
    U, lam = oracle.music_subspace(R, 3)
    assert np.allclose(lam[:3], np.sort(M * P + s2)[::-1], atol=1e-11)
    assert np.allclose(lam[3:], s2, atol=1e-11)
    Pn = np.eye(M) - proj(U)
    assert np.max(np.abs(Pn @ A)) < 1e-11
    assert np.linalg.norm(proj(U) - proj(A / np.sqrt(M))) < 1e-11


# ---------------------------------------------------- QR / SVD / pinv ----
def test_householder_qr_invariants():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((30, 7)) + 1j * rng.standard_normal((30, 7))
    Q, R = oracle.householder_qr(A)
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(7)) < 1e-13
    assert np.linalg.norm(Q @ R - A) < 1e-13 * np.linalg.norm(A)
    assert np.all(np.tril(R, -1) == 0)


def test_svd_jacobi_invariants_and_lapack():
    rng = np.random.default_rng(4)
    A = (rng.standard_normal((25, 6)) + 1j * rng.standard_normal((25, 6))) @ np.diag([1e3, 10, 1, 1, 0.1, 1e-3])
    U, s, W = oracle.svd_jacobi(A)
    assert np.linalg.norm(U.conj().T @ U - np.eye(6)) < 1e-12
    assert np.linalg.norm(W.conj().T @ W - np.eye(6)) < 1e-13
    assert np.linalg.norm(U @ np.diag(s) @ W.conj().T - A) < 1e-12 * np.linalg.norm(A)
    assert np.allclose(s, np.linalg.svd(A, compute_uv=False), rtol=1e-11)


def test_pinv_moore_penrose_conditions():
    rng = np.random.default_rng(5)
    B = rng.standard_normal((8, 3)) + 1j * rng.standard_normal((8, 3))
    H = B @ B.conj().T                       # Hermitian PSD, rank 3
    W, rank = oracle.pinv_hermitian(H)
    assert rank == 3
    for lhs, rhs in [(H @ W @ H, H), (W @ H @ W, W), ((H @ W).conj().T, H @ W), ((W @ H).conj().T, W @ H)]:
        assert np.linalg.norm(lhs - rhs) <= 1e-10 * max(1.0, np.linalg.norm(rhs))
    Hf = rand_herm(rng, 6) + 6 * np.eye(6)   # invertible
    Wf, rf = oracle.pinv_hermitian(Hf)
    assert rf == 6 and np.linalg.norm(Wf @ Hf - np.eye(6)) < 1e-12


# --------------------------------------------------------- fast MUSIC ----
@pytest.mark.parametrize("method,t", [(1, 0), (2, 0), (2, 1), (2, 2), (1, 1)])
def test_fast_music_exact_on_rank_K(method, t):
    """Noise-free rank-K covariance, l >= K: range(S Pi) = range(S), so the randomized
    subspace equals the exact signal subspace (Theorems 1-3 with sigma_{K+1} = 0)."""
    M, K = 48, 4
    rng = np.random.default_rng(6)
    theta = np.array([-31.0, -4.5, 12.0, 40.0])
    A = steering(M, theta)
    R = A @ np.diag([3.0, 1.0, 0.5, 2.0]) @ A.conj().T
    Uk, _ = oracle.music_subspace(R, K)
    for l in (K, K + 3):
        U, lamB, _ = oracle.fast_music(R, K, l, t, method, seed=int(rng.integers(1 << 30)))
        assert np.linalg.norm(proj(U) - proj(Uk)) < 1e-8, (l, np.linalg.norm(proj(U) - proj(Uk)))


def test_fast_music_sampling_all_columns_is_exact():
    """p = M in Algorithm 1: Pi selects every column, S~ = C W C^H = S."""
    X = synth.small_frame().X[:20, :60]
    R = oracle.covariance(X)
    Uk, _ = oracle.music_subspace(R, 3)
    U, lamB, idx = oracle.fast_music(R, 3, 20, 0, 1, seed=1)
    assert np.array_equal(idx, np.arange(20))
    assert np.linalg.norm(proj(U) - proj(Uk)) < 1e-9
    lam = np.sort(np.linalg.eigvalsh(R))[::-1]
    assert np.allclose(lamB, lam, rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("method,t", [(1, 0), (2, 0), (2, 1)])
def test_nystrom_identity_and_forms(method, t):
    """U~ U~^H C = C for the full l-column basis (Lemma 12 of wang2016spsd as used in
    the proofs of Theorems 1-2), and the printed SVD route equals the QR route."""
    fr = synth.small_frame()
    R = oracle.covariance(fr.X)
    l = 13
    Ul, lamB, idx = oracle.fast_music(R, 3, l, t, method, seed=9, ncols=l)
    if method == 1:
        C = R[:, idx]
    else:
        C = R @ oracle.gaussian_test_matrix(9, 0, 64, l)
        for _ in range(t):
            Q, _r = np.linalg.qr(C)
            C = R @ Q
    assert np.linalg.norm(proj(Ul) @ C - C) < 1e-9 * np.linalg.norm(C)
    assert np.linalg.norm(Ul.conj().T @ Ul - np.eye(l)) < 1e-9
    U0, _, _ = oracle.fast_music(R, 3, l, t, method, seed=9, form=0)
    U1, _, _ = oracle.fast_music(R, 3, l, t, method, seed=9, form=1)
    assert np.linalg.norm(proj(U0) - proj(U1)) < 1e-9


def _nystrom_reference(R, method, l, t, seed, frame_id=0):
    """S~ = C pinv(P^H C) C^H written from Eq. 8 with a general Pi (Sec. III-B) and the
    power steps of Eq. 11, with numpy/LAPACK primitives only: C = R Pi (Pi the pinned
    Gaussian test matrix, or the columns R(:, I) for Alg. 1), then t times
    {P = orth(C) by LAPACK QR; C = R P}.  Also returns the two plausible wrong cores
    (W = I, and W built from Pi instead of the last P after power steps)."""
    M = R.shape[0]
    if method == 1:
        idx = oracle.sample_indices(seed, frame_id, M, l)
        Pi = np.zeros((M, l), dtype=complex)
        Pi[idx, np.arange(l)] = 1.0
    else:
        Pi = oracle.gaussian_test_matrix(seed, frame_id, M, l)
    C = R @ Pi
    P = Pi
    for _ in range(t):
        P, _r = np.linalg.qr(C)
        C = R @ P
    H = P.conj().T @ C
    H = (H + H.conj().T) / 2
    S_tilde = C @ np.linalg.pinv(H, hermitian=True) @ C.conj().T
    wrong_identity = C @ C.conj().T
    Hp = Pi.conj().T @ C
    wrong_pi = C @ np.linalg.pinv((Hp + Hp.conj().T) / 2, hermitian=True) @ C.conj().T
    return S_tilde, wrong_identity, wrong_pi


def _top_eig(S, n):
    w, V = np.linalg.eigh((S + S.conj().T) / 2)
    order = np.argsort(w)[::-1][:n]
    return w[order], V[:, order]


@pytest.mark.parametrize("case,method,t", [
    ("small", 2, 0), ("small", 2, 1), ("small", 2, 2), ("small", 1, 1), ("small", 1, 0),
    ("m96", 2, 0), ("m96", 2, 1), ("m96", 2, 2), ("m96", 1, 1)])
def test_core_matrix_is_nystrom_pinv(case, method, t):
    """The core matrix W of Alg. 1/2 is pinv(P^H S P) = pinv(P^H C) (Eq. 8 with a general
    Pi; Alg. 2 with P = the last orth(C)), so B's eigenvalues are the l nonzero eigenvalues
    of the Nystrom approximation S~ = C W C^H and U spans S~'s top-K eigenspace.
    Noisy frames with l > K, where the choice of W decides the result; the two plausible
    slips (W = I; Pi in place of the last P) are shown to miss the check by a wide margin."""
    if case == "small":
        fr = synth.small_frame()
        K, l = fr.K, fr.l
    else:
        fr = synth.massive_mimo_frames(1, seed=4, M=96, T=300, K=4, extra=16, snr_lo=0.0,
                                       snr_hi=12.0).frames[0]
        K, l = fr.K, fr.l
    R = oracle.covariance(fr.X)
    U, lamB, _ = oracle.fast_music(R, K, l, t, method, seed=21)
    S_tilde, wrong_identity, wrong_pi = _nystrom_reference(R, method, l, t, seed=21)
    w_ref, V_ref = _top_eig(S_tilde, l)
    scale = w_ref[0]
    assert np.max(np.abs(lamB - w_ref)) <= 1e-9 * scale, np.max(np.abs(lamB - w_ref)) / scale
    assert np.linalg.norm(proj(U) - proj(V_ref[:, :K])) <= 1e-9
    w_id, _ = _top_eig(wrong_identity, l)
    assert np.max(np.abs(lamB - w_id)) > 1.0 * scale
    if t > 0:
        w_pi, _ = _top_eig(wrong_pi, l)
        assert np.max(np.abs(lamB - w_pi)) > 0.1 * scale


def test_power_iterations_converge():
    """Theorem 2/3: the error decays like (sigma_{K+1}/sigma_K)^{t+1}."""
    fr = synth.massive_mimo_frames(1, seed=3, M=96, T=200, K=4, extra=0, snr_lo=-6, snr_hi=-3).frames[0]
    R = oracle.covariance(fr.X)
    Uk, _ = oracle.music_subspace(R, 4)
    errs = [np.linalg.norm(proj(oracle.fast_music(R, 4, 4, t, 2, seed=5)[0]) - proj(Uk)) for t in range(5)]
    assert errs[4] < errs[0] and errs[4] < 1e-3 and errs[2] < errs[0]


def _theorem_ratios(fr, method, l, t, seed, ncols):
    R = oracle.covariance(fr.X)
    K = fr.K
    Uk, lam = oracle.music_subspace(R, K)
    U, _, _ = oracle.fast_music(R, K, l, t, method, seed=seed, ncols=ncols)
    P = oracle.spectrum(Uk, -90, 0.25, 721, residual_form=True)
    Pt = oracle.spectrum(U, -90, 0.25, 721, residual_form=True)
    return np.sqrt(P / Pt), lam, Uk


def test_theorem1_lower_bound_fast1():
    """Theorem 1 on the Sec. V-C setting scaled down: for p >= 4.5 mu K log(K/delta),
    sqrt(P/P~) <= 1 + 2 sqrt(M^2/p) sigma_{K+1}/sigma_K with prob. >= 1 - delta."""
    delta, fails, runs = 0.1, 0, 0
    for seed in range(8):
        fr = synth.bounds_study_frame(seed, M=64, T=128, K=3, snr_db=1.0)
        R = oracle.covariance(fr.X)
        Uk, lam = oracle.music_subspace(R, 3)
        mu = 64 / 3 * np.max(np.sum(np.abs(Uk) ** 2, axis=1))
        p = int(min(64, np.ceil(4.5 * mu * 3 * np.log(3 / delta))))
        ratio, lam, _ = _theorem_ratios(fr, 1, p, 0, seed, ncols=p)
        bound = 1 + 2 * np.sqrt(64 ** 2 / p) * lam[3] / lam[2]
        runs += 1
        fails += int(np.max(ratio) > bound)
    assert fails <= delta * runs + 1e-9


@pytest.mark.parametrize("t", [1, 2])
def test_theorems2_3_bounds_fast2(t):
    """Theorems 2 and 3 (p = K, the Sec. V-C setting with delta = 0.1):
    1 - a <= sqrt(P/P~) <= 1 + a, a = sqrt(M^2 K)/delta (sigma_{K+1}/sigma_K)^{t+1}."""
    delta, fails, runs = 0.1, 0, 0
    for seed in range(8):
        fr = synth.bounds_study_frame(100 + seed, M=64, T=128, K=3, snr_db=1.0)
        ratio, lam, _ = _theorem_ratios(fr, 2, 3, t, seed, ncols=3)
        a = np.sqrt(64 ** 2 * 3) / delta * (lam[3] / lam[2]) ** (t + 1)
        runs += 1
        fails += int(np.max(ratio) > 1 + a or np.min(ratio) < 1 - a)
    assert fails <= delta * runs + 1e-9


# -------------------------------------------------------------- spectrum --
def test_spectrum_dirichlet_closed_form():
    """With U_K = A/sqrt(M) (DFT-bin sources), P(theta) = 1/(M - sum_k |D_M(u_k)|^2 / M),
    D_M the Dirichlet kernel |sin(pi M u/2)/sin(pi u/2)|, u = sin theta - sin theta_k."""
    M = 40
    R, A, th = dft_bin_population(M, [-7, 3], np.array([2.0, 1.0]), 0.1)
    U, _ = oracle.music_subspace(R, 2)
    grid0, step, L = -89.0, 0.37, 480
    P = oracle.spectrum(U, grid0, step, L)
    thg = np.deg2rad(grid0 + step * np.arange(L))
    acc = np.zeros(L)
    for tk in np.deg2rad(th):
        u = np.sin(thg) - np.sin(tk)
        with np.errstate(invalid="ignore", divide="ignore"):
            D = np.where(np.abs(np.sin(np.pi * u / 2)) < 1e-12, M,
                         np.abs(np.sin(np.pi * M * u / 2) / np.sin(np.pi * u / 2)))
        acc += D ** 2 / M
    expect = 1.0 / (M - acc)
    far = (M - acc) > 1e-3
    assert np.allclose(P[far], expect[far], rtol=1e-9)


def test_spectrum_forms_agree_and_scale():
    fr = synth.small_frame()
    R = oracle.covariance(fr.X)
    U, _ = oracle.music_subspace(R, 3)
    P0 = oracle.spectrum(U, fr.theta0, fr.step, fr.L)
    P1 = oracle.spectrum(U, fr.theta0, fr.step, fr.L, residual_form=True)
    assert np.allclose(P0, P1, rtol=1e-8)
    # away from the targets the spectrum sits near 1/M (Sec. V-C)
    th = fr.theta0 + fr.step * np.arange(fr.L)
    far = np.min(np.abs(th[:, None] - fr.angles_deg[None, :]), axis=1) > 10
    assert 0.5 / 64 < np.median(P0[far]) < 2.0 / 64


# ------------------------------------------------------------------ peaks --
def _brute_peaks(P, K):
    L = len(P)
    cand = [i for i in range(L) if (i == 0 or P[i] > P[i - 1]) and (i == L - 1 or P[i] >= P[i + 1])]
    cand.sort(key=lambda i: (-P[i], i))
    out = cand[:K]
    return out + [-1] * (K - len(out)), len(out)


def test_peaks_brute_force_with_ties():
    rng = np.random.default_rng(8)
    for trial in range(300):
        L = int(rng.integers(1, 40))
        P = rng.integers(0, 6, L).astype(float)       # many ties and plateaus
        K = int(rng.integers(1, 6))
        idx, n = oracle.peaks(P, K)
        bi, bn = _brute_peaks(P, K)
        assert n == bn and list(idx) == bi, (P, K)


def test_frame_peaks_at_true_angles():
    """Peaks of the small ULA frame (3 sources at 10 dB) fall at the true angles."""
    fr = synth.small_frame()
    for method, t in [(0, 0), (2, 2), (1, 0)]:
        P, idx, n = oracle.frame(fr.X, fr.K, fr.l, t, method, 0, 0, fr.theta0, fr.step, fr.L)
        assert n == 3
        est = np.sort(fr.theta0 + fr.step * idx)
        assert np.max(np.abs(est - fr.angles_deg)) <= 0.3, (method, est)


# ------------------------------------------------ non-uniform arrays (Sec. II-A) ---
def test_sparse_lattice_array_reduces_to_zero_padded_ula():
    """An array whose elements sit on the half-wavelength lattice is a subset S of a ULA's
    elements, so a_sparse(theta) = a_ula(theta)[S].  With U' = U placed on rows S of the
    ULA (zeros elsewhere), ||U'^H a_ula|| = ||U^H a_sparse||, hence
    1/P_sparse - M_sparse = 1/P_ula(U') - M_ula at every angle: the position path reduces
    to the pinned uniform-array scan (Dirichlet closed form above)."""
    rng = np.random.default_rng(11)
    N, M, nc = 40, 23, 4
    S = np.sort(rng.choice(N, M, replace=False))
    U = np.linalg.qr(rng.standard_normal((M, nc)) + 1j * rng.standard_normal((M, nc)))[0]
    Up = np.zeros((N, nc), dtype=complex)
    Up[S] = U
    grid = (-89.5, 0.31, 578)
    Ps = oracle.spectrum(U, *grid, pos=0.5 * S)
    Pu = oracle.spectrum(Up, *grid)
    assert np.max(np.abs((1 / Ps - M) - (1 / Pu - N))) < 1e-10


def test_spectrum_position_invariances():
    """Moving the whole array multiplies a(theta) by one phase per angle, and relabelling
    the elements permutes a(theta) and the rows of U together: neither changes
    ||U^H a||, so P is unchanged.  Mirroring the positions conjugates a(theta), which
    conj(U) undoes.  Uniform positions d m give the uniform-array spectrum."""
    rng = np.random.default_rng(12)
    pos = synth.sparse_virtual_array(37, seed=5)
    U = np.linalg.qr(rng.standard_normal((37, 5)) + 1j * rng.standard_normal((37, 5)))[0]
    grid = (-80.0, 0.4, 401)
    P = oracle.spectrum(U, *grid, pos=pos)
    assert np.allclose(oracle.spectrum(U, *grid, pos=pos + 3.25), P, rtol=1e-9)
    perm = rng.permutation(37)
    assert np.allclose(oracle.spectrum(U[perm], *grid, pos=pos[perm]), P, rtol=1e-9)
    assert np.allclose(oracle.spectrum(U.conj(), *grid, pos=-pos), P, rtol=1e-9)
    assert np.allclose(oracle.spectrum(U, *grid, pos=0.5 * np.arange(37)), oracle.spectrum(U, *grid), rtol=1e-11)
    # a shifted but unmirrored array is not the mirrored one: the check above is not vacuous
    assert not np.allclose(oracle.spectrum(U, *grid, pos=-pos), P, rtol=1e-3)


def test_sparse_array_signal_subspace_nulls_the_true_angles():
    """Eq. 4-5 for any geometry: noise-free snapshots of K sources have R = A S A^H with
    A the array's steering matrix, so U_K spans A and the MUSIC denominator
    M - ||U_K^H a(theta)||^2 vanishes at every true angle (P -> inf) while it stays
    well above zero elsewhere.  The data come from the signal model of the input
    generator, the steering of the scan from the oracle: two codes, one geometry."""
    pos = synth.sparse_virtual_array(48, seed=3)
    angles = np.array([-30.0, 7.5, 41.0])
    rng = synth.rng_for(9, 9)
    X = synth.array_snapshots(rng, pos, 400, angles, np.array([1.0, 0.5, 2.0]), 0.0)
    R = oracle.covariance(X)
    U, lam = oracle.music_subspace(R, 3)
    th0, step, L = -60.0, 0.5, 241
    P = oracle.spectrum(U, th0, step, L, pos=pos)
    on = np.round((angles - th0) / step).astype(int)
    den = 1.0 / P
    assert np.all(den[on] < 1e-5 * 48)
    off = np.ones(L, bool)
    for i in on:
        off[max(0, i - 2):i + 3] = False
    assert np.min(den[off]) > 1e-3
    idx, n = oracle.peaks(P, 3)
    assert n == 3 and sorted(idx.tolist()) == sorted(on.tolist())


@pytest.mark.parametrize("method,t", [(2, 1), (1, 0), (0, 0)])
def test_sparse_array_frame_peaks_at_true_angles(method, t):
    """A noisy sparse-array frame (10-20 dB): standard MUSIC and both fast variants put
    their K peaks within one grid step of the true angles."""
    fr = synth.sparse_array_frames(1, seed=2, M=96, T=256, K=4, extra=8, grid=(-60.0, 60.0, 0.05)).frames[0]
    P, idx, n = oracle.frame(fr.X, fr.K, fr.l, t, method, 0, 0, fr.theta0, fr.step, fr.L, pos=fr.pos)
    assert n == fr.K
    est = np.sort(fr.theta0 + fr.step * idx)
    assert np.max(np.abs(est - fr.angles_deg)) <= 0.1, (est, fr.angles_deg)
