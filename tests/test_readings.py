"""CPU pins of reformulations the GPU path relies on (no GPU, no oracle code): each one is
checked against the form the paper writes, in FP64 numpy.

* Implicit Q (Alg. 1 / Alg. 2 final steps with the QR of C in place of its SVD): with
  C^H C = R_c^H R_c (Cholesky) and Q = C R_c^{-1}, the eigenvectors U_B of
  B = R_c W R_c^H give U_s = C (R_c^{-1} U_B[:, :K]), the same subspace as Q U_B[:, :K]
  from a Householder QR of C, and U_s^H U_s = I.
* Sketch on real rows (Sec. III products R V as one real GEMM): an interleaved complex row
  of R times the B rows [Vr, -Vi] and [Vi, Vr] gives Re and Im of R V.
"""
import numpy as np


def _hermitian_psd(rng, M, K, snr=10.0):
    A = np.exp(1j * np.pi * np.outer(np.arange(M), np.sin(rng.uniform(-1.0, 1.0, K))))
    S = (rng.standard_normal((K, 4 * M)) + 1j * rng.standard_normal((K, 4 * M))) * np.sqrt(snr / 2)
    N = (rng.standard_normal((M, 4 * M)) + 1j * rng.standard_normal((M, 4 * M))) / np.sqrt(2)
    X = A @ S + N
    return X @ X.conj().T / X.shape[1]


def _top(B, K):
    w, Z = np.linalg.eigh(B)
    return Z[:, np.argsort(w)[::-1][:K]]


def test_implicit_q_gives_the_qr_subspace_and_an_orthonormal_basis():
    rng = np.random.default_rng(3)
    for M, K, l in ((64, 3, 8), (200, 6, 18), (128, 8, 24)):
        R = _hermitian_psd(rng, M, K)
        Om = rng.standard_normal((M, l)) + 1j * rng.standard_normal((M, l))
        C = R @ Om
        W = np.linalg.pinv(Om.conj().T @ C)          # core matrix of Alg. 2 with t = 0
        # the paper's route with an explicit Q
        Q, Rq = np.linalg.qr(C)
        U1 = Q @ _top(Rq @ W @ Rq.conj().T, K)
        # the GPU's route: R_c from the Cholesky of the Gram, Q never formed
        Rc = np.linalg.cholesky(C.conj().T @ C).conj().T
        U2 = C @ (np.linalg.inv(Rc) @ _top(Rc @ W @ Rc.conj().T, K))
        assert np.linalg.norm(U2.conj().T @ U2 - np.eye(K)) < 1e-9
        assert np.linalg.norm(U1 @ U1.conj().T - U2 @ U2.conj().T) < 1e-9


def test_interleaved_rows_times_split_b_rows_give_the_complex_product():
    rng = np.random.default_rng(4)
    M, l = 37, 5
    R = rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))
    V = rng.standard_normal((M, l)) + 1j * rng.standard_normal((M, l))
    Rrows = np.empty((M, 2 * M))
    Rrows[:, 0::2], Rrows[:, 1::2] = R.real, R.imag
    Brows = np.empty((2 * l, 2 * M))
    Brows[0::2, 0::2], Brows[0::2, 1::2] = V.real.T, -V.imag.T     # -> Re of column j
    Brows[1::2, 0::2], Brows[1::2, 1::2] = V.imag.T, V.real.T      # -> Im of column j
    D = Rrows @ Brows.T
    assert np.allclose(D[:, 0::2] + 1j * D[:, 1::2], R @ V, rtol=0, atol=1e-12)
