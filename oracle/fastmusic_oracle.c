/*
 * fastmusic_oracle.c -- plain, slow FP64 CPU oracle for the fast-MUSIC hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
 * CUDA path is compared against.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header, table
 * or constant generator with the CUDA library, and it never calls it.
 *
 * Everything is double precision (C99 `double complex`), row-major, with
 * naive loops in the order the paper states the steps.  Paper references are
 * to arXiv 1911.07434 ("Ultra-Fast Accurate AoA Estimation via Automotive
 * Massive-MIMO Radar"):
 *   - Sec. II-B, Eq. 2-3 : covariance S = Y Y^H / N of the snapshot matrix
 *   - Sec. II-B, Eq. 4   : SVD/EVD split into signal and noise subspaces
 *   - Sec. II-B, Eq. 5-6 : MUSIC pseudo-spectrum and peak search
 *   - Sec. III-A, Eq. 7-10, Algorithm 1 : fast MUSIC 1 (random sampling,
 *     Nystrom weight W = pinv(Pi^H S Pi), rank restriction via SVD(C), SVD(B))
 *   - Sec. III-B, Eq. 11, Algorithm 2 : fast MUSIC 2 (Gaussian projection,
 *     t power iterations V = orth(C), C = S V, W = pinv(V^H S V))
 *
 * Readings of places where the paper is silent or ambiguous (the same list
 * is kept with the design notes):
 *   - steering vector a_m(theta) = exp(+j 2 pi x_m sin(theta)) with x_m = d m
 *     for the uniform array of Sec. II-A (d in wavelengths) or the given
 *     element positions x_m of a non-uniform virtual array (the trailing ^H in
 *     Sec. II-B is read as a transpose);
 *   - theta is measured from broadside in degrees, grid theta_i = theta0 + i*step;
 *   - sampling draws l DISTINCT indices from {0..M-1}, sorted ascending; the
 *     sqrt(M/p) scale of the sampling matrix cancels in C W C^H and is omitted;
 *   - the Gaussian test matrix is complex with Re, Im ~ N(0,1) i.i.d., drawn from
 *     Philox4x32-10 + Box-Muller with the counter layout documented below;
 *   - Algorithm 2 applies S a total of t+1 times: C = S Pi, then t times
 *     {V = orth(C); C = S V}; W = pinv(V^H C).  For t = 0 the core matrix is
 *     the Nystrom one, W = pinv(Pi^H C) (Eq. 8 with a general Pi).  The same
 *     power steps are applied to a sampling sketch when t > 0;
 *   - pinv of a Hermitian matrix zeroes eigenvalues with |lambda| <=
 *     n * eps64 * max|lambda|;
 *   - the SVD of the Hermitian PSD matrix B is its eigendecomposition ordered by
 *     signed eigenvalue, descending; U_s keeps the first K columns (or all l);
 *   - a local maximum is i with P[i] > P[i-1] and P[i] >= P[i+1] (missing
 *     neighbours at the ends never block); the K largest are returned, ties to
 *     the lower index; a non-positive denominator gives P = +inf.
 */
#define _GNU_SOURCE
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex zc;

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_NOCONV (-2)
#define ORC_ERR_MEM (-3)

/* ------------------------------------------------------------------------ */
/* Counter-based generator: Philox4x32-10 (Salmon, Moraes, Dror, Shaw,       */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11).  One round maps   */
/* (c0,c1,c2,c3) with key (k0,k1) to                                         */
/*   (hi(B*c2) ^ c1 ^ k0, lo(B*c2), hi(A*c0) ^ c3 ^ k1, lo(A*c0)),            */
/* A = 0xD2511F53, B = 0xCD9E8D57; the key is advanced by the Weyl constants */
/* (0x9E3779B9, 0xBB67AE85) before every round after the first.              */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t pa = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t pb = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(pb >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)pb;
        uint32_t n2 = (uint32_t)(pa >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)pa;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Gaussian test matrix Pi (M x l, row-major) of Sec. III-B.
 * Entry (m, j): counter (j, m, frame_lo, frame_hi), key (seed_lo, seed_hi);
 * outputs x0, x1 give u1 = (x0+1)/2^32 in (0,1], u2 = x1/2^32 in [0,1) and the
 * Box-Muller pair  sqrt(-2 ln u1) * (cos 2 pi u2 + j sin 2 pi u2). */
void orc_gaussian_test_matrix(uint64_t seed, uint64_t frame_id, int M, int l, zc* Pi)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int m = 0; m < M; ++m) {
        for (int j = 0; j < l; ++j) {
            uint32_t ctr[4] = {(uint32_t)j, (uint32_t)m, (uint32_t)frame_id,
                               (uint32_t)(frame_id >> 32)};
            uint32_t x[4];
            orc_philox4x32_10(ctr, key, x);
            double u1 = ((double)x[0] + 1.0) / 4294967296.0;
            double u2 = (double)x[1] / 4294967296.0;
            double r = sqrt(-2.0 * log(u1));
            Pi[(size_t)m * l + j] = r * cos(2.0 * M_PI * u2) + I * (r * sin(2.0 * M_PI * u2));
        }
    }
}

/* Random index set of Algorithm 1: l distinct indices from {0..M-1}.
 * Partial Fisher-Yates; draw i uses counter (i, 0xFFFFFFFF, frame_lo, frame_hi)
 * and maps output x0 to j = i + floor(x0 * (M - i) / 2^32).  Returned sorted. */
int orc_sample_indices(uint64_t seed, uint64_t frame_id, int M, int l, int* idx)
{
    if (M < 1 || l < 1 || l > M) return ORC_ERR_ARG;
    int* perm = (int*)malloc(sizeof(int) * (size_t)M);
    if (!perm) return ORC_ERR_MEM;
    for (int m = 0; m < M; ++m) perm[m] = m;
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int i = 0; i < l; ++i) {
        uint32_t ctr[4] = {(uint32_t)i, 0xFFFFFFFFu, (uint32_t)frame_id, (uint32_t)(frame_id >> 32)};
        uint32_t x[4];
        orc_philox4x32_10(ctr, key, x);
        int j = i + (int)(((uint64_t)x[0] * (uint64_t)(M - i)) >> 32);
        int tmp = perm[i];
        perm[i] = perm[j];
        perm[j] = tmp;
    }
    for (int i = 0; i < l; ++i) idx[i] = perm[i];
    free(perm);
    /* insertion sort, ascending */
    for (int i = 1; i < l; ++i) {
        int v = idx[i], k = i - 1;
        while (k >= 0 && idx[k] > v) { idx[k + 1] = idx[k]; --k; }
        idx[k + 1] = v;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Eq. 2: S = (1/N) Y Y^H.  X is complex64 interleaved (re, im), row-major   */
/* M x T with leading dimension ldx (complex elements).                      */
/* ------------------------------------------------------------------------ */
int orc_covariance(const float* X, int M, int T, int64_t ldx, zc* R)
{
    if (M < 1 || T < 1 || ldx < T) return ORC_ERR_ARG;
    for (int i = 0; i < M; ++i) {
        for (int j = 0; j < M; ++j) {
            zc acc = 0.0;
            for (int t = 0; t < T; ++t) {
                const float* xi = X + 2 * ((size_t)i * ldx + t);
                const float* xj = X + 2 * ((size_t)j * ldx + t);
                zc a = (double)xi[0] + I * (double)xi[1];
                zc b = (double)xj[0] + I * (double)xj[1];
                acc += a * conj(b);
            }
            R[(size_t)i * M + j] = acc / (double)T;
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Dense helpers (row-major, naive).                                         */
/* ------------------------------------------------------------------------ */
/* C (m x n) = A (m x k) * B (k x n) */
static void zgemm_nn(int m, int n, int k, const zc* A, const zc* B, zc* C)
{
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j) {
            zc acc = 0.0;
            for (int p = 0; p < k; ++p) acc += A[(size_t)i * k + p] * B[(size_t)p * n + j];
            C[(size_t)i * n + j] = acc;
        }
}
/* C (m x n) = A^H * B, A is k x m, B is k x n */
static void zgemm_hn(int m, int n, int k, const zc* A, const zc* B, zc* C)
{
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j) {
            zc acc = 0.0;
            for (int p = 0; p < k; ++p) acc += conj(A[(size_t)p * m + i]) * B[(size_t)p * n + j];
            C[(size_t)i * n + j] = acc;
        }
}

/* ------------------------------------------------------------------------ */
/* Hermitian eigendecomposition by the cyclic (row-by-row) two-sided Jacobi  */
/* method.  Each rotation first removes the phase of A_pq with D =            */
/* diag(1, e^{-i phi}), then applies the real symmetric 2x2 Jacobi rotation  */
/* (tau = (a_qq - a_pp) / (2|a_pq|), t = sign(tau)/(|tau| + sqrt(1+tau^2)),    */
/* c = 1/sqrt(1+t^2), s = t c), i.e. U = [[c, s], [-s e^{-i phi}, c e^{-i phi}]] */
/* with A <- U^H A U, V <- V U.  Sweeps stop when                              */
/* off(A) <= tol * ||A||_F.  A (n x n, row-major) is overwritten; on return w */
/* holds eigenvalues in descending order and column k of V (row-major, n x n) */
/* the matching unit eigenvector.  Returns the number of sweeps or           */
/* ORC_ERR_NOCONV.                                                            */
/* ------------------------------------------------------------------------ */
int orc_eigh_jacobi(int n, zc* A, double* w, zc* V, double tol, int max_sweeps)
{
    if (n < 1) return ORC_ERR_ARG;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) V[(size_t)i * n + j] = (i == j) ? 1.0 : 0.0;
    /* Hermitise: use the upper triangle as the definition */
    for (int i = 0; i < n; ++i) {
        A[(size_t)i * n + i] = creal(A[(size_t)i * n + i]);
        for (int j = i + 1; j < n; ++j) A[(size_t)j * n + i] = conj(A[(size_t)i * n + j]);
    }
    double fro = 0.0;
    for (size_t e = 0; e < (size_t)n * n; ++e) fro += creal(A[e] * conj(A[e]));
    fro = sqrt(fro);
    int sweep = 0;
    for (;;) {
        double off = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                if (i != j) off += creal(A[(size_t)i * n + j] * conj(A[(size_t)i * n + j]));
        off = sqrt(off);
        if (off <= tol * fro || fro == 0.0) break;
        if (sweep >= max_sweeps) return ORC_ERR_NOCONV;
        ++sweep;
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                zc apq = A[(size_t)p * n + q];
                double mag = cabs(apq);
                if (mag == 0.0) continue;
                double app = creal(A[(size_t)p * n + p]);
                double aqq = creal(A[(size_t)q * n + q]);
                zc ph = apq / mag; /* e^{i phi} */
                double tau = (aqq - app) / (2.0 * mag);
                double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t);
                double s = t * c;
                zc upp = c, upq = s, uqp = -s * conj(ph), uqq = c * conj(ph);
                /* columns: A <- A U */
                for (int i = 0; i < n; ++i) {
                    zc aip = A[(size_t)i * n + p], aiq = A[(size_t)i * n + q];
                    A[(size_t)i * n + p] = aip * upp + aiq * uqp;
                    A[(size_t)i * n + q] = aip * upq + aiq * uqq;
                }
                /* rows: A <- U^H A */
                for (int j = 0; j < n; ++j) {
                    zc apj = A[(size_t)p * n + j], aqj = A[(size_t)q * n + j];
                    A[(size_t)p * n + j] = conj(upp) * apj + conj(uqp) * aqj;
                    A[(size_t)q * n + j] = conj(upq) * apj + conj(uqq) * aqj;
                }
                A[(size_t)p * n + q] = 0.0;
                A[(size_t)q * n + p] = 0.0;
                A[(size_t)p * n + p] = creal(A[(size_t)p * n + p]);
                A[(size_t)q * n + q] = creal(A[(size_t)q * n + q]);
                /* eigenvectors: V <- V U */
                for (int i = 0; i < n; ++i) {
                    zc vip = V[(size_t)i * n + p], viq = V[(size_t)i * n + q];
                    V[(size_t)i * n + p] = vip * upp + viq * uqp;
                    V[(size_t)i * n + q] = vip * upq + viq * uqq;
                }
            }
        }
    }
    for (int i = 0; i < n; ++i) w[i] = creal(A[(size_t)i * n + i]);
    /* selection sort, descending; ties keep the lower index first */
    for (int i = 0; i < n - 1; ++i) {
        int best = i;
        for (int j = i + 1; j < n; ++j)
            if (w[j] > w[best]) best = j;
        if (best != i) {
            double tw = w[i]; w[i] = w[best]; w[best] = tw;
            for (int r = 0; r < n; ++r) {
                zc tv = V[(size_t)r * n + i];
                V[(size_t)r * n + i] = V[(size_t)r * n + best];
                V[(size_t)r * n + best] = tv;
            }
        }
    }
    return sweep;
}

/* ------------------------------------------------------------------------ */
/* Thin SVD A = U diag(s) W^H of an m x n matrix (m >= n) by one-sided        */
/* (Hestenes) Jacobi: rotate column pairs of A until all are orthogonal; the */
/* accumulated rotations form W, the column norms are s, and the normalised  */
/* columns are U.  Columns with zero norm give zero U columns.  Outputs are   */
/* sorted by s descending.  U is m x n, W is n x n (row-major).               */
/* ------------------------------------------------------------------------ */
int orc_svd_jacobi(int m, int n, const zc* A, zc* U, double* s, zc* W, double tol, int max_sweeps)
{
    if (m < n || n < 1) return ORC_ERR_ARG;
    zc* G = (zc*)malloc(sizeof(zc) * (size_t)m * n);
    if (!G) return ORC_ERR_MEM;
    memcpy(G, A, sizeof(zc) * (size_t)m * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) W[(size_t)i * n + j] = (i == j) ? 1.0 : 0.0;
    int sweep = 0, converged = 0;
    while (sweep < max_sweeps) {
        ++sweep;
        int rotated = 0;
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                double alpha = 0.0, beta = 0.0;
                zc gamma = 0.0; /* a_p^H a_q */
                for (int i = 0; i < m; ++i) {
                    zc gp = G[(size_t)i * n + p], gq = G[(size_t)i * n + q];
                    alpha += creal(gp * conj(gp));
                    beta += creal(gq * conj(gq));
                    gamma += conj(gp) * gq;
                }
                double mag = cabs(gamma);
                if (mag == 0.0 || mag <= tol * sqrt(alpha * beta)) continue;
                rotated = 1;
                /* Jacobi rotation of the 2x2 Gram block [[alpha, gamma],[conj(gamma), beta]] */
                zc ph = gamma / mag;
                double tau = (beta - alpha) / (2.0 * mag);
                double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t);
                double sn = t * c;
                zc upp = c, upq = sn, uqp = -sn * conj(ph), uqq = c * conj(ph);
                for (int i = 0; i < m; ++i) {
                    zc gp = G[(size_t)i * n + p], gq = G[(size_t)i * n + q];
                    G[(size_t)i * n + p] = gp * upp + gq * uqp;
                    G[(size_t)i * n + q] = gp * upq + gq * uqq;
                }
                for (int i = 0; i < n; ++i) {
                    zc wp = W[(size_t)i * n + p], wq = W[(size_t)i * n + q];
                    W[(size_t)i * n + p] = wp * upp + wq * uqp;
                    W[(size_t)i * n + q] = wp * upq + wq * uqq;
                }
            }
        }
        if (!rotated) { converged = 1; break; }
    }
    for (int j = 0; j < n; ++j) {
        double nrm = 0.0;
        for (int i = 0; i < m; ++i) nrm += creal(G[(size_t)i * n + j] * conj(G[(size_t)i * n + j]));
        s[j] = sqrt(nrm);
        for (int i = 0; i < m; ++i) U[(size_t)i * n + j] = (s[j] > 0.0) ? G[(size_t)i * n + j] / s[j] : 0.0;
    }
    free(G);
    for (int i = 0; i < n - 1; ++i) {
        int best = i;
        for (int j = i + 1; j < n; ++j)
            if (s[j] > s[best]) best = j;
        if (best != i) {
            double ts = s[i]; s[i] = s[best]; s[best] = ts;
            for (int r = 0; r < m; ++r) {
                zc tu = U[(size_t)r * n + i]; U[(size_t)r * n + i] = U[(size_t)r * n + best]; U[(size_t)r * n + best] = tu;
            }
            for (int r = 0; r < n; ++r) {
                zc tw = W[(size_t)r * n + i]; W[(size_t)r * n + i] = W[(size_t)r * n + best]; W[(size_t)r * n + best] = tw;
            }
        }
    }
    return converged ? sweep : ORC_ERR_NOCONV;
}

/* ------------------------------------------------------------------------ */
/* Thin QR A = Q R (m x n, m >= n) by Householder reflections.  Reflector k   */
/* maps x = A[k:,k] to alpha e1 with alpha = -e^{i arg x0} ||x||.  Q is m x n */
/* with orthonormal columns, R is n x n upper triangular.  This is the       */
/* qr()/orth() of Sec. III-B.                                                 */
/* ------------------------------------------------------------------------ */
int orc_householder_qr(int m, int n, const zc* A, zc* Q, zc* R)
{
    if (m < n || n < 1) return ORC_ERR_ARG;
    zc* Wk = (zc*)malloc(sizeof(zc) * (size_t)m * n);
    zc* vs = (zc*)calloc((size_t)m * n, sizeof(zc)); /* reflector k stored in column k */
    int* used = (int*)calloc((size_t)n, sizeof(int));
    if (!Wk || !vs || !used) { free(Wk); free(vs); free(used); return ORC_ERR_MEM; }
    memcpy(Wk, A, sizeof(zc) * (size_t)m * n);
    for (int k = 0; k < n; ++k) {
        double xn = 0.0;
        for (int i = k; i < m; ++i) xn += creal(Wk[(size_t)i * n + k] * conj(Wk[(size_t)i * n + k]));
        xn = sqrt(xn);
        if (xn == 0.0) continue;
        zc x0 = Wk[(size_t)k * n + k];
        zc ph = (cabs(x0) > 0.0) ? x0 / cabs(x0) : 1.0;
        zc alpha = -ph * xn;
        double vn = 0.0;
        for (int i = k; i < m; ++i) {
            zc v = Wk[(size_t)i * n + k] - ((i == k) ? alpha : 0.0);
            vs[(size_t)i * n + k] = v;
            vn += creal(v * conj(v));
        }
        vn = sqrt(vn);
        if (vn == 0.0) continue;
        for (int i = k; i < m; ++i) vs[(size_t)i * n + k] /= vn;
        used[k] = 1;
        /* apply H = I - 2 v v^H to columns k..n-1 */
        for (int j = k; j < n; ++j) {
            zc d = 0.0;
            for (int i = k; i < m; ++i) d += conj(vs[(size_t)i * n + k]) * Wk[(size_t)i * n + j];
            for (int i = k; i < m; ++i) Wk[(size_t)i * n + j] -= 2.0 * vs[(size_t)i * n + k] * d;
        }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) R[(size_t)i * n + j] = (j >= i) ? Wk[(size_t)i * n + j] : 0.0;
    /* Q = H_0 H_1 ... H_{n-1} [I_n; 0] */
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j) Q[(size_t)i * n + j] = (i == j) ? 1.0 : 0.0;
    for (int k = n - 1; k >= 0; --k) {
        if (!used[k]) continue;
        for (int j = 0; j < n; ++j) {
            zc d = 0.0;
            for (int i = k; i < m; ++i) d += conj(vs[(size_t)i * n + k]) * Q[(size_t)i * n + j];
            for (int i = k; i < m; ++i) Q[(size_t)i * n + j] -= 2.0 * vs[(size_t)i * n + k] * d;
        }
    }
    free(Wk); free(vs); free(used);
    return ORC_OK;
}

/* Moore-Penrose pseudo-inverse of a Hermitian n x n matrix via its Jacobi    */
/* eigendecomposition; eigenvalues with |lambda| <= n*eps64*max|lambda| are   */
/* treated as zero.  Returns the numerical rank.                              */
int orc_pinv_hermitian(int n, const zc* H, zc* Wout)
{
    zc* A = (zc*)malloc(sizeof(zc) * (size_t)n * n);
    zc* V = (zc*)malloc(sizeof(zc) * (size_t)n * n);
    double* w = (double*)malloc(sizeof(double) * (size_t)n);
    if (!A || !V || !w) { free(A); free(V); free(w); return ORC_ERR_MEM; }
    memcpy(A, H, sizeof(zc) * (size_t)n * n);
    int rc = orc_eigh_jacobi(n, A, w, V, 1e-14, 60);
    if (rc < 0) { free(A); free(V); free(w); return rc; }
    double amax = 0.0;
    for (int i = 0; i < n; ++i) if (fabs(w[i]) > amax) amax = fabs(w[i]);
    double thr = (double)n * 2.220446049250313e-16 * amax;
    int rank = 0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Wout[(size_t)i * n + j] = 0.0;
    for (int k = 0; k < n; ++k) {
        if (!(fabs(w[k]) > thr)) continue;
        ++rank;
        double inv = 1.0 / w[k];
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                Wout[(size_t)i * n + j] += V[(size_t)i * n + k] * inv * conj(V[(size_t)j * n + k]);
    }
    free(A); free(V); free(w);
    return rank;
}

/* ------------------------------------------------------------------------ */
/* Standard MUSIC subspace (Eq. 4): U_K = the K leading eigenvectors of S.    */
/* U is M x K row-major; lam (optional, length M) receives all eigenvalues.  */
/* ------------------------------------------------------------------------ */
int orc_music_subspace(const zc* R, int M, int K, zc* U, double* lam)
{
    if (K < 1 || K > M) return ORC_ERR_ARG;
    zc* A = (zc*)malloc(sizeof(zc) * (size_t)M * M);
    zc* V = (zc*)malloc(sizeof(zc) * (size_t)M * M);
    double* w = (double*)malloc(sizeof(double) * (size_t)M);
    if (!A || !V || !w) { free(A); free(V); free(w); return ORC_ERR_MEM; }
    memcpy(A, R, sizeof(zc) * (size_t)M * M);
    int rc = orc_eigh_jacobi(M, A, w, V, 1e-14, 50);
    if (rc >= 0) {
        for (int i = 0; i < M; ++i)
            for (int k = 0; k < K; ++k) U[(size_t)i * K + k] = V[(size_t)i * M + k];
        if (lam) memcpy(lam, w, sizeof(double) * (size_t)M);
    }
    free(A); free(V); free(w);
    return rc < 0 ? rc : ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Fast MUSIC (Algorithms 1 and 2).                                           */
/*   method 1: random sampling (Sec. III-A); method 2: Gaussian projection    */
/*   (Sec. III-B).  l = sketch size p, t = power iterations.                  */
/*   form 0: rank restriction as printed -- SVD C = U_c S_c V_c^H,            */
/*           B = S_c V_c^H W V_c S_c, eig B = U_B L_B U_B^H, U~ = U_c U_B.       */
/*   form 1: the equivalent QR route -- C = Q R_c, B' = R_c W R_c^H,          */
/*           U~ = Q U_B' (Q = U_c Z with Z unitary, so both give one subspace). */
/* Output: U (M x ncols, ncols = K or l), optional lamB (l eigenvalues of B), */
/* optional idx (l sampled indices, method 1).                               */
/* ------------------------------------------------------------------------ */
int orc_fast_music(const zc* R, int M, int K, int l, int t, int method, uint64_t seed,
                   uint64_t frame_id, int ncols, int form, zc* U, double* lamB, int* idx_out)
{
    if (M < 2 || K < 1 || K > l || l > M || t < 0 || (method != 1 && method != 2) ||
        (ncols != K && ncols != l) || (form != 0 && form != 1))
        return ORC_ERR_ARG;
    int rc = ORC_OK;
    size_t Ml = (size_t)M * l, ll = (size_t)l * l;
    zc* Pi = (zc*)calloc(Ml, sizeof(zc));
    zc* C = (zc*)malloc(sizeof(zc) * Ml);
    zc* P = (zc*)malloc(sizeof(zc) * Ml);
    zc* Vq = (zc*)malloc(sizeof(zc) * Ml);
    zc* Rq = (zc*)malloc(sizeof(zc) * ll);
    zc* H = (zc*)malloc(sizeof(zc) * ll);
    zc* W = (zc*)malloc(sizeof(zc) * ll);
    zc* B = (zc*)malloc(sizeof(zc) * ll);
    zc* T1 = (zc*)malloc(sizeof(zc) * ll);
    zc* UB = (zc*)malloc(sizeof(zc) * ll);
    zc* Ub = (zc*)malloc(sizeof(zc) * Ml);
    zc* Wsv = (zc*)malloc(sizeof(zc) * ll);
    double* sv = (double*)malloc(sizeof(double) * (size_t)l);
    double* wl = (double*)malloc(sizeof(double) * (size_t)l);
    int* idx = (int*)malloc(sizeof(int) * (size_t)l);
    if (!Pi || !C || !P || !Vq || !Rq || !H || !W || !B || !T1 || !UB || !Ub || !Wsv || !sv || !wl || !idx) {
        rc = ORC_ERR_MEM;
        goto done;
    }

    /* Step 1: sketch C = S Pi (the sketch step of Algorithms 1 and 2) */
    if (method == 1) {
        rc = orc_sample_indices(seed, frame_id, M, l, idx);
        if (rc < 0) goto done;
        for (int j = 0; j < l; ++j) Pi[(size_t)idx[j] * l + j] = 1.0;
        for (int i = 0; i < M; ++i)
            for (int j = 0; j < l; ++j) C[(size_t)i * l + j] = R[(size_t)i * M + idx[j]];
        if (idx_out) memcpy(idx_out, idx, sizeof(int) * (size_t)l);
    } else {
        orc_gaussian_test_matrix(seed, frame_id, M, l, Pi);
        zgemm_nn(M, l, M, R, Pi, C);
    }
    memcpy(P, Pi, sizeof(zc) * Ml);
    /* power iterations (Eq. 11, Algorithm 2): V = orth(C), C = S V */
    for (int it = 0; it < t; ++it) {
        rc = orc_householder_qr(M, l, C, Vq, Rq);
        if (rc < 0) goto done;
        zgemm_nn(M, l, M, R, Vq, C);
        memcpy(P, Vq, sizeof(zc) * Ml);
    }
    /* core matrix: W = pinv(P^H S P) = pinv(P^H C) (Eq. 8, Algorithm 2) */
    zgemm_hn(l, l, M, P, C, H);
    for (int i = 0; i < l; ++i) /* exact Hermitian part */
        for (int j = i; j < l; ++j) {
            zc h = 0.5 * (H[(size_t)i * l + j] + conj(H[(size_t)j * l + i]));
            H[(size_t)i * l + j] = h;
            H[(size_t)j * l + i] = conj(h);
        }
    rc = orc_pinv_hermitian(l, H, W);
    if (rc < 0) goto done;

    /* Step 2: rank restriction */
    if (form == 0) {
        /* SVD of C (Algorithms 1 and 2): U_c = Vq, Sigma_c = sv, V_c = Wsv */
        rc = orc_svd_jacobi(M, l, C, Vq, sv, Wsv, fmax(1e-14, (double)M * 2.220446049250313e-16), 60);
        if (rc < 0) goto done;
        /* B = Sigma_c V_c^H W V_c Sigma_c (rank restriction, Algorithm 1) */
        zgemm_hn(l, l, l, Wsv, W, T1);   /* V_c^H W */
        zgemm_nn(l, l, l, T1, Wsv, B);   /* (V_c^H W) V_c */
        for (int i = 0; i < l; ++i)
            for (int j = 0; j < l; ++j) B[(size_t)i * l + j] *= sv[i] * sv[j];
    } else {
        /* C = Q R_c, B' = R_c W R_c^H */
        rc = orc_householder_qr(M, l, C, Vq, Rq);
        if (rc < 0) goto done;
        zgemm_nn(l, l, l, Rq, W, T1);
        for (int i = 0; i < l; ++i)
            for (int j = 0; j < l; ++j) {
                zc acc = 0.0;
                for (int p = 0; p < l; ++p) acc += T1[(size_t)i * l + p] * conj(Rq[(size_t)j * l + p]);
                B[(size_t)i * l + j] = acc;
            }
    }
    /* SVD of the Hermitian PSD B = eigendecomposition, descending (Algorithm 1) */
    rc = orc_eigh_jacobi(l, B, wl, UB, 1e-14, 60);
    if (rc < 0) goto done;
    if (lamB) memcpy(lamB, wl, sizeof(double) * (size_t)l);
    /* U~ = U_c U_B (Algorithm 1) */
    zgemm_nn(M, l, l, Vq, UB, Ub);
    for (int i = 0; i < M; ++i)
        for (int k = 0; k < ncols; ++k) U[(size_t)i * ncols + k] = Ub[(size_t)i * l + k];
    rc = ORC_OK;
done:
    free(Pi); free(C); free(P); free(Vq); free(Rq); free(H); free(W); free(B); free(T1);
    free(UB); free(Ub); free(Wsv); free(sv); free(wl); free(idx);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Pseudo-spectrum (Eq. 5 / Eq. 10) on the grid theta_i = theta0 + i*step    */
/* (degrees):  P_i = 1 / (||a||^2 - ||U^H a||^2) with the far-field steering   */
/* vector of Sec. II-A, a_m = exp(j 2 pi x_m sin theta_i), x_m the position   */
/* of element m in wavelengths: x_m = d m for a uniform linear array        */
/* (pos == NULL), else x_m = pos[m].  residual_form = 1 evaluates the same    */
/* quantity as 1 / ||a - U U^H a||^2 (no cancellation).                      */
/* ------------------------------------------------------------------------ */
int orc_spectrum(const zc* U, int M, int ncols, double d, const double* pos, double theta0_deg,
                 double step_deg, int L, int residual_form, double* P)
{
    if (M < 1 || ncols < 1 || L < 1) return ORC_ERR_ARG;
    zc* a = (zc*)malloc(sizeof(zc) * (size_t)M);
    zc* c = (zc*)malloc(sizeof(zc) * (size_t)ncols);
    if (!a || !c) { free(a); free(c); return ORC_ERR_MEM; }
    for (int i = 0; i < L; ++i) {
        double th = (theta0_deg + (double)i * step_deg) * M_PI / 180.0;
        double s = sin(th);
        double an = 0.0;
        for (int m = 0; m < M; ++m) {
            double ph = pos ? 2.0 * M_PI * pos[m] * s : 2.0 * M_PI * d * (double)m * s;
            a[m] = cos(ph) + I * sin(ph);
            an += creal(a[m] * conj(a[m]));
        }
        for (int k = 0; k < ncols; ++k) {
            zc acc = 0.0;
            for (int m = 0; m < M; ++m) acc += conj(U[(size_t)m * ncols + k]) * a[m];
            c[k] = acc;
        }
        double den;
        if (residual_form) {
            den = 0.0;
            for (int m = 0; m < M; ++m) {
                zc r = a[m];
                for (int k = 0; k < ncols; ++k) r -= U[(size_t)m * ncols + k] * c[k];
                den += creal(r * conj(r));
            }
        } else {
            double cn = 0.0;
            for (int k = 0; k < ncols; ++k) cn += creal(c[k] * conj(c[k]));
            den = an - cn;
        }
        P[i] = (den > 0.0) ? 1.0 / den : INFINITY;
    }
    free(a); free(c);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Peak search (Eq. 6): the K largest local maxima of P.                     */
/* Outputs idx[0..K-1] ordered by P descending (ties: lower index first),    */
/* unused slots set to -1; *n_found = number of maxima returned.             */
/* ------------------------------------------------------------------------ */
int orc_peaks(const double* P, int L, int K, int* idx, int* n_found)
{
    if (L < 1 || K < 1) return ORC_ERR_ARG;
    for (int k = 0; k < K; ++k) idx[k] = -1;
    int n = 0;
    for (int i = 0; i < L; ++i) {
        int left_ok = (i == 0) || (P[i] > P[i - 1]);
        int right_ok = (i == L - 1) || (P[i] >= P[i + 1]);
        if (!(left_ok && right_ok)) continue;
        /* insert i into the ordered list (P desc, index asc) if it ranks */
        int pos = n;
        while (pos > 0 && (P[i] > P[idx[pos - 1]])) --pos;
        if (pos >= K) continue;
        int last = (n < K) ? n : K - 1;
        for (int k = last; k > pos; --k) idx[k] = idx[k - 1];
        idx[pos] = i;
        if (n < K) ++n;
    }
    *n_found = n;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* One whole frame: X -> S -> subspace -> spectrum -> peaks.                  */
/* method 0 = standard MUSIC (full eigendecomposition), 1 / 2 = fast MUSIC.   */
/* P (length L) and peak_idx (length K) are outputs.                          */
/* ------------------------------------------------------------------------ */
int orc_frame(const float* X, int M, int T, int64_t ldx, int K, int l, int t, int method,
              uint64_t seed, uint64_t frame_id, double d, const double* pos, double theta0_deg,
              double step_deg, int L, double* P, int* peak_idx, int* n_peaks)
{
    zc* R = (zc*)malloc(sizeof(zc) * (size_t)M * M);
    zc* U = (zc*)malloc(sizeof(zc) * (size_t)M * K);
    if (!R || !U) { free(R); free(U); return ORC_ERR_MEM; }
    int rc = orc_covariance(X, M, T, ldx, R);
    if (rc == ORC_OK) {
        if (method == 0)
            rc = orc_music_subspace(R, M, K, U, NULL);
        else
            rc = orc_fast_music(R, M, K, l, t, method, seed, frame_id, K, 0, U, NULL, NULL);
    }
    if (rc == ORC_OK) rc = orc_spectrum(U, M, K, d, pos, theta0_deg, step_deg, L, 0, P);
    if (rc == ORC_OK) rc = orc_peaks(P, L, K, peak_idx, n_peaks);
    free(R); free(U);
    return rc;
}
