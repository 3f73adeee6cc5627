// small.cu -- per-frame l x l work of Algorithms 1 and 2 (Sec. III), one CTA per frame.
//
//   ORTH  (power step, Eq. 11):  V = orth(C)
//   FINAL (Alg. 1 lines 5-9 / Alg. 2 lines 7-10):
//         H = P^H C  with P = V (t >= 1), the index selection (sampling, t = 0)
//                    or the Gaussian Pi regenerated from Philox (projection, t = 0)
//         W = pinv(H)                                    (Eq. 8)
//         C = Q R_c                                      (QR in place of SVD(C); same subspace)
//         B = R_c W R_c^H, eig(B) = U_B L_B U_B^H        (rank restriction)
//         U_s = Q U_B[:, :ncols]
//
// orth / QR use CholeskyQR2 with a mixed-precision first pass: the Gram matrix
// C^H C is accumulated in double-float arithmetic (each FP32 product split
// exactly with an FMA, sums carried as unevaluated (hi, lo) pairs) and factored
// in FP64, so the first pass survives cond(C) up to ~1/u_fp32; the second pass
// (cond ~ 1) runs in FP32.  The two Hermitian l x l eigenproblems use a
// parallel-ordered (round-robin) two-sided complex Jacobi method in FP32 with
// the relative stopping test |a_pq| <= tol sqrt(|a_pp a_qq|).
#include <float.h>

#include "fm_internal.cuh"

namespace fm {
namespace {

constexpr int kThreads = 256;
constexpr int kRowsChunk = 16;     // rows of an M x l operand staged per step
constexpr int kMaxItems = (kLMax * kLMax + kThreads - 1) / kThreads;  // Gram items per thread
constexpr int kMaxSweeps = 30;
constexpr float kJacobiTol = 1e-6f;

enum Mode { kOrth = 0, kFinal = 1 };
enum Src { kMem = 0, kOmega = 1 };

struct Sm {
    double2* G64;  // l*l   (pass-1 Gram / factor)
    double2* R64;  // l*l   (pass-1 inverse)
    float2* G;     // l*l   (FP32 Gram / factor)
    float2* Ri;    // l*l   (triangular inverse, FP32)
    float2* Rc;    // l*l   (accumulated R factor of the QR)
    float2* H;     // l*l   (core matrix, then B)
    float2* Z;     // l*l   (eigenvectors)
    float2* Y;     // l*l   (temp)
    float2* ca;    // kRowsChunk*l
    float2* cb;    // kRowsChunk*l
    float* w;      // l
    int* perm;     // l
    float4* rot;   // kLMax/2
    int2* pairs;   // kLMax/2
    int* flags;    // 8
    double* dscal; // 8
    double* dinv;  // kLMax
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline size_t smem_layout(int l, Sm* sm, char* base) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align16(off + bytes);
        return base ? base + o : nullptr;
    };
    const size_t ll = (size_t)l * l;
    // G64 and R64 are only live in the first CholQR pass; they alias G/Ri/Y/Z
    char* u0 = take(2 * ll * sizeof(double2));
    char* Rc = take(ll * sizeof(float2));
    char* H = take(ll * sizeof(float2));
    char* ca = take(kRowsChunk * (size_t)l * sizeof(float2));
    char* cb = take(kRowsChunk * (size_t)l * sizeof(float2));
    char* w = take(l * sizeof(float));
    char* perm = take(l * sizeof(int));
    char* rot = take((kLMax / 2 + 1) * sizeof(float4));
    char* pairs = take((kLMax / 2 + 1) * sizeof(int2));
    char* flags = take(8 * sizeof(int));
    char* dscal = take(8 * sizeof(double));
    char* dinv = take(kLMax * sizeof(double));
    if (sm) {
        sm->G64 = reinterpret_cast<double2*>(u0);
        sm->R64 = reinterpret_cast<double2*>(u0) + ll;
        sm->G = reinterpret_cast<float2*>(u0);
        sm->Ri = reinterpret_cast<float2*>(u0) + ll;
        sm->Y = reinterpret_cast<float2*>(u0) + 2 * ll;
        sm->Z = reinterpret_cast<float2*>(u0) + 3 * ll;
        sm->Rc = reinterpret_cast<float2*>(Rc);
        sm->H = reinterpret_cast<float2*>(H);
        sm->ca = reinterpret_cast<float2*>(ca);
        sm->cb = reinterpret_cast<float2*>(cb);
        sm->w = reinterpret_cast<float*>(w);
        sm->perm = reinterpret_cast<int*>(perm);
        sm->rot = reinterpret_cast<float4*>(rot);
        sm->pairs = reinterpret_cast<int2*>(pairs);
        sm->flags = reinterpret_cast<int*>(flags);
        sm->dscal = reinterpret_cast<double*>(dscal);
        sm->dinv = reinterpret_cast<double*>(dinv);
    }
    return off;
}

// ------------------------------------------------------------ double-float --
struct df {
    float hi, lo;
};
__device__ __forceinline__ void df_add_prod(df& s, float a, float b) {
    const float p = a * b;
    const float pe = fmaf(a, b, -p);  // exact: a*b = p + pe
    const float t = s.hi + p;         // TwoSum(s.hi, p) = t + e
    const float bp = t - s.hi;
    const float e = (s.hi - (t - bp)) + (p - bp);
    s.hi = t;
    s.lo += e + pe;
}
__device__ __forceinline__ df df_add(df a, df b) {
    const float t = a.hi + b.hi;
    const float bp = t - a.hi;
    const float e = (a.hi - (t - bp)) + (b.hi - bp);
    df r;
    r.hi = t;
    r.lo = e + a.lo + b.lo;
    return r;
}

// --------------------------------------------------------------- staging ---
// dst[r*l + j] = row (m0 + r) of an M x l operand (zeros past M).
__device__ __forceinline__ void load_chunk(const float2* __restrict__ src, int src_kind, const FrameDesc& d,
                                           int M, int l, int m0, float2* dst) {
    for (int e = threadIdx.x; e < kRowsChunk * l; e += kThreads) {
        const int r = e / l, j = e % l;
        const int m = m0 + r;
        float2 v = make_float2(0.f, 0.f);
        if (m < M) v = (src_kind == kOmega) ? gaussian_entry(d.seed, d.frame_id, m, j) : src[(int64_t)m * l + j];
        dst[e] = v;
    }
}

__device__ __forceinline__ void item_coords(int e, int l, bool herm, int& i, int& j) {
    if (!herm) {
        i = e / l;
        j = e % l;
        return;
    }
    i = 0;
    while (e >= l - i) {
        e -= l - i;
        ++i;
    }
    j = i + e;
}

// G = A^H B (l x l) in FP32 with per-chunk two-level accumulation.  B == nullptr
// means B = A (Hermitian: upper triangle computed, mirrored).
__device__ void gram_fp32(const float2* A, int a_kind, const float2* B, const FrameDesc& d, int M, int l,
                          const Sm& sm, float2* G) {
    const bool herm = (B == nullptr);
    const int nitems = herm ? l * (l + 1) / 2 : l * l;
    int ii[kMaxItems], jj[kMaxItems];
    float2 acc[kMaxItems];
#pragma unroll
    for (int q = 0; q < kMaxItems; ++q) {
        const int e = threadIdx.x + q * kThreads;
        ii[q] = jj[q] = 0;
        if (e < nitems) item_coords(e, l, herm, ii[q], jj[q]);
        acc[q] = make_float2(0.f, 0.f);
    }
    for (int m0 = 0; m0 < M; m0 += kRowsChunk) {
        load_chunk(A, a_kind, d, M, l, m0, sm.ca);
        if (!herm) load_chunk(B, kMem, d, M, l, m0, sm.cb);
        __syncthreads();
        const float2* bb = herm ? sm.ca : sm.cb;
#pragma unroll
        for (int q = 0; q < kMaxItems; ++q) {
            if (threadIdx.x + q * kThreads < nitems) {
                float2 t = make_float2(0.f, 0.f);
#pragma unroll
                for (int r = 0; r < kRowsChunk; ++r) cfmac(t, sm.ca[r * l + ii[q]], bb[r * l + jj[q]]);
                acc[q] = cadd(acc[q], t);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < kMaxItems; ++q) {
        if (threadIdx.x + q * kThreads < nitems) {
            float2 v = acc[q];
            if (herm && ii[q] == jj[q]) v.y = 0.f;
            G[ii[q] * l + jj[q]] = v;
            if (herm && ii[q] != jj[q]) G[jj[q] * l + ii[q]] = cconj(v);
        }
    }
    __syncthreads();
}

// G = A^H A in double-float accumulation, result in FP64.
__device__ void gram_df64(const float2* A, const FrameDesc& d, int M, int l, const Sm& sm, double2* G) {
    const int nitems = l * (l + 1) / 2;
    int ii[kMaxItems], jj[kMaxItems];
    df sre[kMaxItems], sim[kMaxItems];
#pragma unroll
    for (int q = 0; q < kMaxItems; ++q) {
        const int e = threadIdx.x + q * kThreads;
        ii[q] = jj[q] = 0;
        if (e < nitems) item_coords(e, l, true, ii[q], jj[q]);
        sre[q] = df{0.f, 0.f};
        sim[q] = df{0.f, 0.f};
    }
    for (int m0 = 0; m0 < M; m0 += kRowsChunk) {
        load_chunk(A, kMem, d, M, l, m0, sm.ca);
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kMaxItems; ++q) {
            if (threadIdx.x + q * kThreads < nitems) {
                for (int r = 0; r < kRowsChunk; ++r) {
                    const float2 a = sm.ca[r * l + ii[q]], b = sm.ca[r * l + jj[q]];
                    // conj(a) * b = (ar br + ai bi) + j (ar bi - ai br)
                    df_add_prod(sre[q], a.x, b.x);
                    df_add_prod(sre[q], a.y, b.y);
                    df_add_prod(sim[q], a.x, b.y);
                    df_add_prod(sim[q], -a.y, b.x);
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < kMaxItems; ++q) {
        if (threadIdx.x + q * kThreads < nitems) {
            const int i = ii[q], j = jj[q];
            double2 v = make_double2((double)sre[q].hi + (double)sre[q].lo, (double)sim[q].hi + (double)sim[q].lo);
            if (i == j) v.y = 0.0;
            G[i * l + j] = v;
            if (i != j) G[j * l + i] = make_double2(v.x, -v.y);
        }
    }
    __syncthreads();
}

// -------------------------------------------------------------- Cholesky ----
// In place: G (Hermitian) -> upper R with G = R^H R.  Returns false on a
// non-positive pivot (the pivot is then clamped so the factor stays finite).
template <typename T2, typename T>
__device__ bool cholesky_upper(T2* G, int l, int* flag, T* scratch) {
    if (threadIdx.x == 0) flag[0] = 0;
    __syncthreads();
    for (int k = 0; k < l; ++k) {
        if (threadIdx.x == 0) {
            T dkk = G[k * l + k].x;
            if (!(dkk > (T)0)) {
                flag[0] = 1;
                dkk = (T)1e-30;
            }
            const T r = sqrt(dkk);
            G[k * l + k].x = r;
            G[k * l + k].y = (T)0;
            scratch[0] = (T)1 / r;
        }
        __syncthreads();
        const T inv = scratch[0];
        for (int j = k + 1 + threadIdx.x; j < l; j += kThreads) {
            G[k * l + j].x *= inv;
            G[k * l + j].y *= inv;
        }
        __syncthreads();
        const int n = l - k - 1;
        for (int e = threadIdx.x; e < n * n; e += kThreads) {
            const int i = k + 1 + e / n, j = k + 1 + e % n;
            if (i <= j) {
                const T2 a = G[k * l + i], b = G[k * l + j];
                // G_ij -= conj(R_ki) R_kj
                G[i * l + j].x -= a.x * b.x + a.y * b.y;
                G[i * l + j].y -= a.x * b.y - a.y * b.x;
            }
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < l * l; e += kThreads) {
        const int i = e / l, j = e % l;
        if (i > j) {
            G[e].x = (T)0;
            G[e].y = (T)0;
        }
    }
    __syncthreads();
    return flag[0] == 0;
}

// X = R^{-1} for upper triangular R with real positive diagonal, by right-looking
// back substitution: row i of X is finalised as X_ij = (delta_ij - S_ij) / R_ii
// (S_ij = sum_{m>i} R_im X_mj, accumulated in X itself), then its contribution
// R_ki X_ij is added to the partial sums of all rows k < i in parallel.
// dinv: scratch for the l reciprocals of the diagonal.
template <typename T2, typename T>
__device__ void tri_inv_upper(const T2* R, T2* X, int l, T* dinv) {
    for (int e = threadIdx.x; e < l * l; e += kThreads) {
        X[e].x = (T)0;
        X[e].y = (T)0;
    }
    for (int i = threadIdx.x; i < l; i += kThreads) dinv[i] = (T)1 / R[i * l + i].x;
    __syncthreads();
    for (int i = l - 1; i >= 0; --i) {
        const T inv = dinv[i];
        for (int j = i + threadIdx.x; j < l; j += kThreads) {
            T2 x = X[i * l + j];
            x.x = ((j == i) ? (T)1 : (T)0) - x.x;
            x.y = -x.y;
            x.x *= inv;
            x.y *= inv;
            X[i * l + j] = x;
        }
        __syncthreads();
        const int w = l - i;
        for (int e = threadIdx.x; e < i * w; e += kThreads) {
            const int k = e / w, j = i + e % w;
            const T2 a = R[k * l + i], b = X[i * l + j];
            X[k * l + j].x += a.x * b.x - a.y * b.y;
            X[k * l + j].y += a.x * b.y + a.y * b.x;
        }
        __syncthreads();
    }
}

// dst (M x ld_dst) = src (M x l) * Tm (l x n_out, row stride ldt); columns
// n_out..n_pad-1 of dst are zero-filled.  upper: Tm is upper triangular.
// src may equal dst (rows are staged before they are overwritten).
__device__ void apply_rows(const float2* src, float2* dst, const FrameDesc& d, int M, int l, const float2* Tm,
                           int ldt, int n_out, int ld_dst, int n_pad, bool upper, const Sm& sm) {
    for (int m0 = 0; m0 < M; m0 += kRowsChunk) {
        load_chunk(src, kMem, d, M, l, m0, sm.ca);
        __syncthreads();
        for (int e = threadIdx.x; e < kRowsChunk * n_pad; e += kThreads) {
            const int r = e / n_pad, c = e % n_pad;
            const int m = m0 + r;
            if (m >= M) continue;
            float2 out = make_float2(0.f, 0.f);
            if (c < n_out) {
                const int kend = upper ? c : l - 1;
                for (int k = 0; k <= kend; ++k) cfma(out, sm.ca[r * l + k], Tm[k * ldt + c]);
            }
            dst[(int64_t)m * ld_dst + c] = out;
        }
        __syncthreads();
    }
}

// dst (M x l) = src (M x l) * Ri with Ri upper triangular given as an
// unevaluated sum Ri = hi + lo of two FP32 matrices; products with hi are split
// exactly (FMA) and summed in double-float, so the result is the correctly
// scaled combination up to one final rounding even when Ri is ill-conditioned.
__device__ void apply_rows_df(const float2* src, float2* dst, const FrameDesc& d, int M, int l, const float2* Rhi,
                              const float2* Rlo, const Sm& sm) {
    for (int m0 = 0; m0 < M; m0 += kRowsChunk) {
        load_chunk(src, kMem, d, M, l, m0, sm.ca);
        __syncthreads();
        for (int e = threadIdx.x; e < kRowsChunk * l; e += kThreads) {
            const int r = e / l, c = e % l;
            const int m = m0 + r;
            if (m >= M) continue;
            df re{0.f, 0.f}, im{0.f, 0.f};
            for (int k = 0; k <= c; ++k) {
                const float2 a = sm.ca[r * l + k];
                const float2 h = Rhi[k * l + c], w = Rlo[k * l + c];
                df_add_prod(re, a.x, h.x);
                df_add_prod(re, -a.y, h.y);
                df_add_prod(im, a.x, h.y);
                df_add_prod(im, a.y, h.x);
                re.lo = fmaf(a.x, w.x, fmaf(-a.y, w.y, re.lo));
                im.lo = fmaf(a.x, w.y, fmaf(a.y, w.x, im.lo));
            }
            dst[(int64_t)m * l + c] = make_float2(re.hi + re.lo, im.hi + im.lo);
        }
        __syncthreads();
    }
}

// Rc <- Rk * Rc (both l x l upper triangular), using tmp as scratch.
__device__ void upper_mul_inplace(const float2* Rk, float2* Rc, float2* tmp, int l) {
    for (int e = threadIdx.x; e < l * l; e += kThreads) {
        const int i = e / l, j = e % l;
        float2 s = make_float2(0.f, 0.f);
        if (i <= j)
            for (int k = i; k <= j; ++k) cfma(s, Rk[i * l + k], Rc[k * l + j]);
        tmp[e] = s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < l * l; e += kThreads) Rc[e] = tmp[e];
    __syncthreads();
}

// CholeskyQR2: src (M x l) = Q * Rc, Q written to dst (may be src).  Returns
// false if a Cholesky pivot failed.
__device__ bool cholqr2(const float2* src, float2* dst, const FrameDesc& d, int M, int l, const Sm& sm) {
    // pass 1: double-float Gram, FP64 Cholesky and inverse
    gram_df64(src, d, M, l, sm, sm.G64);
    bool ok = cholesky_upper<double2, double>(sm.G64, l, sm.flags + 4, sm.dinv);
    tri_inv_upper<double2, double>(sm.G64, sm.R64, l, sm.dinv);
    // Rc = R1 in FP32, then R1^{-1} (FP64, in R64) as hi + lo FP32 pairs in the
    // slots of G64 (G = hi, Ri = lo), which are free once Rc is taken.
    for (int e = threadIdx.x; e < l * l; e += kThreads) {
        const double2 r = sm.G64[e];
        sm.Rc[e] = make_float2((float)r.x, (float)r.y);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < l * l; e += kThreads) {
        const double2 r = sm.R64[e];
        const float hx = (float)r.x, hy = (float)r.y;
        sm.G[e] = make_float2(hx, hy);
        sm.Ri[e] = make_float2((float)(r.x - (double)hx), (float)(r.y - (double)hy));
    }
    __syncthreads();
    apply_rows_df(src, dst, d, M, l, sm.G, sm.Ri, sm);
    // pass 2 in FP32 (cond ~ 1)
    gram_fp32(dst, kMem, nullptr, d, M, l, sm, sm.G);
    ok = cholesky_upper<float2, float>(sm.G, l, sm.flags + 4, reinterpret_cast<float*>(sm.dinv)) && ok;
    tri_inv_upper<float2, float>(sm.G, sm.Ri, l, reinterpret_cast<float*>(sm.dinv));
    apply_rows(dst, dst, d, M, l, sm.Ri, l, l, l, l, true, sm);
    upper_mul_inplace(sm.G, sm.Rc, sm.Y, l);
    return ok;
}

// ---------------------------------------------------------------- Jacobi ----
// Eigendecomposition of the Hermitian n x n matrix A (destroyed; its diagonal
// ends up holding the eigenvalues).  Z receives the eigenvectors (columns), w
// the eigenvalues, perm the column order by eigenvalue descending (ties: lower
// index).  Returns the number of sweeps, or -1 if the sweep cap was hit.
__device__ int jacobi_herm(float2* A, float2* Z, float* w, int* perm, int n, const Sm& sm) {
    for (int e = threadIdx.x; e < n * n; e += kThreads)
        Z[e] = (e / n == e % n) ? make_float2(1.f, 0.f) : make_float2(0.f, 0.f);
    const int ne = n + (n & 1), npairs = ne / 2, nr = ne - 1;
    int sweeps = -1;
    __syncthreads();
    for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
        if (threadIdx.x == 0) sm.flags[0] = 0;
        __syncthreads();
        for (int r = 0; r < nr; ++r) {
            if (threadIdx.x < npairs) {
                const int k = threadIdx.x;
                const int pa = (k == 0) ? 0 : 1 + ((k - 1 + r) % nr);
                const int pb = 1 + ((ne - 2 - k + r) % nr);
                const int p = min(pa, pb), q = max(pa, pb);
                int2 pr = make_int2(-1, -1);
                float4 rt = make_float4(1.f, 0.f, 1.f, 0.f);
                if (q < n && nr > 0) {
                    const float2 apq = A[p * n + q];
                    const float mag = sqrtf(cabs2(apq));
                    const float app = A[p * n + p].x, aqq = A[q * n + q].x;
                    if (mag > 1e-30f && mag > kJacobiTol * sqrtf(fabsf(app * aqq))) {
                        const float phr = apq.x / mag, phi = apq.y / mag;
                        const float tau = (aqq - app) / (2.f * mag);
                        float t;
                        if (fabsf(tau) > 1e18f)
                            t = 0.5f / tau;
                        else
                            t = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(fmaf(tau, tau, 1.f)));
                        const float c = rsqrtf(fmaf(t, t, 1.f));
                        rt = make_float4(c, t * c, phr, phi);
                        pr = make_int2(p, q);
                        sm.flags[0] = 1;
                    }
                }
                sm.pairs[k] = pr;
                sm.rot[k] = rt;
            }
            __syncthreads();
            // A <- A U and Z <- Z U, U = [[c, s], [-s conj(ph), c conj(ph)]]
            for (int e = threadIdx.x; e < npairs * n; e += kThreads) {
                const int k = e / n, i = e % n;
                const int2 pr = sm.pairs[k];
                if (pr.x < 0) continue;
                const float4 rt = sm.rot[k];
                const float c = rt.x, s = rt.y;
                const float2 phc = make_float2(rt.z, -rt.w);
                const float2 uqp = cscale(phc, -s), uqq = cscale(phc, c);
                float2 x = A[i * n + pr.x], y = A[i * n + pr.y];
                A[i * n + pr.x] = cadd(cscale(x, c), cmul(y, uqp));
                A[i * n + pr.y] = cadd(cscale(x, s), cmul(y, uqq));
                x = Z[i * n + pr.x];
                y = Z[i * n + pr.y];
                Z[i * n + pr.x] = cadd(cscale(x, c), cmul(y, uqp));
                Z[i * n + pr.y] = cadd(cscale(x, s), cmul(y, uqq));
            }
            __syncthreads();
            // A <- U^H A: row p = c row_p - s ph row_q, row q = s row_p + c ph row_q
            for (int e = threadIdx.x; e < npairs * n; e += kThreads) {
                const int k = e / n, j = e % n;
                const int2 pr = sm.pairs[k];
                if (pr.x < 0) continue;
                const float4 rt = sm.rot[k];
                const float c = rt.x, s = rt.y;
                const float2 ph = make_float2(rt.z, rt.w);
                const float2 x = A[pr.x * n + j], y = A[pr.y * n + j];
                float2 np = cadd(cscale(x, c), cmul(y, cscale(ph, -s)));
                float2 nq = cadd(cscale(x, s), cmul(y, cscale(ph, c)));
                if (j == pr.y) {
                    np = make_float2(0.f, 0.f);
                    nq.y = 0.f;
                }
                if (j == pr.x) {
                    np.y = 0.f;
                    nq = make_float2(0.f, 0.f);
                }
                A[pr.x * n + j] = np;
                A[pr.y * n + j] = nq;
            }
            __syncthreads();
        }
        const int any = sm.flags[0];
        __syncthreads();
        if (!any) {
            sweeps = sweep;
            break;
        }
    }
    for (int i = threadIdx.x; i < n; i += kThreads) w[i] = A[i * n + i].x;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += kThreads) {
        int rank = 0;
        const float wi = w[i];
        for (int j = 0; j < n; ++j) rank += (w[j] > wi) || (w[j] == wi && j < i);
        perm[rank] = i;
    }
    __syncthreads();
    return sweeps;
}

// ---------------------------------------------------------------- kernel ----
__global__ void __launch_bounds__(kThreads) small_kernel(const FrameDesc* __restrict__ descs, int mode, int pass) {
    extern __shared__ float4 smem_raw[];
    const FrameDesc d = descs[blockIdx.x];
    if (mode == kOrth && d.t < pass) return;
    const int M = d.M, l = d.l;
    Sm sm;
    smem_layout(l, &sm, reinterpret_cast<char*>(smem_raw));
    bool ok = true;

    if (mode == kOrth) {
        ok = cholqr2(d.C, d.V, d, M, l, sm);
        if (!ok && threadIdx.x == 0) set_status(d.status, FM_ERR_NO_CONVERGENCE);
        return;
    }

    // H = P^H C  (core matrix of Eq. 8 / Alg. 2 line 7)
    if (d.t >= 1) {
        gram_fp32(d.V, kMem, d.C, d, M, l, sm, sm.H);
    } else if (d.method == FM_RAND_SAMPLING) {
        for (int e = threadIdx.x; e < l * l; e += kThreads) {
            const int i = e / l, j = e % l;
            sm.H[e] = d.C[(int64_t)d.idx[i] * l + j];
        }
        __syncthreads();
    } else {
        gram_fp32(nullptr, kOmega, d.C, d, M, l, sm, sm.H);
    }
    // exact Hermitian part
    for (int e = threadIdx.x; e < l * l; e += kThreads) {
        const int i = e / l, j = e % l;
        if (i < j) {
            const float2 a = sm.H[i * l + j], b = sm.H[j * l + i];
            const float2 h = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
            sm.H[i * l + j] = h;
            sm.H[j * l + i] = cconj(h);
        } else if (i == j) {
            sm.H[e].y = 0.f;
        }
    }
    __syncthreads();

    // C = Q R_c ; Q -> V (V is no longer needed once H is formed)
    ok = cholqr2(d.C, d.V, d, M, l, sm) && ok;

    // W = pinv(H) via H = Z diag(w) Z^H
    const int s1 = jacobi_herm(sm.H, sm.Z, sm.w, sm.perm, l, sm);
    if (threadIdx.x == 0) {
        float amax = 0.f;
        for (int i = 0; i < l; ++i) amax = fmaxf(amax, fabsf(sm.w[i]));
        sm.dscal[0] = (double)((float)l * FLT_EPSILON * amax);
    }
    __syncthreads();
    const float thr = (float)sm.dscal[0];
    // Y = R_c Z
    for (int e = threadIdx.x; e < l * l; e += kThreads) {
        const int i = e / l, k = e % l;
        float2 s = make_float2(0.f, 0.f);
        for (int m = i; m < l; ++m) cfma(s, sm.Rc[i * l + m], sm.Z[m * l + k]);
        sm.Y[e] = s;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < l; k += kThreads) sm.w[k] = (fabsf(sm.w[k]) > thr) ? 1.f / sm.w[k] : 0.f;
    __syncthreads();
    // B = Y diag(w+) Y^H -> H
    for (int e = threadIdx.x; e < l * l; e += kThreads) {
        const int i = e / l, j = e % l;
        if (i > j) continue;
        float2 s = make_float2(0.f, 0.f);
        for (int k = 0; k < l; ++k) cfmaconj(s, cscale(sm.Y[i * l + k], sm.w[k]), sm.Y[j * l + k]);
        if (i == j) s.y = 0.f;
        sm.H[i * l + j] = s;
        sm.H[j * l + i] = cconj(s);
    }
    __syncthreads();
    // eig(B): U_B
    const int s2 = jacobi_herm(sm.H, sm.Z, sm.w, sm.perm, l, sm);
    // U_s = Q U_B[:, perm[0..ncols-1]]  (Tp in Ri: l x ncols)
    const int nc = d.ncols;
    for (int e = threadIdx.x; e < l * nc; e += kThreads) {
        const int k = e / nc, c = e % nc;
        sm.Ri[e] = sm.Z[k * l + sm.perm[c]];
    }
    __syncthreads();
    apply_rows(d.V, d.Us, d, M, l, sm.Ri, nc, nc, d.kpad, d.kpad, false, sm);
    if (threadIdx.x == 0 && (s1 < 0 || s2 < 0 || !ok)) set_status(d.status, FM_ERR_NO_CONVERGENCE);
}

}  // namespace

size_t small_smem_bytes(int l) { return smem_layout(l, nullptr, nullptr); }

static cudaError_t launch_small(const FrameDesc* d, int n_frames, int max_l, int mode, int pass, cudaStream_t s) {
    const size_t smem = small_smem_bytes(max_l);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    small_kernel<<<n_frames, kThreads, smem, s>>>(d, mode, pass);
    return cudaGetLastError();
}

cudaError_t launch_orth(const FrameDesc* d, int n_frames, int max_l, int pass, cudaStream_t s) {
    return launch_small(d, n_frames, max_l, kOrth, pass, s);
}

cudaError_t launch_final(const FrameDesc* d, int n_frames, int max_l, cudaStream_t s) {
    return launch_small(d, n_frames, max_l, kFinal, 0, s);
}

}  // namespace fm
