// small.cu -- per-frame l x l work of Algorithms 1 and 2 (Sec. III).
//
//   ORTH  (power step, Eq. 11):  V = orth(C)
//   FINAL (the core-matrix, rank-restriction and eigen steps of Alg. 1 / Alg. 2):
//         H = P^H C   with P = V (t >= 1; for projection with t = 0, V holds Pi)
//                     or H = C(I, :) = R(I, I) (sampling, t = 0)       (Eq. 8)
//         C = Q R_c                         (QR in place of SVD(C): Q = U_c Z, Z unitary)
//         B = R_c W R_c^H, W = H^+          (rank restriction)
//         eig(B) = U_B L_B U_B^H, U_s = Q U_B[:, :ncols] = C (R_c^{-1} U_B[:, :ncols])
//
// One thread-block cluster per frame: CTA r of the cluster keeps rows
// [r*Mr, (r+1)*Mr) of C (and V) in shared memory for the whole kernel, so
// every M-long operation is a row-local pass over shared memory; l x l Gram
// matrices are formed as per-CTA partials and summed over the cluster through
// distributed shared memory in rank order (deterministic), after which every
// CTA holds the same l x l matrix and runs the same l x l algorithms.
//
// Precision (no FP64 -- its rate on GB300 is a small fraction of FP32):
//   - QR: R_c from C^H C accumulated in double-float arithmetic (FP32 products split
//     exactly with an FMA, sums kept as hi + lo pairs), factored and inverted in
//     double-float, which survives cond(C) up to ~1/u_fp32.  ORTH applies R_c^{-1}
//     to the rows (double-float accumulation) to give the power-step basis V.
//     FINAL never forms Q: it keeps R_c^{-1} in double-float and forms U_s =
//     C (R_c^{-1} U_B) at the end with double-float sums, so U_s^H U_s = U_B^H U_B
//     up to double-float rounding and the one FP32 rounding of U_s (the
//     orthonormality a second CholeskyQR pass would give, without the two M-long
//     passes over the rows).
//   - W: H is Hermitian positive definite in exact arithmetic, so
//     B = R_c H^{-1} R_c^H = F F^H with F = R_c R_h^{-1}, H = R_h^H R_h (FP32
//     Cholesky).  If the Cholesky breaks down, W is the eigenvalue pseudo-inverse
//     of H (pivots with |lambda| <= l eps max|lambda| dropped).
//   - eig(B): one-sided Jacobi SVD of F in FP32 (two-sided complex Jacobi on B for
//     the pseudo-inverse branch), round-robin parallel ordering, followed by one
//     Rayleigh-Ritz correction of the leading eigenspace with double-float sums
//     (see refine_subspace) and a double-float re-orthonormalisation of the
//     selected eigenvectors.
#include <cooperative_groups.h>
#include <map>
#include <mutex>
#include <tuple>
#include <float.h>

#include "fm_internal.cuh"
#include "tc_common.cuh"

namespace cg = cooperative_groups;

namespace fm {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxRows = 128;   // rows of C / V held by one CTA
constexpr int kMaxSweeps = 30;
constexpr float kJacobiTol = 1e-6f;
// One-sided: the pair test |f_p^H f_q| <= tol |f_p| |f_q| is on inner products of
// the columns, so it needs a tighter tolerance than the two-sided |b_pq| test for
// the same eigenvector accuracy (1e-6 left projector errors of 1.2e-5 at M = 1024,
// l = 48; 1e-7 gives the two-sided 6e-6).
constexpr float kOneSidedTol = 1e-7f;

enum Mode { kOrth = 0, kFinal = 1 };

// ------------------------------------------------------------ double-float --
// Error-free transformations.  Every product and sum here uses the _rn
// intrinsics, which the compiler never contracts into an FMA: a contraction of
// p = a*b into the following add would change p's rounding and void the exact
// (hi, lo) splits.
struct df {
    float hi, lo;
};
__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return df{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ df quick_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return df{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df dd_add(df x, df y) {
    const df s = two_sum(x.hi, y.hi);
    return quick_two_sum(s.hi, __fadd_rn(__fadd_rn(s.lo, x.lo), y.lo));
}
__device__ __forceinline__ df dd_neg(df x) { return df{-x.hi, -x.lo}; }
__device__ __forceinline__ df dd_mul(df x, df y) {
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return quick_two_sum(p, e);
}
__device__ __forceinline__ df dd_div(df x, df y) {
    const float q1 = __fdiv_rn(x.hi, y.hi);
    const df r = dd_add(x, dd_neg(dd_mul(df{q1, 0.f}, y)));
    return quick_two_sum(q1, __fdiv_rn(r.hi, y.hi));
}
__device__ __forceinline__ df dd_sqrt(df x) {
    if (!(x.hi > 0.f)) return df{0.f, 0.f};
    const float s = __fsqrt_rn(x.hi);
    const float p = __fmul_rn(s, s);
    const float e = __fmaf_rn(s, s, -p);
    const float num = __fadd_rn(__fsub_rn(__fsub_rn(x.hi, p), e), x.lo);
    return quick_two_sum(s, __fdiv_rn(num, __fmul_rn(2.f, s)));
}
// s += a * b with the product split exactly (its error kept in lo)
__device__ __forceinline__ void dd_acc(df& s, float a, float b) {
    const float p = __fmul_rn(a, b);
    const float pe = __fmaf_rn(a, b, -p);
    const df t = two_sum(s.hi, p);
    s.hi = t.hi;
    s.lo = __fadd_rn(s.lo, __fadd_rn(t.lo, pe));
}
// complex double-float, stored as float4 (re.hi, re.lo, im.hi, im.lo)
struct zd {
    df re, im;
};
__device__ __forceinline__ zd zload(const float4& v) { return zd{df{v.x, v.y}, df{v.z, v.w}}; }
__device__ __forceinline__ float4 zpack(const zd& z) { return make_float4(z.re.hi, z.re.lo, z.im.hi, z.im.lo); }
__device__ __forceinline__ zd zadd(zd a, zd b) { return zd{dd_add(a.re, b.re), dd_add(a.im, b.im)}; }
// conj(a) * b
__device__ __forceinline__ zd zmulc(zd a, zd b) {
    return zd{dd_add(dd_mul(a.re, b.re), dd_mul(a.im, b.im)), dd_add(dd_mul(a.re, b.im), dd_neg(dd_mul(a.im, b.re)))};
}
__device__ __forceinline__ zd zmul(zd a, zd b) {
    return zd{dd_add(dd_mul(a.re, b.re), dd_neg(dd_mul(a.im, b.im))), dd_add(dd_mul(a.re, b.im), dd_mul(a.im, b.re))};
}
__device__ __forceinline__ zd zscale(zd a, df s) { return zd{dd_mul(a.re, s), dd_mul(a.im, s)}; }
__device__ __forceinline__ zd zneg(zd a) { return zd{dd_neg(a.re), dd_neg(a.im)}; }

// ------------------------------------------------------------------ layout --
struct Sm {
    float2* Cs;    // Mr x l   rows of C (ORTH: Q after the QR)
    float2* Vs;    // Mr x l   rows of V (FINAL, until H is formed)
    float4* Gd;    // l x l    double-float Gram / Cholesky factor   (aliases Vs)
    float4* Xd;    // l x l    double-float inverse                  (aliases Vs)
    float2* Xf;    // l x l    FP32 scratch of the one-sided Jacobi  (aliases Gd)
    float4* part;  // l x l    per-CTA partial Gram (float4 or float2 view)
    float2* T;     // l x l    temp                                  (aliases part)
    float2* Rc;    // l x l    R factor of C = Q R_c
    float2* H;     // l x l    core matrix, then B
    float2* Z;     // l x l    eigenvectors
    float* w;      // l
    int* perm;     // l
    float4* rot;   // l/2+1
    int2* pairs;   // l/2+1
    int* act;      // l/2+1
    int* items;    // phase-B item table
    int* flags;    // kMaxSweeps + 8
    float* scal;   // 8
    float4* dscal; // 4
};

__host__ __device__ inline size_t a16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline size_t smem_layout(int Mr, int l, Sm* sm, char* base) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = a16(off + bytes);
        return base ? base + o : nullptr;
    };
    const size_t ll = (size_t)l * l, rows = (size_t)Mr * l;
    const int np = (l + 1) / 2 + 1;
    char* Cs = take(rows * sizeof(float2));
    const size_t u1 = rows * sizeof(float2) > 2 * ll * sizeof(float4) ? rows * sizeof(float2) : 2 * ll * sizeof(float4);
    char* U1 = take(u1);
    char* part = take(ll * sizeof(float4));
    char* Rc = take(ll * sizeof(float2));
    char* H = take(ll * sizeof(float2));
    char* Z = take(ll * sizeof(float2));
    char* w = take(l * sizeof(float));
    char* perm = take(l * sizeof(int));
    char* rot = take(np * sizeof(float4));
    char* pairs = take(np * sizeof(int2));
    char* act = take(np * sizeof(int));
    char* items = take((size_t)(np * (np + 1) / 2 + np * l) * sizeof(int));
    char* flags = take((kMaxSweeps + 8) * sizeof(int));
    char* scal = take(8 * sizeof(float));
    char* dscal = take(4 * sizeof(float4));
    if (sm) {
        sm->Cs = reinterpret_cast<float2*>(Cs);
        sm->Vs = reinterpret_cast<float2*>(U1);
        sm->Gd = reinterpret_cast<float4*>(U1);
        sm->Xd = reinterpret_cast<float4*>(U1) + ll;
        sm->Xf = reinterpret_cast<float2*>(U1) + ll;
        sm->part = reinterpret_cast<float4*>(part);
        sm->T = reinterpret_cast<float2*>(part);
        sm->Rc = reinterpret_cast<float2*>(Rc);
        sm->H = reinterpret_cast<float2*>(H);
        sm->Z = reinterpret_cast<float2*>(Z);
        sm->w = reinterpret_cast<float*>(w);
        sm->perm = reinterpret_cast<int*>(perm);
        sm->rot = reinterpret_cast<float4*>(rot);
        sm->pairs = reinterpret_cast<int2*>(pairs);
        sm->act = reinterpret_cast<int*>(act);
        sm->items = reinterpret_cast<int*>(items);
        sm->flags = reinterpret_cast<int*>(flags);
        sm->scal = reinterpret_cast<float*>(scal);
        sm->dscal = reinterpret_cast<float4*>(dscal);
    }
    return off;
}

// --------------------------------------------------------------- helpers ---
__device__ __forceinline__ void tri_coords(int e, int n, int& i, int& j) {
    i = 0;
    while (e >= n - i) {
        e -= n - i;
        ++i;
    }
    j = i + e;
}

__device__ void load_rows(const float2* __restrict__ src, float2* dst, int r0, int rows, int l) {
    const float2* s = src + (int64_t)r0 * l;
    const int n = rows * l;
    if (((reinterpret_cast<uintptr_t>(s) & 15) == 0) && (n % 2 == 0)) {
        const float4* s4 = reinterpret_cast<const float4*>(s);
        float4* d4 = reinterpret_cast<float4*>(dst);
        for (int e = threadIdx.x; e < n / 2; e += kThreads) d4[e] = s4[e];
    } else {
        for (int e = threadIdx.x; e < n; e += kThreads) dst[e] = s[e];
    }
}

__device__ void store_rows(const float2* src, float2* __restrict__ dst, int r0, int rows, int l) {
    for (int e = threadIdx.x; e < rows * l; e += kThreads) dst[(int64_t)r0 * l + e] = src[e];
}

// part <- A^H B over this CTA's rows, FP32 (float2 view of part).  herm: B == A,
// upper triangle only (the reduction mirrors it).
__device__ void gram_part_f(const float2* A, const float2* B, int rows, int l, bool herm, float2* part) {
    const int n = herm ? l * (l + 1) / 2 : l * l;
    for (int e = threadIdx.x; e < n; e += kThreads) {
        int i, j;
        if (herm) {
            tri_coords(e, l, i, j);
        } else {
            i = e / l;
            j = e - i * l;
        }
        float2 acc = make_float2(0.f, 0.f), t = make_float2(0.f, 0.f);
        for (int r = 0; r < rows; ++r) {
            cfmac(t, A[r * l + i], B[r * l + j]);
            if ((r & 15) == 15) {
                acc = cadd(acc, t);
                t = make_float2(0.f, 0.f);
            }
        }
        part[e] = cadd(acc, t);
    }
}

// part <- A^H A over this CTA's rows in double-float (upper triangle, float4 entries).
// Each entry is shared by a lane pair (rows of one parity each, four interleaved
// partial sums per lane) and combined across the pair in a fixed order, so the
// l(l+1)/2 entries spread evenly over the block.
__device__ void gram_part_d(const float2* A, int rows, int l, float4* part) {
    const int n = l * (l + 1) / 2;
    const int ntask = 2 * n;
    const int rounds = (ntask + kThreads - 1) / kThreads;  // block-uniform: every lane reaches every shuffle
    for (int u = 0; u < rounds; ++u) {
        const int task = threadIdx.x + u * kThreads;
        const bool act = task < ntask;
        const int e = act ? task >> 1 : 0, h = task & 1;
        int i, j;
        tri_coords(e, l, i, j);
        df re[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        df im[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        if (act) {
            int r = h;
            for (; r + 6 < rows; r += 8) {  // rows r, r + 2, r + 4, r + 6 of this lane's parity
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const float2 a = A[(r + 2 * v) * l + i], b = A[(r + 2 * v) * l + j];
                    dd_acc(re[v], a.x, b.x);
                    dd_acc(re[v], a.y, b.y);
                    dd_acc(im[v], a.x, b.y);
                    dd_acc(im[v], -a.y, b.x);
                }
            }
            for (; r < rows; r += 2) {
                const float2 a = A[r * l + i], b = A[r * l + j];
                dd_acc(re[0], a.x, b.x);
                dd_acc(re[0], a.y, b.y);
                dd_acc(im[0], a.x, b.y);
                dd_acc(im[0], -a.y, b.x);
            }
        }
        df sr = dd_add(dd_add(re[0], re[1]), dd_add(re[2], re[3]));
        df si = dd_add(dd_add(im[0], im[1]), dd_add(im[2], im[3]));
        // the even-row lane adds its odd-row partner's sums
        const df pr{__shfl_xor_sync(0xffffffffu, sr.hi, 1), __shfl_xor_sync(0xffffffffu, sr.lo, 1)};
        const df pi{__shfl_xor_sync(0xffffffffu, si.hi, 1), __shfl_xor_sync(0xffffffffu, si.lo, 1)};
        if (act && h == 0) {
            sr = dd_add(sr, pr);
            si = dd_add(si, pi);
            part[e] = zpack(zd{quick_two_sum(sr.hi, sr.lo), quick_two_sum(si.hi, si.lo)});
        }
    }
}

// Sum the cluster's double-float partials (upper triangle, rank order) into the
// Hermitian out (l x l).
__device__ void reduce_d(cg::cluster_group& cl, float4* part, float4* out, int l) {
    const int n = l * (l + 1) / 2;
    const unsigned nc = cl.num_blocks();
    cl.sync();
    for (int e = threadIdx.x; e < n; e += kThreads) {
        zd s = zload(cl.map_shared_rank(part, 0u)[e]);
        for (unsigned r = 1; r < nc; ++r) s = zadd(s, zload(cl.map_shared_rank(part, r)[e]));
        int i, j;
        tri_coords(e, l, i, j);
        if (i == j) s.im = df{0.f, 0.f};
        out[i * l + j] = zpack(s);
        if (i != j) out[j * l + i] = zpack(zd{s.re, dd_neg(s.im)});
    }
    cl.sync();
}

// The sums of full l x l FP32 partials (pf -> of) and of double-float upper-triangle
// partials (pd -> od, as reduce_d) over the cluster in rank order, in one pass between
// one pair of cluster barriers.
__device__ void reduce_fd(cg::cluster_group& cl, float2* pf, float2* of, float4* pd, float4* od, int l) {
    const int nf = l * l, nd = l * (l + 1) / 2;
    const unsigned nc = cl.num_blocks();
    cl.sync();
    for (int e = threadIdx.x; e < nf + nd; e += kThreads) {
        if (e < nf) {
            float2 s = make_float2(0.f, 0.f);
            for (unsigned r = 0; r < nc; ++r) s = cadd(s, cl.map_shared_rank(pf, r)[e]);
            of[e] = s;
        } else {
            const int u = e - nf;
            zd s = zload(cl.map_shared_rank(pd, 0u)[u]);
            for (unsigned r = 1; r < nc; ++r) s = zadd(s, zload(cl.map_shared_rank(pd, r)[u]));
            int i, j;
            tri_coords(u, l, i, j);
            if (i == j) s.im = df{0.f, 0.f};
            od[i * l + j] = zpack(s);
            if (i != j) od[j * l + i] = zpack(zd{s.re, dd_neg(s.im)});
        }
    }
    cl.sync();
}

// ------------------------------------------------------ Cholesky / inverse --
// Pivots below 2^-40 x the largest diagonal entry (a numerically rank-deficient
// sketch) are raised to that floor; only a non-finite pivot fails.
__device__ bool chol_d(float4* G, int l, const Sm& sm) {
    if (threadIdx.x == 0) {
        sm.flags[kMaxSweeps + 4] = 0;
        float dmax = 0.f;
        for (int k = 0; k < l; ++k) dmax = fmaxf(dmax, G[k * l + k].x);
        sm.scal[2] = 0x1p-40f * dmax;
    }
    __syncthreads();
    const float dfloor = sm.scal[2];
    for (int k = 0; k < l; ++k) {
        if (threadIdx.x == 0) {
            df d = zload(G[k * l + k]).re;
            if (!isfinite(d.hi)) {
                sm.flags[kMaxSweeps + 4] = 1;
                d = df{1e-30f, 0.f};
            } else if (!(d.hi > dfloor)) {
                d = df{dfloor > 0.f ? dfloor : 1e-30f, 0.f};
            }
            const df r = dd_sqrt(d);
            G[k * l + k] = make_float4(r.hi, r.lo, 0.f, 0.f);
            const df inv = dd_div(df{1.f, 0.f}, r);
            sm.dscal[0] = make_float4(inv.hi, inv.lo, 0.f, 0.f);
        }
        __syncthreads();
        const df inv = df{sm.dscal[0].x, sm.dscal[0].y};
        for (int j = k + 1 + threadIdx.x; j < l; j += kThreads) G[k * l + j] = zpack(zscale(zload(G[k * l + j]), inv));
        __syncthreads();
        const int n = l - k - 1;
        for (int e = threadIdx.x; e < n * n; e += kThreads) {
            const int i = k + 1 + e / n, j = k + 1 + e % n;
            if (i <= j)
                G[i * l + j] = zpack(zadd(zload(G[i * l + j]), zneg(zmulc(zload(G[k * l + i]), zload(G[k * l + j])))));
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < l * l; e += kThreads)
        if (e / l > e % l) G[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    return sm.flags[kMaxSweeps + 4] == 0;
}

// X = R^{-1}, R upper with real positive diagonal; right-looking back
// substitution (row i finalised as (delta_ij - S_ij)/R_ii, then R_ki X_ij added to
// the partial sums S_kj of all rows k < i in parallel).
__device__ void trinv_d(const float4* R, float4* X, int l, const Sm& sm) {
    for (int e = threadIdx.x; e < l * l; e += kThreads) X[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    for (int i = l - 1; i >= 0; --i) {
        if (threadIdx.x == 0) {
            const df inv = dd_div(df{1.f, 0.f}, zload(R[i * l + i]).re);
            sm.dscal[1] = make_float4(inv.hi, inv.lo, 0.f, 0.f);
        }
        __syncthreads();
        const df inv = df{sm.dscal[1].x, sm.dscal[1].y};
        for (int j = i + threadIdx.x; j < l; j += kThreads) {
            zd s = zneg(zload(X[i * l + j]));
            if (j == i) s.re = dd_add(s.re, df{1.f, 0.f});
            X[i * l + j] = zpack(zscale(s, inv));
        }
        __syncthreads();
        const int w = l - i;
        for (int e = threadIdx.x; e < i * w; e += kThreads) {
            const int k = e / w, j = i + e % w;
            X[k * l + j] = zpack(zadd(zload(X[k * l + j]), zmul(zload(R[k * l + i]), zload(X[i * l + j]))));
        }
        __syncthreads();
    }
}

// Cholesky factor and its inverse in one elimination sweep.  Reducing G to R by
// row operations (row k scaled by 1/r_kk, then row i > k minus conj(r_ki) times
// row k) and applying the same operations to the identity beside it leaves that
// identity as E with E G = R, i.e. E = R^{-H} (lower triangular); X = R^{-1} = E^H.
// One block barrier per column: every thread derives the pivot's square root and
// its inverse itself (same inputs, same results), rows i > k are updated from row
// k scaled on the fly, and the finished row k is written where nothing reads it in
// the same phase (R's row parked below G's diagonal, E's row conjugated into
// column k of X), so the next column only waits for the updates.  Aw (l x l) is
// scratch for E.  Task slots of the trailing triangle: rows a and n - 1 - a share
// n + 1 slots, so the triangle packs densely into the block.
__device__ __forceinline__ bool trailing_slot(int t, int n, int& a, int& b) {
    const int p = t / (n + 1), c = t - p * (n + 1);
    if (c < n - p) {
        a = p;
        b = p + c;
        return true;
    }
    a = n - 1 - p;
    b = a + (c - (n - p));
    return a != p;  // odd n: the middle row is listed once
}

// Double-float: pivots below 2^-40 x the largest diagonal entry (a numerically
// rank-deficient sketch) are raised to that floor; only a non-finite pivot fails.
// G (in place) becomes R (upper, zero below), X = R^{-1}.
__device__ bool chol_inv_d(float4* G, float4* X, float4* Aw, int l, const Sm& sm) {
    if (threadIdx.x == 0) {
        sm.flags[kMaxSweeps + 4] = 0;
        float dmax = 0.f;
        for (int k = 0; k < l; ++k) dmax = fmaxf(dmax, G[k * l + k].x);
        sm.scal[2] = 0x1p-40f * dmax;
    }
    for (int e = threadIdx.x; e < l * l; e += kThreads) {
        Aw[e] = make_float4((e / l == e % l) ? 1.f : 0.f, 0.f, 0.f, 0.f);
        X[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    const float dfloor = sm.scal[2];
    df rprev{0.f, 0.f};
    for (int k = 0; k < l; ++k) {
        // the previous pivot's R entry: every thread has read G[k-1][k-1] by now
        if (k > 0 && threadIdx.x == 0) G[(k - 1) * l + k - 1] = make_float4(rprev.hi, rprev.lo, 0.f, 0.f);
        df d = zload(G[k * l + k]).re;
        const bool bad = !isfinite(d.hi);
        if (bad) {
            d = df{1e-30f, 0.f};
        } else if (!(d.hi > dfloor)) {
            d = df{dfloor > 0.f ? dfloor : 1e-30f, 0.f};
        }
        const df r = dd_sqrt(d);
        const df inv = dd_div(df{1.f, 0.f}, r);
        if (bad && threadIdx.x == 0) sm.flags[kMaxSweeps + 4] = 1;
        rprev = r;
        const int n = l - k - 1;
        const int nt = ((n + 1) / 2) * (n + 1);  // trailing upper-triangle slots
        const int na = n * (k + 1);              // E entries of the rows below
        const int ntot = nt + na + n + k + 1;    // + R row k (right of the pivot) + E row k
        for (int t = threadIdx.x; t < ntot; t += kThreads) {
            if (t < nt) {
                int a, b;
                if (!trailing_slot(t, n, a, b)) continue;
                const int i = k + 1 + a, j = k + 1 + b;
                const zd ri = zscale(zload(G[k * l + i]), inv), rj = zscale(zload(G[k * l + j]), inv);
                G[i * l + j] = zpack(zadd(zload(G[i * l + j]), zneg(zmulc(ri, rj))));
            } else if (t < nt + na) {
                const int u = t - nt, a = u / (k + 1), m = u - a * (k + 1);
                const int i = k + 1 + a;
                const zd ri = zscale(zload(G[k * l + i]), inv), em = zscale(zload(Aw[k * l + m]), inv);
                Aw[i * l + m] = zpack(zadd(zload(Aw[i * l + m]), zneg(zmulc(ri, em))));
            } else if (t < nt + na + n) {
                const int j = k + 1 + (t - nt - na);
                G[j * l + k] = zpack(zscale(zload(G[k * l + j]), inv));  // R[k][j], parked
            } else {
                const int m = t - nt - na - n;
                const zd em = zscale(zload(Aw[k * l + m]), inv);
                X[m * l + k] = zpack(zd{em.re, dd_neg(em.im)});
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) G[(l - 1) * l + l - 1] = make_float4(rprev.hi, rprev.lo, 0.f, 0.f);
    // R's rows back above the diagonal, zeros below
    for (int e = threadIdx.x; e < l * l; e += kThreads) {
        const int i = e / l, j = e % l;
        if (i < j) {
            G[e] = G[j * l + i];
            G[j * l + i] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    __syncthreads();
    return sm.flags[kMaxSweeps + 4] == 0;
}

// The double-float sweep of chol_inv_d on the Gram of C and the same sweep in FP32 on
// the core matrix H, side by side: the two chains are independent until
// F = R_c R_h^{-1}, so each column phase takes the tasks of both behind one barrier --
// double-float tasks from the low thread indices, FP32 tasks from the high ones, so
// that a thread takes both only while the double-float phase still fills the block --
// and the FP32 sweep adds no barriers of its own.  Gd becomes R_c and Xd = R_c^{-1}
// (false on a non-finite pivot, pivots floored as in chol_inv_d); Gf becomes R_h and
// the upper triangle of XEf R_h^{-1}, where any non-positive pivot sets *pd false (W
// then falls back to the eigenvalue pseudo-inverse of H).  The FP32 E shares XEf with
// the inverse: E is unit lower triangular (its diagonal is never stored) and its row k
// is read in the phase that writes column k of the inverse above the diagonal.
__device__ bool chol_inv_pair(float4* Gd, float4* Xd, float4* Awd, float2* Gf, float2* XEf, int l, const Sm& sm,
                              bool* pd) {
    if (threadIdx.x == 0) {
        sm.flags[kMaxSweeps + 4] = 0;
        sm.flags[kMaxSweeps + 5] = 0;
        float dmax = 0.f;
        for (int k = 0; k < l; ++k) dmax = fmaxf(dmax, Gd[k * l + k].x);
        sm.scal[2] = 0x1p-40f * dmax;
    }
    for (int e = threadIdx.x; e < l * l; e += kThreads) {
        const float one = (e / l == e % l) ? 1.f : 0.f;
        Awd[e] = make_float4(one, 0.f, 0.f, 0.f);
        Xd[e] = make_float4(0.f, 0.f, 0.f, 0.f);
        XEf[e] = make_float2(0.f, 0.f);
    }
    __syncthreads();
    const float dfloor = sm.scal[2];
    df rprev{0.f, 0.f};
    float rprevf = 0.f;
    for (int k = 0; k < l; ++k) {
        // the previous pivots' R entries: every thread has read them by now
        if (k > 0 && threadIdx.x == 0) Gd[(k - 1) * l + k - 1] = make_float4(rprev.hi, rprev.lo, 0.f, 0.f);
        if (k > 0 && threadIdx.x == kThreads - 1) Gf[(k - 1) * l + k - 1] = make_float2(rprevf, 0.f);
        df d = zload(Gd[k * l + k]).re;
        const bool bad = !isfinite(d.hi);
        if (bad) {
            d = df{1e-30f, 0.f};
        } else if (!(d.hi > dfloor)) {
            d = df{dfloor > 0.f ? dfloor : 1e-30f, 0.f};
        }
        const df r = dd_sqrt(d);
        const df inv = dd_div(df{1.f, 0.f}, r);
        if (bad && threadIdx.x == 0) sm.flags[kMaxSweeps + 4] = 1;
        rprev = r;
        float dff = Gf[k * l + k].x;
        const bool badf = !isfinite(dff) || !(dff > 0.f);
        if (badf) dff = 1e-30f;
        const float rf = sqrtf(dff);
        const float invf = 1.f / rf;
        if (badf && threadIdx.x == kThreads - 1) sm.flags[kMaxSweeps + 5] = 1;
        rprevf = rf;
        const int n = l - k - 1;
        const int nt = ((n + 1) / 2) * (n + 1);  // trailing upper-triangle slots
        const int na = n * (k + 1);              // E entries of the rows below
        const int ntot = nt + na + n + k + 1;    // + R row k (right of the pivot) + E row k
        for (int t = threadIdx.x; t < ntot; t += kThreads) {
            if (t < nt) {
                int a, b;
                if (!trailing_slot(t, n, a, b)) continue;
                const int i = k + 1 + a, j = k + 1 + b;
                const zd ri = zscale(zload(Gd[k * l + i]), inv), rj = zscale(zload(Gd[k * l + j]), inv);
                Gd[i * l + j] = zpack(zadd(zload(Gd[i * l + j]), zneg(zmulc(ri, rj))));
            } else if (t < nt + na) {
                const int u = t - nt, a = u / (k + 1), m = u - a * (k + 1);
                const int i = k + 1 + a;
                const zd ri = zscale(zload(Gd[k * l + i]), inv), em = zscale(zload(Awd[k * l + m]), inv);
                Awd[i * l + m] = zpack(zadd(zload(Awd[i * l + m]), zneg(zmulc(ri, em))));
            } else if (t < nt + na + n) {
                const int j = k + 1 + (t - nt - na);
                Gd[j * l + k] = zpack(zscale(zload(Gd[k * l + j]), inv));  // R[k][j], parked
            } else {
                const int m = t - nt - na - n;
                const zd em = zscale(zload(Awd[k * l + m]), inv);
                Xd[m * l + k] = zpack(zd{em.re, dd_neg(em.im)});
            }
        }
        for (int t = kThreads - 1 - threadIdx.x; t < ntot; t += kThreads) {
            if (t < nt) {
                int a, b;
                if (!trailing_slot(t, n, a, b)) continue;
                const int i = k + 1 + a, j = k + 1 + b;
                Gf[i * l + j] = csub(Gf[i * l + j], cmulc(cscale(Gf[k * l + i], invf), cscale(Gf[k * l + j], invf)));
            } else if (t < nt + na) {
                const int u = t - nt, a = u / (k + 1), m = u - a * (k + 1);
                const int i = k + 1 + a;
                const float2 ekm = (m == k) ? make_float2(1.f, 0.f) : XEf[k * l + m];
                XEf[i * l + m] = csub(XEf[i * l + m], cmulc(cscale(Gf[k * l + i], invf), cscale(ekm, invf)));
            } else if (t < nt + na + n) {
                const int j = k + 1 + (t - nt - na);
                Gf[j * l + k] = cscale(Gf[k * l + j], invf);
            } else {
                const int m = t - nt - na - n;
                const float2 ekm = (m == k) ? make_float2(1.f, 0.f) : XEf[k * l + m];
                XEf[m * l + k] = cconj(cscale(ekm, invf));
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) Gd[(l - 1) * l + l - 1] = make_float4(rprev.hi, rprev.lo, 0.f, 0.f);
    if (threadIdx.x == kThreads - 1) Gf[(l - 1) * l + l - 1] = make_float2(rprevf, 0.f);
    // R's rows back above the diagonal, zeros below
    for (int e = threadIdx.x; e < l * l; e += kThreads) {
        const int i = e / l, j = e % l;
        if (i < j) {
            Gd[e] = Gd[j * l + i];
            Gd[j * l + i] = make_float4(0.f, 0.f, 0.f, 0.f);
            Gf[e] = Gf[j * l + i];
            Gf[j * l + i] = make_float2(0.f, 0.f);
        }
    }
    __syncthreads();
    *pd = sm.flags[kMaxSweeps + 5] == 0;
    return sm.flags[kMaxSweeps + 4] == 0;
}

// In place, row-local: rows of A (rows x l) <- A * X for X upper triangular given
// in double-float (hi, lo) pairs.  Output (r, c) sums k = 0 .. c, so a task pairs
// column c with column l - 1 - c of the same row (l + 1 terms per task whatever c)
// to balance the threads; every result is held in registers until the whole block
// has read A, then written in place.
__device__ void apply_upper_d(float2* A, int rows, int l, const float4* X) {
    constexpr int kMaxTasks = (kMaxRows * ((kLMax + 1) / 2) + kThreads - 1) / kThreads;  // 12 at l = 48
    const int half = (l + 1) / 2;       // column pairs per row (the middle column alone if l is odd)
    const int ntask = rows * half;
    float2 out[kMaxTasks][2];
#pragma unroll
    for (int u = 0; u < kMaxTasks; ++u) {
        const int task = threadIdx.x + u * kThreads;
        out[u][0] = out[u][1] = make_float2(0.f, 0.f);
        if (task >= ntask) continue;
        const int r = task / half, cp = task - r * half;
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const int c = side ? l - 1 - cp : cp;
            if (side && c == cp) continue;  // odd l: the middle column once
            df re{0.f, 0.f}, im{0.f, 0.f};
            for (int k = 0; k <= c; ++k) {
                const float2 a = A[r * l + k];
                const float4 x = X[k * l + c];  // (re.hi, re.lo, im.hi, im.lo)
                dd_acc(re, a.x, x.x);
                dd_acc(re, -a.y, x.z);
                dd_acc(im, a.x, x.z);
                dd_acc(im, a.y, x.x);
                re.lo = fmaf(a.x, x.y, fmaf(-a.y, x.w, re.lo));
                im.lo = fmaf(a.x, x.w, fmaf(a.y, x.y, im.lo));
            }
            out[u][side] = make_float2(re.hi + re.lo, im.hi + im.lo);
        }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kMaxTasks; ++u) {
        const int task = threadIdx.x + u * kThreads;
        if (task >= ntask) continue;
        const int r = task / half, cp = task - r * half;
        A[r * l + cp] = out[u][0];
        if (l - 1 - cp != cp) A[r * l + l - 1 - cp] = out[u][1];
    }
    __syncthreads();
}

// One double-float CholeskyQR pass on the cluster-distributed rows A (in place):
// G = A^H A (double-float sums), G = R^H R (double-float Cholesky),
// A <- A R^{-1} (double-float accumulation).  Rk receives R rounded to FP32.
__device__ bool cholqr_pass_d(cg::cluster_group& cl, float2* A, int rows, int l, const Sm& sm, float2* Rk) {
    gram_part_d(A, rows, l, sm.part);
    reduce_d(cl, sm.part, sm.Gd, l);
    const bool ok = chol_inv_d(sm.Gd, sm.Xd, sm.part, l, sm);  // part is free after the reduction
    for (int e = threadIdx.x; e < l * l; e += kThreads) {
        const float4 g = sm.Gd[e];
        Rk[e] = make_float2(g.x + g.y, g.z + g.w);
    }
    apply_upper_d(A, rows, l, sm.Xd);
    return ok;
}

// perm <- indices of w ordered by value descending, ties by index.  NaN sorts as
// -inf, so perm is a permutation of 0..n-1 whatever w holds (its entries index
// shared-memory arrays).
__device__ void sort_desc(const float* w, int* perm, int n) {
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += kThreads) {
        int rank = 0;
        const float wi = isnan(w[i]) ? -INFINITY : w[i];
        for (int j = 0; j < n; ++j) {
            const float wj = isnan(w[j]) ? -INFINITY : w[j];
            rank += (wj > wi) || (wj == wi && j < i);
        }
        perm[rank] = i;
    }
    __syncthreads();
}

// ---------------------------------------------------------------- Jacobi ----
// Hermitian eigendecomposition of A (n x n, destroyed: its diagonal ends as the
// eigenvalues), eigenvectors in the columns of Z, w the eigenvalues, perm the
// column order by eigenvalue descending (ties: lower index).  One round = one
// set of disjoint rotations: phase A computes them, phase B applies U^H A U as
// independent 2x2 blocks (k, k') and rotates the columns of Z.  Returns the
// number of sweeps or -1 if `cap` sweeps did not converge.
__device__ int jacobi(float2* A, float2* Z, float* w, int* perm, int n, const Sm& sm, int cap) {
    const int ne = n + (n & 1), np = ne / 2, nr = ne - 1;
    const int nblk = np * (np + 1) / 2, nitems = nblk + np * n;
    for (int e = threadIdx.x; e < n * n; e += kThreads)
        Z[e] = (e / n == e % n) ? make_float2(1.f, 0.f) : make_float2(0.f, 0.f);
    for (int e = threadIdx.x; e < nitems; e += kThreads) {
        int a, b;
        if (e < nblk) {
            tri_coords(e, np, a, b);
        } else {
            a = (e - nblk) / n;
            b = (e - nblk) % n;
        }
        sm.items[e] = (a << 16) | b;
    }
    for (int e = threadIdx.x; e < kMaxSweeps; e += kThreads) sm.flags[e] = 0;
    __syncthreads();
    int sweeps = -1;
    for (int sweep = 0; sweep < cap && nr > 0; ++sweep) {
        for (int r = 0; r < nr; ++r) {
            if (threadIdx.x < np) {
                const int k = threadIdx.x;
                const int pa = (k == 0) ? 0 : 1 + (k - 1 + r) % nr;
                const int pb = 1 + (ne - 2 - k + r) % nr;
                const int p = min(pa, pb), q = max(pa, pb);
                float4 rt = make_float4(1.f, 0.f, 1.f, 0.f);
                int on = 0;
                if (q < n) {
                    const float2 apq = A[p * n + q];
                    const float mag = sqrtf(cabs2(apq));
                    const float app = A[p * n + p].x, aqq = A[q * n + q].x;
                    if (mag > 1e-30f && mag > kJacobiTol * sqrtf(fabsf(app * aqq))) {
                        const float tau = (aqq - app) / (2.f * mag);
                        const float t = (fabsf(tau) > 1e18f)
                                            ? 0.5f / tau
                                            : (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(fmaf(tau, tau, 1.f)));
                        const float c = rsqrtf(fmaf(t, t, 1.f));
                        rt = make_float4(c, t * c, apq.x / mag, apq.y / mag);
                        on = 1;
                        sm.flags[sweep] = 1;
                    }
                }
                sm.pairs[k] = make_int2(p, q < n ? q : -1);
                sm.rot[k] = rt;
                sm.act[k] = on;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < nitems; e += kThreads) {
                const int it = sm.items[e];
                const int a = it >> 16, b = it & 0xffff;
                if (e < nblk) {
                    // block (a, b), a <= b: rows (p_a, q_a), cols (p_b, q_b)
                    if (!sm.act[a] && !sm.act[b]) continue;
                    const int2 ra = sm.pairs[a], rb = sm.pairs[b];
                    const float4 ua = sm.rot[a], ub = sm.rot[b];
                    const bool qa = ra.y >= 0, qb = rb.y >= 0;
                    float2 x00 = A[ra.x * n + rb.x];
                    float2 x01 = qb ? A[ra.x * n + rb.y] : make_float2(0.f, 0.f);
                    float2 x10 = qa ? A[ra.y * n + rb.x] : make_float2(0.f, 0.f);
                    float2 x11 = (qa && qb) ? A[ra.y * n + rb.y] : make_float2(0.f, 0.f);
                    {  // X <- X U_b, U = [[c, s], [-s conj(ph), c conj(ph)]]
                        const float c = ub.x, s = ub.y;
                        const float2 phc = make_float2(ub.z, -ub.w);
                        const float2 u10 = cscale(phc, -s), u11 = cscale(phc, c);
                        const float2 y00 = cadd(cscale(x00, c), cmul(x01, u10));
                        const float2 y01 = cadd(cscale(x00, s), cmul(x01, u11));
                        const float2 y10 = cadd(cscale(x10, c), cmul(x11, u10));
                        const float2 y11 = cadd(cscale(x10, s), cmul(x11, u11));
                        x00 = y00;
                        x01 = y01;
                        x10 = y10;
                        x11 = y11;
                    }
                    {  // X <- U_a^H X: row p = c row_p - s ph row_q, row q = s row_p + c ph row_q
                        const float c = ua.x, s = ua.y;
                        const float2 ph = make_float2(ua.z, ua.w);
                        const float2 m01 = cscale(ph, -s), m11 = cscale(ph, c);
                        const float2 y00 = cadd(cscale(x00, c), cmul(m01, x10));
                        const float2 y01 = cadd(cscale(x01, c), cmul(m01, x11));
                        const float2 y10 = cadd(cscale(x00, s), cmul(m11, x10));
                        const float2 y11 = cadd(cscale(x01, s), cmul(m11, x11));
                        x00 = y00;
                        x01 = y01;
                        x10 = y10;
                        x11 = y11;
                    }
                    if (a == b) {
                        x00.y = 0.f;
                        x11.y = 0.f;
                        if (sm.act[a]) x01 = x10 = make_float2(0.f, 0.f);
                    }
                    A[ra.x * n + rb.x] = x00;
                    if (qb) A[ra.x * n + rb.y] = x01;
                    if (qa) A[ra.y * n + rb.x] = x10;
                    if (qa && qb) A[ra.y * n + rb.y] = x11;
                    if (a != b) {
                        A[rb.x * n + ra.x] = cconj(x00);
                        if (qb) A[rb.y * n + ra.x] = cconj(x01);
                        if (qa) A[rb.x * n + ra.y] = cconj(x10);
                        if (qa && qb) A[rb.y * n + ra.y] = cconj(x11);
                    }
                } else {
                    // Z <- Z U_a on row b
                    if (!sm.act[a]) continue;
                    const int2 ra = sm.pairs[a];
                    const float4 ua = sm.rot[a];
                    const float c = ua.x, s = ua.y;
                    const float2 phc = make_float2(ua.z, -ua.w);
                    const float2 x = Z[b * n + ra.x], y = Z[b * n + ra.y];
                    Z[b * n + ra.x] = cadd(cscale(x, c), cmul(y, cscale(phc, -s)));
                    Z[b * n + ra.y] = cadd(cscale(x, s), cmul(y, cscale(phc, c)));
                }
            }
            __syncthreads();
        }
        if (!sm.flags[sweep]) {
            sweeps = sweep;
            break;
        }
    }
    if (nr == 0) sweeps = 0;
    for (int i = threadIdx.x; i < n; i += kThreads) w[i] = A[i * n + i].x;
    __syncthreads();
    sort_desc(w, perm, n);
    return sweeps;
}

// Eigen-decomposition of B = F F^H through the singular value decomposition of
// F (n x n, row-major in Frm) by one-sided (Hestenes) Jacobi in FP32: column
// pairs (p, q) of F are rotated until every pair is orthogonal to the relative
// tolerance, F <- F J with J the 2 x 2 unitary that diagonalises the pair's Gram
// matrix [[a, g], [g*, b]] (a = |f_p|^2, b = |f_q|^2, g = f_p^H f_q).  The columns
// of the converged F are then sigma_k u_k with B u_k = sigma_k^2 u_k.  Pairs follow
// the same round-robin order as the two-sided solver.  Within a round the pairs
// touch disjoint columns: pair k is held by lanes [k kP, (k + 1) kP) of the first
// np kP threads (KE column entries per lane, the inner product reduced over kP
// lanes), and only those threads take part in the sweeps, meeting at named barrier
// 1 once per round.  A round is a chain of latencies (loads, reduction, rotation,
// stores, barrier), so a small group with a short reduction beats spreading a pair
// over more lanes.  The column norms are recomputed at the start of every sweep and
// updated by each rotation (a - t|g|, b + t|g|), so a pair costs one reduced inner
// product.  Working copy column-major in Wc; eigenvectors (row-major, Z[i n + k])
// into Z, eigenvalues into w, and perm orders them descending.  Returns the sweeps
// used, -1 without convergence within `cap` sweeps.
constexpr int kP = 8;  // lanes per pair: 3 warps at n = 24, 6 at n = 48
static_assert((kLMax / 2) * kP <= kThreads, "the sweep group must fit in the block");

__device__ __forceinline__ void named_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

template <int KE>
__device__ int eig_onesided_t(const float2* Frm, float2* Wc, float2* Z, float* w, int* perm, int n, const Sm& sm,
                              int cap) {
    const int ne = n + (n & 1), np = ne / 2, nr = ne - 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nsync = (np * kP + 31) & ~31;  // whole warps; <= kThreads by the assert above
    const int k = threadIdx.x / kP, gl = threadIdx.x % kP;
    const int nent = (n + kP - 1) / kP;  // entries per lane and column (<= KE)
    for (int e = threadIdx.x; e < n * n; e += kThreads) {
        const int i = e / n, p = e % n;
        Wc[p * n + i] = Frm[e];
    }
    for (int e = threadIdx.x; e < kMaxSweeps; e += kThreads) sm.flags[e] = 0;
    // largest |g|^2 / (a b) met in the sweep, as int bits (non-negative floats order as ints)
    int* sweep_max = sm.flags + kMaxSweeps + 6;
    int* s_sweeps = sm.flags + kMaxSweeps + 7;
    if (threadIdx.x == 0) *s_sweeps = -1;
    __syncthreads();
    if (nr > 0 && threadIdx.x < nsync) {
        const bool live_k = k < np;
        const float tol2 = kOneSidedTol * kOneSidedTol;
        int sweeps = -1;
        for (int sweep = 0; sweep < cap; ++sweep) {
            if (threadIdx.x == 0) *sweep_max = 0;
            // round-robin positions, advanced by one each round; the round-0 pairs
            // (k, ne - 1 - k) cover every column once, so each group takes the exact
            // norms of its two columns
            int ia = (k == 0) ? 0 : (k - 1) % nr;
            int ib = (ne - 2 - k + nr) % nr;
            {
                const int c0 = (k == 0) ? 0 : 1 + ia, c1 = 1 + ib;
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    const int c = s ? c1 : c0;
                    const bool own = live_k && c < n;
                    float a = 0.f;
#pragma unroll
                    for (int h = 0; h < KE; ++h) {
                        const int i = gl + kP * h;
                        if (own && h < nent && i < n) {
                            const float2 v = Wc[c * n + i];
                            a = fmaf(v.x, v.x, fmaf(v.y, v.y, a));
                        }
                    }
#pragma unroll
                    for (int o = kP / 2; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o, kP);
                    if (own && gl == 0) w[c] = a;
                }
            }
            float ratio = 0.f;  // this thread's largest pair ratio in the sweep
            bool any = false;
            named_sync(1, nsync);
            for (int r = 0; r < nr; ++r) {
                const int pa = (k == 0) ? 0 : 1 + ia;
                const int pb = 1 + ib;
                const int p = min(pa, pb), q = max(pa, pb);
                const bool live = live_k && q < n;  // q == n: the dummy column of an odd n
                float2* fp = Wc + (live ? p : 0) * n;
                float2* fq = Wc + (live ? q : 0) * n;
                const float na = live ? w[p] : 1.f, nb = live ? w[q] : 1.f;
                float2 xp[KE], xq[KE];
#pragma unroll
                for (int h = 0; h < KE; ++h) {
                    const int i = gl + kP * h;
                    const bool in = live && h < nent && i < n;
                    xp[h] = in ? fp[i] : make_float2(0.f, 0.f);
                    xq[h] = in ? fq[i] : make_float2(0.f, 0.f);
                }
                float gr = 0.f, gi = 0.f;  // conj(f_p) f_q
#pragma unroll
                for (int h = 0; h < KE; ++h) {
                    gr = fmaf(xp[h].x, xq[h].x, fmaf(xp[h].y, xq[h].y, gr));
                    gi = fmaf(xp[h].x, xq[h].y, fmaf(-xp[h].y, xq[h].x, gi));
                }
#pragma unroll
                for (int o = kP / 2; o > 0; o >>= 1) {
                    gr += __shfl_xor_sync(0xffffffffu, gr, o, kP);
                    gi += __shfl_xor_sync(0xffffffffu, gi, o, kP);
                }
                if (++ia == nr) ia = 0;
                if (++ib == nr) ib = 0;
                // rotation of the pair, skipped where it is already orthogonal to the tolerance
                const float mag2 = fmaf(gr, gr, gi * gi);
                const float ab = na * nb;
                const bool rot = live && mag2 > FLT_MIN && mag2 > tol2 * ab;  // uniform over the group
                if (live && ab > 0.f) ratio = fmaxf(ratio, __fdividef(mag2, ab));
                any |= rot;
                if (rot) {
                    const float inv = rsqrtf(mag2);
                    const float mag = mag2 * inv;
                    const float tau = 0.5f * (nb - na) * inv;
                    // smaller root of t^2 + 2 tau t - 1 = 0 (t -> 0 as |tau| -> inf)
                    const float q1 = fmaf(tau, tau, 1.f);
                    const float t = copysignf(__fdividef(1.f, fabsf(tau) + q1 * rsqrtf(q1)), tau);
                    const float c = rsqrtf(fmaf(t, t, 1.f));
                    const float sn = t * c;
                    // F <- F U, U = [[c, s], [-s conj(ph), c conj(ph)]], ph = g / |g|
                    const float2 phc = make_float2(gr * inv, -gi * inv);
                    const float2 u10 = cscale(phc, -sn), u11 = cscale(phc, c);
#pragma unroll
                    for (int h = 0; h < KE; ++h) {
                        const int i = gl + kP * h;
                        if (h < nent && i < n) {
                            fp[i] = cadd(cscale(xp[h], c), cmul(xq[h], u10));
                            fq[i] = cadd(cscale(xp[h], sn), cmul(xq[h], u11));
                        }
                    }
                    if (gl == 0) {
                        w[p] = na - t * mag;
                        w[q] = nb + t * mag;
                    }
                }
                named_sync(1, nsync);
            }
            // sweep summary over the group's warps
            const bool wany = __any_sync(0xffffffffu, any);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) ratio = fmaxf(ratio, __shfl_xor_sync(0xffffffffu, ratio, o));
            if (lane == 0) {
                if (wany) sm.flags[sweep] = 1;
                atomicMax(sweep_max, __float_as_int(ratio));
            }
            named_sync(1, nsync);
            // converged: no rotation in this sweep, or every pair of it was within 1e-4 before its
            // rotation, so after it (quadratic convergence) within 1e-8 < the tolerance
            if (!sm.flags[sweep] || __int_as_float(*sweep_max) < 1e-8f) {
                sweeps = sweep + (sm.flags[sweep] ? 1 : 0);
                break;
            }
            named_sync(1, nsync);  // every thread has read *sweep_max before the next sweep resets it
        }
        if (threadIdx.x == 0) *s_sweeps = sweeps;
    }
    if (nr == 0 && threadIdx.x == 0) *s_sweeps = 0;
    __syncthreads();
    const int sweeps = *s_sweeps;
    // eigenvalues |f_k|^2, eigenvectors f_k / |f_k| (row-major into Z)
    for (int c = warp; c < n; c += kWarps) {
        float a = 0.f;
        for (int i = lane; i < n; i += 32) a = fmaf(Wc[c * n + i].x, Wc[c * n + i].x, fmaf(Wc[c * n + i].y, Wc[c * n + i].y, a));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        const float inv = (a > 0.f) ? rsqrtf(a) : 0.f;
        for (int i = lane; i < n; i += 32) Z[i * n + c] = cscale(Wc[c * n + i], inv);
        __syncwarp();
        if (lane == 0) w[c] = a;
    }
    __syncthreads();
    sort_desc(w, perm, n);
    return sweeps;
}

__device__ int eig_onesided(const float2* Frm, float2* Wc, float2* Z, float* w, int* perm, int n, const Sm& sm,
                             int cap) {
    constexpr int kEMax = (kLMax + kP - 1) / kP;
    return n <= 3 * kP ? eig_onesided_t<3>(Frm, Wc, Z, w, perm, n, sm, cap)
                       : eig_onesided_t<kEMax>(Frm, Wc, Z, w, perm, n, sm, cap);
}

// One Rayleigh-Ritz correction of the leading ncols-dimensional eigenspace of B
// (in T) after the FP32 Jacobi: with Z0 the FP32 eigenvectors (columns ordered by
// perm), B' = Z0^H B Z0 is formed for the (other x leading) block with products
// split exactly and double-float sums, and the leading columns are corrected to
// first order, z_k <- z_k + sum_n z_n B'_nk / (lambda_k - lambda_n).  This removes
// the u ||B|| / gap error of the FP32 eigenvectors without an eigensolve in higher
// precision.  Result (l x ncols) in Rc.  Pairs with a vanishing gap are skipped.
__device__ void refine_subspace(const Sm& sm, int l, int nc) {
    float4* Y = sm.Gd;  // l x nc double-float: B Z0[:, lead]
    for (int e = threadIdx.x; e < l * nc; e += kThreads) {
        const int i = e / nc, k = e % nc;
        const int zk = sm.perm[k];
        df re{0.f, 0.f}, im{0.f, 0.f};
        for (int j = 0; j < l; ++j) {
            const float2 b = sm.T[i * l + j], z = sm.Z[j * l + zk];
            dd_acc(re, b.x, z.x);
            dd_acc(re, -b.y, z.y);
            dd_acc(im, b.x, z.y);
            dd_acc(im, b.y, z.x);
        }
        Y[e] = make_float4(re.hi, re.lo, im.hi, im.lo);
    }
    __syncthreads();
    // E[n][k] = (Z0[:, n]^H Y[:, k]) / (lambda_k - lambda_n), n = nc..l-1 (into H, free after the Jacobi)
    float2* E = sm.H;
    const int no = l - nc;
    float lmax = 0.f;
    for (int i = 0; i < l; ++i) lmax = fmaxf(lmax, fabsf(sm.w[i]));
    for (int e = threadIdx.x; e < no * nc; e += kThreads) {
        const int n = nc + e / nc, k = e % nc;
        const int zn = sm.perm[n], zk = sm.perm[k];
        df re{0.f, 0.f}, im{0.f, 0.f};
        for (int i = 0; i < l; ++i) {
            const float2 z = sm.Z[i * l + zn];
            const float4 y = Y[i * nc + k];
            // conj(z) * y with y = (y.x + y.y) + j (y.z + y.w)
            dd_acc(re, z.x, y.x);
            dd_acc(re, z.y, y.z);
            dd_acc(im, z.x, y.z);
            dd_acc(im, -z.y, y.x);
            re.lo = fmaf(z.x, y.y, fmaf(z.y, y.w, re.lo));
            im.lo = fmaf(z.x, y.w, fmaf(-z.y, y.y, im.lo));
        }
        const float gap = sm.w[zk] - sm.w[zn];
        float2 v = make_float2(0.f, 0.f);
        if (fabsf(gap) > 1e-4f * lmax) v = make_float2((re.hi + re.lo) / gap, (im.hi + im.lo) / gap);
        E[(n - nc) * nc + k] = v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < l * nc; e += kThreads) {
        const int m = e / nc, k = e % nc;
        float2 z = sm.Z[m * l + sm.perm[k]];
        for (int n = 0; n < no; ++n) cfma(z, sm.Z[m * l + sm.perm[nc + n]], E[n * nc + k]);
        sm.Rc[e] = z;
    }
    __syncthreads();
}

// Re-orthonormalise the k columns of Z (n x k, row stride k, every CTA holds the
// same copy) by one double-float CholeskyQR pass: the accumulated FP32 Jacobi
// rotations leave them orthonormal only to ~sqrt(rounds) u, and U_s inherits
// that; the pass keeps their span.  Scratch: part and Gd (Xd is left alone).
__device__ void orthonormalize_cols_d(float2* Z, int n, int k, const Sm& sm) {
    gram_part_d(Z, n, k, sm.part);
    __syncthreads();
    for (int e = threadIdx.x; e < k * (k + 1) / 2; e += kThreads) {
        int i, j;
        tri_coords(e, k, i, j);
        zd g = zload(sm.part[e]);
        if (i == j) g.im = df{0.f, 0.f};
        sm.Gd[i * k + j] = zpack(g);
        if (i != j) sm.Gd[j * k + i] = zpack(zd{g.re, dd_neg(g.im)});
    }
    __syncthreads();
    if (2 * k * k <= n * n) {  // the elimination's scratch fits in part beside the inverse
        chol_inv_d(sm.Gd, sm.part, sm.part + k * k, k, sm);
    } else {
        chol_d(sm.Gd, k, sm);
        trinv_d(sm.Gd, sm.part, k, sm);
    }
    apply_upper_d(Z, n, k, sm.part);
}

// Zt = X W (l x nc, double-float, row stride nc) for X upper triangular l x l in
// double-float and W l x nc FP32 (row stride nc).
__device__ void upper_times_d(const float4* X, const float2* W, float4* Zt, int l, int nc) {
    for (int e = threadIdx.x; e < l * nc; e += kThreads) {
        const int i = e / nc, k = e % nc;
        zd s{df{0.f, 0.f}, df{0.f, 0.f}};
        for (int m = i; m < l; ++m) {
            const float2 w = W[m * nc + k];
            s = zadd(s, zmul(zload(X[i * l + m]), zd{df{w.x, 0.f}, df{w.y, 0.f}}));
        }
        Zt[e] = zpack(s);
    }
    __syncthreads();
}

// dst rows (rows x nc, row stride ld, global) = A rows (rows x l, FP32) * Zt (l x nc,
// double-float): FP32 products split exactly, double-float sums, one final rounding.
__device__ void apply_d(const float2* A, float2* __restrict__ dst, int rows, int l, const float4* Zt, int nc,
                        int64_t ld) {
    for (int e = threadIdx.x; e < rows * nc; e += kThreads) {
        const int r = e / nc, c = e % nc;
        df re{0.f, 0.f}, im{0.f, 0.f};
        for (int k = 0; k < l; ++k) {
            const float2 a = A[r * l + k];
            const float4 x = Zt[k * nc + c];  // (re.hi, re.lo, im.hi, im.lo)
            dd_acc(re, a.x, x.x);
            dd_acc(re, -a.y, x.z);
            dd_acc(im, a.x, x.z);
            dd_acc(im, a.y, x.x);
            re.lo = fmaf(a.x, x.y, fmaf(-a.y, x.w, re.lo));
            im.lo = fmaf(a.x, x.w, fmaf(a.y, x.y, im.lo));
        }
        dst[(int64_t)r * ld + c] = make_float2(re.hi + re.lo, im.hi + im.lo);
    }
}

// B rows of the next tensor-core sketch pass from this CTA's rows of V (rows x l in
// shared memory, entries r0 .. r0 + rows - 1), in the layout sketch_bprep_kernel writes:
// plain, rows [Vr, -Vi] and [Vi, Vr] rounded to TF32 at 2m; split, chunks of 8 entries
// (16 values) as [hi 16 | lo 16], hi = rn_tf32(v), lo = rn_tf32(v - hi).  r0 is a multiple
// of 8 (brows_by_cluster), so the CTA owns whole chunks; the last chunk's entries past M
// are written as zeros.
__device__ void write_brows(const FrameDesc* dp, const float2* Vs, int r0, int rows, int pass) {
    const int M = dp->M, l = dp->l, nrow = 2 * sketch_tc_lpad(l);
    if (!sketch_split(dp->prec, dp->t, pass)) {
        const int64_t rowlen = 2 * (int64_t)M;
        for (int t = threadIdx.x; t < nrow * rows; t += kThreads) {
            const int R = t / rows, r = t - R * rows, j = R >> 1;
            const float2 v = j < l ? Vs[r * l + j] : make_float2(0.f, 0.f);
            const float a = (R & 1) ? v.y : v.x, b = (R & 1) ? v.x : -v.y;
            *reinterpret_cast<float2*>(dp->Bsk + R * rowlen + 2 * (int64_t)(r0 + r)) =
                make_float2(__uint_as_float(tc::tf32_rn(a)), __uint_as_float(tc::tf32_rn(b)));
        }
        return;
    }
    // a row segment of chunk c is 8 pieces of 16 bytes: piece p < 4 holds the hi values
    // of entries 8c + 2p and 8c + 2p + 1, piece p + 4 their lo values.  A thread takes one
    // piece of both B rows of column j (re row 2j, im row 2j + 1: the same two entries).
    const int64_t rowlen = sketch_split_rowlen(M);
    const int nchunks = (2 * M + 15) / 16, c0 = r0 / 8, W = 8 * ((rows + 7) / 8);
    for (int t = threadIdx.x; t < (nrow / 2) * W; t += kThreads) {
        const int j = t / W, q = t - j * W, cc = q >> 3, p = q & 7;
        const int c = c0 + cc;
        if (c >= nchunks) continue;
        const int ra = 8 * cc + 2 * (p & 3);
        float2 va = make_float2(0.f, 0.f), vb = va;
        if (j < l) {
            if (ra < rows) va = Vs[ra * l + j];
            if (ra + 1 < rows) vb = Vs[(ra + 1) * l + j];
        }
        const float xr[4] = {va.x, -va.y, vb.x, -vb.y}, xi[4] = {va.y, va.x, vb.y, vb.x};
        uint4 orr, oi;
        uint32_t* vr = reinterpret_cast<uint32_t*>(&orr);
        uint32_t* vi = reinterpret_cast<uint32_t*>(&oi);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t hr = tc::tf32_rn(xr[u]), hi = tc::tf32_rn(xi[u]);
            vr[u] = p < 4 ? hr : tc::tf32_rn(xr[u] - __uint_as_float(hr));
            vi[u] = p < 4 ? hi : tc::tf32_rn(xi[u] - __uint_as_float(hi));
        }
        float* dst = dp->Bsk + (2 * j) * rowlen + 32 * (int64_t)c + 4 * p;
        *reinterpret_cast<uint4*>(dst) = orr;
        *reinterpret_cast<uint4*>(dst + rowlen) = oi;
    }
}

// ---------------------------------------------------------------- kernel ----
__global__ void __launch_bounds__(kThreads, 3) small_cluster_kernel(const FrameDesc* __restrict__ descs, int mode,
                                                                 int pass) {
    pdl_enter();
    extern __shared__ float4 smem_raw[];
    cg::cluster_group cl = cg::this_cluster();
    const int nc = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();
    const FrameDesc* dp = descs + blockIdx.x / nc;
    // pass < 0: the orth that precedes the FP32 refinement step (frames with refine only)
    if (mode == kOrth && (pass < 0 ? !dp->refine : dp->t < pass)) return;  // uniform over the cluster
    const int M = dp->M, l = dp->l;
    const int Mr = (M + nc - 1) / nc;
    const int r0 = min(M, rank * Mr);
    const int rows = min(Mr, M - r0);
    Sm sm;
    smem_layout(Mr, l, &sm, reinterpret_cast<char*>(smem_raw));
    // sweeps allowed in the eigensolves (a host-set cap below the solver's own exercises
    // the no-convergence report on ordinary data)
    const int cap = dp->sweep_cap > 0 ? min(dp->sweep_cap, kMaxSweeps) : kMaxSweeps;

    load_rows(dp->C, sm.Cs, r0, rows, l);
    if (mode == kOrth) {
        // The power step only needs a well-conditioned basis of range(C): the core
        // matrix H = V^H C and the Nystrom form C H^+ C^H do not depend on which
        // basis V is.  One double-float CholeskyQR pass leaves V orthonormal to about
        // u cond(C) (cond(V) ~ 1), so a second CholeskyQR pass is not taken.
        __syncthreads();
        const bool ok = cholqr_pass_d(cl, sm.Cs, rows, l, sm, sm.Rc);
        store_rows(sm.Cs, dp->V, r0, rows, l);
        // the next sketch pass's B rows, straight from the rows in shared memory (the host
        // planned this cluster size; any other would leave them unwritten)
        if (pass >= 1 && dp->bsk_orth_nc > 0) {
            if (dp->bsk_orth_nc == nc && brows_by_cluster(M, nc))
                write_brows(dp, sm.Cs, r0, rows, pass);
            else if (rank == 0 && threadIdx.x == 0)
                set_status(dp->status, FM_ERR_CUDA);
        }
        if (!ok && rank == 0 && threadIdx.x == 0) set_status(dp->status, FM_ERR_NO_CONVERGENCE);
        return;
    }

    // H = P^H C  (core matrix, Eq. 8 / Alg. 2)
    // sampling without power steps: H = C(I, :) (Alg. 1); after a refinement step the
    // sketch is V-based as in Alg. 2, so H = V^H C
    const bool sampled0 = (dp->method == FM_RAND_SAMPLING && dp->t == 0 && !dp->refine);
    // C = Q R_c with Q = C R_c^{-1} left implicit: R_c from the double-float Gram of C
    // (Cholesky, pivot floor as in CholeskyQR), X = R_c^{-1} kept in Xd until U_s = C (X W)
    // is formed at the end for the ncols selected eigenvectors W only.  U_s^H U_s =
    // W^H X^H (C^H C) X W = W^H W up to double-float rounding, so one pass gives the
    // orthonormality of a second CholeskyQR pass without forming Q.  The Gram partials
    // of H (in Z) and of C (in part) are summed over the cluster in one pass; V rows are
    // dead once H is formed (Gd aliases them).
    if (!sampled0) {
        load_rows(dp->V, sm.Vs, r0, rows, l);
        __syncthreads();
        gram_part_f(sm.Vs, sm.Cs, rows, l, false, sm.Z);
        gram_part_d(sm.Cs, rows, l, sm.part);
        reduce_fd(cl, sm.Z, sm.H, sm.part, sm.Gd, l);
    } else {
        for (int e = threadIdx.x; e < l * l; e += kThreads) {
            const int i = e / l, j = e % l;
            sm.H[e] = dp->C[(int64_t)dp->idx[i] * l + j];
        }
        __syncthreads();
        gram_part_d(sm.Cs, rows, l, sm.part);
        reduce_d(cl, sm.part, sm.Gd, l);
    }
    // exact Hermitian part, kept in H and copied to Z (the FP32 sweep below factors Z in
    // place; H stays for the pseudo-inverse branch)
    for (int e = threadIdx.x; e < l * l; e += kThreads) {
        const int i = e / l, j = e % l;
        if (i < j) {
            const float2 a = sm.H[i * l + j], b = sm.H[j * l + i];
            const float2 h = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
            sm.H[i * l + j] = h;
            sm.H[j * l + i] = cconj(h);
            sm.Z[i * l + j] = h;
            sm.Z[j * l + i] = cconj(h);
        } else if (i == j) {
            sm.H[e].y = 0.f;
            sm.Z[e] = make_float2(sm.H[e].x, 0.f);
        }
    }
    __syncthreads();

    // B = R_c H^+ R_c^H: in the same column sweep as R_c and X (part is free after the
    // reduction), H = R_h^H R_h in FP32 (in Z) with R_h^{-1} into Rc
    bool pd;
    bool ok = chol_inv_pair(sm.Gd, sm.Xd, sm.part, sm.Z, sm.Rc, l, sm, &pd);
    if (pd) {
        // F = R_c R_h^{-1} (upper, R_c rounded to FP32; R_h^{-1} from the upper triangle of
        // Rc) into T, B = F F^H into H
        for (int e = threadIdx.x; e < l * l; e += kThreads) {
            const int i = e / l, j = e % l;
            float2 s = make_float2(0.f, 0.f);
            for (int k = i; k <= j; ++k) {
                const float4 g = sm.Gd[i * l + k];
                cfma(s, make_float2(g.x + g.y, g.z + g.w), sm.Rc[k * l + j]);
            }
            sm.T[e] = s;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < l * l; e += kThreads) {
            const int i = e / l, j = e % l;
            if (i > j) continue;
            float2 s = make_float2(0.f, 0.f);
            for (int k = j; k < l; ++k) cfmaconj(s, sm.T[i * l + k], sm.T[j * l + k]);
            if (i == j) s.y = 0.f;
            sm.H[i * l + j] = s;
            sm.H[j * l + i] = cconj(s);
        }
        __syncthreads();
    } else {
        // eigenvalue pseudo-inverse: H = Z diag(w) Z^H, B = (R_c Z) diag(w+) (R_c Z)^H
        const int s0 = jacobi(sm.H, sm.Z, sm.w, sm.perm, l, sm, cap);
        if (s0 < 0) ok = false;
        if (threadIdx.x == 0) {
            float amax = 0.f;
            for (int i = 0; i < l; ++i) amax = fmaxf(amax, fabsf(sm.w[i]));
            sm.scal[1] = (float)l * FLT_EPSILON * amax;
        }
        __syncthreads();
        const float thr = sm.scal[1];
        for (int e = threadIdx.x; e < l * l; e += kThreads) {
            const int i = e / l, k = e % l;
            float2 s = make_float2(0.f, 0.f);
            for (int m = i; m < l; ++m) {
                const float4 g = sm.Gd[i * l + m];
                cfma(s, make_float2(g.x + g.y, g.z + g.w), sm.Z[m * l + k]);
            }
            sm.T[e] = s;
        }
        __syncthreads();
        for (int k = threadIdx.x; k < l; k += kThreads) sm.w[k] = (fabsf(sm.w[k]) > thr) ? 1.f / sm.w[k] : 0.f;
        __syncthreads();
        for (int e = threadIdx.x; e < l * l; e += kThreads) {
            const int i = e / l, j = e % l;
            if (i > j) continue;
            float2 s = make_float2(0.f, 0.f);
            for (int k = 0; k < l; ++k) cfmaconj(s, cscale(sm.T[i * l + k], sm.w[k]), sm.T[j * l + k]);
            if (i == j) s.y = 0.f;
            sm.H[i * l + j] = s;
            sm.H[j * l + i] = cconj(s);
        }
        __syncthreads();
    }
    // eig(B) = U_B L_B U_B^H in FP32 (B kept in T for the refinement below): with
    // B = F F^H (F in T) through the one-sided Jacobi SVD of F, else two-sided
    // Jacobi on B
    int s2;
    if (pd) {
        s2 = eig_onesided(sm.T, sm.Xf, sm.Z, sm.w, sm.perm, l, sm, cap);  // Gd (under Xf) is dead once F is formed
        for (int e = threadIdx.x; e < l * l; e += kThreads) sm.T[e] = sm.H[e];
        __syncthreads();
    } else {
        for (int e = threadIdx.x; e < l * l; e += kThreads) sm.T[e] = sm.H[e];
        __syncthreads();
        s2 = jacobi(sm.H, sm.Z, sm.w, sm.perm, l, sm, cap);
    }
    const int nc_out = dp->ncols;
    refine_subspace(sm, l, nc_out);
    orthonormalize_cols_d(sm.Rc, l, nc_out, sm);
    // U_s rows = C rows * (R_c^{-1} U_B[:, :ncols]) (U_B refined, in Rc: l x ncols)
    upper_times_d(sm.Xd, sm.Rc, sm.Gd, l, nc_out);
    apply_d(sm.Cs, dp->Us + (int64_t)r0 * dp->kpad, rows, l, sm.Gd, nc_out, dp->kpad);
    if (rank == 0 && threadIdx.x == 0 && (s2 < 0 || !ok)) set_status(dp->status, FM_ERR_NO_CONVERGENCE);
}

int cluster_size_for(int max_M) {
    int nc = 1;
    while (nc < 8 && (max_M + nc - 1) / nc > kMaxRows) nc *= 2;
    return nc;
}

// Clusters of nc CTAs (each with the shared memory of ceil(M / nc) rows) that the device
// can hold at once, as the runtime reports it (clusters sit inside a GPC, so this is
// below SMs x CTAs per SM / nc); cached per device, size and shared memory.
int max_active_clusters(int nc, size_t smem) {
    static std::mutex mu;
    static std::map<std::tuple<int, int, size_t>, int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    const auto key = std::make_tuple(dev, nc, smem);
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    int n = 0;
    if (cudaFuncSetAttribute(small_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)nc, 1, 1);
        cfg.blockDim = dim3(kThreads, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)nc;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if (cudaOccupancyMaxActiveClusters(&n, small_cluster_kernel, &cfg) != cudaSuccess) n = 0;
    }
    cudaGetLastError();
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = n;
    return n;
}

// The cluster size of a launch: the smallest that keeps every CTA at <= kMaxRows rows,
// grown (up to 8, at least 32 rows per CTA) while the launch stays within one CTA per SM
// and every frame's cluster can be resident at once: the row-parallel phases (the loads,
// the Gram partials, V and U_s) shorten.  Beyond one CTA per SM the CTAs that share an
// SM slow each other (every CTA of a cluster repeats the l x l work): measured at 64
// frames of M = 512, clusters of 5-7 took the final solve from 0.164 to 0.186 ms, while
// one frame in a cluster of 8 took 0.38 instead of 0.41 ms end to end.
int cluster_size_for(int max_M, int max_l, int n_frames) {
    int nc = cluster_size_for(max_M);
    int dev = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return nc;
    while (nc < 8 && (max_M + nc) / (nc + 1) >= 32 && (int64_t)(nc + 1) * n_frames <= n_sm) {
        const int next = nc + 1;
        const size_t smem = smem_layout((max_M + next - 1) / next, max_l, nullptr, nullptr);
        if (max_active_clusters(next, smem) < n_frames) break;
        nc = next;
    }
    return nc;
}

cudaError_t launch_small(const FrameDesc* d, int n_frames, int max_M, int max_l, int mode, int pass, cudaStream_t s) {
    const int nc = cluster_size_for(max_M, max_l, n_frames);
    const int Mr = (max_M + nc - 1) / nc;
    const size_t smem = smem_layout(Mr, max_l, nullptr, nullptr);
    cudaError_t e = cudaFuncSetAttribute(small_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nc * n_frames), 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)nc;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;  // a chain kernel (pdl_enter)
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    count_launch();
    e = cudaLaunchKernelEx(&cfg, small_cluster_kernel, d, mode, pass);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace

size_t small_smem_bytes(int max_M, int l) {
    const int nc = cluster_size_for(max_M);
    return smem_layout((max_M + nc - 1) / nc, l, nullptr, nullptr);
}

int orth_cluster_size(int max_M, int max_l, int n_frames) { return cluster_size_for(max_M, max_l, n_frames); }

cudaError_t launch_orth(const FrameDesc* d, int n_frames, int max_M, int max_l, int pass, cudaStream_t s) {
    return launch_small(d, n_frames, max_M, max_l, kOrth, pass, s);
}

cudaError_t launch_final(const FrameDesc* d, int n_frames, int max_M, int max_l, cudaStream_t s) {
    return launch_small(d, n_frames, max_M, max_l, kFinal, 0, s);
}

}  // namespace fm
