// Small dense FP64 complex algebra on the device, one CTA per problem:
//  * eig with right and left eigenvectors ([zr, zl, D] = eig(C), paper Sec. 1
//    notation), eigenvalues ordered by smallest |lambda| (Sec. 2);
//  * the coefficient-space part of Algorithm BiCG-eigen (Sec. 2);
//  * final Ritz pairs of an eigBiCG window (Algorithm eigBiCG, step 4);
//  * LU factorisation / solves for H = U_l^H A U_r (Algorithm Incremental).
//
// Eigen-solver: Householder reduction to Hessenberg form, complex single-shift
// (Wilkinson) implicit QR to Schur form T = Q^H C Q (Golub & Van Loan,
// "Matrix Computations", Sec. 7.4-7.5), eigenvectors of T by back / forward
// substitution, mapped back with Q. Conventions: right vectors have unit
// 2-norm with their largest-modulus entry real positive; left vectors satisfy
// z^H y = 1.
#include <mutex>

#include "../../include/lqcd.h"
#include "dfloat.cuh"
#include "kernels.cuh"

namespace lqcd {
namespace {

constexpr int ET = 128;          // threads per eigen CTA
constexpr double EPS = 2.220446049250313e-16;

__device__ __forceinline__ double2 czero() { return make_double2(0.0, 0.0); }
__device__ __forceinline__ double2 cone() { return make_double2(1.0, 0.0); }

// |re| + |im|: the modulus surrogate used for negligibility tests (no sqrt).
__device__ __forceinline__ double cabs1(double2 a) { return fabs(a.x) + fabs(a.y); }

// 1/sqrt(a) for a > 0 in FP64. FP64 arithmetic issues at 1/64 of the FP32 rate
// on this GPU, so the library's FP64 square root and divide are long serial
// chains; inside FP32's normal range, an FP32 reciprocal square root seeds
// Newton-Raphson for f(y) = 1/y^2 - a, y <- y (3 - a y^2) / 2, which doubles
// the correct bits per step: two steps take the FP32 seed (about 22 bits) to
// FP64 accuracy. Outside that range: 1 / sqrt(a).
__device__ __forceinline__ double rsqrt_fp64(double a) {
    if (!(a > 1e-30 && a < 1e30)) return 1.0 / sqrt(a);
    double y = (double)rsqrtf((float)a);
    const double h = 0.5 * a;
    y = y * fma(-h * y, y, 1.5);
    y = y * fma(-h * y, y, 1.5);
    return y;
}

// 1/a in FP64 the same way: FP32 reciprocal seed, Newton-Raphson for
// f(y) = 1/y - a, y <- y (2 - a y), two steps. Outside FP32's normal range: 1 / a.
__device__ __forceinline__ double rcp_fp64(double a) {
    const double m = fabs(a);
    if (!(m > 1e-30 && m < 1e30)) return 1.0 / a;
    double y = (double)__frcp_rn((float)a);
    y = y * fma(-a, y, 2.0);
    y = y * fma(-a, y, 2.0);
    return y;
}

// Unitary rotation G = [[cx, cy], [-conj(cy), conj(cx)]] with G [x; y] = [n; 0],
// cx = conj(x)/n, cy = conj(y)/n, n = sqrt(|x|^2 + |y|^2): one reciprocal square
// root. (One thread forms it: FP64 issue, not the barriers around it, bounds
// this solver, and every warp forming it would quadruple that work.)
__device__ __forceinline__ void givens(double2 x, double2 y, double2& cx, double2& cy) {
    const double n2 = cabs2(x) + cabs2(y);
    if (n2 == 0.0) { cx = cone(); cy = czero(); return; }
    const double inv = rsqrt_fp64(n2);
    cx = inv * conj_(x);
    cy = inv * conj_(y);
}

// ---------------------------------------------------------------------------
// Block-cooperative eigen-solver on A (n x n, leading dim lda, shared memory).
// On return A holds the Schur form T, Q the Schur vectors. Returns 0 on
// success, 1 if QR failed to converge.
__device__ int schur(double2* A, double2* Q, int n, int lda, double2* v /* n */, double* sh) {
    const int tid = threadIdx.x;
    // Q = I
    for (int e = tid; e < n * lda; e += blockDim.x) Q[e] = ((e / lda) == (e % lda)) ? cone() : czero();
    __syncthreads();
    // Householder reduction to upper Hessenberg. A column with nothing below its
    // subdiagonal is skipped, and a reflection spans only the rows up to the
    // column's last nonzero: the projected matrices of eigBiCG are tridiagonal,
    // or after a restart diagonal + coupling arrow + tridiagonal, so most
    // columns need no work.
    for (int k = 0; k + 2 < n; ++k) {
        // v = x + e^{i theta} ||x|| e1, x = A[k+1:last+1, k]
        if (tid == 0) {
            double nrm2 = 0.0, tail = 0.0;
            int last = k + 1;
            for (int i = k + 1; i < n; ++i) {
                const double a2 = cabs2(A[i * lda + k]);
                nrm2 += a2;
                if (i >= k + 2) tail += a2;
                if (a2 != 0.0) last = i;
            }
            double alpha = sqrt(nrm2);
            double2 x0 = A[(k + 1) * lda + k];
            double ax0 = cabs_(x0);
            double2 ph = ax0 > 0.0 ? make_double2(x0.x / ax0, x0.y / ax0) : cone();
            sh[0] = tail > 0.0 ? alpha : 0.0;   // 0: skip the step
            sh[1] = alpha > 0.0 ? 1.0 / (alpha * (alpha + ax0)) : 0.0;   // tau = 2/||v||^2
            sh[2] = ph.x; sh[3] = ph.y;
            sh[5] = (double)last;
        }
        __syncthreads();
        double alpha = sh[0], tau = sh[1];
        double2 ph = make_double2(sh[2], sh[3]);
        const int last = (int)sh[5];
        if (alpha == 0.0) { __syncthreads(); continue; }
        for (int i = k + 1 + tid; i <= last; i += blockDim.x) v[i - k - 1] = A[i * lda + k];
        __syncthreads();
        if (tid == 0) v[0] = v[0] + alpha * ph;
        __syncthreads();
        const int len = last - k;
        // rows k+1..n-1 of A: A -= tau v (v^H A), columns k..n-1
        for (int j = k + tid; j < n; j += blockDim.x) {
            double2 w = czero();
            for (int i = 0; i < len; ++i) w = w + cdot(v[i], A[(k + 1 + i) * lda + j]);
            w = tau * w;
            for (int i = 0; i < len; ++i) A[(k + 1 + i) * lda + j] = A[(k + 1 + i) * lda + j] - v[i] * w;
        }
        __syncthreads();
        // columns k+1..n-1 of A (all rows) and of Q: X -= tau (X v) v^H
        for (int i = tid; i < 2 * n; i += blockDim.x) {
            double2* row = i < n ? A + i * lda : Q + (i - n) * lda;
            double2 u = czero();
            for (int l = 0; l < len; ++l) u = u + row[k + 1 + l] * v[l];
            u = tau * u;
            for (int l = 0; l < len; ++l) row[k + 1 + l] = row[k + 1 + l] - mulc(u, v[l]);
        }
        __syncthreads();
        for (int i = k + 2 + tid; i <= last; i += blockDim.x) A[i * lda + k] = czero();
        __syncthreads();
    }
    // Frobenius norm for the negligibility tests.
    if (tid == 0) {
        double f = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = (i > 0 ? i - 1 : 0); j < n; ++j) f += cabs2(A[i * lda + j]);
        sh[4] = sqrt(f);
    }
    __syncthreads();
    const double anorm = sh[4] > 0.0 ? sh[4] : 1.0;
    // Single-shift implicit QR with deflation from the bottom.
    __shared__ int s_l, s_hi, s_fail;
    __shared__ double2 s_cx, s_cy, s_mu;
    if (tid == 0) { s_hi = n - 1; s_fail = 0; }
    __syncthreads();
    int iters = 0, total = 0;
    while (true) {
        if (tid == 0) {
            int hi = s_hi;
            int l = hi;
            while (l > 0) {
                double tst = cabs1(A[(l - 1) * lda + l - 1]) + cabs1(A[l * lda + l]);
                if (tst == 0.0) tst = anorm;
                if (cabs1(A[l * lda + l - 1]) <= EPS * tst) { A[l * lda + l - 1] = czero(); break; }
                --l;
            }
            s_l = l;
        }
        __syncthreads();
        int hi = s_hi, l = s_l;
        if (hi <= 0) break;
        if (l == hi) {
            __syncthreads();
            if (tid == 0) s_hi = hi - 1;
            iters = 0;
            __syncthreads();
            continue;
        }
        ++iters; ++total;
        if (iters > 60 || total > 60 * n) { if (tid == 0) s_fail = 1; __syncthreads(); break; }
        if (tid == 0) {
            double2 a = A[(hi - 1) * lda + hi - 1], b = A[(hi - 1) * lda + hi];
            double2 c = A[hi * lda + hi - 1], d = A[hi * lda + hi];
            double2 mu;
            if (iters % 11 == 10) {
                // exceptional shift
                mu = d + make_double2(0.75 * cabs1(c), 0.0);
            } else {
                double2 t = 0.5 * (a - d);
                double2 bc = b * c;
                double2 disc2 = t * t + bc;
                // complex sqrt
                double r = cabs_(disc2);
                double sx = sqrt(0.5 * (r + disc2.x));
                double sy = sqrt(0.5 * (r - disc2.x));
                if (disc2.y < 0) sy = -sy;
                double2 disc = make_double2(sx, sy);
                double2 den1 = t + disc, den2 = t - disc;
                double2 den = cabs2(den1) >= cabs2(den2) ? den1 : den2;
                mu = cabs2(den) > 0.0 ? d - cdiv(bc, den) : d;
            }
            s_mu = mu;
        }
        __syncthreads();
        double2 mu = s_mu;
        for (int k = l; k < hi; ++k) {
            if (tid == 0) {
                double2 x, y;
                if (k == l) { x = A[l * lda + l] - mu; y = A[(l + 1) * lda + l]; }
                else { x = A[k * lda + k - 1]; y = A[(k + 1) * lda + k - 1]; }
                double2 cx, cy;
                givens(x, y, cx, cy);
                s_cx = cx; s_cy = cy;
            }
            __syncthreads();
            const double2 cx = s_cx, cy = s_cy;
            const double2 cxc = conj_(cx), cyc = conj_(cy);
            // rows k, k+1:  [a; b] <- G [a; b]
            const int j0 = (k == l) ? l : k - 1;
            for (int j = j0 + tid; j < n; j += blockDim.x) {
                double2 a = A[k * lda + j], b = A[(k + 1) * lda + j];
                A[k * lda + j] = cx * a + cy * b;
                A[(k + 1) * lda + j] = cxc * b - cyc * a;
            }
            __syncthreads();
            // columns k, k+1 of A (rows 0..min(k+2, hi)) and of Q (all rows):  [a, b] <- [a, b] G^H
            const int i1 = min(k + 2, hi);
            for (int i = tid; i < (i1 + 1) + n; i += blockDim.x) {
                double2* row = i <= i1 ? A + i * lda : Q + (i - i1 - 1) * lda;
                double2 a = row[k], b = row[k + 1];
                row[k] = a * cxc + b * cyc;
                row[k + 1] = b * cx - a * cy;
            }
            __syncthreads();
            if (k > l && tid == 0) A[(k + 1) * lda + k - 1] = czero();
            __syncthreads();
        }
    }
    __syncthreads();
    int fail = s_fail;
    __syncthreads();
    return fail;
}

// ---------------------------------------------------------------------------
// The same reduction in double-float arithmetic (pairs of FP32 numbers, about
// 48 significant bits; Knuth's two-sum and Dekker's FMA two-product, as for the
// reliable-update residual), for the restart's eigen-solves of H^(m) and
// H^(m-1): the FP32 pipeline issues 64 times faster than FP64 on this GPU, and
// the Householder and QR updates are the bulk of the solve. A and Q keep their
// 16-byte slots (one double2 or one double-float complex); the scalars of a
// step (norms, shift, rotation) are formed by one thread in FP64. On return A,
// Q hold T and the Schur vectors in FP64 again.
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
    const float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    const float h = p + e;
    return {h, e - (h - p)};
}
__device__ __forceinline__ dfc dc_mul(dfc a, dfc b) {
    return {df_mul(a.x, b.x) - df_mul(a.y, b.y), df_mul(a.x, b.y) + df_mul(a.y, b.x)};
}
__device__ __forceinline__ dfc dc_conj(dfc a) { return {a.x, -a.y}; }
__device__ __forceinline__ dfc dc_scale(dfl s, dfc a) { return {df_mul(s, a.x), df_mul(s, a.y)}; }
__device__ __forceinline__ dfl dc_abs2(dfc a) { return df_mul(a.x, a.x) + df_mul(a.y, a.y); }
__device__ __forceinline__ float dc_abs1f(dfc a) { return fabsf(a.x.h) + fabsf(a.y.h); }
__device__ __forceinline__ dfc dc_from(double2 a) { return {df_split(a.x), df_split(a.y)}; }
__device__ __forceinline__ double2 dc_to(dfc a) { return make_double2(df_value(a.x), df_value(a.y)); }
__device__ __forceinline__ dfc dc_zero() { return {{0.f, 0.f}, {0.f, 0.f}}; }
__device__ __forceinline__ dfc dc_one() { return {{1.f, 0.f}, {0.f, 0.f}}; }

constexpr float EPS_DF = 1.4e-14f;   // about four units of double-float rounding

__device__ int schur_df(double2* A64, double2* Q64, int n, int lda, double2* v64, double* sh) {
    const int tid = threadIdx.x;
    dfc* A = reinterpret_cast<dfc*>(A64);
    dfc* Q = reinterpret_cast<dfc*>(Q64);
    dfc* v = reinterpret_cast<dfc*>(v64);
    for (int e = tid; e < n * lda; e += blockDim.x) {   // in place: each thread converts its own slots
        if (e % lda < n) {
            const double2 a = A64[e];
            A[e] = dc_from(a);
        }
        Q[e] = ((e / lda) == (e % lda)) ? dc_one() : dc_zero();
    }
    __syncthreads();
    // Householder reduction (columns already Hessenberg skipped, reflections up
    // to the column's last nonzero), as in schur().
    for (int k = 0; k + 2 < n; ++k) {
        if (tid == 0) {
            dfl nrm2 = {0.f, 0.f}, tail = {0.f, 0.f};
            int last = k + 1;
            for (int i = k + 1; i < n; ++i) {
                const dfl a2 = dc_abs2(A[i * lda + k]);
                nrm2 = nrm2 + a2;
                if (i >= k + 2) tail = tail + a2;
                if (a2.h != 0.f) last = i;
            }
            const double alpha = sqrt(df_value(nrm2));
            const double2 x0 = dc_to(A[(k + 1) * lda + k]);
            const double ax0 = cabs_(x0);
            const double2 ph = ax0 > 0.0 ? make_double2(x0.x / ax0, x0.y / ax0) : make_double2(1.0, 0.0);
            sh[0] = tail.h > 0.f ? alpha : 0.0;   // 0: skip the step
            sh[1] = alpha > 0.0 ? 1.0 / (alpha * (alpha + ax0)) : 0.0;
            sh[2] = ph.x; sh[3] = ph.y;
            sh[5] = (double)last;
        }
        __syncthreads();
        const double alpha = sh[0];
        const dfl tau = df_split(sh[1]);
        const double2 ph = make_double2(sh[2], sh[3]);
        const int last = (int)sh[5];
        if (alpha == 0.0) { __syncthreads(); continue; }
        for (int i = k + 1 + tid; i <= last; i += blockDim.x) v[i - k - 1] = A[i * lda + k];
        __syncthreads();
        if (tid == 0) v[0] = v[0] + dc_from(make_double2(alpha * ph.x, alpha * ph.y));
        __syncthreads();
        const int len = last - k;
        for (int j = k + tid; j < n; j += blockDim.x) {
            dfc w = dc_zero();
            for (int i = 0; i < len; ++i) w = w + dc_mul(dc_conj(v[i]), A[(k + 1 + i) * lda + j]);
            w = dc_scale(tau, w);
            for (int i = 0; i < len; ++i) A[(k + 1 + i) * lda + j] = A[(k + 1 + i) * lda + j] - dc_mul(v[i], w);
        }
        __syncthreads();
        for (int i = tid; i < 2 * n; i += blockDim.x) {
            dfc* row = i < n ? A + i * lda : Q + (i - n) * lda;
            dfc u = dc_zero();
            for (int l = 0; l < len; ++l) u = u + dc_mul(row[k + 1 + l], v[l]);
            u = dc_scale(tau, u);
            for (int l = 0; l < len; ++l) row[k + 1 + l] = row[k + 1 + l] - dc_mul(u, dc_conj(v[l]));
        }
        __syncthreads();
        for (int i = k + 2 + tid; i <= last; i += blockDim.x) A[i * lda + k] = dc_zero();
        __syncthreads();
    }
    if (tid == 0) {
        dfl f = {0.f, 0.f};
        for (int i = 0; i < n; ++i)
            for (int j = (i > 0 ? i - 1 : 0); j < n; ++j) f = f + dc_abs2(A[i * lda + j]);
        sh[4] = sqrt(df_value(f));
    }
    __syncthreads();
    const float anorm = sh[4] > 0.0 ? (float)sh[4] : 1.f;
    __shared__ int s_l, s_hi, s_fail;
    __shared__ dfc s_cx, s_cy, s_mu;
    if (tid == 0) { s_hi = n - 1; s_fail = 0; }
    __syncthreads();
    int iters = 0, total = 0;
    while (true) {
        if (tid == 0) {
            const int hi = s_hi;
            int l = hi;
            while (l > 0) {
                float tst = dc_abs1f(A[(l - 1) * lda + l - 1]) + dc_abs1f(A[l * lda + l]);
                if (tst == 0.f) tst = anorm;
                if (dc_abs1f(A[l * lda + l - 1]) <= EPS_DF * tst) { A[l * lda + l - 1] = dc_zero(); break; }
                --l;
            }
            s_l = l;
        }
        __syncthreads();
        const int hi = s_hi, l = s_l;
        if (hi <= 0) break;
        if (l == hi) {
            __syncthreads();
            if (tid == 0) s_hi = hi - 1;
            iters = 0;
            __syncthreads();
            continue;
        }
        ++iters; ++total;
        if (iters > 60 || total > 60 * n) { if (tid == 0) s_fail = 1; __syncthreads(); break; }
        if (tid == 0) {   // Wilkinson shift in FP64
            const double2 a = dc_to(A[(hi - 1) * lda + hi - 1]), b = dc_to(A[(hi - 1) * lda + hi]);
            const double2 c = dc_to(A[hi * lda + hi - 1]), d = dc_to(A[hi * lda + hi]);
            double2 mu;
            if (iters % 11 == 10) {
                mu = d + make_double2(0.75 * cabs1(c), 0.0);
            } else {
                const double2 t = 0.5 * (a - d);
                const double2 bc = b * c;
                const double2 disc2 = t * t + bc;
                const double r = cabs_(disc2);
                const double sx = sqrt(0.5 * (r + disc2.x));
                double sy = sqrt(0.5 * (r - disc2.x));
                if (disc2.y < 0) sy = -sy;
                const double2 disc = make_double2(sx, sy);
                const double2 den1 = t + disc, den2 = t - disc;
                const double2 den = cabs2(den1) >= cabs2(den2) ? den1 : den2;
                mu = cabs2(den) > 0.0 ? d - cdiv(bc, den) : d;
            }
            s_mu = dc_from(mu);
        }
        __syncthreads();
        const dfc mu = s_mu;
        for (int k = l; k < hi; ++k) {
            if (tid == 0) {
                dfc x, y;
                if (k == l) { x = A[l * lda + l] - mu; y = A[(l + 1) * lda + l]; }
                else { x = A[k * lda + k - 1]; y = A[(k + 1) * lda + k - 1]; }
                const double n2 = df_value(dc_abs2(x) + dc_abs2(y));
                if (n2 == 0.0) { s_cx = dc_one(); s_cy = dc_zero(); }
                else {
                    const dfl inv = df_split(rsqrt_fp64(n2));
                    s_cx = dc_scale(inv, dc_conj(x));
                    s_cy = dc_scale(inv, dc_conj(y));
                }
            }
            __syncthreads();
            const dfc cx = s_cx, cy = s_cy;
            const dfc cxc = dc_conj(cx), cyc = dc_conj(cy);
            const int j0 = (k == l) ? l : k - 1;
            for (int j = j0 + tid; j < n; j += blockDim.x) {
                const dfc a = A[k * lda + j], b = A[(k + 1) * lda + j];
                A[k * lda + j] = dc_mul(cx, a) + dc_mul(cy, b);
                A[(k + 1) * lda + j] = dc_mul(cxc, b) - dc_mul(cyc, a);
            }
            __syncthreads();
            const int i1 = min(k + 2, hi);
            for (int i = tid; i < (i1 + 1) + n; i += blockDim.x) {
                dfc* row = i <= i1 ? A + i * lda : Q + (i - i1 - 1) * lda;
                const dfc a = row[k], b = row[k + 1];
                row[k] = dc_mul(a, cxc) + dc_mul(b, cyc);
                row[k + 1] = dc_mul(b, cx) - dc_mul(a, cy);
            }
            __syncthreads();
            if (k > l && tid == 0) A[(k + 1) * lda + k - 1] = dc_zero();
            __syncthreads();
        }
    }
    __syncthreads();
    const int fail = s_fail;
    for (int e = tid; e < n * lda; e += blockDim.x) {   // back to FP64, in place
        if (e % lda < n) {
            const dfc a = A[e];
            A64[e] = dc_to(a);
        }
        const dfc q = Q[e];
        Q64[e] = dc_to(q);
    }
    __syncthreads();
    return fail;
}

// Order of the eigenvalues on the diagonal of T: smallest |lambda|, then Im.
__device__ void order_eigs(const double2* T, int n, int lda, int* ord) {
    if (threadIdx.x == 0) {
        // squared moduli order the same way as moduli (ties included)
        for (int i = 0; i < n; ++i) ord[i] = i;
        for (int i = 1; i < n; ++i) {
            int key = ord[i];
            double2 lk = T[key * lda + key];
            double ak = cabs2(lk);
            int j = i - 1;
            while (j >= 0) {
                double2 lj = T[ord[j] * lda + ord[j]];
                double aj = cabs2(lj);
                bool after = (aj > ak) || (aj == ak && lj.y > lk.y);
                if (!after) break;
                ord[j + 1] = ord[j];
                --j;
            }
            ord[j + 1] = key;
        }
    }
    __syncthreads();
}

// Eigenvectors for the eigenvalues T[ord[i], ord[i]], i < nsel.
// Y, Z (global or shared), column i of an n x nsel row-major array (ld = ldyz).
// W1, W2: scratch of n*nsel each (y', w in Schur coordinates).
__device__ void eigvecs(const double2* T, const double2* Q, int n, int lda, const int* ord, int nsel,
                        double2* Y, double2* Z, int ldyz, double2* W1, double2* W2, double anorm) {
    const int tid = threadIdx.x;
    const double smin = fmax(EPS * anorm, 1e-300);
    // Back / forward substitution, one (vector, side) per thread.
    for (int t = tid; t < 2 * nsel; t += blockDim.x) {
        const int i = t % nsel;
        const bool left = t >= nsel;
        const int k = ord[i];
        const double2 lam = T[k * lda + k];
        double2* w = (left ? W2 : W1) + (size_t)i * n;
        for (int j = 0; j < n; ++j) w[j] = czero();
        w[k] = cone();
        if (!left) {
            for (int j = k - 1; j >= 0; --j) {
                double2 sacc = czero();
                for (int l = j + 1; l <= k; ++l) sacc = sacc + T[j * lda + l] * w[l];
                double2 d = T[j * lda + j] - lam;
                if (cabs1(d) < smin) d = make_double2(smin, 0.0);
                w[j] = -(rcp_fp64(cabs2(d)) * (sacc * conj_(d)));
                if (cabs1(w[j]) > 1e150) {
                    for (int l = j; l <= k; ++l) w[l] = 1e-150 * w[l];
                }
            }
        } else {
            for (int j = k + 1; j < n; ++j) {
                double2 sacc = czero();
                for (int l = k; l < j; ++l) sacc = sacc + w[l] * T[l * lda + j];
                double2 d = T[j * lda + j] - lam;
                if (cabs1(d) < smin) d = make_double2(smin, 0.0);
                w[j] = -(rcp_fp64(cabs2(d)) * (sacc * conj_(d)));
                if (cabs1(w[j]) > 1e150) {
                    for (int l = k; l <= j; ++l) w[l] = 1e-150 * w[l];
                }
            }
        }
    }
    __syncthreads();
    // Y = Q y', Z = Q conj(w)
    for (int e = tid; e < 2 * n * nsel; e += blockDim.x) {
        const bool left = e >= n * nsel;
        const int ee = left ? e - n * nsel : e;
        const int row = ee / nsel, i = ee % nsel;
        const double2* w = (left ? W2 : W1) + (size_t)i * n;
        double2 acc = czero();
        for (int l = 0; l < n; ++l) acc = acc + Q[row * lda + l] * (left ? conj_(w[l]) : w[l]);
        (left ? Z : Y)[row * ldyz + i] = acc;
    }
    __syncthreads();
    // Normalise: ||y|| = 1, largest entry real positive, z^H y = 1.
    for (int i = tid; i < nsel; i += blockDim.x) {
        double nrm2 = 0.0, best = -1.0;
        int arg = 0;
        for (int r = 0; r < n; ++r) {
            double a2 = cabs2(Y[r * ldyz + i]);
            nrm2 += a2;
            if (a2 > best) { best = a2; arg = r; }
        }
        double nrm = sqrt(nrm2);
        double2 pk = Y[arg * ldyz + i];
        double apk = cabs_(pk);
        // factor = conj(pk)/|pk| / nrm
        double2 f = (apk > 0.0 && nrm > 0.0) ? (1.0 / (apk * nrm)) * conj_(pk) : make_double2(nrm > 0.0 ? 1.0 / nrm : 1.0, 0.0);
        double2 d = czero();
        for (int r = 0; r < n; ++r) {
            double2 yv = f * Y[r * ldyz + i];
            Y[r * ldyz + i] = yv;
            d = d + cdot(Z[r * ldyz + i], yv);
        }
        double2 g = cabs2(d) > 0.0 ? cdiv(cone(), conj_(d)) : cone();
        for (int r = 0; r < n; ++r) Z[r * ldyz + i] = g * Z[r * ldyz + i];
    }
    __syncthreads();
}

// Full eigen-solve of the n x n matrix in A (shared). Outputs sorted
// eigenvalues to lam (n), and vectors for the first nsel.
__device__ int eig_block(double2* A, double2* Q, int n, int lda, int nsel, double2* lam, double2* Y,
                         double2* Z, int ldyz, double2* W1, double2* W2, double2* v, double* sh, int* ord,
                         bool dfloat = false) {
    int fail = dfloat ? schur_df(A, Q, n, lda, v, sh) : schur(A, Q, n, lda, v, sh);
    double anorm = sh[4];
    order_eigs(A, n, lda, ord);
    for (int i = threadIdx.x; i < n; i += blockDim.x) lam[i] = A[ord[i] * lda + ord[i]];
    __syncthreads();
    if (nsel > 0) eigvecs(A, Q, n, lda, ord, nsel, Y, Z, ldyz, W1, W2, anorm);
    return fail;
}

// Dynamic shared memory layout for an eigen CTA of capacity nmax.
struct EigSmem {
    double2* A; double2* Q; double2* v; double* sh; int* ord;
    __device__ EigSmem(char* base, int nmax) {
        A = reinterpret_cast<double2*>(base);
        Q = A + nmax * nmax;
        v = Q + nmax * nmax;
        sh = reinterpret_cast<double*>(v + nmax);
        ord = reinterpret_cast<int*>(sh + 8);
    }
    static size_t bytes(int nmax) {
        return (size_t)(2 * nmax * nmax + nmax) * sizeof(double2) + 8 * sizeof(double) + nmax * sizeof(int) + 16;
    }
};

__global__ void __launch_bounds__(ET) small_eig_kernel(int n, const double2* Ain, int lda_in, int nsel,
                                                       double2* lam, double2* Y, double2* Z, int ldyz,
                                                       double2* W, int* info) {
    extern __shared__ __align__(16) char smem[];
    EigSmem S(smem, n);
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) S.A[e] = Ain[(e / n) * lda_in + (e % n)];
    __syncthreads();
    int fail = eig_block(S.A, S.Q, n, n, nsel, lam, Y, Z, ldyz, W, W + (size_t)n * max(nsel, 1), S.v, S.sh, S.ord);
    if (threadIdx.x == 0 && info) *info = fail;
}

// ------------------------------------------------------- BiCG-eigen (coeffs)
// Work arrays (global, per problem) for the restart coefficient computation.
struct RestartWork {
    double2 *y1, *z1, *y2, *z2, *HY, *T, *u, *q, *W1, *W2, *lamtmp, *lamtmp2, *M;
    int *rowp, *colp;
    static size_t elems(int m, int nev) {
        const int r = 2 * nev;
        return (size_t)m * nev * 4 + (size_t)m * r + (size_t)r * r * 3 + (size_t)m * m * 2 + 2 * m + (size_t)nev * nev + 64;
    }
    __device__ RestartWork(double2* base, int m, int nev) {
        const int r = 2 * nev;
        y1 = base; z1 = y1 + m * nev; y2 = z1 + m * nev; z2 = y2 + m * nev;
        HY = z2 + m * nev; T = HY + m * r; u = T + r * r; q = u + r * r;
        W1 = q + r * r; W2 = W1 + m * m; lamtmp = W2 + m * m; lamtmp2 = lamtmp + m; M = lamtmp2 + m;
        rowp = reinterpret_cast<int*>(M + nev * nev);
        colp = rowp + 32;
    }
};

// Algorithm BiCG-eigen in coefficient space, first part: which = 0 computes
// eig(H^(m)) -> y1, z1 (nev smallest); which = 1 computes eig(H^(m-1)) -> y2, z2,
// padded with a zero row. The two parts use disjoint scratch, so two CTAs can
// run them at the same time.
__device__ int restart_eigs_part(const double2* H, int ldh, int m, int nev, int which, EigSmem& S,
                                 RestartWork& Wk) {
    const int tid = threadIdx.x;
    const int n = which ? m - 1 : m;
    for (int e = tid; e < n * n; e += blockDim.x) S.A[e] = H[(e / n) * ldh + (e % n)];
    __syncthreads();
    double2* scratch = which ? Wk.W2 : Wk.W1;   // 2 n nev <= m^2
    int fail = eig_block(S.A, S.Q, n, n, nev, which ? Wk.lamtmp2 : Wk.lamtmp, which ? Wk.y2 : Wk.y1,
                         which ? Wk.z2 : Wk.z1, nev, scratch, scratch + (size_t)n * nev, S.v, S.sh, S.ord, true);
    if (which)
        for (int i = tid; i < nev; i += blockDim.x) { Wk.y2[(m - 1) * nev + i] = czero(); Wk.z2[(m - 1) * nev + i] = czero(); }
    __syncthreads();
    return fail;
}

// Second part: bi-orthogonalize, T = zt^H H yt, eig(T), Yc = yt u, Zc = zt q.
// Writes Yc, Zc (m x r, ld = ldc), lam (r); returns r.
__device__ int restart_finish_part(const double2* H, int ldh, int m, int nev, double2* Yc, double2* Zc, int ldc,
                                   double2* lam, EigSmem& S, RestartWork& Wk, int* fail_out) {
    const int tid = threadIdx.x;
    int fail = 0;
    // 3. y2 -= y1 (z1^H y2), z2 -= z1 (y1^H z2)   (coefficients in S.A as scratch)
    double2* G1 = S.A;                 // nev x nev : z1^H y2
    double2* G2 = S.A + nev * nev;     // nev x nev : y1^H z2
    for (int e = tid; e < 2 * nev * nev; e += blockDim.x) {
        const bool second = e >= nev * nev;
        const int ee = second ? e - nev * nev : e;
        const int i = ee / nev, j = ee % nev;
        const double2* L = second ? Wk.y1 : Wk.z1;
        const double2* R = second ? Wk.z2 : Wk.y2;
        double2 acc = czero();
        for (int r = 0; r < m; ++r) acc = acc + cdot(L[r * nev + i], R[r * nev + j]);
        (second ? G2 : G1)[i * nev + j] = acc;
    }
    __syncthreads();
    for (int e = tid; e < 2 * m * nev; e += blockDim.x) {
        const bool second = e >= m * nev;
        const int ee = second ? e - m * nev : e;
        const int r = ee / nev, j = ee % nev;
        const double2* B = second ? Wk.z1 : Wk.y1;
        const double2* G = second ? G2 : G1;
        double2 acc = czero();
        for (int i = 0; i < nev; ++i) acc = acc + B[r * nev + i] * G[i * nev + j];
        double2* X = second ? Wk.z2 : Wk.y2;
        X[r * nev + j] = X[r * nev + j] - acc;
    }
    __syncthreads();
    // 4. M = z2^H y2, LU with complete pivoting (thread 0), rank by pivot >= 1e-10
    for (int e = tid; e < nev * nev; e += blockDim.x) {
        const int i = e / nev, j = e % nev;
        double2 acc = czero();
        for (int r = 0; r < m; ++r) acc = acc + cdot(Wk.z2[r * nev + i], Wk.y2[r * nev + j]);
        Wk.M[i * nev + j] = acc;
    }
    __syncthreads();
    __shared__ int s_rank;
    if (tid == 0) {
        double2* a = Wk.M;
        int rank = 0;
        for (int i = 0; i < nev; ++i) { Wk.rowp[i] = i; Wk.colp[i] = i; }
        for (int i = 0; i < nev; ++i) {
            double best = -1.0; int pr = i, pc = i;
            for (int r = i; r < nev; ++r)
                for (int c = i; c < nev; ++c) {
                    double v = cabs2(a[r * nev + c]);
                    if (v > best) { best = v; pr = r; pc = c; }
                }
            if (best < 1e-20) break;   // |pivot| < 1e-10
            if (pr != i) {
                for (int c = 0; c < nev; ++c) { double2 t = a[i * nev + c]; a[i * nev + c] = a[pr * nev + c]; a[pr * nev + c] = t; }
                int t = Wk.rowp[i]; Wk.rowp[i] = Wk.rowp[pr]; Wk.rowp[pr] = t;
            }
            if (pc != i) {
                for (int r = 0; r < nev; ++r) { double2 t = a[r * nev + i]; a[r * nev + i] = a[r * nev + pc]; a[r * nev + pc] = t; }
                int t = Wk.colp[i]; Wk.colp[i] = Wk.colp[pc]; Wk.colp[pc] = t;
            }
            for (int r = i + 1; r < nev; ++r) a[r * nev + i] = cdiv(a[r * nev + i], a[i * nev + i]);
            for (int r = i + 1; r < nev; ++r)
                for (int c = i + 1; c < nev; ++c) a[r * nev + c] = a[r * nev + c] - a[r * nev + i] * a[i * nev + c];
            ++rank;
        }
        s_rank = rank;
    }
    __syncthreads();
    const int rank = s_rank;
    const int r = nev + rank;
    // 5. yt = [y1, y2(:,colp) U^{-1}], zt = [z1, z2(:,rowp) L^{-H}]  (in HY/W1 as m x r arrays)
    double2* yt = Wk.W1;   // m x r (ld r)
    double2* zt = Wk.W2;
    for (int e = tid; e < m * nev; e += blockDim.x) {
        const int row = e / nev, i = e % nev;
        yt[row * r + i] = Wk.y1[row * nev + i];
        zt[row * r + i] = Wk.z1[row * nev + i];
    }
    for (int row = tid; row < 2 * m; row += blockDim.x) {
        const bool zs = row >= m;
        const int rr = zs ? row - m : row;
        double2* out = (zs ? zt : yt) + rr * r + nev;
        const double2* in = (zs ? Wk.z2 : Wk.y2) + rr * nev;
        for (int j = 0; j < rank; ++j) {
            double2 acc = in[zs ? Wk.rowp[j] : Wk.colp[j]];
            for (int i = 0; i < j; ++i) {
                if (!zs) acc = acc - out[i] * Wk.M[i * nev + j];            // U_{ij}
                else acc = acc - out[i] * conj_(Wk.M[j * nev + i]);         // conj(L_{ji})
            }
            out[j] = zs ? acc : cdiv(acc, Wk.M[j * nev + j]);
        }
    }
    __syncthreads();
    // 6. T = zt^H H yt (r x r)
    for (int e = tid; e < m * r; e += blockDim.x) {
        const int row = e / r, j = e % r;
        double2 acc = czero();
        for (int l = 0; l < m; ++l) acc = acc + H[row * ldh + l] * yt[l * r + j];
        Wk.HY[row * r + j] = acc;
    }
    __syncthreads();
    for (int e = tid; e < r * r; e += blockDim.x) {
        const int i = e / r, j = e % r;
        double2 acc = czero();
        for (int l = 0; l < m; ++l) acc = acc + cdot(zt[l * r + i], Wk.HY[l * r + j]);
        S.A[e] = acc;
    }
    __syncthreads();
    // 7. eig(T): all r pairs -> u, q, lam
    fail |= eig_block(S.A, S.Q, r, r, r, lam, Wk.u, Wk.q, r, Wk.T, Wk.HY, S.v, S.sh, S.ord);
    // 8. Yc = yt u, Zc = zt q
    for (int e = tid; e < 2 * m * r; e += blockDim.x) {
        const bool zs = e >= m * r;
        const int ee = zs ? e - m * r : e;
        const int row = ee / r, j = ee % r;
        const double2* X = zs ? zt : yt;
        const double2* C = zs ? Wk.q : Wk.u;
        double2 acc = czero();
        for (int l = 0; l < r; ++l) acc = acc + X[row * r + l] * C[l * r + j];
        (zs ? Zc : Yc)[row * ldc + j] = acc;
    }
    __syncthreads();
    *fail_out = fail;
    return r;
}

__global__ void __launch_bounds__(ET) restart_single_kernel(int m, int nev, const double2* H, int* r_out,
                                                            double2* Yc, double2* Zc, double2* lam,
                                                            double2* work, int* info) {
    extern __shared__ __align__(16) char smem[];
    EigSmem S(smem, m);
    RestartWork Wk(work, m, nev);
    int fail = restart_eigs_part(H, m, m, nev, 0, S, Wk);
    fail |= restart_eigs_part(H, m, m, nev, 1, S, Wk);
    int f2 = 0;
    int r = restart_finish_part(H, m, m, nev, Yc, Zc, 2 * nev, lam, S, Wk, &f2);
    if (threadIdx.x == 0) { *r_out = r; *info = fail | f2; }
}

// Restart of every slot whose window is full (vs == m), in two kernels: the two
// eigen-solves (one CTA each, grid (nslots, 2)), then the rest (one CTA per
// slot): coefficients and H = diag(lam).
__global__ void __launch_bounds__(ET) restart_eigs_kernel(SlotState* states, const SlotPtrs* ptrs,
                                                          double2* work_base, size_t work_stride, int* fails) {
    const SlotState& st = states[blockIdx.x];
    const SlotPtrs& P = ptrs[blockIdx.x];
    if (!(st.status == ST_RUNNING && st.m > 0 && st.vs == st.m)) return;
    extern __shared__ __align__(16) char smem[];
    const int m = st.m, nev = st.nev;
    EigSmem S(smem, m);
    RestartWork Wk(work_base + work_stride * blockIdx.x, m, nev);
    int fail = restart_eigs_part(P.H, m, m, nev, blockIdx.y, S, Wk);
    if (threadIdx.x == 0) fails[2 * blockIdx.x + blockIdx.y] = fail;
}

__global__ void __launch_bounds__(ET) restart_slots_kernel(SlotState* states, const SlotPtrs* ptrs,
                                                           double2* work_base, size_t work_stride, const int* fails) {
    SlotState& st = states[blockIdx.x];
    const SlotPtrs& P = ptrs[blockIdx.x];
    __shared__ int go;
    if (threadIdx.x == 0) {
        go = (st.status == ST_RUNNING && st.m > 0 && st.vs == st.m);
        if (!go) st.restart_r = 0;
    }
    __syncthreads();
    if (!go) return;
    extern __shared__ __align__(16) char smem[];
    const int m = st.m, nev = st.nev;
    EigSmem S(smem, m);
    RestartWork Wk(work_base + work_stride * blockIdx.x, m, nev);
    const int ldc = 2 * nev + 1;
    int fail = 0;
    int r = restart_finish_part(P.H, m, m, nev, P.coefY, P.coefZ, ldc, P.lam, S, Wk, &fail);
    fail |= fails[2 * blockIdx.x] | fails[2 * blockIdx.x + 1];
    // H = diag(lam)
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        const int i = e / m, j = e % m;
        P.H[e] = (i == j && i < r) ? P.lam[i] : czero();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (fail) st.status = ST_BREAKDOWN;
        st.restart_r = r;
        st.vs = r;
        st.restarts += 1;
    }
}

// Final Ritz pairs of a window: eig(H^(vs)), nev smallest, scales folded.
// Block j: slot slot0 + j, outputs at Yc + j ostride, Zc + j ostride, lam + j lstride,
// nout[j], work area work + j wstride (the windows' final Ritz pairs of several
// slots at once: each depends only on its own window).
__global__ void __launch_bounds__(ET) final_ritz_kernel(SlotState* states, const SlotPtrs* ptrs, int slot0,
                                                        double2* Yc, double2* Zc, double2* lam, int* nout,
                                                        double2* work, size_t ostride, size_t lstride,
                                                        size_t wstride) {
    const int slot = slot0 + blockIdx.x;
    Yc += blockIdx.x * ostride;
    Zc += blockIdx.x * ostride;
    lam += blockIdx.x * lstride;
    nout += blockIdx.x;
    work += blockIdx.x * wstride;
    const SlotState& st = states[slot];
    const SlotPtrs& P = ptrs[slot];
    const int n = st.vs, m = st.m;
    const int nsel = min(st.nev, n);
    if (n == 0) { if (threadIdx.x == 0) *nout = 0; return; }
    extern __shared__ __align__(16) char smem[];
    EigSmem S(smem, n);
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) S.A[e] = P.H[(e / n) * m + (e % n)];
    __syncthreads();
    eig_block(S.A, S.Q, n, n, nsel, lam, Yc, Zc, nsel, work, work + (size_t)n * nsel, S.v, S.sh, S.ord);
    for (int e = threadIdx.x; e < n * nsel; e += blockDim.x) {
        const int row = e / nsel;
        Yc[e] = P.vscale[row] * Yc[e];
        Zc[e] = P.wscale[row] * Zc[e];
    }
    if (threadIdx.x == 0) *nout = nsel;
}

// LU with partial pivoting, one CTA.
__global__ void lu_factor_kernel(int n, double2* A, int lda, int* piv, int* info) {
    __shared__ int s_p;
    __shared__ int s_bad;
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (threadIdx.x == 0) {
            int p = k; double best = -1.0;
            for (int i = k; i < n; ++i) { double v = cabs2(A[i * lda + k]); if (v > best) { best = v; p = i; } }
            s_p = p; piv[k] = p;
            if (best == 0.0) s_bad = 1;
        }
        __syncthreads();
        const int p = s_p;
        if (p != k)
            for (int j = threadIdx.x; j < n; j += blockDim.x) {
                double2 t = A[k * lda + j]; A[k * lda + j] = A[p * lda + j]; A[p * lda + j] = t;
            }
        __syncthreads();
        const double2 d = A[k * lda + k];
        if (cabs2(d) > 0.0)
            for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) A[i * lda + k] = cdiv(A[i * lda + k], d);
        __syncthreads();
        for (int e = threadIdx.x; e < (n - k - 1) * (n - k - 1); e += blockDim.x) {
            const int i = k + 1 + e / (n - k - 1), j = k + 1 + e % (n - k - 1);
            A[i * lda + j] = A[i * lda + j] - A[i * lda + k] * A[k * lda + j];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && info) *info = s_bad;
}

// Solve with the LU factors; one thread per right-hand-side column.
__global__ void lu_solve_kernel(int n, const double2* LU, int lda, const int* piv, int trans, int nrhs,
                                double2* B, int ldb) {
    for (int c = threadIdx.x; c < nrhs; c += blockDim.x) {
        if (!trans) {
            for (int k = 0; k < n; ++k) {   // P
                int p = piv[k];
                if (p != k) { double2 t = B[k * ldb + c]; B[k * ldb + c] = B[p * ldb + c]; B[p * ldb + c] = t; }
            }
            for (int i = 0; i < n; ++i) {   // L y = b
                double2 acc = B[i * ldb + c];
                for (int j = 0; j < i; ++j) acc = acc - LU[i * lda + j] * B[j * ldb + c];
                B[i * ldb + c] = acc;
            }
            for (int i = n - 1; i >= 0; --i) {   // U x = y
                double2 acc = B[i * ldb + c];
                for (int j = i + 1; j < n; ++j) acc = acc - LU[i * lda + j] * B[j * ldb + c];
                B[i * ldb + c] = cdiv(acc, LU[i * lda + i]);
            }
        } else {
            // A^H x = b with P A = L U:  A^H = U^H L^H P  ->  U^H y = b, L^H w = y, x = P^T w
            for (int i = 0; i < n; ++i) {
                double2 acc = B[i * ldb + c];
                for (int j = 0; j < i; ++j) acc = acc - conj_(LU[j * lda + i]) * B[j * ldb + c];
                B[i * ldb + c] = cdiv(acc, conj_(LU[i * lda + i]));
            }
            for (int i = n - 1; i >= 0; --i) {
                double2 acc = B[i * ldb + c];
                for (int j = i + 1; j < n; ++j) acc = acc - conj_(LU[j * lda + i]) * B[j * ldb + c];
                B[i * ldb + c] = acc;
            }
            for (int k = n - 1; k >= 0; --k) {
                int p = piv[k];
                if (p != k) { double2 t = B[k * ldb + c]; B[k * ldb + c] = B[p * ldb + c]; B[p * ldb + c] = t; }
            }
        }
    }
}

// One factor of P A = L U applied to B (n x nrhs, or nrows x n for LU_RIGHT_U),
// one thread per column (per row for LU_RIGHT_U):
//   LU_LEFT_PL : B <- L^{-1} P B        LU_LEFT_U : B <- U^{-1} B
//   LU_RIGHT_U : B <- B U^{-1}          LU_LEFT_LH: B <- P^T L^{-H} B
__global__ void lu_part_kernel(int n, const double2* LU, int lda, const int* piv, int part, int ncols, double2* B,
                               int ldb) {
    for (int c = threadIdx.x; c < ncols; c += blockDim.x) {
        if (part == LU_LEFT_PL) {
            for (int k = 0; k < n; ++k) {
                const int p = piv[k];
                if (p != k) { double2 t = B[k * ldb + c]; B[k * ldb + c] = B[p * ldb + c]; B[p * ldb + c] = t; }
            }
            for (int i = 0; i < n; ++i) {
                double2 acc = B[i * ldb + c];
                for (int j = 0; j < i; ++j) acc = acc - LU[i * lda + j] * B[j * ldb + c];
                B[i * ldb + c] = acc;
            }
        } else if (part == LU_LEFT_U) {
            for (int i = n - 1; i >= 0; --i) {
                double2 acc = B[i * ldb + c];
                for (int j = i + 1; j < n; ++j) acc = acc - LU[i * lda + j] * B[j * ldb + c];
                B[i * ldb + c] = cdiv(acc, LU[i * lda + i]);
            }
        } else if (part == LU_RIGHT_U) {   // row c: x U = b, x_j = (b_j - sum_{i<j} x_i U_ij) / U_jj
            double2* row = B + (size_t)c * ldb;
            for (int j = 0; j < n; ++j) {
                double2 acc = row[j];
                for (int i = 0; i < j; ++i) acc = acc - row[i] * LU[i * lda + j];
                row[j] = cdiv(acc, LU[j * lda + j]);
            }
        } else {   // LU_LEFT_LH: L^H w = b (unit upper), then x = P^T w
            for (int i = n - 1; i >= 0; --i) {
                double2 acc = B[i * ldb + c];
                for (int j = i + 1; j < n; ++j) acc = acc - conj_(LU[j * lda + i]) * B[j * ldb + c];
                B[i * ldb + c] = acc;
            }
            for (int k = n - 1; k >= 0; --k) {
                const int p = piv[k];
                if (p != k) { double2 t = B[k * ldb + c]; B[k * ldb + c] = B[p * ldb + c]; B[p * ldb + c] = t; }
            }
        }
    }
}

// Rank-revealing selection on a small square block B (n <= 32, row-major, ld):
// LU with complete pivoting on a copy, stopped at the first pivot below
// tau * |first pivot|. out[0] = r (pivots kept), out[1 + i] = row index of pivot
// i, out[1 + n + i] = its column index (i < r). One thread.
__global__ void pivot_select_kernel(int n, const double2* B, int ld, double tau, int* out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double2 a[32][32];
    int rows[32], cols[32];
    for (int i = 0; i < n; ++i) {
        rows[i] = cols[i] = i;
        for (int j = 0; j < n; ++j) a[i][j] = B[i * ld + j];
    }
    double p0 = 0.0;
    int r = 0;
    for (int k = 0; k < n; ++k) {
        int pi = k, pj = k;
        double best = -1.0;
        for (int i = k; i < n; ++i)
            for (int j = k; j < n; ++j) {
                const double v = cabs2(a[i][j]);
                if (v > best) { best = v; pi = i; pj = j; }
            }
        best = sqrt(best);
        if (k == 0) p0 = best;
        if (!(best > tau * p0) || best == 0.0) break;
        if (pi != k) {
            for (int j = 0; j < n; ++j) { double2 t = a[k][j]; a[k][j] = a[pi][j]; a[pi][j] = t; }
            int t = rows[k]; rows[k] = rows[pi]; rows[pi] = t;
        }
        if (pj != k) {
            for (int i = 0; i < n; ++i) { double2 t = a[i][k]; a[i][k] = a[i][pj]; a[i][pj] = t; }
            int t = cols[k]; cols[k] = cols[pj]; cols[pj] = t;
        }
        for (int i = k + 1; i < n; ++i) {
            const double2 l = cdiv(a[i][k], a[k][k]);
            for (int j = k + 1; j < n; ++j) a[i][j] = a[i][j] - l * a[k][j];
        }
        r = k + 1;
    }
    out[0] = r;
    for (int i = 0; i < n; ++i) { out[1 + i] = rows[i]; out[1 + n + i] = cols[i]; }
}

__global__ void small_gemm_kernel(int n, int k, int m, const double2* A, int lda, int transA,
                                  const double2* B, int ldb, double2* C, int ldc) {
    for (int e = threadIdx.x + blockIdx.x * blockDim.x; e < n * m; e += blockDim.x * gridDim.x) {
        const int i = e / m, j = e % m;
        double2 acc = czero();
        for (int l = 0; l < k; ++l) {
            double2 a = transA ? conj_(A[l * lda + i]) : A[i * lda + l];
            acc = acc + a * B[l * ldb + j];
        }
        C[i * ldc + j] = acc;
    }
}

}  // namespace

// ------------------------------------------------------------------ launchers
static cudaError_t set_smem(const void* fn, size_t bytes) {
    if (bytes > 48 * 1024) return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    return cudaSuccess;
}

cudaError_t prepare_eig_kernels() {
    cudaError_t e;
    if ((e = set_smem((const void*)small_eig_kernel, EigSmem::bytes(MAX_SMALL))) != cudaSuccess) return e;
    if ((e = set_smem((const void*)restart_single_kernel, EigSmem::bytes(MAX_M))) != cudaSuccess) return e;
    if ((e = set_smem((const void*)restart_slots_kernel, EigSmem::bytes(MAX_M))) != cudaSuccess) return e;
    if ((e = set_smem((const void*)restart_eigs_kernel, EigSmem::bytes(MAX_M))) != cudaSuccess) return e;
    return set_smem((const void*)final_ritz_kernel, EigSmem::bytes(MAX_M));
}

size_t eig_work_elems() {
    size_t a = RestartWork::elems(MAX_M, MAX_M / 2);
    size_t b = (size_t)2 * MAX_SMALL * MAX_SMALL + 16;
    return a > b ? a : b;
}

cudaError_t launch_small_eig(int n, const double2* A, int lda, int nsel, double2* lam, double2* Y, double2* Z,
                             int ldyz, int* info, double2* w, cudaStream_t st) {
    if (n < 1 || n > MAX_SMALL) return cudaErrorInvalidValue;
    // The kernel's shared-memory limit is only ever set to the largest size
    // (bytes(MAX_SMALL)); a smaller per-call value would lower it for every
    // other caller of this kernel, including the allocation-free entry point.
    cudaError_t e = set_smem((const void*)small_eig_kernel, EigSmem::bytes(MAX_SMALL));
    if (e != cudaSuccess) return e;
    const size_t sm = EigSmem::bytes(n);
    small_eig_kernel<<<1, ET, sm, st>>>(n, A, lda, nsel, lam, Y, Z, ldyz, w, info);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_restart_coeffs_single(int m, int nev, const double2* H, int* r, double2* Yc, double2* Zc,
                                         double2* lam, int* info, double2* w, cudaStream_t st) {
    if (m < 3 || m > MAX_M || 2 * nev >= m || nev < 1) return cudaErrorInvalidValue;
    const size_t sm = EigSmem::bytes(m);
    cudaError_t e = set_smem((const void*)restart_single_kernel, EigSmem::bytes(MAX_M));   // never lowered
    if (e != cudaSuccess) return e;
    restart_single_kernel<<<1, ET, sm, st>>>(m, nev, H, r, Yc, Zc, lam, w, info);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_restart_coeffs(SlotState* states, const SlotPtrs* ptrs, int nslots, double2* w,
                                  cudaStream_t st) {
    // Per-slot work stride: capacity for the largest window; the dynamic shared
    // memory opt-in is done once by prepare_eig_kernels (this launcher runs under
    // graph capture).
    const size_t stride = eig_work_elems();
    int* fails = reinterpret_cast<int*>(w + stride * MAX_SLOTS);   // 2 ints per slot after the slot work areas
    size_t sm = EigSmem::bytes(MAX_M);
    restart_eigs_kernel<<<dim3(nslots, 2), ET, sm, st>>>(states, ptrs, w, stride, fails);
    restart_slots_kernel<<<nslots, ET, sm, st>>>(states, ptrs, w, stride, fails);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_final_ritz(SlotState* states, const SlotPtrs* ptrs, int slot, double2* Yc, double2* Zc,
                              double2* lam, int* nout, double2* w, cudaStream_t st) {
    return launch_final_ritz_slots(states, ptrs, slot, 1, Yc, Zc, lam, nout, 0, 0, w, st);
}

cudaError_t launch_final_ritz_slots(SlotState* states, const SlotPtrs* ptrs, int slot0, int nslots, double2* Yc,
                                    double2* Zc, double2* lam, int* nout, size_t ostride, size_t lstride,
                                    double2* w, cudaStream_t st) {
    if (nslots < 1 || nslots > MAX_SLOTS) return cudaErrorInvalidValue;
    size_t sm = EigSmem::bytes(MAX_M);
    final_ritz_kernel<<<nslots, ET, sm, st>>>(states, ptrs, slot0, Yc, Zc, lam, nout, w, ostride, lstride,
                                              eig_work_elems());
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_lu_factor(int n, double2* A, int lda, int* piv, int* info, cudaStream_t st) {
    lu_factor_kernel<<<1, 256, 0, st>>>(n, A, lda, piv, info);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_lu_solve(int n, const double2* LU, int lda, const int* piv, int trans, int nrhs, double2* B,
                            int ldb, cudaStream_t st) {
    lu_solve_kernel<<<1, 128, 0, st>>>(n, LU, lda, piv, trans, nrhs, B, ldb);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_lu_part(int n, const double2* LU, int lda, const int* piv, int part, int ncols, double2* B,
                           int ldb, cudaStream_t st) {
    lu_part_kernel<<<1, 128, 0, st>>>(n, LU, lda, piv, part, ncols, B, ldb);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_pivot_select(int n, const double2* B, int ld, double tau, int* out, cudaStream_t st) {
    if (n < 1 || n > 32) return cudaErrorInvalidValue;
    pivot_select_kernel<<<1, 32, 0, st>>>(n, B, ld, tau, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_small_gemm(int n, int k, int m, const double2* A, int lda, int transA, const double2* B,
                              int ldb, double2* C, int ldc, cudaStream_t st) {
    int blocks = (n * m + 255) / 256;
    if (blocks < 1) blocks = 1;
    small_gemm_kernel<<<blocks, 256, 0, st>>>(n, k, m, A, lda, transA, B, ldb, C, ldc);
    count_launches(1);
    return cudaGetLastError();
}


// ============================================================================
// Allocation-free variant of the small eigen-solver (no counterpart in the paper).
//
// lqcd_small_eig stages its operands through cudaMalloc'd buffers. Some callers
// cannot allocate device memory at the point where they need an eigen-solve:
// host applications that hand all device memory to their own pool or fixed
// budget up front, and latency-critical loops where the implicit device
// synchronisation of cudaMalloc/cudaFree would stall work on other streams.
// lqcd_small_eig_noalloc takes device pointers for the input and every output
// and keeps its scratch (the substitution vectors and a status word) in the
// file-scope device array below: at most NOALLOC_MAX_N = 80, i.e. 2*80*80 + 16
// complex doubles (about 200 KiB), held by every GPU that loads the library
// until the process exits. The array is shared by all calls on a device and
// keeps the last call's contents: the status word is cleared by each call, the
// substitution vectors are fully rewritten before they are read. Calls whose
// kernels overlap on the GPU (different streams, or host threads) race on it.
// The per-device set-up (the array's address, the shared-memory limit) is kept
// for the life of the process: a cudaDeviceReset between calls is not supported.
// Every other launcher of the same kernel keeps its shared-memory limit at the
// maximum, so no other call can lower it below what this entry point needs.
namespace {

constexpr int NOALLOC_MAX_N = MAX_SMALL;
constexpr size_t NOALLOC_SCRATCH = (size_t)2 * NOALLOC_MAX_N * NOALLOC_MAX_N;

static __device__ __align__(256) double2 g_noalloc_scratch[NOALLOC_SCRATCH + 16];

struct NoAllocSetup {
    bool ready = false;
    double2* scratch = nullptr;   // device address of g_noalloc_scratch on this device
};
constexpr int NOALLOC_MAX_DEVICES = 64;
NoAllocSetup g_noalloc_dev[NOALLOC_MAX_DEVICES];
std::mutex g_noalloc_mutex;

// Once per device, with that device current: the array's device address and the
// kernel's shared-memory opt-in.
cudaError_t noalloc_setup(int dev, double2** scratch) {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    NoAllocSetup& d = g_noalloc_dev[dev];
    if (!d.ready) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        e = set_smem((const void*)small_eig_kernel, EigSmem::bytes(NOALLOC_MAX_N));
        if (e != cudaSuccess) return e;
        d.scratch = reinterpret_cast<double2*>(p);
        d.ready = true;
    }
    *scratch = d.scratch;
    return cudaSuccess;
}

}  // namespace
}  // namespace lqcd

extern "C" lqcd_status lqcd_small_eig_noalloc(int n, const double* C, double* evals, double* Y, double* Z,
                                              void* stream) {
    using namespace lqcd;
    if (n < 1 || n > NOALLOC_MAX_N || !C || !evals || (Y == nullptr) != (Z == nullptr)) return LQCD_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) return LQCD_ERR_CUDA;
    double2* scratch = nullptr;
    if (noalloc_setup(dev, &scratch) != cudaSuccess) return LQCD_ERR_CUDA;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int* info = reinterpret_cast<int*>(scratch + NOALLOC_SCRATCH);
    const int nsel = Y ? n : 0;
    if (cudaMemsetAsync(info, 0, sizeof(int), st) != cudaSuccess) return LQCD_ERR_CUDA;
    (void)cudaGetLastError();   // an earlier, unrelated launch error is not this call's
    small_eig_kernel<<<1, ET, EigSmem::bytes(n), st>>>(n, reinterpret_cast<const double2*>(C), n, nsel,
                                                       reinterpret_cast<double2*>(evals), reinterpret_cast<double2*>(Y),
                                                       reinterpret_cast<double2*>(Z), n, scratch, info);
    count_launches(1);
    if (cudaPeekAtLastError() != cudaSuccess) { (void)cudaGetLastError(); return LQCD_ERR_CUDA; }
    int hinfo = 0;
    if (cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return LQCD_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return LQCD_ERR_CUDA;
    return hinfo ? LQCD_ERR_NOCONV : LQCD_OK;
}
