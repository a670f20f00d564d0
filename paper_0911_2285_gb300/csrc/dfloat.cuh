// Double-FP32 ("double-float") arithmetic for the reliable-update residual.
//
// FP64 runs at a small fraction of the FP32 rate on this GPU, so the in-iteration
// reliable updates evaluate A x in pairs of FP32 numbers: a value is the
// unevaluated sum h + l (|l| <= ulp(h)/2), about 48 significant bits. Sums use
// Knuth's two-sum, products Dekker's two-product through the fused multiply-add,
// and the SU(3) row sums are compensated dot products (Ogita, Rump and Oishi,
// "Accurate sum and dot product", SIAM J. Sci. Comput. 26 (2005), Dot2 with the
// cross terms of the low parts). The convergence certificate of a solve is
// still the native FP64 residual.
#pragma once
#include "common.cuh"

namespace lqcd {

struct dfl { float h, l; };
struct dfc { dfl x, y; };   // complex: x = real part, y = imaginary part

__device__ __forceinline__ dfl operator-(dfl a) { return {-a.h, -a.l}; }
__device__ __forceinline__ dfl operator+(dfl a, dfl b) {
    const float s = a.h + b.h, v = s - a.h;
    float e = (a.h - (s - v)) + (b.h - v);
    e += a.l + b.l;
    const float h = s + e;
    return {h, e - (h - s)};
}
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }
__device__ __forceinline__ dfc operator+(dfc a, dfc b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ dfc operator-(dfc a, dfc b) { return {a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ dfc operator-(dfc a) { return {-a.x, -a.y}; }

__device__ __forceinline__ dfl df_split(double v) {
    const float h = __double2float_rn(v);
    return {h, __double2float_rn(v - (double)h)};
}
__device__ __forceinline__ double df_value(dfl a) { return (double)a.h + (double)a.l; }

// Compensated sum of products a_i b_i: s + c, c collecting every rounding error.
struct Dot2 {
    float s, c;
    __device__ __forceinline__ void first(dfl a, dfl b) {
        s = a.h * b.h;
        float e = fmaf(a.h, b.h, -s);
        e = fmaf(a.h, b.l, e);
        c = fmaf(a.l, b.h, e);
    }
    __device__ __forceinline__ void add(dfl a, dfl b) {
        const float p = a.h * b.h;
        float e = fmaf(a.h, b.h, -p);
        e = fmaf(a.h, b.l, e);
        e = fmaf(a.l, b.h, e);
        const float s2 = s + p, bp = s2 - s;
        const float q = (s - (s2 - bp)) + (p - bp);
        s = s2;
        c += q + e;
    }
    __device__ __forceinline__ dfl done() const {
        const float h = s + c;
        return {h, c - (h - s)};
    }
};

// Link element (mu, e) of site s: float4 (h.re, h.im, l.re, l.im) in [mu][9][V].
struct LinksDF {
    const float4* u;
    int V;
    __device__ __forceinline__ void load(int mu, int s, dfc (&m)[3][3]) const {
#pragma unroll
        for (int e = 0; e < 9; ++e) {
            const float4 t = __ldg(u + (size_t)(mu * 9 + e) * V + s);
            m[e / 3][e % 3] = {{t.x, t.z}, {t.y, t.w}};
        }
    }
};

// Field in double-float form, same complex indexing as the FP64 layout.
struct FieldDF {
    const float4* p;
    int V;
    __device__ __forceinline__ void load(int s, dfc (&v)[12]) const {
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            const float4 t = __ldg(p + ((size_t)(c >> 1) * V + s) * 2 + (c & 1));
            v[c] = {{t.x, t.z}, {t.y, t.w}};
        }
    }
};

__device__ __forceinline__ void su3_mul_df(const dfc (&u)[3][3], const dfc (&h)[2][3], dfc (&o)[2][3]) {
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            Dot2 re, im;
            re.first(u[r][0].x, h[a][0].x);
            re.add(-u[r][0].y, h[a][0].y);
            im.first(u[r][0].x, h[a][0].y);
            im.add(u[r][0].y, h[a][0].x);
#pragma unroll
            for (int c = 1; c < 3; ++c) {
                re.add(u[r][c].x, h[a][c].x);
                re.add(-u[r][c].y, h[a][c].y);
                im.add(u[r][c].x, h[a][c].y);
                im.add(u[r][c].y, h[a][c].x);
            }
            o[a][r] = {re.done(), im.done()};
        }
}
__device__ __forceinline__ void su3_dag_mul_df(const dfc (&u)[3][3], const dfc (&h)[2][3], dfc (&o)[2][3]) {
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            Dot2 re, im;
            re.first(u[0][r].x, h[a][0].x);
            re.add(u[0][r].y, h[a][0].y);
            im.first(u[0][r].x, h[a][0].y);
            im.add(-u[0][r].y, h[a][0].x);
#pragma unroll
            for (int c = 1; c < 3; ++c) {
                re.add(u[c][r].x, h[a][c].x);
                re.add(u[c][r].y, h[a][c].y);
                im.add(u[c][r].x, h[a][c].y);
                im.add(-u[c][r].y, h[a][c].x);
            }
            o[a][r] = {re.done(), im.done()};
        }
}

}  // namespace lqcd
