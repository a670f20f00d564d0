// Wilson hopping term D_hop on one site, both precisions, and its adjoint.
//
//   D_hop psi(x) = sum_mu (1 - gamma_mu) U_mu(x) psi(x+mu) + (1 + gamma_mu) U_mu(x-mu)^+ psi(x-mu)
//   D_hop^+ psi(x) = sum_mu (1 + gamma_mu) U_mu(x) psi(x+mu) + (1 - gamma_mu) U_mu(x-mu)^+ psi(x-mu)
//
// (the operator of the paper's test problems, Sec. 3; the adjoint follows from
// gamma5 (1 -+ gamma_mu) gamma5 = (1 +- gamma_mu), Sec. 4).
//
// Chiral basis: gamma_mu = [[0, M_mu], [M_mu^+, 0]] with M_k = -i sigma_k, M_4 = 1.
// For a sign sg = +-1, (1 + sg gamma_mu) psi = (h, sg M^+ h) with
// h = psi_up + sg M psi_lo (two spin components of three colours), so each
// hop multiplies only the half spinor h by the link and rebuilds the lower
// half with sign/i permutations (no multiplications).
#pragma once
#include "common.cuh"

namespace lqcd {

struct LinksD {   // FP64, all 18 reals
    const double2* u;
    int V;
    __device__ __forceinline__ void load(int mu, int s, double2 (&m)[3][3]) const {
#pragma unroll
        for (int e = 0; e < 9; ++e) m[e / 3][e % 3] = __ldg(u + (size_t)(mu * 9 + e) * V + s);
    }
};

// conj(a b - c d) as two fused chains.
__device__ __forceinline__ float2 cross_conj(float2 a, float2 b, float2 c, float2 d) {
    float re = a.x * b.x;
    re = fmaf(-a.y, b.y, re);
    re = fmaf(-c.x, d.x, re);
    re = fmaf(c.y, d.y, re);
    float im = c.x * d.y;
    im = fmaf(c.y, d.x, im);
    im = fmaf(-a.x, b.y, im);
    im = fmaf(-a.y, b.x, im);
    return make_float2(re, im);
}

struct LinksF {   // FP32 rows 0, 1; row 2 rebuilt as conj(row0 x row1)
    const float4* u;
    int V;
    __device__ __forceinline__ void load(int mu, int s, float2 (&m)[3][3]) const {
        float4 a = __ldg(u + (size_t)(mu * 3 + 0) * V + s);
        float4 b = __ldg(u + (size_t)(mu * 3 + 1) * V + s);
        float4 c = __ldg(u + (size_t)(mu * 3 + 2) * V + s);
        m[0][0] = make_float2(a.x, a.y); m[0][1] = make_float2(a.z, a.w);
        m[0][2] = make_float2(b.x, b.y); m[1][0] = make_float2(b.z, b.w);
        m[1][1] = make_float2(c.x, c.y); m[1][2] = make_float2(c.z, c.w);
        m[2][0] = cross_conj(m[0][1], m[1][2], m[0][2], m[1][1]);
        m[2][1] = cross_conj(m[0][2], m[1][0], m[0][0], m[1][2]);
        m[2][2] = cross_conj(m[0][0], m[1][1], m[0][1], m[1][0]);
    }
};

template <typename T> struct LinkSel;
template <> struct LinkSel<float> { using type = LinksF; };
template <> struct LinkSel<double> { using type = LinksD; };

// h_a = psi_a + sg (M_mu psi_lo)_a, a = 0, 1; psi index = spin*3 + colour.
template <int MU, int SG, typename C>
__device__ __forceinline__ void project(const C (&psi)[12], C (&h)[2][3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        C p0 = psi[c], p1 = psi[3 + c], p2 = psi[6 + c], p3 = psi[9 + c];
        C m0, m1;
        if (MU == 0) { m0 = mul_mi(p3); m1 = mul_mi(p2); }
        else if (MU == 1) { m0 = -p3; m1 = p2; }
        else if (MU == 2) { m0 = mul_mi(p2); m1 = mul_i(p3); }
        else { m0 = p2; m1 = p3; }
        if (SG > 0) { h[0][c] = p0 + m0; h[1][c] = p1 + m1; }
        else { h[0][c] = p0 - m0; h[1][c] = p1 - m1; }
    }
}

// acc += (uh, sg M_mu^+ uh)
template <int MU, int SG, typename C>
__device__ __forceinline__ void reconstruct(const C (&uh)[2][3], C (&acc)[12]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        C a = uh[0][c], b = uh[1][c];
        C l0, l1;   // M^+ (a, b)
        if (MU == 0) { l0 = mul_i(b); l1 = mul_i(a); }
        else if (MU == 1) { l0 = b; l1 = -a; }
        else if (MU == 2) { l0 = mul_i(a); l1 = mul_mi(b); }
        else { l0 = a; l1 = b; }
        acc[c] = acc[c] + a;
        acc[3 + c] = acc[3 + c] + b;
        if (SG > 0) { acc[6 + c] = acc[6 + c] + l0; acc[9 + c] = acc[9 + c] + l1; }
        else { acc[6 + c] = acc[6 + c] - l0; acc[9 + c] = acc[9 + c] - l1; }
    }
}

// Fused multiply-add chains (one rounding per term, no separate product and
// sum instructions): o = u h and o = u^+ h for the two spin rows of h.
__device__ __forceinline__ float fma_(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return fma(a, b, c); }

template <typename C>
__device__ __forceinline__ void su3_mul(const C (&u)[3][3], const C (&h)[2][3], C (&o)[2][3]) {
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            auto re = u[r][0].x * h[a][0].x;
            auto im = u[r][0].x * h[a][0].y;
            re = fma_(-u[r][0].y, h[a][0].y, re);
            im = fma_(u[r][0].y, h[a][0].x, im);
#pragma unroll
            for (int c = 1; c < 3; ++c) {
                re = fma_(u[r][c].x, h[a][c].x, re);
                im = fma_(u[r][c].x, h[a][c].y, im);
                re = fma_(-u[r][c].y, h[a][c].y, re);
                im = fma_(u[r][c].y, h[a][c].x, im);
            }
            o[a][r].x = re;
            o[a][r].y = im;
        }
}
template <typename C>
__device__ __forceinline__ void su3_dag_mul(const C (&u)[3][3], const C (&h)[2][3], C (&o)[2][3]) {
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            auto re = u[0][r].x * h[a][0].x;
            auto im = u[0][r].x * h[a][0].y;
            re = fma_(u[0][r].y, h[a][0].y, re);
            im = fma_(-u[0][r].y, h[a][0].x, im);
#pragma unroll
            for (int c = 1; c < 3; ++c) {
                re = fma_(u[c][r].x, h[a][c].x, re);
                im = fma_(u[c][r].x, h[a][c].y, im);
                re = fma_(u[c][r].y, h[a][c].y, re);
                im = fma_(-u[c][r].y, h[a][c].x, im);
            }
            o[a][r].x = re;
            o[a][r].y = im;
        }
}

// Input accessors: in.load(site, psi) fills 12 complex values.
template <typename S> struct FieldIn {
    const void* p;
    int V;
    template <typename C> __device__ __forceinline__ void load(int s, C (&v)[12]) const { Field<S>::load(p, V, s, v); }
};
// x_hi (FP64) + x_lo (storage S), summed in FP64.
template <typename S> struct SumIn {
    const void* hi;
    const void* lo;
    int V;
    __device__ __forceinline__ void load(int s, double2 (&v)[12]) const {
        double2 a[12], b[12];
        Field<double>::load(hi, V, s, a);
        Field<S>::load(lo, V, s, b);
#pragma unroll
        for (int c = 0; c < 12; ++c) v[c] = a[c] + b[c];
    }
};

template <int MU, bool DAG, typename T, class LK, class IN>
__device__ __forceinline__ void hop_dir(const Nbr& nb, const LK& U, const IN& in, int s,
                                        cplx<T> (&acc)[12]) {
    using C = cplx<T>;
    constexpr int SF = DAG ? +1 : -1;   // forward projector sign
    C psi[12], h[2][3], uh[2][3], u[3][3];
    {
        int sf = nb.f[MU];
        in.load(sf, psi);
        project<MU, SF>(psi, h);
        U.load(MU, s, u);
        su3_mul(u, h, uh);
        reconstruct<MU, SF>(uh, acc);
    }
    {
        int sb = nb.b[MU];
        in.load(sb, psi);
        project<MU, -SF>(psi, h);
        U.load(MU, sb, u);
        su3_dag_mul(u, h, uh);
        reconstruct<MU, -SF>(uh, acc);
    }
}

// acc = D_hop psi (DAG = false) or D_hop^+ psi (DAG = true) at site s.
template <bool DAG, typename T, class LK, class IN>
__device__ __forceinline__ void hop_site(const Geom& g, const LK& U, const IN& in, int s,
                                         cplx<T> (&acc)[12]) {
    const Nbr nb(g, s);
#pragma unroll
    for (int c = 0; c < 12; ++c) acc[c] = mk<T>(T(0), T(0));
    hop_dir<0, DAG, T>(nb, U, in, s, acc);
    hop_dir<1, DAG, T>(nb, U, in, s, acc);
    hop_dir<2, DAG, T>(nb, U, in, s, acc);
    hop_dir<3, DAG, T>(nb, U, in, s, acc);
}

// Both operators of a BiCG pair at one site, sharing every link load:
// a = D_hop p (projectors 1 -+ gamma), b = D_hop^+ phat (projectors 1 +- gamma).
template <int MU, typename T, class LK, class IN>
__device__ __forceinline__ void hop_dir_pair(const Nbr& nb, const LK& U, const IN& inp, const IN& inh, int s,
                                             cplx<T> (&a)[12], cplx<T> (&b)[12]) {
    using C = cplx<T>;
    C psi[12], h[2][3], uh[2][3], u[3][3];
    U.load(MU, s, u);
    inp.load(nb.f[MU], psi);
    project<MU, -1>(psi, h);
    su3_mul(u, h, uh);
    reconstruct<MU, -1>(uh, a);
    inh.load(nb.f[MU], psi);
    project<MU, +1>(psi, h);
    su3_mul(u, h, uh);
    reconstruct<MU, +1>(uh, b);
    U.load(MU, nb.b[MU], u);
    inp.load(nb.b[MU], psi);
    project<MU, +1>(psi, h);
    su3_dag_mul(u, h, uh);
    reconstruct<MU, +1>(uh, a);
    inh.load(nb.b[MU], psi);
    project<MU, -1>(psi, h);
    su3_dag_mul(u, h, uh);
    reconstruct<MU, -1>(uh, b);
}

template <typename T, class LK, class IN>
__device__ __forceinline__ void hop_site_pair(const Geom& g, const LK& U, const IN& inp, const IN& inh, int s,
                                              cplx<T> (&a)[12], cplx<T> (&b)[12]) {
    const Nbr nb(g, s);
#pragma unroll
    for (int c = 0; c < 12; ++c) { a[c] = mk<T>(T(0), T(0)); b[c] = a[c]; }
    hop_dir_pair<0, T>(nb, U, inp, inh, s, a, b);
    hop_dir_pair<1, T>(nb, U, inp, inh, s, a, b);
    hop_dir_pair<2, T>(nb, U, inp, inh, s, a, b);
    hop_dir_pair<3, T>(nb, U, inp, inh, s, a, b);
}

}  // namespace lqcd
