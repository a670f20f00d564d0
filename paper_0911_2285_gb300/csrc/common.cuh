// Shared device definitions: complex arithmetic, field and link layouts,
// lattice geometry, per-slot solver state.
//
// Field layout in HBM (both precisions share the same complex ordering, so a
// flat element-wise map converts between them):
//   a site's 12 spin-colour components c = spin*3 + colour are grouped in 6
//   pairs ("chunks") q = c/2; chunk q of all sites is contiguous:
//     FP32: float4  f[q*V + s]          = (re c0, im c0, re c1, im c1)
//     FP64: double2 d[(q*V + s)*2 + e]  = (re, im) of c = 2q + e
//   so a warp over consecutive sites reads each chunk fully coalesced.
// Link layout:
//   FP64: double2 u[(mu*9 + 3*row + col)*V + s]           (all 18 reals)
//   FP32: float4  u[(mu*3 + q)*V + s], q = 0..2 hold rows 0 and 1
//         (u00,u01) (u02,u10) (u11,u12); row 2 = conj(row0 x row1) (SU(3)).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lqcd {

// ----------------------------------------------------------------- complex
template <typename T> struct cplx_t;
template <> struct cplx_t<float> { using type = float2; };
template <> struct cplx_t<double> { using type = double2; };
template <typename T> using cplx = typename cplx_t<T>::type;

template <typename T> __host__ __device__ __forceinline__ cplx<T> mk(T re, T im) {
    cplx<T> z; z.x = re; z.y = im; return z;
}
__host__ __device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 operator*(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__host__ __device__ __forceinline__ float2 operator*(float a, float2 b) { return make_float2(a * b.x, a * b.y); }
__host__ __device__ __forceinline__ float2 operator-(float2 a) { return make_float2(-a.x, -a.y); }
__host__ __device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 operator*(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__host__ __device__ __forceinline__ double2 operator*(double a, double2 b) { return make_double2(a * b.x, a * b.y); }
__host__ __device__ __forceinline__ double2 operator-(double2 a) { return make_double2(-a.x, -a.y); }

template <typename C> __host__ __device__ __forceinline__ C conj_(C a) { a.y = -a.y; return a; }
// i * a, -i * a
template <typename C> __host__ __device__ __forceinline__ C mul_i(C a) { C r; r.x = -a.y; r.y = a.x; return r; }
template <typename C> __host__ __device__ __forceinline__ C mul_mi(C a) { C r; r.x = a.y; r.y = -a.x; return r; }
// conj(a) * b
template <typename C> __host__ __device__ __forceinline__ C cdot(C a, C b) {
    C r; r.x = a.x * b.x + a.y * b.y; r.y = a.x * b.y - a.y * b.x; return r;
}
// a * conj(b)
template <typename C> __host__ __device__ __forceinline__ C mulc(C a, C b) {
    C r; r.x = a.x * b.x + a.y * b.y; r.y = a.y * b.x - a.x * b.y; return r;
}
__host__ __device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    // Smith's algorithm for a / b.
    if (fabs(b.x) >= fabs(b.y)) {
        double r = b.y / b.x, den = b.x + b.y * r;
        return make_double2((a.x + a.y * r) / den, (a.y - a.x * r) / den);
    } else {
        double r = b.x / b.y, den = b.x * r + b.y;
        return make_double2((a.x * r + a.y) / den, (a.y * r - a.x) / den);
    }
}
__host__ __device__ __forceinline__ double cabs_(double2 a) { return hypot(a.x, a.y); }

__host__ __device__ __forceinline__ float2 to_f(double2 a) { return make_float2((float)a.x, (float)a.y); }
__host__ __device__ __forceinline__ double2 to_d(float2 a) { return make_double2(a.x, a.y); }
__host__ __device__ __forceinline__ double2 to_d(double2 a) { return a; }
template <typename T> __host__ __device__ __forceinline__ cplx<T> cvt(double2 a);
template <> __host__ __device__ __forceinline__ float2 cvt<float>(double2 a) { return to_f(a); }
template <> __host__ __device__ __forceinline__ double2 cvt<double>(double2 a) { return a; }

// ---------------------------------------------------------------- geometry
struct Geom {
    int L[4];        // Lx, Ly, Lz, Lt
    int stride[4];   // 1, Lx, Lx*Ly, Lx*Ly*Lz
    int V;
    __device__ __forceinline__ int coord(int s, int mu) const { return (s / stride[mu]) % L[mu]; }
    __device__ __forceinline__ int fwd(int s, int mu) const {
        return coord(s, mu) == L[mu] - 1 ? s - (L[mu] - 1) * stride[mu] : s + stride[mu];
    }
    __device__ __forceinline__ int bwd(int s, int mu) const {
        return coord(s, mu) == 0 ? s + (L[mu] - 1) * stride[mu] : s - stride[mu];
    }
};

// The eight neighbour sites of s (periodic), from one coordinate decomposition.
struct Nbr {
    int f[4], b[4];
    __device__ __forceinline__ Nbr(const Geom& g, int s) {
        int r = s;
        int c[4];
        c[0] = r % g.L[0]; r /= g.L[0];
        c[1] = r % g.L[1]; r /= g.L[1];
        c[2] = r % g.L[2];
        c[3] = r / g.L[2];
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            const int st = g.stride[mu], wrap = (g.L[mu] - 1) * st;
            f[mu] = c[mu] == g.L[mu] - 1 ? s - wrap : s + st;
            b[mu] = c[mu] == 0 ? s + wrap : s - st;
        }
    }
};

// ------------------------------------------------------------ field access
// Storage type S (float or double); values returned in arithmetic type T.
template <typename S> struct Field;

template <> struct Field<float> {
    static __device__ __forceinline__ void load(const void* base, int V, int s, float2 (&v)[12]) {
        const float4* f = reinterpret_cast<const float4*>(base);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            float4 t = __ldg(f + (size_t)q * V + s);
            v[2 * q] = make_float2(t.x, t.y);
            v[2 * q + 1] = make_float2(t.z, t.w);
        }
    }
    static __device__ __forceinline__ void load(const void* base, int V, int s, double2 (&v)[12]) {
        float2 t[12];
        load(base, V, s, t);
#pragma unroll
        for (int c = 0; c < 12; ++c) v[c] = to_d(t[c]);
    }
    static __device__ __forceinline__ void store(void* base, int V, int s, const float2 (&v)[12]) {
        float4* f = reinterpret_cast<float4*>(base);
#pragma unroll
        for (int q = 0; q < 6; ++q) f[(size_t)q * V + s] = make_float4(v[2 * q].x, v[2 * q].y, v[2 * q + 1].x, v[2 * q + 1].y);
    }
    static __device__ __forceinline__ void store(void* base, int V, int s, const double2 (&v)[12]) {
        float2 t[12];
#pragma unroll
        for (int c = 0; c < 12; ++c) t[c] = to_f(v[c]);
        store(base, V, s, t);
    }
};

template <> struct Field<double> {
    static __device__ __forceinline__ void load(const void* base, int V, int s, double2 (&v)[12]) {
        const double2* d = reinterpret_cast<const double2*>(base);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            v[2 * q] = __ldg(d + ((size_t)q * V + s) * 2);
            v[2 * q + 1] = __ldg(d + ((size_t)q * V + s) * 2 + 1);
        }
    }
    static __device__ __forceinline__ void load(const void* base, int V, int s, float2 (&v)[12]) {
        double2 t[12];
        load(base, V, s, t);
#pragma unroll
        for (int c = 0; c < 12; ++c) v[c] = to_f(t[c]);
    }
    static __device__ __forceinline__ void store(void* base, int V, int s, const double2 (&v)[12]) {
        double2* d = reinterpret_cast<double2*>(base);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            d[((size_t)q * V + s) * 2] = v[2 * q];
            d[((size_t)q * V + s) * 2 + 1] = v[2 * q + 1];
        }
    }
    static __device__ __forceinline__ void store(void* base, int V, int s, const float2 (&v)[12]) {
        double2 t[12];
#pragma unroll
        for (int c = 0; c < 12; ++c) t[c] = to_d(v[c]);
        store(base, V, s, t);
    }
};

// Flat complex element e (0 <= e < 12 V) of a field in storage S.
template <typename S> __device__ __forceinline__ cplx<S> ld_elem(const void* base, size_t e) {
    return reinterpret_cast<const cplx<S>*>(base)[e];
}
template <typename S> __device__ __forceinline__ void st_elem(void* base, size_t e, cplx<S> v) {
    reinterpret_cast<cplx<S>*>(base)[e] = v;
}

// ---------------------------------------------------------------- reductions
template <typename C> __device__ __forceinline__ C warp_sum(C v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum of NV complex values per thread (float2 or double2, summed in
// that precision); result valid in thread 0.
// blockDim.x must be a multiple of 32 and <= 1024. smem: 32*NV values of type C.
template <int NV, typename C> __device__ __forceinline__ void block_sum(C (&v)[NV], C* smem) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = warp_sum(v[i]);
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) smem[w * NV + i] = v[i];
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            C t;
            t.x = 0; t.y = 0;
            if (lane < nw) t = smem[lane * NV + i];
            v[i] = warp_sum(t);
        }
    }
}

// "Last block done" handshake: every block calls this after publishing its
// partials; returns true in exactly one block (the last to arrive), which then
// sees all partials. The partials must be written by thread 0 of the block, or
// fenced (__threadfence) by the thread that wrote them before this call; the
// other threads' stores need no fence. counter must be zero before the launch;
// it is reset here.
__device__ __forceinline__ bool last_block(unsigned* counter, unsigned nblocks) {
    __shared__ bool am_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned prev = atomicAdd(counter, 1u);
        am_last = (prev == nblocks - 1);
        if (am_last) *counter = 0;   // ready for the next launch
    }
    __syncthreads();
    if (am_last) __threadfence();
    return am_last;
}

}  // namespace lqcd
