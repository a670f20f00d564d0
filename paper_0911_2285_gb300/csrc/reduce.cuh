// Per-slot two-level reductions shared by the lattice kernels.
#pragma once
#include "kernels.cuh"

namespace lqcd {

constexpr int RED_MAX_THREADS = 256;   // blocks that reduce have at most this many threads

__device__ __forceinline__ double2* part(const SlotPtrs& P, int kind) { return P.partials + (size_t)kind * PARTIAL_STRIDE; }

// Sum NV complex values per block into part[kind][block*NV + i]; in the last
// block returns true with tot[] = sum over blocks (thread 0 only).
template <int NV>
__device__ bool reduce_slot(const SlotPtrs& P, int kind, double2 (&v)[NV], double2 (&tot)[NV], unsigned nblocks,
                            unsigned bid) {
    __shared__ double2 sm[(RED_MAX_THREADS / 32) * NV];   // blockDim.x <= RED_MAX_THREADS
    block_sum<NV>(v, sm);
    double2* pp = part(P, kind);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) pp[(size_t)bid * NV + i] = v[i];
    }
    bool last = last_block(P.counters + kind, nblocks);
    if (last) {
        // the last block adds the partials in block order (deterministic)
        double2 acc[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) acc[i] = make_double2(0.0, 0.0);
        for (unsigned b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
            for (int i = 0; i < NV; ++i) acc[i] = acc[i] + __ldcg(pp + (size_t)b * NV + i);
        // fixed-order tree over threads
        block_sum<NV>(acc, sm);
#pragma unroll
        for (int i = 0; i < NV; ++i) tot[i] = acc[i];
    }
    return last;
}

// Per-thread partial sums accumulate in the storage precision (FP32 for the
// mixed solver: FP64 arithmetic is a small fraction of FP32 throughput on this
// GPU and would bound these bandwidth kernels); the block and cross-block sums
// are FP64.
template <typename S> struct Acc {
    cplx<S> z;      // complex sum
    S a, b;         // two real sums
    __device__ __forceinline__ Acc() : z(mk<S>(S(0), S(0))), a(S(0)), b(S(0)) {}
    __device__ __forceinline__ void to(double2 (&v)[2]) const { v[0] = to_d(z); v[1] = make_double2((double)a, (double)b); }
};
template <typename C> __device__ __forceinline__ auto abs2(C a) -> decltype(a.x) { return a.x * a.x + a.y * a.y; }


}  // namespace lqcd
