// Per-slot two-level reductions shared by the lattice kernels.
#pragma once
#include "kernels.cuh"

namespace lqcd {

constexpr int RED_MAX_THREADS = 256;   // blocks that reduce have at most this many threads

__device__ __forceinline__ double2* part(const SlotPtrs& P, int kind) { return P.partials + (size_t)kind * PARTIAL_STRIDE; }

// Sum NV complex values per block into part[kind][block*NV + i]; in the last
// block returns true with tot[] = sum over blocks (thread 0 only). The block
// sum runs in the precision of v (FP32 for the mixed solver), the cross-block
// sum in FP64.
template <int NV, typename C>
__device__ bool reduce_slot(const SlotPtrs& P, int kind, C (&v)[NV], double2 (&tot)[NV], unsigned nblocks,
                            unsigned bid) {
    __shared__ C sm[(RED_MAX_THREADS / 32) * NV];   // blockDim.x <= RED_MAX_THREADS
    __shared__ double2 smd[(RED_MAX_THREADS / 32) * NV];
    block_sum<NV>(v, sm);
    double2* pp = part(P, kind);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) pp[(size_t)bid * NV + i] = to_d(v[i]);
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
        block_sum<NV>(acc, smd);
#pragma unroll
        for (int i = 0; i < NV; ++i) tot[i] = acc[i];
    }
    return last;
}

// Per-thread and per-block partial sums accumulate in the storage precision
// (FP32 for the mixed solver: FP64 arithmetic runs at a small fraction of the
// FP32 rate on this GPU and would bound these bandwidth kernels); only the
// cross-block sum is FP64.
template <typename S> struct Acc {
    cplx<S> z;      // complex sum
    S a, b;         // two real sums
    __device__ __forceinline__ Acc() : z(mk<S>(S(0), S(0))), a(S(0)), b(S(0)) {}
    __device__ __forceinline__ void to(cplx<S> (&v)[2]) const { v[0] = z; v[1] = mk<S>(a, b); }
};
template <typename C> __device__ __forceinline__ auto abs2(C a) -> decltype(a.x) { return a.x * a.x + a.y * a.y; }


}  // namespace lqcd
