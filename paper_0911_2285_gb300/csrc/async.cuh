// Asynchronous-copy and tensor-core primitives for sm_103a, as inline PTX:
// mbarriers with bounded waits, TMA bulk and tensor copies, and the tcgen05
// family (tensor-memory allocation, MMA issue/commit, tensor-memory loads).
//
// Every wait is bounded (wait_cycles()): a kernel that gives up sets an error
// word for the host instead of spinning forever.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lqcd {

// Bound of every device-side wait, in SM clock cycles (default about 2 s at
// 2 GHz). Each translation unit that includes this header holds its own copy
// on each device; set_wait_cycles_here() sets the copy of the including unit on
// the current device (the C ABI's lqcd_set_wait_limit sets all of them).
constexpr long long DEFAULT_WAIT_CYCLES = 4000000000ll;
static __device__ long long g_wait_cycles = DEFAULT_WAIT_CYCLES;
__device__ __forceinline__ long long wait_cycles() { return *(volatile long long*)&g_wait_cycles; }
static inline cudaError_t set_wait_cycles_here(long long cycles) {
    if (cycles <= 0) cycles = DEFAULT_WAIT_CYCLES;
    return cudaMemcpyToSymbol(g_wait_cycles, &cycles, sizeof(cycles));
}

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// ------------------------------------------------------------------ mbarrier
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for the phase of the given parity to complete, at most wait_cycles().
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
    const long long t0 = clock64(), lim = wait_cycles();
    while (!mbar_test(bar, parity))
        if (clock64() - t0 > lim) return false;
    return true;
}
// Wait for a device word to become nonzero, at most wait_cycles().
__device__ __forceinline__ bool flag_wait(const volatile int* flag) {
    const long long t0 = clock64(), lim = wait_cycles();
    while (*flag == 0)
        if (clock64() - t0 > lim) return false;
    return true;
}

// ----------------------------------------------------------------- TMA copies
// 1-D bulk copy global -> shared (16-byte aligned addresses, size multiple of 16).
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
// 2-D tiled tensor copy global -> shared of the box at (x, y); x is the inner
// (contiguous) coordinate and must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_2d(void* dst, const void* tmap, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_addr(dst)),
        "l"(tmap), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}
// Generic-proxy shared-memory writes -> visible to the async proxy (TMA, tcgen05).
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// -------------------------------------------------------------------- tcgen05
// Tensor-memory allocation: one full warp executes alloc / dealloc. The base
// address (lane 0, first column) is written to *dst in shared memory.
__device__ __forceinline__ void tmem_alloc(unsigned* dst, unsigned ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst)), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(unsigned taddr, unsigned ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A[smem] * B[smem]^T, both operands K-major, TF32 inputs, FP32 accumulate.
__device__ __forceinline__ void mma_tf32(unsigned d, uint64_t adesc, uint64_t bdesc, unsigned idesc, unsigned accum) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}
// The mbarrier completes one arrival once all earlier MMAs of this thread are done.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}
// 16 consecutive 32-bit columns of this thread's tensor-memory lane (warp w
// reads lanes 32 (w % 4) .. +31), waiting for the load to land.
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float (&v)[16]) {
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor of a K-major operand tile in the 128-byte
// swizzled layout (rows of 128 bytes, 8-row atoms of 1024 bytes, the layout a
// TMA tensor copy with 128-byte swizzle writes): start address, leading byte
// offset (unused for this layout, 16), stride byte offset 1024 (one 8-row
// atom to the next), descriptor version 1, layout type 2 (128-byte swizzle).
__device__ __forceinline__ uint64_t sdesc_k128(const void* p) {
    const uint64_t a = smem_addr(p);
    return ((a & 0x3FFFFull) >> 4) | (1ull << 16) | ((1024ull >> 4) << 32) | (1ull << 46) | (2ull << 61);
}
// Instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both
// K-major, M x N tile.
__host__ __device__ constexpr unsigned idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}
// Round to TF32 (10-bit mantissa, round to nearest, ties away from zero).
__device__ __forceinline__ float to_tf32(float x) {
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

}  // namespace lqcd
