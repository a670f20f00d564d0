// Tall-skinny complex inner-product matrices on the tensor cores (tcgen05):
//   C[i][j] = sum_e conj(X_i(e)) Y_j(e),   i < a, j < b,
// over FP32 fields of N complex numbers. These are the Galerkin projections
// of the deflation and of the eigenspace growth (Alg. Incremental eigBiCG:
// U_l^H r, U_l^H A U_r and the oblique orthogonalisation of new Ritz vectors).
//
// Real form: with x' = (re x, im x) interleaved along K (K = 2N reals),
//   Re C_ij = x'_i . y'_j,   Im C_ij = x'_i . z_j,  z = (im y, -re y),
// so one real GEMM of the a x K matrix X' against the 2b x K matrix [Y'; Z]
// gives both parts (M = 128 rows of X per CTA tile, N = 16 = 8 Y columns and
// their Z twins, FP32 accumulators in tensor memory).
//
// Precision: 3xTF32. Each operand v is split into big = tf32(v) and
// small = v - big, and the tile product is big.big + big.small + small.big,
// which keeps FP32-level accuracy. Each run of TC_FLUSH K-tiles accumulates in
// tensor memory (FP32); the runs and the CTAs (split-K) are summed in FP64.
//
// Data movement: TMA tensor copies with 128-byte swizzle bring 32-real K-tiles
// of X (128 rows) and Y (8 rows) into a 4-stage shared-memory ring; the split
// is elementwise in place (the swizzle moves 16-byte granules only, so every
// complex pair keeps its position), the Z twins go to the second 8-row atom.
// Warp-specialised: one thread issues the TMA copies, one the MMAs (committed
// to the stage's mbarrier, which frees the stage for the next copy), eight
// warps split the tiles; two tensor-memory accumulators alternate between
// runs so that reading one run overlaps the MMAs of the next.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <mutex>

#include "async.cuh"
#include "common.cuh"
#include "kernels.cuh"

namespace lqcd {
namespace {

constexpr int TC_KT = 32;        // reals per row per K-tile (128 bytes)
constexpr int TC_M = 128;        // X rows per CTA tile
constexpr int TC_NB = 8;         // Y fields per launch (N = 2 * TC_NB)
constexpr int TC_STAGES = 5;
constexpr int TC_FLUSH = 16;     // K-tiles per FP32 accumulation run in tensor memory
constexpr int TC_XW = 8;         // split (transform) warps
constexpr int TC_THREADS = 32 * (2 + TC_XW);
constexpr unsigned TC_TMEM_COLS = 32;   // two accumulators of 16 columns

struct __align__(1024) TcStage {
    float xa[TC_M * TC_KT];      // TMA X tile, then its TF32 big part in place
    float xs[TC_M * TC_KT];      // small part of X
    float yb[2 * TC_NB * TC_KT]; // rows 0-7: TMA Y tile -> big part; rows 8-15: big part of Z
    float ys[2 * TC_NB * TC_KT]; // small parts of Y and Z
};
static_assert(sizeof(TcStage) % 1024 == 0, "stage must keep 1024-byte alignment");
struct TcBars {
    uint64_t full[TC_STAGES], ready[TC_STAGES], empty[TC_STAGES], accfull[2], accempty[2];
    unsigned tmem;
    int abort;
};
constexpr size_t TC_SMEM = TC_STAGES * sizeof(TcStage) + 1024 /*align slack*/ + sizeof(TcBars);

__device__ __forceinline__ void split4(float4 v, float4& big, float4& small) {
    big = make_float4(to_tf32(v.x), to_tf32(v.y), to_tf32(v.z), to_tf32(v.w));
    small = make_float4(v.x - big.x, v.y - big.y, v.z - big.z, v.w - big.w);
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
// Bounded wait that also gives up once another role has aborted.
__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, unsigned parity, volatile int* abort) {
    const long long t0 = clock64();
    while (!mbar_test(bar, parity)) {
        if (*abort) return false;
        if (clock64() - t0 > WAIT_CYCLES) { *abort = 1; return false; }
    }
    return true;
}

// Warp roles: warp 0 allocates tensor memory and (lane 0) issues the TMA
// copies; warp 1 (lane 0) issues the MMAs; warps 2.. split the tiles into
// TF32 big/small parts, and warps 2-5 (one per tensor-memory lane quarter)
// also move each finished accumulation run into their FP64 sums.
// Grid (split-K CTAs, row tiles of 128). part: [gridDim.y][gridDim.x][128][16] FP64.
__global__ void __launch_bounds__(TC_THREADS, 1)
    dots_tc_kernel(const __grid_constant__ CUtensorMap mx, const __grid_constant__ CUtensorMap my, int box_rows,
                   long long tiles, double* part, int* err) {
    extern __shared__ unsigned char smem_raw[];
    TcStage* st = reinterpret_cast<TcStage*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    TcBars* B = reinterpret_cast<TcBars*>(st + TC_STAGES);
    volatile int* abort = &B->abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int y0 = blockIdx.y * TC_M;
    const long long t0 = (long long)blockIdx.x * tiles / gridDim.x;
    const long long t1 = (long long)(blockIdx.x + 1) * tiles / gridDim.x;
    const int n = (int)(t1 - t0);
    const int ngroups = (n + TC_FLUSH - 1) / TC_FLUSH;
    const unsigned tx = (unsigned)(box_rows + TC_NB) * TC_KT * 4;

    if (tid == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(&B->full[s], 1);
            mbar_init(&B->ready[s], TC_XW);
            mbar_init(&B->empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) { mbar_init(&B->accfull[b], 1); mbar_init(&B->accempty[b], 4); }
        B->abort = 0;
        mbar_init_fence();
    }
    if (warp == 0) {
        __syncwarp();
        tmem_alloc(&B->tmem, TC_TMEM_COLS);
        tmem_relinquish();
    }
    if (warp >= 2) {   // rows the TMA box does not cover stay zero in both X buffers
        for (int p = box_rows * TC_KT / 4 + (tid - 64); p < TC_M * TC_KT / 4; p += 32 * TC_XW)
            for (int s = 0; s < TC_STAGES; ++s) {
                reinterpret_cast<float4*>(st[s].xa)[p] = make_float4(0.f, 0.f, 0.f, 0.f);
                reinterpret_cast<float4*>(st[s].xs)[p] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        fence_proxy_async();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = B->tmem;
    constexpr unsigned IDESC = idesc_tf32(TC_M, 2 * TC_NB);

    double acc[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) acc[c] = 0.0;

    if (warp == 0) {
        if (lane == 0) {   // ---------------- TMA producer
            int j = 0;
            for (; j < n; ++j) {
                const int s = j % TC_STAGES;
                if (j >= TC_STAGES &&
                    !wait_or_abort(&B->empty[s], (unsigned)(j / TC_STAGES - 1) & 1u, abort))
                    break;
                const int x = (int)((t0 + j) * TC_KT);
                mbar_arrive_expect_tx(&B->full[s], tx);
                tma_load_2d(st[s].xa, &mx, x, y0, &B->full[s]);
                tma_load_2d(st[s].yb, &my, x, 0, &B->full[s]);
            }
            // every issued copy must land before the CTA may exit
            for (int q = j - TC_STAGES > 0 ? j - TC_STAGES : 0; q < j; ++q)
                mbar_wait(&B->full[q % TC_STAGES], (unsigned)(q / TC_STAGES) & 1u);
        }
    } else if (warp == 1) {
        if (lane == 0) {   // ---------------- MMA issuer
            int i = 0;
            for (; i < n; ++i) {
                const int s = i % TC_STAGES, g = i / TC_FLUSH, b = g & 1;
                if (i % TC_FLUSH == 0 && g >= 2 &&
                    !wait_or_abort(&B->accempty[b], (unsigned)(g / 2 - 1) & 1u, abort))
                    break;
                if (!wait_or_abort(&B->ready[s], (unsigned)(i / TC_STAGES) & 1u, abort)) break;
                tc_fence_after();
                TcStage& S = st[s];
                const unsigned d = tmem + (unsigned)(b * 16);
#pragma unroll
                for (int kk = 0; kk < TC_KT / 8; ++kk) {   // K = 8 reals (32 bytes) per MMA
                    const uint64_t ab = sdesc_k128(S.xa + 8 * kk), as = sdesc_k128(S.xs + 8 * kk);
                    const uint64_t bb = sdesc_k128(S.yb + 8 * kk), bs = sdesc_k128(S.ys + 8 * kk);
                    mma_tf32(d, ab, bb, IDESC, (i % TC_FLUSH != 0 || kk > 0) ? 1u : 0u);
                    mma_tf32(d, ab, bs, IDESC, 1u);
                    mma_tf32(d, as, bb, IDESC, 1u);
                }
                mma_commit(&B->empty[s]);
                if (i % TC_FLUSH == TC_FLUSH - 1 || i == n - 1) mma_commit(&B->accfull[b]);
            }
            if (i > 0)   // the last MMAs must finish before tensor memory is released
                mbar_wait(&B->empty[(i - 1) % TC_STAGES], (unsigned)((i - 1) / TC_STAGES) & 1u);
        }
    } else {   // ---------------------------- split warps (+ accumulator readers)
        const int xt = tid - 64;
        const bool reader = warp < 6;
        const unsigned lane_base = (unsigned)((warp & 3) * 32) << 16;
        int next_group = 0;
        auto read_group = [&](int g) -> bool {
            // warp-uniform outcome: tcgen05.ld below needs the whole warp
            if (!__all_sync(0xffffffffu, wait_or_abort(&B->accfull[g & 1], (unsigned)(g / 2) & 1u, abort)))
                return false;
            tc_fence_after();
            float v[16];
            tmem_ld16(tmem + lane_base + (unsigned)((g & 1) * 16), v);
#pragma unroll
            for (int c = 0; c < 16; ++c) acc[c] += (double)v[c];
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&B->accempty[g & 1]);
            return true;
        };
        bool ok = true;
        for (int i = 0; i < n && ok; ++i) {
            const int s = i % TC_STAGES;
            if (!__all_sync(0xffffffffu, wait_or_abort(&B->full[s], (unsigned)(i / TC_STAGES) & 1u, abort))) {
                ok = false;
                break;
            }
            TcStage& S = st[s];
            float4* xa = reinterpret_cast<float4*>(S.xa);
            float4* xs = reinterpret_cast<float4*>(S.xs);
            for (int p = xt; p < box_rows * TC_KT / 4; p += 32 * TC_XW) {
                float4 big, small;
                split4(xa[p], big, small);
                xa[p] = big;
                xs[p] = small;
            }
            if (xt < TC_NB * TC_KT / 4) {   // Y and its Z twin
                float4* yb = reinterpret_cast<float4*>(S.yb);
                float4* ys = reinterpret_cast<float4*>(S.ys);
                const float4 y = yb[xt];
                float4 big, small;
                split4(y, big, small);
                yb[xt] = big;
                ys[xt] = small;
                split4(make_float4(y.y, -y.x, y.w, -y.z), big, small);
                yb[TC_NB * TC_KT / 4 + xt] = big;
                ys[TC_NB * TC_KT / 4 + xt] = small;
            }
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(&B->ready[s]);
            if (reader && i % TC_FLUSH == 1 && i > TC_FLUSH) ok = read_group(next_group++);
        }
        if (reader)
            while (ok && next_group < ngroups) ok = read_group(next_group++);
        if (ok && reader) {
            const int r = (warp & 3) * 32 + lane;
            double* out = part + (((size_t)blockIdx.y * gridDim.x + blockIdx.x) * TC_M + r) * 16;
#pragma unroll
            for (int c = 0; c < 16; ++c) out[c] = acc[c];
        }
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && *abort) atomicExch(err, 1);
    if (warp == 0) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem, TC_TMEM_COLS);
    }
}

// C[i][j] (or conj into C[j][i]) = sum over the split-K partials, FP64.
__global__ void dots_tc_reduce_kernel(int a, int b, int nblk, const double* part, double2* Cm, int ldc,
                                      int conj_store) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= a * b) return;
    const int i = q / b, j = q % b, ty = i / TC_M, r = i % TC_M;
    double re = 0.0, im = 0.0;
    for (int k = 0; k < nblk; ++k) {
        const double* p = part + (((size_t)ty * nblk + k) * TC_M + r) * 16;
        re += p[j];
        im += p[TC_NB + j];
    }
    if (conj_store) Cm[(size_t)j * ldc + i] = make_double2(re, -im);
    else Cm[(size_t)i * ldc + j] = make_double2(re, im);
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;
std::once_flag g_prepare_once;
cudaError_t g_prepare_err = cudaSuccess;
int g_num_sms = 0;
__device__ int g_tc_err;   // error word for callers that pass none

int num_sms() {
    if (g_num_sms == 0) {
        int dev = 0, n = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        g_num_sms = n > 0 ? n : 148;
    }
    return g_num_sms;
}

cudaError_t get_encode() {
    std::call_once(g_encode_once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    return g_encode ? cudaSuccess : cudaErrorNotSupported;
}

// rows x (2N reals) FP32 matrix, row stride in bytes; box = 32 reals x box_rows, 128-byte swizzle.
bool encode_rows(CUtensorMap* m, const void* base, size_t n_complex, int rows, size_t row_bytes, int box_rows) {
    // box = TC_KT reals x box_rows rows; rows past the tensor read as zero
    cuuint64_t dims[2] = {(cuuint64_t)(2 * n_complex), (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)row_bytes};
    cuuint32_t box[2] = {(cuuint32_t)TC_KT, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return g_encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool dots_tc_supported(int a, const void* X, const void* Y, size_t N) {
    return a > 0 && a <= 4 * TC_M && N > 0 && (2 * N) % TC_KT == 0 && ((uintptr_t)X & 15) == 0 &&
           ((uintptr_t)Y & 15) == 0 && get_encode() == cudaSuccess;
}

size_t dots_tc_scratch_doubles(int a) { return (size_t)((a + TC_M - 1) / TC_M) * num_sms() * TC_M * 16; }

cudaError_t prepare_dots_tc() {
    std::call_once(g_prepare_once, [] {
        g_prepare_err = cudaFuncSetAttribute((const void*)dots_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)TC_SMEM);
    });
    return g_prepare_err;
}

// FP32 fields only: X = a fields, Y = b fields, each N complex, consecutive
// fields x_stride / y_stride bytes apart.
cudaError_t launch_dots_tc(int a, const void* X, size_t x_stride, int b, const void* Y, size_t y_stride, size_t N,
                           double2* Cm, int ldc, int conj_store, double* scratch, size_t scratch_doubles, int* err,
                           cudaStream_t st) {
    if (a <= 0 || b <= 0) return cudaSuccess;
    if (!dots_tc_supported(a, X, Y, N) || (x_stride & 15) || (y_stride & 15)) return cudaErrorInvalidValue;
    cudaError_t pe = prepare_dots_tc();
    if (pe != cudaSuccess) return pe;
    if (!err) {
        void* p = nullptr;
        pe = cudaGetSymbolAddress(&p, g_tc_err);
        if (pe != cudaSuccess) return pe;
        err = reinterpret_cast<int*>(p);
    }
    const long long tiles = (long long)(2 * N / TC_KT);
    const int ty = (a + TC_M - 1) / TC_M;
    int nblk = num_sms();
    if (nblk > tiles) nblk = (int)tiles;
    if ((size_t)ty * nblk * TC_M * 16 > scratch_doubles) return cudaErrorInvalidValue;
    const int box_rows = ty > 1 ? TC_M : (a + 7) / 8 * 8;
    CUtensorMap mx;
    if (!encode_rows(&mx, X, N, a, x_stride, box_rows)) return cudaErrorInvalidValue;
    for (int j0 = 0; j0 < b; j0 += TC_NB) {
        const int bb = b - j0 < TC_NB ? b - j0 : TC_NB;
        CUtensorMap my;
        const char* Yj = reinterpret_cast<const char*>(Y) + (size_t)j0 * y_stride;
        if (!encode_rows(&my, Yj, N, bb, y_stride, TC_NB)) return cudaErrorInvalidValue;
        dots_tc_kernel<<<dim3(nblk, ty), TC_THREADS, TC_SMEM, st>>>(mx, my, box_rows, tiles, scratch, err);
        count_launches(1);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        double2* Cj = conj_store ? Cm + (size_t)j0 * ldc : Cm + j0;
        dots_tc_reduce_kernel<<<(int)(((size_t)a * bb + 127) / 128), 128, 0, st>>>(a, bb, nblk, scratch, Cj, ldc,
                                                                            conj_store);
        count_launches(1);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace lqcd
