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
// which keeps FP32-level accuracy. The tensor core truncates as it
// accumulates, so big.big and the corrections accumulate in separate
// tensor-memory columns over short runs (TC_FLUSH K-tiles, 8 MMAs each); the
// runs and the CTAs (split-K) are summed in FP64.
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
constexpr int TC_NB = 8;         // Y fields per launch, narrow form (N = 2 * TC_NB)
constexpr int TC_NB_WIDE = 24;   // wide form (N = 48): one launch serves up to 24 Y fields, so X is
                                 // read once and each MMA instruction does three times the work
constexpr int TC_STAGES = 5;
constexpr int TC_FLUSH = 2;      // K-tiles per FP32 accumulation run in tensor memory
constexpr int TC_XW = 8;         // split (transform) warps
constexpr int TC_THREADS = 32 * (2 + TC_XW);
constexpr int TC_NBUF = 4;       // accumulator sets in flight (runs the readers may lag behind)
constexpr int TC_SUPER = 16;     // runs summed in FP32 before an FP64 add
// tensor-memory columns: TC_NBUF runs x (big.big, correction) x 2 NB columns, as a power of two
__host__ __device__ constexpr unsigned tc_tmem_cols(int nb) {
    return (unsigned)(TC_NBUF * 2 * 2 * nb) <= 128u ? 128u : (unsigned)(TC_NBUF * 2 * 2 * nb) <= 256u ? 256u : 512u;
}

template <int NB> struct __align__(1024) TcStage {
    float xa[TC_M * TC_KT];      // TMA X tile, then its TF32 big part in place
    float xs[TC_M * TC_KT];      // small part of X
    float yb[2 * NB * TC_KT];    // rows 0..NB-1: TMA Y tile -> big part; rows NB..2NB-1: big part of Z
    float ys[2 * NB * TC_KT];    // small parts of Y and Z
};
static_assert(sizeof(TcStage<TC_NB>) % 1024 == 0, "stage must keep 1024-byte alignment");
static_assert(sizeof(TcStage<TC_NB_WIDE>) % 1024 == 0, "stage must keep 1024-byte alignment");
struct TcBars {
    uint64_t full[TC_STAGES], ready[TC_STAGES], empty[TC_STAGES], accfull[TC_NBUF], accempty[TC_NBUF];
    unsigned tmem;
    int abort;
};
template <int NB> constexpr size_t tc_smem() { return TC_STAGES * sizeof(TcStage<NB>) + 1024 /*align slack*/ + sizeof(TcBars); }

__device__ __forceinline__ void split4(float4 v, float4& big, float4& small) {
    big = make_float4(to_tf32(v.x), to_tf32(v.y), to_tf32(v.z), to_tf32(v.w));
    small = make_float4(v.x - big.x, v.y - big.y, v.z - big.z, v.w - big.w);
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
// Bounded wait that also gives up once another role has aborted.
__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, unsigned parity, volatile int* abort) {
    const long long t0 = clock64(), lim = wait_cycles();
    while (!mbar_test(bar, parity)) {
        if (*abort) return false;
        if (clock64() - t0 > lim) { *abort = 1; return false; }
    }
    return true;
}

// Warp roles: warp 0 allocates tensor memory and (lane 0) issues the TMA
// copies; warp 1 (lane 0) issues the MMAs; warps 2.. split the tiles into
// TF32 big/small parts, and warps 2-5 (one per tensor-memory lane quarter)
// also move each finished accumulation run into their FP64 sums.
// Grid (split-K CTAs, row tiles of 128). part: [gridDim.y][gridDim.x][128][16] FP64.
// NB: Y fields per launch (N = 2 NB columns: the Y fields and their Z twins).
template <int NB>
__global__ void __launch_bounds__(TC_THREADS, 1)
    dots_tc_kernel(const __grid_constant__ CUtensorMap mx, const __grid_constant__ CUtensorMap my, int box_rows,
                   long long tiles, double* part, int* err) {
    constexpr int NC = 2 * NB;                       // accumulator columns
    constexpr unsigned TMEM_COLS = tc_tmem_cols(NB);
    extern __shared__ unsigned char smem_raw[];
    using Stage = TcStage<NB>;
    Stage* st = reinterpret_cast<Stage*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    TcBars* B = reinterpret_cast<TcBars*>(st + TC_STAGES);
    volatile int* abort = &B->abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int y0 = blockIdx.y * TC_M;
    const long long t0 = (long long)blockIdx.x * tiles / gridDim.x;
    const long long t1 = (long long)(blockIdx.x + 1) * tiles / gridDim.x;
    const int n = (int)(t1 - t0);
    const int ngroups = (n + TC_FLUSH - 1) / TC_FLUSH;
    const unsigned tx = (unsigned)(box_rows + NB) * TC_KT * 4;

    if (tid == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(&B->full[s], 1);
            mbar_init(&B->ready[s], TC_XW);
            mbar_init(&B->empty[s], 1);
        }
        for (int b = 0; b < TC_NBUF; ++b) { mbar_init(&B->accfull[b], 1); mbar_init(&B->accempty[b], 4); }
        B->abort = 0;
        mbar_init_fence();
    }
    if (warp == 0) {
        __syncwarp();
        tmem_alloc(&B->tmem, TMEM_COLS);
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
    constexpr unsigned IDESC = idesc_tf32(TC_M, NC);

    double acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = 0.0;

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
                const int s = i % TC_STAGES, g = i / TC_FLUSH, b = g % TC_NBUF;
                if (i % TC_FLUSH == 0 && g >= TC_NBUF &&
                    !wait_or_abort(&B->accempty[b], (unsigned)(g / TC_NBUF - 1) & 1u, abort))
                    break;
                if (!wait_or_abort(&B->ready[s], (unsigned)(i / TC_STAGES) & 1u, abort)) break;
                tc_fence_after();
                Stage& S = st[s];
                // big.big and the two correction products go to separate accumulators
                // (the tensor core truncates as it accumulates: keeping the small
                // terms apart and the runs short keeps the sum at FP32 accuracy)
                const unsigned dm = tmem + (unsigned)(b * 2 * NC), dc = dm + NC;
#pragma unroll
                for (int kk = 0; kk < TC_KT / 8; ++kk) {   // K = 8 reals (32 bytes) per MMA
                    const uint64_t ab = sdesc_k128(S.xa + 8 * kk), as = sdesc_k128(S.xs + 8 * kk);
                    const uint64_t bb = sdesc_k128(S.yb + 8 * kk), bs = sdesc_k128(S.ys + 8 * kk);
                    const unsigned keep = (i % TC_FLUSH != 0 || kk > 0) ? 1u : 0u;
                    mma_tf32(dm, ab, bb, IDESC, keep);
                    mma_tf32(dc, ab, bs, IDESC, keep);
                    mma_tf32(dc, as, bb, IDESC, 1u);
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
        float sum32[NC];   // FP32 sum of up to TC_SUPER runs (FP64 adds are slow on this GPU)
#pragma unroll
        for (int c = 0; c < NC; ++c) sum32[c] = 0.f;
        auto read_group = [&](int g) -> bool {
            const int b = g % TC_NBUF;
            // warp-uniform outcome: tcgen05.ld below needs the whole warp
            if (!__all_sync(0xffffffffu, wait_or_abort(&B->accfull[b], (unsigned)(g / TC_NBUF) & 1u, abort)))
                return false;
            tc_fence_after();
#pragma unroll
            for (int c0 = 0; c0 < NC; c0 += 16) {
                float v[16], w[16];
                tmem_ld16(tmem + lane_base + (unsigned)(b * 2 * NC + c0), v);
                tmem_ld16(tmem + lane_base + (unsigned)(b * 2 * NC + NC + c0), w);
#pragma unroll
                for (int c = 0; c < 16; ++c) sum32[c0 + c] += v[c] + w[c];
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&B->accempty[b]);
            if (g % TC_SUPER == TC_SUPER - 1 || g == ngroups - 1) {
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    acc[c] += (double)sum32[c];
                    sum32[c] = 0.f;
                }
            }
            return true;
        };
        bool ok = true;
        for (int i = 0; i < n && ok; ++i) {
            const int s = i % TC_STAGES;
            if (!__all_sync(0xffffffffu, wait_or_abort(&B->full[s], (unsigned)(i / TC_STAGES) & 1u, abort))) {
                ok = false;
                break;
            }
            Stage& S = st[s];
            float4* xa = reinterpret_cast<float4*>(S.xa);
            float4* xs = reinterpret_cast<float4*>(S.xs);
            for (int p = xt; p < box_rows * TC_KT / 4; p += 32 * TC_XW) {
                float4 big, small;
                split4(xa[p], big, small);
                xa[p] = big;
                xs[p] = small;
            }
            for (int yt = xt; yt < NB * TC_KT / 4; yt += 32 * TC_XW) {   // Y and its Z twin
                float4* yb = reinterpret_cast<float4*>(S.yb);
                float4* ys = reinterpret_cast<float4*>(S.ys);
                const float4 y = yb[yt];
                float4 big, small;
                split4(y, big, small);
                yb[yt] = big;
                ys[yt] = small;
                split4(make_float4(y.y, -y.x, y.w, -y.z), big, small);
                yb[NB * TC_KT / 4 + yt] = big;
                ys[NB * TC_KT / 4 + yt] = small;
            }
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(&B->ready[s]);
            // run g is read TC_NBUF - 2 runs after it was issued
            if (reader && i % TC_FLUSH == 1 && i > (TC_NBUF - 1) * TC_FLUSH) ok = read_group(next_group++);
        }
        if (reader)
            while (ok && next_group < ngroups) ok = read_group(next_group++);
        if (ok && reader) {
            const int r = (warp & 3) * 32 + lane;
            double* out = part + (((size_t)blockIdx.y * gridDim.x + blockIdx.x) * TC_M + r) * NC;
#pragma unroll
            for (int c = 0; c < NC; ++c) out[c] = acc[c];
        }
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && *abort) atomicExch(err, 1);
    if (warp == 0) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem, TMEM_COLS);
    }
}

// C[i][j] (or conj into C[j][i]) = sum over the split-K partials, FP64.
__global__ void dots_tc_reduce_kernel(int a, int b, int nb, int nblk, const double* part, double2* Cm, int ldc,
                                      int conj_store) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= a * b) return;
    const int i = q / b, j = q % b, ty = i / TC_M, r = i % TC_M;
    double re = 0.0, im = 0.0;
    for (int k = 0; k < nblk; ++k) {
        const double* p = part + (((size_t)ty * nblk + k) * TC_M + r) * (2 * nb);
        re += p[j];
        im += p[nb + j];
    }
    if (conj_store) Cm[(size_t)j * ldc + i] = make_double2(re, -im);
    else Cm[(size_t)i * ldc + j] = make_double2(re, im);
}

// ------------------------------------------------------------------------
// In-place window product of the BiCG-eigen restart on the tensor cores
// (Alg. BiCG-eigen: V <- V Yc, W <- W Zc, FP32 windows), one job per
// (slot, side):
//   new slot k = sum_{i<m} s_i c_ik old slot i   (k < r),   new slot r = old slot m,
// plus the coupling dots of the new vectors with (A p - beta q) or
// (A^+ phat - conj(beta) s), and the new H row/column (same contract as the
// CUDA-core window_gemm_kernel).
//
// Real form per element e: y(e)[2k + c'] = sum_{i, c} x(e)[2i + c] B[2k + c'][2i + c]
// with the 2 x 2 blocks B = [[cr, -ci], [ci, cr]] of s_i c_ik: an MMA with
// M = 128 elements, N = 2 r (padded to 48), K = 2 m reals in K-chunks of 16
// fields. The fields are element-contiguous, so 1-D bulk copies bring 16
// field rows of 128 elements into a raw stage and eight warps transpose them
// into the 128-byte-swizzled K-major operand (3xTF32 split on the way).
// Roles: warp 0 copies, warp 1 issues MMAs, warps 2-9 transpose, warps 10-13
// (one per tensor-memory lane quarter) drain the two alternating accumulators
// and store, copy slot m and form the coupling dots.
constexpr int RT_E = 128;        // elements per tile
constexpr int RT_KF = 16;        // fields per K-chunk (32 reals, one 128-byte row)
constexpr int RT_QMAX = 4;       // K-chunks: m <= 64
constexpr int RT_RMAX = 24;      // kept vectors r <= 24
constexpr int RT_N = 2 * RT_RMAX;
constexpr int RT_STAGES = 3;
constexpr int RT_XW = 8;         // transpose warps
constexpr int RT_EW = 4;         // epilogue warps
constexpr int RT_THREADS = 32 * (2 + RT_XW + RT_EW);
constexpr unsigned RT_TMEM_COLS = 512;   // two tiles x (one big.big accumulator per K-chunk + corrections)
constexpr int RT_ACC_STRIDE = 256;       // columns per tile accumulator set: 4 x 48 main + 48 correction

struct __align__(1024) RtSmem {
    float bb[RT_QMAX][RT_N * 32];    // coefficients, big part (K-major, swizzled), per K-chunk
    float bs[RT_QMAX][RT_N * 32];    // small part
    float ab[2][RT_E * 32];          // transposed X chunk, big part (two buffers)
    float as[2][RT_E * 32];          // small part
    float raw[RT_STAGES][RT_KF * RT_E * 2];   // field rows as copied: [field][element][re, im]
    uint64_t raw_full[RT_STAGES], raw_empty[RT_STAGES], a_full[2], a_empty[2], acc_full[2], acc_empty[2];
    double2 dots[RT_EW][RT_RMAX];
    unsigned tmem;
    int abort;
};
constexpr size_t RT_SMEM = sizeof(RtSmem) + 1024;

// byte offset of the 16-byte granule j of row n in a 128-byte-swizzled K-major tile
__device__ __forceinline__ int sw128(int n, int j) { return n * 128 + ((j ^ (n & 7)) << 4); }

__global__ void __launch_bounds__(RT_THREADS, 1)
    restart_tc_kernel(SlotState* states, const SlotPtrs* ptrs, size_t N, int* err) {
    const int slot = blockIdx.y >> 1, side = blockIdx.y & 1;
    SlotState& st = states[slot];
    const SlotPtrs& P = ptrs[slot];
    if (st.status != ST_RUNNING || st.restart_r == 0) return;   // uniform over the CTA
    extern __shared__ unsigned char smem_raw[];
    RtSmem* S = reinterpret_cast<RtSmem*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    volatile int* abort = &S->abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m = st.m, r = st.restart_r, ldc = 2 * st.nev + 1;
    const int Q = (m + RT_KF - 1) / RT_KF;
    const int par = st.iter & 1;
    char* base = reinterpret_cast<char*>(side ? P.W : P.V);
    const size_t fbytes = N * 8;
    const long long tiles = (long long)(N / RT_E);
    const long long t0 = (long long)blockIdx.x * tiles / gridDim.x;
    const long long t1 = (long long)(blockIdx.x + 1) * tiles / gridDim.x;
    const int nt = (int)(t1 - t0);
    const int nchunks = nt * Q;

    if (tid == 0) {
        for (int s = 0; s < RT_STAGES; ++s) { mbar_init(&S->raw_full[s], 1); mbar_init(&S->raw_empty[s], RT_XW); }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&S->a_full[b], RT_XW);
            mbar_init(&S->a_empty[b], 1);
            mbar_init(&S->acc_full[b], 1);
            mbar_init(&S->acc_empty[b], RT_EW);
        }
        S->abort = 0;
        mbar_init_fence();
    }
    if (warp == 0) {
        __syncwarp();
        tmem_alloc(&S->tmem, RT_TMEM_COLS);
        tmem_relinquish();
    }
    // coefficient operand: row n = 2k + c', K index 2i + c, blocks [[cr, -ci], [ci, cr]] of s_i c_ik
    {
        const double2* coef = side ? P.coefZ : P.coefY;
        for (int w = tid; w < RT_QMAX * RT_N * 8; w += RT_THREADS) {
            const int q = w / (RT_N * 8), n = (w / 8) % RT_N, j = w % 8;
            const int k = n >> 1, co = n & 1;
            float v[4];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int i = q * RT_KF + 2 * j + h;
                double2 c = make_double2(0.0, 0.0);
                if (k < r && i < m) {
                    const double2 sc = side ? P.wscale[i] : make_double2(P.vscale[i], 0.0);
                    c = sc * coef[i * ldc + k];
                }
                v[2 * h] = co ? (float)c.y : (float)c.x;
                v[2 * h + 1] = co ? (float)c.x : -(float)c.y;
            }
            float4 big, small;
            split4(make_float4(v[0], v[1], v[2], v[3]), big, small);
            *reinterpret_cast<float4*>(reinterpret_cast<char*>(S->bb[q]) + sw128(n, j)) = big;
            *reinterpret_cast<float4*>(reinterpret_cast<char*>(S->bs[q]) + sw128(n, j)) = small;
        }
        fence_proxy_async();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = S->tmem;
    constexpr unsigned IDESC = idesc_tf32(RT_E, RT_N);

    if (warp == 0) {
        if (lane == 0) {   // ------------------------------ copies
            int g = 0;
            for (; g < nchunks; ++g) {
                const int s = g % RT_STAGES, q = g % Q;
                const long long e0 = (t0 + g / Q) * RT_E;
                if (g >= RT_STAGES &&
                    !wait_or_abort(&S->raw_empty[s], (unsigned)(g / RT_STAGES - 1) & 1u, abort))
                    break;
                const int nf = min(RT_KF, m - q * RT_KF);
                mbar_arrive_expect_tx(&S->raw_full[s], (unsigned)nf * RT_E * 8);
                for (int f = 0; f < nf; ++f)
                    bulk_copy_g2s(S->raw[s] + f * RT_E * 2, base + (size_t)(q * RT_KF + f) * fbytes + e0 * 8,
                                  RT_E * 8, &S->raw_full[s]);
            }
            for (int h = g - RT_STAGES > 0 ? g - RT_STAGES : 0; h < g; ++h)
                mbar_wait(&S->raw_full[h % RT_STAGES], (unsigned)(h / RT_STAGES) & 1u);
        }
    } else if (warp == 1) {
        if (lane == 0) {   // ------------------------------ MMAs
            int g = 0;
            for (; g < nchunks; ++g) {
                const int t = g / Q, q = g % Q, b = g & 1, acc = t & 1;
                if (q == 0 && t >= 2 &&
                    !wait_or_abort(&S->acc_empty[acc], (unsigned)(t / 2 - 1) & 1u, abort))
                    break;
                if (!wait_or_abort(&S->a_full[b], (unsigned)(g / 2) & 1u, abort)) break;
                tc_fence_after();
                // big.big of each K-chunk in its own accumulator, all corrections in one:
                // the tensor core truncates as it accumulates, so short sums of
                // like-sized terms keep the product at FP32 accuracy
                const unsigned dm = tmem + (unsigned)(acc * RT_ACC_STRIDE + q * RT_N);
                const unsigned dc = tmem + (unsigned)(acc * RT_ACC_STRIDE + RT_QMAX * RT_N);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const uint64_t ab = sdesc_k128(S->ab[b] + 8 * kk), as = sdesc_k128(S->as[b] + 8 * kk);
                    const uint64_t bb = sdesc_k128(S->bb[q] + 8 * kk), bs = sdesc_k128(S->bs[q] + 8 * kk);
                    mma_tf32(dm, ab, bb, IDESC, kk > 0 ? 1u : 0u);
                    mma_tf32(dc, ab, bs, IDESC, (q > 0 || kk > 0) ? 1u : 0u);
                    mma_tf32(dc, as, bb, IDESC, 1u);
                }
                mma_commit(&S->a_empty[b]);
                if (q == Q - 1) mma_commit(&S->acc_full[acc]);
            }
            if (g > 0) mbar_wait(&S->a_empty[(g - 1) & 1], (unsigned)((g - 1) / 2) & 1u);
        }
    } else if (warp < 2 + RT_XW) {   // ------------------- transpose + 3xTF32 split
        const int xt = tid - 64;
        for (int g = 0; g < nchunks; ++g) {
            const int s = g % RT_STAGES, q = g % Q, b = g & 1;
            bool ok = wait_or_abort(&S->raw_full[s], (unsigned)(g / RT_STAGES) & 1u, abort);
            if (ok && g >= 2) ok = wait_or_abort(&S->a_empty[b], (unsigned)(g / 2 - 1) & 1u, abort);
            if (!__all_sync(0xffffffffu, ok)) break;
            const float2* raw = reinterpret_cast<const float2*>(S->raw[s]);
            const int nf = min(RT_KF, m - q * RT_KF);
#pragma unroll
            for (int w = 0; w < RT_E * 8 / (32 * RT_XW); ++w) {
                const int item = w * 32 * RT_XW + xt;       // (element e, granule j): e fastest
                const int e = item % RT_E, j = item / RT_E;
                const float2 x0 = 2 * j < nf ? raw[(2 * j) * RT_E + e] : make_float2(0.f, 0.f);
                const float2 x1 = 2 * j + 1 < nf ? raw[(2 * j + 1) * RT_E + e] : make_float2(0.f, 0.f);
                float4 big, small;
                split4(make_float4(x0.x, x0.y, x1.x, x1.y), big, small);
                *reinterpret_cast<float4*>(reinterpret_cast<char*>(S->ab[b]) + sw128(e, j)) = big;
                *reinterpret_cast<float4*>(reinterpret_cast<char*>(S->as[b]) + sw128(e, j)) = small;
            }
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&S->a_full[b]);
                mbar_arrive(&S->raw_empty[s]);
            }
        }
    } else {   // ------------------------------------------- epilogue
        const int quarter = warp & 3, e = quarter * 32 + lane;
        const unsigned lane_base = (unsigned)(quarter * 32) << 16;
        const float2 bp = to_f(side ? st.beta_prev : conj_(st.beta_prev));
        const char* cur = reinterpret_cast<const char*>(side ? P.Ap[par] : P.Ahp[par]);
        const char* prv = reinterpret_cast<const char*>(side ? P.Ap[par ^ 1] : P.Ahp[par ^ 1]);
        float2 dot[RT_RMAX];
#pragma unroll
        for (int k = 0; k < RT_RMAX; ++k) dot[k] = make_float2(0.f, 0.f);
        for (int t = 0; t < nt; ++t) {
            const int acc = t & 1;
            if (!__all_sync(0xffffffffu, wait_or_abort(&S->acc_full[acc], (unsigned)(t / 2) & 1u, abort))) break;
            tc_fence_after();
            float y[RT_N];
            const unsigned ta = tmem + lane_base + (unsigned)(acc * RT_ACC_STRIDE);
#pragma unroll
            for (int h = 0; h < RT_N / 16; ++h)   // corrections first, then each chunk's main sum
                tmem_ld16(ta + (unsigned)(RT_QMAX * RT_N + 16 * h), *reinterpret_cast<float(*)[16]>(y + 16 * h));
            for (int q = 0; q < Q; ++q)
#pragma unroll
                for (int h = 0; h < RT_N / 16; ++h) {
                    float v[16];
                    tmem_ld16(ta + (unsigned)(q * RT_N + 16 * h), v);
#pragma unroll
                    for (int c = 0; c < 16; ++c) y[16 * h + c] += v[c];
                }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&S->acc_empty[acc]);
            const size_t el = (size_t)(t0 + t) * RT_E + e;
            const float2 c = reinterpret_cast<const float2*>(cur)[el];
            const float2 pv = reinterpret_cast<const float2*>(prv)[el];
            const float2 cv = c - bp * pv;
            const float2 last = reinterpret_cast<const float2*>(base + (size_t)m * fbytes)[el];
#pragma unroll
            for (int k = 0; k < RT_RMAX; ++k)
                if (k < r) {
                    const float2 o = make_float2(y[2 * k], y[2 * k + 1]);
                    reinterpret_cast<float2*>(base + (size_t)k * fbytes)[el] = o;
                    dot[k] = dot[k] + (side ? cdot(o, cv) : cdot(cv, o));
                }
            reinterpret_cast<float2*>(base + (size_t)r * fbytes)[el] = last;
        }
#pragma unroll
        for (int k = 0; k < RT_RMAX; ++k) {
            const float2 d = warp_sum(dot[k]);
            if (lane == 0) S->dots[quarter][k] = to_d(d);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem, RT_TMEM_COLS);
    }
    // per-CTA partials of the coupling dots, then the last CTA of this (slot, side)
    const int kind = side ? CNT_GEMM_W : CNT_GEMM_V;
    double2* pp = P.partials + (size_t)kind * PARTIAL_STRIDE;
    if (tid < RT_RMAX) {
        double2 a = make_double2(0.0, 0.0);
        for (int q = 0; q < RT_EW; ++q) a = a + S->dots[q][tid];
        pp[(size_t)blockIdx.x * RT_RMAX + tid] = a;
        __threadfence();
    }
    if (tid == 0 && *abort) atomicExch(err, 1);
    if (!last_block(P.counters + kind, gridDim.x)) return;
    if (tid < r) {
        double2 tot = make_double2(0.0, 0.0);
        for (unsigned b = 0; b < gridDim.x; ++b) tot = tot + __ldcg(pp + (size_t)b * RT_RMAX + tid);
        if (side) {
            P.H[tid * m + r] = (1.0 / st.rnorm) * tot;
            P.wscale[tid] = make_double2(1.0, 0.0);
        } else {
            P.H[r * m + tid] = cdiv(make_double2(st.rnorm, 0.0), st.rho) * tot;
            P.vscale[tid] = 1.0;
        }
    }
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

bool encode_tensor_map_f32(void* map, const void* base, int rank, const uint64_t* dims, const uint64_t* strides,
                           const uint32_t* box) {
    if (get_encode() != cudaSuccess || rank < 1 || rank > 5) return false;
    cuuint64_t d[5], st[4];
    cuuint32_t b[5], e[5];
    for (int i = 0; i < rank; ++i) {
        d[i] = dims[i];
        b[i] = box[i];
        e[i] = 1;
        if (i + 1 < rank) st[i] = strides[i];
    }
    return g_encode(reinterpret_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank,
                    const_cast<void*>(base), d, st, b, e, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool dots_tc_supported(int a, const void* X, const void* Y, size_t N) {
    return a > 0 && a <= 4 * TC_M && N > 0 && (2 * N) % TC_KT == 0 && ((uintptr_t)X & 15) == 0 &&
           ((uintptr_t)Y & 15) == 0 && get_encode() == cudaSuccess;
}

size_t dots_tc_scratch_doubles(int a) {
    return (size_t)((a + TC_M - 1) / TC_M) * num_sms() * TC_M * 2 * TC_NB_WIDE;
}

cudaError_t prepare_dots_tc() {
    std::call_once(g_prepare_once, [] {
        g_prepare_err = cudaFuncSetAttribute((const void*)dots_tc_kernel<TC_NB>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem<TC_NB>());
        if (g_prepare_err == cudaSuccess)
            g_prepare_err = cudaFuncSetAttribute((const void*)dots_tc_kernel<TC_NB_WIDE>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)tc_smem<TC_NB_WIDE>());
        if (g_prepare_err == cudaSuccess)
            g_prepare_err = cudaFuncSetAttribute((const void*)restart_tc_kernel,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RT_SMEM);
    });
    return g_prepare_err;
}

bool restart_tc_supported(int m, int two_nev, size_t N) {
    return m <= RT_QMAX * RT_KF && two_nev <= RT_RMAX && N % RT_E == 0 && N / RT_E >= 1;
}

cudaError_t launch_restart_tc(SlotState* states, const SlotPtrs* ptrs, int nslots, size_t N, int* err,
                              cudaStream_t st) {
    cudaError_t e = prepare_dots_tc();
    if (e != cudaSuccess) return e;
    if (!err) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_tc_err);
        if (e != cudaSuccess) return e;
        err = reinterpret_cast<int*>(p);
    }
    long long tiles = (long long)(N / RT_E);
    int nblk = (2 * num_sms()) / (2 * nslots);
    if (nblk < 1) nblk = 1;
    if (nblk > tiles) nblk = (int)tiles;
    if (nblk * RT_RMAX > PARTIAL_STRIDE) nblk = PARTIAL_STRIDE / RT_RMAX;
    restart_tc_kernel<<<dim3(nblk, 2 * nslots), RT_THREADS, RT_SMEM, st>>>(states, ptrs, N, err);
    count_launches(1);
    return cudaGetLastError();
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
    // up to 8 Y fields per launch in the narrow form (N = 16), more in the wide one
    // (N = 48), which reads X once for 24 fields
    const int nb = b > TC_NB ? TC_NB_WIDE : TC_NB;
    if ((size_t)ty * nblk * TC_M * 2 * nb > scratch_doubles) return cudaErrorInvalidValue;
    const int box_rows = ty > 1 ? TC_M : (a + 7) / 8 * 8;
    CUtensorMap mx;
    if (!encode_rows(&mx, X, N, a, x_stride, box_rows)) return cudaErrorInvalidValue;
    for (int j0 = 0; j0 < b; j0 += nb) {
        const int bb = b - j0 < nb ? b - j0 : nb;
        CUtensorMap my;
        const char* Yj = reinterpret_cast<const char*>(Y) + (size_t)j0 * y_stride;
        if (!encode_rows(&my, Yj, N, bb, y_stride, nb)) return cudaErrorInvalidValue;
        if (nb == TC_NB)
            dots_tc_kernel<TC_NB><<<dim3(nblk, ty), TC_THREADS, tc_smem<TC_NB>(), st>>>(mx, my, box_rows, tiles,
                                                                                     scratch, err);
        else
            dots_tc_kernel<TC_NB_WIDE><<<dim3(nblk, ty), TC_THREADS, tc_smem<TC_NB_WIDE>(), st>>>(
                mx, my, box_rows, tiles, scratch, err);
        count_launches(1);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        double2* Cj = conj_store ? Cm + (size_t)j0 * ldc : Cm + j0;
        dots_tc_reduce_kernel<<<(int)(((size_t)a * bb + 127) / 128), 128, 0, st>>>(a, bb, nb, nblk, scratch, Cj,
                                                                            ldc, conj_store);
        count_launches(1);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// ------------------------------------------------------------ bounded waits
// One thread waits, with the same bounded wait as the copy pipelines above, for
// a device word to become nonzero; status = 1 if the wait gave up.
namespace {
__global__ void flag_wait_kernel(const int* flag, int* status) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *status = flag_wait(flag) ? 0 : 1;
}
}  // namespace

cudaError_t set_wait_cycles_tc(long long cycles) { return set_wait_cycles_here(cycles); }

cudaError_t launch_flag_wait(const int* flag, int* status, cudaStream_t st) {
    flag_wait_kernel<<<1, 32, 0, st>>>(flag, status);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace lqcd
