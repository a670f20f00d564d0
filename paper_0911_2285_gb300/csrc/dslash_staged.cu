// Operator pair of one BiCG iteration (A p, A^+ phat and sigma = (phat, A p)
// for every slot of the batch, Sec. 2's two products per step), FP32, with
// every operand staged in shared memory by TMA tensor copies.
//
// A block (one per SM, one thread per site) owns a brick of 8 x BY x BZ x BT =
// 256 sites at a time and walks the brick's phases: for each running slot,
// first the field p (A p), then phat (A^+ phat). Shared memory holds
//   * the brick's links (two stored rows per direction) and the links of its
//     four backward faces, loaded once per brick and used by all 2k operators;
//   * two tile buffers; a tile is one field's interior plus its eight face
//     layers (nine 5-D tensor boxes), and the tile of the next phase streams
//     in while the current one is computed.
// Every spinor byte of a tile is read from L2 once per brick, so a field costs
// 1 + 2 (1/8 + 1/BY + 1/BZ + 1/BT) reads per site instead of the ~4-6 of the
// kernels that gather neighbours through L1, and the links are read once per
// brick instead of once per slot. The 8-site x rows are the 128-byte rows of
// the chunk-major field layout.
//
// All Krylov fields p, phat of the batch lie in one allocation, slot s at
// 6 s Krylov fields from its start (p, phat, Ap[2], Ahp[2]); one tensor map over
// it with a "chunk" dimension of 36 k_max float4 planes addresses any slot's
// field (chunk 36 s + 6 f + q).
//
// sigma, |phat|^2, |A p|^2: FP32 per thread (A p of the site is kept in
// registers from the p phase to the phat phase), warp sums accumulated per
// (warp, slot) in shared memory, one FP64 partial per (block, slot) and the last
// block adds them in block order (fixed grid: independent of the batch).
// Every mbarrier wait is bounded; a timeout sets the error word, waits
// (bounded) for the block's copies in flight and stops the block.
#include <cuda.h>

#include "async.cuh"
#include "dslash.cuh"
#include "kernels.cuh"
#include "reduce.cuh"

namespace lqcd {
namespace {

constexpr int SG_THREADS = 256;   // one thread per site of the brick
constexpr double SG_BREAK_TOL = 1e-14;

__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* tmap, int c0, int c1, int c2, int c3,
                                            int c4, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
        "%6}], [%7];" ::"r"(smem_addr(dst)),
        "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_addr(bar))
        : "memory");
}

template <int BY_, int BZ_, int BT_> struct SBrick {
    static constexpr int BX = 8, BY = BY_, BZ = BZ_, BT = BT_;
    static constexpr int NB = BX * BY * BZ * BT;
    static constexpr int FX = BY * BZ * BT, FY = BX * BZ * BT, FZ = BX * BY * BT, FT = BX * BY * BZ;
    // tile of one field (float4 offsets): interior [q][site], then faces [q][face site]
    static constexpr int T_XB = 6 * NB, T_XF = T_XB + 6 * FX, T_YB = T_XF + 6 * FX, T_YF = T_YB + 6 * FY,
                         T_ZB = T_YF + 6 * FY, T_ZF = T_ZB + 6 * FZ, T_TB = T_ZF + 6 * FZ, T_TF = T_TB + 6 * FT,
                         T_END = T_TF + 6 * FT;
    // links: interior [mu*3 + q][site], then the backward faces [q][face site] of mu = 0..3
    static constexpr int L_XB = 12 * NB, L_YB = L_XB + 3 * FX, L_ZB = L_YB + 3 * FY, L_TB = L_ZB + 3 * FZ,
                         L_END = L_TB + 3 * FT;
    static constexpr unsigned TILE_BYTES = T_END * 16u, LINK_BYTES = L_END * 16u;
    static constexpr size_t SMEM = (size_t)(L_END + 2 * T_END) * 16 + 64;   // + three mbarriers
    static_assert(NB == SG_THREADS, "one site per thread");
    // every region starts on a 128-byte boundary (8 float4): TMA destinations
    static_assert(FX % 8 == 0 && FY % 8 == 0 && FZ % 8 == 0 && FT % 8 == 0, "");
};

// Tensor maps: [0..4] spinor tiles (interior, x, y, z, t faces; 6 chunks),
// [5..9] links (interior 12 chunks; x, y, z, t backward faces, 3 chunks).
// Nine boxes per tile: the TMA unit's cost per copy makes a few large boxes
// much cheaper than one box per chunk.
struct StageMaps {
    CUtensorMap m[10];
};

// 6 float4 of a site from a tile region with chunk stride st.
__device__ __forceinline__ void tile_load(const float4* t, int st, float2 (&v)[12]) {
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const float4 a = t[q * st];
        v[2 * q] = make_float2(a.x, a.y);
        v[2 * q + 1] = make_float2(a.z, a.w);
    }
}

__device__ __forceinline__ void link_load(const float4* b, int st, float2 (&m)[3][3]) {
    const float4 a = b[0], c = b[st], d = b[2 * st];
    m[0][0] = make_float2(a.x, a.y); m[0][1] = make_float2(a.z, a.w);
    m[0][2] = make_float2(c.x, c.y); m[1][0] = make_float2(c.z, c.w);
    m[1][1] = make_float2(d.x, d.y); m[1][2] = make_float2(d.z, d.w);
    m[2][0] = cross_conj(m[0][1], m[1][2], m[0][2], m[1][1]);
    m[2][1] = cross_conj(m[0][2], m[1][0], m[0][0], m[1][2]);
    m[2][2] = cross_conj(m[0][0], m[1][1], m[0][1], m[1][0]);
}

// Per-thread neighbour addressing (independent of the brick): tile offset and
// chunk stride of the forward (2 mu) and backward (2 mu + 1) neighbour, and of
// the backward link U_mu(x - mu).
template <class B> struct SAddr {
    int toff[8], tst[8], loff[4], lst[4];
    __device__ __forceinline__ SAddr(int tid) {
        const int x = tid & 7, y = (tid >> 3) % B::BY, z = (tid / (8 * B::BY)) % B::BZ,
                  t = tid / (8 * B::BY * B::BZ);
        const int fidx[4] = {y + B::BY * (z + B::BZ * t), x + 8 * (z + B::BZ * t), x + 8 * (y + B::BY * t),
                             x + 8 * (y + B::BY * z)};
        const int ls[4] = {1, 8, 8 * B::BY, 8 * B::BY * B::BZ};
        const bool lo[4] = {x == 0, y == 0, z == 0, t == 0};
        const bool hi[4] = {x == 7, y == B::BY - 1, z == B::BZ - 1, t == B::BT - 1};
        const int fsz[4] = {B::FX, B::FY, B::FZ, B::FT};
        const int tf[4] = {B::T_XF, B::T_YF, B::T_ZF, B::T_TF};
        const int tb[4] = {B::T_XB, B::T_YB, B::T_ZB, B::T_TB};
        const int lb[4] = {B::L_XB, B::L_YB, B::L_ZB, B::L_TB};
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            toff[2 * mu] = hi[mu] ? tf[mu] + fidx[mu] : tid + ls[mu];
            tst[2 * mu] = hi[mu] ? fsz[mu] : B::NB;
            toff[2 * mu + 1] = lo[mu] ? tb[mu] + fidx[mu] : tid - ls[mu];
            tst[2 * mu + 1] = lo[mu] ? fsz[mu] : B::NB;
            loff[mu] = lo[mu] ? lb[mu] + fidx[mu] : mu * 3 * B::NB + tid - ls[mu];
            lst[mu] = lo[mu] ? fsz[mu] : B::NB;
        }
    }
};

// acc += hop in direction mu of D_hop psi (DAG = false: projectors 1 - gamma
// forward, 1 + gamma backward) or of D_hop^+ psi, from a staged tile and links.
template <int MU, bool DAG, class B>
__device__ __forceinline__ void staged_dir(const float4* tile, const float4* lk, const SAddr<B>& ad, int tid,
                                           float2 (&acc)[12]) {
    constexpr int SF = DAG ? +1 : -1;
    // both neighbours' spinors and links first (shared-memory latency overlaps)
    float2 pf[12], pb[12], uf[3][3], ub[3][3], h[2][3], uh[2][3];
    tile_load(tile + ad.toff[2 * MU], ad.tst[2 * MU], pf);
    tile_load(tile + ad.toff[2 * MU + 1], ad.tst[2 * MU + 1], pb);
    link_load(lk + MU * 3 * B::NB + tid, B::NB, uf);
    link_load(lk + ad.loff[MU], ad.lst[MU], ub);
    project<MU, SF>(pf, h);
    su3_mul(uf, h, uh);
    reconstruct<MU, SF>(uh, acc);
    project<MU, -SF>(pb, h);
    su3_dag_mul(ub, h, uh);
    reconstruct<MU, -SF>(uh, acc);
}

template <bool DAG, class B>
__device__ __forceinline__ void staged_hop(const float4* tile, const float4* lk, const SAddr<B>& ad, int tid,
                                           float2 (&acc)[12]) {
#pragma unroll
    for (int c = 0; c < 12; ++c) acc[c] = make_float2(0.f, 0.f);
    staged_dir<0, DAG, B>(tile, lk, ad, tid, acc);
    staged_dir<1, DAG, B>(tile, lk, ad, tid, acc);
    staged_dir<2, DAG, B>(tile, lk, ad, tid, acc);
    staged_dir<3, DAG, B>(tile, lk, ad, tid, acc);
}

__device__ __forceinline__ int wrap(int c, int L) { return c < 0 ? c + L : (c >= L ? c - L : c); }

template <int BY, int BZ, int BT>
__global__ void __launch_bounds__(SG_THREADS, 1)
    matvec_staged_kernel(const __grid_constant__ StageMaps maps, Geom g, float kappa, SlotState* states,
                         const SlotPtrs* ptrs, int nslots, int* err) {
    using B = SBrick<BY, BZ, BT>;
    extern __shared__ __align__(1024) float4 sg_sm[];
    float4* lk = sg_sm;
    float4* tbuf0 = sg_sm + B::L_END;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sg_sm + B::L_END + 2 * B::T_END);   // tile 0, tile 1, links
    __shared__ float4 acc_sm[MAX_SLOTS][SG_THREADS / 32];   // (Re sigma, Im sigma, |phat|^2, |Ap|^2)
    __shared__ int run_list[MAX_SLOTS];
    __shared__ int nrun_s;
    __shared__ unsigned par_mask_s;
    __shared__ int issued[3];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        int n = 0;
        unsigned pm = 0;
        for (int j = 0; j < nslots; ++j)
            if (states[j].status == ST_RUNNING && !states[j].stab) {
                run_list[n++] = j;
                pm |= (unsigned)(states[j].iter & 1) << j;
            }
        nrun_s = n;
        par_mask_s = pm;
        for (int i = 0; i < 3; ++i) { mbar_init(&bars[i], 1); issued[i] = 0; }
        mbar_init_fence();
    }
    if (tid < MAX_SLOTS * (SG_THREADS / 32))
        acc_sm[tid / (SG_THREADS / 32)][tid % (SG_THREADS / 32)] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    const int nrun = nrun_s;
    const unsigned pmask = par_mask_s;
    if (nrun == 0) return;   // uniform over the grid: nothing arrives, the counter stays zero
    const int nph = 2 * nrun;   // phases per brick
    const int Lx = g.L[0], Ly = g.L[1], Lz = g.L[2], Lt = g.L[3];
    const int nbx = Lx / 8, nby = Ly / BY, nbz = Lz / BZ;
    const int nbricks = nbx * nby * nbz * (Lt / BT);

    auto origin = [&](int br, int (&o)[4]) {
        o[0] = (br % nbx) * 8; br /= nbx;
        o[1] = (br % nby) * BY; br /= nby;
        o[2] = (br % nbz) * BZ;
        o[3] = (br / nbz) * BT;
    };
    // thread 0: the tile of phase k of brick br into buffer b
    auto issue_tile = [&](int b, int br, int k) {
        int o[4];
        origin(br, o);
        const int cq = 36 * run_list[k >> 1] + 6 * (k & 1);
        float4* t = tbuf0 + b * B::T_END;
        uint64_t* bar = &bars[b];
        mbar_arrive_expect_tx(bar, B::TILE_BYTES);
        issued[b] += 1;
        tma_load_5d(t, &maps.m[0], 4 * o[0], o[1], o[2], o[3], cq, bar);
        tma_load_5d(t + B::T_XB, &maps.m[1], 4 * wrap(o[0] - 1, Lx), o[1], o[2], o[3], cq, bar);
        tma_load_5d(t + B::T_XF, &maps.m[1], 4 * wrap(o[0] + 8, Lx), o[1], o[2], o[3], cq, bar);
        tma_load_5d(t + B::T_YB, &maps.m[2], 4 * o[0], wrap(o[1] - 1, Ly), o[2], o[3], cq, bar);
        tma_load_5d(t + B::T_YF, &maps.m[2], 4 * o[0], wrap(o[1] + BY, Ly), o[2], o[3], cq, bar);
        tma_load_5d(t + B::T_ZB, &maps.m[3], 4 * o[0], o[1], wrap(o[2] - 1, Lz), o[3], cq, bar);
        tma_load_5d(t + B::T_ZF, &maps.m[3], 4 * o[0], o[1], wrap(o[2] + BZ, Lz), o[3], cq, bar);
        tma_load_5d(t + B::T_TB, &maps.m[4], 4 * o[0], o[1], o[2], wrap(o[3] - 1, Lt), cq, bar);
        tma_load_5d(t + B::T_TF, &maps.m[4], 4 * o[0], o[1], o[2], wrap(o[3] + BT, Lt), cq, bar);
    };
    auto issue_links = [&](int br) {
        int o[4];
        origin(br, o);
        uint64_t* bar = &bars[2];
        mbar_arrive_expect_tx(bar, B::LINK_BYTES);
        issued[2] += 1;
        tma_load_5d(lk, &maps.m[5], 4 * o[0], o[1], o[2], o[3], 0, bar);
        tma_load_5d(lk + B::L_XB, &maps.m[6], 4 * wrap(o[0] - 1, Lx), o[1], o[2], o[3], 0, bar);
        tma_load_5d(lk + B::L_YB, &maps.m[7], 4 * o[0], wrap(o[1] - 1, Ly), o[2], o[3], 3, bar);
        tma_load_5d(lk + B::L_ZB, &maps.m[8], 4 * o[0], o[1], wrap(o[2] - 1, Lz), o[3], 6, bar);
        tma_load_5d(lk + B::L_TB, &maps.m[9], 4 * o[0], o[1], o[2], wrap(o[3] - 1, Lt), 9, bar);
    };

    const int br0 = blockIdx.x;
    if (tid == 0 && br0 < nbricks) {
        issue_links(br0);
        issue_tile(0, br0, 0);
        if (nph > 1) issue_tile(1, br0, 1);
        else if (br0 + (int)gridDim.x < nbricks) issue_tile(1, br0 + gridDim.x, 0);
    }
    const SAddr<B> ad(tid);
    const float k = kappa;
    const int sx = tid & 7, sy = (tid >> 3) % BY, sz = (tid / (8 * BY)) % BZ, st_ = tid / (8 * BY * BZ);
    bool ok = true;
    int gp = 0, nit = 0;
    float2 ap[12];   // A p of this site, from the p phase to the phat phase
    for (int br = br0; br < nbricks && ok; br += gridDim.x, ++nit) {
        int o[4];
        origin(br, o);
        const int s = (o[0] + sx) + Lx * ((o[1] + sy) + Ly * ((o[2] + sz) + Lz * (o[3] + st_)));
        if (!mbar_wait(&bars[2], nit & 1)) ok = false;
        for (int kk = 0; kk < nph; ++kk, ++gp) {
            const int b = gp & 1;
            // a thread whose wait gave up computes on whatever the buffer holds; the
            // block stops at the barrier below and the host discards the launch
            if (ok && !mbar_wait(&bars[b], (gp >> 1) & 1)) ok = false;
            const float4* tile = tbuf0 + b * B::T_END;
            const int slot = run_list[kk >> 1];
            const SlotPtrs& P = ptrs[slot];
            const int par = (pmask >> slot) & 1;
            float2 acc[12], self[12];
            tile_load(tile + tid, B::NB, self);
            if ((kk & 1) == 0) {
                staged_hop<false, B>(tile, lk, ad, tid, acc);
#pragma unroll
                for (int c = 0; c < 12; ++c) ap[c] = self[c] - k * acc[c];
#pragma unroll
                for (int q = 0; q < 6; ++q)
                    __stcs(reinterpret_cast<float4*>(P.Ap[par]) + (size_t)q * g.V + s,
                           make_float4(ap[2 * q].x, ap[2 * q].y, ap[2 * q + 1].x, ap[2 * q + 1].y));
            } else {
                staged_hop<true, B>(tile, lk, ad, tid, acc);
                Acc<float> sacc;
#pragma unroll
                for (int c = 0; c < 12; ++c) {
                    acc[c] = self[c] - k * acc[c];
                    sacc.z = sacc.z + cdot(self[c], ap[c]);
                    sacc.a += abs2(self[c]);
                    sacc.b += abs2(ap[c]);
                }
#pragma unroll
                for (int q = 0; q < 6; ++q)
                    __stcs(reinterpret_cast<float4*>(P.Ahp[par]) + (size_t)q * g.V + s,
                           make_float4(acc[2 * q].x, acc[2 * q].y, acc[2 * q + 1].x, acc[2 * q + 1].y));
                const float2 z = warp_sum(sacc.z);
                const float2 ab = warp_sum(make_float2(sacc.a, sacc.b));
                if (lane == 0) {
                    const float4 t = acc_sm[slot][warp];
                    acc_sm[slot][warp] = make_float4(t.x + z.x, t.y + z.y, t.z + ab.x, t.w + ab.y);
                }
            }
            // every thread is done with tile b (and, after the last phase, the links);
            // a timeout anywhere stops the whole block here
            if (!__syncthreads_and(ok)) { ok = false; break; }
            if (tid == 0) {
                int br2 = br, k2 = kk + 2;
                while (k2 >= nph) { k2 -= nph; br2 += gridDim.x; }
                if (br2 < nbricks) issue_tile(b, br2, k2);
                if (kk == nph - 1 && br + (int)gridDim.x < nbricks) issue_links(br + gridDim.x);
            }
        }
    }
    ok = __syncthreads_and(ok);
    if (!ok) {
        // timed out: report, wait (bounded) for this block's copies in flight so
        // none lands in shared memory after the block exits, and stop
        if (tid == 0) {
            atomicExch(err, 1);
            for (int i = 0; i < 3; ++i)
                if (issued[i] > 0) mbar_wait(&bars[i], (unsigned)((issued[i] - 1) & 1));
        }
        __syncthreads();
        return;
    }
    // one FP64 partial per (block, slot), warps added in order
    if (tid < nrun) {
        const int slot = run_list[tid];
        double2 z = make_double2(0.0, 0.0), ab = make_double2(0.0, 0.0);
        for (int w = 0; w < SG_THREADS / 32; ++w) {
            const float4 t = acc_sm[slot][w];
            z = z + make_double2(t.x, t.y);
            ab = ab + make_double2(t.z, t.w);
        }
        double2* pp = ptrs[slot].partials + (size_t)CNT_MATVEC * PARTIAL_STRIDE + (size_t)blockIdx.x * 2;
        pp[0] = z;
        pp[1] = ab;
        __threadfence();
    }
    if (!last_block(ptrs[0].counters + CNT_GROUP, gridDim.x)) return;
    for (int i = warp; i < nrun; i += SG_THREADS / 32) {
        const int slot = run_list[i];
        SlotState& st = states[slot];
        const double2* pp = ptrs[slot].partials + (size_t)CNT_MATVEC * PARTIAL_STRIDE;
        double2 z = make_double2(0.0, 0.0), ab = make_double2(0.0, 0.0);
        for (int b = lane; b < (int)gridDim.x; b += 32) {
            z = z + __ldcg(pp + 2 * b);
            ab = ab + __ldcg(pp + 2 * b + 1);
        }
        z = warp_sum(z);
        ab = warp_sum(ab);
        if (lane == 0) {
            st.sigma = z;
            st.phat_norm = sqrt(ab.x);
            st.ap_norm = sqrt(ab.y);
            st.matvecs += 2;
            if (!(cabs_(st.sigma) >= SG_BREAK_TOL * st.phat_norm * st.ap_norm) || cabs2(st.sigma) == 0.0) {
                st.status = ST_BREAKDOWN;
            } else {
                st.alpha = cdiv(st.rho, st.sigma);
            }
        }
    }
}

using Brick8442 = SBrick<4, 4, 2>;

bool encode5(CUtensorMap* m, const void* base, const Geom& g, int nchunks, int b0, int b1, int b2, int b3, int b4) {
    cuuint64_t dims[5] = {(cuuint64_t)4 * g.L[0], (cuuint64_t)g.L[1], (cuuint64_t)g.L[2], (cuuint64_t)g.L[3],
                          (cuuint64_t)nchunks};
    cuuint64_t strides[4] = {(cuuint64_t)16 * g.L[0], (cuuint64_t)16 * g.L[0] * g.L[1],
                             (cuuint64_t)16 * g.L[0] * g.L[1] * g.L[2], (cuuint64_t)16 * g.V};
    cuuint32_t box[5] = {(cuuint32_t)b0, (cuuint32_t)b1, (cuuint32_t)b2, (cuuint32_t)b3, (cuuint32_t)b4};
    return encode_tensor_map_f32(m, base, 5, dims, strides, box);
}

}  // namespace

bool staged_variant_ok(const Geom& g) {
    using B = Brick8442;
    return g.L[0] % 8 == 0 && g.L[1] % B::BY == 0 && g.L[2] % B::BZ == 0 && g.L[3] % B::BT == 0;
}

size_t staged_maps_bytes() { return sizeof(StageMaps); }

cudaError_t prepare_staged(const Geom& g, const void* krylov_base, int kmax, const void* links32, void* maps_out) {
    using B = Brick8442;
    if (!staged_variant_ok(g) || ((uintptr_t)krylov_base & 15) || ((uintptr_t)links32 & 15))
        return cudaErrorInvalidValue;
    StageMaps* M = reinterpret_cast<StageMaps*>(maps_out);
    const int nk = 36 * kmax;
    bool ok = encode5(&M->m[0], krylov_base, g, nk, 32, B::BY, B::BZ, B::BT, 6) &&
              encode5(&M->m[1], krylov_base, g, nk, 4, B::BY, B::BZ, B::BT, 6) &&
              encode5(&M->m[2], krylov_base, g, nk, 32, 1, B::BZ, B::BT, 6) &&
              encode5(&M->m[3], krylov_base, g, nk, 32, B::BY, 1, B::BT, 6) &&
              encode5(&M->m[4], krylov_base, g, nk, 32, B::BY, B::BZ, 1, 6) &&
              encode5(&M->m[5], links32, g, 12, 32, B::BY, B::BZ, B::BT, 12) &&
              encode5(&M->m[6], links32, g, 12, 4, B::BY, B::BZ, B::BT, 3) &&
              encode5(&M->m[7], links32, g, 12, 32, 1, B::BZ, B::BT, 3) &&
              encode5(&M->m[8], links32, g, 12, 32, B::BY, 1, B::BT, 3) &&
              encode5(&M->m[9], links32, g, 12, 32, B::BY, B::BZ, 1, 3);
    if (!ok) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(matvec_staged_kernel<B::BY, B::BZ, B::BT>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B::SMEM);
}

cudaError_t launch_matvec_staged(const Geom& g, const void* maps, double kappa, SlotState* states,
                                 const SlotPtrs* ptrs, int nslots, int* err, int nsm, cudaStream_t s) {
    using B = Brick8442;
    if (!staged_variant_ok(g) || nslots > MAX_SLOTS || nsm < 1) return cudaErrorInvalidValue;
    const int nbricks = (g.L[0] / 8) * (g.L[1] / B::BY) * (g.L[2] / B::BZ) * (g.L[3] / B::BT);
    int grid = nbricks < nsm ? nbricks : nsm;
    if (grid > PARTIAL_STRIDE / 2) grid = PARTIAL_STRIDE / 2;
    matvec_staged_kernel<B::BY, B::BZ, B::BT><<<grid, SG_THREADS, B::SMEM, s>>>(
        *reinterpret_cast<const StageMaps*>(maps), g, (float)kappa, states, ptrs, nslots, err);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace lqcd
