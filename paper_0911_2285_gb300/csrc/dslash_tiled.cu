// Plane-streaming operator pair (FP32 fields, two-row links): A p and A^+ phat
// with the fused sigma = (phat, A p), for lattices whose x-y planes tile into
// row blocks.
//
// A CTA owns YB consecutive y-rows of the (x, y) plane at one z and sweeps t
// through a segment. Shared memory holds a four-deep ring of t-planes of its
// rows plus one halo row on each side in y (both fields of the pair), filled by
// TMA bulk copies that complete on mbarriers, and a buffer with the z-1, z+1
// rows of the current t. While step t computes from planes t-1, t, t+1, the
// plane t+2 streams in. Each spinor thus leaves L2 about (YB+2)/YB + 2 times per
// field instead of nine, and one thread applies both operators at its site so
// every link load serves two products. All mbarrier waits are bounded: a
// timeout sets an error word for the host and the CTA stops issuing work.
#include <stdint.h>

#include "async.cuh"
#include "dslash.cuh"
#include "kernels.cuh"
#include "reduce.cuh"

namespace lqcd {
namespace {

constexpr int TILE_MAX_THREADS = 256;
struct SmemTile {
    const float4* s;   // base of one plane-row block: [6 chunks][ld sites]
    int ld;
    __device__ __forceinline__ void load(int i, float2 (&v)[12]) const {
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            float4 t = s[q * ld + i];
            v[2 * q] = make_float2(t.x, t.y);
            v[2 * q + 1] = make_float2(t.z, t.w);
        }
    }
};

// One direction of both operators at a site, neighbours given as shared-memory
// spinors (forward fp/fh, backward bp/bh) and links from global memory.
template <int MU>
__device__ __forceinline__ void pair_hop(const LinksF& U, int s, int sb, const float2 (&pf)[12], const float2 (&hf)[12],
                                         const float2 (&pb)[12], const float2 (&hb)[12], float2 (&a)[12],
                                         float2 (&b)[12]) {
    float2 h[2][3], uh[2][3], u[3][3];
    U.load(MU, s, u);
    project<MU, -1>(pf, h);
    su3_mul(u, h, uh);
    reconstruct<MU, -1>(uh, a);
    project<MU, +1>(hf, h);
    su3_mul(u, h, uh);
    reconstruct<MU, +1>(uh, b);
    U.load(MU, sb, u);
    project<MU, +1>(pb, h);
    su3_dag_mul(u, h, uh);
    reconstruct<MU, +1>(uh, a);
    project<MU, -1>(hb, h);
    su3_dag_mul(u, h, uh);
    reconstruct<MU, -1>(uh, b);
}

__global__ void __launch_bounds__(TILE_MAX_THREADS, 1)
    matvec_tiled_kernel(Geom g, TileGeom tg, const float4* links, float kappa, SlotState* states,
                        const SlotPtrs* ptrs, int* err) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int Lx = g.L[0], Ly = g.L[1], Lz = g.L[2], Lt = g.L[3], V = g.V, plane = Lx * Ly;
    const int YB = tg.YB, rows = YB + 2, nsites = YB * Lx, rs = rows * Lx;
    int bid = blockIdx.x;
    const int slot = bid % tg.nslots;
    bid /= tg.nslots;
    const int yb = bid % tg.nyb;
    bid /= tg.nyb;
    const int z = bid % Lz;
    const int seg = bid / Lz;
    SlotState& st = states[slot];
    const SlotPtrs& P = ptrs[slot];
    if (st.status != ST_RUNNING || st.stab) return;
    const int par = st.iter & 1;
    const float4* src[2] = {reinterpret_cast<const float4*>(P.p), reinterpret_cast<const float4*>(P.phat)};
    float4* dst[2] = {reinterpret_cast<float4*>(P.Ap[par]), reinterpret_cast<float4*>(P.Ahp[par])};

    float4* ring = reinterpret_cast<float4*>(smem);          // [4][2 fields][6][rs]
    float4* zbuf = ring + 4 * 2 * 6 * rs;                    // [2 dirs][2 fields][6][nsites]
    uint64_t* bars = reinterpret_cast<uint64_t*>(zbuf + 2 * 2 * 6 * nsites);   // 4 ring + 1 z

    const int y0 = yb * YB;
    const int t0 = seg * tg.tseg;
    const int t1 = min(t0 + tg.tseg, Lt);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    __shared__ int issued[5];   // phases started on each barrier (copies possibly in flight)
    if (threadIdx.x == 0) {
        for (int i = 0; i < 5; ++i) { mbar_init(&bars[i], 1); issued[i] = 0; }
        mbar_init_fence();
    }
    __syncthreads();

    // Plane tt (periodic) into ring slot (tt - t0 + 1) & 3, issued by warp 0.
    auto load_plane = [&](int tt) {
        const int tm = ((tt % Lt) + Lt) % Lt;
        const int rslot = (tt - t0 + 1) & 3;
        uint64_t* bar = &bars[rslot];
        if (lane == 0) { mbar_arrive_expect_tx(bar, (unsigned)(2 * 6 * rows * Lx * 16)); issued[rslot] += 1; }
        __syncwarp();
        const int pbase = plane * (z + Lz * tm);
        for (int c = lane; c < 2 * 6 * rows; c += 32) {
            const int f = c / (6 * rows), q = (c / rows) % 6, r = c % rows;
            const int yy = (y0 - 1 + r + Ly) % Ly;
            const float4* s = src[f] + (size_t)q * V + pbase + yy * Lx;
            float4* d = ring + ((size_t)(rslot * 2 + f) * 6 + q) * rs + r * Lx;
            bulk_copy_g2s(d, s, (unsigned)(Lx * 16), bar);
        }
    };
    // Rows y0..y0+YB-1 of planes (z-1, t) and (z+1, t) into zbuf.
    auto load_z = [&](int tt) {
        uint64_t* bar = &bars[4];
        if (lane == 0) { mbar_arrive_expect_tx(bar, (unsigned)(2 * 2 * 6 * nsites * 16)); issued[4] += 1; }
        __syncwarp();
        for (int c = lane; c < 2 * 2 * 6; c += 32) {
            const int d = c / 12, f = (c / 6) % 2, q = c % 6;
            const int zz = (z + (d ? 1 : -1) + Lz) % Lz;
            const float4* s = src[f] + (size_t)q * V + plane * (zz + Lz * tt) + y0 * Lx;
            float4* dd = zbuf + ((size_t)(d * 2 + f) * 6 + q) * nsites;
            bulk_copy_g2s(dd, s, (unsigned)(nsites * 16), bar);
        }
    };

    if (warp == 0) {
        load_plane(t0 - 1);
        load_plane(t0);
        load_plane(t0 + 1);
    }
    LinksF U{links, V};
    const float k = kappa;
    Acc<float> sacc;
    bool ok = true;
    const int tid = threadIdx.x;
    const int x = tid % Lx, yy = tid / Lx;
    for (int tt = t0; tt < t1; ++tt) {
        // step tt-1 finished reading the slot of plane tt-2 and zbuf; a timeout
        // anywhere in the CTA stops every thread here (uniform decision)
        if (!__syncthreads_and(ok)) { ok = false; break; }
        if (warp == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            if (tt + 2 <= t1) load_plane(tt + 2);
            load_z(tt);
        }
        // planes tt-1, tt, tt+1 (the first step waits for all three)
        for (int d = (tt == t0 ? -1 : 1); d <= 1; ++d) {
            const int rslot = (tt + d - t0 + 1) & 3;
            const unsigned parity = ((tt + d - t0 + 1) >> 2) & 1;
            if (!mbar_wait(&bars[rslot], parity)) ok = false;
        }
        if (!__syncthreads_and(ok)) { ok = false; break; }
        if (tid < nsites) {
            const int sc = (tt - t0 + 1) & 3, sn = (tt - t0 + 2) & 3, sp = (tt - t0) & 3;
            const int s = x + Lx * (y0 + yy) + plane * (z + Lz * tt);
            auto tile = [&](int rslot, int f) { return SmemTile{ring + (size_t)(rslot * 2 + f) * 6 * rs, rs}; };
            const int ic = (yy + 1) * Lx + x;                 // own site in a ring plane
            const int xf = (x + 1) % Lx, xb = (x + Lx - 1) % Lx;
            float2 a[12], b[12];
#pragma unroll
            for (int c = 0; c < 12; ++c) { a[c] = make_float2(0.f, 0.f); b[c] = a[c]; }
            const Nbr nb(g, s);
            {
                float2 pf[12], hf[12], pb[12], hb[12];
                tile(sc, 0).load((yy + 1) * Lx + xf, pf); tile(sc, 1).load((yy + 1) * Lx + xf, hf);
                tile(sc, 0).load((yy + 1) * Lx + xb, pb); tile(sc, 1).load((yy + 1) * Lx + xb, hb);
                pair_hop<0>(U, s, nb.b[0], pf, hf, pb, hb, a, b);
            }
            {
                float2 pf[12], hf[12], pb[12], hb[12];
                tile(sc, 0).load((yy + 2) * Lx + x, pf); tile(sc, 1).load((yy + 2) * Lx + x, hf);
                tile(sc, 0).load(yy * Lx + x, pb); tile(sc, 1).load(yy * Lx + x, hb);
                pair_hop<1>(U, s, nb.b[1], pf, hf, pb, hb, a, b);
            }
            {
                float2 pf[12], hf[12], pb[12], hb[12];
                tile(sn, 0).load(ic, pf); tile(sn, 1).load(ic, hf);
                tile(sp, 0).load(ic, pb); tile(sp, 1).load(ic, hb);
                pair_hop<3>(U, s, nb.b[3], pf, hf, pb, hb, a, b);
            }
            if (!mbar_wait(&bars[4], (tt - t0) & 1)) ok = false;
            if (ok) {
                float2 pf[12], hf[12], pb[12], hb[12];
                const int iz = yy * Lx + x;
                SmemTile{zbuf + (size_t)(1 * 2 + 0) * 6 * nsites, nsites}.load(iz, pf);
                SmemTile{zbuf + (size_t)(1 * 2 + 1) * 6 * nsites, nsites}.load(iz, hf);
                SmemTile{zbuf + (size_t)(0 * 2 + 0) * 6 * nsites, nsites}.load(iz, pb);
                SmemTile{zbuf + (size_t)(0 * 2 + 1) * 6 * nsites, nsites}.load(iz, hb);
                pair_hop<2>(U, s, nb.b[2], pf, hf, pb, hb, a, b);
                float2 ps[12], hs[12];
                tile(sc, 0).load(ic, ps);
                tile(sc, 1).load(ic, hs);
#pragma unroll
                for (int c = 0; c < 12; ++c) {
                    a[c] = ps[c] - k * a[c];
                    b[c] = hs[c] - k * b[c];
                    sacc.z = sacc.z + cdot(hs[c], a[c]);
                    sacc.a += abs2(hs[c]);
                    sacc.b += abs2(a[c]);
                }
                Field<float>::store(dst[0], V, s, a);
                Field<float>::store(dst[1], V, s, b);
            }
        } else {
            if (!mbar_wait(&bars[4], (tt - t0) & 1)) ok = false;
        }
    }
    ok = __syncthreads_and(ok);
    if (!ok) {
        // Timed out: report, wait (bounded) for this CTA's copies in flight so
        // none lands in shared memory after the CTA exits, and stop.
        if (threadIdx.x == 0) {
            atomicExch(err, 1);
            for (int i = 0; i < 5; ++i)
                if (issued[i] > 0) mbar_wait(&bars[i], (unsigned)((issued[i] - 1) & 1));
        }
        __syncthreads();
        return;
    }
    float2 v[2];
    sacc.to(v);
    double2 tot[2];
    const unsigned nblk = (unsigned)(tg.nyb * Lz * tg.nseg);
    const unsigned myblk = (unsigned)(yb + tg.nyb * (z + Lz * seg));
    if (reduce_slot<2>(P, CNT_MATVEC, v, tot, nblk, myblk) && threadIdx.x == 0) {
        st.sigma = tot[0];
        st.phat_norm = sqrt(tot[1].x);
        st.ap_norm = sqrt(tot[1].y);
        st.matvecs += 2;
        if (!(cabs_(st.sigma) >= 1e-14 * st.phat_norm * st.ap_norm) || cabs2(st.sigma) == 0.0) {
            st.status = ST_BREAKDOWN;
        } else {
            st.alpha = cdiv(st.rho, st.sigma);
        }
    }
}

}  // namespace

size_t tiled_smem_bytes(int Lx, int YB) {
    return (size_t)4 * 2 * 6 * (YB + 2) * Lx * 16 + (size_t)2 * 2 * 6 * YB * Lx * 16 + 5 * 8;
}

bool tiled_plan(const Geom& g, int nslots, TileGeom* tg) {
    const int Lx = g.L[0], Ly = g.L[1], Lz = g.L[2], Lt = g.L[3];
    int best = 0;
    for (int yb = 1; yb <= Ly; ++yb) {
        if (Ly % yb) continue;
        if (yb * Lx > TILE_MAX_THREADS) continue;
        if (tiled_smem_bytes(Lx, yb) > 220 * 1024) continue;
        best = yb;
    }
    if (best == 0 || best * Lx < 64 || Lt < 3 || Lz < 2) return false;
    tg->YB = best;
    tg->nyb = Ly / best;
    tg->nslots = nslots;
    const int tiles = nslots * Lz * tg->nyb;
    int nseg = (2 * 152 + tiles - 1) / tiles;
    if (nseg < 1) nseg = 1;
    while (nseg > 1 && (Lt + nseg - 1) / nseg < 8) --nseg;
    tg->tseg = (Lt + nseg - 1) / nseg;
    tg->nseg = (Lt + tg->tseg - 1) / tg->tseg;
    if (tg->nyb * Lz * tg->nseg > PARTIAL_STRIDE / 2) return false;
    return true;
}

cudaError_t prepare_tiled_kernel() {
    return cudaFuncSetAttribute((const void*)matvec_tiled_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                220 * 1024);
}

cudaError_t launch_matvec_tiled(const Geom& g, const TileGeom& tg, const void* links32, double kappa,
                                SlotState* states, const SlotPtrs* ptrs, int* err, cudaStream_t s) {
    const int threads = ((tg.YB * g.L[0] + 31) / 32) * 32;
    const int blocks = tg.nslots * tg.nyb * g.L[2] * tg.nseg;
    matvec_tiled_kernel<<<blocks, threads, tiled_smem_bytes(g.L[0], tg.YB), s>>>(
        g, tg, reinterpret_cast<const float4*>(links32), (float)kappa, states, ptrs, err);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t set_wait_cycles_tiled(long long cycles) { return set_wait_cycles_here(cycles); }

}  // namespace lqcd
