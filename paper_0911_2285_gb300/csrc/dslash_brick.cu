// Operator pair of one BiCG iteration (A p and A^+ phat for every slot of the
// batch, Sec. 2's two products per step) on 4-D bricks of 256 sites, FP32.
//
// A block owns one brick of BX x BY x BZ x BT sites at a time (one site per
// thread) and computes both operators for EVERY running slot of the batch:
//   * the brick's links (two rows per direction) and the links of its four
//     backward faces are staged in shared memory once and serve all 2k
//     operator applications of the brick (the other operator shapes fetch them
//     once per slot from L2);
//   * the spinors p, phat of a slot are read through L1 while the block works
//     on that slot, so a brick site's value serves its in-brick neighbours and
//     only the eight faces come from L2 (1 + 2 (1/BX + 1/BY + 1/BZ + 1/BT)
//     reads per site per field instead of about 4);
//   * outputs are stored with an evict-first hint: they are not read again
//     inside the launch and would otherwise push the face spinors of the
//     neighbouring bricks out of L2.
// sigma = (phat, A p) and the two norms: FP32 per thread, warp sums, one
// accumulator per (warp, slot) in shared memory across the block's bricks,
// one FP64 partial per (block, slot); the last block adds each slot's partials
// in block order. The grid depends only on the lattice, so each slot's sums
// do not depend on which other slots share the batch.
#include "dslash.cuh"
#include "kernels.cuh"
#include "reduce.cuh"

namespace lqcd {
namespace {

constexpr int BR_THREADS = 256;
constexpr double BR_BREAK_TOL = 1e-14;

__device__ __forceinline__ void stcs4(void* base, size_t i, float4 v) {
    __stcs(reinterpret_cast<float4*>(base) + i, v);
}

// Link (two stored rows, third rebuilt) from shared memory: rows in three
// float4 at base[0], base[stride], base[2 stride].
__device__ __forceinline__ void sm_link(const float4* base, int stride, float2 (&m)[3][3]) {
    const float4 a = base[0], b = base[stride], c = base[2 * stride];
    m[0][0] = make_float2(a.x, a.y); m[0][1] = make_float2(a.z, a.w);
    m[0][2] = make_float2(b.x, b.y); m[1][0] = make_float2(b.z, b.w);
    m[1][1] = make_float2(c.x, c.y); m[1][2] = make_float2(c.z, c.w);
    m[2][0] = cross_conj(m[0][1], m[1][2], m[0][2], m[1][1]);
    m[2][1] = cross_conj(m[0][2], m[1][0], m[0][0], m[1][2]);
    m[2][2] = cross_conj(m[0][0], m[1][1], m[0][1], m[1][0]);
}

template <int BX, int BY, int BZ, int BT> struct Brick {
    static constexpr int NB = BX * BY * BZ * BT;
    static constexpr int F0 = NB / BX, F1 = NB / BY, F2 = NB / BZ, F3 = NB / BT;   // face sizes
    static constexpr int FTOT = F0 + F1 + F2 + F3;
    static constexpr size_t SMEM = (size_t)(12 * NB + 3 * FTOT) * sizeof(float4);
    static constexpr __device__ int foff(int mu) {
        return mu == 0 ? 0 : mu == 1 ? F0 : mu == 2 ? F0 + F1 : F0 + F1 + F2;
    }
    static constexpr __device__ int lstride(int mu) {
        return mu == 0 ? 1 : mu == 1 ? BX : mu == 2 ? BX * BY : BX * BY * BZ;
    }
    // index on the face normal to mu of local coordinates c (the other three, in order)
    static __device__ __forceinline__ int face_index(int mu, const int (&c)[4]) {
        if (mu == 0) return c[1] + BY * (c[2] + BZ * c[3]);
        if (mu == 1) return c[0] + BX * (c[2] + BZ * c[3]);
        if (mu == 2) return c[0] + BX * (c[1] + BY * c[3]);
        return c[0] + BX * (c[1] + BY * c[2]);
    }
};

// One direction of both operators at a site: a += hop of p (projectors 1 -+ gamma),
// b += hop of phat (1 +- gamma), links from shared memory (sm: the brick's
// links [mu*3 + q][NB], then the backward faces [q][FTOT]).
template <int MU, class B>
__device__ __forceinline__ void brick_dir(const Nbr& nb, const float4* sm, int tid, const int (&lc)[4],
                                          const void* p, const void* ph, int V, float2 (&a)[12],
                                          float2 (&b)[12]) {
    float2 psi[12], h[2][3], uh[2][3], u[3][3];
    sm_link(sm + MU * 3 * B::NB + tid, B::NB, u);
    Field<float>::load(p, V, nb.f[MU], psi);
    project<MU, -1>(psi, h);
    su3_mul(u, h, uh);
    reconstruct<MU, -1>(uh, a);
    Field<float>::load(ph, V, nb.f[MU], psi);
    project<MU, +1>(psi, h);
    su3_mul(u, h, uh);
    reconstruct<MU, +1>(uh, b);
    // U_mu(x - mu): in the brick, or on its backward face
    if (lc[MU] > 0) sm_link(sm + MU * 3 * B::NB + tid - B::lstride(MU), B::NB, u);
    else sm_link(sm + 12 * B::NB + B::foff(MU) + B::face_index(MU, lc), B::FTOT, u);
    Field<float>::load(p, V, nb.b[MU], psi);
    project<MU, +1>(psi, h);
    su3_dag_mul(u, h, uh);
    reconstruct<MU, +1>(uh, a);
    Field<float>::load(ph, V, nb.b[MU], psi);
    project<MU, -1>(psi, h);
    su3_dag_mul(u, h, uh);
    reconstruct<MU, -1>(uh, b);
}

template <int BX, int BY, int BZ, int BT, int MINB>
__global__ void __launch_bounds__(BR_THREADS, MINB)
    matvec_brick_kernel(Geom g, const float4* __restrict__ links, float kappa, SlotState* states,
                        const SlotPtrs* ptrs, int nslots) {
    using B = Brick<BX, BY, BZ, BT>;
    static_assert(B::NB == BR_THREADS, "one site per thread");
    constexpr int NB = B::NB, FTOT = B::FTOT;
    extern __shared__ float4 br_sm[];
    float4* sl = br_sm;              // [mu*3 + q][NB]: the brick's links
    float4* sh = br_sm + 12 * NB;    // [q][FTOT]: links U_mu at the backward face of mu
    __shared__ float4 acc_sm[MAX_SLOTS][BR_THREADS / 32];   // (Re sigma, Im sigma, |phat|^2, |Ap|^2)
    __shared__ unsigned run_mask, par_mask;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        unsigned rm = 0, pm = 0;
        for (int j = 0; j < nslots; ++j)
            if (states[j].status == ST_RUNNING && !states[j].stab) {
                rm |= 1u << j;
                pm |= (unsigned)(states[j].iter & 1) << j;
            }
        run_mask = rm;
        par_mask = pm;
    }
    if (tid < MAX_SLOTS * (BR_THREADS / 32)) acc_sm[tid / (BR_THREADS / 32)][tid % (BR_THREADS / 32)] =
        make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    const unsigned rmask = run_mask, pmask = par_mask;
    if (rmask == 0) return;   // uniform over the grid: nothing arrives, the counter stays zero

    const int nbx = g.L[0] / BX, nby = g.L[1] / BY, nbz = g.L[2] / BZ;
    const int nbricks = nbx * nby * nbz * (g.L[3] / BT);
    int lc[4];
    lc[0] = tid % BX;
    lc[1] = (tid / BX) % BY;
    lc[2] = (tid / (BX * BY)) % BZ;
    lc[3] = tid / (BX * BY * BZ);
    const float k = kappa;
    for (int br = blockIdx.x; br < nbricks; br += gridDim.x) {
        int r = br;
        int o[4];
        o[0] = (r % nbx) * BX; r /= nbx;
        o[1] = (r % nby) * BY; r /= nby;
        o[2] = (r % nbz) * BZ;
        o[3] = (r / nbz) * BT;
        const int s = (o[0] + lc[0]) + g.L[0] * ((o[1] + lc[1]) + g.L[1] * ((o[2] + lc[2]) + g.L[2] * (o[3] + lc[3])));
#pragma unroll
        for (int e = 0; e < 12; ++e) sl[e * NB + tid] = __ldg(links + (size_t)e * g.V + s);
        for (int i = tid; i < 3 * FTOT; i += NB) {
            const int q = i / FTOT, fi = i % FTOT;
            // face site: local coordinate mu = -1 (periodic), the other three from the face index
            int x, y, z, t, mu;
            if (fi < B::F0) {
                mu = 0; x = (o[0] == 0 ? g.L[0] : o[0]) - 1;
                y = o[1] + fi % BY; z = o[2] + (fi / BY) % BZ; t = o[3] + fi / (BY * BZ);
            } else if (fi < B::F0 + B::F1) {
                const int j = fi - B::F0;
                mu = 1; y = (o[1] == 0 ? g.L[1] : o[1]) - 1;
                x = o[0] + j % BX; z = o[2] + (j / BX) % BZ; t = o[3] + j / (BX * BZ);
            } else if (fi < B::F0 + B::F1 + B::F2) {
                const int j = fi - B::F0 - B::F1;
                mu = 2; z = (o[2] == 0 ? g.L[2] : o[2]) - 1;
                x = o[0] + j % BX; y = o[1] + (j / BX) % BY; t = o[3] + j / (BX * BY);
            } else {
                const int j = fi - B::F0 - B::F1 - B::F2;
                mu = 3; t = (o[3] == 0 ? g.L[3] : o[3]) - 1;
                x = o[0] + j % BX; y = o[1] + (j / BX) % BY; z = o[2] + j / (BX * BY);
            }
            const int fs = x + g.L[0] * (y + g.L[1] * (z + g.L[2] * t));
            sh[q * FTOT + fi] = __ldg(links + (size_t)(mu * 3 + q) * g.V + fs);
        }
        __syncthreads();

        const Nbr nb(g, s);
        for (int j = 0; j < nslots; ++j) {
            if (!((rmask >> j) & 1u)) continue;
            const SlotPtrs& P = ptrs[j];
            const int par = (pmask >> j) & 1;
            const void* p = P.p;
            const void* ph = P.phat;
            float2 a[12], b[12];
#pragma unroll
            for (int c = 0; c < 12; ++c) { a[c] = make_float2(0.f, 0.f); b[c] = a[c]; }
            brick_dir<0, B>(nb, br_sm, tid, lc, p, ph, g.V, a, b);
            brick_dir<1, B>(nb, br_sm, tid, lc, p, ph, g.V, a, b);
            brick_dir<2, B>(nb, br_sm, tid, lc, p, ph, g.V, a, b);
            brick_dir<3, B>(nb, br_sm, tid, lc, p, ph, g.V, a, b);
            float2 self[12];
            Field<float>::load(p, g.V, s, self);
#pragma unroll
            for (int c = 0; c < 12; ++c) a[c] = self[c] - k * a[c];
#pragma unroll
            for (int q = 0; q < 6; ++q)
                stcs4(P.Ap[par], (size_t)q * g.V + s, make_float4(a[2 * q].x, a[2 * q].y, a[2 * q + 1].x, a[2 * q + 1].y));
            Field<float>::load(ph, g.V, s, self);
            Acc<float> sacc;
#pragma unroll
            for (int c = 0; c < 12; ++c) {
                b[c] = self[c] - k * b[c];
                sacc.z = sacc.z + cdot(self[c], a[c]);
                sacc.a += abs2(self[c]);
                sacc.b += abs2(a[c]);
            }
#pragma unroll
            for (int q = 0; q < 6; ++q)
                stcs4(P.Ahp[par], (size_t)q * g.V + s, make_float4(b[2 * q].x, b[2 * q].y, b[2 * q + 1].x, b[2 * q + 1].y));
            const float2 z = warp_sum(sacc.z);
            const float2 ab = warp_sum(make_float2(sacc.a, sacc.b));
            if (lane == 0) {
                float4 t = acc_sm[j][warp];
                acc_sm[j][warp] = make_float4(t.x + z.x, t.y + z.y, t.z + ab.x, t.w + ab.y);
            }
        }
        __syncthreads();   // the next brick overwrites the staged links
    }
    // one FP64 partial per (block, slot), warps added in order
    if (tid < nslots && ((rmask >> tid) & 1u)) {
        double2 z = make_double2(0.0, 0.0), ab = make_double2(0.0, 0.0);
        for (int w = 0; w < BR_THREADS / 32; ++w) {
            const float4 t = acc_sm[tid][w];
            z = z + make_double2(t.x, t.y);
            ab = ab + make_double2(t.z, t.w);
        }
        double2* pp = ptrs[tid].partials + (size_t)CNT_MATVEC * PARTIAL_STRIDE + (size_t)blockIdx.x * 2;
        pp[0] = z;
        pp[1] = ab;
        __threadfence();
    }
    if (!last_block(ptrs[0].counters + CNT_GROUP, gridDim.x)) return;
    for (int sl_ = warp; sl_ < nslots; sl_ += BR_THREADS / 32) {
        if (!((rmask >> sl_) & 1u)) continue;
        SlotState& st = states[sl_];
        const double2* pp = ptrs[sl_].partials + (size_t)CNT_MATVEC * PARTIAL_STRIDE;
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
            if (!(cabs_(st.sigma) >= BR_BREAK_TOL * st.phat_norm * st.ap_norm) || cabs2(st.sigma) == 0.0) {
                st.status = ST_BREAKDOWN;
            } else {
                st.alpha = cdiv(st.rho, st.sigma);
            }
        }
    }
}

template <int BX, int BY, int BZ, int BT, int MINB>
cudaError_t brick_launch(const Geom& g, const void* links, double kappa, SlotState* states, const SlotPtrs* ptrs,
                         int nslots, cudaStream_t s) {
    using Bk = Brick<BX, BY, BZ, BT>;
    auto kern = matvec_brick_kernel<BX, BY, BZ, BT, MINB>;
    static unsigned configured = 0;   // one bit per device
    int dev = 0;
    cudaError_t e0 = cudaGetDevice(&dev);
    if (e0 != cudaSuccess) return e0;
    if (dev >= 32) return cudaErrorInvalidDevice;
    if (!((configured >> dev) & 1u)) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Bk::SMEM);
        if (e != cudaSuccess) return e;
        // shared memory for MINB blocks, the rest of the 256 KB stays L1 (the spinor reuse)
        int pct = (int)((MINB * (Bk::SMEM + 4096) * 100 + 228 * 1024 - 1) / (228 * 1024));
        if (pct > 100) pct = 100;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
        if (e != cudaSuccess) return e;
        configured |= 1u << dev;
    }
    const int nbricks = (g.L[0] / BX) * (g.L[1] / BY) * (g.L[2] / BZ) * (g.L[3] / BT);
    int grid = nbricks < PARTIAL_STRIDE / 2 ? nbricks : PARTIAL_STRIDE / 2;
    kern<<<grid, BR_THREADS, Bk::SMEM, s>>>(g, reinterpret_cast<const float4*>(links), (float)kappa, states, ptrs,
                                            nslots);
    return cudaGetLastError();
}

}  // namespace

bool brick_variant_ok(const Geom& g, int v) {
    int b[4];
    switch (v) {
        case 25: case 29: b[0] = 4; b[1] = 4; b[2] = 4; b[3] = 4; break;
        case 27: b[0] = 8; b[1] = 4; b[2] = 4; b[3] = 2; break;
        case 28: b[0] = 4; b[1] = 4; b[2] = 8; b[3] = 2; break;
        default: return false;
    }
    for (int mu = 0; mu < 4; ++mu)
        if (g.L[mu] % b[mu] != 0) return false;
    return true;
}

cudaError_t launch_matvec_brick(const Geom& g, const void* links, double kappa, SlotState* states,
                                const SlotPtrs* ptrs, int nslots, cudaStream_t s, int variant) {
    if (!brick_variant_ok(g, variant) || nslots > MAX_SLOTS) return cudaErrorInvalidValue;
    cudaError_t e;
    switch (variant) {
        case 25: e = brick_launch<4, 4, 4, 4, 2>(g, links, kappa, states, ptrs, nslots, s); break;
        case 27: e = brick_launch<8, 4, 4, 2, 2>(g, links, kappa, states, ptrs, nslots, s); break;
        case 28: e = brick_launch<4, 4, 8, 2, 2>(g, links, kappa, states, ptrs, nslots, s); break;
        default: e = brick_launch<4, 4, 4, 4, 1>(g, links, kappa, states, ptrs, nslots, s); break;
    }
    count_launches(1);
    return e;
}

}  // namespace lqcd
