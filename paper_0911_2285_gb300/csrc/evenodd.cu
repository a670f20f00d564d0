// Even-odd (Schur complement) form of the Wilson operator (the paper's test
// matrices are even-odd preconditioned, Sec. 3). D_hop connects only sites of
// opposite parity (x + y + z + t) mod 2, so with A = [[1, -k D_eo], [-k D_oe, 1]]
// the odd unknowns solve
//
//     A_hat x_o = b_hat,   A_hat = 1 - k^2 D_oe D_eo,   b_hat = b_o + k D_oe b_e,
//
// and x_e = b_e + k D_eo x_o. A_hat^+ = 1 - k^2 (D^+)_oe (D^+)_eo: the adjoint
// hops in the same two stages.
//
// Half-lattice fields (one parity, all extents even): site s of parity P has the
// half index h = s >> 1 (Lx even, so each pair of sites 2h, 2h + 1 holds one site
// of each parity); a half field is the chunk layout of common.cuh over V/2 sites.
#include "dslash.cuh"
#include "kernels.cuh"
#include "reduce.cuh"

namespace lqcd {
namespace {

constexpr int EO_THREADS = 128;
constexpr double EO_BREAK_TOL = 1e-14;

// Full site index of half index h in parity P.
__device__ __forceinline__ int eo_site(const Geom& g, int h, int P) {
    const int s0 = 2 * h;
    int r = s0 / g.L[0];
    const int y = r % g.L[1];
    r /= g.L[1];
    const int z = r % g.L[2], t = r / g.L[2];
    // x of s0 is even, so the parity of s0 is that of y + z + t
    return s0 + ((((y + z + t) & 1) != P) ? 1 : 0);
}

// A half field read at full site indices (the neighbours of a site of the other parity).
template <typename S> struct HalfIn {
    const void* p;
    int Vh;
    template <typename C> __device__ __forceinline__ void load(int s, C (&v)[12]) const {
        Field<S>::load(p, Vh, s >> 1, v);
    }
};

int eo_blocks(int Vh) {
    int nb = (Vh + EO_THREADS - 1) / EO_THREADS;
    if (nb > PARTIAL_STRIDE / 2) nb = PARTIAL_STRIDE / 2;
    return nb;
}

// ------------------------------------------------------------- host applies
// Stage 1 (jobs): out = D in (or D^+ in), in of parity 1 - P, out of parity P.
// Grid: site blocks x jobs, jobs fastest.
template <typename S>
__global__ void __launch_bounds__(EO_THREADS) eo_hop_kernel(Geom g, const void* links, const EoJob* jobs, int njobs,
                                                           int P) {
    const int jid = blockIdx.x % njobs, sblock = blockIdx.x / njobs, nsb = gridDim.x / njobs;
    const EoJob jb = jobs[jid];
    const int Vh = g.V / 2;
    typename LinkSel<S>::type U{reinterpret_cast<decltype(U.u)>(links), g.V};
    HalfIn<S> in{jb.hop_in, Vh};
    for (int h = sblock * blockDim.x + threadIdx.x; h < Vh; h += nsb * blockDim.x) {
        const int s = eo_site(g, h, P);
        cplx<S> acc[12];
        if (jb.dagger) hop_site<true, S>(g, U, in, s, acc);
        else hop_site<false, S>(g, U, in, s, acc);
        Field<S>::store(jb.out, Vh, h, acc);
    }
}

// Stage 2 (jobs): out = self - k^2 D tmp (odd sites), or aux - (self - k^2 D tmp)
// with aux (FP64) when RES.
template <typename S, bool RES>
__global__ void __launch_bounds__(EO_THREADS) eo_combine_kernel(Geom g, const void* links, double kappa,
                                                               const EoJob* jobs, int njobs) {
    const int jid = blockIdx.x % njobs, sblock = blockIdx.x / njobs, nsb = gridDim.x / njobs;
    const EoJob jb = jobs[jid];
    const int Vh = g.V / 2;
    typename LinkSel<S>::type U{reinterpret_cast<decltype(U.u)>(links), g.V};
    HalfIn<S> in{jb.hop_in, Vh};
    const S k2 = (S)(kappa * kappa);
    for (int h = sblock * blockDim.x + threadIdx.x; h < Vh; h += nsb * blockDim.x) {
        const int s = eo_site(g, h, 1);
        cplx<S> acc[12], self[12];
        if (jb.dagger) hop_site<true, S>(g, U, in, s, acc);
        else hop_site<false, S>(g, U, in, s, acc);
        Field<S>::load(jb.self, Vh, h, self);
#pragma unroll
        for (int c = 0; c < 12; ++c) acc[c] = self[c] - k2 * acc[c];
        if (RES) {
            double2 b[12];
            Field<double>::load(jb.aux, Vh, h, b);
#pragma unroll
            for (int c = 0; c < 12; ++c) acc[c] = cvt<S>(b[c] - to_d(acc[c]));
        }
        Field<S>::store(jb.out, Vh, h, acc);
    }
}

// b_hat = b_o + k D_oe b_e from full FP64 fields (k fields, consecutive).
__global__ void __launch_bounds__(EO_THREADS) eo_prepare_kernel(Geom g, const void* links64, double kappa,
                                                               const double2* bfull, double2* bhat, int k) {
    const int Vh = g.V / 2;
    const size_t fN = (size_t)12 * g.V, hN = (size_t)12 * Vh;
    LinksD U{reinterpret_cast<const double2*>(links64), g.V};
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < (size_t)Vh * k; q += (size_t)gridDim.x * blockDim.x) {
        const int f = (int)(q / Vh), h = (int)(q % Vh);
        const int s = eo_site(g, h, 1);
        FieldIn<double> in{bfull + f * fN, g.V};
        double2 acc[12], self[12];
        hop_site<false, double>(g, U, in, s, acc);
        in.load(s, self);
#pragma unroll
        for (int c = 0; c < 12; ++c) acc[c] = self[c] + kappa * acc[c];
        Field<double>::store(bhat + f * hN, Vh, h, acc);
    }
}

// x_o (half) from a full FP64 field (k fields).
__global__ void eo_extract_kernel(Geom g, const double2* xfull, double2* xhalf, int k) {
    const int Vh = g.V / 2;
    const size_t fN = (size_t)12 * g.V, hN = (size_t)12 * Vh;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < (size_t)Vh * k; q += (size_t)gridDim.x * blockDim.x) {
        const int f = (int)(q / Vh), h = (int)(q % Vh);
        double2 v[12];
        Field<double>::load(xfull + f * fN, g.V, eo_site(g, h, 1), v);
        Field<double>::store(xhalf + f * hN, Vh, h, v);
    }
}

// Full solution: x_o from the half field, x_e = b_e + k D_eo x_o (k fields).
__global__ void __launch_bounds__(EO_THREADS) eo_reconstruct_kernel(Geom g, const void* links64, double kappa,
                                                                   const double2* bfull, const double2* xhalf,
                                                                   double2* xfull, int k) {
    const int Vh = g.V / 2;
    const size_t fN = (size_t)12 * g.V, hN = (size_t)12 * Vh;
    LinksD U{reinterpret_cast<const double2*>(links64), g.V};
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < (size_t)g.V * k; q += (size_t)gridDim.x * blockDim.x) {
        const int f = (int)(q / g.V), s = (int)(q % g.V);
        int r = s / g.L[0];
        const int x = s % g.L[0];
        const int y = r % g.L[1];
        r /= g.L[1];
        const int z = r % g.L[2], t = r / g.L[2];
        double2 v[12];
        if ((x + y + z + t) & 1) {
            Field<double>::load(xhalf + f * hN, Vh, s >> 1, v);
        } else {
            HalfIn<double> in{xhalf + f * hN, Vh};
            double2 bb[12];
            hop_site<false, double>(g, U, in, s, v);
            Field<double>::load(bfull + f * fN, g.V, s, bb);
#pragma unroll
            for (int c = 0; c < 12; ++c) v[c] = bb[c] + kappa * v[c];
        }
        Field<double>::store(xfull + f * fN, g.V, s, v);
    }
}

// ------------------------------------------------------------ BiCG kernels
// The pair kernels: a block takes a contiguous run of THREADS-site units of
// the half lattice (neighbouring sites stay on one SM; FP32: 256 threads, two
// blocks per SM, two units per block, like the full operator's best
// gather-through-L1 shape).
struct HalfRun {
    int u0, u1;
    __device__ __forceinline__ HalfRun(int Vh, int threads, int nsb, int sblock) {
        const int nunits = (Vh + threads - 1) / threads;
        const int per = (nunits + nsb - 1) / nsb;
        u0 = sblock * per;
        u1 = min(nunits, u0 + per);
    }
};

// Operator pair of one BiCG iteration on A_hat, stage 1 (one thread per (half
// site, slot)): t = D_eo p, that = (D^+)_eo phat into the slot's stage buffers.
template <typename S, int THREADS, int MINB>
__global__ void __launch_bounds__(THREADS, MINB) eo_pair1_kernel(Geom g, const void* links, SlotState* states,
                                                                const SlotPtrs* ptrs, int nslots) {
    const int slot = blockIdx.x % nslots, sblock = blockIdx.x / nslots, nsb = gridDim.x / nslots;
    const SlotState& st = states[slot];
    const SlotPtrs& P = ptrs[slot];
    if (st.status != ST_RUNNING || st.stab) return;
    const int Vh = g.V / 2;
    typename LinkSel<S>::type U{reinterpret_cast<decltype(U.u)>(links), g.V};
    HalfIn<S> inp{P.p, Vh}, inh{P.phat, Vh};
    const HalfRun run(Vh, THREADS, nsb, sblock);
    for (int u = run.u0; u < run.u1; ++u) {
        const int h = u * THREADS + (int)threadIdx.x;
        if (h >= Vh) continue;
        const int s = eo_site(g, h, 0);
        cplx<S> a[12], b[12];
        hop_site_pair<S>(g, U, inp, inh, s, a, b);
        Field<S>::store(P.eo_t, Vh, h, a);
        Field<S>::store(P.eo_th, Vh, h, b);
    }
}

// Stage 2: A_hat p = p - k^2 D_oe t, A_hat^+ phat = phat - k^2 (D^+)_oe that, and
// sigma = (phat, A_hat p), alpha = rho / sigma in the last block.
template <typename S, int THREADS, int MINB>
__global__ void __launch_bounds__(THREADS, MINB) eo_pair2_kernel(Geom g, const void* links, double kappa,
                                                                SlotState* states, const SlotPtrs* ptrs, int nslots) {
    const int slot = blockIdx.x % nslots, sblock = blockIdx.x / nslots, nsb = gridDim.x / nslots;
    SlotState& st = states[slot];
    const SlotPtrs& P = ptrs[slot];
    if (st.status != ST_RUNNING || st.stab) return;
    const int Vh = g.V / 2;
    const int par = st.iter & 1;
    typename LinkSel<S>::type U{reinterpret_cast<decltype(U.u)>(links), g.V};
    HalfIn<S> int_{P.eo_t, Vh}, inth{P.eo_th, Vh};
    const S k2 = (S)(kappa * kappa);
    Acc<S> sacc;   // sigma, |phat|^2, |Ap|^2
    const HalfRun run(Vh, THREADS, nsb, sblock);
    for (int u = run.u0; u < run.u1; ++u) {
        const int h = u * THREADS + (int)threadIdx.x;
        if (h >= Vh) continue;
        const int s = eo_site(g, h, 1);
        cplx<S> a[12], b[12], self[12];
        hop_site_pair<S>(g, U, int_, inth, s, a, b);
        Field<S>::load(P.p, Vh, h, self);
#pragma unroll
        for (int c = 0; c < 12; ++c) a[c] = self[c] - k2 * a[c];
        Field<S>::store(P.Ap[par], Vh, h, a);
        Field<S>::load(P.phat, Vh, h, self);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            b[c] = self[c] - k2 * b[c];
            sacc.z = sacc.z + cdot(self[c], a[c]);
            sacc.a += abs2(self[c]);
            sacc.b += abs2(a[c]);
        }
        Field<S>::store(P.Ahp[par], Vh, h, b);
    }
    cplx<S> v[2];
    sacc.to(v);
    double2 tot[2];
    if (reduce_slot<2>(P, CNT_MATVEC, v, tot, nsb, sblock) && threadIdx.x == 0) {
        st.sigma = tot[0];
        st.phat_norm = sqrt(tot[1].x);
        st.ap_norm = sqrt(tot[1].y);
        st.matvecs += 2;
        if (!(cabs_(st.sigma) >= EO_BREAK_TOL * st.phat_norm * st.ap_norm) || cabs2(st.sigma) == 0.0)
            st.status = ST_BREAKDOWN;
        else
            st.alpha = cdiv(st.rho, st.sigma);
    }
}

// FP64 Schur residual r = b_hat - A_hat x_hi of the slots that asked for it
// (in-iteration, check_only = 0) or of every started slot (check_only = 1):
// stage 1 t = D_eo x_hi into the slot's FP64 stage buffer, stage 2 the residual.
__global__ void __launch_bounds__(EO_THREADS) eo_res1_kernel(Geom g, const void* links64, SlotState* states,
                                                            const SlotPtrs* ptrs, int check_only) {
    const SlotState& st = states[blockIdx.y];
    const SlotPtrs& P = ptrs[blockIdx.y];
    if (check_only ? st.status == ST_IDLE : (st.status != ST_RUNNING || !st.need_ru)) return;
    const int Vh = g.V / 2;
    LinksD U{reinterpret_cast<const double2*>(links64), g.V};
    HalfIn<double> in{P.x_hi, Vh};
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < Vh; h += gridDim.x * blockDim.x) {
        double2 acc[12];
        hop_site<false, double>(g, U, in, eo_site(g, h, 0), acc);
        Field<double>::store(P.eo64, Vh, h, acc);
    }
}

__global__ void __launch_bounds__(EO_THREADS) eo_res2_kernel(Geom g, const void* links64, double kappa,
                                                            SlotState* states, const SlotPtrs* ptrs, int check_only) {
    SlotState& st = states[blockIdx.y];
    const SlotPtrs& P = ptrs[blockIdx.y];
    if (check_only ? st.status == ST_IDLE : (st.status != ST_RUNNING || !st.need_ru)) return;
    const int Vh = g.V / 2;
    LinksD U{reinterpret_cast<const double2*>(links64), g.V};
    HalfIn<double> in{P.eo64, Vh};
    const double k2 = kappa * kappa;
    double2 v[1] = {make_double2(0, 0)};
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < Vh; h += gridDim.x * blockDim.x) {
        double2 acc[12], self[12], b[12];
        hop_site<false, double>(g, U, in, eo_site(g, h, 1), acc);
        Field<double>::load(P.x_hi, Vh, h, self);
        Field<double>::load(P.b, Vh, h, b);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            acc[c] = b[c] - (self[c] - k2 * acc[c]);
            v[0].x += cabs2(acc[c]);
        }
        Field<double>::store(P.r_true, Vh, h, acc);
    }
    double2 tot[1];
    if (reduce_slot<1>(P, CNT_RU, v, tot, gridDim.x, blockIdx.x) && threadIdx.x == 0) {
        st.true_rnorm = sqrt(tot[0].x);
        st.matvecs += 1;
        if (!check_only && st.true_rnorm <= st.tol * st.bnorm) st.status = ST_CONVERGED;
    }
}

}  // namespace

// ------------------------------------------------------------------ launchers
cudaError_t launch_eo_apply(const Geom& g, const void* links, double kappa, int prec, const EoJob* d_stage1,
                            const EoJob* d_stage2, int njobs, int residual, cudaStream_t st) {
    const int grid = eo_blocks(g.V / 2) * njobs;
    if (prec == 0) {
        eo_hop_kernel<double><<<grid, EO_THREADS, 0, st>>>(g, links, d_stage1, njobs, 0);
        if (residual) eo_combine_kernel<double, true><<<grid, EO_THREADS, 0, st>>>(g, links, kappa, d_stage2, njobs);
        else eo_combine_kernel<double, false><<<grid, EO_THREADS, 0, st>>>(g, links, kappa, d_stage2, njobs);
    } else {
        if (residual) return cudaErrorInvalidValue;
        eo_hop_kernel<float><<<grid, EO_THREADS, 0, st>>>(g, links, d_stage1, njobs, 0);
        eo_combine_kernel<float, false><<<grid, EO_THREADS, 0, st>>>(g, links, kappa, d_stage2, njobs);
    }
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_eo_prepare(const Geom& g, const void* links64, double kappa, const double2* bfull, double2* bhat,
                              int k, cudaStream_t st) {
    eo_prepare_kernel<<<eo_blocks(g.V / 2) * k, EO_THREADS, 0, st>>>(g, links64, kappa, bfull, bhat, k);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_eo_extract(const Geom& g, const double2* xfull, double2* xhalf, int k, cudaStream_t st) {
    eo_extract_kernel<<<eo_blocks(g.V / 2) * k, EO_THREADS, 0, st>>>(g, xfull, xhalf, k);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_eo_reconstruct(const Geom& g, const void* links64, double kappa, const double2* bfull,
                                  const double2* xhalf, double2* xfull, int k, cudaStream_t st) {
    eo_reconstruct_kernel<<<eo_blocks(g.V) * k, EO_THREADS, 0, st>>>(g, links64, kappa, bfull, xhalf, xfull, k);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_eo_pair(const Geom& g, const void* links, double kappa, int prec, SlotState* states,
                           const SlotPtrs* ptrs, int nslots, cudaStream_t st) {
    if (prec == 0) {
        const int grid = eo_blocks(g.V / 2) * nslots;
        eo_pair1_kernel<double, EO_THREADS, 1><<<grid, EO_THREADS, 0, st>>>(g, links, states, ptrs, nslots);
        eo_pair2_kernel<double, EO_THREADS, 1><<<grid, EO_THREADS, 0, st>>>(g, links, kappa, states, ptrs, nslots);
    } else {
        constexpr int T = 256, UNITS = 2;
        int nb = (g.V / 2 + T * UNITS - 1) / (T * UNITS);
        if (nb > PARTIAL_STRIDE / 2) nb = PARTIAL_STRIDE / 2;
        eo_pair1_kernel<float, T, 2><<<nb * nslots, T, 0, st>>>(g, links, states, ptrs, nslots);
        eo_pair2_kernel<float, T, 2><<<nb * nslots, T, 0, st>>>(g, links, kappa, states, ptrs, nslots);
    }
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_eo_true_resid(const Geom& g, const void* links64, double kappa, SlotState* states,
                                 const SlotPtrs* ptrs, int nslots, int check_only, cudaStream_t st) {
    const dim3 grid(eo_blocks(g.V / 2), nslots);
    eo_res1_kernel<<<grid, EO_THREADS, 0, st>>>(g, links64, states, ptrs, check_only);
    eo_res2_kernel<<<grid, EO_THREADS, 0, st>>>(g, links64, kappa, states, ptrs, check_only);
    count_launches(2);
    return cudaGetLastError();
}

}  // namespace lqcd
