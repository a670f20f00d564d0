// Lattice-sized kernels: the Wilson operator applications, the BiCG iteration
// (Algorithm eigBiCG, steps 1-3 of the paper, Sec. 2), the window product of
// the BiCG-eigen restart with its coupling row/column, and the tall-skinny
// products of the oblique deflation (Algorithm Incremental eigBiCG).
//
// All reductions are two-level and deterministic: each block writes its
// partial sums to a fixed slot, and the last block to finish adds them in
// block order (same result alone or inside a batch).
#include "dslash.cuh"
#include "dfloat.cuh"
#include "kernels.cuh"
#include "reduce.cuh"

namespace lqcd {
namespace {

constexpr int DS_THREADS = 128;   // operator kernels
constexpr int BL_THREADS = 256;   // vector kernels
constexpr double BREAK_TOL = 1e-14;

inline int div_up(size_t a, size_t b) { return (int)((a + b - 1) / b); }

int blas_blocks(size_t units) {
    int nb = div_up(units, BL_THREADS);
    if (nb > 1216) nb = 1216;   // 8 blocks of 256 per SM on 152 SMs
    if (nb < 1) nb = 1;
    return nb;
}
int ds_blocks(int V) {
    int nb = div_up((size_t)V, DS_THREADS);
    if (nb > PARTIAL_STRIDE / 2) nb = PARTIAL_STRIDE / 2;
    return nb;
}

// ------------------------------------------------------------------- apply
// r = b - A x with FP64 x, b, r and the hop in FP32 arithmetic on FP32 links:
// the starting and deflation residuals of the mixed-precision solver, which
// are consumed in FP32 (the reliable updates and the final residual use
// FP64-class arithmetic). jobs: in = x, aux = b, out = r.
__global__ void __launch_bounds__(DS_THREADS) residual32_kernel(Geom g, const float4* links, double kappa,
                                                                const ApplyJob* jobs, int njobs) {
    const int jid = blockIdx.x % njobs, sblock = blockIdx.x / njobs, nsb = gridDim.x / njobs;
    const ApplyJob jb = jobs[jid];
    LinksF U{links, g.V};
    FieldIn<double> in{jb.in, g.V};
    const double k = kappa;
    for (int s = sblock * blockDim.x + threadIdx.x; s < g.V; s += nsb * blockDim.x) {
        float2 acc[12];
        hop_site<false, float>(g, U, in, s, acc);
        double2 x[12], b[12];
        Field<double>::load(jb.in, g.V, s, x);
        Field<double>::load(jb.aux, g.V, s, b);
#pragma unroll
        for (int c = 0; c < 12; ++c) b[c] = b[c] - (x[c] - k * to_d(acc[c]));
        Field<double>::store(jb.out, g.V, s, b);
    }
}

template <typename S, bool RES>
__global__ void __launch_bounds__(DS_THREADS) apply_kernel(Geom g, const void* links, double kappa,
                                                           const ApplyJob* jobs, int njobs) {
    using C = cplx<S>;
    const int jid = blockIdx.x % njobs, sblock = blockIdx.x / njobs, nsb = gridDim.x / njobs;
    const ApplyJob jb = jobs[jid];
    typename LinkSel<S>::type U{reinterpret_cast<decltype(U.u)>(links), g.V};
    FieldIn<S> in{jb.in, g.V};
    const S k = (S)kappa;
    for (int s = sblock * blockDim.x + threadIdx.x; s < g.V; s += nsb * blockDim.x) {
        C acc[12], self[12];
        if (jb.dagger) hop_site<true, S>(g, U, in, s, acc);
        else hop_site<false, S>(g, U, in, s, acc);
        in.load(s, self);
#pragma unroll
        for (int c = 0; c < 12; ++c) acc[c] = self[c] - k * acc[c];
        if (RES) {
            double2 b[12];
            Field<double>::load(jb.aux, g.V, s, b);
#pragma unroll
            for (int c = 0; c < 12; ++c) acc[c] = cvt<S>(b[c] - to_d(acc[c]));
        }
        Field<S>::store(jb.out, g.V, s, acc);
    }
}

// -------------------------------------------------------------- pack/unpack
// Host layout AoS [site][12] complex128 <-> device chunk layout.
template <typename S>
__global__ void pack_kernel(const double2* aos, void* dev, int V, int k) {
    const size_t total = (size_t)V * 12 * k;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t f = i / ((size_t)V * 12);
        const size_t r = i % ((size_t)V * 12);
        const int s = (int)(r / 12), c = (int)(r % 12);
        const size_t e = f * (size_t)V * 12 + ((size_t)(c >> 1) * V + s) * 2 + (c & 1);
        st_elem<S>(dev, e, cvt<S>(aos[i]));
    }
}
template <typename S>
__global__ void unpack_kernel(const void* dev, double2* aos, int V, int k) {
    const size_t total = (size_t)V * 12 * k;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t f = i / ((size_t)V * 12);
        const size_t r = i % ((size_t)V * 12);
        const int s = (int)(r / 12), c = (int)(r % 12);
        const size_t e = f * (size_t)V * 12 + ((size_t)(c >> 1) * V + s) * 2 + (c & 1);
        aos[i] = to_d(ld_elem<S>(dev, e));
    }
}
template <typename SI, typename SO>
__global__ void convert_kernel(const void* src, void* dst, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        st_elem<SO>(dst, i, cvt<SO>(to_d(ld_elem<SI>(src, i))));
}

// ------------------------------------------------------------- multidot
// C[i][j] = sum_e conj(X_i(e)) Y_j(e) for i in [i0, i0+TI), j < b <= BMAX.
constexpr int MD_TI = 4, MD_BMAX = 8;
// Grid: (element chunk x column group) flattened with the column group fastest,
// so the groups that read the same Y chunk run together (Y leaves DRAM once).
template <typename SX, typename SY, typename T>
__global__ void __launch_bounds__(BL_THREADS) multidot_kernel(int a, const void* X, int b, const void* Y, size_t N,
                                                              double2* scratch, int nby) {
    using C = cplx<T>;
    const int by = blockIdx.x % nby, bx = blockIdx.x / nby, nbx = gridDim.x / nby;
    const int i0 = by * MD_TI;
    C acc[MD_TI][MD_BMAX];
#pragma unroll
    for (int i = 0; i < MD_TI; ++i)
#pragma unroll
        for (int j = 0; j < MD_BMAX; ++j) acc[i][j] = mk<T>(T(0), T(0));
    for (size_t e = bx * (size_t)blockDim.x + threadIdx.x; e < N; e += (size_t)nbx * blockDim.x) {
        C y[MD_BMAX];
#pragma unroll
        for (int j = 0; j < MD_BMAX; ++j)
            if (j < b) {
                auto v = ld_elem<SY>(reinterpret_cast<const char*>(Y) + (size_t)j * N * sizeof(cplx<SY>), e);
                y[j] = mk<T>((T)v.x, (T)v.y);
            }
#pragma unroll
        for (int i = 0; i < MD_TI; ++i)
            if (i0 + i < a) {
                auto v = ld_elem<SX>(reinterpret_cast<const char*>(X) + (size_t)(i0 + i) * N * sizeof(cplx<SX>), e);
                C x = mk<T>((T)v.x, (T)v.y);
#pragma unroll
                for (int j = 0; j < MD_BMAX; ++j)
                    if (j < b) acc[i][j] = acc[i][j] + cdot(x, y[j]);
            }
    }
    C v[MD_TI * MD_BMAX];
#pragma unroll
    for (int i = 0; i < MD_TI; ++i)
#pragma unroll
        for (int j = 0; j < MD_BMAX; ++j) v[i * MD_BMAX + j] = acc[i][j];
    __shared__ C sm[(BL_THREADS / 32) * MD_TI * MD_BMAX];
    block_sum<MD_TI * MD_BMAX>(v, sm);   // in the accumulation precision T
    if (threadIdx.x == 0) {
        double2* out = scratch + ((size_t)by * nbx + bx) * (MD_TI * MD_BMAX);
#pragma unroll
        for (int q = 0; q < MD_TI * MD_BMAX; ++q) out[q] = to_d(v[q]);
    }
}
__global__ void multidot_reduce_kernel(int a, int b, int nbx, const double2* scratch, double2* Cm, int ldc,
                                       int conj_store) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;   // (i, j) pair
    if (q >= a * b) return;
    const int i = q / b, j = q % b;
    const int by = i / MD_TI, ii = i % MD_TI;
    double2 acc = make_double2(0.0, 0.0);
    for (int bx = 0; bx < nbx; ++bx) acc = acc + scratch[((size_t)by * nbx + bx) * (MD_TI * MD_BMAX) + ii * MD_BMAX + j];
    if (conj_store) Cm[(size_t)j * ldc + i] = conj_(acc);
    else Cm[(size_t)i * ldc + j] = acc;
}

// ------------------------------------------------------------- vupdate
// mode 0: Y_j += sum_i X_i D[i][j];  mode 1: Y_j = sum_i X_i D[i][j]  (j < b <= MD_BMAX).
template <typename SX, typename SY, typename T>
__global__ void __launch_bounds__(BL_THREADS) vupdate_kernel(int a, const void* X, const double2* D, int ldd, int b,
                                                             void* Y, int overwrite, size_t N) {
    using C = cplx<T>;
    __shared__ C Ds[MAX_SMALL * MD_BMAX];
    for (int q = threadIdx.x; q < a * b; q += blockDim.x) {
        const int i = q / b, j = q % b;
        double2 d = D[(size_t)i * ldd + j];
        Ds[i * MD_BMAX + j] = mk<T>((T)d.x, (T)d.y);
    }
    __syncthreads();
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < N; e += (size_t)gridDim.x * blockDim.x) {
        C acc[MD_BMAX];
#pragma unroll
        for (int j = 0; j < MD_BMAX; ++j) acc[j] = mk<T>(T(0), T(0));
        for (int i = 0; i < a; ++i) {
            auto v = ld_elem<SX>(reinterpret_cast<const char*>(X) + (size_t)i * N * sizeof(cplx<SX>), e);
            C x = mk<T>((T)v.x, (T)v.y);
#pragma unroll
            for (int j = 0; j < MD_BMAX; ++j)
                if (j < b) acc[j] = acc[j] + x * Ds[i * MD_BMAX + j];
        }
#pragma unroll
        for (int j = 0; j < MD_BMAX; ++j)
            if (j < b) {
                char* yj = reinterpret_cast<char*>(Y) + (size_t)j * N * sizeof(cplx<SY>);
                double2 upd = to_d(acc[j]);
                if (!overwrite) upd = upd + to_d(ld_elem<SY>(yj, e));   // add in the target precision
                st_elem<SY>(yj, e, cvt<SY>(upd));
            }
    }
}

// Per-field squared 2-norms of b fields: block partials (FP64) for a second pass.
template <typename S>
__global__ void __launch_bounds__(BL_THREADS) norms_kernel(const void* Y, size_t N, double2* scratch) {
    const int j = blockIdx.y;
    const cplx<S>* y = reinterpret_cast<const cplx<S>*>(Y) + (size_t)j * N;
    S acc = S(0);
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < N; e += (size_t)gridDim.x * blockDim.x)
        acc += abs2(y[e]);
    cplx<S> v[1] = {mk<S>(acc, S(0))};
    __shared__ cplx<S> sm[BL_THREADS / 32];
    block_sum<1>(v, sm);
    if (threadIdx.x == 0) scratch[(size_t)j * gridDim.x + blockIdx.x] = to_d(v[0]);
}
__global__ void norms_reduce_kernel(int b, int nb, const double2* scratch, double* out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= b) return;
    double acc = 0.0;
    for (int i = 0; i < nb; ++i) acc += scratch[(size_t)j * nb + i].x;
    out[j] = sqrt(acc);
}

// Y_j *= s_j (per-field scale), j < b.
template <typename S>
__global__ void scale_fields_kernel(int b, void* Y, const double2* sc, size_t N) {
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < N * b; q += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(q / N);
        const double2 s = sc[j];
        st_elem<S>(Y, q, cvt<S>(s * to_d(ld_elem<S>(Y, q))));
    }
}

// ------------------------------------------------------------ BiCG kernels
// Vector units: two complex numbers (one float4 in FP32, two double2 in FP64).
template <typename S> struct Unit;
template <> struct Unit<float> {
    float2 a, b;
    __device__ __forceinline__ static Unit load(const void* p, size_t u) {
        float4 t = reinterpret_cast<const float4*>(p)[u];
        return Unit{make_float2(t.x, t.y), make_float2(t.z, t.w)};
    }
    __device__ __forceinline__ void store(void* p, size_t u) const {
        reinterpret_cast<float4*>(p)[u] = make_float4(a.x, a.y, b.x, b.y);
    }
};
template <> struct Unit<double> {
    double2 a, b;
    __device__ __forceinline__ static Unit load(const void* p, size_t u) {
        const double2* d = reinterpret_cast<const double2*>(p);
        return Unit{d[2 * u], d[2 * u + 1]};
    }
    __device__ __forceinline__ void store(void* p, size_t u) const {
        double2* d = reinterpret_cast<double2*>(p);
        d[2 * u] = a; d[2 * u + 1] = b;
    }
};

// Compensated FP32 accumulation of a complex sum (Knuth's two-sum per term), for
// the gamma5 variant's inner products rho = r^H gamma5 r and sigma = p^H gamma5 A p:
// their terms have both signs and cancel down to about ||r||^2 / sqrt(N), so a
// plain FP32 sum would lose three to four digits of them. The per-thread value
// goes to FP64 block and cross-block sums.
struct CompC {
    float sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f;
    __device__ __forceinline__ static void add1(float& s, float& c, float v) {
        const float t = s + v, bp = t - s;
        c += (s - (t - bp)) + (v - bp);
        s = t;
    }
    __device__ __forceinline__ void add(float2 v) { add1(sx, cx, v.x); add1(sy, cy, v.y); }
    __device__ __forceinline__ double2 value() const { return make_double2((double)sx + cx, (double)sy + cy); }
};

// Block and cross-block sum of (z, (a, b)) per slot: in the storage precision,
// or (gamma5 variant with FP32 storage, compensated z) in FP64 throughout.
template <typename S>
__device__ __forceinline__ bool reduce2(const SlotPtrs& P, int kind, bool comp, const CompC& cz, const Acc<S>& acc,
                                        double2 (&tot)[2], unsigned nblocks, unsigned bid) {
    if (comp) {
        double2 v[2] = {cz.value(), make_double2((double)acc.a, (double)acc.b)};
        return reduce_slot<2>(P, kind, v, tot, nblocks, bid);
    }
    cplx<S> v[2];
    acc.to(v);
    return reduce_slot<2>(P, kind, v, tot, nblocks, bid);
}

// gamma5 = diag(1, 1, -1, -1) on a vector unit: units u < N/4 hold spins 0 and 1
// (chunks q = 0..2 of the field layout), the rest spins 2 and 3.
template <typename S> __device__ __forceinline__ Unit<S> g5u(Unit<S> v, size_t u, size_t N) {
    if (u >= N / 4) { v.a = -v.a; v.b = -v.b; }
    return v;
}

// Start: r0 = b - A x_hi (already in r_true, FP64), rhat0 = r0 (gamma5 r0 in the
// gamma5 variant), p = r, phat = rhat, x_lo = 0; rho_0 = (rhat_0, r_0), ||r_0||,
// ||b||  (Algorithm eigBiCG, steps 1-2).
template <typename S>
__global__ void __launch_bounds__(BL_THREADS) start_kernel(SlotState* states, const SlotPtrs* ptrs, size_t N) {
    SlotState& st = states[blockIdx.y];
    const SlotPtrs& P = ptrs[blockIdx.y];
    if (st.status != ST_RUNNING) return;
    if (st.m > 0 && blockIdx.x == 0)   // a fresh window: H is tridiagonal until the first restart
        for (int e = threadIdx.x; e < st.m * st.m; e += blockDim.x) P.H[e] = make_double2(0.0, 0.0);
    using C = cplx<S>;
    Acc<S> acc;   // rho, |r|^2, |b|^2
    CompC cz;     // rho of the gamma5 variant (FP32 storage)
    const bool comp = st.g5 && sizeof(S) == 4;
    const size_t units = N / 2;
    Unit<S> zero{mk<S>(0, 0), mk<S>(0, 0)};
    for (size_t u = blockIdx.x * (size_t)blockDim.x + threadIdx.x; u < units; u += (size_t)gridDim.x * blockDim.x) {
        Unit<double> rt = Unit<double>::load(P.r_true, u);
        Unit<double> bb = Unit<double>::load(P.b, u);
        Unit<S> r{cvt<S>(rt.a), cvt<S>(rt.b)};
        r.store(P.V, u);
        r.store(P.p, u);
        Unit<S> h = r;
        if (st.g5) {   // rhat0 = gamma5 r0: only the window keeps it
            h = g5u(r, u, N);
            if (st.m > 0) h.store(P.W, u);
        } else {
            r.store(P.W, u);
            r.store(P.phat, u);
        }
        zero.store(P.x_lo, u);
        if (comp) {
            if constexpr (sizeof(S) == 4) { cz.add(cdot(h.a, r.a)); cz.add(cdot(h.b, r.b)); }
        } else {
            acc.z = acc.z + cdot(h.a, r.a) + cdot(h.b, r.b);
        }
        acc.a += abs2(r.a) + abs2(r.b);
        acc.b += (S)(cabs2(bb.a) + cabs2(bb.b));
    }
    double2 tot[2];
    if (reduce2<S>(P, CNT_START, comp, cz, acc, tot, gridDim.x, blockIdx.x) && threadIdx.x == 0) {
        st.rho = tot[0];
        st.rnorm = sqrt(tot[1].x);
        st.bnorm = P.bnorm_ref ? *P.bnorm_ref : sqrt(tot[1].y);   // even-odd: ||b|| of the full system
        st.rhat_norm = st.rnorm;
        st.rmax = st.rnorm;
        st.r_ru = st.rnorm;
        st.true_rnorm = st.rnorm;
        st.iter = 0; st.vs = 0; st.need_ru = 0; st.ru_count = 0; st.restarts = 0; st.restart_r = 0;
        st.matvecs = 1; st.live = 1;
        st.alpha_prev = make_double2(0, 0); st.beta_prev = make_double2(0, 0);
        if (st.rnorm <= st.tol * st.bnorm) { st.status = ST_CONVERGED; st.live = 0; }
        // rho_0 = (rhat_0, r_0) must not vanish (e.g. the gamma5 shadow start on a
        // source whose upper and lower spin halves have equal norms)
        else if (!(cabs_(st.rho) >= BREAK_TOL * st.rhat_norm * st.rnorm)) { st.status = ST_BREAKDOWN; st.live = 0; }
    }
    (void)sizeof(C);
}

// Operator pair of one iteration: A p -> Ap[par], A^+ phat -> Ahp[par];
// sigma = (phat, A p) and alpha = rho / sigma in the last block.
// Grid: (site blocks x jobs) flattened with the job index fastest, so the jobs
// that share a block of sites (and its links) run together and the links come
// from DRAM once per launch. Variants (picked by the autotuner):
//   PAIR = false: one thread per (site, operator) job, 2 jobs per slot;
//   PAIR = true : one thread per (site, slot) computes both operators and
//                 shares each link load between them.
//   BZ > 0: a block covers an 8 x 8 x BZ brick of sites (THREADS = 64 BZ) instead
//           of THREADS consecutive sites, so more y and z neighbours are L1 hits.
//   TM (t march, with BZ > 0): the units of a brick at consecutive t are
//           consecutive, so a block walks one brick through several t-planes
//           and the t neighbours of a step are the centres of the steps before
//           and after it (L1 hits instead of L2 reads).
template <int THREADS, int BZ, bool TM = false> struct SiteMap {
    int nunits;
    __device__ __forceinline__ SiteMap(const Geom& g) {
        nunits = BZ > 0 ? (g.L[0] / 8) * (g.L[1] / 8) * (g.L[2] / (BZ > 0 ? BZ : 1)) * g.L[3]
                        : (g.V + THREADS - 1) / THREADS;
    }
    __device__ __forceinline__ int site(const Geom& g, int u) const {   // -1: none
        if (BZ == 0) {
            const int s = u * THREADS + (int)threadIdx.x;
            return s < g.V ? s : -1;
        }
        const int nbx = g.L[0] / 8, nby = g.L[1] / 8, nbz = g.L[2] / (BZ > 0 ? BZ : 1);
        int b = u, t = 0;
        if (TM) { t = u % g.L[3]; b = u / g.L[3]; }
        const int bx = b % nbx, r1 = b / nbx, by = r1 % nby, r2 = r1 / nby, bz = r2 % nbz;
        if (!TM) t = r2 / nbz;
        const int x = bx * 8 + (threadIdx.x & 7), y = by * 8 + ((threadIdx.x >> 3) & 7);
        const int z = bz * BZ + (threadIdx.x >> 6);
        return x + g.L[0] * (y + g.L[1] * (z + g.L[2] * t));
    }
};

//   G5   = true : the gamma5 variant (Sec. 4): one job per slot, A p only, with
//                 phat = gamma5 p formed in registers for sigma; windowed slots
//                 also store A^+ phat = gamma5 A p for the restart's coupling.
template <typename S, int THREADS, int MINB, bool PAIR, int BZ = 0, bool G5 = false, bool TM = false>
__global__ void __launch_bounds__(THREADS, MINB) matvec_kernel(Geom g, const void* links, double kappa,
                                                               SlotState* states, const SlotPtrs* ptrs,
                                                               int njobs) {
    const int job = blockIdx.x % njobs, sblock = blockIdx.x / njobs, nsb = gridDim.x / njobs;
    const SiteMap<THREADS, BZ, TM> map(g);
    // each block takes a contiguous run of site units (neighbouring sites stay on one SM)
    const int per = (map.nunits + nsb - 1) / nsb;
    const int u0 = sblock * per, u1 = min(map.nunits, u0 + per);
    const int slot = (PAIR || G5) ? job : job >> 1, which = (PAIR || G5) ? 0 : job & 1;
    SlotState& st = states[slot];
    const SlotPtrs& P = ptrs[slot];
    if (st.status != ST_RUNNING || st.stab) return;   // BiCGStab slots run their own kernels
    using C = cplx<S>;
    const int par = st.iter & 1;
    typename LinkSel<S>::type U{reinterpret_cast<decltype(U.u)>(links), g.V};
    const S k = (S)kappa;
    Acc<S> sacc;   // sigma, |phat|^2, |Ap|^2
    CompC scomp;   // sigma of the gamma5 variant (FP32)
    if (PAIR) {
        FieldIn<S> inp{P.p, g.V}, inh{P.phat, g.V};
        for (int u = u0; u < u1; ++u) {
            const int s = map.site(g, u);
            if (s < 0) continue;
            C a[12], b[12], self[12];
            hop_site_pair<S>(g, U, inp, inh, s, a, b);
            inp.load(s, self);
#pragma unroll
            for (int c = 0; c < 12; ++c) a[c] = self[c] - k * a[c];
            Field<S>::store(P.Ap[par], g.V, s, a);
            inh.load(s, self);
#pragma unroll
            for (int c = 0; c < 12; ++c) {
                b[c] = self[c] - k * b[c];
                sacc.z = sacc.z + cdot(self[c], a[c]);
                sacc.a += abs2(self[c]);
                sacc.b += abs2(a[c]);
            }
            Field<S>::store(P.Ahp[par], g.V, s, b);
        }
    } else {
        FieldIn<S> in{which ? P.phat : P.p, g.V};
        void* out = which ? P.Ahp[par] : P.Ap[par];
        const bool win = G5 && st.m > 0;
        for (int u = u0; u < u1; ++u) {
            const int s = map.site(g, u);
            if (s < 0) continue;
            C acc[12], self[12];
            if (which) hop_site<true, S>(g, U, in, s, acc);
            else hop_site<false, S>(g, U, in, s, acc);
            in.load(s, self);
            const C (&self_p)[12] = self;
#pragma unroll
            for (int c = 0; c < 12; ++c) acc[c] = self[c] - k * acc[c];
            Field<S>::store(out, g.V, s, acc);
            if (G5) {   // phat = gamma5 p: spins 0, 1 (c < 6) keep their sign
#pragma unroll
                for (int c = 0; c < 12; ++c) {
                    const C ph = c < 6 ? self_p[c] : -self_p[c];
                    if constexpr (sizeof(S) == 4) scomp.add(cdot(ph, acc[c]));
                    else sacc.z = sacc.z + cdot(ph, acc[c]);
                    sacc.a += abs2(ph);
                    sacc.b += abs2(acc[c]);
                }
                if (win) {
#pragma unroll
                    for (int c = 6; c < 12; ++c) acc[c] = -acc[c];
                    Field<S>::store(P.Ahp[par], g.V, s, acc);
                }
            } else if (!which) {
                C ph[12];
                Field<S>::load(P.phat, g.V, s, ph);
#pragma unroll
                for (int c = 0; c < 12; ++c) {
                    sacc.z = sacc.z + cdot(ph[c], acc[c]);
                    sacc.a += abs2(ph[c]);
                    sacc.b += abs2(acc[c]);
                }
            }
        }
        if (which) return;
    }
    double2 tot[2];
    if (reduce2<S>(P, CNT_MATVEC, G5 && sizeof(S) == 4, scomp, sacc, tot, nsb, sblock) && threadIdx.x == 0) {
        st.sigma = tot[0];
        st.phat_norm = sqrt(tot[1].x);
        st.ap_norm = sqrt(tot[1].y);
        st.matvecs += G5 ? 1 : 2;   // the gamma5 variant applies A only
        if (!(cabs_(st.sigma) >= BREAK_TOL * st.phat_norm * st.ap_norm) || cabs2(st.sigma) == 0.0) {
            st.status = ST_BREAKDOWN;
        } else {
            st.alpha = cdiv(st.rho, st.sigma);
        }
    }
}

// Operator pair with one warp per (32-site group, job): a block holds the
// jobs (slot, operator) of up to JPB/2 slots for the same sites, so the link
// loads of one site group are shared through L1 by every job of the block.
// Blocks loop over site groups (grid-stride, a fixed grid independent of the
// number of slots, so each slot's sigma partition does not depend on the
// batch). sigma: per-lane FP32 sums, warp sums, one FP64 partial per (block,
// slot) in that slot's partial buffer; the last block of the launch (one
// counter in slot 0) adds each slot's partials in block order.
constexpr int GRP_BLOCKS = 4 * 152;   // blocks per job half (fixed)
template <int JPB, int MINB>
__global__ void __launch_bounds__(32 * JPB, MINB)
    matvec_group_kernel(Geom g, const void* links, float kappa, SlotState* states, const SlotPtrs* ptrs,
                        int nslots) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int njobs = 2 * nslots;
    const int job = blockIdx.y * JPB + warp;
    const int slot = job >> 1, which = job & 1;
    const int ngroups = (g.V + 31) >> 5;
    LinksF U{reinterpret_cast<const float4*>(links), g.V};
    Acc<float> sacc;
    if (job < njobs && states[slot].status == ST_RUNNING && !states[slot].stab) {
        const SlotState& st = states[slot];
        const SlotPtrs& P = ptrs[slot];
        const int par = st.iter & 1;
        FieldIn<float> in{which ? P.phat : P.p, g.V};
        void* out = which ? P.Ahp[par] : P.Ap[par];
        for (int grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
            const int s = (grp << 5) + lane;
            if (s >= g.V) break;
            float2 acc[12], self[12];
            if (which) hop_site<true, float>(g, U, in, s, acc);
            else hop_site<false, float>(g, U, in, s, acc);
            in.load(s, self);
#pragma unroll
            for (int c = 0; c < 12; ++c) acc[c] = self[c] - kappa * acc[c];
            Field<float>::store(out, g.V, s, acc);
            if (!which) {
                float2 ph[12];
                Field<float>::load(P.phat, g.V, s, ph);
#pragma unroll
                for (int c = 0; c < 12; ++c) {
                    sacc.z = sacc.z + cdot(ph[c], acc[c]);
                    sacc.a += abs2(ph[c]);
                    sacc.b += abs2(acc[c]);
                }
            }
        }
        if (!which) {
            float2 z = warp_sum(sacc.z);
            float2 ab = warp_sum(make_float2(sacc.a, sacc.b));
            if (lane == 0) {
                double2* pp = P.partials + (size_t)CNT_MATVEC * PARTIAL_STRIDE + (size_t)blockIdx.x * 2;
                pp[0] = to_d(z);
                pp[1] = to_d(ab);
                __threadfence();
            }
        }
    }
    // one arrival per block; the last block finishes every slot
    if (!last_block(ptrs[0].counters + CNT_GROUP, gridDim.x * gridDim.y)) return;
    for (int sl = warp; sl < nslots; sl += JPB) {
        SlotState& st = states[sl];
        if (st.status != ST_RUNNING || st.stab) continue;
        const double2* pp = ptrs[sl].partials + (size_t)CNT_MATVEC * PARTIAL_STRIDE;
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
            if (!(cabs_(st.sigma) >= BREAK_TOL * st.phat_norm * st.ap_norm) || cabs2(st.sigma) == 0.0) {
                st.status = ST_BREAKDOWN;
            } else {
                st.alpha = cdiv(st.rho, st.sigma);
            }
        }
    }
}

// r_j = r_{j-1} - alpha A p; rhat_j = rhat_{j-1} - conj(alpha) A^+ phat;
// rho_j, ||r_j||, ||rhat_j||; flags for the FP64 residual check. The solution
// update x_lo += alpha p is owed (x_owed): the direction update, which reads p
// anyway, or the reliable-update fold, or the final fold adds it.
template <typename S>
__global__ void __launch_bounds__(BL_THREADS) update_kernel(SlotState* states, const SlotPtrs* ptrs, size_t N) {
    SlotState& st = states[blockIdx.y];
    const SlotPtrs& P = ptrs[blockIdx.y];
    if (st.status != ST_RUNNING || st.stab) return;   // BiCGStab slots run their own kernels
    using C = cplx<S>;
    const int par = st.iter & 1;
    const C al = cvt<S>(st.alpha), alc = conj_(al);
    const void* rin = slot_field<S>(P.V, cur_slot(st), N);
    void* rout = slot_field<S>(P.V, next_slot(st), N);
    const void* hin = slot_field<S>(P.W, cur_slot(st), N);
    void* hout = slot_field<S>(P.W, next_slot(st), N);
    const void* ap = P.Ap[par];
    const void* ahp = P.Ahp[par];
    Acc<S> acc;   // rho_j, |r_j|^2, |rhat_j|^2
    CompC cz;     // rho_j of the gamma5 variant (FP32 storage)
    const bool comp = st.g5 && sizeof(S) == 4;
    const size_t units = N / 2;
    if (st.g5) {   // rhat_j = gamma5 r_j: one vector update, the window keeps gamma5 r_j
        const bool win = st.m > 0;
        for (size_t u = blockIdx.x * (size_t)blockDim.x + threadIdx.x; u < units; u += (size_t)gridDim.x * blockDim.x) {
            Unit<S> r = Unit<S>::load(rin, u), a = Unit<S>::load(ap, u);
            r.a = r.a - al * a.a; r.b = r.b - al * a.b;
            r.store(rout, u);
            const Unit<S> h = g5u(r, u, N);
            if (win) h.store(hout, u);
            if constexpr (sizeof(S) == 4) { cz.add(cdot(h.a, r.a)); cz.add(cdot(h.b, r.b)); }
            else acc.z = acc.z + cdot(h.a, r.a) + cdot(h.b, r.b);
            acc.a += abs2(r.a) + abs2(r.b);
        }
        acc.b = acc.a;
    } else {
        for (size_t u = blockIdx.x * (size_t)blockDim.x + threadIdx.x; u < units; u += (size_t)gridDim.x * blockDim.x) {
            Unit<S> r = Unit<S>::load(rin, u), a = Unit<S>::load(ap, u);
            Unit<S> h = Unit<S>::load(hin, u), ah = Unit<S>::load(ahp, u);
            r.a = r.a - al * a.a; r.b = r.b - al * a.b;
            h.a = h.a - alc * ah.a; h.b = h.b - alc * ah.b;
            r.store(rout, u);
            h.store(hout, u);
            acc.z = acc.z + cdot(h.a, r.a) + cdot(h.b, r.b);
            acc.a += abs2(r.a) + abs2(r.b);
            acc.b += abs2(h.a) + abs2(h.b);
        }
    }
    double2 tot[2];
    if (reduce2<S>(P, CNT_UPDATE, comp, cz, acc, tot, gridDim.x, blockIdx.x) && threadIdx.x == 0) {
        st.rho_new = tot[0];
        st.rnorm_new = sqrt(tot[1].x);
        st.rhat_norm = sqrt(tot[1].y);
        st.x_owed = 1;
        if (!isfinite(st.rnorm_new) || !isfinite(st.rho_new.x) || !isfinite(st.rho_new.y)) {
            st.status = ST_BREAKDOWN;
        } else {
            // Reliable update (FP32 Krylov vectors): when the residual has dropped by
            // delta since the last update, or far below the largest residual seen
            // since then (the recursion's rounding error scales with that maximum);
            // and always to confirm convergence. A slot with rec_stop set (the
            // eigBiCG leg of a mixed-precision solve) never replaces r, which
            // would break the Lanczos relation of its window, and stops at the
            // first recursive convergence candidate instead.
            if (st.rnorm_new <= st.tol * st.bnorm) {
                if (st.rec_stop) st.status = ST_CONVERGED;
                else st.need_ru = 1;
            }
            if (st.rnorm_new > st.rmax) st.rmax = st.rnorm_new;
            if (st.delta > 0.0 && (st.rnorm_new < st.delta * st.r_ru || st.rnorm_new < 1e-3 * st.rmax)) st.need_ru = 1;
        }
    }
}

// FP64 true residual r = b - A x_hi for slots that asked for it (x_lo has been
// folded into x_hi just before).
// check_only = 0: inside the iteration (converged if ||r|| <= tol ||b||);
// check_only = 1: final report for every slot that was started.
template <int THREADS, int MINB>
__global__ void __launch_bounds__(THREADS, MINB) true_resid_kernel(Geom g, const void* links64, double kappa,
                                                                   SlotState* states, const SlotPtrs* ptrs,
                                                                   int check_only) {
    SlotState& st = states[blockIdx.y];
    const SlotPtrs& P = ptrs[blockIdx.y];
    if (check_only) {
        if (st.status == ST_IDLE) return;
    } else if (st.status != ST_RUNNING || !st.need_ru) {
        return;
    }
    LinksD U{reinterpret_cast<const double2*>(links64), g.V};
    FieldIn<double> in{P.x_hi, g.V};
    double2 v[1] = {make_double2(0, 0)};
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < g.V; s += gridDim.x * blockDim.x) {
        double2 acc[12], self[12], b[12];
        hop_site<false, double>(g, U, in, s, acc);
        in.load(s, self);
        Field<double>::load(P.b, g.V, s, b);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            acc[c] = b[c] - (self[c] - kappa * acc[c]);
            v[0].x += cabs2(acc[c]);
        }
        Field<double>::store(P.r_true, g.V, s, acc);
    }
    double2 tot[1];
    if (reduce_slot<1>(P, CNT_RU, v, tot, gridDim.x, blockIdx.x) && threadIdx.x == 0) {
        st.true_rnorm = sqrt(tot[0].x);
        st.matvecs += 1;
        if (!check_only && st.true_rnorm <= st.tol * st.bnorm) st.status = ST_CONVERGED;
    }
}

// The in-iteration reliable-update residual b - A x_hi with A x_hi in
// double-float arithmetic (dfloat.cuh): same contract as true_resid_kernel
// with check_only = 0.
// One hop in double-float: each colour row of U h (or U^+ h) is formed and
// added into the accumulator at once, and the link is read row by row, so
// only a row of U and one colour of U h are live next to h and the sums.
template <int MU, int SG>
__device__ __forceinline__ void recon_row_df(dfc a, dfc b, int c, dfc (&acc)[12]) {
    dfc l0, l1;   // M^+ (a, b)
    if (MU == 0) { l0 = mul_i(b); l1 = mul_i(a); }
    else if (MU == 1) { l0 = b; l1 = -a; }
    else if (MU == 2) { l0 = mul_i(a); l1 = mul_mi(b); }
    else { l0 = a; l1 = b; }
    acc[c] = acc[c] + a;
    acc[3 + c] = acc[3 + c] + b;
    if (SG > 0) { acc[6 + c] = acc[6 + c] + l0; acc[9 + c] = acc[9 + c] + l1; }
    else { acc[6 + c] = acc[6 + c] - l0; acc[9 + c] = acc[9 + c] - l1; }
}
template <int MU, bool BWD>
__device__ __forceinline__ void hop_df(const Nbr& nb, const LinksDF& U, const FieldDF& in, int s, dfc (&acc)[12]) {
    constexpr int SG = BWD ? +1 : -1;
    dfc h[2][3];
    {
        dfc psi[12];
        in.load(BWD ? nb.b[MU] : nb.f[MU], psi);
        project<MU, SG>(psi, h);
    }
    const int ls = BWD ? nb.b[MU] : s;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        dfc u[3];   // row r of U (forward) or column r (backward, conjugated below)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float4 t = __ldg(U.u + (size_t)(MU * 9 + (BWD ? 3 * c + r : 3 * r + c)) * U.V + ls);
            u[c] = {{t.x, t.z}, {t.y, t.w}};
        }
        dfc o[2];
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            Dot2 re, im;
            if (!BWD) {
                re.first(u[0].x, h[a][0].x); re.add(-u[0].y, h[a][0].y);
                im.first(u[0].x, h[a][0].y); im.add(u[0].y, h[a][0].x);
#pragma unroll
                for (int c = 1; c < 3; ++c) {
                    re.add(u[c].x, h[a][c].x); re.add(-u[c].y, h[a][c].y);
                    im.add(u[c].x, h[a][c].y); im.add(u[c].y, h[a][c].x);
                }
            } else {
                re.first(u[0].x, h[a][0].x); re.add(u[0].y, h[a][0].y);
                im.first(u[0].x, h[a][0].y); im.add(-u[0].y, h[a][0].x);
#pragma unroll
                for (int c = 1; c < 3; ++c) {
                    re.add(u[c].x, h[a][c].x); re.add(u[c].y, h[a][c].y);
                    im.add(u[c].x, h[a][c].y); im.add(-u[c].y, h[a][c].x);
                }
            }
            o[a] = {re.done(), im.done()};
        }
        recon_row_df<MU, SG>(o[0], o[1], r, acc);
    }
}
template <int THREADS, int MINB>
__global__ void __launch_bounds__(THREADS, MINB) true_resid_df_kernel(Geom g, const float4* links_df, double kappa,
                                                                      SlotState* states, const SlotPtrs* ptrs) {
    SlotState& st = states[blockIdx.y];
    const SlotPtrs& P = ptrs[blockIdx.y];
    if (st.status != ST_RUNNING || !st.need_ru) return;
    const LinksDF U{links_df, g.V};
    const FieldDF in{P.x_df, g.V};
    double2 v[1] = {make_double2(0, 0)};
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < g.V; s += gridDim.x * blockDim.x) {
        const Nbr nb(g, s);
        dfc acc[12];
#pragma unroll
        for (int c = 0; c < 12; ++c) acc[c] = {{0.f, 0.f}, {0.f, 0.f}};
        hop_df<0, false>(nb, U, in, s, acc);
        hop_df<0, true>(nb, U, in, s, acc);
        hop_df<1, false>(nb, U, in, s, acc);
        hop_df<1, true>(nb, U, in, s, acc);
        hop_df<2, false>(nb, U, in, s, acc);
        hop_df<2, true>(nb, U, in, s, acc);
        hop_df<3, false>(nb, U, in, s, acc);
        hop_df<3, true>(nb, U, in, s, acc);
        double2 self[12], b[12];
        Field<double>::load(P.x_hi, g.V, s, self);
        Field<double>::load(P.b, g.V, s, b);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            const double2 a = make_double2(df_value(acc[c].x), df_value(acc[c].y));
            b[c] = b[c] - (self[c] - kappa * a);
            v[0].x += cabs2(b[c]);
        }
        Field<double>::store(P.r_true, g.V, s, b);
    }
    double2 tot[1];
    if (reduce_slot<1>(P, CNT_RU, v, tot, gridDim.x, blockIdx.x) && threadIdx.x == 0) {
        st.true_rnorm = sqrt(tot[0].x);
        st.matvecs += 1;
        if (st.true_rnorm <= st.tol * st.bnorm) st.status = ST_CONVERGED;
    }
}

// Reliable update, first half: x_hi += x_lo, x_lo = 0 for slots that asked for it.
template <typename S>
__global__ void __launch_bounds__(BL_THREADS) fold_ru_kernel(SlotState* states, const SlotPtrs* ptrs, size_t N) {
    const SlotState& st = states[blockIdx.y];
    const SlotPtrs& P = ptrs[blockIdx.y];
    if (st.status != ST_RUNNING || !st.need_ru) return;
    const size_t units = N / 2;
    const cplx<S> al = cvt<S>(st.alpha);
    Unit<S> zero{mk<S>(0, 0), mk<S>(0, 0)};
    for (size_t u = blockIdx.x * (size_t)blockDim.x + threadIdx.x; u < units; u += (size_t)gridDim.x * blockDim.x) {
        Unit<double> xh = Unit<double>::load(P.x_hi, u);
        Unit<S> xl = Unit<S>::load(P.x_lo, u);
        if (st.x_owed) {   // alpha p of this iteration's residual update
            const Unit<S> p = Unit<S>::load(P.p, u);
            xl.a = xl.a + al * p.a; xl.b = xl.b + al * p.b;
        }
        xh.a = xh.a + to_d(xl.a); xh.b = xh.b + to_d(xl.b);
        xh.store(P.x_hi, u);
        zero.store(P.x_lo, u);
        if (P.x_df) {   // the double-float copy read by the reliable-update residual
            const dfl ar = df_split(xh.a.x), ai = df_split(xh.a.y), br = df_split(xh.b.x), bi = df_split(xh.b.y);
            P.x_df[2 * u] = make_float4(ar.h, ai.h, ar.l, ai.l);
            P.x_df[2 * u + 1] = make_float4(br.h, bi.h, br.l, bi.l);
        }
    }
}

// Reliable update, second half: unless converged, the recursive residual r_j is
// replaced by the true one and rho_j recomputed.
template <typename S>
__global__ void __launch_bounds__(BL_THREADS) replace_kernel(SlotState* states, const SlotPtrs* ptrs, size_t N) {
    SlotState& st = states[blockIdx.y];
    const SlotPtrs& P = ptrs[blockIdx.y];
    if (!st.live || !st.need_ru || (st.status != ST_RUNNING && st.status != ST_CONVERGED)) return;
    const bool run = st.status == ST_RUNNING;
    void* rcur = slot_field<S>(P.V, next_slot(st), N);
    void* hcur = slot_field<S>(P.W, next_slot(st), N);
    cplx<S> rho = mk<S>(S(0), S(0));
    CompC cz;   // gamma5 variant, FP32 storage
    const bool comp = st.g5 && sizeof(S) == 4;
    const size_t units = N / 2;
    for (size_t u = blockIdx.x * (size_t)blockDim.x + threadIdx.x; u < units; u += (size_t)gridDim.x * blockDim.x) {
        if (run) {
            Unit<double> rt = Unit<double>::load(P.r_true, u);
            Unit<S> r{cvt<S>(rt.a), cvt<S>(rt.b)};
            r.store(rcur, u);
            Unit<S> h;
            if (st.g5) {   // the shadow residual follows: rhat = gamma5 r
                h = g5u(r, u, N);
                if (st.m > 0) h.store(hcur, u);
            } else {
                h = Unit<S>::load(hcur, u);
            }
            if (comp) {
                if constexpr (sizeof(S) == 4) { cz.add(cdot(h.a, r.a)); cz.add(cdot(h.b, r.b)); }
            } else {
                rho = rho + cdot(h.a, r.a) + cdot(h.b, r.b);
            }
        }
    }
    double2 tot[1];
    bool last;
    if (comp) {
        double2 v[1] = {cz.value()};
        last = reduce_slot<1>(P, CNT_REPLACE, v, tot, gridDim.x, blockIdx.x);
    } else {
        cplx<S> v[1] = {rho};
        last = reduce_slot<1>(P, CNT_REPLACE, v, tot, gridDim.x, blockIdx.x);
    }
    if (last && threadIdx.x == 0) {
        if (run) {
            st.rho_new = tot[0];
            st.rnorm_new = st.true_rnorm;
            st.rmax = st.true_rnorm;
            st.r_ru = st.true_rnorm;
        }
        st.need_ru = 0;
        st.ru_count += 1;
        st.x_owed = 0;   // the fold added alpha p
    }
}

// Scalar bookkeeping of one iteration (one thread per slot):
// beta_{j-1} = rho_j / rho_{j-1}; window append v = r/||r||, w = (||r||/conj(rho)) rhat;
// tridiagonal entries of H (Algorithm eigBiCG, step 3); iteration counters.
__global__ void scalars_kernel(SlotState* states, const SlotPtrs* ptrs) {
    if (threadIdx.x != 0) return;
    SlotState& st = states[blockIdx.x];
    const SlotPtrs& P = ptrs[blockIdx.x];
    if (!st.live || st.stab) return;
    if (st.status == ST_BREAKDOWN) { st.live = 0; return; }
    const double2 beta = cdiv(st.rho_new, st.rho);
    if (st.m > 0) {
        const int k = st.vs;   // 0-based index of the appended vector
        const int m = st.m;
        P.vscale[k] = 1.0 / st.rnorm;
        P.wscale[k] = cdiv(make_double2(st.rnorm, 0.0), conj_(st.rho));
        const double2 inv_a = cdiv(make_double2(1.0, 0.0), st.alpha);
        double2 diag = inv_a;
        if (st.iter > 0) diag = diag + cdiv(st.beta_prev, st.alpha_prev);
        P.H[k * m + k] = diag;
        if (k + 1 < m) {
            P.H[k * m + k + 1] = -(st.rnorm / st.rnorm_new) * cdiv(beta, st.alpha);
            P.H[(k + 1) * m + k] = -(st.rnorm_new / st.rnorm) * inv_a;
        }
        st.vs = k + 1;
    }
    st.beta = beta;
    st.alpha_prev = st.alpha;
    st.beta_prev = beta;
    st.rho = st.rho_new;
    st.rnorm = st.rnorm_new;
    st.iter += 1;
    if (st.status == ST_RUNNING) {
        if (st.iter >= st.maxiter) st.status = ST_NOCONV;
        else if (!(cabs_(st.rho) >= BREAK_TOL * st.rhat_norm * st.rnorm)) st.status = ST_BREAKDOWN;
    }
    if (st.status != ST_RUNNING) st.live = 0;
    // the direction update adds the owed alpha p; a slot that stops here keeps it
    // owed for the final fold
    if (st.status == ST_RUNNING) { st.x_dir = st.x_owed; st.x_owed = 0; }
    else st.x_dir = 0;
}

// p_j = r_j + beta p_{j-1}, phat_j = rhat_j + conj(beta) phat_{j-1}.
template <typename S>
__global__ void __launch_bounds__(BL_THREADS) direction_kernel(SlotState* states, const SlotPtrs* ptrs, size_t N) {
    const SlotState& st = states[blockIdx.y];
    const SlotPtrs& P = ptrs[blockIdx.y];
    if (st.status != ST_RUNNING || st.stab) return;   // BiCGStab slots run their own kernels
    using C = cplx<S>;
    const C be = cvt<S>(st.beta), bec = conj_(be);
    const C al = cvt<S>(st.alpha);
    const bool addx = st.x_dir != 0;
    const bool g5 = st.g5 != 0;   // gamma5 variant: phat = gamma5 p is never stored
    const void* r = slot_field<S>(P.V, cur_slot(st), N);
    const void* h = slot_field<S>(P.W, cur_slot(st), N);
    const size_t units = N / 2;
    for (size_t u = blockIdx.x * (size_t)blockDim.x + threadIdx.x; u < units; u += (size_t)gridDim.x * blockDim.x) {
        Unit<S> p = Unit<S>::load(P.p, u), ph, hh, rr = Unit<S>::load(r, u);
        if (!g5) { ph = Unit<S>::load(P.phat, u); hh = Unit<S>::load(h, u); }
        if (addx) {   // x_lo += alpha p_{j-1} (owed by the residual update)
            Unit<S> x = Unit<S>::load(P.x_lo, u);
            x.a = x.a + al * p.a; x.b = x.b + al * p.b;
            x.store(P.x_lo, u);
        }
        p.a = rr.a + be * p.a; p.b = rr.b + be * p.b;
        p.store(P.p, u);
        if (!g5) {
            ph.a = hh.a + bec * ph.a; ph.b = hh.b + bec * ph.b;
            ph.store(P.phat, u);
        }
    }
}

// ------------------------------------------------------------- BiCGStab
// The phase-2 solver of Alg. Incremental eigBiCG as the paper runs it (Sec. 2),
// BiCGStab (van der Vorst) with the shadow start rhat = r_0 (W slot 0):
//   p = r + beta (p - omega v);  v = A p;  alpha = rho / (rhat, v);  s = r - alpha v;
//   t = A s;  omega = (t, s) / (t, t);  x += alpha p + omega s;  r = s - omega t;
//   rho' = (rhat, r);  beta = (rho' / rho) (alpha / omega).
// Buffers of a slot: r in V slot 0, rhat in W slot 0, p, v = Ap[0], s in the phat
// buffer, t = Ahp[0]. Two products with A per step, none with A^+.

// p = r + beta (p - omega v); the first step (iter 0) takes p = r.
template <typename S>
__global__ void __launch_bounds__(BL_THREADS) stab_dir_kernel(SlotState* states, const SlotPtrs* ptrs, size_t N) {
    const SlotState& st = states[blockIdx.y];
    const SlotPtrs& P = ptrs[blockIdx.y];
    if (st.status != ST_RUNNING || !st.stab) return;
    using C = cplx<S>;
    const C be = cvt<S>(st.beta), om = cvt<S>(st.omega);
    const bool first = st.iter == 0;
    const size_t units = N / 2;
    for (size_t u = blockIdx.x * (size_t)blockDim.x + threadIdx.x; u < units; u += (size_t)gridDim.x * blockDim.x) {
        Unit<S> r = Unit<S>::load(P.V, u);
        if (!first) {
            const Unit<S> p = Unit<S>::load(P.p, u), v = Unit<S>::load(P.Ap[0], u);
            r.a = r.a + be * (p.a - om * v.a);
            r.b = r.b + be * (p.b - om * v.b);
        }
        r.store(P.p, u);
    }
}

// PHASE 1: v = A p, sigma = (rhat, v), alpha = rho / sigma.
// PHASE 2: t = A s, (t, s), (t, t), omega = (t, s) / (t, t).
// One job per slot (grid: site blocks x slots, slots fastest).
template <typename S, int THREADS, int MINB, int PHASE>
__global__ void __launch_bounds__(THREADS, MINB) stab_matvec_kernel(Geom g, const void* links, double kappa,
                                                                    SlotState* states, const SlotPtrs* ptrs,
                                                                    int nslots) {
    const int slot = blockIdx.x % nslots, sblock = blockIdx.x / nslots, nsb = gridDim.x / nslots;
    SlotState& st = states[slot];
    const SlotPtrs& P = ptrs[slot];
    if (st.status != ST_RUNNING || !st.stab) return;
    using C = cplx<S>;
    typename LinkSel<S>::type U{reinterpret_cast<decltype(U.u)>(links), g.V};
    FieldIn<S> in{PHASE == 1 ? P.p : P.phat, g.V};
    void* out = PHASE == 1 ? P.Ap[0] : P.Ahp[0];
    const S k = (S)kappa;
    Acc<S> acc;   // PHASE 1: (rhat, v), |rhat|^2, |v|^2;  PHASE 2: (t, s), (t, t), |s|^2
    for (int s = sblock * blockDim.x + threadIdx.x; s < g.V; s += nsb * blockDim.x) {
        C o[12], self[12];
        hop_site<false, S>(g, U, in, s, o);
        in.load(s, self);
#pragma unroll
        for (int c = 0; c < 12; ++c) o[c] = self[c] - k * o[c];
        Field<S>::store(out, g.V, s, o);
        if (PHASE == 1) {
            C h[12];
            Field<S>::load(P.W, g.V, s, h);
#pragma unroll
            for (int c = 0; c < 12; ++c) {
                acc.z = acc.z + cdot(h[c], o[c]);
                acc.a += abs2(h[c]);
                acc.b += abs2(o[c]);
            }
        } else {
#pragma unroll
            for (int c = 0; c < 12; ++c) {
                acc.z = acc.z + cdot(o[c], self[c]);
                acc.a += abs2(o[c]);
                acc.b += abs2(self[c]);
            }
        }
    }
    cplx<S> v[2];
    acc.to(v);
    double2 tot[2];
    if (reduce_slot<2>(P, CNT_MATVEC, v, tot, nsb, sblock) && threadIdx.x == 0) {
        st.matvecs += 1;
        if (PHASE == 1) {
            st.sigma = tot[0];
            st.phat_norm = sqrt(tot[1].x);
            st.ap_norm = sqrt(tot[1].y);
            if (!(cabs_(st.sigma) >= BREAK_TOL * st.phat_norm * st.ap_norm) || cabs2(st.sigma) == 0.0)
                st.status = ST_BREAKDOWN;
            else
                st.alpha = cdiv(st.rho, st.sigma);
        } else {
            st.ts = tot[0];
            st.tt = tot[1].x;
            st.omega = st.tt > 0.0 ? cdiv(st.ts, make_double2(st.tt, 0.0)) : make_double2(0.0, 0.0);
        }
    }
}

// s = r - alpha v  (into the phat buffer)
template <typename S>
__global__ void __launch_bounds__(BL_THREADS) stab_s_kernel(SlotState* states, const SlotPtrs* ptrs, size_t N) {
    const SlotState& st = states[blockIdx.y];
    const SlotPtrs& P = ptrs[blockIdx.y];
    if (st.status != ST_RUNNING || !st.stab) return;
    const cplx<S> al = cvt<S>(st.alpha);
    const size_t units = N / 2;
    for (size_t u = blockIdx.x * (size_t)blockDim.x + threadIdx.x; u < units; u += (size_t)gridDim.x * blockDim.x) {
        Unit<S> r = Unit<S>::load(P.V, u);
        const Unit<S> v = Unit<S>::load(P.Ap[0], u);
        r.a = r.a - al * v.a;
        r.b = r.b - al * v.b;
        r.store(P.phat, u);
    }
}

// x_lo += alpha p + omega s;  r = s - omega t;  rho' = (rhat, r), ||r||; the
// reliable-update flags as in the BiCG residual update.
template <typename S>
__global__ void __launch_bounds__(BL_THREADS) stab_update_kernel(SlotState* states, const SlotPtrs* ptrs, size_t N) {
    SlotState& st = states[blockIdx.y];
    const SlotPtrs& P = ptrs[blockIdx.y];
    if (st.status != ST_RUNNING || !st.stab) return;
    using C = cplx<S>;
    const C al = cvt<S>(st.alpha), om = cvt<S>(st.omega);
    Acc<S> acc;   // rho', |r|^2
    const size_t units = N / 2;
    for (size_t u = blockIdx.x * (size_t)blockDim.x + threadIdx.x; u < units; u += (size_t)gridDim.x * blockDim.x) {
        Unit<S> x = Unit<S>::load(P.x_lo, u);
        const Unit<S> p = Unit<S>::load(P.p, u), sv = Unit<S>::load(P.phat, u), t = Unit<S>::load(P.Ahp[0], u);
        const Unit<S> h = Unit<S>::load(P.W, u);
        x.a = x.a + al * p.a + om * sv.a;
        x.b = x.b + al * p.b + om * sv.b;
        x.store(P.x_lo, u);
        Unit<S> r{sv.a - om * t.a, sv.b - om * t.b};
        r.store(P.V, u);
        acc.z = acc.z + cdot(h.a, r.a) + cdot(h.b, r.b);
        acc.a += abs2(r.a) + abs2(r.b);
    }
    cplx<S> v[2];
    acc.to(v);
    double2 tot[2];
    if (reduce_slot<2>(P, CNT_UPDATE, v, tot, gridDim.x, blockIdx.x) && threadIdx.x == 0) {
        st.rho_new = tot[0];
        st.rnorm_new = sqrt(tot[1].x);
        st.x_owed = 0;   // x is complete after this step
        if (!isfinite(st.rnorm_new) || !isfinite(st.rho_new.x) || !isfinite(st.rho_new.y)) {
            st.status = ST_BREAKDOWN;
        } else {
            if (st.rnorm_new <= st.tol * st.bnorm) st.need_ru = 1;
            if (st.rnorm_new > st.rmax) st.rmax = st.rnorm_new;
            if (st.delta > 0.0 && (st.rnorm_new < st.delta * st.r_ru || st.rnorm_new < 1e-3 * st.rmax)) st.need_ru = 1;
        }
    }
}

// beta = (rho' / rho) (alpha / omega); counters; maxiter and breakdown (rho or omega).
__global__ void stab_scalars_kernel(SlotState* states) {
    if (threadIdx.x != 0) return;
    SlotState& st = states[blockIdx.x];
    if (!st.live || !st.stab) return;
    if (st.status == ST_BREAKDOWN) { st.live = 0; return; }
    st.iter += 1;
    const bool om0 = cabs2(st.omega) == 0.0;
    if (!om0) st.beta = cdiv(st.rho_new, st.rho) * cdiv(st.alpha, st.omega);
    st.rho = st.rho_new;
    st.rnorm = st.rnorm_new;
    if (st.status == ST_RUNNING) {
        if (st.iter >= st.maxiter) st.status = ST_NOCONV;
        else if (om0 || !(cabs_(st.rho) >= BREAK_TOL * st.rhat_norm * st.rnorm)) st.status = ST_BREAKDOWN;
    }
    if (st.status != ST_RUNNING) st.live = 0;
}

// Fold x_lo into x_hi at the end of a solve (x = 0 for a zero source).
template <typename S>
__global__ void fold_kernel(SlotState* states, const SlotPtrs* ptrs, size_t N) {
    const SlotState& st = states[blockIdx.y];
    const SlotPtrs& P = ptrs[blockIdx.y];
    if (st.status == ST_IDLE) return;
    const bool zero_src = st.bnorm == 0.0;
    const bool owed = st.x_owed != 0;   // the last residual update's alpha p (no direction update ran)
    const cplx<S> al = cvt<S>(st.alpha);
    const size_t units = N / 2;
    Unit<S> zero{mk<S>(0, 0), mk<S>(0, 0)};
    for (size_t u = blockIdx.x * (size_t)blockDim.x + threadIdx.x; u < units; u += (size_t)gridDim.x * blockDim.x) {
        Unit<double> xh = Unit<double>::load(P.x_hi, u);
        Unit<S> xl = Unit<S>::load(P.x_lo, u);
        if (owed) {
            const Unit<S> p = Unit<S>::load(P.p, u);
            xl.a = xl.a + al * p.a; xl.b = xl.b + al * p.b;
        }
        if (zero_src) { xh.a = make_double2(0, 0); xh.b = make_double2(0, 0); }
        else { xh.a = xh.a + to_d(xl.a); xh.b = xh.b + to_d(xl.b); }
        xh.store(P.x_hi, u);
        zero.store(P.x_lo, u);
    }
}

// -------------------------------------------------------- restart product
// In-place window product of the BiCG-eigen restart (one job per slot and side):
//   new slot k = sum_{i<m} scale_i coef[i][k] old slot i   (k < r)
//   new slot r = old slot m                                  (r_{j-1}, appended next)
// with the coupling dots of the new vectors:
//   V side: H[r][k] = (||r_{j-1}|| / rho_{j-1}) (A^+ phat - conj(beta_{j-2}) s)^H v_k
//   W side: H[k][r] = (1 / ||r_{j-1}||) w_k^H (A p - beta_{j-2} q)
// where q, s are the products of the previous iteration (Algorithm eigBiCG).
//
// Register tiling: a block covers tiles of WG_E * WG_T elements; each of the
// RMAX / WG_K column groups computes WG_K output columns for WG_E elements per
// thread, so one shared-memory coefficient read serves WG_E elements. All
// groups read a tile's inputs before any group overwrites them (one block
// barrier per tile: the product is in place).
constexpr int WG_E = 4, WG_K = 8, WG_T = 64;

template <typename S, int RMAX>
__global__ void __launch_bounds__(WG_T * ((RMAX + WG_K - 1) / WG_K))
    window_gemm_kernel(SlotState* states, const SlotPtrs* ptrs, size_t N) {
    constexpr int G = (RMAX + WG_K - 1) / WG_K;
    const int slot = blockIdx.y >> 1, side = blockIdx.y & 1;
    SlotState& st = states[slot];
    const SlotPtrs& P = ptrs[slot];
    if (st.status != ST_RUNNING || st.restart_r == 0) return;
    using C = cplx<S>;
    const int m = st.m, r = st.restart_r, ldc = 2 * st.nev + 1;
    const int par = st.iter & 1;
    __shared__ C Cs[MAX_M * RMAX];
    const double2* coef = side ? P.coefZ : P.coefY;
    for (int q = threadIdx.x; q < m * RMAX; q += blockDim.x) {
        const int i = q / RMAX, k = q % RMAX;
        double2 v = make_double2(0.0, 0.0);
        if (k < r) {
            double2 sc = side ? P.wscale[i] : make_double2(P.vscale[i], 0.0);
            v = sc * coef[i * ldc + k];
        }
        Cs[q] = cvt<S>(v);
    }
    __syncthreads();
    const int g = threadIdx.x / WG_T, t = threadIdx.x % WG_T, k0 = g * WG_K;
    // coupling vector: V side c = A^+phat - conj(beta) s ; W side a = A p - beta q
    const C bp = cvt<S>(side ? st.beta_prev : conj_(st.beta_prev));
    const void* cur = side ? P.Ap[par] : P.Ahp[par];
    const void* prv = side ? P.Ap[par ^ 1] : P.Ahp[par ^ 1];
    void* base = side ? P.W : P.V;
    C dot[WG_K];
#pragma unroll
    for (int kk = 0; kk < WG_K; ++kk) dot[kk] = mk<S>(S(0), S(0));
    const size_t tile = (size_t)WG_E * WG_T;
    for (size_t e0 = (size_t)blockIdx.x * tile; e0 < N; e0 += (size_t)gridDim.x * tile) {
        const size_t eb = e0 + (size_t)t * WG_E;
        const int ne = eb >= N ? 0 : (int)min((size_t)WG_E, N - eb);
        C out[WG_E][WG_K];
#pragma unroll
        for (int e = 0; e < WG_E; ++e)
#pragma unroll
            for (int kk = 0; kk < WG_K; ++kk) out[e][kk] = mk<S>(S(0), S(0));
        // inputs of slot i+1 are loaded while slot i is multiplied (software pipelining)
        C x[WG_E], xn[WG_E];
        {
            const C* src = reinterpret_cast<const C*>(base) + eb;
#pragma unroll
            for (int e = 0; e < WG_E; ++e) x[e] = e < ne ? src[e] : mk<S>(S(0), S(0));
        }
        for (int i = 0; i < m; ++i) {
            if (i + 1 < m) {
                const C* src = reinterpret_cast<const C*>(slot_field<S>(base, i + 1, N)) + eb;
#pragma unroll
                for (int e = 0; e < WG_E; ++e) xn[e] = e < ne ? src[e] : mk<S>(S(0), S(0));
            }
#pragma unroll
            for (int kk = 0; kk < WG_K; ++kk) {
                const C c = Cs[i * RMAX + k0 + kk];
#pragma unroll
                for (int e = 0; e < WG_E; ++e) out[e][kk] = out[e][kk] + x[e] * c;
            }
#pragma unroll
            for (int e = 0; e < WG_E; ++e) x[e] = xn[e];
        }
        C last[WG_E], cv[WG_E];
        {
            const C* lsrc = reinterpret_cast<const C*>(slot_field<S>(base, m, N)) + eb;
            const C* cs = reinterpret_cast<const C*>(cur) + eb;
            const C* ps = reinterpret_cast<const C*>(prv) + eb;
#pragma unroll
            for (int e = 0; e < WG_E; ++e) {
                last[e] = (g == 0 && e < ne) ? lsrc[e] : mk<S>(S(0), S(0));
                cv[e] = e < ne ? cs[e] - bp * ps[e] : mk<S>(S(0), S(0));
            }
        }
        __syncthreads();   // every group has read this tile's inputs
#pragma unroll
        for (int kk = 0; kk < WG_K; ++kk) {
            const int k = k0 + kk;
            if (k < r) {
                C* dst = reinterpret_cast<C*>(slot_field<S>(base, k, N)) + eb;
#pragma unroll
                for (int e = 0; e < WG_E; ++e)
                    if (e < ne) {
                        dst[e] = out[e][kk];
                        dot[kk] = dot[kk] + (side ? cdot(out[e][kk], cv[e]) : cdot(cv[e], out[e][kk]));
                    }
            }
        }
        if (g == 0) {
            C* dst = reinterpret_cast<C*>(slot_field<S>(base, r, N)) + eb;
#pragma unroll
            for (int e = 0; e < WG_E; ++e)
                if (e < ne) dst[e] = last[e];
        }
    }
    // block sums of the coupling dots: warp shuffles, then one value per thread
    __shared__ double2 wdot[(WG_T * G / 32) * WG_K];
    __shared__ bool am_last;
#pragma unroll
    for (int kk = 0; kk < WG_K; ++kk) {
        double2 d = warp_sum(to_d(dot[kk]));
        if ((threadIdx.x & 31) == 0) wdot[(threadIdx.x >> 5) * WG_K + kk] = d;
    }
    __syncthreads();
    constexpr int WPG = WG_T / 32;   // warps per column group
    double2* pp = P.partials + (size_t)(side ? CNT_GEMM_W : CNT_GEMM_V) * PARTIAL_STRIDE;
    const int q = threadIdx.x;       // output column q = group * WG_K + kk
    if (q < G * WG_K) {
        double2 acc = make_double2(0.0, 0.0);
        for (int w = 0; w < WPG; ++w) acc = acc + wdot[((q / WG_K) * WPG + w) * WG_K + q % WG_K];
        pp[(size_t)blockIdx.x * (G * WG_K) + q] = acc;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned prev = atomicAdd(P.counters + (side ? CNT_GEMM_W : CNT_GEMM_V), 1u);
        am_last = (prev == gridDim.x - 1);
        if (am_last) P.counters[side ? CNT_GEMM_W : CNT_GEMM_V] = 0;
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    if (q < r) {
        // the last block adds the partials in block order (deterministic)
        double2 tot = make_double2(0.0, 0.0);
        for (unsigned b = 0; b < gridDim.x; ++b) tot = tot + __ldcg(pp + (size_t)b * (G * WG_K) + q);
        // the new basis vectors are stored normalised: their window scale is 1
        if (side) {
            P.H[q * m + r] = (1.0 / st.rnorm) * tot;
            P.wscale[q] = make_double2(1.0, 0.0);
        } else {
            P.H[r * m + q] = cdiv(make_double2(st.rnorm, 0.0), st.rho) * tot;
            P.vscale[q] = 1.0;
        }
    }
}

}  // namespace

// FP64 links [mu][9][V] double2 -> double-float float4 (h.re, h.im, l.re, l.im).
__global__ void links_df_kernel(const double2* l64, float4* ldf, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double2 v = l64[i];
        const dfl r = df_split(v.x), m = df_split(v.y);
        ldf[i] = make_float4(r.h, m.h, r.l, m.l);
    }
}

// ------------------------------------------------------------------ launchers
static Geom geom_of(const Geom& g) { return g; }

static long long g_launches = 0;
void count_launches(long long n) { g_launches += n; }
long long launches_so_far() { return g_launches; }
void set_launches(long long n) { g_launches = n; }

cudaError_t launch_apply(const Geom& g, const void* links, double kappa, int precision, const ApplyJob* d_jobs,
                         int njobs, int residual, cudaStream_t st) {
    const int grid = ds_blocks(g.V) * njobs;   // jobs fastest: they share each block's links
    if (precision == 0) {
        if (residual) apply_kernel<double, true><<<grid, DS_THREADS, 0, st>>>(geom_of(g), links, kappa, d_jobs, njobs);
        else apply_kernel<double, false><<<grid, DS_THREADS, 0, st>>>(geom_of(g), links, kappa, d_jobs, njobs);
    } else {
        if (residual) return cudaErrorInvalidValue;
        apply_kernel<float, false><<<grid, DS_THREADS, 0, st>>>(geom_of(g), links, kappa, d_jobs, njobs);
    }
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_residual32(const Geom& g, const void* links32, double kappa, const ApplyJob* d_jobs, int njobs,
                              cudaStream_t st) {
    const int grid = ds_blocks(g.V) * njobs;
    residual32_kernel<<<grid, DS_THREADS, 0, st>>>(g, reinterpret_cast<const float4*>(links32), kappa, d_jobs, njobs);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_pack(const double* aos, void* dev, int V, int k, int precision, cudaStream_t st) {
    int nb = blas_blocks((size_t)V * 12 * k);
    if (precision == 0) pack_kernel<double><<<nb, BL_THREADS, 0, st>>>(reinterpret_cast<const double2*>(aos), dev, V, k);
    else pack_kernel<float><<<nb, BL_THREADS, 0, st>>>(reinterpret_cast<const double2*>(aos), dev, V, k);
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t launch_unpack(const void* dev, double* aos, int V, int k, int precision, cudaStream_t st) {
    int nb = blas_blocks((size_t)V * 12 * k);
    if (precision == 0) unpack_kernel<double><<<nb, BL_THREADS, 0, st>>>(dev, reinterpret_cast<double2*>(aos), V, k);
    else unpack_kernel<float><<<nb, BL_THREADS, 0, st>>>(dev, reinterpret_cast<double2*>(aos), V, k);
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t launch_convert(const void* src, int sp, void* dst, int dp, size_t n, cudaStream_t st) {
    int nb = blas_blocks(n);
    if (sp == 0 && dp == 1) convert_kernel<double, float><<<nb, BL_THREADS, 0, st>>>(src, dst, n);
    else if (sp == 1 && dp == 0) convert_kernel<float, double><<<nb, BL_THREADS, 0, st>>>(src, dst, n);
    else if (sp == 0 && dp == 0) convert_kernel<double, double><<<nb, BL_THREADS, 0, st>>>(src, dst, n);
    else convert_kernel<float, float><<<nb, BL_THREADS, 0, st>>>(src, dst, n);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_multidot(int a, const void* X, int xp, int b, const void* Y, int yp, size_t N, double2* Cm,
                            int ldc, int conj_store, double2* scratch, size_t scratch_elems, cudaStream_t st,
                            int* err, int tensor_cores) {
    if (a <= 0 || b <= 0) return cudaSuccess;
    if (tensor_cores && xp == 1 && yp == 1 && dots_tc_supported(a, X, Y, N) &&
        dots_tc_scratch_doubles(a) <= 2 * scratch_elems)
        return launch_dots_tc(a, X, N * 8, b, Y, N * 8, N, Cm, ldc, conj_store, reinterpret_cast<double*>(scratch),
                              2 * scratch_elems, err, st);
    for (int j0 = 0; j0 < b; j0 += MD_BMAX) {
        const int bb = b - j0 < MD_BMAX ? b - j0 : MD_BMAX;
        const int nby = div_up(a, MD_TI);
        int nbx = blas_blocks(N) / 2;
        if (nbx < 1) nbx = 1;
        while ((size_t)nbx * nby * MD_TI * MD_BMAX > scratch_elems && nbx > 1) nbx /= 2;
        if ((size_t)nbx * nby * MD_TI * MD_BMAX > scratch_elems) return cudaErrorInvalidValue;
        const char* Yj = reinterpret_cast<const char*>(Y) + (size_t)j0 * N * (yp == 0 ? 16 : 8);
        const int grid = nbx * nby;
        if (xp == 1 && yp == 1) multidot_kernel<float, float, float><<<grid, BL_THREADS, 0, st>>>(a, X, bb, Yj, N, scratch, nby);
        else if (xp == 1 && yp == 0) multidot_kernel<float, double, double><<<grid, BL_THREADS, 0, st>>>(a, X, bb, Yj, N, scratch, nby);
        else if (xp == 0 && yp == 1) multidot_kernel<double, float, double><<<grid, BL_THREADS, 0, st>>>(a, X, bb, Yj, N, scratch, nby);
        else multidot_kernel<double, double, double><<<grid, BL_THREADS, 0, st>>>(a, X, bb, Yj, N, scratch, nby);
        count_launches(2);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        double2* Cj = conj_store ? Cm + j0 * ldc : Cm + j0;
        multidot_reduce_kernel<<<div_up((size_t)a * bb, 128), 128, 0, st>>>(a, bb, nbx, scratch, Cj, ldc, conj_store);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_vupdate(int a, const void* X, int xp, const double2* D, int ldd, int b, void* Y, int yp,
                           int overwrite, size_t N, cudaStream_t st, int fp64_arith) {
    if (a > MAX_SMALL) return cudaErrorInvalidValue;
    for (int j0 = 0; j0 < b; j0 += MD_BMAX) {
        const int bb = b - j0 < MD_BMAX ? b - j0 : MD_BMAX;
        char* Yj = reinterpret_cast<char*>(Y) + (size_t)j0 * N * (yp == 0 ? 16 : 8);
        const double2* Dj = D + j0;
        int nb = blas_blocks(N);
        if (xp == 1 && yp == 1) vupdate_kernel<float, float, float><<<nb, BL_THREADS, 0, st>>>(a, X, Dj, ldd, bb, Yj, overwrite, N);
        else if (xp == 1 && yp == 0 && fp64_arith) vupdate_kernel<float, double, double><<<nb, BL_THREADS, 0, st>>>(a, X, Dj, ldd, bb, Yj, overwrite, N);
        else if (xp == 1 && yp == 0) vupdate_kernel<float, double, float><<<nb, BL_THREADS, 0, st>>>(a, X, Dj, ldd, bb, Yj, overwrite, N);
        else if (xp == 0 && yp == 1) vupdate_kernel<double, float, double><<<nb, BL_THREADS, 0, st>>>(a, X, Dj, ldd, bb, Yj, overwrite, N);
        else vupdate_kernel<double, double, double><<<nb, BL_THREADS, 0, st>>>(a, X, Dj, ldd, bb, Yj, overwrite, N);
        count_launches(1);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_norms(int b, const void* Y, int yp, size_t N, double* out, double2* scratch,
                         size_t scratch_elems, cudaStream_t st) {
    if (b <= 0) return cudaSuccess;
    int nb = blas_blocks(N) / 2;
    if (nb < 1) nb = 1;
    while ((size_t)nb * b > scratch_elems && nb > 1) nb /= 2;
    dim3 grid(nb, b);
    if (yp == 0) norms_kernel<double><<<grid, BL_THREADS, 0, st>>>(Y, N, scratch);
    else norms_kernel<float><<<grid, BL_THREADS, 0, st>>>(Y, N, scratch);
    norms_reduce_kernel<<<(b + 63) / 64, 64, 0, st>>>(b, nb, scratch, out);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_links_df(const double2* l64, float4* ldf, size_t n, cudaStream_t st) {
    links_df_kernel<<<1216, 256, 0, st>>>(l64, ldf, n);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_scale_fields(int b, void* Y, int yp, const double2* sc, size_t N, cudaStream_t st) {
    int nb = blas_blocks(N * b);
    if (yp == 0) scale_fields_kernel<double><<<nb, BL_THREADS, 0, st>>>(b, Y, sc, N);
    else scale_fields_kernel<float><<<nb, BL_THREADS, 0, st>>>(b, Y, sc, N);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_bicg_start(const Geom& g, const void* links64, double kappa, int prec, SlotState* states,
                              const SlotPtrs* ptrs, int nslots, size_t N, cudaStream_t s) {
    (void)g; (void)links64; (void)kappa;
    dim3 grid(blas_blocks(N / 2), nslots);
    if (prec == 0) start_kernel<double><<<grid, BL_THREADS, 0, s>>>(states, ptrs, N);
    else start_kernel<float><<<grid, BL_THREADS, 0, s>>>(states, ptrs, N);
    count_launches(1);
    return cudaGetLastError();
}

// SPT: sites per thread (grid-stride), which amortises each block's set-up and
// reduction tail over more sites.
template <typename S, int THREADS, int MINB, bool PAIR, int BZ = 0, int SPT = 1, bool G5 = false, bool TM = false>
static void matvec_launch(const Geom& g, const void* links, double kappa, SlotState* states, const SlotPtrs* ptrs,
                          int nslots, cudaStream_t s) {
    const int njobs = (PAIR || G5) ? nslots : 2 * nslots;
    int nb = div_up((size_t)g.V, (size_t)THREADS * SPT);
    if (nb > PARTIAL_STRIDE / 2) nb = PARTIAL_STRIDE / 2;
    matvec_kernel<S, THREADS, MINB, PAIR, BZ, G5, TM><<<nb * njobs, THREADS, 0, s>>>(g, links, kappa, states, ptrs,
                                                                                    njobs);
}
// The brick shapes need Lx, Ly multiples of 8 and Lz a multiple of BZ.
static bool brick_ok(const Geom& g, int bz) { return g.L[0] % 8 == 0 && g.L[1] % 8 == 0 && g.L[2] % bz == 0; }

template <int JPB, int MINB>
static void matvec_group_launch(const Geom& g, const void* links, double kappa, SlotState* states,
                                const SlotPtrs* ptrs, int nslots, cudaStream_t s) {
    const int njobs = 2 * nslots;
    dim3 grid(GRP_BLOCKS, (njobs + JPB - 1) / JPB);
    matvec_group_kernel<JPB, MINB><<<grid, 32 * JPB, 0, s>>>(g, links, (float)kappa, states, ptrs, nslots);
}

int matvec_variants() { return 30; }
bool matvec_variant_ok(const Geom& g, int v) {
    if (v == STAGED_VARIANT) return staged_variant_ok(g);
    if (v >= 25 && v < 30) return brick_variant_ok(g, v);
    if (v == 13 || v == 14) return brick_ok(g, 4);
    if (v == 15 || v == 23) return brick_ok(g, 2);
    if (v >= 19 && v < 25) return brick_ok(g, 4);
    return v >= 0 && v < 25;
}

cudaError_t launch_bicg_matvec(const Geom& g, const void* links, double kappa, int prec, SlotState* states,
                               const SlotPtrs* ptrs, int nslots, cudaStream_t s, int variant) {
    if (prec != 0 && variant == STAGED_VARIANT) return cudaErrorInvalidValue;   // needs the context's tensor maps
    if (prec != 0 && variant >= 25 && variant < 30)   // 4-D bricks, every slot per block (dslash_brick.cu)
        return launch_matvec_brick(g, links, kappa, states, ptrs, nslots, s, variant);
    if (prec == 0) {
        matvec_launch<double, 128, 1, false>(g, links, kappa, states, ptrs, nslots, s);
    } else {
        switch (variant) {
            case 1: matvec_launch<float, 128, 6, false>(g, links, kappa, states, ptrs, nslots, s); break;
            case 2: matvec_launch<float, 256, 3, false>(g, links, kappa, states, ptrs, nslots, s); break;
            case 3: matvec_launch<float, 128, 1, true>(g, links, kappa, states, ptrs, nslots, s); break;
            case 4: matvec_launch<float, 128, 4, true>(g, links, kappa, states, ptrs, nslots, s); break;
            case 5: matvec_launch<float, 128, 4, false>(g, links, kappa, states, ptrs, nslots, s); break;
            case 6: matvec_launch<float, 128, 5, false>(g, links, kappa, states, ptrs, nslots, s); break;
            case 7: matvec_launch<float, 128, 3, true>(g, links, kappa, states, ptrs, nslots, s); break;
            case 8: matvec_launch<float, 256, 2, true>(g, links, kappa, states, ptrs, nslots, s); break;
            case 9: matvec_launch<float, 64, 8, false>(g, links, kappa, states, ptrs, nslots, s); break;
            case 10: matvec_group_launch<8, 3>(g, links, kappa, states, ptrs, nslots, s); break;
            case 11: matvec_group_launch<8, 2>(g, links, kappa, states, ptrs, nslots, s); break;
            case 12: matvec_group_launch<16, 1>(g, links, kappa, states, ptrs, nslots, s); break;
            case 13: matvec_launch<float, 256, 3, false, 4>(g, links, kappa, states, ptrs, nslots, s); break;
            case 14: matvec_launch<float, 256, 2, true, 4>(g, links, kappa, states, ptrs, nslots, s); break;
            case 15: matvec_launch<float, 128, 4, true, 2>(g, links, kappa, states, ptrs, nslots, s); break;
            case 16: matvec_launch<float, 256, 3, false, 0, 4>(g, links, kappa, states, ptrs, nslots, s); break;
            case 17: matvec_launch<float, 128, 4, true, 0, 4>(g, links, kappa, states, ptrs, nslots, s); break;
            case 18: matvec_launch<float, 256, 2, true, 0, 2>(g, links, kappa, states, ptrs, nslots, s); break;
            // t march over 8 x 8 x BZ bricks (SPT consecutive t-planes per block)
            case 19: matvec_launch<float, 256, 1, true, 4, 8, false, true>(g, links, kappa, states, ptrs, nslots, s); break;
            case 20: matvec_launch<float, 256, 2, true, 4, 4, false, true>(g, links, kappa, states, ptrs, nslots, s); break;
            case 21: matvec_launch<float, 256, 1, false, 4, 8, false, true>(g, links, kappa, states, ptrs, nslots, s); break;
            case 22: matvec_launch<float, 256, 2, false, 4, 8, false, true>(g, links, kappa, states, ptrs, nslots, s); break;
            case 23: matvec_launch<float, 128, 2, true, 2, 8, false, true>(g, links, kappa, states, ptrs, nslots, s); break;
            case 24: matvec_launch<float, 256, 1, true, 4, 16, false, true>(g, links, kappa, states, ptrs, nslots, s); break;
            default: matvec_launch<float, 128, 1, false>(g, links, kappa, states, ptrs, nslots, s); break;
        }
    }
    count_launches(1);
    return cudaGetLastError();
}

// The gamma5 variant's operator (A p only, sigma with phat = gamma5 p): the
// one-operator shapes of the list above (per-site threads, no operator pairing).
bool matvec_g5_variant_ok(const Geom& g, int v) {
    switch (v) {
        case 0: case 1: case 2: case 5: case 6: case 9: case 16: return true;
        case 13: case 21: case 22: return brick_ok(g, 4);
        default: return false;
    }
}

cudaError_t launch_bicg_matvec_g5(const Geom& g, const void* links, double kappa, int prec, SlotState* states,
                                  const SlotPtrs* ptrs, int nslots, cudaStream_t s, int variant) {
    if (prec == 0) {
        matvec_launch<double, 128, 1, false, 0, 1, true>(g, links, kappa, states, ptrs, nslots, s);
    } else {
        switch (variant) {
            case 1: matvec_launch<float, 128, 6, false, 0, 1, true>(g, links, kappa, states, ptrs, nslots, s); break;
            case 2: matvec_launch<float, 256, 3, false, 0, 1, true>(g, links, kappa, states, ptrs, nslots, s); break;
            case 5: matvec_launch<float, 128, 4, false, 0, 1, true>(g, links, kappa, states, ptrs, nslots, s); break;
            case 6: matvec_launch<float, 128, 5, false, 0, 1, true>(g, links, kappa, states, ptrs, nslots, s); break;
            case 9: matvec_launch<float, 64, 8, false, 0, 1, true>(g, links, kappa, states, ptrs, nslots, s); break;
            case 13: matvec_launch<float, 256, 3, false, 4, 1, true>(g, links, kappa, states, ptrs, nslots, s); break;
            case 16: matvec_launch<float, 256, 3, false, 0, 4, true>(g, links, kappa, states, ptrs, nslots, s); break;
            case 21: matvec_launch<float, 256, 1, false, 4, 8, true, true>(g, links, kappa, states, ptrs, nslots, s); break;
            case 22: matvec_launch<float, 256, 2, false, 4, 8, true, true>(g, links, kappa, states, ptrs, nslots, s); break;
            default: matvec_launch<float, 128, 1, false, 0, 1, true>(g, links, kappa, states, ptrs, nslots, s); break;
        }
    }
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_bicg_update(int prec, SlotState* states, const SlotPtrs* ptrs, int nslots, size_t N, cudaStream_t s) {
    dim3 grid(blas_blocks(N / 2), nslots);
    if (prec == 0) update_kernel<double><<<grid, BL_THREADS, 0, s>>>(states, ptrs, N);
    else update_kernel<float><<<grid, BL_THREADS, 0, s>>>(states, ptrs, N);
    count_launches(1);
    return cudaGetLastError();
}

// FP64 true-residual shapes (threads, blocks per SM): FP64 arithmetic runs at a
// small fraction of the FP32 rate, so occupancy (latency hiding for the FP64
// pipe) decides; the library times them at init.
template <int THREADS, int MINB>
static void true_resid_launch(const Geom& g, const void* links64, double kappa, SlotState* states,
                              const SlotPtrs* ptrs, int nslots, int check_only, cudaStream_t s) {
    int nb = div_up((size_t)g.V, THREADS);
    if (nb > PARTIAL_STRIDE / 2) nb = PARTIAL_STRIDE / 2;
    true_resid_kernel<THREADS, MINB><<<dim3(nb, nslots), THREADS, 0, s>>>(g, links64, kappa, states, ptrs, check_only);
}
int true_resid_variants() { return 6; }
static void launch_true_resid(int variant, const Geom& g, const void* links64, const float4* links_df,
                              double kappa, SlotState* states, const SlotPtrs* ptrs, int nslots, int check_only,
                              cudaStream_t s) {
    if ((variant == RU_DF || variant == RU_DF + 1) && !check_only && links_df) {
        int nb = div_up((size_t)g.V, 128);
        if (nb > PARTIAL_STRIDE / 2) nb = PARTIAL_STRIDE / 2;
        if (variant == RU_DF)
            true_resid_df_kernel<128, 4><<<dim3(nb, nslots), 128, 0, s>>>(g, links_df, kappa, states, ptrs);
        else
            true_resid_df_kernel<128, 2><<<dim3(nb, nslots), 128, 0, s>>>(g, links_df, kappa, states, ptrs);
        return;
    }
    switch (variant) {
        case 1: true_resid_launch<128, 3>(g, links64, kappa, states, ptrs, nslots, check_only, s); break;
        case 2: true_resid_launch<128, 4>(g, links64, kappa, states, ptrs, nslots, check_only, s); break;
        case 3: true_resid_launch<64, 6>(g, links64, kappa, states, ptrs, nslots, check_only, s); break;
        default: true_resid_launch<128, 1>(g, links64, kappa, states, ptrs, nslots, check_only, s); break;
    }
}

cudaError_t launch_bicg_ru(const Geom& g, const void* links64, double kappa, int prec, SlotState* states,
                           const SlotPtrs* ptrs, int nslots, size_t N, cudaStream_t s, int ru_variant,
                           const float4* links_df, int eo) {
    dim3 g2(blas_blocks(N / 2), nslots);
    if (prec == 0) fold_ru_kernel<double><<<g2, BL_THREADS, 0, s>>>(states, ptrs, N);
    else fold_ru_kernel<float><<<g2, BL_THREADS, 0, s>>>(states, ptrs, N);
    count_launches(1);
    if (eo) {
        cudaError_t e = launch_eo_true_resid(g, links64, kappa, states, ptrs, nslots, 0, s);
        if (e != cudaSuccess) return e;
    } else {
        launch_true_resid(ru_variant, g, links64, links_df, kappa, states, ptrs, nslots, 0, s);
        count_launches(1);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (prec == 0) replace_kernel<double><<<g2, BL_THREADS, 0, s>>>(states, ptrs, N);
    else replace_kernel<float><<<g2, BL_THREADS, 0, s>>>(states, ptrs, N);
    count_launches(1);
    return cudaGetLastError();
}

template <typename S, int THREADS, int MINB, int PHASE>
static void stab_matvec_launch(const Geom& g, const void* links, double kappa, SlotState* states,
                               const SlotPtrs* ptrs, int nslots, cudaStream_t s) {
    int nb = div_up((size_t)g.V, (size_t)THREADS * 2);
    if (nb > PARTIAL_STRIDE / 2) nb = PARTIAL_STRIDE / 2;
    stab_matvec_kernel<S, THREADS, MINB, PHASE><<<nb * nslots, THREADS, 0, s>>>(g, links, kappa, states, ptrs, nslots);
}

cudaError_t launch_stab_step(const Geom& g, const void* links, double kappa, int prec, SlotState* states,
                             const SlotPtrs* ptrs, int nslots, size_t N, cudaStream_t s) {
    dim3 grid(blas_blocks(N / 2), nslots);
    if (prec == 0) {
        stab_dir_kernel<double><<<grid, BL_THREADS, 0, s>>>(states, ptrs, N);
        stab_matvec_launch<double, 128, 1, 1>(g, links, kappa, states, ptrs, nslots, s);
        stab_s_kernel<double><<<grid, BL_THREADS, 0, s>>>(states, ptrs, N);
        stab_matvec_launch<double, 128, 1, 2>(g, links, kappa, states, ptrs, nslots, s);
        stab_update_kernel<double><<<grid, BL_THREADS, 0, s>>>(states, ptrs, N);
    } else {
        stab_dir_kernel<float><<<grid, BL_THREADS, 0, s>>>(states, ptrs, N);
        stab_matvec_launch<float, 128, 4, 1>(g, links, kappa, states, ptrs, nslots, s);
        stab_s_kernel<float><<<grid, BL_THREADS, 0, s>>>(states, ptrs, N);
        stab_matvec_launch<float, 128, 4, 2>(g, links, kappa, states, ptrs, nslots, s);
        stab_update_kernel<float><<<grid, BL_THREADS, 0, s>>>(states, ptrs, N);
    }
    count_launches(5);
    return cudaGetLastError();
}

cudaError_t launch_stab_scalars(SlotState* states, int nslots, cudaStream_t s) {
    stab_scalars_kernel<<<nslots, 32, 0, s>>>(states);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_bicg_scalars(SlotState* states, const SlotPtrs* ptrs, int nslots, cudaStream_t s) {
    scalars_kernel<<<nslots, 32, 0, s>>>(states, ptrs);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_bicg_direction(int prec, SlotState* states, const SlotPtrs* ptrs, int nslots, size_t N,
                                  cudaStream_t s) {
    dim3 grid(blas_blocks(N / 2), nslots);
    if (prec == 0) direction_kernel<double><<<grid, BL_THREADS, 0, s>>>(states, ptrs, N);
    else direction_kernel<float><<<grid, BL_THREADS, 0, s>>>(states, ptrs, N);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_bicg_finish(const Geom& g, const void* links64, double kappa, int prec, SlotState* states,
                               const SlotPtrs* ptrs, int nslots, size_t N, cudaStream_t s, int ru_variant, int eo) {
    dim3 g2(blas_blocks(N / 2), nslots);
    if (prec == 0) fold_kernel<double><<<g2, BL_THREADS, 0, s>>>(states, ptrs, N);
    else fold_kernel<float><<<g2, BL_THREADS, 0, s>>>(states, ptrs, N);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (eo) return launch_eo_true_resid(g, links64, kappa, states, ptrs, nslots, 1, s);
    launch_true_resid(ru_variant >= RU_DF ? 0 : ru_variant, g, links64, nullptr, kappa, states, ptrs, nslots, 1, s);
    count_launches(1);
    return cudaGetLastError();
}

template <typename S, int RMAX>
static void window_gemm_launch(SlotState* states, const SlotPtrs* ptrs, int nslots, size_t N, cudaStream_t s) {
    constexpr int threads = WG_T * ((RMAX + WG_K - 1) / WG_K);
    int nb = div_up(N, (size_t)WG_E * WG_T);
    if (nb > 2 * 152) nb = 2 * 152;
    if (nb > PARTIAL_STRIDE / RMAX) nb = PARTIAL_STRIDE / RMAX;
    window_gemm_kernel<S, RMAX><<<dim3(nb, 2 * nslots), threads, 0, s>>>(states, ptrs, N);
}

template <typename S>
static cudaError_t window_gemm_dispatch(int rmax_needed, SlotState* states, const SlotPtrs* ptrs, int nslots,
                                        size_t N, cudaStream_t s) {
    if (rmax_needed <= 8) window_gemm_launch<S, 8>(states, ptrs, nslots, N, s);
    else if (rmax_needed <= 16) window_gemm_launch<S, 16>(states, ptrs, nslots, N, s);
    else if (rmax_needed <= 24) window_gemm_launch<S, 24>(states, ptrs, nslots, N, s);
    else if (rmax_needed <= 32) window_gemm_launch<S, 32>(states, ptrs, nslots, N, s);
    else return cudaErrorInvalidValue;
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_window_gemm(int prec, int two_nev, SlotState* states, const SlotPtrs* ptrs, int nslots, size_t N,
                               cudaStream_t s) {
    if (prec == 0) return window_gemm_dispatch<double>(two_nev, states, ptrs, nslots, N, s);
    return window_gemm_dispatch<float>(two_nev, states, ptrs, nslots, N, s);
}

}  // namespace lqcd
