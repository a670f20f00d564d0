// Host side of the library: context, device memory, the solve driver and the
// C ABI declared in include/lqcd.h.
//
// The driver follows Algorithm Incremental eigBiCG (paper Sec. 2): deflate the
// initial guesses against the accumulated eigenspace, solve a batch of
// right-hand sides with BiCG (eigBiCG while the eigenspace is still being
// built), then bi-orthogonalize the new Ritz vectors against the eigenspace
// and grow H = U_l^H A U_r. Every arithmetic step runs in the kernels of
// kernels.cu / eig.cu; the host only launches, polls status words and copies
// small matrices.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <string>
#include <vector>

#include "../../include/lqcd.h"
#include "kernels.cuh"

#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define LQCD_HAVE_NVTX 1
#endif

using namespace lqcd;

namespace {

thread_local std::string g_last_error;

// Named host range for timeline tools (Nsight Systems): the stages of a solve
// (sources in, deflation, iterations, eigenspace growth, solutions out), the
// autotuners and the serving calls. NVTX is inert unless a tool is attached.
struct Range {
    explicit Range(const char* name) {
#ifdef LQCD_HAVE_NVTX
        nvtxRangePushA(name);
#else
        (void)name;
#endif
    }
    ~Range() {
#ifdef LQCD_HAVE_NVTX
        nvtxRangePop();
#endif
    }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

void set_error(const char* what, cudaError_t e) {
    char buf[512];
    snprintf(buf, sizeof(buf), "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
    g_last_error = buf;
}

#define CK(call)                                                      \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) {                                      \
            set_error(#call, e_);                                     \
            return e_ == cudaErrorMemoryAllocation ? LQCD_ERR_OOM     \
                                                   : LQCD_ERR_CUDA;   \
        }                                                             \
    } while (0)

constexpr int CHECK_EVERY = 8;   // iterations per graph launch / status poll
constexpr int TILED = 100;       // dslash_variant value of the plane-streaming kernel
constexpr size_t RITZ_STRIDE = (size_t)2 * MAX_M * MAX_M + MAX_M;   // double2 per slot in ritz_all

}  // namespace

struct lqcd_ctx {
    lqcd_params p{};
    Geom g{};
    int V = 0;
    size_t N = 0;            // complex numbers per field
    int kprec = 0;           // Krylov storage: 0 = FP64, 1 = FP32
    size_t kbytes = 0;       // bytes per Krylov field
    size_t dbytes = 0;       // bytes per FP64 field
    int kmax = 1, m = 0, nev = 0, n_def_max = 0, nslot_win = 0;
    int kbatch = 1;                 // right-hand sides per batched launch (<= kmax; autotuned for k_max = 0)
    bool k_auto = false;
    double k_ms[MAX_SLOTS + 1] = {};   // autotuner: ms of one iteration (operator, updates) per batch size
    cudaStream_t stream = nullptr;
    int device = 0;                 // the CUDA device current at init
    bool own_stream = false;
    std::vector<void*> allocs;

    double2* links64 = nullptr;
    float4* links_df = nullptr;     // double-float links for the reliable-update residual (mixed)
    float4* xdf_all = nullptr;      // per slot: x_hi as double-float pairs (mixed)
    float4* links32 = nullptr;

    SlotState* d_state = nullptr;
    SlotPtrs* d_ptrs = nullptr;
    SlotState* h_state = nullptr;   // pinned mirror
    std::vector<SlotPtrs> h_ptrs;

    char* x_lo_all = nullptr;       // kmax Krylov fields
    double2* x_hi_all = nullptr;    // kmax FP64 fields
    double2* b_all = nullptr;
    double2* rt_all = nullptr;
    char* vw_base = nullptr;        // 2 kmax Krylov fields: [V_0 .. V_{K-1}][W_0 .. W_{K-1}], the
                                    // residual and shadow residual of a slot without a window
    // eigBiCG windows (2 (m+1) Krylov fields each), attached to a slot while it
    // runs windowed: allocated from the context's stream-ordered pool when the
    // memory plan has room (hbm_budget_bytes, or free device memory), freed after
    cudaMemPool_t win_pool = nullptr;
    void* win[MAX_SLOTS] = {};
    size_t win_bytes = 0;           // bytes of one window
    size_t plan_bytes = 0;          // memory plan of everything else (fixed at init)
    int win_attached = 0;
    char* vec_all = nullptr;        // kmax * 6 Krylov fields (p, phat, Ap[2], Ahp[2])
    double2* small_all = nullptr;   // per-slot small matrices
    size_t small_stride = 0;
    double2* partials = nullptr;
    unsigned* counters = nullptr;
    double2* eigwork = nullptr;     // kmax * eig_work_elems()
    double2* ritz_all = nullptr;    // per slot: final Ritz coefficients Yc, Zc (MAX_M^2 each) and values
    int* ritz_n = nullptr;          // per slot: number of final Ritz pairs
    double2* mdscratch = nullptr;
    size_t mdscratch_elems = 0;
    ApplyJob* d_jobs = nullptr;
    double2* staging = nullptr;     // kmax FP64 full fields (host AoS I/O)
    // even-odd (Schur complement) operator: the solver works on the odd half
    // lattice (N = 6 V); sources and solutions stay full fields (Nfull = 12 V)
    bool eo = false;
    size_t Nfull = 0;
    double2* bfull_all = nullptr;   // kmax full FP64 sources
    double2* xfull_all = nullptr;   // kmax full FP64 solutions (and initial guesses)
    double2* eo64_all = nullptr;    // kmax FP64 half fields: stage buffer of the Schur residual
    char* eot_all = nullptr;        // 2 kmax Krylov half fields: stage buffers of the operator pair
    double* bnorm_all = nullptr;    // kmax ||b|| of the full systems
    char* eo_scr = nullptr;         // 2 kmax FP64 half fields: stage buffers of host applies
    EoJob* d_eojobs = nullptr;      // 2 x 2 kmax stage jobs

    // eigenspace
    int n_def = 0;
    int eig_rhs_done = 0;
    char* Ur = nullptr;
    char* Ul = nullptr;
    double2* Hdef = nullptr;        // n_def_max^2, ld n_def_max
    double2* Mdef = nullptr;
    double2* Hlu = nullptr;
    double2* Mlu = nullptr;
    int* Hpiv = nullptr;
    int* Mpiv = nullptr;
    double2* dsmall = nullptr;      // scratch for small matrices (n_def_max * 16 * ...)
    int* dinfo = nullptr;
    double2* dconst = nullptr;      // constants

    int dslash_variant = 0;         // operator-kernel shape (autotuned at init); TILED = plane streaming
    int use_tc = 1;                 // FP32 projections and restart products on the tensor cores
    int ru_variant = 0;             // FP64 true-residual kernel shape (timed at init)
    TileGeom tgeo[MAX_SLOTS + 1] = {};
    bool tile_ok[MAX_SLOTS + 1] = {};
    long long deflations_discarded = 0;   // oblique projections undone (deflate_range)
    bool staged_ok = false;         // shape 26: tensor maps of the Krylov fields and links encoded
    int nsm = 0;                    // SMs of the device (grid of the staged operator kernel)
    alignas(64) unsigned char staged_maps[2048] = {};
    int* d_err = nullptr;           // device error word of the bounded waits
    std::vector<double> tune_ms;    // autotuner timings per variant

    // CUDA graphs of CHECK_EVERY iterations, keyed by (nslots, kernel groups CH_*)
    cudaGraphExec_t graphs[MAX_SLOTS + 1][8] = {};
    long long graph_nodes[MAX_SLOTS + 1][8] = {};

    // serving session (lqcd_submit / lqcd_progress / lqcd_poll): requests wait in
    // a queue, take a batch slot as soon as one is free, and leave it when done
    struct Request {
        long long ticket = 0;
        const double* b = nullptr;
        double* x = nullptr;
        int on_device = 0;
        lqcd_mode mode = LQCD_MODE_AUTO;
    };
    struct SlotJob {
        bool busy = false;
        Request req;
        lqcd_mode md = LQCD_MODE_PLAIN;
        bool windowed = false;
        bool deftol_pending = false;   // first leg of the DefTol restart still running
        bool correction_pending = false;   // mixed eigBiCG: the window leg is still running
        int first_iters = 0, first_matvecs = 0, first_ru = 0, first_restarts = 0, outer = 0;
        std::chrono::steady_clock::time_point t0;
    };
    struct Finished {
        lqcd_solve_info info;
        lqcd_status status;
    };
    std::deque<Request> queue;
    SlotJob jobs[MAX_SLOTS];
    std::map<long long, Finished> finished;
    long long next_ticket = 1;
    int eig_inflight = 0;
    bool chunk_inflight = false;
    cudaEvent_t chunk_ev = nullptr;    // recorded after each session chunk
    bool session_busy() const {
        if (!queue.empty() || chunk_inflight) return true;
        for (int s = 0; s < kmax; ++s)
            if (jobs[s].busy) return true;
        return false;
    }

    // last eigBiCG window info (per slot): final Ritz values
    std::vector<std::vector<double2>> last_ritz;
    std::vector<int> last_vs, last_restarts;
    int last_window_valid = 0;

    // Host-side fault injection (LQCD_FAULT=alloc:N in the environment at init):
    // the N-th device allocation of the context reports cudaErrorMemoryAllocation
    // without allocating, to exercise the clean-up paths. Nothing runs on the GPU.
    int fault_alloc = -1, n_alloc = 0;

    template <typename T> cudaError_t alloc(T** p, size_t bytes) {
        void* q = nullptr;
        if (++n_alloc == fault_alloc) return cudaErrorMemoryAllocation;
        cudaError_t e = cudaMalloc(&q, bytes < 16 ? 16 : bytes);
        if (e != cudaSuccess) return e;
        allocs.push_back(q);
        *p = reinterpret_cast<T*>(q);
        return cudaSuccess;
    }
    void* krylov(char* base, size_t i) const { return base + i * kbytes; }
};

namespace {

size_t small_stride_elems(int m, int nev) {
    // H (m*m), wscale (m+1), coefY, coefZ ((m+1)*(2nev+1)), lam (2nev+2), vscale ((m+1) doubles -> as double2), ritz (nev)
    return (size_t)m * m + (m + 1) + 2 * (size_t)(m + 1) * (2 * nev + 1) + (2 * nev + 2) + (m + 1) + nev + 16;
}

lqcd_status validate(const lqcd_params* p) {
    if (!p) return LQCD_ERR_ARG;
    for (int d = 0; d < 4; ++d)
        if (p->dims[d] < 2 || p->dims[d] > 4096) return LQCD_ERR_ARG;
    double V = (double)p->dims[0] * p->dims[1] * p->dims[2] * p->dims[3];
    if (V * 12.0 > 2.0e9) return LQCD_ERR_ARG;
    if (!(p->kappa >= 0.0) || !std::isfinite(p->kappa)) return LQCD_ERR_ARG;
    if (p->nev < 1 || p->m <= 2 * p->nev || p->m > MAX_M || 2 * p->nev > 32) return LQCD_ERR_ARG;
    if (!(p->tol > 0.0) || p->maxiter < 1) return LQCD_ERR_ARG;
    if (p->precision != LQCD_FP64 && p->precision != LQCD_MIXED) return LQCD_ERR_ARG;
    if (p->k_max < 0 || p->k_max > MAX_SLOTS) return LQCD_ERR_ARG;
    if (p->n_def_max < 0 || p->n_def_max > MAX_SMALL) return LQCD_ERR_ARG;
    if (p->n1 < 0 || p->deftol < 0.0 || p->delta < 0.0 || p->delta >= 1.0) return LQCD_ERR_ARG;
    if (p->gamma5 != 0 && p->gamma5 != 1) return LQCD_ERR_ARG;
    if (p->bicgstab != 0 && p->bicgstab != 1) return LQCD_ERR_ARG;
    if (p->bicgstab && p->gamma5) return LQCD_ERR_ARG;   // the gamma5 variant is a BiCG recursion
    if (p->evenodd != 0 && p->evenodd != 1) return LQCD_ERR_ARG;
    if (p->evenodd) {   // parities need even extents; the variants keep the full operator
        for (int d = 0; d < 4; ++d)
            if (p->dims[d] % 2) return LQCD_ERR_ARG;
        if (p->gamma5 || p->bicgstab) return LQCD_ERR_ARG;
    }
    return LQCD_OK;
}

lqcd_status set_ptrs(lqcd_ctx* c) {
    c->h_ptrs.resize(c->kmax);
    for (int s = 0; s < c->kmax; ++s) {
        SlotPtrs& P = c->h_ptrs[s];
        P.x_lo = c->krylov(c->x_lo_all, s);
        P.x_hi = c->x_hi_all + (size_t)s * c->N;
        P.b = c->b_all + (size_t)s * c->N;
        P.r_true = c->rt_all + (size_t)s * c->N;
        P.x_df = c->xdf_all ? c->xdf_all + (size_t)s * c->N : nullptr;
        P.V = c->win[s] ? c->win[s] : c->krylov(c->vw_base, s);
        P.W = c->win[s] ? reinterpret_cast<char*>(c->win[s]) + (size_t)(c->m + 1) * c->kbytes
                        : c->krylov(c->vw_base, (size_t)c->kmax + s);
        char* vb = c->vec_all + (size_t)s * 6 * c->kbytes;
        P.p = vb;
        P.phat = vb + c->kbytes;
        P.Ap[0] = vb + 2 * c->kbytes;
        P.Ap[1] = vb + 3 * c->kbytes;
        P.Ahp[0] = vb + 4 * c->kbytes;
        P.Ahp[1] = vb + 5 * c->kbytes;
        double2* sm = c->small_all + (size_t)s * c->small_stride;
        const int m = c->m, nev = c->nev;
        P.H = sm; sm += (size_t)m * m;
        P.wscale = sm; sm += m + 1;
        P.coefY = sm; sm += (size_t)(m + 1) * (2 * nev + 1);
        P.coefZ = sm; sm += (size_t)(m + 1) * (2 * nev + 1);
        P.lam = sm; sm += 2 * nev + 2;
        P.vscale = reinterpret_cast<double*>(sm); sm += m + 1;
        P.partials = c->partials + (size_t)s * CNT_COUNT * PARTIAL_STRIDE;
        P.counters = c->counters + (size_t)s * CNT_COUNT;
        P.eo_t = c->eo ? c->krylov(c->eot_all, 2 * (size_t)s) : nullptr;
        P.eo_th = c->eo ? c->krylov(c->eot_all, 2 * (size_t)s + 1) : nullptr;
        P.eo64 = c->eo ? c->eo64_all + (size_t)s * c->N : nullptr;
        P.bnorm_ref = c->eo ? c->bnorm_all + s : nullptr;
    }
    CK(cudaMemcpy(c->d_ptrs, c->h_ptrs.data(), sizeof(SlotPtrs) * c->kmax, cudaMemcpyHostToDevice));
    return LQCD_OK;
}

// A caller's buffer matches on_device: device (or managed) memory of the
// context's GPU for on_device = 1, host memory (pageable, pinned or managed) for
// on_device = 0. A host buffer passed as device memory would be read by the
// kernels, a device buffer passed as host memory by a host copy: both refused.
bool user_buffer_ok(const lqcd_ctx* c, const void* p, int on_device) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return !on_device;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    if (on_device) return a.type == cudaMemoryTypeDevice && a.device == c->device;
    return a.type != cudaMemoryTypeDevice;
}

lqcd_status check_buffers(const lqcd_ctx* c, const void* a, const void* b, int on_device, const char* where) {
    if (user_buffer_ok(c, a, on_device) && user_buffer_ok(c, b, on_device)) return LQCD_OK;
    g_last_error = std::string(where) + (on_device ? ": a buffer is not device memory of the context's GPU"
                                                   : ": a buffer is device memory but on_device = 0");
    return LQCD_ERR_ARG;
}

// Point slot s's V and W at its window (attached) or at its base fields.
lqcd_status upload_ptrs(lqcd_ctx* c, int s) {
    SlotPtrs& P = c->h_ptrs[s];
    P.V = c->win[s] ? c->win[s] : c->krylov(c->vw_base, s);
    P.W = c->win[s] ? reinterpret_cast<char*>(c->win[s]) + (size_t)(c->m + 1) * c->kbytes
                    : c->krylov(c->vw_base, (size_t)c->kmax + s);
    CK(cudaMemcpyAsync(c->d_ptrs + s, &P, sizeof(SlotPtrs), cudaMemcpyHostToDevice, c->stream));
    return LQCD_OK;
}

constexpr size_t WIN_RESERVE = (size_t)1 << 30;   // device memory left free when there is no budget

// Admission by device memory: give slot s an eigBiCG window if the memory plan has
// room for one more (hbm_budget_bytes, else the free device memory less a reserve).
// *ok = false (and LQCD_OK) when it does not fit now.
lqcd_status attach_window(lqcd_ctx* c, int s, bool* ok) {
    *ok = false;
    if (c->win[s]) { *ok = true; return LQCD_OK; }
    if (c->p.hbm_budget_bytes) {
        if (c->plan_bytes + (size_t)(c->win_attached + 1) * c->win_bytes > c->p.hbm_budget_bytes) return LQCD_OK;
    } else {
        // free device memory, plus what this context's pool keeps mapped but unused
        size_t fr = 0, tot = 0;
        CK(cudaMemGetInfo(&fr, &tot));
        uint64_t reserved = 0, used = 0;
        CK(cudaMemPoolGetAttribute(c->win_pool, cudaMemPoolAttrReservedMemCurrent, &reserved));
        CK(cudaMemPoolGetAttribute(c->win_pool, cudaMemPoolAttrUsedMemCurrent, &used));
        if (fr + (reserved > used ? reserved - used : 0) < c->win_bytes + WIN_RESERVE) return LQCD_OK;
    }
    void* p = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(&p, c->win_bytes, c->win_pool, c->stream);
    if (e == cudaErrorMemoryAllocation) {
        (void)cudaGetLastError();
        return LQCD_OK;
    }
    CK(e);
    CK(cudaMemsetAsync(p, 0, c->win_bytes, c->stream));
    c->win[s] = p;
    c->win_attached += 1;
    *ok = true;
    return upload_ptrs(c, s);
}

lqcd_status detach_window(lqcd_ctx* c, int s) {
    if (!c->win[s]) return LQCD_OK;
    void* p = c->win[s];
    c->win[s] = nullptr;
    c->win_attached -= 1;
    lqcd_status r = upload_ptrs(c, s);
    if (r != LQCD_OK) return r;
    CK(cudaFreeAsync(p, c->stream));
    return LQCD_OK;
}

// Links: host [4][V][3][3] complex128 -> FP64 [mu][9][V] and FP32 two-row [mu][3][V].
__global__ void links_kernel(const double2* host_layout, double2* l64, float4* l32, int V) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < 4 * V; q += gridDim.x * blockDim.x) {
        const int mu = q / V, s = q % V;
        const double2* u = host_layout + (size_t)q * 9;
        for (int e = 0; e < 9; ++e) l64[(size_t)(mu * 9 + e) * V + s] = u[e];
        if (l32) {
            l32[(size_t)(mu * 3 + 0) * V + s] = make_float4((float)u[0].x, (float)u[0].y, (float)u[1].x, (float)u[1].y);
            l32[(size_t)(mu * 3 + 1) * V + s] = make_float4((float)u[2].x, (float)u[2].y, (float)u[3].x, (float)u[3].y);
            l32[(size_t)(mu * 3 + 2) * V + s] = make_float4((float)u[4].x, (float)u[4].y, (float)u[5].x, (float)u[5].y);
        }
    }
}

__global__ void negate_kernel(double2* a, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a[i] = -a[i];
}
__global__ void copy_block_kernel(const double2* src, int lds, double2* dst, int ldd, int rows, int cols) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < rows * cols; q += gridDim.x * blockDim.x) {
        const int i = q / cols, j = q % cols;
        dst[(size_t)i * ldd + j] = src[(size_t)i * lds + j];
    }
}
// sc[j] = 1/sqrt(diag(G)[j]) for G (n x n, ld), and nrm[j] = sqrt(diag)
__global__ void inv_norm_kernel(const double2* G, int ld, int n, double2* sc, double* nrm) {
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double d = sqrt(fmax(G[(size_t)j * ld + j].x, 0.0));
        nrm[j] = d;
        sc[j] = make_double2(d > 0.0 ? 1.0 / d : 0.0, 0.0);
    }
}

}  // namespace

static lqcd_status autotune(lqcd_ctx* c);
static lqcd_status autotune_batch(lqcd_ctx* c);

// ============================================================== lifecycle
extern "C" lqcd_status lqcd_eigbicg_init(lqcd_ctx** out, const lqcd_params* params, const double* links,
                                         void* cuda_stream) {
    Range nvtx_("lqcd_eigbicg_init");
    if (!out || !links) return LQCD_ERR_ARG;
    *out = nullptr;
    lqcd_status vs = validate(params);
    if (vs != LQCD_OK) return vs;
    lqcd_ctx* c = new lqcd_ctx();
    c->p = *params;
    c->k_auto = params->k_max == 0;
    if (const char* f = getenv("LQCD_FAULT")) {
        int n = 0;
        if (sscanf(f, "alloc:%d", &n) == 1 && n > 0) c->fault_alloc = n;
    }
    if (c->p.k_max == 0) c->p.k_max = MAX_SLOTS;
    if (c->p.delta == 0.0) c->p.delta = 0.01;
    c->kmax = c->p.k_max;
    c->m = c->p.m;
    c->nev = c->p.nev;
    c->n_def_max = c->p.n_def_max ? c->p.n_def_max : std::min(MAX_SMALL, std::max(c->p.n1, 1) * c->nev);
    for (int d = 0; d < 4; ++d) c->g.L[d] = c->p.dims[d];
    c->g.stride[0] = 1;
    for (int d = 1; d < 4; ++d) c->g.stride[d] = c->g.stride[d - 1] * c->g.L[d - 1];
    c->V = c->g.stride[3] * c->g.L[3];
    c->g.V = c->V;
    c->eo = c->p.evenodd != 0;
    c->Nfull = (size_t)12 * c->V;
    c->N = c->eo ? c->Nfull / 2 : c->Nfull;
    c->kprec = c->p.precision == LQCD_MIXED ? 1 : 0;
    c->kbytes = c->N * (c->kprec ? 8 : 16);
    c->dbytes = c->N * 16;
    c->small_stride = small_stride_elems(c->m, c->nev);
    c->mdscratch_elems = (size_t)((MAX_SMALL + 3) / 4) * 1216 * 32;

    // Memory plan (bytes) for the HBM budget check.
    const size_t K = (size_t)c->kmax;
    size_t plan = (size_t)c->V * 4 * 9 * 16 + (c->kprec ? (size_t)c->V * 4 * (3 + 9) * 16 + K * c->N * 16 : 0);
    plan += K * c->kbytes * (1 + 2 + 6) + K * c->dbytes * 3 + K * c->Nfull * 16;
    if (c->eo) plan += K * c->Nfull * 16 * 2 + K * c->dbytes * 3 + 2 * K * c->kbytes;
    plan += 2 * (size_t)c->n_def_max * c->kbytes;
    plan += (MAX_SLOTS * eig_work_elems() + 16) * 16 + c->mdscratch_elems * 16 + K * CNT_COUNT * PARTIAL_STRIDE * 16;
    plan += MAX_SLOTS * RITZ_STRIDE * 16 + MAX_SLOTS * sizeof(int);
    c->plan_bytes = plan;
    c->win_bytes = (size_t)2 * (c->m + 1) * c->kbytes;
    if (c->p.hbm_budget_bytes && plan > c->p.hbm_budget_bytes) {
        g_last_error = "memory plan exceeds hbm_budget_bytes";
        delete c;
        return LQCD_ERR_OOM;
    }

    auto fail = [&](lqcd_status s) { lqcd_destroy(c); return s; };
    cudaError_t e;
#define AL(ptr, bytes)                                                                   \
    do {                                                                                 \
        e = c->alloc(&(ptr), (bytes));                                                   \
        if (e != cudaSuccess) { set_error("cudaMalloc " #ptr, e); return fail(e == cudaErrorMemoryAllocation ? LQCD_ERR_OOM : LQCD_ERR_CUDA); } \
    } while (0)

    e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) { set_error("cudaGetDevice", e); delete c; return LQCD_ERR_CUDA; }
    if (cuda_stream) {
        c->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { set_error("cudaStreamCreate", e); delete c; return LQCD_ERR_CUDA; }
        c->own_stream = true;
    }
    AL(c->links64, (size_t)c->V * 4 * 9 * 16);
    if (c->kprec) AL(c->links32, (size_t)c->V * 4 * 3 * 16);
    if (c->kprec) AL(c->links_df, (size_t)c->V * 4 * 9 * 16);
    if (c->kprec) AL(c->xdf_all, K * c->N * 16);
    AL(c->d_state, sizeof(SlotState) * K);
    AL(c->d_ptrs, sizeof(SlotPtrs) * K);
    e = cudaMallocHost(&c->h_state, sizeof(SlotState) * K);
    if (e != cudaSuccess) { set_error("cudaMallocHost", e); return fail(LQCD_ERR_OOM); }
    AL(c->x_lo_all, K * c->kbytes);
    AL(c->x_hi_all, K * c->dbytes);
    AL(c->b_all, K * c->dbytes);
    AL(c->rt_all, K * c->dbytes);
    AL(c->vw_base, K * 2 * c->kbytes);
    AL(c->vec_all, K * 6 * c->kbytes);
    AL(c->small_all, K * c->small_stride * 16);
    AL(c->partials, K * CNT_COUNT * PARTIAL_STRIDE * 16);
    AL(c->counters, K * CNT_COUNT * sizeof(unsigned));
    AL(c->eigwork, ((size_t)MAX_SLOTS * eig_work_elems() + 16) * 16);
    AL(c->ritz_all, (size_t)MAX_SLOTS * RITZ_STRIDE * 16);
    AL(c->ritz_n, MAX_SLOTS * sizeof(int));
    AL(c->mdscratch, c->mdscratch_elems * 16);
    AL(c->d_jobs, sizeof(ApplyJob) * 2 * K);
    AL(c->staging, K * c->Nfull * 16);
    if (c->eo) {
        AL(c->bfull_all, K * c->Nfull * 16);
        AL(c->xfull_all, K * c->Nfull * 16);
        AL(c->eo64_all, K * c->dbytes);
        AL(c->eot_all, 2 * K * c->kbytes);
        AL(c->bnorm_all, K * sizeof(double));
        AL(c->eo_scr, 2 * K * c->dbytes);
        AL(c->d_eojobs, 4 * K * sizeof(EoJob));
    }
    AL(c->Ur, (size_t)std::max(c->n_def_max, 1) * c->kbytes);
    AL(c->Ul, (size_t)std::max(c->n_def_max, 1) * c->kbytes);
    const size_t nd2 = (size_t)c->n_def_max * c->n_def_max + 16;
    AL(c->Hdef, nd2 * 16);
    AL(c->Mdef, nd2 * 16);
    AL(c->Hlu, nd2 * 16);
    AL(c->Mlu, nd2 * 16);
    AL(c->Hpiv, (size_t)(c->n_def_max + 1) * sizeof(int));
    AL(c->Mpiv, (size_t)(c->n_def_max + 1) * sizeof(int));
    AL(c->dsmall, (size_t)(MAX_SMALL * MAX_SMALL * 6 + 4096) * 16);
    AL(c->dinfo, (64 + MAX_SMALL) * sizeof(int));
    AL(c->dconst, 64 * 16);
    AL(c->d_err, 16);
#undef AL
    if ((e = cudaMemset(c->counters, 0, K * CNT_COUNT * sizeof(unsigned))) != cudaSuccess ||
        (e = cudaMemset(c->small_all, 0, K * c->small_stride * 16)) != cudaSuccess ||
        (e = cudaMemset(c->vw_base, 0, K * 2 * c->kbytes)) != cudaSuccess ||
        (e = cudaMemset(c->vec_all, 0, K * 6 * c->kbytes)) != cudaSuccess ||
        (e = cudaMemset(c->x_lo_all, 0, K * c->kbytes)) != cudaSuccess ||
        (e = cudaMemset(c->d_err, 0, 16)) != cudaSuccess) {
        set_error("cudaMemset", e);
        return fail(LQCD_ERR_CUDA);
    }
    for (int s = 0; s < c->kmax; ++s) {
        memset(&c->h_state[s], 0, sizeof(SlotState));
        c->h_state[s].status = ST_IDLE;
    }
    if ((e = cudaMemcpy(c->d_state, c->h_state, sizeof(SlotState) * K, cudaMemcpyHostToDevice)) != cudaSuccess) {
        set_error("cudaMemcpy state", e);
        return fail(LQCD_ERR_CUDA);
    }
    {
        int dev = 0;
        cudaMemPoolProps pp;
        memset(&pp, 0, sizeof(pp));
        pp.allocType = cudaMemAllocationTypePinned;
        pp.location.type = cudaMemLocationTypeDevice;
        if ((e = cudaGetDevice(&dev)) == cudaSuccess) {
            pp.location.id = dev;
            e = cudaMemPoolCreate(&c->win_pool, &pp);
        }
        if (e != cudaSuccess) { set_error("cudaMemPoolCreate", e); c->win_pool = nullptr; return fail(LQCD_ERR_CUDA); }
        // keep up to kmax released windows mapped in the pool (a job re-acquires them
        // at every eigBiCG batch; unmapping and mapping 10 GB windows costs ~0.1 s)
        uint64_t keep = (uint64_t)K * c->win_bytes;
        if ((e = cudaMemPoolSetAttribute(c->win_pool, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess) {
            set_error("cudaMemPoolSetAttribute", e);
            return fail(LQCD_ERR_CUDA);
        }
    }
    lqcd_status st = set_ptrs(c);
    if (st != LQCD_OK) return fail(st);
    // links: host -> staging (reuse rt_all as FP64 scratch of >= 4*V*9 complex? use a temp)
    double2* tmp = nullptr;
    if ((e = cudaMalloc(&tmp, (size_t)c->V * 4 * 9 * 16)) != cudaSuccess) { set_error("cudaMalloc links tmp", e); return fail(LQCD_ERR_OOM); }
    e = cudaMemcpy(tmp, links, (size_t)c->V * 4 * 9 * 16, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        links_kernel<<<1216, 256, 0, c->stream>>>(tmp, c->links64, c->links32, c->V);
        count_launches(1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && c->links_df) e = launch_links_df(c->links64, c->links_df, (size_t)c->V * 4 * 9, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) { set_error("links upload", e); return fail(LQCD_ERR_CUDA); }
    c->last_ritz.assign(c->kmax, {});
    c->last_vs.assign(c->kmax, 0);
    c->last_restarts.assign(c->kmax, 0);
    if ((e = prepare_eig_kernels()) != cudaSuccess) { set_error("prepare_eig_kernels", e); return fail(LQCD_ERR_CUDA); }
    if ((e = prepare_tiled_kernel()) != cudaSuccess) { set_error("prepare_tiled_kernel", e); return fail(LQCD_ERR_CUDA); }
    for (int n = 1; n <= c->kmax; ++n)
        c->tile_ok[n] = c->kprec && !c->p.gamma5 && !c->eo && tiled_plan(c->g, n, &c->tgeo[n]);
    if (c->kprec && !c->p.gamma5 && !c->eo && staged_variant_ok(c->g) && staged_maps_bytes() <= sizeof(c->staged_maps)) {
        int dev = 0;
        if ((e = cudaGetDevice(&dev)) == cudaSuccess)
            e = cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = prepare_staged(c->g, c->vec_all, c->kmax, c->links32, c->staged_maps);
        // a lattice or device the tensor maps cannot describe keeps the other shapes
        c->staged_ok = e == cudaSuccess;
        if (e == cudaErrorInvalidValue) { cudaGetLastError(); e = cudaSuccess; }
        if (e != cudaSuccess) { set_error("prepare_staged", e); return fail(LQCD_ERR_CUDA); }
    }
    st = c->p.no_autotune ? LQCD_OK : autotune(c);
    if (st != LQCD_OK) return fail(st);
    c->kbatch = c->kmax;
    if (c->k_auto && !c->p.no_autotune) {
        st = autotune_batch(c);
        if (st != LQCD_OK) return fail(st);
    }
    *out = c;
    return LQCD_OK;
}

extern "C" void lqcd_destroy(lqcd_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (int i = 0; i <= MAX_SLOTS; ++i)
        for (int j = 0; j < 8; ++j)
            if (c->graphs[i][j]) cudaGraphExecDestroy(c->graphs[i][j]);
    for (int s = 0; s < MAX_SLOTS; ++s)
        if (c->win[s]) cudaFreeAsync(c->win[s], c->stream);
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->win_pool) cudaMemPoolDestroy(c->win_pool);
    for (void* p : c->allocs) cudaFree(p);
    if (c->h_state) cudaFreeHost(c->h_state);
    if (c->chunk_ev) cudaEventDestroy(c->chunk_ev);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

extern "C" const char* lqcd_status_str(lqcd_status s) {
    switch (s) {
        case LQCD_OK: return "ok";
        case LQCD_ERR_ARG: return "invalid argument";
        case LQCD_ERR_OOM: return "out of device memory";
        case LQCD_ERR_CUDA: return "CUDA error";
        case LQCD_ERR_NOCONV: return "no convergence within maxiter";
        case LQCD_ERR_BREAKDOWN: return "BiCG breakdown";
        case LQCD_ERR_TIMEOUT: return "device wait timed out";
        case LQCD_ERR_STATE: return "invalid state";
    }
    return "unknown status";
}

extern "C" const char* lqcd_last_error(void) { return g_last_error.c_str(); }

extern "C" int lqcd_eigspace_size(const lqcd_ctx* c) { return c ? c->n_def : 0; }

// ============================================================ field I/O
namespace {

// Copy k fields from user memory (host or device, AoS FP64) into device fields
// of precision prec (0 FP64, 1 FP32), via the staging buffer for host input.
// nc: complex numbers per field (0 = the solver's field length c->N; Nfull for
// the full sources and solutions of an even-odd context).
lqcd_status upload(lqcd_ctx* c, const double* src, int k, void* dst, int prec, int on_device, size_t nc = 0) {
    if (!nc) nc = c->N;
    for (int j0 = 0; j0 < k; j0 += c->kmax) {
        const int kb = std::min(c->kmax, k - j0);
        const double* s = src + (size_t)j0 * 2 * nc;
        const double* dev_src = s;
        if (!on_device) {
            CK(cudaMemcpyAsync(c->staging, s, (size_t)kb * nc * 16, cudaMemcpyHostToDevice, c->stream));
            dev_src = reinterpret_cast<const double*>(c->staging);
        }
        char* d = reinterpret_cast<char*>(dst) + (size_t)j0 * nc * (prec ? 8 : 16);
        CK(launch_pack(dev_src, d, (int)(nc / 12), kb, prec, c->stream));
    }
    return LQCD_OK;
}

lqcd_status download(lqcd_ctx* c, const void* src, int prec, int k, double* dst, int on_device, size_t nc = 0) {
    if (!nc) nc = c->N;
    for (int j0 = 0; j0 < k; j0 += c->kmax) {
        const int kb = std::min(c->kmax, k - j0);
        const char* s = reinterpret_cast<const char*>(src) + (size_t)j0 * nc * (prec ? 8 : 16);
        double* d = dst + (size_t)j0 * 2 * nc;
        if (on_device) {
            CK(launch_unpack(s, d, (int)(nc / 12), kb, prec, c->stream));
        } else {
            CK(launch_unpack(s, reinterpret_cast<double*>(c->staging), (int)(nc / 12), kb, prec, c->stream));
            CK(cudaMemcpyAsync(d, c->staging, (size_t)kb * nc * 16, cudaMemcpyDeviceToHost, c->stream));
        }
    }
    return LQCD_OK;
}

// out_j = A in_j (or A^+, or b_j - A in_j) for nf device fields in precision prec:
// the solver's operator (A_hat on the odd half lattice in an even-odd context),
// or with full = true the full-lattice A (fields of Nfull complex).
lqcd_status apply_fields(lqcd_ctx* c, int prec, int dagger, int nf, const void* in, size_t in_stride, void* out,
                         size_t out_stride, const double2* aux, bool full = false) {
    const void* links = prec ? (const void*)c->links32 : (const void*)c->links64;
    if (prec && !c->links32) return LQCD_ERR_ARG;
    if (c->eo && !full) {   // two stages through the half-field scratch
        std::vector<EoJob> st1(2 * c->kmax), st2(2 * c->kmax);
        const size_t sb = c->N * (prec ? 8 : 16);
        for (int j0 = 0; j0 < nf; j0 += 2 * c->kmax) {
            const int nb = std::min(2 * c->kmax, nf - j0);
            for (int j = 0; j < nb; ++j) {
                const char* fin = reinterpret_cast<const char*>(in) + (j0 + j) * in_stride;
                char* scr = c->eo_scr + (size_t)j * sb;
                st1[j] = EoJob{fin, nullptr, scr, nullptr, dagger};
                st2[j] = EoJob{scr, fin, reinterpret_cast<char*>(out) + (j0 + j) * out_stride,
                               aux ? aux + (size_t)(j0 + j) * c->N : nullptr, dagger};
            }
            CK(cudaMemcpyAsync(c->d_eojobs, st1.data(), sizeof(EoJob) * nb, cudaMemcpyHostToDevice, c->stream));
            CK(cudaMemcpyAsync(c->d_eojobs + 2 * c->kmax, st2.data(), sizeof(EoJob) * nb, cudaMemcpyHostToDevice,
                               c->stream));
            CK(launch_eo_apply(c->g, links, c->p.kappa, prec, c->d_eojobs, c->d_eojobs + 2 * c->kmax, nb,
                               aux != nullptr, c->stream));
            CK(cudaStreamSynchronize(c->stream));   // the job tables are reused
        }
        return LQCD_OK;
    }
    const size_t an = full ? c->Nfull : c->N;
    std::vector<ApplyJob> jobs(2 * c->kmax);
    for (int j0 = 0; j0 < nf; j0 += 2 * c->kmax) {
        const int nb = std::min(2 * c->kmax, nf - j0);
        for (int j = 0; j < nb; ++j) {
            jobs[j].in = reinterpret_cast<const char*>(in) + (j0 + j) * in_stride;
            jobs[j].out = reinterpret_cast<char*>(out) + (j0 + j) * out_stride;
            jobs[j].aux = aux ? aux + (size_t)(j0 + j) * an : nullptr;
            jobs[j].dagger = dagger;
        }
        CK(cudaMemcpyAsync(c->d_jobs, jobs.data(), sizeof(ApplyJob) * nb, cudaMemcpyHostToDevice, c->stream));
        CK(launch_apply(c->g, links, c->p.kappa, prec, c->d_jobs, nb, aux != nullptr, c->stream));
        // the job table is reused: wait before overwriting it
        CK(cudaStreamSynchronize(c->stream));
    }
    return LQCD_OK;
}

// r = b - A x for nf FP64 fields (consecutive slots): FP32 hop arithmetic in
// mixed precision (the result feeds FP32 work), FP64 otherwise or when precise
// is set (a residual far below ||A|| ||x||, e.g. after a first solve leg, where
// FP32 hop rounding would swamp it).
lqcd_status residual_fields(lqcd_ctx* c, int nf, const double2* x, double2* r, const double2* b,
                            bool precise = false) {
    if (!c->kprec || precise || c->eo) return apply_fields(c, 0, 0, nf, x, c->dbytes, r, c->dbytes, b);
    std::vector<ApplyJob> jobs(2 * c->kmax);
    for (int j0 = 0; j0 < nf; j0 += 2 * c->kmax) {
        const int nb = std::min(2 * c->kmax, nf - j0);
        for (int j = 0; j < nb; ++j) {
            jobs[j].in = x + (size_t)(j0 + j) * c->N;
            jobs[j].out = r + (size_t)(j0 + j) * c->N;
            jobs[j].aux = b + (size_t)(j0 + j) * c->N;
            jobs[j].dagger = 0;
        }
        CK(cudaMemcpyAsync(c->d_jobs, jobs.data(), sizeof(ApplyJob) * nb, cudaMemcpyHostToDevice, c->stream));
        CK(launch_residual32(c->g, c->links32, c->p.kappa, c->d_jobs, nb, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    return LQCD_OK;
}

// Sources and initial guesses of slots s0 .. s0+k-1 from user memory (full
// fields): b into b_all and x0 into x_hi_all; in an even-odd context through the
// full buffers, b_hat = b_o + k D_oe b_e, x0 -> its odd half, and ||b|| of the
// full systems for the tolerance.
lqcd_status load_sources(lqcd_ctx* c, int s0, int k, const double* b, const double* x0, int on_device) {
    Range nvtx_("sources to device");
    if (!c->eo) {
        lqcd_status s = upload(c, b, k, c->b_all + (size_t)s0 * c->N, 0, on_device);
        if (s != LQCD_OK) return s;
        return upload(c, x0, k, c->x_hi_all + (size_t)s0 * c->N, 0, on_device);
    }
    double2* bf = c->bfull_all + (size_t)s0 * c->Nfull;
    double2* xf = c->xfull_all + (size_t)s0 * c->Nfull;
    lqcd_status s = upload(c, b, k, bf, 0, on_device, c->Nfull);
    if (s != LQCD_OK) return s;
    s = upload(c, x0, k, xf, 0, on_device, c->Nfull);
    if (s != LQCD_OK) return s;
    CK(launch_norms(k, bf, 0, c->Nfull, c->bnorm_all + s0, c->mdscratch, c->mdscratch_elems, c->stream));
    CK(launch_eo_prepare(c->g, c->links64, c->p.kappa, bf, c->b_all + (size_t)s0 * c->N, k, c->stream));
    CK(launch_eo_extract(c->g, xf, c->x_hi_all + (size_t)s0 * c->N, k, c->stream));
    return LQCD_OK;
}

// Solutions of slots s0 .. s0+k-1 to user memory (full fields). In an even-odd
// context x_e = b_e + k D_eo x_o is reconstructed first and, when resid is given,
// resid[j] = ||b - A x|| / ||b|| of the full system in FP64 (the certificate).
lqcd_status store_solutions(lqcd_ctx* c, int s0, int k, double* x, int on_device, double* resid = nullptr) {
    Range nvtx_("solutions from device");
    if (!c->eo) return download(c, c->x_hi_all + (size_t)s0 * c->N, 0, k, x, on_device);
    double2* bf = c->bfull_all + (size_t)s0 * c->Nfull;
    double2* xf = c->xfull_all + (size_t)s0 * c->Nfull;
    CK(launch_eo_reconstruct(c->g, c->links64, c->p.kappa, bf, c->x_hi_all + (size_t)s0 * c->N, xf, k, c->stream));
    if (resid) {
        double2* rf = reinterpret_cast<double2*>(c->eo_scr);   // room for kmax full FP64 fields
        lqcd_status s = apply_fields(c, 0, 0, k, xf, c->Nfull * 16, rf, c->Nfull * 16, bf, true);
        if (s != LQCD_OK) return s;
        double* rn = reinterpret_cast<double*>(c->dsmall);
        CK(launch_norms(k, rf, 0, c->Nfull, rn, c->mdscratch, c->mdscratch_elems, c->stream));
        std::vector<double> hr(k), hb(k);
        CK(cudaMemcpyAsync(hr.data(), rn, sizeof(double) * k, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaMemcpyAsync(hb.data(), c->bnorm_all + s0, sizeof(double) * k, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        for (int j = 0; j < k; ++j) resid[j] = hb[j] > 0 ? hr[j] / hb[j] : 0.0;
    }
    return download(c, xf, 0, k, x, on_device, c->Nfull);
}

}  // namespace

extern "C" lqcd_status lqcd_apply(lqcd_ctx* c, int dagger, lqcd_precision prec, int k, const double* in, double* out,
                                  int on_device) {
    if (!c || !in || !out || k < 0) return LQCD_ERR_ARG;
    const int pr = prec == LQCD_MIXED ? 1 : 0;
    if (pr && !c->links32) return LQCD_ERR_ARG;
    if (k > 0) {
        lqcd_status s = check_buffers(c, in, out, on_device, "lqcd_apply");
        if (s != LQCD_OK) return s;
    }
    // work in chunks of kmax fields: input in x_hi_all / x_lo_all, output in rt_all / win
    for (int j0 = 0; j0 < k; j0 += c->kmax) {
        const int kb = std::min(c->kmax, k - j0);
        void* fin = pr ? (void*)c->x_lo_all : (void*)c->x_hi_all;
        void* fout = pr ? (void*)c->vw_base : (void*)c->rt_all;
        const size_t fb = c->N * (pr ? 8 : 16);
        lqcd_status s = upload(c, in + (size_t)j0 * 2 * c->N, kb, fin, pr, on_device);
        if (s != LQCD_OK) return s;
        s = apply_fields(c, pr, dagger ? 1 : 0, kb, fin, fb, fout, fb, nullptr);
        if (s != LQCD_OK) return s;
        s = download(c, fout, pr, kb, out + (size_t)j0 * 2 * c->N, on_device);
        if (s != LQCD_OK) return s;
    }
    CK(cudaStreamSynchronize(c->stream));
    return LQCD_OK;
}

// ============================================================ deflation
namespace {

// Residual growth beyond which an oblique projection is discarded (see deflate_range).
constexpr double DEFLATE_GROWTH_MAX = 4.0;

// x_hi[j] += U_r H^{-1} U_l^H (b_j - A x_hi[j]) for slots s0 .. s0+k-1
// (precise: FP64 residual, see residual_fields). first (the first deflation of
// a source's initial guess) in the gamma5 variant: a slot whose residual norm
// the projection multiplies by more than DEFLATE_GROWTH_MAX keeps its guess.
// The left vectors are gamma5 images of the right ones, so U_l^H A U_r is close
// to the indefinite Hermitian U_r^H gamma5 A U_r and can be nearly singular; the
// correction is then noise that the FP32 gamma5 recursion may not recover from
// (the general BiCG does). With the guard, rt holds b - A x_hi on return.
lqcd_status deflate_range(lqcd_ctx* c, int s0, int k, bool precise = false, bool first = false) {
    Range nvtx_("deflation");
    const int n = c->n_def;
    if (n == 0 || k == 0) return LQCD_OK;
    const bool guard = first && c->p.gamma5;
    double2* xh = c->x_hi_all + (size_t)s0 * c->N;
    double2* rt = c->rt_all + (size_t)s0 * c->N;
    const double2* bs = c->b_all + (size_t)s0 * c->N;
    lqcd_status s = residual_fields(c, k, xh, rt, bs, precise);
    if (s != LQCD_OK) return s;
    double2* scr = c->dsmall + (size_t)MAX_SMALL * MAX_SMALL * 6;   // norms before / after, reverting C
    double* nrm = reinterpret_cast<double*>(scr);
    double2* Crev = scr + MAX_SLOTS;
    if (guard) CK(launch_norms(k, rt, 0, c->N, nrm, c->mdscratch, c->mdscratch_elems, c->stream));
    double2* C = c->dsmall;   // n x k, ld k
    const void* R = rt;
    int rp = 0;
    if (c->kprec) {   // FP32 projections: convert the residuals first (into these slots' x_lo)
        void* xl = c->krylov(c->x_lo_all, s0);
        CK(launch_convert(rt, 0, xl, 1, (size_t)k * c->N, c->stream));
        R = xl;
        rp = 1;
    }
    CK(launch_multidot(n, c->Ul, c->kprec, k, R, rp, c->N, C, k, 0, c->mdscratch, c->mdscratch_elems, c->stream, c->d_err, c->use_tc));
    CK(launch_lu_solve(n, c->Hlu, c->n_def_max, c->Hpiv, 0, k, C, k, c->stream));
    CK(launch_vupdate(n, c->Ur, c->kprec, C, k, k, xh, 0, 0, c->N, c->stream));
    if (!guard) return LQCD_OK;
    s = residual_fields(c, k, xh, rt, bs, precise);
    if (s != LQCD_OK) return s;
    CK(launch_norms(k, rt, 0, c->N, nrm + MAX_SLOTS, c->mdscratch, c->mdscratch_elems, c->stream));
    double hn[2 * MAX_SLOTS];
    CK(cudaMemcpyAsync(hn, nrm, sizeof(hn), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    bool bad[MAX_SLOTS] = {}, any = false;
    for (int j = 0; j < k; ++j) {
        bad[j] = !(hn[MAX_SLOTS + j] <= DEFLATE_GROWTH_MAX * hn[j]);
        any = any || bad[j];
    }
    if (any) {   // take the correction back from those slots: x_hi -= U_r C
        std::vector<double2> hc((size_t)n * k);
        CK(cudaMemcpyAsync(hc.data(), C, sizeof(double2) * n * k, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < k; ++j) {
                double2& v = hc[(size_t)i * k + j];
                v = bad[j] ? make_double2(-v.x, -v.y) : make_double2(0.0, 0.0);
            }
        CK(cudaMemcpyAsync(Crev, hc.data(), sizeof(double2) * n * k, cudaMemcpyHostToDevice, c->stream));
        CK(launch_vupdate(n, c->Ur, c->kprec, Crev, k, k, xh, 0, 0, c->N, c->stream));
        s = residual_fields(c, k, xh, rt, bs, precise);
        if (s != LQCD_OK) return s;
        for (int j = 0; j < k; ++j) c->deflations_discarded += bad[j] ? 1 : 0;
    }
    return LQCD_OK;
}
lqcd_status deflate_slots(lqcd_ctx* c, int k, bool precise = false, bool first = false) {
    return deflate_range(c, 0, k, precise, first);
}

lqcd_status refactor(lqcd_ctx* c) {
    const int n = c->n_def, ld = c->n_def_max;
    if (n == 0) return LQCD_OK;
    copy_block_kernel<<<64, 256, 0, c->stream>>>(c->Hdef, ld, c->Hlu, ld, n, n);
    copy_block_kernel<<<64, 256, 0, c->stream>>>(c->Mdef, ld, c->Mlu, ld, n, n);
    count_launches(2);
    CK(cudaGetLastError());
    CK(launch_lu_factor(n, c->Hlu, ld, c->Hpiv, c->dinfo, c->stream));
    CK(launch_lu_factor(n, c->Mlu, ld, c->Mpiv, c->dinfo + 1, c->stream));
    return LQCD_OK;
}

// Append nn new pairs (already stored at columns n_def.. of Ur/Ul) after
// bi-orthogonalizing them against the existing space (Algorithm Incremental,
// step 2), scaling to unit norm and growing H = U_l^H A U_r and M = U_l^H U_r.
// work: at least 4*nn Krylov fields (A V', V', A^H W', W').
lqcd_status grow_space(lqcd_ctx* c, int nn, void* work) {
    Range nvtx_("eigenspace growth");
    const int n = c->n_def, ld = c->n_def_max;
    nn = std::min(nn, c->n_def_max - n);
    if (nn <= 0) return LQCD_OK;
    void* Vn = c->krylov(c->Ur, n);
    void* Wn = c->krylov(c->Ul, n);
    const int kp = c->kprec;
    double2* G = c->dsmall;                        // n x nn
    double2* G2 = G + (size_t)MAX_SMALL * 16;      // n x nn
    double2* T1 = G2 + (size_t)MAX_SMALL * 16;     // (n+nn) x 2nn
    double2* T2 = T1 + (size_t)MAX_SMALL * 32;     // n x 2nn (conjugate-transposed store: 2nn x n)
    double2* sc = T2 + (size_t)MAX_SMALL * 32;     // nn scales (V), nn (W)
    double* nrm = reinterpret_cast<double*>(sc + 64);   // 4*nn doubles
    // norms before the projection
    CK(launch_norms(nn, Vn, kp, c->N, nrm, c->mdscratch, c->mdscratch_elems, c->stream));
    CK(launch_norms(nn, Wn, kp, c->N, nrm + nn, c->mdscratch, c->mdscratch_elems, c->stream));
    if (n > 0) {
        // V' = V - U_r M^{-1} U_l^H V ;  W' = W - U_l M^{-H} U_r^H W
        CK(launch_multidot(n, c->Ul, kp, nn, Vn, kp, c->N, G, nn, 0, c->mdscratch, c->mdscratch_elems, c->stream, c->d_err, c->use_tc));
        CK(launch_multidot(n, c->Ur, kp, nn, Wn, kp, c->N, G2, nn, 0, c->mdscratch, c->mdscratch_elems, c->stream, c->d_err, c->use_tc));
        CK(launch_lu_solve(n, c->Mlu, ld, c->Mpiv, 0, nn, G, nn, c->stream));
        CK(launch_lu_solve(n, c->Mlu, ld, c->Mpiv, 1, nn, G2, nn, c->stream));
        negate_kernel<<<1, 256, 0, c->stream>>>(G, n * nn);
        negate_kernel<<<1, 256, 0, c->stream>>>(G2, n * nn);
        count_launches(2);
        CK(cudaGetLastError());
        CK(launch_vupdate(n, c->Ur, kp, G, nn, nn, Vn, kp, 0, c->N, c->stream));
        CK(launch_vupdate(n, c->Ul, kp, G2, nn, nn, Wn, kp, 0, c->N, c->stream));
    }
    CK(launch_norms(nn, Vn, kp, c->N, nrm + 2 * nn, c->mdscratch, c->mdscratch_elems, c->stream));
    CK(launch_norms(nn, Wn, kp, c->N, nrm + 3 * nn, c->mdscratch, c->mdscratch_elems, c->stream));
    std::vector<double> hn(4 * nn);
    CK(cudaMemcpyAsync(hn.data(), nrm, sizeof(double) * 4 * nn, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    // keep pairs whose projected columns retain more than drop of their norm:
    // 1e-8 with FP64 vectors; with FP32 vectors the projection itself carries
    // errors of order 1e-6 of the column, so a column that keeps less than 1e-3
    // is mostly rounding noise and would only make the bases nearly dependent
    const double drop = c->kprec ? 1e-3 : 1e-8;
    std::vector<int> keep;
    std::vector<double2> hsc(2 * nn, make_double2(0.0, 0.0));
    for (int i = 0; i < nn; ++i) {
        const double nv0 = hn[i], nw0 = hn[nn + i], nv = hn[2 * nn + i], nw = hn[3 * nn + i];
        if (nv > drop * nv0 && nw > drop * nw0 && std::isfinite(nv) && std::isfinite(nw)) keep.push_back(i);
        hsc[i] = make_double2(nv > 0 ? 1.0 / nv : 0.0, 0.0);
        hsc[nn + i] = make_double2(nw > 0 ? 1.0 / nw : 0.0, 0.0);
    }
    CK(cudaMemcpyAsync(sc, hsc.data(), sizeof(double2) * 2 * nn, cudaMemcpyHostToDevice, c->stream));
    // scale to unit norm, then compact the kept columns
    CK(launch_scale_fields(nn, Vn, kp, sc, c->N, c->stream));
    CK(launch_scale_fields(nn, Wn, kp, sc + nn, c->N, c->stream));
    int kk = 0;
    for (int i : keep) {
        if (i != kk) {
            CK(cudaMemcpyAsync(c->krylov(c->Ur, n + kk), c->krylov(c->Ur, n + i), c->kbytes, cudaMemcpyDeviceToDevice, c->stream));
            CK(cudaMemcpyAsync(c->krylov(c->Ul, n + kk), c->krylov(c->Ul, n + i), c->kbytes, cudaMemcpyDeviceToDevice, c->stream));
        }
        ++kk;
    }
    if (kk == 0) return LQCD_OK;
    if (kp && kk > 1) {
        // FP32 vectors: the Ritz pairs of one window can be nearly dependent among
        // themselves (repeated copies of a converged pair in a finite-precision
        // Lanczos run), which the column norms above do not see. A complete-pivoting
        // LU of the block W'^H V' keeps a well-conditioned subset: columns of V' and
        // W' of the pivots down to 1e-3 of the first.
        double2* Mb = T1;
        int* sel = reinterpret_cast<int*>(nrm + 4 * nn + 8);
        CK(launch_multidot(kk, Wn, kp, kk, Vn, kp, c->N, Mb, kk, 0, c->mdscratch, c->mdscratch_elems, c->stream,
                           c->d_err, c->use_tc));
        CK(launch_pivot_select(kk, Mb, kk, 1e-3, sel, c->stream));
        std::vector<int> hsel(1 + 2 * kk);
        CK(cudaMemcpyAsync(hsel.data(), sel, sizeof(int) * (1 + 2 * kk), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        const int r = std::max(0, std::min(hsel[0], kk));
        if (r < kk) {
            std::vector<int> wi(hsel.begin() + 1, hsel.begin() + 1 + r);
            std::vector<int> vi(hsel.begin() + 1 + kk, hsel.begin() + 1 + kk + r);
            std::sort(wi.begin(), wi.end());
            std::sort(vi.begin(), vi.end());
            for (int t = 0; t < r; ++t) {   // ascending subsets: each copy moves a column down
                if (vi[t] != t)
                    CK(cudaMemcpyAsync(c->krylov(c->Ur, n + t), c->krylov(c->Ur, n + vi[t]), c->kbytes,
                                       cudaMemcpyDeviceToDevice, c->stream));
                if (wi[t] != t)
                    CK(cudaMemcpyAsync(c->krylov(c->Ul, n + t), c->krylov(c->Ul, n + wi[t]), c->kbytes,
                                       cudaMemcpyDeviceToDevice, c->stream));
            }
            kk = r;
        }
        if (kk == 0) return LQCD_OK;
    }
    // [A V' | V'] and [A^H W' | W'] side by side in the work area, in the storage
    // precision (FP32 operator with two-row links for FP32 storage: the
    // projections are FP32 sums as well, and lqcd_eigs recomputes its pencil in FP64)
    char* AV = reinterpret_cast<char*>(work);
    char* AW = AV + (size_t)2 * kk * c->kbytes;
    lqcd_status s = apply_fields(c, kp, 0, kk, Vn, c->kbytes, AV, c->kbytes, nullptr);
    if (s != LQCD_OK) return s;
    s = apply_fields(c, kp, 1, kk, Wn, c->kbytes, AW, c->kbytes, nullptr);
    if (s != LQCD_OK) return s;
    CK(cudaMemcpyAsync(AV + (size_t)kk * c->kbytes, Vn, (size_t)kk * c->kbytes, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(AW + (size_t)kk * c->kbytes, Wn, (size_t)kk * c->kbytes, cudaMemcpyDeviceToDevice, c->stream));
    // [U_l W']^H [A V' | V'] -> H[:, n:n+kk] and M[:, n:n+kk]  (rows 0..n+kk)
    const int nt = n + kk;
    CK(launch_multidot(nt, c->Ul, kp, 2 * kk, AV, kp, c->N, T1, 2 * kk, 0, c->mdscratch, c->mdscratch_elems, c->stream, c->d_err, c->use_tc));
    copy_block_kernel<<<16, 256, 0, c->stream>>>(T1, 2 * kk, c->Hdef + n, ld, nt, kk);
    copy_block_kernel<<<16, 256, 0, c->stream>>>(T1 + kk, 2 * kk, c->Mdef + n, ld, nt, kk);
    count_launches(2);
    CK(cudaGetLastError());
    if (n > 0) {
        // (A^H W')^H U_r -> H[n:n+kk, 0:n] ;  W'^H U_r -> M[n:n+kk, 0:n]
        CK(launch_multidot(n, c->Ur, kp, 2 * kk, AW, kp, c->N, T2, n, 1, c->mdscratch, c->mdscratch_elems, c->stream, c->d_err, c->use_tc));
        copy_block_kernel<<<16, 256, 0, c->stream>>>(T2, n, c->Hdef + (size_t)n * ld, ld, kk, n);
        copy_block_kernel<<<16, 256, 0, c->stream>>>(T2 + (size_t)kk * n, n, c->Mdef + (size_t)n * ld, ld, kk, n);
        count_launches(2);
        CK(cudaGetLastError());
    }
    c->n_def = n + kk;
    return refactor(c);
}

}  // namespace

extern "C" lqcd_status lqcd_deflate(lqcd_ctx* c, int k, const double* b, double* x0, int on_device) {
    if (!c || !b || !x0 || k < 0) return LQCD_ERR_ARG;
    if (c->n_def == 0) return LQCD_ERR_STATE;
    if (k > 0) {
        lqcd_status s = check_buffers(c, b, x0, on_device, "lqcd_deflate");
        if (s != LQCD_OK) return s;
    }
    for (int j0 = 0; j0 < k; j0 += c->kmax) {
        const int kb = std::min(c->kmax, k - j0);
        lqcd_status s = load_sources(c, 0, kb, b + (size_t)j0 * 2 * c->Nfull, x0 + (size_t)j0 * 2 * c->Nfull,
                                     on_device);
        if (s != LQCD_OK) return s;
        s = deflate_slots(c, kb);
        if (s != LQCD_OK) return s;
        s = store_solutions(c, 0, kb, x0 + (size_t)j0 * 2 * c->Nfull, on_device);
        if (s != LQCD_OK) return s;
    }
    CK(cudaStreamSynchronize(c->stream));
    return LQCD_OK;
}

// ============================================================ the solve
namespace {

// Operator-kernel shape v usable on this context (FP32 Krylov vectors; the
// gamma5 variant has its own list; the staged shape needs its tensor maps).
bool shape_ok(const lqcd_ctx* c, int v) {
    if (c->p.gamma5) return matvec_g5_variant_ok(c->g, v);
    if (v == STAGED_VARIANT && !c->staged_ok) return false;
    return matvec_variant_ok(c->g, v);
}

// The operator pair of one iteration in the autotuned kernel shape.
cudaError_t launch_matvec(lqcd_ctx* c, int nslots, int variant) {
    if (c->eo) {
        const void* links = c->kprec ? (const void*)c->links32 : (const void*)c->links64;
        return launch_eo_pair(c->g, links, c->p.kappa, c->kprec, c->d_state, c->d_ptrs, nslots, c->stream);
    }
    if (c->p.gamma5) {
        const void* links = c->kprec ? (const void*)c->links32 : (const void*)c->links64;
        return launch_bicg_matvec_g5(c->g, links, c->p.kappa, c->kprec, c->d_state, c->d_ptrs, nslots, c->stream,
                                     variant);
    }
    if (variant == TILED && c->tile_ok[nslots])
        return launch_matvec_tiled(c->g, c->tgeo[nslots], c->links32, c->p.kappa, c->d_state, c->d_ptrs, c->d_err,
                                   c->stream);
    if (variant == STAGED_VARIANT && c->kprec && c->staged_ok)
        return launch_matvec_staged(c->g, c->staged_maps, c->p.kappa, c->d_state, c->d_ptrs, nslots, c->d_err, c->nsm,
                                    c->stream);
    const void* links = c->kprec ? (const void*)c->links32 : (const void*)c->links64;
    return launch_bicg_matvec(c->g, links, c->p.kappa, c->kprec, c->d_state, c->d_ptrs, nslots, c->stream,
                              variant == TILED ? 0 : variant);
}

// One chunk of CHECK_EVERY iterations for nslots slots (graph body).
// Kernel groups of an iteration chunk (bit mask): BiCG iteration, its eigBiCG
// window (restart), BiCGStab iteration. Each kernel skips the slots of the
// other kind, so a chunk can serve a mix of slots.
constexpr int CH_BICG = 1, CH_WINDOW = 2, CH_STAB = 4;

lqcd_status enqueue_chunk(lqcd_ctx* c, int nslots, int kinds) {
    const void* links = c->kprec ? (const void*)c->links32 : (const void*)c->links64;
    for (int it = 0; it < CHECK_EVERY; ++it) {
        if (kinds & (CH_BICG | CH_WINDOW)) {
            CK(launch_matvec(c, nslots, c->dslash_variant));
            if (kinds & CH_WINDOW) {
                CK(launch_restart_coeffs(c->d_state, c->d_ptrs, nslots, c->eigwork, c->stream));
                if (c->kprec && c->use_tc && restart_tc_supported(c->m, 2 * c->nev, c->N))
                    CK(launch_restart_tc(c->d_state, c->d_ptrs, nslots, c->N, c->d_err, c->stream));
                else
                    CK(launch_window_gemm(c->kprec, 2 * c->nev, c->d_state, c->d_ptrs, nslots, c->N, c->stream));
            }
            CK(launch_bicg_update(c->kprec, c->d_state, c->d_ptrs, nslots, c->N, c->stream));
            CK(launch_bicg_ru(c->g, c->links64, c->p.kappa, c->kprec, c->d_state, c->d_ptrs, nslots, c->N,
                              c->stream, c->ru_variant, c->links_df, c->eo ? 1 : 0));
            CK(launch_bicg_scalars(c->d_state, c->d_ptrs, nslots, c->stream));
            CK(launch_bicg_direction(c->kprec, c->d_state, c->d_ptrs, nslots, c->N, c->stream));
        }
        if (kinds & CH_STAB) {
            CK(launch_stab_step(c->g, links, c->p.kappa, c->kprec, c->d_state, c->d_ptrs, nslots, c->N, c->stream));
            CK(launch_bicg_ru(c->g, c->links64, c->p.kappa, c->kprec, c->d_state, c->d_ptrs, nslots, c->N,
                              c->stream, c->ru_variant, c->links_df, c->eo ? 1 : 0));
            CK(launch_stab_scalars(c->d_state, nslots, c->stream));
        }
    }
    return LQCD_OK;
}

lqcd_status run_chunk(lqcd_ctx* c, int nslots, int kinds) {
    cudaGraphExec_t& ge = c->graphs[nslots][kinds];
    if (!ge) {
        cudaGraph_t graph = nullptr;
        const long long before = launches_so_far();   // captured launches are not executions
        CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        lqcd_status s = enqueue_chunk(c, nslots, kinds);
        cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
        set_launches(before);
        if (s != LQCD_OK) { if (graph) cudaGraphDestroy(graph); return s; }
        if (e != cudaSuccess) { set_error("cudaStreamEndCapture", e); return LQCD_ERR_CUDA; }
        size_t nodes = 0;
        cudaGraphGetNodes(graph, nullptr, &nodes);
        c->graph_nodes[nslots][kinds] = (long long)nodes;
        e = cudaGraphInstantiate(&ge, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) { ge = nullptr; set_error("cudaGraphInstantiate", e); return LQCD_ERR_CUDA; }
    }
    CK(cudaGraphLaunch(ge, c->stream));
    count_launches(c->graph_nodes[nslots][kinds]);
    return LQCD_OK;
}

// Solve the right-hand sides already in slots 0..k-1 (b_all, x_hi_all) to
// tolerance tol; windowed = eigBiCG window on. rec_stop: stop at the recursive
// convergence candidate without reliable updates (the eigBiCG leg of a
// mixed-precision solve). precise: FP64 starting residual. maxiter[s] (may be
// null) replaces the iteration limit of slot s; a slot whose limit is 0 sits
// the solve out (idle).
lqcd_status solve_slots(lqcd_ctx* c, int k, int windowed, double tol, bool rec_stop = false, bool precise = false,
                        const int* maxiter = nullptr, bool stab = false) {
    Range nvtx_("BiCG iterations");
    for (int s = 0; s < c->kmax; ++s) {
        SlotState& st = c->h_state[s];
        memset(&st, 0, sizeof(SlotState));
        st.maxiter = maxiter && s < k ? maxiter[s] : c->p.maxiter;
        st.status = s < k && st.maxiter > 0 ? ST_RUNNING : ST_IDLE;
        st.tol = tol;
        st.delta = c->kprec && !rec_stop ? c->p.delta : 0.0;
        st.rec_stop = rec_stop ? 1 : 0;
        st.m = windowed ? c->m : 0;
        st.nev = c->nev;
        st.g5 = c->p.gamma5;
        st.stab = stab && !windowed ? 1 : 0;
    }
    CK(cudaMemcpyAsync(c->d_state, c->h_state, sizeof(SlotState) * c->kmax, cudaMemcpyHostToDevice, c->stream));
    // r0 = b - A x0 (FP64), then the Krylov start vectors
    lqcd_status s = residual_fields(c, k, c->x_hi_all, c->rt_all, c->b_all, precise);
    if (s != LQCD_OK) return s;
    CK(launch_bicg_start(c->g, c->links64, c->p.kappa, c->kprec, c->d_state, c->d_ptrs, k, c->N, c->stream));
    while (true) {
        int herr = 0;
        CK(cudaMemcpyAsync(c->h_state, c->d_state, sizeof(SlotState) * k, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaMemcpyAsync(&herr, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        if (herr) {
            // a bounded device wait gave up: the reduction counters may be stale
            CK(cudaMemsetAsync(c->counters, 0, (size_t)c->kmax * CNT_COUNT * sizeof(unsigned), c->stream));
            CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
            CK(cudaStreamSynchronize(c->stream));
            g_last_error = "operator kernel: bounded wait on a TMA copy timed out";
            return LQCD_ERR_TIMEOUT;
        }
        bool any = false;
        for (int j = 0; j < k; ++j) any = any || c->h_state[j].status == ST_RUNNING;
        if (!any) break;
        s = run_chunk(c, k, stab && !windowed ? CH_STAB : (windowed ? CH_BICG | CH_WINDOW : CH_BICG));
        if (s != LQCD_OK) return s;
    }
    CK(launch_bicg_finish(c->g, c->links64, c->p.kappa, c->kprec, c->d_state, c->d_ptrs, k, c->N, c->stream,
                          c->ru_variant, c->eo ? 1 : 0));
    CK(cudaMemcpyAsync(c->h_state, c->d_state, sizeof(SlotState) * k, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return LQCD_OK;
}

// Final Ritz vectors of one finished eigBiCG slot, appended to the eigenspace.
// ritz_ready: the slot's final Ritz pairs are already in ritz_all (grow_from_windows).
lqcd_status grow_slot(lqcd_ctx* c, int s, bool ritz_ready = false) {
    const SlotState& st = c->h_state[s];
    c->last_vs[s] = st.vs;
    c->last_restarts[s] = st.restarts;
    c->last_ritz[s].clear();
    if (st.status != ST_CONVERGED) return LQCD_OK;
    const int vs = st.vs;
    const int nsel = std::min(c->nev, vs);
    if (nsel == 0) return LQCD_OK;
    const int room = c->n_def_max - c->n_def;
    if (room <= 0) return LQCD_OK;
    const int take = std::min(nsel, room);
    // this slot's final Ritz pairs, formed for every slot of the batch at once
    // (grow_from_windows)
    double2* Yc = c->ritz_all + (size_t)s * RITZ_STRIDE;
    double2* Zc = Yc + (size_t)MAX_M * MAX_M;
    double2* lam = Zc + (size_t)MAX_M * MAX_M;
    if (!ritz_ready)
        CK(launch_final_ritz_slots(c->d_state, c->d_ptrs, s, 1, Yc, Zc, lam, c->ritz_n + s, 0, 0, c->eigwork,
                                   c->stream));
    std::vector<double2> hl(nsel);
    CK(cudaMemcpyAsync(hl.data(), lam, sizeof(double2) * nsel, cudaMemcpyDeviceToHost, c->stream));
    const SlotPtrs& P = c->h_ptrs[s];
    // U = V Yc, Q = W Zc  into the next eigenspace columns (first 'take' of nsel)
    CK(launch_vupdate(vs, P.V, c->kprec, Yc, nsel, take, c->krylov(c->Ur, c->n_def), c->kprec, 1, c->N, c->stream));
    CK(launch_vupdate(vs, P.W, c->kprec, Zc, nsel, take, c->krylov(c->Ul, c->n_def), c->kprec, 1, c->N, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->last_ritz[s] = hl;
    // work fields for [A V' | V'], [A^H W' | W']: this slot's window, which
    // holds 2(m+1) > 4 nev Krylov fields
    lqcd_status r = grow_space(c, take, P.V);
    if (r != LQCD_OK) return r;
    c->eig_rhs_done += 1;
    return LQCD_OK;
}

// After an eigBiCG batch: final Ritz vectors of every slot, appended in slot order.
lqcd_status grow_from_windows(lqcd_ctx* c, int k) {
    Range nvtx_("final Ritz vectors");
    c->last_window_valid = 1;
    if (k > 0) {   // final Ritz pairs of every window in one launch (each depends on its window only)
        double2* Yc = c->ritz_all;
        CK(launch_final_ritz_slots(c->d_state, c->d_ptrs, 0, k, Yc, Yc + (size_t)MAX_M * MAX_M,
                                   Yc + (size_t)2 * MAX_M * MAX_M, c->ritz_n, RITZ_STRIDE, RITZ_STRIDE,
                                   c->eigwork, c->stream));
    }
    for (int s = 0; s < k; ++s) {
        lqcd_status r = grow_slot(c, s, true);
        if (r != LQCD_OK) return r;
    }
    return LQCD_OK;
}

lqcd_status status_of(const SlotState& st) {
    switch (st.status) {
        case ST_CONVERGED: return LQCD_OK;
        case ST_BREAKDOWN: return LQCD_ERR_BREAKDOWN;
        case ST_NOCONV: return LQCD_ERR_NOCONV;
        default: return LQCD_OK;
    }
}

}  // namespace

extern "C" lqcd_status lqcd_solve(lqcd_ctx* c, int k, const double* b, double* x, int on_device, lqcd_mode mode,
                                  lqcd_solve_info* info) {
    Range nvtx_("lqcd_solve");
    if (!c || k < 0 || (k > 0 && (!b || !x))) return LQCD_ERR_ARG;
    if (mode < LQCD_MODE_AUTO || mode > LQCD_MODE_PLAIN) return LQCD_ERR_ARG;
    if (c->session_busy()) {
        g_last_error = "lqcd_solve: requests submitted with lqcd_submit are still in flight";
        return LQCD_ERR_STATE;
    }
    if (k > 0) {
        lqcd_status s = check_buffers(c, b, x, on_device, "lqcd_solve");
        if (s != LQCD_OK) return s;
    }
    lqcd_status worst = LQCD_OK;
    for (int j0 = 0, kb = 0; j0 < k; j0 += kb) {
        auto t0 = std::chrono::steady_clock::now();
        kb = std::min(c->kbatch, k - j0);
        lqcd_mode md = mode;
        if (md == LQCD_MODE_AUTO) md = c->eig_rhs_done < c->p.n1 ? LQCD_MODE_EIGBICG : LQCD_MODE_DEFLATED;
        if (md == LQCD_MODE_EIGBICG) {
            // windows for as many sources of the batch as the memory plan admits
            int got = 0;
            for (; got < kb; ++got) {
                bool ok = false;
                lqcd_status s = attach_window(c, got, &ok);
                if (s != LQCD_OK) return s;
                if (!ok) break;
            }
            if (got == 0) {
                g_last_error = "no device memory (or hbm_budget_bytes) for an eigBiCG window";
                return LQCD_ERR_OOM;
            }
            kb = got;
        }
        lqcd_status s = load_sources(c, 0, kb, b + (size_t)j0 * 2 * c->Nfull, x + (size_t)j0 * 2 * c->Nfull,
                                     on_device);
        if (s != LQCD_OK) return s;
        int outer = 0;
        if (md != LQCD_MODE_PLAIN && c->n_def > 0) {
            s = deflate_slots(c, kb, false, true);
            if (s != LQCD_OK) return s;
        }
        std::vector<SlotState> first;
        const bool windowed = md == LQCD_MODE_EIGBICG;
        if (windowed) c->last_window_valid = 0;
        if (md == LQCD_MODE_DEFLATED && c->p.deftol > c->p.tol && c->n_def > 0) {
            // DefTol restart: solve to deftol, re-deflate, solve to tol
            s = solve_slots(c, kb, 0, c->p.deftol, false, false, nullptr, c->p.bicgstab != 0);
            if (s != LQCD_OK) return s;
            first.assign(c->h_state, c->h_state + kb);
            s = deflate_slots(c, kb, c->kprec != 0);
            if (s != LQCD_OK) return s;
            outer = 1;
        }
        // Mixed-precision eigBiCG runs in two legs: the windowed iteration without
        // reliable updates (replacing r by the true residual would break the
        // Lanczos relation W^H A V = H of the window) until the recursive residual
        // reaches tol; its Ritz vectors grow the eigenspace; then a deflated
        // correction leg from the FP64 residual, with reliable updates, to tol.
        const bool two_leg = windowed && c->kprec;
        s = solve_slots(c, kb, windowed ? 1 : 0, c->p.tol, two_leg, outer > 0 && c->kprec, nullptr,
                        c->p.bicgstab != 0);
        if (s != LQCD_OK) return s;
        std::vector<SlotState> fin(c->h_state, c->h_state + kb);
        if (windowed) {
            s = grow_from_windows(c, kb);
            if (s != LQCD_OK) return s;
            for (int j = 0; j < kb; ++j) {
                s = detach_window(c, j);
                if (s != LQCD_OK) return s;
            }
        }
        if (two_leg) {
            first = fin;
            std::vector<int> left(kb, 0);
            for (int j = 0; j < kb; ++j)
                if (first[j].status == ST_CONVERGED) left[j] = std::max(c->p.maxiter - first[j].iter, 0);
            if (std::count(left.begin(), left.end(), 0) == 0) {
                s = deflate_slots(c, kb, true);
            } else {   // a slot whose first leg failed keeps its iterate
                for (int j = 0; j < kb && s == LQCD_OK; ++j)
                    if (left[j] > 0) s = deflate_range(c, j, 1, true);
            }
            if (s != LQCD_OK) return s;
            s = solve_slots(c, kb, 0, c->p.tol, false, true, left.data());
            if (s != LQCD_OK) return s;
            outer = 1;
            for (int j = 0; j < kb; ++j) {
                if (left[j] > 0) {
                    const int restarts = first[j].restarts;
                    fin[j] = c->h_state[j];
                    fin[j].restarts = restarts;
                } else {
                    first[j] = SlotState{};   // the first leg stopped short: report it alone
                }
            }
        }
        std::vector<double> full_resid(kb, -1.0);
        s = store_solutions(c, 0, kb, x + (size_t)j0 * 2 * c->Nfull, on_device, c->eo ? full_resid.data() : nullptr);
        if (s != LQCD_OK) return s;
        CK(cudaStreamSynchronize(c->stream));
        const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        for (int j = 0; j < kb; ++j) {
            SlotState& st = fin[j];
            if (full_resid[j] >= 0.0) st.true_rnorm = full_resid[j] * st.bnorm;   // the full system's certificate
            lqcd_status sj = status_of(st);
            if (sj == LQCD_OK && st.bnorm > 0 && st.true_rnorm > c->p.tol * st.bnorm) sj = LQCD_ERR_NOCONV;
            if (sj != LQCD_OK && worst == LQCD_OK) worst = sj;
            if (info) {
                lqcd_solve_info& in = info[j0 + j];
                in.iters = st.iter + (first.empty() ? 0 : first[j].iter);
                in.matvecs = st.matvecs + (first.empty() ? 0 : first[j].matvecs);
                in.restarts = st.restarts;
                in.reliable_updates = st.ru_count + (first.empty() ? 0 : first[j].ru_count);
                in.outer_steps = outer;
                in.true_resid = st.bnorm > 0 ? st.true_rnorm / st.bnorm : 0.0;
                in.seconds = secs;
                in.mode_used = md;
            }
        }
    }
    return worst;
}

// ============================================================ eigenspace I/O
extern "C" lqcd_status lqcd_eigspace_get(lqcd_ctx* c, double* Ur, double* Ul, double* H) {
    if (!c) return LQCD_ERR_ARG;
    const int n = c->n_def;
    if (Ur) { lqcd_status s = download(c, c->Ur, c->kprec, n, Ur, 0); if (s != LQCD_OK) return s; }
    if (Ul) { lqcd_status s = download(c, c->Ul, c->kprec, n, Ul, 0); if (s != LQCD_OK) return s; }
    if (H && n > 0) {
        CK(cudaMemcpy2DAsync(H, sizeof(double2) * n, c->Hdef, sizeof(double2) * c->n_def_max, sizeof(double2) * n, n,
                             cudaMemcpyDeviceToHost, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    return LQCD_OK;
}

namespace {

// H = U_l^H A U_r and M = U_l^H U_r over the first n pairs, in FP64 arithmetic
// (FP32-stored columns are converted to FP64 first), into Hout / Mout (ld).
lqcd_status project_fp64(lqcd_ctx* c, int n, double2* Hout, double2* Mout, int ld) {
    for (int j0 = 0; j0 < n; j0 += c->kmax) {
        const int kb = std::min(c->kmax, n - j0);
        const void* src = c->krylov(c->Ur, j0);
        const void* in = src;
        if (c->kprec) {
            CK(launch_convert(src, 1, c->x_hi_all, 0, (size_t)kb * c->N, c->stream));
            in = c->x_hi_all;
        }
        lqcd_status s = apply_fields(c, 0, 0, kb, in, c->kprec ? c->dbytes : c->kbytes, c->rt_all, c->dbytes, nullptr);
        if (s != LQCD_OK) return s;
        CK(launch_multidot(n, c->Ul, c->kprec, kb, c->rt_all, 0, c->N, Hout + j0, ld, 0, c->mdscratch,
                           c->mdscratch_elems, c->stream, c->d_err, c->use_tc));
        CK(launch_multidot(n, c->Ul, c->kprec, kb, in, 0, c->N, Mout + j0, ld, 0, c->mdscratch,
                           c->mdscratch_elems, c->stream, c->d_err, c->use_tc));
    }
    return LQCD_OK;
}

}  // namespace

extern "C" lqcd_status lqcd_eigspace_set(lqcd_ctx* c, int n, const double* Ur, const double* Ul) {
    if (!c || n < 0 || n > c->n_def_max) return LQCD_ERR_ARG;
    if (n > 0 && (!Ur || !Ul)) return LQCD_ERR_ARG;
    c->n_def = 0;
    c->eig_rhs_done = 0;
    if (n == 0) return LQCD_OK;
    lqcd_status s = upload(c, Ur, n, c->Ur, c->kprec, 0);
    if (s != LQCD_OK) return s;
    s = upload(c, Ul, n, c->Ul, c->kprec, 0);
    if (s != LQCD_OK) return s;
    s = project_fp64(c, n, c->Hdef, c->Mdef, c->n_def_max);
    if (s != LQCD_OK) return s;
    c->n_def = n;
    c->eig_rhs_done = c->p.n1;   // a loaded eigenspace counts as complete for LQCD_MODE_AUTO
    s = refactor(c);
    if (s != LQCD_OK) return s;
    CK(cudaStreamSynchronize(c->stream));
    return LQCD_OK;
}

// ============================================================ Rayleigh-Ritz
extern "C" lqcd_status lqcd_eigs(lqcd_ctx* c, int* n_inout, double* evals, double* evecs_r, double* evecs_l,
                                 double* resid) {
    Range nvtx_("Rayleigh-Ritz");
    if (!c || !n_inout || !evals) return LQCD_ERR_ARG;
    const int n = c->n_def;
    if (n == 0) return LQCD_ERR_STATE;
    const int nout = std::min(*n_inout, n);
    const int ld = c->n_def_max;
    // Pencil (H, M) with P M = L U: G = L^{-1} P H U^{-1} (n x n, ld n), eig(G) ->
    // lam, Yhat, Zhat; right vectors y = U^{-1} yhat, left z = P^T L^{-H} zhat.
    // The two-sided form splits M's conditioning between the factors (the
    // accumulated bases are nearly dependent: cond(M) reaches 1e13) and keeps the
    // eigenvalues at the accuracy of a QZ solve of the pencil, where M^{-1} H loses
    // three or more digits.
    double2* G = c->dsmall;
    double2* Y = G + (size_t)n * n;
    double2* Z = Y + (size_t)n * n;
    double2* lam = Z + (size_t)n * n;
    // Pencil (U_l^H A U_r, U_l^H U_r) in FP64 arithmetic. With FP32-stored vectors
    // the projections kept for deflation were summed in FP32, so recompute them.
    const double2* Hp = c->Hdef;
    const double2* Mp = c->Mlu;
    const int* Mpiv = c->Mpiv;
    int ldp = ld;
    if (c->kprec) {
        double2* Hr = c->dsmall + (size_t)MAX_SMALL * MAX_SMALL * 4;
        double2* Mr = Hr + (size_t)n * n;
        int* piv = c->dinfo + 24;
        lqcd_status s = project_fp64(c, n, Hr, Mr, n);
        if (s != LQCD_OK) return s;
        CK(launch_lu_factor(n, Mr, n, piv, c->dinfo + 20, c->stream));
        Hp = Hr; Mp = Mr; Mpiv = piv; ldp = n;
    }
    copy_block_kernel<<<64, 256, 0, c->stream>>>(Hp, ldp, G, n, n, n);
    count_launches(1);
    CK(cudaGetLastError());
    CK(launch_lu_part(n, Mp, ldp, Mpiv, LU_LEFT_PL, n, G, n, c->stream));
    CK(launch_lu_part(n, Mp, ldp, Mpiv, LU_RIGHT_U, n, G, n, c->stream));
    CK(launch_small_eig(n, G, n, n, lam, Y, Z, n, c->dinfo + 16, c->eigwork, c->stream));
    CK(launch_lu_part(n, Mp, ldp, Mpiv, LU_LEFT_U, n, Y, n, c->stream));
    CK(launch_lu_part(n, Mp, ldp, Mpiv, LU_LEFT_LH, n, Z, n, c->stream));
    std::vector<double2> hl(n);
    CK(cudaMemcpyAsync(hl.data(), lam, sizeof(double2) * n, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int i = 0; i < nout; ++i) { evals[2 * i] = hl[i].x; evals[2 * i + 1] = hl[i].y; }
    // vectors in chunks of kmax: u = U_r y (FP64 in x_hi_all), w = U_l z (rt_all)
    std::vector<double> hres(nout, 0.0);
    for (int j0 = 0; j0 < nout; j0 += c->kmax) {
        const int kb = std::min(c->kmax, nout - j0);
        CK(launch_vupdate(n, c->Ur, c->kprec, Y + j0, n, kb, c->x_hi_all, 0, 1, c->N, c->stream, 1));
        if (evecs_r) {
            lqcd_status s = download(c, c->x_hi_all, 0, kb, evecs_r + (size_t)j0 * 2 * c->N, 0);
            if (s != LQCD_OK) return s;
        }
        if (evecs_l) {
            CK(launch_vupdate(n, c->Ul, c->kprec, Z + j0, n, kb, c->rt_all, 0, 1, c->N, c->stream, 1));
            lqcd_status s = download(c, c->rt_all, 0, kb, evecs_l + (size_t)j0 * 2 * c->N, 0);
            if (s != LQCD_OK) return s;
        }
        if (resid) {
            // r_j = A u_j - lam_j u_j ; |r_j| / |u_j|
            lqcd_status s = apply_fields(c, 0, 0, kb, c->x_hi_all, c->dbytes, c->rt_all, c->dbytes, nullptr);
            if (s != LQCD_OK) return s;
            double2* D = c->dsmall + (size_t)MAX_SMALL * MAX_SMALL * 6;
            std::vector<double2> hd((size_t)kb * kb, make_double2(0, 0));
            for (int j = 0; j < kb; ++j) hd[(size_t)j * kb + j] = make_double2(-hl[j0 + j].x, -hl[j0 + j].y);
            CK(cudaMemcpyAsync(D, hd.data(), sizeof(double2) * kb * kb, cudaMemcpyHostToDevice, c->stream));
            CK(launch_vupdate(kb, c->x_hi_all, 0, D, kb, kb, c->rt_all, 0, 0, c->N, c->stream));
            double2* gr = D + 256;
            double2* gu = gr + 256;
            CK(launch_multidot(kb, c->rt_all, 0, kb, c->rt_all, 0, c->N, gr, kb, 0, c->mdscratch, c->mdscratch_elems, c->stream, c->d_err, c->use_tc));
            CK(launch_multidot(kb, c->x_hi_all, 0, kb, c->x_hi_all, 0, c->N, gu, kb, 0, c->mdscratch, c->mdscratch_elems, c->stream, c->d_err, c->use_tc));
            std::vector<double2> hr((size_t)kb * kb), hu((size_t)kb * kb);
            CK(cudaMemcpyAsync(hr.data(), gr, sizeof(double2) * kb * kb, cudaMemcpyDeviceToHost, c->stream));
            CK(cudaMemcpyAsync(hu.data(), gu, sizeof(double2) * kb * kb, cudaMemcpyDeviceToHost, c->stream));
            CK(cudaStreamSynchronize(c->stream));
            for (int j = 0; j < kb; ++j)
                hres[j0 + j] = std::sqrt(std::max(hr[(size_t)j * kb + j].x, 0.0)) / std::sqrt(std::max(hu[(size_t)j * kb + j].x, 1e-300));
        }
    }
    CK(cudaStreamSynchronize(c->stream));
    if (resid)
        for (int i = 0; i < nout; ++i) resid[i] = hres[i];
    *n_inout = nout;
    return LQCD_OK;
}

// ============================================================ inspection
extern "C" lqcd_status lqcd_last_window(lqcd_ctx* c, int slot, int* vs, double* H, double* ritz, int* restarts) {
    if (!c || slot < 0 || slot >= c->kmax) return LQCD_ERR_ARG;
    if (!c->last_window_valid) return LQCD_ERR_STATE;
    const int nvs = c->last_vs[slot];
    if (vs) *vs = nvs;
    if (restarts) *restarts = c->last_restarts[slot];
    if (H) {
        std::vector<double2> h((size_t)c->m * c->m);
        CK(cudaMemcpy(h.data(), c->h_ptrs[slot].H, sizeof(double2) * c->m * c->m, cudaMemcpyDeviceToHost));
        for (int i = 0; i < nvs; ++i)
            for (int j = 0; j < nvs; ++j) {
                H[2 * ((size_t)i * nvs + j)] = h[(size_t)i * c->m + j].x;
                H[2 * ((size_t)i * nvs + j) + 1] = h[(size_t)i * c->m + j].y;
            }
    }
    if (ritz) {
        const auto& r = c->last_ritz[slot];
        for (size_t i = 0; i < r.size(); ++i) { ritz[2 * i] = r[i].x; ritz[2 * i + 1] = r[i].y; }
    }
    return LQCD_OK;
}

// ============================================================ test hooks
extern "C" lqcd_status lqcd_small_eig(int n, const double* C, double* evals, double* Yout, double* Zout) {
    if (n < 1 || n > MAX_SMALL || !C || !evals) return LQCD_ERR_ARG;
    double2 *dA = nullptr, *dl = nullptr, *dY = nullptr, *dZ = nullptr, *dw = nullptr;
    int* dinfo = nullptr;
    size_t nn = (size_t)n * n;
    lqcd_status ret = LQCD_OK;
    cudaError_t e;
    if ((e = cudaMalloc(&dA, nn * 16)) != cudaSuccess || (e = cudaMalloc(&dl, n * 16)) != cudaSuccess ||
        (e = cudaMalloc(&dY, nn * 16)) != cudaSuccess || (e = cudaMalloc(&dZ, nn * 16)) != cudaSuccess ||
        (e = cudaMalloc(&dw, eig_work_elems() * 16)) != cudaSuccess || (e = cudaMalloc(&dinfo, 16)) != cudaSuccess) {
        set_error("cudaMalloc", e);
        ret = LQCD_ERR_OOM;
    }
    int info = 0;
    if (ret == LQCD_OK) {
        e = cudaMemcpy(dA, C, nn * 16, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = launch_small_eig(n, dA, n, n, dl, dY, dZ, n, dinfo, dw, 0);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e == cudaSuccess) e = cudaMemcpy(evals, dl, n * 16, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && Yout) e = cudaMemcpy(Yout, dY, nn * 16, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && Zout) e = cudaMemcpy(Zout, dZ, nn * 16, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(&info, dinfo, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) { set_error("small eig", e); ret = LQCD_ERR_CUDA; }
        else if (info) { g_last_error = "QR iteration did not converge"; ret = LQCD_ERR_NOCONV; }
    }
    cudaFree(dA); cudaFree(dl); cudaFree(dY); cudaFree(dZ); cudaFree(dw); cudaFree(dinfo);
    return ret;
}

extern "C" lqcd_status lqcd_field_dots(int a, const float* X, int b, const float* Y, long long n, int path, int reps,
                                       double* C, double* avg_ms) {
    if (a < 1 || b < 1 || n < 1 || !X || !Y || !C || (path != 0 && path != 1) || reps < 0 || (reps > 0 && !avg_ms))
        return LQCD_ERR_ARG;
    const size_t N = (size_t)n;
    if (path == 1 && !dots_tc_supported(a, X, Y, N)) {
        g_last_error = "tensor-core path needs 2n % 32 == 0, a <= 512 and 16-byte aligned fields";
        return LQCD_ERR_ARG;
    }
    const size_t md_elems = std::max((size_t)((a + 3) / 4) * 1216 * 32, dots_tc_scratch_doubles(a) / 2 + 1);
    double2 *scratch = nullptr, *dC = nullptr;
    int* derr = nullptr;
    lqcd_status ret = LQCD_OK;
    cudaError_t e;
    if ((e = cudaMalloc(&scratch, md_elems * 16)) != cudaSuccess || (e = cudaMalloc(&dC, (size_t)a * b * 16)) != cudaSuccess ||
        (e = cudaMalloc(&derr, 16)) != cudaSuccess) {
        set_error("cudaMalloc", e);
        ret = LQCD_ERR_OOM;
    }
    if (ret == LQCD_OK) {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        e = cudaMemset(derr, 0, 16);
        if (e == cudaSuccess) e = cudaEventCreate(&e0);
        if (e == cudaSuccess) e = cudaEventCreate(&e1);
        for (int r = 0; e == cudaSuccess && r <= reps; ++r) {
            if (r == 1) e = cudaEventRecord(e0, 0);
            if (e == cudaSuccess)
                e = launch_multidot(a, X, 1, b, Y, 1, N, dC, b, 0, scratch, md_elems, 0, derr, path);
        }
        if (e == cudaSuccess && reps > 0) e = cudaEventRecord(e1, 0);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e == cudaSuccess && reps > 0) {
            float ms = 0.f;
            e = cudaEventElapsedTime(&ms, e0, e1);
            *avg_ms = ms / reps;
        }
        int herr = 0;
        if (e == cudaSuccess) e = cudaMemcpy(C, dC, (size_t)a * b * 16, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) { set_error("field dots", e); ret = LQCD_ERR_CUDA; }
        else if (herr) { g_last_error = "tensor-core dots: a bounded wait timed out"; ret = LQCD_ERR_TIMEOUT; }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
    cudaFree(scratch); cudaFree(dC); cudaFree(derr);
    return ret;
}

extern "C" lqcd_status lqcd_restart_coefficients(int m, int nev, const double* H, int* r, double* Yc, double* Zc,
                                                 double* lam) {
    if (m < 3 || m > MAX_M || nev < 1 || 2 * nev >= m || !H || !r) return LQCD_ERR_ARG;
    double2 *dH = nullptr, *dY = nullptr, *dZ = nullptr, *dl = nullptr, *dw = nullptr;
    int* di = nullptr;
    lqcd_status ret = LQCD_OK;
    cudaError_t e;
    const size_t cs = (size_t)m * 2 * nev;
    if ((e = cudaMalloc(&dH, (size_t)m * m * 16)) != cudaSuccess || (e = cudaMalloc(&dY, cs * 16)) != cudaSuccess ||
        (e = cudaMalloc(&dZ, cs * 16)) != cudaSuccess || (e = cudaMalloc(&dl, 2 * nev * 16)) != cudaSuccess ||
        (e = cudaMalloc(&dw, eig_work_elems() * 16)) != cudaSuccess || (e = cudaMalloc(&di, 16)) != cudaSuccess) {
        set_error("cudaMalloc", e);
        ret = LQCD_ERR_OOM;
    }
    int hi[2] = {0, 0};
    if (ret == LQCD_OK) {
        e = cudaMemcpy(dH, H, (size_t)m * m * 16, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = launch_restart_coeffs_single(m, nev, dH, di, dY, dZ, dl, di + 1, dw, 0);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e == cudaSuccess) e = cudaMemcpy(hi, di, 2 * sizeof(int), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && Yc) e = cudaMemcpy(Yc, dY, cs * 16, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && Zc) e = cudaMemcpy(Zc, dZ, cs * 16, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && lam) e = cudaMemcpy(lam, dl, 2 * nev * 16, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) { set_error("restart coefficients", e); ret = LQCD_ERR_CUDA; }
        else {
            *r = hi[0];
            if (hi[1]) { g_last_error = "QR iteration did not converge"; ret = LQCD_ERR_NOCONV; }
        }
    }
    cudaFree(dH); cudaFree(dY); cudaFree(dZ); cudaFree(dl); cudaFree(dw); cudaFree(di);
    return ret;
}

// ============================================================ measurement
extern "C" long long lqcd_kernel_launches(void) { return launches_so_far(); }

constexpr int TIME_TILED = 99;   // lqcd_time_kernel id of the plane-streaming shape

static lqcd_status time_kernel_impl(lqcd_ctx* c, int kernel, int k, int reps, double* avg_ms) {
    if (!c || !avg_ms || k < 1 || k > c->kmax || reps < 1) return LQCD_ERR_ARG;
    if (kernel < 0 || (kernel > 3 && kernel < 10) ||
        (kernel >= 10 + matvec_variants() && kernel != TIME_TILED && !(kernel >= 40 && kernel < 40 + true_resid_variants())))
        return LQCD_ERR_ARG;
    if (kernel == TIME_TILED && !c->tile_ok[k]) return LQCD_ERR_ARG;
    if (c->eo && kernel >= 10) return LQCD_ERR_ARG;   // one operator shape
    if (kernel >= 10 && kernel < 10 + matvec_variants() && !shape_ok(c, kernel - 10)) return LQCD_ERR_ARG;
    const int ru_saved = c->ru_variant;
    if (kernel >= 40 && kernel < 40 + true_resid_variants()) {   // reliable update with FP64 shape v
        c->ru_variant = kernel - 40;
        kernel = 3;
    }
    // Slots 0..k-1 iterate with fixed scalars on whatever their buffers hold.
    std::vector<SlotState> tmpl(c->kmax);
    for (int s = 0; s < c->kmax; ++s) {
        SlotState& st = tmpl[s];
        memset(&st, 0, sizeof(SlotState));
        st.status = s < k ? ST_RUNNING : ST_IDLE;
        st.live = s < k;
        st.need_ru = 1;
        st.tol = 0.0;
        st.maxiter = 1 << 30;
        st.rho = make_double2(1.0, 0.0);
        st.rnorm = 1.0; st.bnorm = 1.0; st.rmax = 1.0; st.r_ru = 1.0;
        st.alpha = make_double2(0.1, 0.0);
        st.beta = make_double2(0.1, 0.0);
        st.g5 = c->p.gamma5;
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    double total = 0.0;
    for (int r = 0; r < reps; ++r) {
        CK(cudaMemcpyAsync(c->d_state, tmpl.data(), sizeof(SlotState) * c->kmax, cudaMemcpyHostToDevice, c->stream));
        CK(cudaEventRecord(e0, c->stream));
        if (kernel == 0) CK(launch_matvec(c, k, c->dslash_variant));
        else if (kernel == TIME_TILED) CK(launch_matvec(c, k, TILED));
        else if (kernel >= 10) CK(launch_matvec(c, k, kernel - 10));
        else if (kernel == 1) CK(launch_bicg_update(c->kprec, c->d_state, c->d_ptrs, k, c->N, c->stream));
        else if (kernel == 2) CK(launch_bicg_direction(c->kprec, c->d_state, c->d_ptrs, k, c->N, c->stream));
        else CK(launch_bicg_ru(c->g, c->links64, c->p.kappa, c->kprec, c->d_state, c->d_ptrs, k, c->N, c->stream,
                               c->ru_variant, c->links_df, c->eo ? 1 : 0));
        CK(cudaEventRecord(e1, c->stream));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        total += ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->ru_variant = ru_saved;
    // leave the slots idle
    for (int s = 0; s < c->kmax; ++s) { tmpl[s].status = ST_IDLE; tmpl[s].live = 0; }
    CK(cudaMemcpyAsync(c->d_state, tmpl.data(), sizeof(SlotState) * c->kmax, cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    *avg_ms = total / reps;
    return LQCD_OK;
}

extern "C" lqcd_status lqcd_time_kernel(lqcd_ctx* c, int kernel, int k, int reps, double* avg_ms) {
    return time_kernel_impl(c, kernel, k, reps, avg_ms);
}

extern "C" int lqcd_dslash_variant(const lqcd_ctx* c) { return c ? c->dslash_variant : -1; }

static void drop_graphs(lqcd_ctx* c) {
    for (int i = 0; i <= MAX_SLOTS; ++i)   // the iteration graphs hold the old kernels
        for (int j = 0; j < 8; ++j)
            if (c->graphs[i][j]) {
                cudaGraphExecDestroy(c->graphs[i][j]);
                c->graphs[i][j] = nullptr;
            }
}

extern "C" lqcd_status lqcd_set_tensor_cores(lqcd_ctx* c, int on) {
    if (!c) return LQCD_ERR_ARG;
    if (c->session_busy()) {
        g_last_error = "lqcd_set_tensor_cores: requests are in flight";
        return LQCD_ERR_STATE;
    }
    CK(cudaStreamSynchronize(c->stream));
    c->use_tc = on ? 1 : 0;
    drop_graphs(c);
    return LQCD_OK;
}

extern "C" lqcd_status lqcd_set_dslash_variant(lqcd_ctx* c, int variant) {
    if (!c) return LQCD_ERR_ARG;
    if (c->session_busy()) {
        g_last_error = "lqcd_set_dslash_variant: requests are in flight";
        return LQCD_ERR_STATE;
    }
    const bool ok = variant == TILED ? (c->kprec && !c->eo && !c->p.gamma5 && c->tile_ok[c->kmax])
                                     : variant >= 0 && variant < matvec_variants() && !c->eo &&
                                           (c->kprec || variant == 0) && shape_ok(c, variant);
    if (!ok) {
        g_last_error = "lqcd_set_dslash_variant: shape not available on this context";
        return LQCD_ERR_ARG;
    }
    CK(cudaStreamSynchronize(c->stream));
    c->dslash_variant = variant;
    drop_graphs(c);
    return LQCD_OK;
}

// Autotuner: time every operator-kernel variant on this lattice with a full
// batch and keep the fastest (FP32 operator only; FP64 has one shape).
static lqcd_status autotune(lqcd_ctx* c) {
    Range nvtx_("autotune operator shapes");
    if (c->eo) return LQCD_OK;   // the even-odd operator and its FP64 residual have one shape each
    {   // FP64 true-residual shape
        double best_ru = 1e300;
        for (int v = 0; v < true_resid_variants(); ++v) {
            double ms = 0.0;
            if (v >= RU_DF && !c->links_df) continue;
            lqcd_status s = time_kernel_impl(c, 40 + v, 1, 1, &ms);
            if (s != LQCD_OK) return s;
            s = time_kernel_impl(c, 40 + v, 1, 2, &ms);
            if (s != LQCD_OK) return s;
            if (ms < best_ru) { best_ru = ms; c->ru_variant = v; }
        }
    }
    if (!c->kprec) return LQCD_OK;
    const int nv = matvec_variants();
    c->tune_ms.assign(nv, 0.0);
    double best = 1e300;
    for (int v = 0; v < nv; ++v) {
        double ms = 0.0;
        if (!shape_ok(c, v)) {
            c->tune_ms[v] = -1.0;
            continue;
        }
        lqcd_status s = time_kernel_impl(c, 10 + v, c->kmax, 1, &ms);   // warm-up
        if (s != LQCD_OK) return s;
        s = time_kernel_impl(c, 10 + v, c->kmax, 3, &ms);
        if (s != LQCD_OK) return s;
        c->tune_ms[v] = ms;
        if (ms < best) { best = ms; c->dslash_variant = v; }
    }
    if (c->tile_ok[c->kmax]) {
        double ms = 0.0;
        lqcd_status s = time_kernel_impl(c, TIME_TILED, c->kmax, 1, &ms);
        if (s != LQCD_OK) return s;
        s = time_kernel_impl(c, TIME_TILED, c->kmax, 3, &ms);
        if (s != LQCD_OK) return s;
        c->tune_ms.push_back(ms);
        if (ms < best) { best = ms; c->dslash_variant = TILED; }
    }
    int herr = 0;
    CK(cudaMemcpy(&herr, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr) {
        // the plane-streaming kernel timed out on a copy: never use it on this context
        CK(cudaMemset(c->d_err, 0, sizeof(int)));
        CK(cudaMemset(c->counters, 0, (size_t)c->kmax * CNT_COUNT * sizeof(unsigned)));
        for (int n = 0; n <= MAX_SLOTS; ++n) c->tile_ok[n] = false;
        if (c->dslash_variant == TILED) c->dslash_variant = 0;
    }
    return LQCD_OK;
}

// Batch-size autotuner (k_max = 0): time one BiCG iteration (operator, residual
// update, direction update) over k = 1, 2, 4, 8 slots and keep the k with the most
// right-hand sides per second (ties to the larger k, which needs fewer launches).
static lqcd_status autotune_batch(lqcd_ctx* c) {
    Range nvtx_("autotune batch size");
    double best = 0.0;
    int kbest = c->kmax;
    for (int k = 1; k <= c->kmax; k *= 2) {
        double t = 0.0;
        for (int kernel = 0; kernel < 3; ++kernel) {
            double ms = 0.0;
            lqcd_status s = time_kernel_impl(c, kernel, k, 1, &ms);   // warm-up
            if (s != LQCD_OK) return s;
            s = time_kernel_impl(c, kernel, k, 3, &ms);
            if (s != LQCD_OK) return s;
            t += ms;
        }
        c->k_ms[k] = t;
        const double rate = k / t;
        if (rate >= best * 0.99) { best = std::max(best, rate); kbest = k; }
    }
    c->kbatch = kbest;
    return LQCD_OK;
}

extern "C" int lqcd_batch_size(const lqcd_ctx* c) { return c ? c->kbatch : 0; }

extern "C" lqcd_status lqcd_memory_info(const lqcd_ctx* c, size_t* plan_bytes, size_t* window_bytes,
                                        int* windows_attached) {
    if (!c) return LQCD_ERR_ARG;
    if (plan_bytes) *plan_bytes = c->plan_bytes;
    if (window_bytes) *window_bytes = c->win_bytes;
    if (windows_attached) *windows_attached = c->win_attached;
    return LQCD_OK;
}

extern "C" lqcd_status lqcd_batch_timings(const lqcd_ctx* c, double* ms) {
    if (!c || !ms) return LQCD_ERR_ARG;
    for (int k = 0; k <= MAX_SLOTS; ++k) ms[k] = c->k_ms[k];
    return c->k_auto ? LQCD_OK : LQCD_ERR_STATE;
}

// ============================================================ pair-kernel hook
extern "C" lqcd_status lqcd_apply_pair(lqcd_ctx* c, int variant, int k, const double* p, const double* phat,
                                       double* Ap, double* Ahp, double* sigma) {
    if (!c || !p || !phat || !Ap || !Ahp || k < 1 || k > c->kmax) return LQCD_ERR_ARG;
    if (c->eo && variant != 0) return LQCD_ERR_ARG;
    if (variant == TILED) {
        if (!c->tile_ok[k]) return LQCD_ERR_ARG;
    } else if (variant < 0 || variant >= matvec_variants() || (!c->kprec && variant != 0) ||
               !shape_ok(c, variant)) {
        return LQCD_ERR_ARG;
    }
    const size_t fb = 2 * c->N;   // doubles per host field
    for (int s = 0; s < k; ++s) {
        lqcd_status r = upload(c, p + s * fb, 1, c->h_ptrs[s].p, c->kprec, 0);
        if (r != LQCD_OK) return r;
        r = upload(c, phat + s * fb, 1, c->h_ptrs[s].phat, c->kprec, 0);
        if (r != LQCD_OK) return r;
    }
    std::vector<SlotState> tmpl(c->kmax);
    for (int s = 0; s < c->kmax; ++s) {
        memset(&tmpl[s], 0, sizeof(SlotState));
        tmpl[s].status = s < k ? ST_RUNNING : ST_IDLE;
        tmpl[s].rho = make_double2(1.0, 0.0);
        tmpl[s].g5 = c->p.gamma5;
        tmpl[s].m = c->p.gamma5 ? 1 : 0;   // gamma5 shapes then also store A^+ phat = gamma5 A p
    }
    CK(cudaMemcpyAsync(c->d_state, tmpl.data(), sizeof(SlotState) * c->kmax, cudaMemcpyHostToDevice, c->stream));
    CK(launch_matvec(c, k, variant));
    std::vector<SlotState> out(c->kmax);
    int herr = 0;
    CK(cudaMemcpyAsync(out.data(), c->d_state, sizeof(SlotState) * c->kmax, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&herr, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    for (int s = 0; s < k; ++s) {
        lqcd_status r = download(c, c->h_ptrs[s].Ap[0], c->kprec, 1, Ap + s * fb, 0);
        if (r != LQCD_OK) return r;
        r = download(c, c->h_ptrs[s].Ahp[0], c->kprec, 1, Ahp + s * fb, 0);
        if (r != LQCD_OK) return r;
    }
    for (int s = 0; s < c->kmax; ++s) { tmpl[s].status = ST_IDLE; }
    CK(cudaMemcpyAsync(c->d_state, tmpl.data(), sizeof(SlotState) * c->kmax, cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (herr) {
        CK(cudaMemset(c->d_err, 0, sizeof(int)));
        CK(cudaMemset(c->counters, 0, (size_t)c->kmax * CNT_COUNT * sizeof(unsigned)));
        return LQCD_ERR_TIMEOUT;
    }
    if (sigma)
        for (int s = 0; s < k; ++s) { sigma[2 * s] = out[s].sigma.x; sigma[2 * s + 1] = out[s].sigma.y; }
    return LQCD_OK;
}

// ============================================================ serving session
namespace {

// One BiCG run in slot s from the x_hi and b already there: deflation of the
// initial guess (phases 1 and 2 of Alg. Incremental eigBiCG), initial residual
// and start vectors, with tolerance tol. windowed: eigBiCG window on;
// rec_stop: the eigBiCG leg of a mixed-precision solve (no reliable updates,
// stop at the recursive convergence candidate); precise: FP64 residuals for
// the deflation and the start (a leg that continues from an earlier iterate).
lqcd_status begin_slot(lqcd_ctx* c, int s, lqcd_mode md, double tol, bool windowed, bool rec_stop, bool precise,
                       int maxiter, bool stab = false, bool first = false) {
    if (md != LQCD_MODE_PLAIN && c->n_def > 0) {
        lqcd_status r = deflate_range(c, s, 1, precise, first);
        if (r != LQCD_OK) return r;
    }
    SlotState& st = c->h_state[s];
    memset(&st, 0, sizeof(SlotState));
    st.status = ST_RUNNING;
    st.tol = tol;
    st.maxiter = maxiter;
    st.delta = c->kprec && !rec_stop ? c->p.delta : 0.0;
    st.rec_stop = rec_stop ? 1 : 0;
    st.m = windowed ? c->m : 0;
    st.nev = c->nev;
    st.g5 = c->p.gamma5;
    st.stab = stab && !windowed ? 1 : 0;
    CK(cudaMemcpyAsync(c->d_state + s, &st, sizeof(SlotState), cudaMemcpyHostToDevice, c->stream));
    lqcd_status r = residual_fields(c, 1, c->x_hi_all + (size_t)s * c->N, c->rt_all + (size_t)s * c->N,
                                    c->b_all + (size_t)s * c->N, precise);
    if (r != LQCD_OK) return r;
    CK(launch_bicg_start(c->g, c->links64, c->p.kappa, c->kprec, c->d_state + s, c->d_ptrs + s, 1, c->N, c->stream));
    return LQCD_OK;
}

// Start request req in free slot s. A deflated request with deftol > tol first
// runs to deftol, is deflated again and then runs to tol (the DefTol restart),
// exactly as lqcd_solve does.
lqcd_status admit(lqcd_ctx* c, int s, const lqcd_ctx::Request& req, lqcd_mode md) {
    Range nvtx_("admit request");
    lqcd_ctx::SlotJob& job = c->jobs[s];
    lqcd_status r = load_sources(c, s, 1, req.b, req.x, req.on_device);
    if (r != LQCD_OK) return r;
    const bool two_legs = md == LQCD_MODE_DEFLATED && c->p.deftol > c->p.tol && c->n_def > 0;
    const bool windowed = md == LQCD_MODE_EIGBICG;
    const bool eig_legs = windowed && c->kprec;   // mixed eigBiCG: window leg, then correction leg
    r = begin_slot(c, s, md, two_legs ? c->p.deftol : c->p.tol, windowed, eig_legs, false, c->p.maxiter,
                   c->p.bicgstab != 0, true);
    if (r != LQCD_OK) return r;
    job.busy = true;
    job.req = req;
    job.md = md;
    job.windowed = windowed;
    job.deftol_pending = two_legs;
    job.correction_pending = eig_legs;
    job.first_iters = job.first_matvecs = job.first_ru = job.first_restarts = job.outer = 0;
    job.t0 = std::chrono::steady_clock::now();
    if (job.windowed) c->eig_inflight += 1;
    return LQCD_OK;
}

// Slot s has stopped iterating: final FP64 residual; then either the second
// leg of the DefTol restart, or eigenspace growth for an eigBiCG request and
// the solution back to the caller's buffer.
lqcd_status retire(lqcd_ctx* c, int s) {
    Range nvtx_("retire request");
    lqcd_ctx::SlotJob& job = c->jobs[s];
    CK(launch_bicg_finish(c->g, c->links64, c->p.kappa, c->kprec, c->d_state + s, c->d_ptrs + s, 1, c->N, c->stream,
                          c->ru_variant, c->eo ? 1 : 0));
    CK(cudaMemcpyAsync(c->h_state + s, c->d_state + s, sizeof(SlotState), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (job.deftol_pending) {
        const SlotState& f = c->h_state[s];
        job.first_iters = f.iter;
        job.first_matvecs = f.matvecs;
        job.first_ru = f.ru_count;
        job.outer = 1;
        job.deftol_pending = false;
        return begin_slot(c, s, job.md, c->p.tol, false, false, c->kprec != 0, c->p.maxiter, c->p.bicgstab != 0);
    }
    if (job.windowed) {
        lqcd_status r = grow_slot(c, s);
        if (r != LQCD_OK) return r;
        c->last_window_valid = 1;
        c->eig_inflight -= 1;
        job.windowed = false;
        r = detach_window(c, s);   // its memory is free for the next eigBiCG request
        if (r != LQCD_OK) return r;
    }
    if (job.correction_pending) {
        // mixed eigBiCG: the window leg stopped at the recursive tolerance; the
        // deflated correction leg (FP64 residual, reliable updates) finishes it
        const SlotState f = c->h_state[s];
        job.correction_pending = false;
        if (f.status == ST_CONVERGED && f.iter < c->p.maxiter) {
            job.first_iters = f.iter;
            job.first_matvecs = f.matvecs;
            job.first_ru = f.ru_count;
            job.first_restarts = f.restarts;
            job.outer = 1;
            return begin_slot(c, s, LQCD_MODE_DEFLATED, c->p.tol, false, false, true, c->p.maxiter - f.iter);
        }
    }
    double full_resid = -1.0;
    lqcd_status r = store_solutions(c, s, 1, job.req.x, job.req.on_device, c->eo ? &full_resid : nullptr);
    if (r != LQCD_OK) return r;
    CK(cudaStreamSynchronize(c->stream));
    SlotState& st = c->h_state[s];
    if (full_resid >= 0.0) st.true_rnorm = full_resid * st.bnorm;   // the full system's certificate
    lqcd_ctx::Finished f;
    memset(&f.info, 0, sizeof(f.info));
    f.info.iters = st.iter + job.first_iters;
    f.info.matvecs = st.matvecs + job.first_matvecs;
    f.info.restarts = st.restarts + job.first_restarts;
    f.info.reliable_updates = st.ru_count + job.first_ru;
    f.info.outer_steps = job.outer;
    f.info.true_resid = st.bnorm > 0 ? st.true_rnorm / st.bnorm : 0.0;
    f.info.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - job.t0).count();
    f.info.mode_used = job.md;
    f.status = status_of(st);
    if (f.status == LQCD_OK && st.bnorm > 0 && st.true_rnorm > c->p.tol * st.bnorm) f.status = LQCD_ERR_NOCONV;
    c->finished[job.req.ticket] = f;
    job.busy = false;
    c->h_state[s].status = ST_IDLE;
    return LQCD_OK;
}

}  // namespace

extern "C" lqcd_status lqcd_submit(lqcd_ctx* c, const double* b, double* x, int on_device, lqcd_mode mode,
                                   long long* ticket) {
    if (!c || !b || !x || !ticket) return LQCD_ERR_ARG;
    if (mode < LQCD_MODE_AUTO || mode > LQCD_MODE_PLAIN) return LQCD_ERR_ARG;
    {
        lqcd_status s = check_buffers(c, b, x, on_device ? 1 : 0, "lqcd_submit");
        if (s != LQCD_OK) return s;
    }
    lqcd_ctx::Request r;
    r.ticket = c->next_ticket++;
    r.b = b;
    r.x = x;
    r.on_device = on_device ? 1 : 0;
    r.mode = mode;
    c->queue.push_back(r);
    *ticket = r.ticket;
    return LQCD_OK;
}

extern "C" lqcd_status lqcd_progress(lqcd_ctx* c, int wait, int* pending) {
    Range nvtx_("lqcd_progress");
    if (!c) return LQCD_ERR_ARG;
    if (!wait && c->chunk_inflight) {
        cudaError_t q = cudaEventQuery(c->chunk_ev);
        if (q == cudaErrorNotReady) {
            if (pending) {
                int busy = 0;
                for (int s = 0; s < c->kmax; ++s) busy += c->jobs[s].busy ? 1 : 0;
                *pending = busy + (int)c->queue.size();
            }
            return LQCD_OK;
        }
        if (q != cudaSuccess) { set_error("cudaEventQuery", q); return LQCD_ERR_CUDA; }
    }
    // 1. wait for the chunk in flight and read every slot's status
    int herr = 0;
    CK(cudaMemcpyAsync(c->h_state, c->d_state, sizeof(SlotState) * c->kmax, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&herr, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->chunk_inflight = false;
    if (herr) {
        CK(cudaMemsetAsync(c->counters, 0, (size_t)c->kmax * CNT_COUNT * sizeof(unsigned), c->stream));
        CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
        CK(cudaStreamSynchronize(c->stream));
        g_last_error = "operator kernel: bounded wait on a TMA copy timed out";
        return LQCD_ERR_TIMEOUT;
    }
    // 2. retire slots that stopped iterating
    for (int s = 0; s < c->kmax; ++s)
        if (c->jobs[s].busy && c->h_state[s].status != ST_RUNNING) {
            lqcd_status r = retire(c, s);
            if (r != LQCD_OK) return r;
        }
    // 3. admit queued requests into free slots, in arrival order, by device memory:
    // an eigBiCG request needs a window (attach_window); one that does not fit now
    // waits for memory to free up while later requests that need no window pass it.
    // If no window is held (nothing will free), AUTO requests run deflated and
    // explicit eigBiCG requests finish with LQCD_ERR_OOM.
    for (int s = 0; s < c->kbatch && !c->queue.empty(); ++s) {
        if (c->jobs[s].busy) continue;
        for (auto it = c->queue.begin(); it != c->queue.end(); ++it) {
            lqcd_mode md = it->mode;
            if (md == LQCD_MODE_AUTO)
                md = c->eig_rhs_done + c->eig_inflight < c->p.n1 ? LQCD_MODE_EIGBICG : LQCD_MODE_DEFLATED;
            if (md == LQCD_MODE_EIGBICG) {
                bool ok = false;
                lqcd_status r = attach_window(c, s, &ok);
                if (r != LQCD_OK) return r;
                if (!ok) {
                    if (c->win_attached > 0) continue;   // wait for a window to be freed
                    if (it->mode == LQCD_MODE_AUTO) {
                        md = LQCD_MODE_DEFLATED;
                    } else {
                        lqcd_ctx::Finished f;
                        memset(&f.info, 0, sizeof(f.info));
                        f.info.mode_used = LQCD_MODE_EIGBICG;
                        f.status = LQCD_ERR_OOM;
                        c->finished[it->ticket] = f;
                        c->queue.erase(it);
                        --s;   // the slot is still free
                        break;
                    }
                }
            }
            const lqcd_ctx::Request req = *it;
            c->queue.erase(it);
            lqcd_status r = admit(c, s, req, md);
            if (r != LQCD_OK) return r;
            break;
        }
    }
    // 4. next chunk of iterations for every busy slot (asynchronous)
    int busy = 0, kinds = 0;
    for (int s = 0; s < c->kmax; ++s)
        if (c->jobs[s].busy) {
            ++busy;
            kinds |= c->h_state[s].stab ? CH_STAB : (c->jobs[s].windowed ? CH_BICG | CH_WINDOW : CH_BICG);
        }
    if (busy) {
        lqcd_status r = run_chunk(c, c->kmax, kinds);
        if (r != LQCD_OK) return r;
        if (!c->chunk_ev) CK(cudaEventCreateWithFlags(&c->chunk_ev, cudaEventDisableTiming));
        CK(cudaEventRecord(c->chunk_ev, c->stream));
        c->chunk_inflight = true;
    }
    if (pending) *pending = busy + (int)c->queue.size();
    return LQCD_OK;
}

extern "C" lqcd_status lqcd_poll(lqcd_ctx* c, long long ticket, int* done, lqcd_solve_info* info,
                                 lqcd_status* result) {
    if (!c || !done) return LQCD_ERR_ARG;
    auto it = c->finished.find(ticket);
    if (it == c->finished.end()) {
        *done = 0;
        return ticket > 0 && ticket < c->next_ticket ? LQCD_OK : LQCD_ERR_ARG;
    }
    *done = 1;
    if (info) *info = it->second.info;
    if (result) *result = it->second.status;
    c->finished.erase(it);
    return LQCD_OK;
}

// ============================================================ bounded waits
namespace {
__device__ int g_flag_status;   // status word of lqcd_wait_flag
}

extern "C" lqcd_status lqcd_set_wait_limit(long long cycles) {
    CK(set_wait_cycles_tc(cycles));
    CK(set_wait_cycles_tiled(cycles));
    return LQCD_OK;
}

extern "C" lqcd_status lqcd_wait_flag(const int* flag, void* cuda_stream) {
    if (!flag) return LQCD_ERR_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    void* p = nullptr;
    CK(cudaGetSymbolAddress(&p, g_flag_status));
    int* status = reinterpret_cast<int*>(p);
    CK(cudaMemsetAsync(status, 0, sizeof(int), st));
    CK(launch_flag_wait(flag, status, st));
    int h = 0;
    CK(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (h) {
        g_last_error = "lqcd_wait_flag: the bounded wait gave up";
        return LQCD_ERR_TIMEOUT;
    }
    return LQCD_OK;
}
