// Per-slot solver state kept in device memory, and the kernel launchers
// shared between translation units.
//
// One "slot" is one right-hand side in flight. All BiCG scalars live on the
// device; every iteration kernel reads them, so the host only launches a fixed
// kernel sequence and polls the status words between chunks of iterations.
#pragma once
#include "common.cuh"

namespace lqcd {

enum SlotStatus : int { ST_RUNNING = 0, ST_CONVERGED = 1, ST_BREAKDOWN = 2, ST_NOCONV = 3, ST_IDLE = 4 };

struct SlotState {
    double2 rho;          // rho_{j-1} = (rhat_{j-1}, r_{j-1})
    double2 rho_new;      // rho_j
    double2 sigma;        // sigma_{j-1} = (phat_{j-1}, A p_{j-1})
    double2 alpha, beta;  // alpha_{j-1}, beta_{j-1}
    double2 alpha_prev, beta_prev;   // alpha_{j-2}, beta_{j-2}
    double rnorm;         // ||r_{j-1}||
    double rnorm_new;     // ||r_j||
    double bnorm;
    double rmax;          // largest ||r|| since the last reliable update
    double r_ru;          // ||r|| at the last reliable update (or the start)
    double true_rnorm;    // last FP64 ||b - A x||
    double tol;           // relative tolerance
    double delta;         // reliable-update factor (0: only at convergence)
    double phat_norm, ap_norm, rhat_norm;   // scales for the breakdown tests
    int iter;             // completed iterations
    int maxiter;
    int vs;               // vectors in the window (eigBiCG)
    int m, nev;           // window size (0 = plain BiCG), Ritz pairs
    int status;           // SlotStatus
    int need_ru;          // 1: recompute the FP64 residual in this iteration
    int ru_count;
    int restarts;
    int restart_r;        // vectors kept by the restart in this iteration (0 = none)
    int matvecs;
    int live;             // 1 while the slot takes part in the current iteration
    int x_owed;           // 1: x_lo has not yet received alpha p of the last residual update
    int x_dir;            // 1: the direction update adds alpha p to x_lo in this iteration
    int rec_stop;         // 1: stop at the first recursive convergence candidate, without
                          // replacing r (the eigBiCG leg of a mixed-precision solve)
    int g5;               // 1: gamma5-Hermitian variant (Sec. 4): rhat = gamma5 r, phat = gamma5 p,
                          // A^+ phat = gamma5 A p; one operator product per iteration
    int stab;             // 1: BiCGStab iteration (phase-2 solver of Alg. Incremental eigBiCG)
    double2 omega;        // BiCGStab: omega_j of the minimal-residual step
    double2 ts;           // BiCGStab: (t, s) of the current step
    double tt;            // BiCGStab: (t, t)
};

// Device pointers of one slot. Krylov vectors are in the precision of the
// solve (FP32 for MIXED, FP64 for FP64); x_hi, b, r_true are FP64.
struct SlotPtrs {
    void* x_lo;            // accumulated alpha p since the last reliable update
    double2* x_hi;         // FP64 solution
    const double2* b;      // FP64 source
    double2* r_true;       // FP64 scratch for b - A x
    float4* x_df;          // x_hi as double-float pairs (mixed precision; written by the reliable-update fold)
    void* V;               // residual window: (m+1) fields (windowed) or 1 field
    void* W;               // shadow residual window, same shape
    void* p;
    void* phat;
    void* Ap[2];           // A p of this and the previous iteration
    void* Ahp[2];
    double2* H;            // m x m projection matrix, row-major
    double* vscale;        // v_i = vscale[i] * V slot i
    double2* wscale;       // w_i = wscale[i] * W slot i
    double2* coefY;        // restart coefficients, (m+1) x (2nev+1), row-major
    double2* coefZ;
    double2* lam;          // restart eigenvalues (2nev)
    double2* partials;     // per-block reduction scratch of this slot
    unsigned* counters;    // last-block counters of this slot (one per kernel kind)
    void* eo_t;            // even-odd operator: even half fields of the two hop stages
    void* eo_th;           //   (D_eo p and (D^+)_eo phat, Krylov precision)
    double2* eo64;         //   and of the FP64 Schur residual (D_eo x_hi)
    const double* bnorm_ref;   // if set: ||b|| of the full system (the Schur system's tolerance reference)
};

enum CounterId { CNT_MATVEC = 0, CNT_UPDATE = 1, CNT_RU = 2, CNT_REPLACE = 3, CNT_START = 4,
                 CNT_GEMM_V = 5, CNT_GEMM_W = 6, CNT_GROUP = 7, CNT_COUNT = 8 };

// Slot of the current residual r_{j-1} at the start of an iteration.
__device__ __forceinline__ int cur_slot(const SlotState& st) { return st.m > 0 ? st.vs : 0; }
// Slot the update writes r_j into.
__device__ __forceinline__ int next_slot(const SlotState& st) { return st.m > 0 ? st.vs + 1 : 0; }

__device__ __forceinline__ bool running(const SlotState& st) { return st.status == ST_RUNNING; }

template <typename S> __device__ __forceinline__ void* slot_field(void* base, int i, size_t N) {
    return reinterpret_cast<char*>(base) + (size_t)i * N * sizeof(cplx<S>);
}

}  // namespace lqcd
