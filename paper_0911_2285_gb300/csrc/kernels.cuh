// Host-side declarations of the kernel launchers (implemented in kernels.cu,
// eig.cu). Every launcher enqueues on the given stream and returns the launch
// error (cudaSuccess on success).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "solver.cuh"

namespace lqcd {

// Process-wide count of kernels launched by this library (graph replays add
// their node count). Used by the benchmark to report its launch count.
void count_launches(long long n);
long long launches_so_far();
void set_launches(long long n);

constexpr int PARTIAL_STRIDE = 16384;  // double2 per counter kind per slot
constexpr int MAX_SLOTS = 8;
constexpr int MAX_M = 64;              // window size limit
constexpr int MAX_SMALL = 80;          // largest dense eigenproblem / eigenspace

// Even-odd operator, host-driven applies in two stages (evenodd.cu):
// stage 1 out = D hop_in (even sites), stage 2 out = self - k^2 D hop_in (odd
// sites) or aux - (self - k^2 D hop_in) (FP64 aux).
struct EoJob {
    const void* hop_in;
    const void* self;
    void* out;
    const void* aux;
    int dagger;
};

struct ApplyJob {            // out = A in, A^+ in, or aux - A in
    const void* in;
    void* out;
    const void* aux;         // FP64 b for the residual form
    int dagger;
};

// precision: 0 = FP64 storage/arith (FP64 links), 1 = FP32 storage/arith (FP32 links)
cudaError_t launch_apply(const Geom& g, const void* links, double kappa, int precision,
                         const ApplyJob* d_jobs, int njobs, int residual, cudaStream_t st);

// r = b - A x (FP64 fields) with the hop in FP32 on FP32 links; jobs: in = x, aux = b, out = r.
cudaError_t launch_residual32(const Geom& g, const void* links32, double kappa, const ApplyJob* d_jobs, int njobs,
                              cudaStream_t st);

// Host AoS complex128 [site][12] <-> device layout in storage precision.
cudaError_t launch_pack(const double* aos, void* dev, int V, int k, int precision, cudaStream_t st);
cudaError_t launch_unpack(const void* dev, double* aos, int V, int k, int precision, cudaStream_t st);
// FP64 layout -> storage precision (element-wise), k fields.
cudaError_t launch_convert(const void* src, int src_prec, void* dst, int dst_prec, size_t n_elems, cudaStream_t st);

// C[i*ldc + j] (+)= sum_e conj(X_i(e)) Y_j(e), i < a, j < b; X, Y fields of N complex.
// conj_store: store conj(C) transposed, C[j*ldc + i] instead.
cudaError_t launch_multidot(int a, const void* X, int xprec, int b, const void* Y, int yprec,
                            size_t N, double2* C, int ldc, int conj_store, double2* scratch,
                            size_t scratch_elems, cudaStream_t st, int* err = nullptr, int tensor_cores = 1);
// tensor_cores = 1: FP32 x FP32 products go to the tensor-core path where the shape allows.
// Tensor-core form of launch_multidot for FP32 X and Y (gemm_tc.cu): 3xTF32
// tcgen05 MMAs, split-K over the SMs, partials summed in FP64. Fields of X
// (resp. Y) are x_stride (y_stride) bytes apart. scratch: dots_tc_scratch_doubles(a)
// doubles. err: device word set to 1 if a bounded wait gave up.
bool dots_tc_supported(int a, const void* X, const void* Y, size_t N);
// Tensor-core form of the FP32 restart window product (gemm_tc.cu), same
// contract as launch_window_gemm; supported for m <= 64, 2 nev <= 24, N % 128 == 0.
bool restart_tc_supported(int m, int two_nev, size_t N);
cudaError_t launch_restart_tc(SlotState* states, const SlotPtrs* ptrs, int nslots, size_t N, int* err,
                              cudaStream_t st);
size_t dots_tc_scratch_doubles(int a);
cudaError_t prepare_dots_tc();
cudaError_t launch_dots_tc(int a, const void* X, size_t x_stride, int b, const void* Y, size_t y_stride, size_t N,
                           double2* C, int ldc, int conj_store, double* scratch, size_t scratch_doubles, int* err,
                           cudaStream_t st);
// overwrite = 0: Y_j += sum_i X_i D[i*ldd + j];  overwrite = 1: Y_j = sum_i X_i D[i*ldd + j].
// The arithmetic is FP32 when X is FP32 (the sum is added to an FP64 Y in FP64),
// unless fp64_arith is set and Y is FP64 (coefficients with large, cancelling
// entries, e.g. eigenvectors in a nearly dependent basis).
cudaError_t launch_vupdate(int a, const void* X, int xprec, const double2* D, int ldd, int b,
                           void* Y, int yprec, int overwrite, size_t N, cudaStream_t st, int fp64_arith = 0);
// out[j] = ||Y_j|| (FP64 result, device) for b fields.
cudaError_t launch_norms(int b, const void* Y, int yprec, size_t N, double* out, double2* scratch,
                         size_t scratch_elems, cudaStream_t st);
// Y_j *= sc[j] for b fields (sc on the device).
cudaError_t launch_scale_fields(int b, void* Y, int yprec, const double2* sc, size_t N, cudaStream_t st);

// BiCG iteration kernels over nslots slots (see kernels.cu for the contract).
cudaError_t launch_bicg_start(const Geom& g, const void* links, double kappa, int prec,
                              SlotState* st_, const SlotPtrs* ptrs, int nslots, size_t N, cudaStream_t s);
// Plane-streaming operator pair (dslash_tiled.cu): YB rows per CTA tile, nyb
// tiles along y, t segments of tseg planes (nseg of them), nslots batch slots.
struct TileGeom {
    int YB, nyb, tseg, nseg, nslots;
};
// Plan a tiling for this lattice and batch; false if the lattice does not tile.
bool tiled_plan(const Geom& g, int nslots, TileGeom* tg);
size_t tiled_smem_bytes(int Lx, int YB);
cudaError_t prepare_tiled_kernel();
// err: device word set to 1 if a bounded wait timed out.
cudaError_t launch_matvec_tiled(const Geom& g, const TileGeom& tg, const void* links32, double kappa,
                                SlotState* states, const SlotPtrs* ptrs, int* err, cudaStream_t s);

// variant: operator-kernel shape chosen by the autotuner (0 .. matvec_variants()-1)
int matvec_variants();
// false when shape v cannot run on this lattice (brick shapes need Lx, Ly % 8 == 0, Lz % BZ == 0)
bool matvec_variant_ok(const Geom& g, int v);
// Tiled tensor map (FP32 elements, no swizzle, rank <= 5) into the 128-byte
// CUtensorMap at map; dims innermost first, strides in bytes (rank - 1 of them).
bool encode_tensor_map_f32(void* map, const void* base, int rank, const uint64_t* dims, const uint64_t* strides,
                           const uint32_t* box);
// Operator pair with links and spinor tiles staged in shared memory by TMA
// (dslash_staged.cu; FP32; shape 26). The Krylov fields of all k_max slots lie
// in one allocation krylov_base (slot s at 6 s fields); prepare_staged encodes
// the tensor maps into maps_out (staged_maps_bytes(), 64-byte aligned).
bool staged_variant_ok(const Geom& g);
size_t staged_maps_bytes();
cudaError_t prepare_staged(const Geom& g, const void* krylov_base, int kmax, const void* links32, void* maps_out);
cudaError_t launch_matvec_staged(const Geom& g, const void* maps, double kappa, SlotState* states,
                                 const SlotPtrs* ptrs, int nslots, int* err, int nsm, cudaStream_t s);
constexpr int STAGED_VARIANT = 26;
// Operator pair on 4-D bricks of 256 sites with every slot of the batch in one
// block (dslash_brick.cu; FP32; variants 25, 27, 28, 29 of launch_bicg_matvec).
bool brick_variant_ok(const Geom& g, int v);
cudaError_t launch_matvec_brick(const Geom& g, const void* links, double kappa, SlotState* states,
                                const SlotPtrs* ptrs, int nslots, cudaStream_t s, int variant);
cudaError_t launch_bicg_matvec(const Geom& g, const void* links, double kappa, int prec,
                               SlotState* st_, const SlotPtrs* ptrs, int nslots, cudaStream_t s, int variant);
// gamma5 variant (Sec. 4): A p only, phat = gamma5 p; shapes v with matvec_g5_variant_ok.
bool matvec_g5_variant_ok(const Geom& g, int v);
cudaError_t launch_bicg_matvec_g5(const Geom& g, const void* links, double kappa, int prec,
                                  SlotState* st_, const SlotPtrs* ptrs, int nslots, cudaStream_t s, int variant);
cudaError_t launch_bicg_update(int prec, SlotState* st_, const SlotPtrs* ptrs, int nslots, size_t N, cudaStream_t s);
// ru_variant: true-residual kernel shape (0 .. true_resid_variants()-1, timed at init);
// RU_DF and RU_DF + 1 evaluate A x_hi in double-float arithmetic (needs links_df
// and the slots' x_df); the final residual of launch_bicg_finish is always native FP64.
constexpr int RU_DF = 4;
int true_resid_variants();
// eo: the even-odd Schur residual (FP64) instead of the full-lattice one.
cudaError_t launch_bicg_ru(const Geom& g, const void* links64, double kappa, int prec,
                           SlotState* st_, const SlotPtrs* ptrs, int nslots, size_t N, cudaStream_t s,
                           int ru_variant = 0, const float4* links_df = nullptr, int eo = 0);
// FP64 links -> double-float links (n complex elements).
cudaError_t launch_links_df(const double2* l64, float4* ldf, size_t n, cudaStream_t st);
cudaError_t launch_bicg_scalars(SlotState* st_, const SlotPtrs* ptrs, int nslots, cudaStream_t s);
// BiCGStab step over the slots with stab set (direction, v = A p with alpha, s,
// t = A s with omega, x and r update with rho and the reliable-update flags),
// then (after launch_bicg_ru) the scalars: beta, counters, maxiter, breakdown.
cudaError_t launch_stab_step(const Geom& g, const void* links, double kappa, int prec, SlotState* st_,
                             const SlotPtrs* ptrs, int nslots, size_t N, cudaStream_t s);
cudaError_t launch_stab_scalars(SlotState* st_, int nslots, cudaStream_t s);
cudaError_t launch_bicg_direction(int prec, SlotState* st_, const SlotPtrs* ptrs, int nslots, size_t N, cudaStream_t s);
cudaError_t launch_bicg_finish(const Geom& g, const void* links64, double kappa, int prec,
                               SlotState* st_, const SlotPtrs* ptrs, int nslots, size_t N, cudaStream_t s,
                               int ru_variant = 0, int eo = 0);

// eigBiCG restart: coefficient kernel (one CTA per slot) and window product.
// Work buffers: eig_work_elems() double2 per slot (restart; the buffer holds MAX_SLOTS
// slot areas plus 16 double2 for status words) or per call (the others).
size_t eig_work_elems();
// Opt the eigen kernels into large dynamic shared memory (call once, outside graph capture).
cudaError_t prepare_eig_kernels();
cudaError_t launch_restart_coeffs(SlotState* st_, const SlotPtrs* ptrs, int nslots, double2* work, cudaStream_t s);
cudaError_t launch_window_gemm(int prec, int two_nev, SlotState* st_, const SlotPtrs* ptrs, int nslots, size_t N,
                               cudaStream_t s);

// Small dense FP64 algebra on the device (one CTA).
// eig of an n x n row-major matrix; Y, Z (n x nsel row-major columns) for the
// nsel smallest-|lambda| eigenvalues; lam gets all n eigenvalues (sorted).
cudaError_t launch_small_eig(int n, const double2* A, int lda, int nsel, double2* lam,
                             double2* Y, double2* Z, int ldyz, int* info, double2* work, cudaStream_t st);
cudaError_t launch_restart_coeffs_single(int m, int nev, const double2* H, int* r, double2* Yc,
                                         double2* Zc, double2* lam, int* info, double2* work, cudaStream_t st);
// LU with partial pivoting of n x n (row-major, in place), piv[n]; info != 0 if singular.
cudaError_t launch_lu_factor(int n, double2* A, int lda, int* piv, int* info, cudaStream_t st);
// Solve A X = B (trans = 0) or A^H X = B (trans = 1) with the LU factors; B is n x nrhs (ldb), in place.
cudaError_t launch_lu_solve(int n, const double2* LU, int lda, const int* piv, int trans, int nrhs,
                            double2* B, int ldb, cudaStream_t st);
// One factor of P A = L U (from launch_lu_factor) applied to B:
// LU_LEFT_PL: B <- L^{-1} P B; LU_LEFT_U: B <- U^{-1} B (n x ncols);
// LU_RIGHT_U: B <- B U^{-1} (ncols rows of n); LU_LEFT_LH: B <- P^T L^{-H} B.
enum LuPart { LU_LEFT_PL = 0, LU_LEFT_U = 1, LU_RIGHT_U = 2, LU_LEFT_LH = 3 };
cudaError_t launch_lu_part(int n, const double2* LU, int lda, const int* piv, int part, int ncols, double2* B,
                           int ldb, cudaStream_t st);
// Rank-revealing selection of a small square block B (n <= 32): complete-pivoting
// LU stopped at the first pivot below tau * |first pivot|; out[0] = pivots kept r,
// out[1 + i], out[1 + n + i] = row and column index of pivot i.
cudaError_t launch_pivot_select(int n, const double2* B, int ld, double tau, int* out, cudaStream_t st);
// Final Ritz pairs of one slot's window: eig(H^(vs)), nev smallest;
// coefficients Y (vs x nev) and Z into Yc/Zc with the window scales folded in.
cudaError_t launch_final_ritz(SlotState* st_, const SlotPtrs* ptrs, int slot, double2* Yc, double2* Zc,
                              double2* lam, int* nout, double2* work, cudaStream_t st);
// The same for slots slot0 .. slot0+nslots-1 in one launch (one block each):
// slot slot0 + j writes Yc/Zc + j ostride, lam + j lstride, nout[j], and uses
// the work area work + j eig_work_elems().
cudaError_t launch_final_ritz_slots(SlotState* st_, const SlotPtrs* ptrs, int slot0, int nslots, double2* Yc,
                                    double2* Zc, double2* lam, int* nout, size_t ostride, size_t lstride,
                                    double2* work, cudaStream_t st);
// Small matrix helpers: C = A B (all row-major, n x k x m), one CTA.
cudaError_t launch_small_gemm(int n, int k, int m, const double2* A, int lda, int transA,
                              const double2* B, int ldb, double2* C, int ldc, cudaStream_t st);

// Even-odd (Schur complement) operator A_hat = 1 - k^2 D_oe D_eo on the odd half
// lattice (evenodd.cu). Half fields: V/2 sites, half index h = s >> 1.
// A_hat (A_hat^+ with job.dagger) of njobs fields: d_stage1 jobs (D_eo in -> tmp),
// d_stage2 jobs (in - k^2 D_oe tmp, or aux - that with residual).
cudaError_t launch_eo_apply(const Geom& g, const void* links, double kappa, int prec, const EoJob* d_stage1,
                            const EoJob* d_stage2, int njobs, int residual, cudaStream_t st);
// b_hat = b_o + k D_oe b_e (k full FP64 fields -> k half fields).
cudaError_t launch_eo_prepare(const Geom& g, const void* links64, double kappa, const double2* bfull, double2* bhat,
                              int k, cudaStream_t st);
// The odd half of k full FP64 fields.
cudaError_t launch_eo_extract(const Geom& g, const double2* xfull, double2* xhalf, int k, cudaStream_t st);
// Full solutions: x_o from the half fields, x_e = b_e + k D_eo x_o.
cudaError_t launch_eo_reconstruct(const Geom& g, const void* links64, double kappa, const double2* bfull,
                                  const double2* xhalf, double2* xfull, int k, cudaStream_t st);
// BiCG operator pair on A_hat over the slots (two stages through eo_t, eo_th) with sigma and alpha.
cudaError_t launch_eo_pair(const Geom& g, const void* links, double kappa, int prec, SlotState* states,
                           const SlotPtrs* ptrs, int nslots, cudaStream_t st);
// FP64 Schur residual b_hat - A_hat x_hi (through eo64): in-iteration (check_only 0) or final.
cudaError_t launch_eo_true_resid(const Geom& g, const void* links64, double kappa, SlotState* states,
                                 const SlotPtrs* ptrs, int nslots, int check_only, cudaStream_t st);

// Bound of the device-side waits (SM clock cycles) of the kernels of gemm_tc.cu
// and dslash_tiled.cu on the current device; cycles <= 0 restores the default.
cudaError_t set_wait_cycles_tc(long long cycles);
cudaError_t set_wait_cycles_tiled(long long cycles);
// One-thread kernel: bounded wait for *flag != 0; *status = 1 if it gave up.
cudaError_t launch_flag_wait(const int* flag, int* status, cudaStream_t st);

}  // namespace lqcd
