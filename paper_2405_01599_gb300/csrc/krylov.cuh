// Device-side state of the Krylov solvers (internal).
#pragma once
#include "common.cuh"

namespace xb {

// GMRES(m) state in device memory, M = restart-length capacity.
//   H: column-major (M+1) x M Hessenberg (column j at H + j*(M+1))
//   cs, sn: Givens rotations; g: rotated right-hand side (M+1)
//   sc: 1/||w|| of each stored (unnormalised) basis vector (M+1)
//   scf: the same scales in FP32 (for the FP32 basis)
//   y: least-squares solution times the basis scales (M)
//   coef: pending update coefficients of the block Gram-Schmidt passes (M+1)
//   misc: named scalars (below)
struct GmDev {
    double *H, *cs, *sn, *g, *sc, *y, *coef, *misc;
    float *scf;
    int M;
};
enum GmMisc {
    GM_BNORM = 0,   // ||b|| (relative-residual denominator)
    GM_RES = 1,     // |g_{k+1}| / ||b||
    GM_COEF = 2,    // MGS coefficient for the pending axpy
    GM_LEN2 = 3,    // sum_i h_ij^2 of the current column
    GM_K = 4,       // Arnoldi steps completed in this cycle
    GM_STOP = 5,    // 0 running, 1 converged/happy breakdown, 2 singular
    GM_TAU = 6,     // implicit threshold (relative)
    GM_BETA = 7,    // ||r0|| of the cycle
    GM_RAW = 8,     // 1: plain MGS sweep, keep column j unrotated (no Givens)
    GM_NMISC = 9
};
inline size_t gm_doubles(int M) { return (size_t)(M + 1) * M + 2 * (size_t)M + 3 * (size_t)(M + 1) + M + GM_NMISC + (M + 2) / 2 + 8; }
GmDev gm_layout(double *base, int M);

// BiCGStab scalars (indices into a device double array).
enum BiScal {
    BI_RHO = 0, BI_RHO_OLD, BI_ALPHA, BI_OMEGA, BI_SNORM2, BI_RNORM2, BI_FLAG, BI_TAU2, BI_N
};

// ---- launchers (krylov.cu) ----
int gm_cycle_init(xb_plan *p, GmDev st, int64_t n, const double *r0, double tau, cudaStream_t s);
// MGS sweep of Arnoldi step j against basis rows V_0..V_j (row stride ld);
// w holds A v_j on entry and the orthogonalised vector on exit.
template <typename VB>
int gm_mgs_step(xb_plan *p, GmDev st, int64_t n, const VB *V, int64_t ld, VB *w, int j,
                cudaStream_t s);
// Orthogonalisation of Arnoldi step j with XB_ORTHO_MGS / CGS / DGKS / BCGS
// (the policy value is resolved by the caller); ends with h_{j+1,j} and the
// Givens update like gm_mgs_step.
template <typename VB>
int gm_ortho_step(xb_plan *p, GmDev st, int64_t n, const VB *V, int64_t ld, VB *w, int j,
                  int ortho, cudaStream_t s);
// Algorithmic vector passes (multiples of n elements read + written) of one
// orthogonalisation of step j.
double ortho_passes(int ortho, int j);
// The accuracy policy of Sec. 3.3.2: MGS for tol <= 1e-10, else BCGS; DGKS
// once a fault convergence was seen.  Non-AUTO values pass through.
int ortho_choice(int ortho, double tol, bool faulted);
template <typename VB, typename VX>
int gm_update(xb_plan *p, GmDev st, int64_t n, const VB *V, int64_t ld, int k, VX *x,
              cudaStream_t s);
int gm_cycle_init_f32(xb_plan *p, GmDev st, int64_t n, const float *r0, double tau,
                      cudaStream_t s);

int bi_init(xb_plan *p, double *scal, int64_t n, const double *r, double tau2, cudaStream_t s);
int bi_p_update(double *scal, int64_t n, const double *r, double *pv, const double *v,
                cudaStream_t s);
int bi_sigma(xb_plan *p, double *scal, int64_t n, const double *rh, const double *v,
             cudaStream_t s);
int bi_s_update(xb_plan *p, double *scal, int64_t n, const double *r, const double *v, double *sv,
                cudaStream_t s);
int bi_omega(xb_plan *p, double *scal, int64_t n, const double *t, const double *sv,
             cudaStream_t s);
int bi_xr_update(xb_plan *p, double *scal, int64_t n, double *x, const double *pv,
                 const double *sv, const double *sx, const double *t, double *r, const double *rh,
                 cudaStream_t s);
int residual(xb_plan *p, const double *b, const double *x, double *r, cudaStream_t s);
int cast_f64_to_f32_scaled(int64_t n, const double *a, const double *scale_dev, float *b,
                           cudaStream_t s);
int add_scaled_f32(int64_t n, double *x, const double *scale_dev, const float *d, cudaStream_t s);

// SpMV with alpha read from device memory (beta = 0).
int spmv_launch_dalpha(xb_plan *p, int variant, int block, int ipt, const double *alpha_dev,
                       const double *x, double *y, cudaStream_t s);
int spmv_launch_dalpha_f32(xb_plan *p, int variant, int block, int ipt, const float *alpha_dev,
                           const float *x, float *y, cudaStream_t s);

}  // namespace xb
