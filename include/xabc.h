/*
 * xabc.h -- C ABI of the GB300 (sm_103a) CRS SpMV + restarted Krylov library.
 *
 * The operation throughout is the paper's linear system A x = b with A in
 * compressed row storage (CRS, Sec. 4.2 of Katagiri et al., "Xabclib: A Fully
 * Auto-tuned Sparse Iterative Solver"), optionally symmetric with only the
 * upper triangle stored (Sec. 4.2).
 *
 * Conventions for every entry point
 *   - Matrix and vector pointers are DEVICE pointers owned by the caller (for
 *     example torch tensors).  The library never frees caller memory.
 *   - CRS is 0-based: rowptr[n+1], col[nnz] ascending within each row, no
 *     duplicates, val[nnz] FP64.  n and nnz are < 2^31 - 64 (int32 indices).
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *     default stream.  Work is enqueued on it in stream order; functions that
 *     must read a device result on the host (solvers, tuners) synchronise
 *     that stream.
 *   - Return value: XB_OK (0) or a negative XB_E* code.  The message of the
 *     last error on the calling host thread is returned by xb_last_error().
 *   - A plan (xb_plan) owns library workspace in device memory, created by
 *     xb_plan_create and released by xb_plan_destroy.  A plan may be used by
 *     one host thread / one stream at a time.
 */
#ifndef XABC_H
#define XABC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define XB_OK 0
#define XB_EINVAL (-1)       /* bad argument or malformed CRS                  */
#define XB_ENOMEM (-2)       /* device or host allocation failed               */
#define XB_ECUDA (-3)        /* CUDA runtime error (message: xb_last_error)    */
#define XB_ENOCONV (-4)      /* iteration/time limit hit; x holds the iterate  */
#define XB_EBREAKDOWN (-5)   /* Krylov breakdown (singular/indefinite pivot)   */
#define XB_ETIMEOUT (-6)     /* a bounded device-side wait expired            */
#define XB_EFAULT (-7)       /* fault convergence (Sec. 3.3.2): the implicit   */
                             /*   residual met tol, the true one did not, and  */
                             /*   fault_check was off; x holds the iterate     */

/* ---- SpMV implementation variants (Sec. 3.2.2: U1-U3, S1-S3) ---------- */
#define XB_VAR_AUTO (-1)     /* plan's tuned / default choice                  */
#define XB_VAR_ROW 0         /* U1: one thread per row (conventional)          */
#define XB_VAR_NNZ 1         /* U2: nnz-balanced row-aligned tiles             */
#define XB_VAR_SEGSCAN 2     /* U3: flat nnz split + segmented sum (BSS)       */
#define XB_VAR_SYM_ATOMIC 3  /* S1-like: every transpose term a global atomic  */
#define XB_VAR_SYM_TILE 4    /* S2/S3-like: nnz-balanced tiles, in-tile        */
                             /*   transpose terms in shared memory, only the   */
                             /*   out-of-tile (non-zero region) ones global    */
#define XB_VAR_SELL 5        /* format conversion (Sec. 5): SELL-C-sigma copy,  */
                             /*   C = 32 rows per slice, rows sorted by length */
                             /*   in windows of sigma = 32 * ipt rows; a thread */
                             /*   per row, coalesced slice columns; built on   */
                             /*   first use (general storage only)             */
#define XB_VAR_SYM_PART 6    /* S3: S2 tiles; transposes beyond the tile summed */
                             /*   in per-CTA partial vectors over only the     */
                             /*   256-row granules they reach, then one pass   */
                             /*   adds each reached granule's partials in tile */
                             /*   order (granules nothing reaches are skipped);*/
                             /*   no device atomics.  XB_EINVAL when a tile    */
                             /*   reaches more than 8 granules beyond itself   */
#define XB_VAR_SYM_WAGG 7    /* S1 with warp-aggregated atomics: lanes whose   */
                             /*   transpose terms target the same row add them */
                             /*   first, one device atomic per distinct row    */
#define XB_VAR_BCSR 8        /* format conversion (Sec. 5): block CRS with     */
                             /*   r x r blocks, r = ipt in {2, 3, 4}, zero-   */
                             /*   filled; a thread per row walks its block    */
                             /*   row (one column index per block, x read r   */
                             /*   at a time); built on first use, rejected    */
                             /*   when the blocks hold more than 2 nnz + 16 r */
                             /*   entries (general storage only)              */
#define XB_NUM_VARIANTS 9

/* Re-orthogonalisation in the Arnoldi step (Sec. 3.2.2) and the accuracy
 * policy choosing it (Sec. 3.3.2). */
#define XB_ORTHO_MGS 0       /* modified Gram-Schmidt (the default)            */
#define XB_ORTHO_CGS 1       /* classical Gram-Schmidt                         */
#define XB_ORTHO_DGKS 2      /* DGKS: classical Gram-Schmidt run two times     */
#define XB_ORTHO_BCGS 3      /* blocked CGS, block length 4: CGS inside a      */
                             /*   block, MGS between blocks                    */
#define XB_ORTHO_AUTO 4      /* policy: MGS if tol <= 1e-10 else BCGS; DGKS    */
                             /*   after a fault convergence                    */

#define XB_PREC_FP64 0
#define XB_PREC_MIXED 1      /* FP32 SpMV + Arnoldi basis inside FP64          */
                             /*   iterative refinement                         */

/* Numerical computation policy (Sec. 2.3.2, 3.3).  Any value but NONE sets
 * tuner, variant, m / m_max, dafrt, ortho and fault_check before the solve:
 *   TIME     fastest: exhaustive SpMV tuning, the restart rule on (m up to
 *            m_max >= 128), BCGS for tol > 1e-10 else MGS, fault_check 0;
 *   ACCURACY as TIME, but fault_check 1 and the orthogonalisation policy
 *            (DGKS after a fault convergence);
 *   MEMORY   least memory: the SpMV without plan metadata (thread per row,
 *            or atomic transposes for symmetric storage), m = 10 fixed, MGS,
 *            FP64, fault_check 0;
 *   STABLE   no auto-tuning: the plan's SpMV, m as given, MGS, no restart
 *            rule, fault_check 0. */
#define XB_POLICY_NONE 0     /* every option as given (default)               */
#define XB_POLICY_TIME 1
#define XB_POLICY_ACCURACY 2
#define XB_POLICY_MEMORY 3
#define XB_POLICY_STABLE 4

/* Preconditioner (Sec. 4.3 runs the solvers with ILU(0)). */
#define XB_PRECOND_NONE 0
#define XB_PRECOND_ILU0 1    /* incomplete LU in A's pattern, right-applied:  */
                             /*   the solvers iterate on A M^{-1} and report   */
                             /*   residuals of A x = b                         */

/* Solvers a policy file can name (SOLVER keyword, Sec. 2.3.2). */
#define XB_SOLVER_GMRES 0
#define XB_SOLVER_BICGSTAB 1
#define XB_SOLVER_LANCZOS 2
#define XB_SOLVER_ARNOLDI 3

/* Wanted end of the spectrum for the Arnoldi eigensolver. */
#define XB_EIG_LR 0          /* largest real part first                        */
#define XB_EIG_LM 1          /* largest modulus first                          */

#define XB_TUNER_NONE 0      /* fixed variant (options.variant or default)     */
#define XB_TUNER_EXHAUSTIVE 1 /* time every candidate (Sec. 3.1)              */
#define XB_TUNER_MLP 2       /* learned tuner (xb_mlp_*)                       */

typedef struct xb_csr {
    int32_t n;               /* rows = columns                                 */
    int32_t nnz;             /* stored entries                                 */
    const int32_t *rowptr;   /* device, n+1                                    */
    const int32_t *col;      /* device, nnz                                    */
    const double *val;       /* device, nnz                                    */
    int32_t sym_upper;       /* 1: symmetric, only entries with col >= row     */
} xb_csr;

typedef struct xb_options {
    double tol;              /* ||b - A x|| / ||b|| target (default 1e-8)      */
    int32_t maxiter;         /* Arnoldi steps / BiCGStab iterations cap        */
    double maxtime_s;        /* wall-clock cap, seconds (default 1000)        */
    int32_t m;               /* GMRES restart length (default 30)             */
    int32_t m_max;           /* cap for the restart rule (default 120)        */
    int32_t dafrt;           /* 1: MM-ratio restart rule on (Eq. 1, Sec. 4.3)  */
    double dafrt_theta;      /* judgement threshold (default 10)              */
    int32_t dafrt_window;    /* samples per judgement (default 5, Fig. 2)     */
    int32_t dafrt_dm;        /* restart-length increment (default 5)          */
    int32_t ortho;           /* XB_ORTHO_*                                     */
    int32_t precision;       /* XB_PREC_*                                      */
    double tol_inner;        /* inner FP32 solve tolerance (default 1e-4)     */
    int32_t maxiter_inner;   /* inner FP32 Arnoldi steps per refinement step  */
    int32_t max_outer;       /* refinement steps cap (default 60)             */
    int32_t variant;         /* XB_VAR_* for the SpMV inside solvers          */
    int32_t block;           /* CTA size for SpMV (0 = plan default)          */
    int32_t ipt;             /* items per thread (segscan / tile size; SELL:  */
                             /*   sorting window sigma = 32 * ipt rows)        */
    int32_t tuner;           /* XB_TUNER_*                                     */
    int32_t check_every;     /* host reads the residual every k steps (>=1)   */
    int32_t timing;          /* 1: record per-SpMV CUDA-event times in info   */
    int32_t policy;          /* XB_POLICY_* (numerical computation policy)     */
    int32_t fault_check;     /* 1 (default): after an implicit convergence the */
                             /*   true residual decides; a false claim narrows */
                             /*   the implicit threshold and the solve goes on */
                             /*   (Sec. 3.3.2); 0: stop at the first claim and */
                             /*   return XB_EFAULT if the true residual misses */
    int32_t precond;         /* XB_PRECOND_*: right preconditioner (FP64      */
                             /*   GMRES and BiCGStab on general CRS)           */
    int32_t ir_fallback;     /* mixed precision only.  0: plain refinement    */
                             /*   (FP64 residual, FP32 inner GMRES, x += ||r|| */
                             /*   d) until tol or max_outer.  1 (default): a   */
                             /*   library safeguard, not part of the method:   */
                             /*   when the FP64 residual fails to halve in two */
                             /*   consecutive refinement steps (FP32 cannot    */
                             /*   resolve the system: kappa * 6e-8 near 1),    */
                             /*   the solve continues as FP64 GMRES(m) from    */
                             /*   the current x and xb_info.fallback = 1       */
    int32_t small_n;         /* GMRES: systems with n <= small_n run as one  */
                             /*   persistent launch when the options allow it */
                             /*   and one of the persistent kernels takes     */
                             /*   the size (see gmres_solve); default 8192    */
                             /*   (the environment variable XB_SMALL_N        */
                             /*   changes the default), 0 = never             */
} xb_options;

typedef struct xb_info {
    int32_t status;          /* same as the return value                      */
    int32_t iters;           /* Arnoldi steps / BiCGStab iterations           */
    int32_t restarts;        /* GMRES cycles completed / BiCGStab restarts    */
    int32_t m_final;         /* restart length at exit                        */
    int32_t faults;          /* fault-convergence events (Sec. 3.3.2)         */
    int32_t outer;           /* refinement steps (mixed precision)            */
    int32_t inner_iters;     /* FP32 Arnoldi steps (mixed precision)          */
    int32_t fallback;        /* 1: mixed solve finished in FP64               */
    int32_t variant_used;    /* XB_VAR_* of the SpMV                          */
    int32_t block_used;
    int32_t ipt_used;
    int32_t spmv_calls;      /* SpMV launches in the solve                    */
    int32_t ortho_used;      /* XB_ORTHO_* in use at exit (GMRES)             */
    double res_implicit;     /* last implicit (recursive) relative residual   */
    double res_true;         /* ||b - A x|| / ||b|| at exit, FP64             */
    double t_solve_s;        /* host wall time of the solve                   */
    double spmv_ms;          /* summed CUDA-event SpMV time (opt.timing)      */
    double bytes_alg;        /* algorithmic bytes of all launches (see docs)  */
    double mem_bytes;        /* device memory the solve used: workspace it    */
                             /*   requested, the SpMV variant's plan data and */
                             /*   the FP32 matrix copy (mixed precision)      */
    int32_t persistent;      /* GMRES ran as one persistent launch (small     */
                             /*   systems, see gmres_solve): 2 = from one     */
                             /*   cluster's shared memory, 1 = the batched    */
                             /*   kernel's single-system path; 0 = neither    */
} xb_info;

typedef struct xb_plan xb_plan;

typedef struct xb_choice {
    int32_t variant, block, ipt;
    float ms;                /* best measured time (exhaustive)               */
} xb_choice;

/* ---- setup -------------------------------------------------------------- */

/* Fill *opt with the defaults listed in the struct comments (the paper's
 * OpenATI_INIT: set default parameters, Table 1). */
void xb_options_default(xb_options *opt);

/* Message of the last failing call on this host thread ("" if none). */
const char *xb_last_error(void);

/* Build a plan for A (the paper's *_Setup functions, Table 1): validates
 * sizes, copies rowptr to the host once, picks the default SpMV variant and
 * allocates the reduction scratch.  Each variant's plan data (tile
 * partitions, the segmented scan's row-end bitmask, warp start rows and data
 * format copy, the S3 granule lists, the SELL and BCSR copies) is built on the
 * variant's first use.  opt may be NULL (defaults).  The plan keeps A's
 * pointers: A's arrays must outlive the plan and stay unmodified.
 * XB_EINVAL: n < 0, nnz < 0, NULL arrays with n > 0, rowptr[0] != 0,
 * rowptr[n] != nnz or rowptr decreasing, n or nnz >= 2^31 - 64 (use
 * xb_plan_create64).  Columns are checked (0 <= col < n, ascending, and
 * col >= row when sym_upper) only when the environment variable
 * XB_VALIDATE=1 is set. */
int xb_plan_create(const xb_csr *A, const xb_options *opt, void *stream, xb_plan **out);
int xb_plan_destroy(xb_plan *plan);

/* A in CRS with 64-bit row offsets (nnz up to 2^62; n, the columns and every
 * row's length stay below 2^31 - 64).  Same rules as xb_csr otherwise. */
typedef struct xb_csr64 {
    int32_t n;
    int64_t nnz;
    const int64_t *rowptr;   /* device, n+1                                    */
    const int32_t *col;      /* device, nnz                                    */
    const double *val;       /* device, nnz                                    */
    int32_t sym_upper;
} xb_csr64;
/* Plan for A with 64-bit row offsets.  When nnz < 2^31 - 64 the plan narrows
 * rowptr to an int32 copy it owns and is an ordinary plan.  Larger matrices
 * (general storage only) are cut into consecutive row blocks of at most
 * 2^31 - 64 non-zeros each (xb_split_rows64; the environment variable
 * XB_PLAN_SPLIT_NNZ lowers the block limit, for testing); each block is
 * planned with int32 offsets into A's col/val from the block's first entry,
 * and every SpMV runs the chosen variant block by block on the whole x.  Such
 * a plan supports the general SpMV variants (ROW, NNZ, SEGSCAN, SELL, BCSR),
 * the tuner and the FP64 / mixed-precision GMRES and BiCGStab solvers; ILU(0)
 * and the symmetric storage return XB_EINVAL.  Errors as xb_plan_create, plus
 * XB_EINVAL for a row longer than the block limit. */
int xb_plan_create64(const xb_csr64 *A, const xb_options *opt, void *stream, xb_plan **out);
/* The row blocks xb_plan_create64 cuts (host logic, no device work; exposed
 * for testing): consecutive rows, each block at most max_nnz non-zeros,
 * greedily as many rows as fit.  HOST rowptr (n + 1 int64); starts receives
 * the first row of each block and then n (capacity cap entries); *nblocks the
 * block count (always set).  XB_EINVAL when a row alone has more than max_nnz
 * non-zeros, max_nnz < 1 or rowptr is not non-decreasing from 0. */
int xb_split_rows64(int32_t n, const int64_t *rowptr, int64_t max_nnz, int32_t *starts,
                    int32_t cap, int32_t *nblocks);

/* Set the SpMV variant and launch shape used by XB_VAR_AUTO calls and by the
 * solvers.  block in {64,128,256,512}; ipt in [1,32].  XB_EINVAL for a
 * variant that does not fit the storage (sym variants need sym_upper=1,
 * general variants sym_upper=0). */
int xb_plan_set_choice(xb_plan *plan, int32_t variant, int32_t block, int32_t ipt);
int xb_plan_get_choice(const xb_plan *plan, xb_choice *out);

/* ---- SpMV entry points: y = alpha*A*x + beta*y ---------------------------
 * x, y: device FP64 vectors of length n; y may not alias x.  beta == 0 means
 * y is write-only (its old contents, even NaN, are ignored).  Stream-ordered,
 * no host synchronisation. */

/* General CRS SpMV, nnz-balanced row-aligned tiles (U2 of Sec. 3.2.2; the
 * partition follows Fig. 3: rows grouped so each tile holds about the same
 * number of non-zeros; a row is never split across tiles unless it alone
 * exceeds a tile).  Deterministic.  XB_EINVAL if the plan is sym_upper. */
int spmv_crs(xb_plan *plan, double alpha, const double *x, double beta, double *y, void *stream);

/* Symmetric SpMV from upper storage: y = alpha*(U + U^T - diag U) x + beta*y
 * (S1-S3 of Sec. 3.2.2).  Uses the plan's sym variant (XB_VAR_SYM_TILE unless
 * set otherwise): transpose contributions that land inside the tile are summed
 * in shared memory, only the non-zero region outside a tile goes through
 * device atomics (so the result is not bitwise reproducible run to run; it
 * agrees to rounding).  XB_EINVAL if the plan is not sym_upper. */
int spmv_sym(xb_plan *plan, double alpha, const double *x, double beta, double *y, void *stream);

/* General CRS SpMV by the branchless segmented-scan idea (U3/BSS, Sec. 3.2.2,
 * Sec. 4.4.1.3): the non-zeros are split into equal flat segments regardless
 * of row boundaries (ipt consecutive non-zeros per thread, 32*ipt per warp);
 * the plan's "continuous location" data -- one row-end bit per non-zero and
 * the start row of each warp -- lets each thread sum its segment with row
 * breaks as predicated stores, and row sums that straddle threads or warps
 * are combined by a segmented warp scan and a deterministic carry fix-up.
 * Deterministic.  Launch shapes: block <= 256, ipt in {4, 8, 16, 32}.
 * XB_EINVAL if the plan is sym_upper. */
int spmv_segscan(xb_plan *plan, double alpha, const double *x, double beta, double *y, void *stream);

/* Allocation-free variant of spmv_segscan (the paper has no counterpart).
 * For callers that cannot allocate device memory -- their device memory is
 * owned by another allocator, or an allocation's implicit synchronisation is
 * not allowed where they call -- and therefore cannot create a plan either.
 * Takes the CRS arrays directly (device pointers, laid out as xb_csr with
 * sym_upper = 0) and computes y = alpha*A*x + beta*y with a staged per-CTA
 * segmented-scan kernel at a fixed shape of 256 threads x 8 non-zeros per
 * thread.  The arrays are NOT validated (there is no plan to do it): the
 * caller guarantees rowptr[0] = 0, rowptr non-decreasing, rowptr[n] = nnz and
 * 0 <= col < n.  The kernel only keeps its own accesses inside x and y when
 * they do not hold (an out-of-range column adds nothing, a row index past n
 * is not stored); the result is then meaningless.  x and y must not overlap
 * (XB_EINVAL).  Its scratch (16 bytes
 * per 2048 non-zeros) lives in one 4 MiB array compiled into the library,
 * which every GPU that loads the library holds until the process exits; it
 * calls no cudaMalloc/cudaFree.  Limit: nnz <= 262,142 * 2048 (about 5.4e8);
 * larger inputs return XB_EINVAL with that limit in the message.  Every call
 * looks up the array's device address on the current device
 * (cudaGetSymbolAddress; after cudaDeviceReset the next call finds the
 * reloaded array).  The first call on a device also loads the library's
 * device code there, so make that first call before any stream capture.
 * All calls share the one array: calls that overlap on the GPU (for example
 * on two streams) race and must be serialised by the caller.  Each row is
 * summed in CRS order up to the final combination of partial sums, so
 * results agree with spmv_segscan within rounding (the library's 1e-12 row
 * tolerance), not bit for bit. */
int spmv_segscan_noalloc(int32_t n, int32_t nnz, const int32_t *rowptr, const int32_t *col,
                         const double *val, double alpha, const double *x, double beta,
                         double *y, void *stream);

/* The SELL-32-sigma layout that XB_VAR_SELL builds (host logic, no device
 * work; exposed for testing): rows sorted by length, longest first and
 * stable, inside windows of sigma rows; slot q of slice q / 32 holds sorted
 * row q.  HOST arrays: rowptr (n + 1); perm (32 ceil(n / 32): the row of each
 * slot, -1 past n); slen (same length: the slot's row length); off
 * (ceil(n / 32) + 1: entry offset of each slice, a slice being 32 times its
 * longest row wide).  perm, slen, off may each be NULL; *total receives the
 * padded entry count. */
int xb_sell_layout(int32_t n, const int32_t *rowptr, int32_t sigma, int32_t *perm,
                   int32_t *slen, int64_t *off, int64_t *total);

/* The warp tiles that XB_VAR_NNZ (U2) builds for items per thread ipt (host
 * logic, no device work; exposed for testing).  Rows are cut, in order, into
 * tiles [r0, r1) whose non-zeros fit the 32*ipt-entry window starting at
 * rowptr[r0] rounded down to a multiple of ipt; a tile takes rows while they
 * fit, and stops at 32 rows while none of its rows is longer than ipt (kind 0,
 * thread per row; otherwise kind 1, flat).  A row that overflows a window on
 * its own is a long row (CTA per row).  HOST arrays: rowptr (n + 1); tiles
 * (4 int32 per tile: r0, r1, number of non-empty rows before r0, kind + 4 if
 * the tile has an empty row), filled up to cap_tiles tiles; longs, filled up
 * to cap_long rows.  *ntiles and *nlong receive the full counts.  tiles and
 * longs may be NULL (capacity 0) to query the counts. */
int xb_u2_layout(int32_t n, const int32_t *rowptr, int32_t ipt, int32_t *tiles, int32_t cap_tiles,
                 int32_t *ntiles, int32_t *longs, int32_t cap_long, int32_t *nlong);

/* The block-CRS structure that XB_VAR_BCSR builds for r x r blocks (host
 * logic, no device work; exposed for testing): block row b covers rows
 * [r b, r b + r); its blocks are the distinct col / r of those rows' entries,
 * ascending.  HOST arrays: rowptr (n + 1), col (nnz); bptr (ceil(n / r) + 1)
 * receives the block-row offsets, bcol (capacity cap) the block columns;
 * *nblocks the block count (always set).  bptr and bcol may be NULL (cap 0)
 * to query the count. */
int xb_bcsr_layout(int32_t n, const int32_t *rowptr, const int32_t *col, int32_t r, int32_t *bptr,
                   int32_t *bcol, int64_t cap, int64_t *nblocks);

/* Any variant (XB_VAR_*; XB_VAR_AUTO = plan choice) with an explicit launch
 * shape (block/ipt 0 = plan choice).  XB_VAR_SELL builds the SELL-32-sigma
 * copy of the matrix on its first use with that sigma (device memory held by
 * the plan: 12 B per stored entry including padding plus 8 B per row) and
 * returns XB_EINVAL when the padding would exceed 3 nnz + 32 per slice of 32
 * rows; results equal XB_VAR_ROW's bit for bit. */
int xb_spmv(xb_plan *plan, int32_t variant, int32_t block, int32_t ipt, double alpha,
            const double *x, double beta, double *y, void *stream);

/* FP32 SpMV on the plan's FP32 copy of A (made on first use, library-owned):
 * y32 = alpha*A32*x32 + beta*y32 with FP32 accumulation (the inner operator
 * of the mixed-precision refinement). */
int xb_spmv_f32(xb_plan *plan, int32_t variant, float alpha, const float *x, float beta,
                float *y, void *stream);

/* ---- Krylov solvers -------------------------------------------------------
 * b: device FP64 right-hand side; x: device FP64, in = initial guess,
 * out = iterate.  opt NULL = defaults.  info may be NULL.  The solve ends
 * when the TRUE residual ||b - A x|| / ||b|| <= opt->tol (checked in FP64
 * after every claimed convergence: the fault-convergence test of Sec. 3.1 and
 * 3.3.2, which narrows the implicit threshold and continues when the claim
 * was false), or with XB_ENOCONV at maxiter / maxtime_s, or XB_EBREAKDOWN.
 * b == 0 gives x = 0.  The host synchronises `stream` every
 * opt->check_every steps to read the residual. */

/* Restarted GMRES(m) (Sec. 2.2, Sec. 4.3): Arnoldi with the
 * orthogonalisation opt->ortho -- MGS, CGS, DGKS (CGS run twice) or BCGS
 * (blocks of 4), Sec. 3.2.2, or XB_ORTHO_AUTO, the accuracy policy of
 * Sec. 3.3.2 (MGS for tol <= 1e-10, else BCGS; DGKS after a fault
 * convergence) -- and Givens least squares; opt->dafrt enables the MM-ratio
 * restart rule of Eq. (1) / Fig. 2 / Sec. 4.3 (m += dafrt_dm, at most m_max).
 * opt->precond == XB_PRECOND_ILU0 preconditions on the right with ILU(0)
 * (Sec. 4.3; FP64 only, general storage).  opt->precision == XB_PREC_MIXED
 * runs FP32 GMRES(m) (FP32 SpMV and basis, FP64 Hessenberg/Givens/least
 * squares) inside FP64 iterative refinement (see opt->ir_fallback).
 * Small systems -- n <= opt->small_n (default 8192), general storage, FP64,
 * no preconditioner,
 * MGS or BCGS, m (and m_max with the restart rule, whose window and
 * increment must then be the default 5) <= XB_BATCH_MAX_M,
 * fault_check on -- run the same GMRES(m) as one persistent launch, because
 * each Arnoldi step of the multi-launch path is bound by launch and
 * synchronisation latency at that size.  When a cluster of 2, 4, 8 or 16
 * CTAs can hold the system in shared memory (at most 1024 rows per CTA, rows
 * at most 64 long, the basis slice, the ELL copy of the rows and the
 * Hessenberg matrix within the opt-in shared memory of a CTA) that cluster
 * runs it with no global-memory traffic per step (xb_info.persistent = 2;
 * the environment variable XB_RESIDENT_CL = 0 turns this off, a cluster size
 * forces it); otherwise, while nnz + m n <= 32 small_n, the batched kernel's
 * single-system path does (one 8-CTA cluster, basis in global memory;
 * xb_info.persistent = 1), and beyond that the multi-launch path.  spmv_ms
 * and res_implicit are 0 on both.  A column index outside [0, n) makes the
 * shared-memory path return XB_EINVAL without touching x. */
int gmres_solve(xb_plan *plan, const double *b, double *x, const xb_options *opt,
                xb_info *info, void *stream);

/* BiCGStab (Sec. 2.2, Sec. 4.3; van der Vorst's iteration), two SpMVs per
 * step, optionally right-preconditioned with ILU(0) (opt->precond ==
 * XB_PRECOND_ILU0: two preconditioner applications per step). */
int bicgstab_solve(xb_plan *plan, const double *b, double *x, const xb_options *opt,
                   xb_info *info, void *stream);

/* ---- Krylov vector operations (FP64, device) ------------------------------
 * Deterministic two-stage reductions; `out` is a DEVICE pointer to one
 * double.  n >= 0. */
int xb_dot(xb_plan *plan, int32_t n, const double *x, const double *y, double *out, void *stream);
int xb_axpy(int32_t n, double a, const double *x, double *y, void *stream); /* y += a x */
/* One modified Gram-Schmidt sweep (Sec. 3.2.2, MGS): for i = 0..k-1,
 * h[i] = (w, V_i); w -= h[i] V_i, with V row-major k x ld (ld >= n), then
 * h[k] = ||w||.  h: device, k+1 doubles. */
int xb_mgs(xb_plan *plan, int32_t n, int32_t k, const double *V, int64_t ld, double *w,
           double *h, void *stream);
/* Orthogonalise w against the k rows of V (row-major k x ld, ld >= n, rows
 * orthonormal) with ortho = XB_ORTHO_MGS / CGS / DGKS / BCGS (Sec. 3.2.2):
 * on return w is the orthogonalised vector, h[0..k-1] the projection
 * coefficients (for DGKS the sum of both passes) and h[k] = ||w||.
 * h: device, k+1 doubles; 1 <= k <= 512; XB_ORTHO_AUTO is rejected. */
int xb_orth(xb_plan *plan, int32_t n, int32_t k, const double *V, int64_t ld, double *w,
            double *h, int32_t ortho, void *stream);

/* ---- restarted Lanczos eigensolver (OpenATI_EIGENSOLVE, Sec. 2.2 / 4.3) ---
 * The nev largest eigenvalues of a symmetric A (general storage holding both
 * triangles, or sym_upper) by thick-restart Lanczos with full DGKS
 * re-orthogonalisation: cycles of m basis vectors (nev < m <= min(n, 512)),
 * restarts keeping nev + (m - nev)/2 Ritz vectors, until every wanted Ritz
 * pair has residual ||A y - theta y|| <= tol |theta| or maxrestart restarts.
 * m_max > m turns on the restart rule (Eq. 1, Sec. 4.3): the worst relative
 * wanted residual of each cycle is a sample, every 5 samples the MM ratio is
 * compared with theta and m grows by 5 (up to m_max <= min(n, 512)) when the
 * residuals stagnate.  The plan's SpMV choice is used.  policy: as for
 * xb_arnoldi (SpMV, cycle, restart rule, true-residual check, outer loop;
 * MEMORY's cycle is m = max(nev + 1, min(m, 20))), but the Gram-Schmidt stays
 * DGKS under every policy.  v0: DEVICE start vector (n), or NULL for a
 * fixed pseudo-random one.  evals, resid: HOST arrays (nev), largest first;
 * evecs: DEVICE n x nev column-major (unit Ritz vectors) or NULL; counts:
 * HOST int[5] = {Lanczos steps (SpMVs), restarts, final m, Gram-Schmidt used
 * at the end, outer passes} or NULL; stats: HOST double[2] as for xb_arnoldi
 * or NULL.  Returns XB_OK, XB_ENOCONV (restart limit; evals hold the current
 * Ritz values), XB_EFAULT (a policy's true-residual check failed) or
 * XB_EBREAKDOWN (the start vector spans an invariant subspace of dimension
 * < m).  Synchronises the stream. */
int xb_lanczos(xb_plan *plan, int32_t nev, int32_t m, int32_t m_max, double theta, double tol,
               int32_t maxrestart, int32_t policy, const double *v0, double *evals,
               double *evecs, double *resid, int32_t *counts, double *stats, void *stream);

/* ---- restarted Arnoldi eigensolver (OpenATI_EIGENSOLVE, Sec. 2.2 / 4.3) ---
 * nev eigenvalues of a general A at the wanted end (which = XB_EIG_LR or
 * XB_EIG_LM) by restarted Arnoldi in Krylov-Schur form: cycles of m basis
 * vectors (nev + 2 <= m <= min(n, 512)) orthogonalised on the device with
 * ortho = XB_ORTHO_MGS / CGS / DGKS / BCGS / AUTO (Sec. 3.2.2; AUTO = the
 * accuracy rule of Sec. 3.3.2); the m x m projected matrix is put in complex
 * Schur form on the host and reordered so that the wanted eigenvalues lead;
 * a restart keeps the real invariant subspace of the k = nev + (m - nev)/2
 * leading ones (k + 1 when k would split a conjugate pair).  Stops when every
 * wanted Ritz pair has residual ||A y - theta y|| <= tol |theta| or after
 * maxrestart restarts.  m_max > m turns on the restart rule (Eq. 1, Sec. 4.3)
 * exactly as for xb_lanczos.  policy (Sec. 2.3.2, 3.3): XB_POLICY_NONE runs
 * the arguments as given; TIME tunes the SpMV (exhaustive), turns the restart
 * rule on with m_max >= 128 and picks the Gram-Schmidt by the accuracy rule;
 * MEMORY uses the SpMV without plan metadata (U1, S1 for sym_upper), a fixed
 * m = max(nev + 2, min(m, 20)) and MGS; STABLE keeps the plan's SpMV and m,
 * MGS, no rule; ACCURACY is TIME plus the outer loop of Sec. 3.3.2.  Under
 * every policy but NONE, a claimed convergence is checked with the true
 * residuals ||A y - theta y|| / |theta| (2 nev SpMVs): ACCURACY narrows the
 * threshold by tol / (worst true residual), switches to DGKS and iterates
 * on; the others return XB_EFAULT.  v0: DEVICE start vector (n) or NULL for
 * a fixed pseudo-random one.  evals_re, evals_im, resid: HOST arrays (nev),
 * wanted order; a conjugate pair is adjacent, positive imaginary part first.
 * evecs_re / evecs_im: DEVICE n x nev column-major real and imaginary parts of
 * the unit Ritz vectors (either may be NULL).  counts: HOST int[5] = {Arnoldi
 * steps (SpMVs), restarts, final m, Gram-Schmidt used at the end, outer
 * passes} or NULL.  stats: HOST double[2] = {device bytes of the call's
 * workspace and SpMV metadata, worst true relative residual of the last check
 * (-1 if none)} or NULL.  Returns XB_OK, XB_ENOCONV, XB_EFAULT,
 * XB_EBREAKDOWN (the start vector spans an invariant subspace of dimension
 * < m) or XB_EINVAL.  Synchronises the stream. */
int xb_arnoldi(xb_plan *plan, int32_t nev, int32_t m, int32_t m_max, double theta, double tol,
               int32_t maxrestart, int32_t which, int32_t ortho, int32_t policy, const double *v0,
               double *evals_re, double *evals_im, double *evecs_re, double *evecs_im,
               double *resid, int32_t *counts, double *stats, void *stream);

/* Eigen-decomposition of a small general matrix, the dense step inside
 * xb_arnoldi (host code, no device work): A is a HOST row-major n x n array
 * (1 <= n <= 512); eigenvalues wr + i wi (HOST, n) in the order of `which`,
 * conjugate pairs adjacent; vr / vi (HOST n x n column-major, both or
 * neither NULL) the unit eigenvectors, largest entry real and positive. */
int xb_dense_eig(int32_t n, const double *A, int32_t which, double *wr, double *wi, double *vr,
                 double *vi);
/* The restart step of xb_arnoldi on a small dense matrix (host logic,
 * exposed for testing): the k leading wanted eigenvalues of the HOST
 * row-major n x n matrix A (2 <= n <= 512, 1 <= k < n; k moved by one when it
 * would split a conjugate pair), their invariant subspace as an orthonormal
 * real basis in Q (HOST, n x (k + 1) column-major room), *kout = its
 * dimension. */
int xb_dense_restart_basis(int32_t n, const double *A, int32_t which, int32_t k, double *Q,
                           int32_t *kout);

/* ---- ILU(0) preconditioner (Sec. 4.3) -------------------------------------
 * Built once per plan on first use (dependency levels of the two triangles
 * from the pattern on the host, numeric factorization on the device, level
 * by level); general CRS only (XB_EINVAL for sym_upper plans).  A row without
 * a stored diagonal or a zero pivot gives XB_EBREAKDOWN. */
int xb_ilu0_setup(xb_plan *plan, void *stream);
/* z = (L U)^{-1} r: forward then backward substitution, one launch per
 * dependency level.  r and z: DEVICE, n doubles, distinct. */
int xb_ilu0_apply(xb_plan *plan, const double *r, double *z, void *stream);
/* Which substitution path the plan's ILU(0) applications take, and the
 * persistent path's barrier poll limit (a control for tests and diagnosis).
 * mode: -1 = automatic (the default; the environment variable XB_ILU_MODE
 * = 0/1 overrides it), 0 = the captured graph of level launches, 1 = one
 * cooperative launch with a grid barrier between levels (used only when the
 * device supports cooperative launches).  barrier_polls: how many times a CTA
 * polls a level barrier before it gives up (0 = default, about 0.5 s of
 * polling); a CTA that gives up sets an error flag and returns, every other
 * CTA returns at its next barrier, and the apply or solve reports
 * XB_ETIMEOUT.  XB_EINVAL for mode outside -1..1 or barrier_polls < 0. */
int xb_ilu0_config(xb_plan *plan, int32_t mode, int32_t barrier_polls);
/* Copy the factors (aligned with the plan's col array: strict lower part = L
 * with unit diagonal not stored, the rest = U) to the DEVICE array lu (nnz). */
int xb_ilu0_factors(xb_plan *plan, double *lu, void *stream);
/* The dependency levels xb_ilu0_setup schedules by (host logic, no device
 * work; exposed for testing): for the row pattern (HOST rowptr n + 1, col
 * nnz, sorted rows), lev[i] = 1 + max lev over the row's strictly-lower
 * columns (0 if none) and ulev[i] = 1 + max ulev over its strictly-upper
 * columns; nlevels[0..1] = the level counts.  lev, ulev (n) and nlevels (2)
 * are HOST arrays or NULL.  XB_EBREAKDOWN for a row without a diagonal. */
int xb_ilu_levels(int32_t n, const int32_t *rowptr, const int32_t *col, int32_t *lev,
                  int32_t *ulev, int32_t *nlevels);

/* ---- numerical policy file (Sec. 2.3.2) -----------------------------------
 * The meta-solvers' user input: lines "<keyword> = <value>", keywords in any
 * case, blank lines and lines starting with '#' or '!' skipped, keywords the
 * file does not register ignored.  POLICY = TIME / ACCURACY / MEMORY / STABLE
 * sets opt->policy (any other value: TIME, the default policy); RESIDUAL (a
 * real, Fortran's D exponent accepted) sets opt->tol; MAXTIME (seconds) sets
 * opt->maxtime_s; PRECONDITIONER = NONE / ILU0 / ILU(0) sets opt->precond;
 * SOLVER = GMRES / BICGSTAB / LANCZOS / ARNOLDI goes to *solver
 * (XB_SOLVER_*); MAXMEMORY (bytes, optional K / M / G / T suffix, powers of
 * 1024) to *max_memory; CPU (the paper's thread count; the device is the
 * caller's choice) to *cpu.  opt is updated in place (start from
 * xb_options_default); solver, max_memory and cpu may be NULL and are left
 * unchanged when their keyword is absent.  text: HOST, NUL-terminated.
 * XB_EINVAL, with the line number in xb_last_error, for a line without '='
 * or a value that does not parse.  Host only: no device work. */
int xb_policy_parse(const char *text, xb_options *opt, int32_t *solver, double *max_memory,
                    int32_t *cpu);
/* Reads "OPENATI_POLICY_INPUT.<id>" (id: the caller's thread or device
 * number) from directory dir (NULL or "" = the current directory) and parses
 * it as xb_policy_parse does; XB_EINVAL if the file cannot be opened. */
int xb_policy_read(const char *dir, int32_t id, xb_options *opt, int32_t *solver,
                   double *max_memory, int32_t *cpu);

/* ---- run-time auto-tuning ------------------------------------------------ */

/* Before-execution AT (Sec. 3.1): time every candidate (variant x CTA size x
 * items per thread) that fits the plan's storage, each at most 4 times after
 * one warm-up, with CUDA events on `stream`; keep the minimum.  Sets the
 * plan's choice and returns it in *out (may be NULL). */
int xb_tune_exhaustive(xb_plan *plan, xb_choice *out, void *stream);

/* The sweep behind xb_tune_exhaustive: every candidate that fits, with its
 * best time, written to the HOST array out (at most cap entries); *count
 * receives the number of candidates timed.  Does not change the plan. */
int xb_tune_sweep(xb_plan *plan, xb_choice *out, int32_t cap, int32_t *count, void *stream);

/* MM ratio of Eq. (1): R(s,t) = max / min of r(s-t+1..s), r 1-based on the
 * HOST array r (r[z-1] = r(z)); 1 <= t <= s.  Returns +inf for a zero min. */
double xb_mm_ratio(const double *r, int32_t s, int32_t t);
/* OpenATI_DAFRT judgement: 1 if R(I, I) over samp[0..I-1] < theta, else 0. */
int xb_dafrt(int32_t I, const double *samp, double theta);

/* ---- learned tuner --------------------------------------------------------
 * Matrix features on the device (host output): raw[7] = n, nnz, mean row
 * length, population variance, max row length, bandwidth max|i-j|, symmetry
 * (1 if sym_upper or the stored pattern and values equal their transpose);
 * feat[8] = ln(1+n), ln(1+nnz), ln(1+mean), ln(1+var), ln(1+max),
 * ln(1+bandwidth), sym, ln(1+max) - ln(1+mean).  Either output may be NULL. */
int xb_features(const xb_csr *A, double *raw, float *feat, void *stream);

/* ---- learned tuner: MLP with hand-written training and inference kernels --
 * d_in -> h1 (ReLU) -> h2 (ReLU) -> sum(heads) logits, one softmax
 * cross-entropy per head; FP32 parameters on the device.  Inputs are
 * standardised by (x - mu) / sd (identity until xb_mlp_set_norm).  Parameter
 * blob layout: W1[h1][d_in], b1[h1], W2[h2][h1], b2[h2], W3[o][h2], b3[o],
 * o = sum(heads).  Every batch reduction is a fixed-order loop, so results
 * are deterministic.  d_in <= 16, nheads <= 8, each head >= 2 classes. */
typedef struct xb_mlp xb_mlp;
int xb_mlp_create(int32_t d_in, int32_t h1, int32_t h2, int32_t nheads, const int32_t *heads,
                  uint64_t seed, xb_mlp **out);
int xb_mlp_destroy(xb_mlp *m);
int64_t xb_mlp_param_count(const xb_mlp *m);
/* Parameters host <-> device (host pointer, param_count floats). */
int xb_mlp_get_params(const xb_mlp *m, float *host);
int xb_mlp_set_params(xb_mlp *m, const float *host);
/* Input standardisation (host arrays of d_in floats, sd > 0). */
int xb_mlp_set_norm(xb_mlp *m, const float *mu, const float *sd);
/* Forward: X device [B][d_in] FP32 -> logits device [B][o]. */
int xb_mlp_forward(xb_mlp *m, const float *X, int32_t B, float *logits, void *stream);
/* Mean over the batch of the summed per-head softmax cross-entropy, and its
 * gradient (kept in the model for xb_mlp_adam; copied to the DEVICE array
 * grad_out when it is not NULL).  labels: device [B][nheads]; a negative
 * label leaves that head of that sample out of the loss.  *loss: host. */
int xb_mlp_loss_grad(xb_mlp *m, const float *X, const int32_t *labels, int32_t B, float *loss,
                     float *grad_out, void *stream);
/* One Adam step (Kingma & Ba; t counts from 1) with the stored gradient. */
int xb_mlp_adam(xb_mlp *m, int32_t t, float lr, float b1, float b2, float eps, void *stream);
/* Minibatch Adam training on device data X [N][d_in], labels [N][nheads]:
 * `epochs` passes in a seeded shuffled order; *final_loss (host, may be
 * NULL) receives the full-set loss after training. */
int xb_mlp_train(xb_mlp *m, const float *X, const int32_t *labels, int32_t N, int32_t epochs,
                 int32_t batch, float lr, uint64_t seed, float *final_loss, void *stream);
/* Argmax per head: out_host [B][nheads]. */
int xb_mlp_predict(xb_mlp *m, const float *X, int32_t B, int32_t *out_host, void *stream);
/* Binary model file (header, standardisation, parameters). */
int xb_mlp_save(const xb_mlp *m, const char *path);
int xb_mlp_load(const char *path, xb_mlp **out);

/* Learned run-time tuning: features of A (xb_features) through the model,
 * whose heads are (variant: 5 classes XB_VAR_0..4, CTA size: 64/128/256/512,
 * items per thread: 1/4/8/16/32, GMRES restart m: 10/20/30/50/80/120).  The
 * arg-max over the choices that fit the plan's storage and the variant's
 * supported shapes becomes the plan's choice (returned in *out); *m_out (may
 * be NULL) receives the predicted restart length.  A must be the matrix the
 * plan was built on. */
int xb_tune_mlp(xb_plan *plan, const xb_csr *A, xb_mlp *model, xb_choice *out, int32_t *m_out,
                void *stream);

/* ---- batched solve: many uneven systems in one persistent launch ----------
 * Each system is an independent A x = b in general CRS (device pointers, the
 * xb_csr rules with sym_upper = 0) solved by restarted GMRES(m) with MGS,
 * the same algorithm as gmres_solve.  One persistent kernel (captured once in
 * a CUDA graph, replayed by xb_batch_run) holds as many CTAs as fit on the
 * GPU, in 8-CTA clusters; work comes from two atomic queues.  A system with
 * n >= 30000 (XB_BATCH_COOP_MIN_N in the environment overrides the
 * threshold) is solved by a whole cluster, its dot products combined through
 * distributed shared memory; these are taken first, largest first.  Once
 * they are all taken, every CTA pulls the smaller systems (largest first)
 * one at a time as soon as it is free, with no inter-CTA synchronisation.  opt: tol, maxiter (per
 * system), maxtime_s (whole launch; checked at every restart), dafrt /
 * dafrt_theta / m_max (the restart-length rule, per system), ortho
 * (XB_ORTHO_MGS, XB_ORTHO_BCGS, or XB_ORTHO_AUTO: BCGS for tol > 1e-10,
 * else MGS; others are rejected).  Per system:
 * m in [1, XB_BATCH_MAX_M] and the SpMV mode inside the CTA (0: thread per
 * row; 1: thread per row in warp-sized row blocks, rows longer than 32
 * non-zeros taken by the whole warp, rows longer than 1024 by the whole CTA
 * after the blocks -- xb_batch_create reads each mode-1 system's row pointer
 * once to list them), as chosen by a tuner; zero_x = 1 makes the kernel
 * start from x = 0 (so a replay repeats the same solve). */
#define XB_BATCH_MAX_M 128
typedef struct xb_batch_sys {
    int32_t n, nnz;
    const int32_t *rowptr, *col;
    const double *val, *b;
    double *x;
    int32_t m, mode, zero_x;
} xb_batch_sys;
typedef struct xb_batch_info {
    int32_t status, iters, restarts, m, mode;
    double res_true;         /* ||b - A x|| / ||b|| at exit                   */
    double ms;               /* device time spent on this system              */
} xb_batch_info;
typedef struct xb_batch xb_batch;
/* Validate, allocate the per-system workspace ((m+1)(n+31) doubles each) and
 * capture the graph.  Does not run it. */
int xb_batch_create(int32_t count, const xb_batch_sys *sys, const xb_options *opt, void *stream,
                    xb_batch **out);
/* Replay the captured launch on `stream` (asynchronous). */
int xb_batch_run(xb_batch *b, void *stream);
/* Wait for `stream` and copy the per-system results to the HOST array infos;
 * returns the first non-OK system status, else XB_OK. */
int xb_batch_results(xb_batch *b, xb_batch_info *infos, void *stream);
int xb_batch_destroy(xb_batch *b);
/* create + run + results + destroy. */
int xb_batch_solve(int32_t count, const xb_batch_sys *sys, const xb_options *opt,
                   xb_batch_info *infos, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* XABC_H */
