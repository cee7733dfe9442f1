// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/xabc.h"

namespace xb {

// ---- error handling -------------------------------------------------------
int set_error(int code, const char *fmt, ...);
int cuda_error(cudaError_t e, const char *where);

#define XB_CUDA(call)                                                  \
    do {                                                               \
        cudaError_t e__ = (call);                                      \
        if (e__ != cudaSuccess) return ::xb::cuda_error(e__, #call);   \
    } while (0)
#define XB_LAUNCHED(where)                                             \
    do {                                                               \
        cudaError_t e__ = cudaGetLastError();                          \
        if (e__ != cudaSuccess) return ::xb::cuda_error(e__, where);    \
    } while (0)
#define XB_TRY(...)                                                    \
    do {                                                               \
        int r__ = (__VA_ARGS__);                                       \
        if (r__ != XB_OK) return r__;                                  \
    } while (0)

// ---- device constants ------------------------------------------------------
constexpr int kRedSlots = 2048;     // max CTAs of a reduction grid
constexpr int kRedValues = 16;      // max values reduced together by one grid
constexpr int kScalars = 4096;      // device scalar scratch per plan (doubles)

int num_sms();                      // cached cudaDevAttrMultiProcessorCount
int reduce_grid(int64_t n, int block);  // CTAs for a streaming reduction
// CTAs of a grid-stride launch of kernel fn: every CTA resident at once (the
// occupancy limit times the SM count, at most kRedSlots), fewer for small n
// (per_thread elements per thread).
int resident_grid(const void *fn, int block, int64_t n, int per_thread);

// ---- partitions -------------------------------------------------------------
// Row-aligned nnz-balanced tiles (U2 / S2): tile t covers rows
// [row[t], row[t+1]); at most T = block*ipt non-zeros and `block` rows, except
// a single row longer than T which forms a tile of its own.
struct TilePart {
    int block = 0, ipt = 0;
    int ntiles = 0;
    int *d_row = nullptr;    // ntiles+1
};
// Row-aligned nnz-balanced warp tiles (U2).  Warp tile t covers rows
// [r0, r1) whose non-zeros [k0, k1) fit the 32*ipt-entry window that starts
// at k0 rounded down to a multiple of ipt; rows never cross tiles.  Kind:
//   0  thread per row: at most 32 rows, none longer than ipt;
//   1  flat: lane l sums window entries [l*ipt, (l+1)*ipt) inside [k0, k1),
//      row ends from the BSS bitmask, rows joined by a segmented warp scan.
// A row too long for a window is listed in d_long and gets a CTA.  When every
// tile is 32 rows of kind 0 (uniform short rows) the tiles are implicit
// (tile t = rows [32t, 32t + 32)) and no table is read.
struct U2Part {
    int ipt = 0;
    int ntiles = 0, nlong = 0, nflat = 0;
    bool implicit = false;
    int4 *d_tile = nullptr;  // {r0, r1, ne0 (non-empty-row index of the first
                             //  non-empty row >= r0), kind | 4 if it has empty rows}
    int *d_long = nullptr;
};
// S3 partial vectors (XB_VAR_SYM_PART) over the S2 tiles (TilePart with the
// same block, ipt): slots tslot[t] .. tslot[t+1]-1 of tile t hold the granules
// (kS3Gran rows each, sgran[slot]) its transposes reach beyond the tile, at
// most kS3Max per tile; reached granule c (gid[c]) adds slots
// gslot[gptr[c] .. gptr[c+1]-1] (tile order).  part: nslots * kS3Gran values.
constexpr int kS3Gran = 256;
constexpr int kS3Max = 8;
struct S3Part {
    int block = 0, ipt = 0;
    int ntiles = 0, nslots = 0, ngran = 0;
    int *d_tslot = nullptr, *d_sgran = nullptr;
    int *d_gid = nullptr, *d_gptr = nullptr, *d_gslot = nullptr;
    double *d_part = nullptr;  // FP32 use reads it as floats
};
// Block CRS copy (format conversion, XB_VAR_BCSR): r x r blocks, block row
// b = rows [r b, r b + r), blocks ascending by block column, values row-major
// inside a block and zero where A has no entry.
struct BcsrPart {
    int r = 0;
    int nbr = 0;                     // block rows
    int64_t nblocks = 0;
    int *d_bptr = nullptr;           // nbr + 1
    int *d_bcol = nullptr;           // nblocks
    double *d_val = nullptr;         // nblocks * r * r
    float *d_val32 = nullptr;        // built on the first FP32 use
};
// Flat nnz segments (U3, BSS): warp w owns non-zeros [w*W, (w+1)*W), W =
// 32*ipt; d_row[w] is the (non-empty-row) index of the row holding non-zero
// w*W; one carry slot per warp feeds the fix-up.
struct SegPart {
    int block = 0, ipt = 0;
    int nblk = 0;            // warps
    int *d_row = nullptr;    // nblk+1
    int *d_carry_row = nullptr;
    double *d_carry_val = nullptr;   // raw partial sums (float in FP32 use)
};
// SELL-C-sigma copy (C = 32): rows sorted by length (longest first, stable)
// inside windows of sigma rows; slice q holds sorted rows 32q..32q+31, its
// entries stored column by column (entry j of its 32 rows at off[q] + 32 j +
// lane), as wide as its longest row.  Padding is never read (a row stops at
// its own length), so it is left unset.
struct SellPart {
    int sigma = 0;
    int nslices = 0;
    int64_t total = 0;               // entries including padding
    int64_t *d_off = nullptr;        // nslices + 1
    int *d_perm = nullptr;           // nslices * 32 row of each slot, -1 past n
    int *d_len = nullptr;            // nslices * 32 length of each slot's row
    int *d_col = nullptr;            // total
    double *d_val = nullptr;         // total
    float *d_val32 = nullptr;        // total, built on the first FP32 use
};
// The BSS "continuous location" data of the plan (independent of the launch
// shape): bit e of d_endbits is set when non-zero e is the last one of its
// row; with empty rows present, rows are renumbered over the non-empty ones
// (d_ne_rows maps back, d_crp is the rowptr of the non-empty rows).
// The BSS data format: A's values and columns copied in the order the
// segmented-scan warps read them.  Warp chunk g holds non-zeros
// [g*W, (g+1)*W), W = 32*ipt, and lane l of its warp owns the ipt consecutive
// ones from g*W + l*ipt.  The copy stores the lane's values as vectors of VN
// consecutive elements (VN = 2 for FP64, 4 for FP32): vector q of lane l sits
// at g*W + (q*32 + l)*VN; columns likewise in vectors of 4.  The q-th vector
// load of a warp therefore reads 32 consecutive 16-byte vectors (512 bytes,
// four whole 128-byte lines) instead of 32 vectors 16*ipt/VN bytes apart.
// Padded with zero values (column 0) to whole chunks.
struct BssCopy {
    int ipt = 0;
    int64_t total = 0;               // entries including padding
    int *d_col = nullptr;
    double *d_val = nullptr;
    float *d_val32 = nullptr;        // built on the first FP32 use
};
struct BssData {
    unsigned *d_endbits = nullptr;   // ceil(nnz/32) + 1 words
    int *d_ne_rows = nullptr;        // n_ne, or null when no row is empty
    int *d_crp = nullptr;            // n_ne + 1, or null (then rowptr)
    int n_ne = 0;
    bool built = false;
    std::vector<BssCopy> copies;     // one per ipt in use
};

// ILU(0) preconditioner data (built on first use): factors in A's pattern
// (strict lower part L with unit diagonal, the rest U), the diagonal
// positions, and the rows grouped by dependency level for the forward (L)
// and backward (U) substitutions: every row of a level depends only on rows
// of earlier levels.
struct IluData {
    bool built = false;
    int status = 0;                  // XB_OK or XB_EBREAKDOWN (zero pivot)
    double *d_lu = nullptr;          // nnz
    int *d_dpos = nullptr;           // n
    int *d_lrows = nullptr, *d_urows = nullptr;  // n each, ordered by level
    std::vector<int> loff, uoff;     // level offsets (levels + 1)
    // Inside a level rows are ordered by tier: short rows (<= 8 entries in the
    // triangle) first, stored again level by level in ELL form (entry t of
    // slot s at eoff[l] + t * count + s, padded with zero values) so a thread
    // loads its row with no dependent index loads; then rows of up to 512
    // entries (thread or warp per row, CSR); then longer rows (CTA per row).
    std::vector<int> ln0, ln1, un0, un1;  // per level: ELL-tier and CSR-tier counts
    std::vector<int> lw, uw;              // per level: ELL width
    std::vector<long long> leoff, ueoff;  // per level: ELL base offset
    int *d_lecol = nullptr, *d_uecol = nullptr;
    double *d_leval = nullptr, *d_ueval = nullptr;
    int *d_lesrc = nullptr, *d_uesrc = nullptr;  // factor position of each ELL entry (-1: pad)
    double *d_udiag = nullptr;            // u_ii in backward level order
    int *d_flag = nullptr;           // zero-pivot flag
    double *d_in = nullptr, *d_out = nullptr;  // fixed operands of the captured solve
    cudaGraph_t graph = nullptr;     // both substitutions, every level, captured once
    cudaGraphExec_t exec = nullptr;
    // persistent substitution (one cooperative launch, a bounded grid barrier
    // between levels): level tables on the device, barrier state, error flag
    int *d_lmeta = nullptr, *d_umeta = nullptr;        // per level: off, n0, n1, w
    long long *d_leo = nullptr, *d_ueo = nullptr;      // per level: ELL base offset
    unsigned *d_bar = nullptr;                          // count, generation
    int *d_err = nullptr;                               // 1: a barrier wait ran out
    int pgrid = 0;                                      // CTAs of the persistent launch
};

}  // namespace xb

struct xb_plan {
    int n = 0, nnz = 0, sym = 0;
    int ncols = 0;                       // columns (= n but for the row blocks of a split plan)
    int64_t nnz64 = 0;                   // non-zeros (nnz saturates in a split plan)
    int *d_rp32_own = nullptr;           // int32 row offsets the plan narrowed from 64-bit ones
    struct Sub {
        int r0;
        xb_plan *plan;
    };
    std::vector<Sub> subs;               // row blocks of a plan with more than 2^31 - 64 non-zeros
    const int *rowptr = nullptr, *col = nullptr;
    const double *val = nullptr;
    float *val32 = nullptr;              // FP32 copy (mixed precision)
    std::vector<int> h_rowptr;           // host copy, used to build partitions
    int max_row = 0;
    int n_empty = 0;
    int *d_empty = nullptr;              // rows with no stored entry
    std::vector<xb::TilePart> tiles;     // cache by (block, ipt)
    std::vector<xb::SegPart> segs;       // cache by (block, ipt)
    std::vector<xb::U2Part> u2;          // cache by ipt
    std::vector<xb::S3Part> s3;          // cache by (block, ipt)
    std::vector<xb::BcsrPart> bcsr;      // cache by block size r
    std::vector<xb::SellPart> sells;     // cache by sigma
    xb::BssData bss;
    xb::IluData ilu;
    int ilu_mode = -1;                   // substitution path: -1 auto, 0 graph, 1 persistent
    int ilu_polls = 0;                   // persistent barrier poll limit (0: default)
    bool vec_ok = false;                 // val and col 16-byte aligned
    // reduction scratch
    double *d_part = nullptr;            // kRedSlots * kRedValues partials
    unsigned *d_ticket = nullptr;        // 64 counters (one in use per reduction)
    double *d_scal = nullptr;            // kScalars
    // solver workspace (grown on demand)
    void *d_work = nullptr;
    size_t work_bytes = 0;
    double *h_pin = nullptr;             // pinned host mirror of a few scalars
    // tuned choice
    int variant = XB_VAR_NNZ, block = 256, ipt = 8;
    float tuned_ms = 0.f;
    cudaEvent_t ev[2] = {nullptr, nullptr};
};

namespace xb {

const TilePart *get_tiles(xb_plan *p, int block, int ipt, cudaStream_t s, int *err);
const SegPart *get_segs(xb_plan *p, int block, int ipt, cudaStream_t s, int *err);
const U2Part *get_u2(xb_plan *p, int ipt, cudaStream_t s, int *err);
// Row starts of the S2 / U2-CTA tiles (host): at most block rows and
// block*ipt non-zeros per tile, a longer row alone.
std::vector<int> tile_rows(int n, const int *rp, int block, int ipt);
// The S3 slots and cover lists (XB_EINVAL when a tile reaches more than
// kS3Max granules beyond itself).
const S3Part *get_s3(xb_plan *p, int block, int ipt, cudaStream_t s, int *err);
// Block CRS structure on the host from the pattern; returns the block count.
int64_t bcsr_layout(int n, const int *rp, const int *col, int r, std::vector<int> &bptr,
                    std::vector<int> &bcol);
// BCSR copy with r x r blocks (FP32 values too when f32); XB_EINVAL when the
// blocks would hold more than 2 nnz + 16 r entries.
const BcsrPart *get_bcsr(xb_plan *p, int r, bool f32, cudaStream_t s, int *err);
// The U2 warp tiles on the host from the row pointer (n + 1 entries); returns
// the number of flat tiles.  tiles: {r0, r1, ne0, kind | 4 * has_empty}.
int u2_layout(int n, const int *rp, int ipt, std::vector<int4> &tiles, std::vector<int> &longs);
// SELL-32-sigma copy (FP32 values too when f32); XB_EINVAL when the padding
// would exceed 3 nnz + 32 per slice.
const SellPart *get_sell(xb_plan *p, int sigma, bool f32, cudaStream_t s, int *err);
// The SELL-32-sigma layout on the host from the row pointer (n + 1 entries):
// perm (slot -> row, -1 past n), slen (slot -> row length), off (slice entry
// offsets, nslices + 1); returns the padded entry count.
int64_t sell_layout(int n, const int *rp, int sigma, std::vector<int> &perm,
                    std::vector<int> &slen, std::vector<int64_t> &off);
const BssData *get_bss(xb_plan *p, cudaStream_t s, int *err);
// BSS data format copy for ipt (FP32 values too when f32), built on first use.
const BssCopy *get_bss_copy(xb_plan *p, int ipt, bool f32, cudaStream_t s, int *err);
// Free the BSS copies of every ipt but keep_ipt (0: all of them).
void bss_trim(xb_plan *p, int keep_ipt);
int ensure_val32(xb_plan *p, cudaStream_t s);
int ensure_work(xb_plan *p, size_t bytes);
// ILU(0): build (levels on the host from the pattern, factorization on the
// device), apply z = (LU)^{-1} r on stream s, and the algorithmic bytes of one
// application.
int ensure_ilu(xb_plan *p, cudaStream_t s);
// Dependency levels of the two triangles from the pattern (host): lev[i] = 1 +
// the largest lev of the row's strictly-lower columns (0 if none), ulev[i]
// likewise over its strictly-upper columns; dpos = each row's diagonal entry;
// *nl, *nu = level counts.  XB_EBREAKDOWN for a row without a diagonal entry.
int ilu_levels(int n, const int *rp, const int *ci, std::vector<int> &dpos, std::vector<int> &lev,
               std::vector<int> &ulev, int *nl, int *nu);
int ilu_apply(xb_plan *p, const double *r, double *z, cudaStream_t s);
// GMRES(m) of the plan's system in one persistent launch (the batched
// kernel with a single system): FP64, general storage, MGS or BCGS, m <= 128.
int batch_single(xb_plan *p, const double *b, double *x, const xb_options &o, int mode,
                 xb_info &inf, double *alg_bytes, cudaStream_t s);
// The same solve from one cluster's shared memory when the system fits
// (resident.cu); *ran = false when it does not (nothing launched).
int resident_gmres(xb_plan *p, const double *b, double *x, const xb_options &o, xb_info &inf,
                   double *alg_bytes, cudaStream_t s, bool *ran);
double ilu_apply_bytes(const xb_plan *p);
int ilu_check(xb_plan *p);  // XB_ETIMEOUT if a substitution's barrier wait ran out
void ilu_free(xb_plan *p);
bool variant_fits(const xb_plan *p, int variant);
// Consecutive row blocks of a 64-bit row pointer, each holding at most
// max_nnz non-zeros (rows never split): starts[b] = first row of block b,
// plus n at the end.  XB_EINVAL when one row alone has more than max_nnz.
int split_rows64(int n, const int64_t *rp, int64_t max_nnz, std::vector<int> &starts);

// SpMV dispatch: y = alpha*A*x + beta*y in value type double or float.
int spmv_launch(xb_plan *p, int variant, int block, int ipt, double alpha, const double *x,
                double beta, double *y, cudaStream_t s);
int spmv_launch_f32(xb_plan *p, int variant, int block, int ipt, float alpha, const float *x,
                    float beta, float *y, cudaStream_t s);
// Algorithmic bytes of one SpMV (val+col once, rowptr once, x once, y once,
// y read again when beta != 0).
double spmv_alg_bytes(const xb_plan *p, bool beta_nonzero, int val_bytes);
// Device bytes of the plan data a variant reads besides the matrix (tile
// starts, BSS bitmask and warp rows, segment tables).
double spmv_meta_bytes(const xb_plan *p, int variant, int block, int ipt);

// ---- vector kernels (vec.cu) ------------------------------------------------
// Deterministic reductions write their result to a device double.
int vdot(xb_plan *p, int64_t n, const double *x, const double *y, double *out, cudaStream_t s);
int vnrm2(xb_plan *p, int64_t n, const double *x, double *out, cudaStream_t s);
int vaxpy(int64_t n, double a, const double *x, double *y, cudaStream_t s);
int vcopy(int64_t n, const double *x, double *y, cudaStream_t s);
int vscale(int64_t n, double a, double *x, cudaStream_t s);
int vfill(int64_t n, double a, double *x, cudaStream_t s);

}  // namespace xb

// ---- device helpers ----------------------------------------------------------
namespace xbd {

template <typename V>
__device__ __forceinline__ V warp_sum(V v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the block; result valid in thread 0.  `sh` holds >= 32 V.
template <typename V>
__device__ __forceinline__ V block_sum(V v, V *sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    if (w == 0) {
        v = lane < nw ? sh[lane] : V(0);
        v = warp_sum(v);
    }
    return v;
}

}  // namespace xbd
