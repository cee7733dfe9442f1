// CRS SpMV kernels for sm_103a: y = alpha*A*x + beta*y.
//
// The paper's OpenMP implementations (Sec. 3.2.2) are the prior art: U1
// row-based decomposition, U2 non-zero-balanced row decomposition, U3
// branchless segmented scan (BSS), and for symmetric upper storage S1-S3
// (S3: skip the reduction work on all-zero parts of the per-thread vectors).
// On GB300 the FP64 pipe delivers ~2 DFMA/clk/SM (~0.6 T DFMA/s), barely
// above what HBM needs for 12 B per non-zero, so every kernel here spends
// one FP64 instruction per non-zero and keeps all other work (index math,
// staging, row search, transpose scatter) on integer, shared-memory or L2
// atomic paths.
//
// mode: 0 -> y = s, 1 -> y = alpha*s, 2 -> y = alpha*s + beta*y.
#include "common.cuh"
#include "krylov.cuh"

#include <algorithm>
#include <climits>
#include <mutex>
#include <unordered_set>

namespace {

template <typename V>
__device__ __forceinline__ void store_row(V *__restrict__ y, int r, V s, V alpha, V beta, int mode) {
    if (mode == 0)
        y[r] = s;
    else if (mode == 1)
        y[r] = alpha * s;
    else
        y[r] = fma(alpha, s, beta * y[r]);
}

// ---------------------------------------------------------------------------
// U1: one thread per row, operands straight from global memory.
// ---------------------------------------------------------------------------
template <typename V>
__global__ void __launch_bounds__(512) k_row(int n, const int *__restrict__ rowptr,
                                             const int *__restrict__ col, const V *__restrict__ val,
                                             const V *__restrict__ x, V alpha, V beta, int mode,
                                             V *__restrict__ y, const V *__restrict__ adev) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    if (adev) alpha = *adev;
    const int a = rowptr[r], b = rowptr[r + 1];
    V s = V(0);
    for (int k = a; k < b; k++) s = fma(val[k], x[col[k]], s);
    store_row(y, r, s, alpha, beta, mode);
}

// ---------------------------------------------------------------------------
// SELL-C-sigma (format conversion, C = 32): thread per row of a slice; the
// warp's loads of entry j are 32 consecutive values and columns.  A row reads
// its own length of entries (padding is never read) in CRS order, so the sum
// is the one k_row forms.
// ---------------------------------------------------------------------------
template <typename V>
__global__ void __launch_bounds__(512) k_sell(int nslices, const int64_t *__restrict__ off,
                                              const int *__restrict__ perm,
                                              const int *__restrict__ slen,
                                              const int *__restrict__ col,
                                              const V *__restrict__ val, const V *__restrict__ x,
                                              V alpha, V beta, int mode, V *__restrict__ y,
                                              const V *__restrict__ adev) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if ((t >> 5) >= nslices) return;
    const int r = perm[t];
    if (r < 0) return;
    if (adev) alpha = *adev;
    const int len = slen[t];
    const int64_t base = off[t >> 5] + (t & 31);
    V s = V(0);
#pragma unroll 4
    for (int j = 0; j < len; j++) {
        const int64_t k = base + 32LL * j;
        s = fma(val[k], x[col[k]], s);
    }
    store_row(y, r, s, alpha, beta, mode);
}

// ---------------------------------------------------------------------------
// BCSR (format conversion, R x R blocks): a thread per row walks its block
// row's blocks; the R threads of a block row share each block's column index
// and x segment and read consecutive rows of the block.  Zero-filled entries
// add fma(0, x, s) = s, and the entries come in ascending column order, so the
// row sum is the one k_row forms, bit for bit.
// ---------------------------------------------------------------------------
template <typename V, int R>
__global__ void __launch_bounds__(512) k_bcsr(int n, int ncols, const int *__restrict__ bptr,
                                              const int *__restrict__ bcol,
                                              const V *__restrict__ bval, const V *__restrict__ x,
                                              V alpha, V beta, int mode, V *__restrict__ y,
                                              const V *__restrict__ adev) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    if (adev) alpha = *adev;
    const int b = r / R, li = r - b * R;
    const int q0 = __ldg(bptr + b), q1 = __ldg(bptr + b + 1);
    V s = V(0);
    for (int q = q0; q < q1; q++) {
        const int c0 = __ldg(bcol + q) * R;
        const V *blk = bval + ((int64_t)q * R + li) * R;
        if (c0 + R <= ncols) {
#pragma unroll
            for (int j = 0; j < R; j++) s = fma(__ldg(blk + j), __ldg(x + c0 + j), s);
        } else {  // last block column when the column count is not a multiple of R
            for (int j = 0; c0 + j < ncols; j++) s = fma(__ldg(blk + j), __ldg(x + c0 + j), s);
        }
    }
    store_row(y, r, s, alpha, beta, mode);
}

template <typename V>
const V *bcsr_values(const xb::BcsrPart *bp);
template <>
const double *bcsr_values<double>(const xb::BcsrPart *bp) { return bp->d_val; }
template <>
const float *bcsr_values<float>(const xb::BcsrPart *bp) { return bp->d_val32; }

template <typename V>
int launch_bcsr(xb_plan *p, int block, int ipt, V alpha, const V *x, V beta, int mode, V *y,
                const V *adev, cudaStream_t s) {
    int err = XB_OK;
    const xb::BcsrPart *bp = xb::get_bcsr(p, ipt, sizeof(V) == sizeof(float), s, &err);
    if (!bp) return err;
    const int grid = (p->n + block - 1) / block;
    const V *bv = bcsr_values<V>(bp);
    switch (ipt) {
        case 2:
            k_bcsr<V, 2><<<grid, block, 0, s>>>(p->n, p->ncols, bp->d_bptr, bp->d_bcol, bv, x, alpha, beta,
                                                mode, y, adev);
            break;
        case 3:
            k_bcsr<V, 3><<<grid, block, 0, s>>>(p->n, p->ncols, bp->d_bptr, bp->d_bcol, bv, x, alpha, beta,
                                                mode, y, adev);
            break;
        case 4:
            k_bcsr<V, 4><<<grid, block, 0, s>>>(p->n, p->ncols, bp->d_bptr, bp->d_bcol, bv, x, alpha, beta,
                                                mode, y, adev);
            break;
        default:
            return xb::set_error(XB_EINVAL, "BCSR: block size %d not in {2, 3, 4}", ipt);
    }
    XB_LAUNCHED("k_bcsr");
    return XB_OK;
}

template <typename V>
const V *sell_values(const xb::SellPart *sp);
template <>
const double *sell_values<double>(const xb::SellPart *sp) { return sp->d_val; }
template <>
const float *sell_values<float>(const xb::SellPart *sp) { return sp->d_val32; }

template <typename V>
int launch_sell(xb_plan *p, int block, int ipt, V alpha, const V *x, V beta, int mode, V *y,
                const V *adev, cudaStream_t s) {
    if (ipt < 1 || ipt > 32) return xb::set_error(XB_EINVAL, "SELL: ipt %d not in 1..32", ipt);
    int err = XB_OK;
    const xb::SellPart *sp = xb::get_sell(p, 32 * ipt, sizeof(V) == sizeof(float), s, &err);
    if (!sp) return err;
    const int64_t threads = (int64_t)sp->nslices * 32;
    k_sell<V><<<(unsigned)((threads + block - 1) / block), block, 0, s>>>(
        sp->nslices, sp->d_off, sp->d_perm, sp->d_len, sp->d_col, sell_values<V>(sp), x, alpha,
        beta, mode, y, adev);
    XB_LAUNCHED("k_sell");
    return XB_OK;
}

template <typename V>
struct Vec2;
template <>
struct Vec2<double> {
    using T = double2;
    static constexpr int N = 2;
};
template <>
struct Vec2<float> {
    using T = float4;
    static constexpr int N = 4;
};

// ---------------------------------------------------------------------------
// U2: non-zero-balanced row decomposition (Sec. 3.2.2, Fig. 3) at warp
// granularity.  The plan cuts the rows into consecutive warp tiles of about
// equal non-zero count (at most 32*IPT, rows never split); a row too long for
// a tile gets a CTA.  Inside a tile the rows are binned by length:
//   kind 0 (every row at most IPT long, at most 32 rows): a thread per row,
//          operands straight from global memory -- on uniform short rows this
//          is the row decomposition U1 with 32 rows per warp;
//   kind 1 (some row longer): the tile's non-zeros are split flat over the
//          lanes, IPT consecutive ones each from an IPT-aligned window (16-byte
//          vector loads), row ends from the plan's bitmask, rows joined by a
//          key-segmented warp scan.  No row leaves the tile, so there is no
//          carry between warps and no fix-up launch.
// Long-row CTAs come first in the grid (they are the longest-running).
// ---------------------------------------------------------------------------
template <typename V, int IPT, int M>
__global__ void __launch_bounds__(512, (IPT <= 8 ? 3 : 1)) k_u2(int ntiles, int implicit, int nlong,
                                                               int n, int nnz,
                                            const int4 *__restrict__ tiles,
                                            const int *__restrict__ lrows,
                                            const int *__restrict__ rowptr,
                                            const int *__restrict__ col,
                                            const V *__restrict__ val, const V *__restrict__ x,
                                            V alpha, V beta, V *__restrict__ y,
                                            const unsigned *__restrict__ endbits,
                                            const int *__restrict__ ne_rows,
                                            const V *__restrict__ adev, int vec) {
    static_assert(IPT == 4 || IPT == 8 || IPT == 16, "IPT");
    __shared__ V red[32];
    const unsigned FULL = 0xffffffffu;
    if (adev) alpha = *adev;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((int)blockIdx.x < nlong) {  // one long row, whole CTA (CTA-uniform branch)
        const int r = lrows[blockIdx.x];
        const int a = rowptr[r], b = rowptr[r + 1], B = blockDim.x;
        V s0 = V(0), s1 = V(0);
        int k = a + threadIdx.x;
        for (; k + B < b; k += 2 * B) {
            const int c0 = __ldg(col + k), c1 = __ldg(col + k + B);
            const V v0 = __ldg(val + k), v1 = __ldg(val + k + B);
            s0 = fma(v0, __ldg(x + c0), s0);
            s1 = fma(v1, __ldg(x + c1), s1);
        }
        if (k < b) s0 = fma(__ldg(val + k), __ldg(x + __ldg(col + k)), s0);
        const V sum = xbd::block_sum(s0 + s1, red);
        if (threadIdx.x == 0) store_row(y, r, sum, alpha, beta, M);
        return;
    }
    const int t = ((int)blockIdx.x - nlong) * nw + wib;
    if (t >= ntiles) return;  // warp-uniform
    int r0, r1, ne0 = 0, kind = 0;
    if (implicit) {
        r0 = 32 * t;
        r1 = min(n, r0 + 32);
    } else {
        const int4 d = __ldg(tiles + t);
        r0 = d.x;
        r1 = d.y;
        ne0 = d.z;
        kind = d.w;
    }
    if ((kind & 3) == 0) {  // thread per row
        const int r = r0 + lane;
        if (r < r1) {
            const int a = __ldg(rowptr + r), b = __ldg(rowptr + r + 1);
            V s = V(0);
            for (int k = a; k < b; k++) s = fma(__ldg(val + k), __ldg(x + __ldg(col + k)), s);
            store_row(y, r, s, alpha, beta, M);
        }
        return;
    }
    // flat over the tile's IPT-aligned window
    const int k0 = __ldg(rowptr + r0), k1 = __ldg(rowptr + r1);
    const int e0 = k0 - k0 % IPT + lane * IPT;
    const int lo = max(0, k0 - e0), hi = min(IPT, k1 - e0);
    const unsigned vm = (hi > lo) ? (((1u << hi) - 1u) & ~((1u << lo) - 1u)) : 0u;
    unsigned fl = 0;
    if (vm) {  // IPT divides 32 and e0 is a multiple of IPT: one bitmask word
        const unsigned w = __ldg(endbits + (e0 >> 5));
        fl = (w >> (unsigned)(e0 & 31)) & vm;
    }
    const int cnt = __popc(fl);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += u;
    }
    int row = ne0 + incl - cnt;  // non-empty-row index of the lane's first entry
    V v[IPT];
    int c[IPT];
    if (vm && vec && e0 + IPT <= nnz) {
        using T2 = typename Vec2<V>::T;
        constexpr int VN = Vec2<V>::N;
        const T2 *vp = reinterpret_cast<const T2 *>(val + e0);
#pragma unroll
        for (int q = 0; q < IPT / VN; q++) {
            const T2 u = __ldg(vp + q);
            if constexpr (VN == 2) {
                v[2 * q] = u.x;
                v[2 * q + 1] = u.y;
            } else {
                v[4 * q] = u.x;
                v[4 * q + 1] = u.y;
                v[4 * q + 2] = u.z;
                v[4 * q + 3] = u.w;
            }
        }
        const int4 *cp = reinterpret_cast<const int4 *>(col + e0);
#pragma unroll
        for (int q = 0; q < IPT / 4; q++) {
            const int4 u = __ldg(cp + q);
            c[4 * q] = u.x;
            c[4 * q + 1] = u.y;
            c[4 * q + 2] = u.z;
            c[4 * q + 3] = u.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < IPT; j++) {
            const bool ok = (vm >> j) & 1u;
            c[j] = ok ? __ldg(col + e0 + j) : 0;
            v[j] = ok ? __ldg(val + e0 + j) : V(0);
        }
    }
    V xv[IPT];
#pragma unroll
    for (int j = 0; j < IPT; j++) {  // window entries of other tiles count as 0
        const bool ok = (vm >> j) & 1u;
        xv[j] = ok ? __ldg(x + c[j]) : V(0);
        v[j] = ok ? v[j] : V(0);
    }
    V sum = V(0), head = V(0);
    int hrow = -1, hkey = -1;
#pragma unroll
    for (int j = 0; j < IPT; j++) {
        sum = fma(v[j], xv[j], sum);
        if ((fl >> j) & 1u) {
            const int rid = ne_rows ? __ldg(ne_rows + row) : row;
            if (hkey < 0) {
                head = sum;
                hrow = rid;
                hkey = row;
            } else {
                store_row(y, rid, sum, alpha, beta, M);
            }
            sum = V(0);
            row++;
        }
    }
    // key-segmented inclusive scan of (row, sum); keys ascend with the lane
    int k = vm ? row : INT_MAX;
    V s = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int ku = __shfl_up_sync(FULL, k, o);
        const bool need = lane >= o && ku == k;
        if (!__any_sync(FULL, need)) break;
        const V su = __shfl_up_sync(FULL, s, o);
        if (need) s += su;
    }
    const int kp = __shfl_up_sync(FULL, k, 1);
    const V sp = __shfl_up_sync(FULL, s, 1);
    const bool addc = lane > 0 && hkey >= 0 && kp == hkey;
    if (__any_sync(FULL, addc))
        if (addc) head += sp;
    if (hkey >= 0) store_row(y, hrow, head, alpha, beta, M);
    if (kind & 4)  // the tile's empty rows
        for (int r = r0 + lane; r < r1; r += 32)
            if (__ldg(rowptr + r) == __ldg(rowptr + r + 1))
                y[r] = (M == 2) ? beta * y[r] : V(0);
}

// Thread-per-row U2 tiles when the balanced partition is 32-row blocks of
// short rows (every tile kind 0, implicit): U1's loop with 32 rows per warp.
template <typename V, int M>
__global__ void __launch_bounds__(512) k_u2_rows(int n, const int *__restrict__ rowptr,
                                                 const int *__restrict__ col,
                                                 const V *__restrict__ val,
                                                 const V *__restrict__ x, V alpha, V beta,
                                                 V *__restrict__ y, const V *__restrict__ adev) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    if (adev) alpha = *adev;
    const int a = __ldg(rowptr + r), b = __ldg(rowptr + r + 1);
    V s = V(0);
    for (int k = a; k < b; k++) s = fma(__ldg(val + k), __ldg(x + __ldg(col + k)), s);
    store_row(y, r, s, alpha, beta, M);
}

// ---------------------------------------------------------------------------
// U3 (BSS): flat nnz segments.  CTA b owns non-zeros [b*T, b*T+T); thread t
// owns IPT consecutive ones.  val and col are staged with coalesced loads
// into a padded shared layout (stride IPT+1, conflict-free per-thread reads),
// the thread's start row comes from a binary search in the CTA's staged
// rowptr slice, and each thread runs its IPT FMAs with row breaks as
// predicated stores (no data-dependent loop).  Partial sums of rows that
// straddle threads are combined by a key-segmented scan (warp shuffles, then
// across warps), rows straddling CTAs by a deterministic carry fix-up.
// ---------------------------------------------------------------------------
template <typename V, int IPT>
__global__ void __launch_bounds__(512) k_seg(int n, int nnz, const int *__restrict__ rowptr,
                                             const int *__restrict__ col,
                                             const V *__restrict__ val, const V *__restrict__ x,
                                             V alpha, V beta, int mode, V *__restrict__ y,
                                             const int *__restrict__ brow, V *__restrict__ cval,
                                             int *__restrict__ crow, const V *__restrict__ adev) {
    extern __shared__ __align__(16) unsigned char sm_[];
    const int B = blockDim.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (adev) alpha = *adev;
    const int T = B * IPT, TP = T + B;
    const int E0 = blockIdx.x * T;
    const int cnt = min(T, nnz - E0);
    const int rb = brow[blockIdx.x], re = brow[blockIdx.x + 1];
    V *sv = reinterpret_cast<V *>(sm_);
    V *wsum = sv + TP;   // 32
    V *wtot = wsum + 32; // 32
    int *sc = reinterpret_cast<int *>(wtot + 32);
    int *srp = sc + TP;  // T + 2
    int *wkf = srp + T + 2, *wkl = wkf + 32;

    {
        int c[IPT];
        V v[IPT];
#pragma unroll
        for (int j = 0; j < IPT; j++) {
            const int e = tid + j * B;
            if (e < cnt) {
                c[j] = col[E0 + e];
                v[j] = val[E0 + e];
            }
        }
#pragma unroll
        for (int j = 0; j < IPT; j++) {
            const int e = tid + j * B;
            if (e < cnt) {
                const int p = e + e / IPT;
                sv[p] = v[j];
                sc[p] = c[j];
            }
        }
    }
    const int nr = re - rb + 2;  // rowptr[rb .. re+1], clamped to n
    const bool big = nr > T + 2;
    if (!big)
        for (int i = tid; i < nr; i += B) srp[i] = rowptr[min(rb + i, n)];
    __syncthreads();
#define RP(r) (big ? rowptr[min((r), n)] : srp[(r) - rb])

    const int el = tid * IPT;
    const int ecnt = max(0, min(IPT, cnt - el));
    const int p0 = tid * (IPT + 1);
    int row = INT_MAX;
    V sum = V(0), head = V(0);
    int hrow = -1;
    if (ecnt > 0) {
        const int target = E0 + el;
        int lo = rb, hi = re;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (RP(mid) <= target) lo = mid;
            else hi = mid - 1;
        }
        row = lo;
        V xv[IPT];
#pragma unroll
        for (int j = 0; j < IPT; j++)
            if (j < ecnt) {  // unvalidated caller arrays: a column outside [0, n) adds 0
                const int cj = sc[p0 + j];
                xv[j] = ((unsigned)cj < (unsigned)n) ? x[cj] : V(0);
            }
        int nend = RP(row + 1) - E0;
#pragma unroll
        for (int j = 0; j < IPT; j++) {
            if (j < ecnt) {
                sum = fma(sv[p0 + j], xv[j], sum);
                const int le = el + j + 1;
                if (le == nend) {
                    if (hrow < 0) {
                        head = sum;
                        hrow = row;
                    } else if (row < n) {
                        store_row(y, row, sum, alpha, beta, mode);
                    }
                    sum = V(0);
                    do {
                        row++;
                        nend = RP(row + 1) - E0;
                    } while (nend == le && row < n);
                }
            }
        }
    }
#undef RP
    // key-segmented inclusive scan of (row, sum) over the CTA
    V s = sum;
    int k = row;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const V su = __shfl_up_sync(0xffffffffu, s, o);
        const int ku = __shfl_up_sync(0xffffffffu, k, o);
        if (lane >= o && ku == k) s += su;
    }
    if (lane == 31) {
        wsum[wid] = s;
        wkl[wid] = k;
    }
    if (lane == 0) wkf[wid] = k;
    __syncthreads();
    const int nw = B >> 5;
    if (wid == 0) {
        // segmented scan over warp tails: warp l continues warp l-1's tail run
        // when the whole warp carries that one key.
        V ts = lane < nw ? wsum[lane] : V(0);
        int f = 1;
        if (lane < nw && lane > 0) f = !(wkf[lane] == wkl[lane] && wkl[lane - 1] == wkl[lane]);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const V su = __shfl_up_sync(0xffffffffu, ts, o);
            const int fu = __shfl_up_sync(0xffffffffu, f, o);
            if (lane >= o && !f) {
                ts += su;
                f |= fu;
            }
        }
        if (lane < nw) wtot[lane] = ts;
    }
    __syncthreads();
    if (wid > 0 && k == wkf[wid] && wkl[wid - 1] == k) s += wtot[wid - 1];
    V sp = __shfl_up_sync(0xffffffffu, s, 1);
    int kp = __shfl_up_sync(0xffffffffu, k, 1);
    if (lane == 0) {
        if (wid > 0) {
            sp = wtot[wid - 1];
            kp = wkl[wid - 1];
        } else {
            sp = V(0);
            kp = -1;
        }
    }
    if (hrow >= 0 && hrow < n) store_row(y, hrow, head + (kp == hrow ? sp : V(0)), alpha, beta, mode);
    if (cnt > 0 && tid == (cnt - 1) / IPT) {
        crow[blockIdx.x] = k;
        cval[blockIdx.x] = s;
    }
}

// ---------------------------------------------------------------------------
// U3 (BSS) with the plan's row-end bitmask ("a data format representing the
// continuous location", Sec. 3.2.2).  Warp w owns non-zeros [w*32*IPT, ...),
// lane l the IPT consecutive ones from w*32*IPT + l*IPT.  The lane's values
// and columns come from the plan's BSS data format copy (values and columns in
// the order the warps read them), so each 16-byte vector load of the warp
// reads 512 consecutive bytes; no staging, no row search: the lane's start
// row is the warp's start row plus the row ends that precede it (integer warp
// scan of popcounts of its flag bits).  The inner loop is IPT FMAs with row
// ends as predicated stores.  Row sums that straddle lanes are joined by a
// key-segmented warp scan that stops as soon as no lane needs another step
// (most steps cost no FP64 instruction); rows that straddle warps go through
// one carry slot per warp and the fix-up.
//
// On GB300 this kernel is bound by the rate of L1 -> L2 requests (about one
// per SM per clock): every x gather of a random column is one request, so
// what is left to save is the streamed operands' requests.  With the copy a
// warp's 256 values and columns (IPT = 8) take 24 line requests instead of
// the 80 that lane-strided loads of the caller's arrays need.
// ---------------------------------------------------------------------------
template <typename V, int IPT, int M, bool NE>
__global__ void __launch_bounds__(256) k_bss(int nnz, int nwarps, const int *__restrict__ col_il,
                                             const V *__restrict__ val_il, const V *__restrict__ x,
                                             V alpha, V beta, V *__restrict__ y,
                                             const unsigned *__restrict__ endbits,
                                             const int *__restrict__ wrow,
                                             const int *__restrict__ ne_rows, int n_ne, int n,
                                             V *__restrict__ cval, int *__restrict__ crow,
                                             const V *__restrict__ adev) {
    static_assert(IPT == 4 || IPT == 8 || IPT == 16 || IPT == 32, "IPT");
    // the carry fix-up may be scheduled as soon as every CTA of this grid has
    // started (it waits for this grid's completion before reading anything)
    asm volatile("griddepcontrol.launch_dependents;");
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (gw >= nwarps) return;  // warp-uniform
    if (adev) alpha = *adev;
    const long long E = gw * 32 * IPT;
    const long long e0 = E + lane * IPT;
    const int ecnt = (int)max(0LL, min((long long)IPT, (long long)nnz - e0));
    unsigned fl = 0;
    if (ecnt > 0) {
        const unsigned w = __ldg(endbits + (e0 >> 5));
        fl = (IPT == 32) ? w : (w >> (unsigned)(e0 & 31)) & ((1u << IPT) - 1u);
        if (ecnt < IPT) fl &= (1u << ecnt) - 1u;
    }
    const int cnt = __popc(fl);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += t;
    }
    int row = __ldg(wrow + gw) + incl - cnt;  // index over non-empty rows
    // The copy is padded to whole warp chunks: every load is a full vector.
    V v[IPT];
    int c[IPT];
    {
        using T2 = typename Vec2<V>::T;
        constexpr int VN = Vec2<V>::N;
        const T2 *vp = reinterpret_cast<const T2 *>(val_il + E);
#pragma unroll
        for (int q = 0; q < IPT / VN; q++) {
            const T2 t = __ldg(vp + q * 32 + lane);
            if constexpr (VN == 2) {
                v[2 * q] = t.x;
                v[2 * q + 1] = t.y;
            } else {
                v[4 * q] = t.x;
                v[4 * q + 1] = t.y;
                v[4 * q + 2] = t.z;
                v[4 * q + 3] = t.w;
            }
        }
        const int4 *cp = reinterpret_cast<const int4 *>(col_il + E);
#pragma unroll
        for (int q = 0; q < IPT / 4; q++) {
            const int4 t = __ldg(cp + q * 32 + lane);
            c[4 * q] = t.x;
            c[4 * q + 1] = t.y;
            c[4 * q + 2] = t.z;
            c[4 * q + 3] = t.w;
        }
    }
    V xv[IPT];
#pragma unroll
    for (int j = 0; j < IPT; j++) xv[j] = (j < ecnt) ? __ldg(x + c[j]) : V(0);
    V sum = V(0), head = V(0);
    int hrow = -1, hkey = -1;
#pragma unroll
    for (int j = 0; j < IPT; j++) {
        sum = fma(v[j], xv[j], sum);
        if ((fl >> j) & 1u) {
            const int rid = NE ? __ldg(ne_rows + row) : row;
            if (hkey < 0) {
                head = sum;
                hrow = rid;
                hkey = row;
            } else {
                store_row(y, rid, sum, alpha, beta, M);
            }
            sum = V(0);
            row++;
        }
    }
    // key-segmented inclusive scan of (row, sum); keys ascend with the lane
    int k = (ecnt > 0) ? row : INT_MAX;
    V s = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int ku = __shfl_up_sync(FULL, k, o);
        const bool need = lane >= o && ku == k;
        if (!__any_sync(FULL, need)) break;  // no longer run at this distance: done
        const V su = __shfl_up_sync(FULL, s, o);
        if (need) s += su;
    }
    const int kp = __shfl_up_sync(FULL, k, 1);
    const V sp = __shfl_up_sync(FULL, s, 1);
    const bool addc = lane > 0 && hkey >= 0 && kp == hkey;
    if (__any_sync(FULL, addc))
        if (addc) head += sp;
    if (hkey >= 0) store_row(y, hrow, head, alpha, beta, M);
    // the warp's carry: the last lane holding a non-zero
    const long long left = (long long)nnz - gw * 32 * IPT;
    const int last = (int)min(31LL, (left - 1) / IPT);
    if (lane == last) {
        crow[gw] = (k < n_ne) ? (NE ? __ldg(ne_rows + k) : k) : n;
        cval[gw] = s;
    }
}

// Adds each run of equal carry rows, in CTA order (deterministic).  Launched
// as a programmatic dependent of k_bss, it waits here until k_bss has
// finished and its writes are visible (a no-op for an ordinary launch).
template <typename V>
__global__ void k_seg_fix(int nblk, int n, const int *__restrict__ crow, const V *__restrict__ cval,
                          V alpha, int mode, V *__restrict__ y, const V *__restrict__ adev) {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nblk) return;
    if (adev) alpha = *adev;
    const int r = crow[b];
    if (r >= n || (b > 0 && crow[b - 1] == r)) return;
    // the run of carries of row r, added in storage order; eight carries are
    // loaded per round, so a row spanning many warps costs few round trips
    V s = cval[b];
    for (int q = b + 1; q < nblk; q += 8) {
        int rr[8];
        V cc[8];
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const bool in = q + u < nblk;
            rr[u] = in ? crow[q + u] : -1;
            cc[u] = in ? cval[q + u] : V(0);
        }
        bool more = true;
#pragma unroll
        for (int u = 0; u < 8; u++) {
            more = more && rr[u] == r;
            if (more) s += cc[u];
        }
        if (!more) break;
    }
    y[r] += (mode == 0) ? s : alpha * s;
}

template <typename V>
__global__ void k_empty_rows(int cnt, const int *__restrict__ rows, V beta, int mode,
                             V *__restrict__ y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    const int r = rows[i];
    y[r] = (mode == 2) ? beta * y[r] : V(0);
}

template <typename V>
__global__ void k_yscale(int n, V beta, V *__restrict__ y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = (beta == V(0)) ? V(0) : beta * y[i];
}

// ---------------------------------------------------------------------------
// S1-like baseline: thread per upper row; the row part is a plain FMA sum,
// every transpose term u*x_i goes to y[j] through a device FP64 atomic (an
// L2 reduction, no FP64 work on the SM).  y must hold beta*y beforehand.
// ---------------------------------------------------------------------------
template <typename V, bool A1>
__global__ void __launch_bounds__(512) k_sym_atomic(int n, const int *__restrict__ rowptr,
                                                    const int *__restrict__ col,
                                                    const V *__restrict__ val,
                                                    const V *__restrict__ x, V alpha,
                                                    V *__restrict__ y, const V *__restrict__ adev) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    if (!A1 && adev) alpha = *adev;
    const int a = rowptr[r], b = rowptr[r + 1];
    const V axi = A1 ? x[r] : alpha * x[r];
    V s = V(0);
    for (int k = a; k < b; k++) {
        const int j = col[k];
        const V u = val[k];
        s = fma(u, x[j], s);
        if (j != r) atomicAdd(&y[j], u * axi);
    }
    atomicAdd(&y[r], A1 ? s : alpha * s);
}

// ---------------------------------------------------------------------------
// S2/S3-like: the U2 tile partition over the upper rows.  Transpose terms
// whose target row lies inside the tile are summed in a shared-memory
// vector for the tile's rows; only the tile's out-of-tile targets (the
// non-zero region beyond the tile) reach device memory, as FP64 atomics.
// Each tile row is then added to y once.  y must hold beta*y beforehand.
// ---------------------------------------------------------------------------
template <typename V, int IPT, bool A1>
__global__ void __launch_bounds__(512) k_sym_tile(const int *__restrict__ rowptr,
                                                  const int *__restrict__ col,
                                                  const V *__restrict__ val,
                                                  const V *__restrict__ x, V alpha,
                                                  V *__restrict__ y,
                                                  const int *__restrict__ trow,
                                                  const V *__restrict__ adev) {
    extern __shared__ __align__(16) unsigned char sm_[];
    const int B = blockDim.x, tid = threadIdx.x;
    const int T = B * IPT;
    if (!A1 && adev) alpha = *adev;
    const int r0 = trow[blockIdx.x], r1 = trow[blockIdx.x + 1];
    const int k0 = rowptr[r0], k1 = rowptr[r1];
    const int cnt = k1 - k0;
    V *red = reinterpret_cast<V *>(sm_);  // 32
    if (cnt > T) {  // one long row r0: whole CTA
        const V axi = A1 ? x[r0] : alpha * x[r0];
        V s = V(0);
        for (int e = k0 + tid; e < k1; e += B) {
            const int j = col[e];
            const V u = val[e];
            s = fma(u, x[j], s);
            if (j != r0) atomicAdd(&y[j], u * axi);
        }
        s = xbd::block_sum(s, red);
        if (tid == 0) atomicAdd(&y[r0], A1 ? s : alpha * s);
        return;
    }
    V *acc = red + 32;     // B
    V *sv = acc + B;       // T
    int *sc = reinterpret_cast<int *>(sv + T);  // T
    int *srp = sc + T;     // B + 1
    {
        int c[IPT];
        V v[IPT];
#pragma unroll
        for (int j = 0; j < IPT; j++) {
            const int e = tid + j * B;
            if (e < cnt) {
                c[j] = col[k0 + e];
                v[j] = val[k0 + e];
            }
        }
#pragma unroll
        for (int j = 0; j < IPT; j++) {
            const int e = tid + j * B;
            if (e < cnt) {
                sc[e] = c[j];
                sv[e] = v[j];
            }
        }
    }
    const int nr = r1 - r0;
    for (int i = tid; i <= nr; i += B) srp[i] = rowptr[r0 + i] - k0;
    for (int i = tid; i < nr; i += B) acc[i] = V(0);
    __syncthreads();
    V s = V(0);
    if (tid < nr) {
        const int r = r0 + tid;
        const V axi = A1 ? x[r] : alpha * x[r];
        const int a = srp[tid], b = srp[tid + 1];
        for (int e = a; e < b; e++) {
            const int j = sc[e];
            const V u = sv[e];
            s = fma(u, x[j], s);
            if (j != r) {
                if (j < r1) atomicAdd(&acc[j - r0], u * axi);
                else atomicAdd(&y[j], u * axi);
            }
        }
    }
    __syncthreads();
    if (tid < nr) atomicAdd(&y[r0 + tid], A1 ? s + acc[tid] : fma(alpha, s, acc[tid]));
}

// ---------------------------------------------------------------------------
// S3: zero-element omission (Sec. 3.2.2, S3).  The S2 tile partition; each
// CTA sums the transpose terms of its rows into shared-memory partial vectors
// that cover only where they land: the tile's own rows, and the granules of
// kS3Gran rows beyond the tile that the plan listed for it (at most kS3Max).
// The CTA writes each of its rows once (alpha * (row sum + in-tile transposes)
// + beta * y) and its granule partials to its slots in device memory; the
// reduction launch then adds, for every granule some tile reaches, its slots
// in tile order.  Granules no tile reaches -- the all-zero parts of the
// partial vectors -- are neither stored nor read.  No device atomics; the
// shared-memory sums are atomic (their order varies between launches).
// ---------------------------------------------------------------------------
template <typename V, int IPT, bool A1>
__global__ void __launch_bounds__(512) k_sym_s3(const int *__restrict__ rowptr,
                                                const int *__restrict__ col,
                                                const V *__restrict__ val, const V *__restrict__ x,
                                                V alpha, V beta, int mode, V *__restrict__ y,
                                                const int *__restrict__ trow,
                                                const int *__restrict__ tslot,
                                                const int *__restrict__ sgran, V *__restrict__ part,
                                                const V *__restrict__ adev) {
    extern __shared__ __align__(16) unsigned char sm_[];
    const int B = blockDim.x, tid = threadIdx.x;
    const int T = B * IPT;
    if (!A1 && adev) alpha = *adev;
    const int t = blockIdx.x;
    const int r0 = trow[t], r1 = trow[t + 1];
    const int k0 = rowptr[r0], k1 = rowptr[r1];
    const int cnt = k1 - k0, nr = r1 - r0;
    const int s0 = tslot[t], ns = tslot[t + 1] - s0;
    V *gp = reinterpret_cast<V *>(sm_);      // kS3Max * kS3Gran
    V *acc = gp + xb::kS3Max * xb::kS3Gran;  // B
    V *red = acc + B;                        // 32
    V *sv = red + 32;                        // T
    int *sc = reinterpret_cast<int *>(sv + T);  // T
    int *srp = sc + T;                       // B + 1
    int *gid = srp + B + 1;                  // kS3Max
    for (int i = tid; i < ns * xb::kS3Gran; i += B) gp[i] = V(0);
    for (int i = tid; i < B; i += B) acc[i] = V(0);
    if (tid < ns) gid[tid] = sgran[s0 + tid];
    // transpose term u * x_r of stored (r, j, u), j != r: in-tile row or granule slot
    auto scatter = [&](int j, V tv) {
        if (j < r1) {
            atomicAdd(&acc[j - r0], tv);
        } else {
            const int g = j / xb::kS3Gran;
            int q = 0;
            while (q + 1 < ns && gid[q] != g) q++;
            atomicAdd(&gp[q * xb::kS3Gran + (j - g * xb::kS3Gran)], tv);
        }
    };
    if (cnt > T) {  // one long row r0, whole CTA
        __syncthreads();
        const V xr = x[r0];
        V sr = V(0);
        for (int e = k0 + tid; e < k1; e += B) {
            const int j = col[e];
            const V u = val[e];
            sr = fma(u, x[j], sr);
            if (j != r0) scatter(j, u * xr);
        }
        sr = xbd::block_sum(sr, red);
        __syncthreads();
        if (tid == 0) store_row(y, r0, sr + acc[0], alpha, beta, mode);
    } else {
        {
            int c[IPT];
            V v[IPT];
#pragma unroll
            for (int j = 0; j < IPT; j++) {
                const int e = tid + j * B;
                if (e < cnt) {
                    c[j] = col[k0 + e];
                    v[j] = val[k0 + e];
                }
            }
#pragma unroll
            for (int j = 0; j < IPT; j++) {
                const int e = tid + j * B;
                if (e < cnt) {
                    sc[e] = c[j];
                    sv[e] = v[j];
                }
            }
        }
        for (int i = tid; i <= nr; i += B) srp[i] = rowptr[r0 + i] - k0;
        __syncthreads();
        V sr = V(0);
        if (tid < nr) {
            const int r = r0 + tid;
            const V xr = x[r];
            for (int e = srp[tid]; e < srp[tid + 1]; e++) {
                const int j = sc[e];
                const V u = sv[e];
                sr = fma(u, x[j], sr);
                if (j != r) scatter(j, u * xr);
            }
        }
        __syncthreads();
        if (tid < nr) store_row(y, r0 + tid, sr + acc[tid], alpha, beta, mode);
    }
    __syncthreads();
    for (int i = tid; i < ns * xb::kS3Gran; i += B) part[(size_t)s0 * xb::kS3Gran + i] = gp[i];
}

// Adds the partials of one reached granule (one CTA of kS3Gran threads).
template <typename V>
__global__ void __launch_bounds__(xb::kS3Gran) k_sym_s3_red(int n, const int *__restrict__ gid,
                                                            const int *__restrict__ gptr,
                                                            const int *__restrict__ gslot,
                                                            const V *__restrict__ part, V alpha,
                                                            V *__restrict__ y,
                                                            const V *__restrict__ adev) {
    if (adev) alpha = *adev;
    const int c = blockIdx.x;
    const int i = gid[c] * xb::kS3Gran + threadIdx.x;
    if (i >= n) return;
    V sum = V(0);
    for (int q = gptr[c]; q < gptr[c + 1]; q++)
        sum += part[(size_t)gslot[q] * xb::kS3Gran + threadIdx.x];
    y[i] += alpha * sum;
}

// ---------------------------------------------------------------------------
// S1 with warp-aggregated atomics: a thread per upper row; the warp walks its
// rows' entries in lock step, and lanes whose transpose terms go to the same
// row add them (in lane order) before one device atomic per distinct row.
// y must hold beta*y beforehand.
// ---------------------------------------------------------------------------
template <typename V, bool A1>
__global__ void __launch_bounds__(512) k_sym_wagg(int n, const int *__restrict__ rowptr,
                                                  const int *__restrict__ col,
                                                  const V *__restrict__ val,
                                                  const V *__restrict__ x, V alpha,
                                                  V *__restrict__ y, const V *__restrict__ adev) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (!A1 && adev) alpha = *adev;
    const bool has = r < n;
    const int a = has ? rowptr[r] : 0, b = has ? rowptr[r + 1] : 0;
    int len = b - a, L = len;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) L = max(L, __shfl_xor_sync(FULL, L, o));
    const V axi = has ? (A1 ? x[r] : alpha * x[r]) : V(0);
    V s = V(0);
    for (int q = 0; q < L; q++) {  // warp-uniform trip count
        const bool act = q < len;
        int j = -1;
        V tv = V(0);
        if (act) {
            j = col[a + q];
            const V u = val[a + q];
            s = fma(u, x[j], s);
            if (j != r) tv = u * axi;
            else j = -1;
        }
        const int key = (j >= 0) ? j : -1 - lane;  // lanes with no transpose term: own key
        const unsigned m = __match_any_sync(FULL, key);
        V tot = tv;
        if (__popc(m) > 1) {  // add the group's terms in lane order
            tot = V(0);
            for (unsigned mm = m; mm; mm &= mm - 1) tot += __shfl_sync(m, tv, __ffs(mm) - 1);
        }
        if (j >= 0 && lane == __ffs(m) - 1) atomicAdd(&y[j], tot);
    }
    if (has) atomicAdd(&y[r], A1 ? s : alpha * s);
}

// Opt every kernel instantiation into the device's full shared-memory
// capacity once (the launch size decides the occupancy).
int smem_limit() {
    static int maxs = -1;
    if (maxs < 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&maxs, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    }
    return maxs;
}

int smem_optin(const void *fn, size_t need) {
    static std::mutex mu;
    static std::unordered_set<const void *> done;
    if (need > (size_t)smem_limit())
        return xb::set_error(XB_EINVAL, "launch shape needs %zu B shared memory (> %d)", need,
                             smem_limit());
    std::lock_guard<std::mutex> g(mu);
    if (!done.count(fn)) {
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_limit());
        done.insert(fn);
    }
    return XB_OK;
}

template <typename V>
int launch_u2(xb_plan *p, const int *rp, const int *ci, const V *va, int block, int ipt, V alpha,
              const V *x, V beta, int mode, V *y, const V *adev, cudaStream_t s) {
    int err = XB_OK;
    const xb::U2Part *up = xb::get_u2(p, ipt, s, &err);
    if (!up) return err;
    if (up->ntiles + up->nlong == 0) return XB_OK;
    const int nw = block / 32;
    const int grid = up->nlong + (up->ntiles + nw - 1) / nw;
    const int vec = (((uintptr_t)va % 16) == 0 && ((uintptr_t)ci % 16) == 0) ? 1 : 0;
    const xb::BssData &bd = p->bss;
#define XB_U2(I)                                                                            \
    case I:                                                                                 \
        if (mode == 0) XB_U2M(I, 0) else if (mode == 1) XB_U2M(I, 1) else XB_U2M(I, 2)      \
        break;
#define XB_U2M(I, MM)                                                                       \
    {                                                                                       \
        k_u2<V, I, MM><<<grid, block, 0, s>>>(up->ntiles, up->implicit ? 1 : 0, up->nlong,    \
                                              p->n, p->nnz, up->d_tile, up->d_long, rp, ci,  \
                                              va, x, alpha, beta, y, bd.d_endbits,           \
                                              bd.d_ne_rows, adev, vec);                      \
    }
    if (up->implicit) {  // uniform short rows: the light thread-per-row kernel
        const int g = (p->n + block - 1) / block;
        if (mode == 0)
            k_u2_rows<V, 0><<<g, block, 0, s>>>(p->n, rp, ci, va, x, alpha, beta, y, adev);
        else if (mode == 1)
            k_u2_rows<V, 1><<<g, block, 0, s>>>(p->n, rp, ci, va, x, alpha, beta, y, adev);
        else
            k_u2_rows<V, 2><<<g, block, 0, s>>>(p->n, rp, ci, va, x, alpha, beta, y, adev);
        XB_LAUNCHED("k_u2_rows");
        return XB_OK;
    }
    switch (ipt) {
        XB_U2(4) XB_U2(8) XB_U2(16)
        default: return xb::set_error(XB_EINVAL, "nnz-balanced: unsupported ipt %d", ipt);
    }
#undef XB_U2
#undef XB_U2M
    XB_LAUNCHED("k_u2");
    return XB_OK;
}

template <typename V>
const V *bss_values(const xb::BssCopy *c);
template <>
const double *bss_values<double>(const xb::BssCopy *c) { return c->d_val; }
template <>
const float *bss_values<float>(const xb::BssCopy *c) { return c->d_val32; }

template <typename V>
int launch_seg(xb_plan *p, const int *rp, const int *ci, const V *va, int block, int ipt, V alpha,
               const V *x, V beta, int mode, V *y, const V *adev, cudaStream_t s) {
    (void)rp;
    (void)ci;
    (void)va;
    if (block > 256)
        return xb::set_error(XB_EINVAL, "segscan: block %d > 256", block);
    int err = XB_OK;
    const xb::SegPart *sp = xb::get_segs(p, block, ipt, s, &err);
    if (!sp) return err;
    const xb::BssData &bd = p->bss;
    if (sp->nblk > 0) {
        const xb::BssCopy *cp = xb::get_bss_copy(p, ipt, sizeof(V) == sizeof(float), s, &err);
        if (!cp) return err;
        const V *vil = bss_values<V>(cp);
        V *cv = reinterpret_cast<V *>(sp->d_carry_val);
        const int wpb = block / 32;
        const int grid = (sp->nblk + wpb - 1) / wpb;
#define XB_BSS(I)                                                                            \
    case I:                                                                                  \
        if (mode == 0) XB_BSSM(I, 0) else if (mode == 1) XB_BSSM(I, 1) else XB_BSSM(I, 2)     \
        break;
#define XB_BSSM(I, MM)                                                                       \
    {                                                                                        \
        if (bd.d_ne_rows)                                                                    \
            k_bss<V, I, MM, true><<<grid, block, 0, s>>>(                                    \
                p->nnz, sp->nblk, cp->d_col, vil, x, alpha, beta, y, bd.d_endbits, sp->d_row, \
                bd.d_ne_rows, bd.n_ne, p->n, cv, sp->d_carry_row, adev);                     \
        else                                                                                 \
            k_bss<V, I, MM, false><<<grid, block, 0, s>>>(                                   \
                p->nnz, sp->nblk, cp->d_col, vil, x, alpha, beta, y, bd.d_endbits, sp->d_row, \
                bd.d_ne_rows, bd.n_ne, p->n, cv, sp->d_carry_row, adev);                     \
    }
        switch (ipt) {
            XB_BSS(4) XB_BSS(8) XB_BSS(16) XB_BSS(32)
            default: return xb::set_error(XB_EINVAL, "segscan: unsupported ipt %d", ipt);
        }
#undef XB_BSS
#undef XB_BSSM
        XB_LAUNCHED("k_bss");
        {  // programmatic dependent launch: no idle gap between the two kernels
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3((unsigned)((sp->nblk + 255) / 256));
            cfg.blockDim = dim3(256);
            cfg.stream = s;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            at[0].val.programmaticStreamSerializationAllowed = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            const int *cr = sp->d_carry_row;
            const V *cvc = cv;
            XB_CUDA(cudaLaunchKernelEx(&cfg, k_seg_fix<V>, sp->nblk, p->n, cr, cvc, alpha, mode, y,
                                       adev));
        }
        XB_LAUNCHED("k_seg_fix");
    }
    if (p->n_empty > 0) {
        k_empty_rows<V><<<(p->n_empty + 255) / 256, 256, 0, s>>>(p->n_empty, p->d_empty, beta,
                                                                  mode, y);
        XB_LAUNCHED("k_empty_rows");
    }
    return XB_OK;
}

template <typename V>
int launch_sym(xb_plan *p, int variant, const int *rp, const int *ci, const V *va, int block,
               int ipt, V alpha, const V *x, V beta, V *y, const V *adev, cudaStream_t s) {
    const int n = p->n;
    if (n == 0) return XB_OK;
    const bool a1 = (adev == nullptr && alpha == V(1));
    if (variant == XB_VAR_SYM_PART) {
        int err = XB_OK;
        const xb::TilePart *tp = xb::get_tiles(p, block, ipt, s, &err);
        if (!tp) return err;
        const xb::S3Part *sp = xb::get_s3(p, block, ipt, s, &err);
        if (!sp) return err;
        const int mode = adev ? 1 : (beta == V(0)) ? (alpha == V(1) ? 0 : 1) : 2;
        const size_t sm = ((size_t)xb::kS3Max * xb::kS3Gran + block + 32 + (size_t)block * ipt) *
                              sizeof(V) +
                          (size_t)block * ipt * 4 + (block + 1) * 4 + xb::kS3Max * 4;
        V *part = reinterpret_cast<V *>(sp->d_part);
#define XB_S3(I)                                                                                \
    case I:                                                                                     \
        if (a1) {                                                                               \
            XB_TRY(smem_optin((const void *)k_sym_s3<V, I, true>, sm));                          \
            k_sym_s3<V, I, true><<<sp->ntiles, block, sm, s>>>(rp, ci, va, x, alpha, beta, mode,  \
                                                              y, tp->d_row, sp->d_tslot,        \
                                                              sp->d_sgran, part, adev);         \
        } else {                                                                                \
            XB_TRY(smem_optin((const void *)k_sym_s3<V, I, false>, sm));                         \
            k_sym_s3<V, I, false><<<sp->ntiles, block, sm, s>>>(rp, ci, va, x, alpha, beta,      \
                                                               mode, y, tp->d_row, sp->d_tslot, \
                                                               sp->d_sgran, part, adev);        \
        }                                                                                       \
        break;
        switch (ipt) {
            XB_S3(1) XB_S3(2) XB_S3(4) XB_S3(8) XB_S3(16)
            default: return xb::set_error(XB_EINVAL, "sym S3: unsupported ipt %d", ipt);
        }
#undef XB_S3
        XB_LAUNCHED("k_sym_s3");
        if (sp->ngran > 0) {
            k_sym_s3_red<V><<<sp->ngran, xb::kS3Gran, 0, s>>>(n, sp->d_gid, sp->d_gptr, sp->d_gslot,
                                                              part, alpha, y, adev);
            XB_LAUNCHED("k_sym_s3_red");
        }
        return XB_OK;
    }
    k_yscale<V><<<(n + 255) / 256, 256, 0, s>>>(n, beta, y);
    XB_LAUNCHED("k_yscale");
    if (variant == XB_VAR_SYM_WAGG) {
        if (a1)
            k_sym_wagg<V, true><<<(n + block - 1) / block, block, 0, s>>>(n, rp, ci, va, x, alpha, y, adev);
        else
            k_sym_wagg<V, false><<<(n + block - 1) / block, block, 0, s>>>(n, rp, ci, va, x, alpha, y, adev);
        XB_LAUNCHED("k_sym_wagg");
        return XB_OK;
    }
    if (variant == XB_VAR_SYM_ATOMIC) {
        if (a1)
            k_sym_atomic<V, true><<<(n + block - 1) / block, block, 0, s>>>(n, rp, ci, va, x, alpha, y, adev);
        else
            k_sym_atomic<V, false><<<(n + block - 1) / block, block, 0, s>>>(n, rp, ci, va, x, alpha, y, adev);
        XB_LAUNCHED("k_sym_atomic");
        return XB_OK;
    }
    int err = XB_OK;
    const xb::TilePart *tp = xb::get_tiles(p, block, ipt, s, &err);
    if (!tp) return err;
    if (tp->ntiles == 0) return XB_OK;
    const size_t sm = (32 + (size_t)block + (size_t)block * ipt) * sizeof(V) +
                      (size_t)block * ipt * 4 + (block + 1) * 4;
#define XB_SYM(I)                                                                         \
    case I:                                                                               \
        if (a1) {                                                                         \
            XB_TRY(smem_optin((const void *)k_sym_tile<V, I, true>, sm));                  \
            k_sym_tile<V, I, true><<<tp->ntiles, block, sm, s>>>(rp, ci, va, x, alpha, y,   \
                                                                tp->d_row, adev);         \
        } else {                                                                          \
            XB_TRY(smem_optin((const void *)k_sym_tile<V, I, false>, sm));                 \
            k_sym_tile<V, I, false><<<tp->ntiles, block, sm, s>>>(rp, ci, va, x, alpha, y,  \
                                                                 tp->d_row, adev);        \
        }                                                                                 \
        break;
    switch (ipt) {
        XB_SYM(1) XB_SYM(2) XB_SYM(4) XB_SYM(8) XB_SYM(16)
        default: return xb::set_error(XB_EINVAL, "sym tile: unsupported ipt %d", ipt);
    }
#undef XB_SYM
    XB_LAUNCHED("k_sym_tile");
    return XB_OK;
}

template <typename V>
int spmv_any(xb_plan *p, int variant, int block, int ipt, V alpha, const V *x, V beta, V *y,
             const V *va, const V *adev, cudaStream_t s) {
    if (variant == XB_VAR_AUTO) variant = p->variant;
    if (block <= 0) block = p->block;
    if (ipt <= 0) ipt = p->ipt;
    if (!xb::variant_fits(p, variant))
        return xb::set_error(XB_EINVAL, "SpMV variant %d does not fit %s storage", variant,
                             p->sym ? "symmetric-upper" : "general");
    if (block != 64 && block != 128 && block != 256 && block != 512)
        return xb::set_error(XB_EINVAL, "SpMV block %d not in {64,128,256,512}", block);
    const int n = p->n;
    if (n == 0) return XB_OK;
    if (!p->subs.empty()) {  // a split plan: the variant on each row block, the whole x
        for (const auto &sb : p->subs) {
            const V *vs = sizeof(V) == sizeof(float) ? reinterpret_cast<const V *>(sb.plan->val32)
                                                     : reinterpret_cast<const V *>(sb.plan->val);
            XB_TRY(spmv_any<V>(sb.plan, variant, block, ipt, alpha, x, beta, y + sb.r0, vs, adev, s));
        }
        return XB_OK;
    }
    if (adev) beta = V(0);
    const int mode = adev ? 1 : (beta == V(0)) ? (alpha == V(1) ? 0 : 1) : 2;
    switch (variant) {
        case XB_VAR_ROW:
            k_row<V><<<(n + block - 1) / block, block, 0, s>>>(n, p->rowptr, p->col, va, x, alpha,
                                                               beta, mode, y, adev);
            XB_LAUNCHED("k_row");
            return XB_OK;
        case XB_VAR_NNZ:
            return launch_u2<V>(p, p->rowptr, p->col, va, block, ipt, alpha, x, beta, mode, y, adev,
                                s);
        case XB_VAR_SEGSCAN:
            return launch_seg<V>(p, p->rowptr, p->col, va, block, ipt, alpha, x, beta, mode, y, adev,
                                 s);
        case XB_VAR_SYM_ATOMIC:
        case XB_VAR_SYM_TILE:
        case XB_VAR_SYM_PART:
        case XB_VAR_SYM_WAGG:
            return launch_sym<V>(p, variant, p->rowptr, p->col, va, block, ipt, alpha, x, beta, y,
                                 adev, s);
        case XB_VAR_SELL:
            return launch_sell<V>(p, block, ipt, alpha, x, beta, mode, y, adev, s);
        case XB_VAR_BCSR:
            return launch_bcsr<V>(p, block, ipt, alpha, x, beta, mode, y, adev, s);
    }
    return xb::set_error(XB_EINVAL, "unknown SpMV variant %d", variant);
}

}  // namespace

namespace xb {

int spmv_launch(xb_plan *p, int variant, int block, int ipt, double alpha, const double *x,
                double beta, double *y, cudaStream_t s) {
    return spmv_any<double>(p, variant, block, ipt, alpha, x, beta, y, p->val, nullptr, s);
}

int spmv_launch_dalpha(xb_plan *p, int variant, int block, int ipt, const double *alpha_dev,
                       const double *x, double *y, cudaStream_t s) {
    return spmv_any<double>(p, variant, block, ipt, 1.0, x, 0.0, y, p->val, alpha_dev, s);
}

int spmv_launch_dalpha_f32(xb_plan *p, int variant, int block, int ipt, const float *alpha_dev,
                           const float *x, float *y, cudaStream_t s) {
    XB_TRY(ensure_val32(p, s));
    return spmv_any<float>(p, variant, block, ipt, 1.0f, x, 0.0f, y, p->val32, alpha_dev, s);
}

int spmv_launch_f32(xb_plan *p, int variant, int block, int ipt, float alpha, const float *x,
                    float beta, float *y, cudaStream_t s) {
    XB_TRY(ensure_val32(p, s));
    return spmv_any<float>(p, variant, block, ipt, alpha, x, beta, y, p->val32, nullptr, s);
}

double spmv_alg_bytes(const xb_plan *p, bool beta_nonzero, int val_bytes) {
    const double n = p->n, nnz = (double)p->nnz64;
    const int vb = val_bytes;
    return (vb + 4.0) * nnz + 4.0 * (n + 1) + vb * n + vb * n + (beta_nonzero ? vb * n : 0.0);
}

}  // namespace xb

// ---------------------------------------------------------------------------
// Allocation-free segmented-scan SpMV.
//
// Some callers cannot call cudaMalloc at all: applications whose device
// memory is entirely owned by another allocator (a framework that reserves
// the free HBM at start-up and hands out sub-buffers), and code on a path
// where an allocation's implicit device synchronisation and latency are not
// allowed.  Such callers cannot create an xb_plan either, since a plan owns
// device workspace.  spmv_segscan_noalloc runs the staged per-CTA
// segmented-scan kernel k_seg (nothing else launches it; spmv_segscan runs
// the bitmask-driven k_bss, which needs plan data) with its scratch (per-CTA
// start rows and carries) in one file-scope device array instead of plan
// memory.  Its rows agree with spmv_segscan within the 1e-12 row tolerance,
// not bit for bit.  Every GPU that loads the library holds that array until
// the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr int kNaBlock = 256;
constexpr int kNaIpt = 8;
constexpr size_t kNaScratchBytes = size_t(4) << 20;  // 4 MiB
// per CTA: start row (int) + carry row (int) + carry value (double)
constexpr long long kNaMaxCtas = (long long)(kNaScratchBytes / 16) - 1;

static __device__ __align__(256) unsigned char g_na_scratch[kNaScratchBytes];

// Row holding non-zero b*T for each CTA b (last entry n).
__global__ void k_na_rows(int n, const int *__restrict__ rowptr, long long T, int nblk,
                          int *__restrict__ out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b > nblk) return;
    if (b == nblk) {
        out[b] = n;
        return;
    }
    const long long target = (long long)b * T;
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (int)(((long long)lo + hi + 1) >> 1);
        if ((long long)rowptr[mid] <= target) lo = mid;
        else hi = mid - 1;
    }
    out[b] = lo;
}

// Rows without stored entries get beta*y (or 0); no other row is touched.
__global__ void k_na_empty(int n, const int *__restrict__ rowptr, double beta, int mode,
                           double *__restrict__ y) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n || rowptr[r] != rowptr[r + 1]) return;
    y[r] = (mode == 2) ? beta * y[r] : 0.0;
}

// Device address of the scratch array on the current device.  Looked up on
// every call: once the library's module is loaded on the device this is a
// host-side table lookup, and it stays right after cudaDeviceReset, which
// reloads the module (a cached address could then be stale).  The first call
// on a device loads the module, so it should come before any stream capture.
int na_scratch(unsigned char **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
    if (e != cudaSuccess)
        return xb::cuda_error(e, "spmv_segscan_noalloc: cudaGetSymbolAddress(scratch)");
    *out = static_cast<unsigned char *>(p);
    return XB_OK;
}

}  // namespace

extern "C" int spmv_segscan_noalloc(int32_t n, int32_t nnz, const int32_t *rowptr,
                                    const int32_t *col, const double *val, double alpha,
                                    const double *x, double beta, double *y, void *stream) {
    if (n < 0 || nnz < 0) return xb::set_error(XB_EINVAL, "spmv_segscan_noalloc: n=%d nnz=%d", n, nnz);
    if (n == 0) return XB_OK;
    if (!rowptr || !x || !y || (nnz > 0 && (!col || !val)))
        return xb::set_error(XB_EINVAL, "spmv_segscan_noalloc: NULL array");
    {  // y is written while other CTAs still read x: the ranges must be disjoint
        const uintptr_t xa = (uintptr_t)x, ya = (uintptr_t)y, len = (uintptr_t)n * sizeof(double);
        if (xa < ya + len && ya < xa + len)
            return xb::set_error(XB_EINVAL, "spmv_segscan_noalloc: x and y overlap");
    }
    const long long T = (long long)kNaBlock * kNaIpt;
    const long long nblk = ((long long)nnz + T - 1) / T;
    if (nblk + 1 > kNaMaxCtas)
        return xb::set_error(XB_EINVAL,
                             "spmv_segscan_noalloc: nnz=%d needs %lld scratch slots; the built-in "
                             "scratch holds %lld (nnz <= %lld)", nnz, nblk + 1, kNaMaxCtas,
                             (kNaMaxCtas - 1) * T);
    unsigned char *base = nullptr;
    XB_TRY(na_scratch(&base));
    cudaStream_t s = (cudaStream_t)stream;
    const int mode = (beta == 0.0) ? (alpha == 1.0 ? 0 : 1) : 2;
    int *brow = reinterpret_cast<int *>(base);
    int *crow = brow + (nblk + 1);
    double *cval = reinterpret_cast<double *>(base + 8 * (size_t)(nblk + 1));
    if (nblk > 0) {
        k_na_rows<<<(int)((nblk + 1 + 255) / 256), 256, 0, s>>>(n, rowptr, T, (int)nblk, brow);
        XB_LAUNCHED("k_na_rows");
        const int TP = (int)T + kNaBlock;
        const size_t sm = (size_t)TP * sizeof(double) + 64 * sizeof(double) + (size_t)TP * 4 +
                          (size_t)(T + 2) * 4 + 64 * 4;
        XB_TRY(smem_optin((const void *)k_seg<double, kNaIpt>, sm));
        k_seg<double, kNaIpt><<<(int)nblk, kNaBlock, sm, s>>>(n, nnz, rowptr, col, val, x, alpha,
                                                              beta, mode, y, brow, cval, crow,
                                                              nullptr);
        XB_LAUNCHED("k_seg (noalloc)");
        k_seg_fix<double><<<(int)((nblk + 255) / 256), 256, 0, s>>>((int)nblk, n, crow, cval,
                                                                     alpha, mode, y, nullptr);
        XB_LAUNCHED("k_seg_fix (noalloc)");
    }
    k_na_empty<<<(n + 255) / 256, 256, 0, s>>>(n, rowptr, beta, mode, y);
    XB_LAUNCHED("k_na_empty");
    return XB_OK;
}
