// Plans (the paper's *_Setup functions, Table 1): validation, partitions for
// every SpMV variant, FP32 copy of A, reduction scratch, matrix features.
#include "common.cuh"

#include <algorithm>
#include <climits>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>

namespace xb {

static thread_local std::string g_err;

int set_error(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_error(cudaError_t e, const char *where) {
    return set_error(XB_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

int num_sms() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

int reduce_grid(int64_t n, int block) {
    int64_t want = (n + block * 4 - 1) / (block * 4);
    int64_t cap = std::min<int64_t>(kRedSlots, (int64_t)num_sms() * 8);
    return (int)std::max<int64_t>(1, std::min(want, cap));
}

int resident_grid(const void *fn, int block, int64_t n, int per_thread) {
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, int> cache;  // (kernel, device) -> CTAs/SM
    int dev = 0;
    cudaGetDevice(&dev);
    int per_sm = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find({fn, dev});
        if (it != cache.end()) {
            per_sm = it->second;
        } else {
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block, 0) != cudaSuccess ||
                per_sm < 1)
                per_sm = 1;
            cache[{fn, dev}] = per_sm;
        }
    }
    const int64_t want = (n + (int64_t)block * per_thread - 1) / ((int64_t)block * per_thread);
    const int64_t cap = std::min<int64_t>(kRedSlots, (int64_t)per_sm * num_sms());
    return (int)std::max<int64_t>(1, std::min(want, cap));
}

bool variant_fits(const xb_plan *p, int v) {
    if (p->sym)
        return v == XB_VAR_SYM_ATOMIC || v == XB_VAR_SYM_TILE || v == XB_VAR_SYM_PART ||
               v == XB_VAR_SYM_WAGG;
    return v == XB_VAR_ROW || v == XB_VAR_NNZ || v == XB_VAR_SEGSCAN || v == XB_VAR_SELL ||
           v == XB_VAR_BCSR;
}

// ---- partitions -------------------------------------------------------------

std::vector<int> tile_rows(int n, const int *rp, int block, int ipt) {
    const int64_t T = (int64_t)block * ipt;
    std::vector<int> rows;
    rows.reserve(n / std::max(1, block / 2) + 16);
    rows.push_back(0);
    int r = 0;
    while (r < n) {
        const int64_t k0 = rp[r];
        int r1 = r + 1;
        if ((int64_t)rp[r + 1] - k0 <= T)
            while (r1 < n && r1 - r < block && (int64_t)rp[r1 + 1] - k0 <= T) r1++;
        rows.push_back(r1);
        r = r1;
    }
    return rows;
}

const TilePart *get_tiles(xb_plan *p, int block, int ipt, cudaStream_t s, int *err) {
    for (auto &t : p->tiles)
        if (t.block == block && t.ipt == ipt) return &t;
    std::vector<int> rows = tile_rows(p->n, p->h_rowptr.data(), block, ipt);
    TilePart t;
    t.block = block;
    t.ipt = ipt;
    t.ntiles = (int)rows.size() - 1;
    cudaError_t e = cudaMalloc(&t.d_row, rows.size() * sizeof(int));
    if (e != cudaSuccess) {
        *err = cuda_error(e, "cudaMalloc(tiles)");
        return nullptr;
    }
    e = cudaMemcpyAsync(t.d_row, rows.data(), rows.size() * sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaFree(t.d_row);
        *err = cuda_error(e, "upload tiles");
        return nullptr;
    }
    p->tiles.push_back(t);
    return &p->tiles.back();
}

const S3Part *get_s3(xb_plan *p, int block, int ipt, cudaStream_t s, int *err) {
    for (auto &t : p->s3)
        if (t.block == block && t.ipt == ipt) return &t;
    const TilePart *tp = get_tiles(p, block, ipt, s, err);
    if (!tp) return nullptr;
    const int n = p->n;
    const int *rp = p->h_rowptr.data();
    std::vector<int> rows = tile_rows(n, rp, block, ipt);
    std::vector<int> hcol(p->nnz);
    cudaError_t e = cudaSuccess;
    if (p->nnz > 0)
        e = cudaMemcpy(hcol.data(), p->col, (size_t)p->nnz * sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        *err = cuda_error(e, "S3 layout: columns to host");
        return nullptr;
    }
    const int ngr = (n + kS3Gran - 1) / kS3Gran;
    std::vector<int> tslot(1, 0), sgran;
    std::vector<std::vector<int>> cover(ngr);
    for (size_t t = 0; t + 1 < rows.size(); t++) {
        const int r1 = rows[t + 1];
        std::vector<int> g;  // granules reached beyond the tile, ascending
        for (int k = rp[rows[t]]; k < rp[r1]; k++)
            if (hcol[k] >= r1) {
                const int q = hcol[k] / kS3Gran;
                if (std::find(g.begin(), g.end(), q) == g.end()) {
                    if ((int)g.size() == kS3Max) {
                        *err = set_error(XB_EINVAL,
                                         "S3 layout: tile %zu reaches more than %d granules of "
                                         "%d rows beyond itself", t, kS3Max, kS3Gran);
                        return nullptr;
                    }
                    g.push_back(q);
                }
            }
        std::sort(g.begin(), g.end());
        for (int q : g) {
            cover[q].push_back((int)sgran.size());
            sgran.push_back(q);
        }
        tslot.push_back((int)sgran.size());
    }
    std::vector<int> gid, gptr(1, 0), gslot;
    for (int q = 0; q < ngr; q++)
        if (!cover[q].empty()) {
            gid.push_back(q);
            gslot.insert(gslot.end(), cover[q].begin(), cover[q].end());
            gptr.push_back((int)gslot.size());
        }
    S3Part t;
    t.block = block;
    t.ipt = ipt;
    t.ntiles = (int)rows.size() - 1;
    t.nslots = (int)sgran.size();
    t.ngran = (int)gid.size();
    auto up = [&](int **d, const std::vector<int> &h) {
        if (e != cudaSuccess) return;
        e = cudaMalloc(d, std::max<size_t>(1, h.size()) * sizeof(int));
        if (e == cudaSuccess && !h.empty())
            e = cudaMemcpy(*d, h.data(), h.size() * sizeof(int), cudaMemcpyHostToDevice);
    };
    up(&t.d_tslot, tslot);
    up(&t.d_sgran, sgran);
    up(&t.d_gid, gid);
    up(&t.d_gptr, gptr);
    up(&t.d_gslot, gslot);
    if (e == cudaSuccess)
        e = cudaMalloc(&t.d_part, std::max<size_t>(1, (size_t)t.nslots * kS3Gran) * sizeof(double));
    if (e != cudaSuccess) {
        cudaFree(t.d_tslot);
        cudaFree(t.d_sgran);
        cudaFree(t.d_gid);
        cudaFree(t.d_gptr);
        cudaFree(t.d_gslot);
        cudaFree(t.d_part);
        *err = cuda_error(e, "S3 layout");
        return nullptr;
    }
    p->s3.push_back(t);
    return &p->s3.back();
}

int64_t bcsr_layout(int n, const int *rp, const int *col, int r, std::vector<int> &bptr,
                    std::vector<int> &bcol) {
    const int nbr = (n + r - 1) / r;
    bptr.assign(1, 0);
    bcol.clear();
    std::vector<int> cur;
    for (int b = 0; b < nbr; b++) {
        cur.clear();
        for (int i = b * r; i < std::min(n, b * r + r); i++)
            for (int k = rp[i]; k < rp[i + 1]; k++) cur.push_back(col[k] / r);
        std::sort(cur.begin(), cur.end());
        cur.erase(std::unique(cur.begin(), cur.end()), cur.end());
        bcol.insert(bcol.end(), cur.begin(), cur.end());
        bptr.push_back((int)bcol.size());
    }
    return (int64_t)bcol.size();
}

// Places A's entries in the zero-filled blocks: thread per row, merging the
// row's block columns (ascending) with its block row's block list (ascending).
template <typename T>
__global__ void k_bcsr_fill(int n, int r, const int *__restrict__ rowptr,
                            const int *__restrict__ col, const T *__restrict__ val,
                            const int *__restrict__ bptr, const int *__restrict__ bcol,
                            T *__restrict__ bval) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int b = i / r, li = i - b * r;
    int q = bptr[b];
    const int qe = bptr[b + 1];
    for (int k = rowptr[i]; k < rowptr[i + 1]; k++) {
        const int c = col[k], cb = c / r;
        while (q < qe && bcol[q] < cb) q++;
        if (q < qe && bcol[q] == cb) bval[((int64_t)q * r + li) * r + (c - cb * r)] = val[k];
    }
}

const BcsrPart *get_bcsr(xb_plan *p, int r, bool f32, cudaStream_t s, int *err) {
    if (r < 2 || r > 4) {
        *err = set_error(XB_EINVAL, "BCSR: block size %d not in {2, 3, 4}", r);
        return nullptr;
    }
    BcsrPart *bp = nullptr;
    for (auto &t : p->bcsr)
        if (t.r == r) bp = &t;
    cudaError_t e = cudaSuccess;
    if (!bp) {
        std::vector<int> hcol(p->nnz), bptr, bcol;
        if (p->nnz > 0)
            e = cudaMemcpy(hcol.data(), p->col, (size_t)p->nnz * sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            *err = cuda_error(e, "BCSR: columns to host");
            return nullptr;
        }
        BcsrPart t;
        t.r = r;
        t.nbr = (p->n + r - 1) / r;
        t.nblocks = bcsr_layout(p->n, p->h_rowptr.data(), hcol.data(), r, bptr, bcol);
        const int64_t entries = t.nblocks * r * r;
        if (entries > 2LL * p->nnz + 16LL * r) {
            *err = set_error(XB_EINVAL, "BCSR %dx%d: blocks hold %lld entries for %d non-zeros", r,
                             r, (long long)entries, p->nnz);
            return nullptr;
        }
        const size_t ent = (size_t)std::max<int64_t>(entries, 1);
        e = cudaMalloc(&t.d_bptr, bptr.size() * sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc(&t.d_bcol, std::max<size_t>(bcol.size(), 1) * sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc(&t.d_val, ent * sizeof(double));
        if (e == cudaSuccess)
            e = cudaMemcpy(t.d_bptr, bptr.data(), bptr.size() * sizeof(int), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && !bcol.empty())
            e = cudaMemcpy(t.d_bcol, bcol.data(), bcol.size() * sizeof(int), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemsetAsync(t.d_val, 0, ent * sizeof(double), s);
        if (e == cudaSuccess && p->n > 0) {
            k_bcsr_fill<double><<<(p->n + 255) / 256, 256, 0, s>>>(p->n, r, p->rowptr, p->col, p->val,
                                                                  t.d_bptr, t.d_bcol, t.d_val);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) {
            cudaFree(t.d_bptr);
            cudaFree(t.d_bcol);
            cudaFree(t.d_val);
            *err = cuda_error(e, "BCSR copy");
            return nullptr;
        }
        p->bcsr.push_back(t);
        bp = &p->bcsr.back();
    }
    if (f32 && !bp->d_val32) {
        int rc = ensure_val32(p, s);
        if (rc != XB_OK) {
            *err = rc;
            return nullptr;
        }
        const size_t ent = (size_t)std::max<int64_t>(bp->nblocks * r * r, 1);
        e = cudaMalloc(&bp->d_val32, ent * sizeof(float));
        if (e == cudaSuccess) e = cudaMemsetAsync(bp->d_val32, 0, ent * sizeof(float), s);
        if (e == cudaSuccess && p->n > 0) {
            k_bcsr_fill<float><<<(p->n + 255) / 256, 256, 0, s>>>(p->n, r, p->rowptr, p->col, p->val32,
                                                                 bp->d_bptr, bp->d_bcol, bp->d_val32);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) {
            cudaFree(bp->d_val32);
            bp->d_val32 = nullptr;
            *err = cuda_error(e, "BCSR FP32 copy");
            return nullptr;
        }
    }
    return bp;
}

int u2_layout(int n, const int *rp, int ipt, std::vector<int4> &tiles, std::vector<int> &longs) {
    tiles.clear();
    longs.clear();
    const int64_t W = 32LL * ipt;
    int nflat = 0, r = 0, ne = 0;
    while (r < n) {
        const int64_t A = rp[r] - rp[r] % ipt;  // window start
        if ((int64_t)rp[r + 1] - A > W) {        // the row alone overflows a window
            longs.push_back(r);
            ne += rp[r + 1] > rp[r];
            r++;
            continue;
        }
        const int r0 = r, ne0 = ne;
        int maxlen = 0, empty = 0;
        while (r < n && (int64_t)rp[r + 1] - A <= W) {
            const int len = rp[r + 1] - rp[r];
            const int nm = std::max(maxlen, len);
            if (nm <= ipt && r - r0 == 32) break;  // a thread-per-row tile holds 32 rows
            maxlen = nm;
            empty |= (len == 0);
            ne += (len > 0);
            r++;
        }
        const int kind = maxlen <= ipt ? 0 : 1;
        nflat += kind;
        tiles.push_back(make_int4(r0, r, ne0, kind | (empty ? 4 : 0)));
    }
    return nflat;
}

const U2Part *get_u2(xb_plan *p, int ipt, cudaStream_t s, int *err) {
    for (auto &t : p->u2)
        if (t.ipt == ipt) return &t;
    std::vector<int4> tiles;
    std::vector<int> longs;
    U2Part t;
    t.ipt = ipt;
    t.nflat = u2_layout(p->n, p->h_rowptr.data(), ipt, tiles, longs);
    t.ntiles = (int)tiles.size();
    t.nlong = (int)longs.size();
    if (t.nflat > 0 && !get_bss(p, s, err)) return nullptr;  // flat tiles read the row-end bits
    t.implicit = t.nlong == 0 && t.nflat == 0;
    for (int i = 0; t.implicit && i < t.ntiles; i++)
        t.implicit = tiles[i].x == 32 * i && tiles[i].y == std::min(p->n, 32 * i + 32);
    cudaError_t e = cudaSuccess;
    if (!t.implicit && t.ntiles > 0) {
        e = cudaMalloc(&t.d_tile, tiles.size() * sizeof(int4));
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(t.d_tile, tiles.data(), tiles.size() * sizeof(int4),
                                cudaMemcpyHostToDevice, s);
    }
    if (e == cudaSuccess && t.nlong > 0) {
        e = cudaMalloc(&t.d_long, longs.size() * sizeof(int));
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(t.d_long, longs.data(), longs.size() * sizeof(int),
                                cudaMemcpyHostToDevice, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaFree(t.d_tile);
        cudaFree(t.d_long);
        *err = cuda_error(e, "U2 tiles");
        return nullptr;
    }
    p->u2.push_back(t);
    return &p->u2.back();
}

// Index (over the rows of crp) of the row holding non-zero w*W, per warp w.
__global__ void k_seg_rows(int nrows, const int *__restrict__ crp, long long W, int nw,
                           int *__restrict__ out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b > nw) return;
    if (b == nw) {
        out[b] = nrows;
        return;
    }
    const long long target = (long long)b * W;
    int lo = 0, hi = nrows;
    while (lo < hi) {
        const int mid = (int)(((long long)lo + hi + 1) >> 1);
        if ((long long)crp[mid] <= target) lo = mid;
        else hi = mid - 1;
    }
    out[b] = lo;
}

// Bit (rowptr[r+1]-1) for every non-empty row r: the row-end flags.
__global__ void k_endbits(int n, const int *__restrict__ rowptr, unsigned *__restrict__ bits) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int a = rowptr[r], b = rowptr[r + 1];
    if (b > a) atomicOr(&bits[(b - 1) >> 5], 1u << ((b - 1) & 31));
}

const BssData *get_bss(xb_plan *p, cudaStream_t s, int *err) {
    BssData &d = p->bss;
    if (d.built) return &d;
    const size_t words = (size_t)p->nnz / 32 + 2;
    cudaError_t e = cudaMalloc(&d.d_endbits, words * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemsetAsync(d.d_endbits, 0, words * sizeof(unsigned), s);
    if (e == cudaSuccess && p->n > 0) {
        k_endbits<<<(p->n + 255) / 256, 256, 0, s>>>(p->n, p->rowptr, d.d_endbits);
        e = cudaGetLastError();
    }
    d.n_ne = p->n - p->n_empty;
    if (e == cudaSuccess && p->n_empty > 0) {
        std::vector<int> ne, crp;
        ne.reserve(d.n_ne);
        crp.reserve(d.n_ne + 1);
        const int *rp = p->h_rowptr.data();
        for (int r = 0; r < p->n; r++)
            if (rp[r + 1] > rp[r]) {
                ne.push_back(r);
                crp.push_back(rp[r]);
            }
        crp.push_back(p->nnz);
        e = cudaMalloc(&d.d_ne_rows, std::max<size_t>(1, ne.size()) * sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc(&d.d_crp, crp.size() * sizeof(int));
        if (e == cudaSuccess && !ne.empty())
            e = cudaMemcpy(d.d_ne_rows, ne.data(), ne.size() * sizeof(int), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(d.d_crp, crp.data(), crp.size() * sizeof(int), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        *err = cuda_error(e, "BSS plan data");
        return nullptr;
    }
    d.built = true;
    return &d;
}

// Entry p of the BSS copy (VN-element vectors) comes from non-zero e.
template <typename T, int VN>
__global__ void k_bss_copy(int64_t total, int64_t nnz, int ipt, const T *__restrict__ src,
                           T *__restrict__ dst) {
    const int64_t W = 32LL * ipt;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < total;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = p / W;
        const int off = (int)(p - g * W);
        const int vec = off / VN, h = off - vec * VN;
        const int q = vec >> 5, l = vec & 31;
        const int64_t e = g * W + (int64_t)l * ipt + q * VN + h;
        dst[p] = (e < nnz) ? src[e] : T(0);
    }
}

const BssCopy *get_bss_copy(xb_plan *p, int ipt, bool f32, cudaStream_t s, int *err) {
    BssCopy *c = nullptr;
    for (auto &t : p->bss.copies)
        if (t.ipt == ipt) c = &t;
    const int64_t W = 32LL * ipt;
    const int64_t total = (p->nnz + W - 1) / W * W;
    const int grid = num_sms() * 8;
    cudaError_t e = cudaSuccess;
    if (!c) {
        BssCopy t;
        t.ipt = ipt;
        t.total = total;
        e = cudaMalloc(&t.d_col, std::max<int64_t>(total, 1) * sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc(&t.d_val, std::max<int64_t>(total, 1) * sizeof(double));
        if (e == cudaSuccess && total > 0) {
            k_bss_copy<int, 4><<<grid, 256, 0, s>>>(total, p->nnz, ipt, p->col, t.d_col);
            k_bss_copy<double, 2><<<grid, 256, 0, s>>>(total, p->nnz, ipt, p->val, t.d_val);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) {
            cudaFree(t.d_col);
            cudaFree(t.d_val);
            *err = cuda_error(e, "BSS data format copy");
            return nullptr;
        }
        p->bss.copies.push_back(t);
        c = &p->bss.copies.back();
    }
    if (f32 && !c->d_val32) {
        int r = ensure_val32(p, s);
        if (r != XB_OK) {
            *err = r;
            return nullptr;
        }
        e = cudaMalloc(&c->d_val32, std::max<int64_t>(total, 1) * sizeof(float));
        if (e == cudaSuccess && total > 0) {
            k_bss_copy<float, 4><<<grid, 256, 0, s>>>(total, p->nnz, ipt, p->val32, c->d_val32);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) {
            cudaFree(c->d_val32);
            c->d_val32 = nullptr;
            *err = cuda_error(e, "BSS data format copy (FP32)");
            return nullptr;
        }
    }
    return c;
}

void bss_trim(xb_plan *p, int keep_ipt) {
    for (auto &sb : p->subs) bss_trim(sb.plan, keep_ipt);
    auto &v = p->bss.copies;
    bool any = false;
    for (auto &t : v)
        if (t.ipt != keep_ipt) any = true;
    if (!any) return;
    cudaDeviceSynchronize();  // no launch may still read a copy being freed
    std::vector<BssCopy> kept;
    for (auto &t : v) {
        if (t.ipt == keep_ipt) {
            kept.push_back(t);
        } else {
            cudaFree(t.d_col);
            cudaFree(t.d_val);
            cudaFree(t.d_val32);
        }
    }
    v.swap(kept);
}

const SegPart *get_segs(xb_plan *p, int block, int ipt, cudaStream_t s, int *err) {
    for (auto &t : p->segs)
        if (t.block == block && t.ipt == ipt) return &t;
    const BssData *bd = get_bss(p, s, err);
    if (!bd) return nullptr;
    SegPart t;
    t.block = block;
    t.ipt = ipt;
    const long long W = 32LL * ipt;
    t.nblk = (int)((p->nnz + W - 1) / W);
    const size_t nb = (size_t)t.nblk + 1;
    cudaError_t e = cudaMalloc(&t.d_row, nb * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&t.d_carry_row, nb * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&t.d_carry_val, nb * sizeof(double));
    if (e != cudaSuccess) {
        cudaFree(t.d_row);
        cudaFree(t.d_carry_row);
        cudaFree(t.d_carry_val);
        *err = cuda_error(e, "cudaMalloc(segments)");
        return nullptr;
    }
    const int *crp = bd->d_crp ? bd->d_crp : p->rowptr;
    k_seg_rows<<<(t.nblk + 1 + 255) / 256, 256, 0, s>>>(bd->n_ne, crp, W, t.nblk, t.d_row);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        *err = cuda_error(e, "k_seg_rows");
        return nullptr;
    }
    p->segs.push_back(t);
    return &p->segs.back();
}

__global__ void k_to_f32(int64_t n, const double *__restrict__ a, float *__restrict__ b) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

int ensure_val32(xb_plan *p, cudaStream_t s) {
    for (auto &sb : p->subs) XB_TRY(ensure_val32(sb.plan, s));  // a split plan's blocks
    if (!p->subs.empty() || p->val32 || p->nnz == 0) return XB_OK;
    XB_CUDA(cudaMalloc(&p->val32, (size_t)p->nnz * sizeof(float)));
    k_to_f32<<<num_sms() * 8, 256, 0, s>>>(p->nnz, p->val, p->val32);
    XB_LAUNCHED("k_to_f32");
    return XB_OK;
}

// Copy row perm[t]'s entries into slot t of the SELL layout (the slot's
// lane of its slice, one column per entry); thread per slot.
template <typename V>
__global__ void k_sell_scatter(int64_t nslots, const int *__restrict__ perm,
                               const int64_t *__restrict__ off, const int *__restrict__ rowptr,
                               const int *__restrict__ col, const V *__restrict__ val,
                               int *__restrict__ scol, V *__restrict__ sval) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nslots) return;
    const int r = perm[t];
    if (r < 0) return;
    const int a = rowptr[r], len = rowptr[r + 1] - a;
    const int64_t base = off[t >> 5] + (t & 31);
    for (int j = 0; j < len; j++) {
        if (scol) scol[base + 32LL * j] = col[a + j];
        sval[base + 32LL * j] = val[a + j];
    }
}

int64_t sell_layout(int n, const int *rp, int sigma, std::vector<int> &perm,
                    std::vector<int> &slen, std::vector<int64_t> &off) {
    const int nslices = (n + 31) / 32;
    const size_t nslots = (size_t)nslices * 32;
    perm.assign(nslots, -1);
    for (int i = 0; i < n; i++) perm[i] = i;
    auto len = [&](int r) { return rp[r + 1] - rp[r]; };
    for (int w0 = 0; w0 < n; w0 += sigma) {
        const int w1 = (int)std::min<int64_t>(n, (int64_t)w0 + sigma);
        std::stable_sort(perm.begin() + w0, perm.begin() + w1,
                         [&](int a, int b) { return len(a) > len(b); });
    }
    slen.assign(nslots, 0);
    for (size_t q = 0; q < nslots; q++)
        if (perm[q] >= 0) slen[q] = len(perm[q]);
    off.assign((size_t)nslices + 1, 0);
    for (int q = 0; q < nslices; q++) {
        int wd = 0;
        for (int l = 0; l < 32; l++) wd = std::max(wd, slen[(size_t)q * 32 + l]);
        off[q + 1] = off[q] + 32LL * wd;
    }
    return off[nslices];
}

const SellPart *get_sell(xb_plan *p, int sigma, bool f32, cudaStream_t s, int *err) {
    SellPart *sp = nullptr;
    for (auto &t : p->sells)
        if (t.sigma == sigma) sp = &t;
    if (!sp) {
        SellPart t;
        t.sigma = sigma;
        t.nslices = (p->n + 31) / 32;
        const size_t nslots = (size_t)t.nslices * 32;
        std::vector<int> perm, slen;
        std::vector<int64_t> off;
        t.total = sell_layout(p->n, p->h_rowptr.data(), sigma, perm, slen, off);
        if (t.total > 3LL * p->nnz + 32LL * t.nslices) {
            *err = set_error(XB_EINVAL, "SELL-32-%d: padding to %lld entries for %d non-zeros",
                             sigma, (long long)t.total, p->nnz);
            return nullptr;
        }
        const size_t tot = (size_t)std::max<int64_t>(t.total, 1);
        cudaError_t e = cudaMalloc(&t.d_off, off.size() * sizeof(int64_t));
        if (e == cudaSuccess) e = cudaMalloc(&t.d_perm, nslots * sizeof(int) + 4);
        if (e == cudaSuccess) e = cudaMalloc(&t.d_len, nslots * sizeof(int) + 4);
        if (e == cudaSuccess) e = cudaMalloc(&t.d_col, tot * sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc(&t.d_val, tot * sizeof(double));
        if (e == cudaSuccess)
            e = cudaMemcpy(t.d_off, off.data(), off.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && nslots)
            e = cudaMemcpy(t.d_perm, perm.data(), nslots * sizeof(int), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && nslots)
            e = cudaMemcpy(t.d_len, slen.data(), nslots * sizeof(int), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(t.d_off);
            cudaFree(t.d_perm);
            cudaFree(t.d_len);
            cudaFree(t.d_col);
            cudaFree(t.d_val);
            *err = cuda_error(e, "SELL copy");
            return nullptr;
        }
        if (nslots) {
            k_sell_scatter<double><<<(unsigned)((nslots + 255) / 256), 256, 0, s>>>(
                (int64_t)nslots, t.d_perm, t.d_off, p->rowptr, p->col, p->val, t.d_col, t.d_val);
            e = cudaGetLastError();
        }
        p->sells.push_back(t);  // owned by the plan from here (freed with it)
        if (e != cudaSuccess) {
            *err = cuda_error(e, "k_sell_scatter");
            return nullptr;
        }
        sp = &p->sells.back();
    }
    if (f32 && !sp->d_val32) {
        int r = ensure_val32(p, s);
        if (r != XB_OK) {
            *err = r;
            return nullptr;
        }
        const size_t tot = (size_t)std::max<int64_t>(sp->total, 1);
        cudaError_t e = cudaMalloc(&sp->d_val32, tot * sizeof(float));
        if (e != cudaSuccess) {
            *err = cuda_error(e, "SELL FP32 copy");
            return nullptr;
        }
        const size_t nslots = (size_t)sp->nslices * 32;
        if (nslots && p->nnz) {
            k_sell_scatter<float><<<(unsigned)((nslots + 255) / 256), 256, 0, s>>>(
                (int64_t)nslots, sp->d_perm, sp->d_off, p->rowptr, p->col, p->val32, nullptr,
                sp->d_val32);
            e = cudaGetLastError();
            if (e != cudaSuccess) {
                *err = cuda_error(e, "k_sell_scatter");
                return nullptr;
            }
        }
    }
    return sp;
}

int ensure_work(xb_plan *p, size_t bytes) {
    if (p->work_bytes >= bytes) return XB_OK;
    if (p->d_work) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_error(e, "sync before workspace growth");
        cudaFree(p->d_work);
        p->d_work = nullptr;
        p->work_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&p->d_work, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(XB_ENOMEM, "solver workspace of %zu bytes: %s", bytes,
                         cudaGetErrorString(e));
    }
    p->work_bytes = bytes;
    return XB_OK;
}

// ---- features -----------------------------------------------------------------

__global__ void k_feat(int n, const int *__restrict__ rowptr, const int *__restrict__ col,
                       unsigned long long *__restrict__ acc /* [0] sum L^2, [1] max L, [2] max bw */) {
    __shared__ unsigned long long s2[32];
    __shared__ unsigned int mx[2];
    if (threadIdx.x == 0) mx[0] = mx[1] = 0;
    __syncthreads();
    unsigned long long sq = 0;
    unsigned int ml = 0, mb = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int a = rowptr[i], b = rowptr[i + 1];
        const unsigned int L = (unsigned int)(b - a);
        sq += (unsigned long long)L * L;
        ml = max(ml, L);
        if (b > a) {  // columns ascending: the extremes are the first and last
            mb = max(mb, (unsigned int)abs(col[a] - i));
            mb = max(mb, (unsigned int)abs(col[b - 1] - i));
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        sq += __shfl_xor_sync(0xffffffffu, sq, o);
        ml = max(ml, __shfl_xor_sync(0xffffffffu, ml, o));
        mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
    }
    if ((threadIdx.x & 31) == 0) {
        s2[threadIdx.x >> 5] = sq;
        atomicMax(&mx[0], ml);
        atomicMax(&mx[1], mb);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += s2[w];
        atomicAdd(&acc[0], t);
        atomicMax(&acc[1], (unsigned long long)mx[0]);
        atomicMax(&acc[2], (unsigned long long)mx[1]);
    }
}

// Exact symmetry test: every stored (i, j, v) has a stored (j, i, v).
__global__ void k_feat_sym(int n, const int *__restrict__ rowptr, const int *__restrict__ col,
                           const double *__restrict__ val, unsigned long long *__restrict__ bad) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        for (int k = rowptr[i]; k < rowptr[i + 1]; k++) {
            const int j = col[k];
            int lo = rowptr[j], hi = rowptr[j + 1] - 1;
            int found = -1;
            while (lo <= hi) {
                const int mid = (lo + hi) >> 1;
                const int c = col[mid];
                if (c == i) {
                    found = mid;
                    break;
                }
                if (c < i) lo = mid + 1;
                else hi = mid - 1;
            }
            if (found < 0 || val[found] != val[k]) {
                atomicOr(bad, 1ull);
                return;
            }
        }
    }
}

}  // namespace xb

using namespace xb;

namespace xb {
// Reduction scratch, pinned host mirror and timing events of a plan.
int plan_scratch(xb_plan *p, cudaStream_t s) {
    cudaError_t e = cudaMalloc(&p->d_part, (size_t)kRedSlots * kRedValues * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&p->d_ticket, 64 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&p->d_scal, (size_t)kScalars * sizeof(double));
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_ticket, 0, 64 * sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_scal, 0, (size_t)kScalars * sizeof(double), s);
    if (e == cudaSuccess) e = cudaMallocHost(&p->h_pin, 64 * sizeof(double));
    if (e == cudaSuccess) e = cudaEventCreate(&p->ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&p->ev[1]);
    return e == cudaSuccess ? XB_OK : cuda_error(e, "plan_create: scratch");
}

// A plan over A whose columns index an x of ncols entries (ncols = n except
// for the row blocks of a split plan).
int plan_create_impl(const xb_csr *A, int ncols, cudaStream_t s, xb_plan **out) {
    const int n = A->n, nnz = A->nnz;
    if (n < 0 || nnz < 0 || n > INT_MAX - 64 || nnz > INT_MAX - 64)
        return set_error(XB_EINVAL, "plan_create: n=%d nnz=%d (int32 indices, < 2^31 - 64)", n,
                         nnz);
    if (n > 0 && (!A->rowptr || (nnz > 0 && (!A->col || !A->val))))
        return set_error(XB_EINVAL, "plan_create: NULL CRS array");
    xb_plan *p = new (std::nothrow) xb_plan();
    if (!p) return set_error(XB_ENOMEM, "plan_create: host allocation");
    p->n = n;
    p->nnz = nnz;
    p->ncols = ncols;
    p->nnz64 = nnz;
    p->sym = A->sym_upper ? 1 : 0;
    p->rowptr = A->rowptr;
    p->col = A->col;
    p->val = A->val;
    auto fail = [&](int code) {
        xb_plan_destroy(p);
        return code;
    };
    p->h_rowptr.resize((size_t)n + 1, 0);
    if (n > 0) {
        cudaError_t e = cudaMemcpyAsync(p->h_rowptr.data(), A->rowptr, ((size_t)n + 1) * sizeof(int),
                                        cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return fail(cuda_error(e, "plan_create: read rowptr"));
    }
    const int *rp = p->h_rowptr.data();
    if (rp[0] != 0 || rp[n] != nnz)
        return fail(set_error(XB_EINVAL, "plan_create: rowptr[0]=%d rowptr[n]=%d nnz=%d", rp[0],
                              rp[n], nnz));
    std::vector<int> empty;
    for (int i = 0; i < n; i++) {
        const int L = rp[i + 1] - rp[i];
        if (L < 0) return fail(set_error(XB_EINVAL, "plan_create: rowptr decreases at row %d", i));
        p->max_row = std::max(p->max_row, L);
        if (L == 0) empty.push_back(i);
    }
    const char *val_env = std::getenv("XB_VALIDATE");
    if (val_env && val_env[0] == '1' && nnz > 0) {
        std::vector<int> hc(nnz);
        cudaError_t e = cudaMemcpy(hc.data(), A->col, (size_t)nnz * sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return fail(cuda_error(e, "plan_create: read col"));
        for (int i = 0; i < n; i++)
            for (int k = rp[i]; k < rp[i + 1]; k++) {
                const int c = hc[k];
                if (c < 0 || c >= ncols || (k > rp[i] && c <= hc[k - 1]) || (p->sym && c < i))
                    return fail(set_error(XB_EINVAL, "plan_create: bad column %d at row %d (k=%d)",
                                          c, i, k));
            }
    }
    p->n_empty = (int)empty.size();
    if (p->n_empty) {
        cudaError_t e = cudaMalloc(&p->d_empty, empty.size() * sizeof(int));
        if (e == cudaSuccess)
            e = cudaMemcpy(p->d_empty, empty.data(), empty.size() * sizeof(int), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail(cuda_error(e, "plan_create: empty rows"));
    }
    {
        const int r = plan_scratch(p, s);
        if (r != XB_OK) return fail(r);
    }
    // default choice (Sec. 3.3.1 STABLE policy: no tuning): power-law rows go to
    // the segmented scan, everything else to the nnz-balanced tiles.
    if (p->sym) {
        p->variant = XB_VAR_SYM_TILE;
    } else {
        const double mean = n > 0 ? (double)nnz / n : 0.0;
        p->variant = (p->max_row > 64 && p->max_row > 16.0 * mean) ? XB_VAR_SEGSCAN : XB_VAR_NNZ;
    }
    p->block = 256;
    p->ipt = 8;
    p->vec_ok = ((uintptr_t)A->val % 16 == 0) && ((uintptr_t)A->col % 16 == 0);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(cuda_error(e, "plan_create"));
    *out = p;
    return XB_OK;
}

}  // namespace xb

extern "C" {

const char *xb_last_error(void) { return g_err.c_str(); }

void xb_options_default(xb_options *o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->tol = 1e-8;
    o->maxiter = 1000000;
    o->maxtime_s = 1000.0;
    o->m = 30;
    o->m_max = 120;
    o->dafrt = 0;
    o->dafrt_theta = 10.0;
    o->dafrt_window = 5;
    o->dafrt_dm = 5;
    o->ortho = XB_ORTHO_MGS;
    o->precision = XB_PREC_FP64;
    o->tol_inner = 1e-4;
    o->maxiter_inner = 300;
    o->max_outer = 60;
    o->variant = XB_VAR_AUTO;
    o->block = 0;
    o->ipt = 0;
    o->tuner = XB_TUNER_NONE;
    o->check_every = 1;
    o->timing = 0;
    o->policy = XB_POLICY_NONE;
    o->fault_check = 1;
    o->precond = XB_PRECOND_NONE;
    o->ir_fallback = 1;
    o->small_n = 8192;
    if (const char *e = std::getenv("XB_SMALL_N")) o->small_n = std::max(0, std::atoi(e));
}


int xb_plan_create(const xb_csr *A, const xb_options *opt, void *stream, xb_plan **out) {
    (void)opt;
    if (!A || !out) return set_error(XB_EINVAL, "plan_create: NULL argument");
    *out = nullptr;
    return xb::plan_create_impl(A, A->n, (cudaStream_t)stream, out);
}


int xb_plan_destroy(xb_plan *p) {
    if (!p) return XB_OK;
    cudaDeviceSynchronize();
    for (auto &sb : p->subs) xb_plan_destroy(sb.plan);
    cudaFree(p->d_rp32_own);
    for (auto &t : p->tiles) cudaFree(t.d_row);
    for (auto &t : p->u2) {
        cudaFree(t.d_tile);
        cudaFree(t.d_long);
    }
    for (auto &t : p->bcsr) {
        cudaFree(t.d_bptr);
        cudaFree(t.d_bcol);
        cudaFree(t.d_val);
        cudaFree(t.d_val32);
    }
    for (auto &t : p->s3) {
        cudaFree(t.d_tslot);
        cudaFree(t.d_sgran);
        cudaFree(t.d_gid);
        cudaFree(t.d_gptr);
        cudaFree(t.d_gslot);
        cudaFree(t.d_part);
    }
    for (auto &t : p->segs) {
        cudaFree(t.d_row);
        cudaFree(t.d_carry_row);
        cudaFree(t.d_carry_val);
    }
    for (auto &t : p->sells) {
        cudaFree(t.d_off);
        cudaFree(t.d_perm);
        cudaFree(t.d_len);
        cudaFree(t.d_col);
        cudaFree(t.d_val);
        cudaFree(t.d_val32);
    }
    cudaFree(p->val32);
    cudaFree(p->bss.d_endbits);
    cudaFree(p->bss.d_ne_rows);
    cudaFree(p->bss.d_crp);
    for (auto &t : p->bss.copies) {
        cudaFree(t.d_col);
        cudaFree(t.d_val);
        cudaFree(t.d_val32);
    }
    cudaFree(p->d_empty);
    cudaFree(p->d_part);
    cudaFree(p->d_ticket);
    cudaFree(p->d_scal);
    cudaFree(p->d_work);
    xb::ilu_free(p);
    if (p->h_pin) cudaFreeHost(p->h_pin);
    for (auto &e : p->ev)
        if (e) cudaEventDestroy(e);
    delete p;
    return XB_OK;
}

int xb_plan_set_choice(xb_plan *p, int32_t variant, int32_t block, int32_t ipt) {
    if (!p) return set_error(XB_EINVAL, "set_choice: NULL plan");
    if (!variant_fits(p, variant))
        return set_error(XB_EINVAL, "set_choice: variant %d does not fit this storage", variant);
    if (block != 64 && block != 128 && block != 256 && block != 512)
        return set_error(XB_EINVAL, "set_choice: block %d", block);
    if (ipt < 1 || ipt > 32) return set_error(XB_EINVAL, "set_choice: ipt %d", ipt);
    p->variant = variant;
    p->block = block;
    p->ipt = ipt;
    return XB_OK;
}

int xb_plan_get_choice(const xb_plan *p, xb_choice *out) {
    if (!p || !out) return set_error(XB_EINVAL, "get_choice: NULL argument");
    out->variant = p->variant;
    out->block = p->block;
    out->ipt = p->ipt;
    out->ms = p->tuned_ms;
    return XB_OK;
}

int xb_features(const xb_csr *A, double *raw, float *feat, void *stream) {
    if (!A) return set_error(XB_EINVAL, "features: NULL matrix");
    cudaStream_t s = (cudaStream_t)stream;
    const int n = A->n, nnz = A->nnz;
    unsigned long long h[4] = {0, 0, 0, 0};
    if (n > 0) {
        unsigned long long *d = nullptr;
        XB_CUDA(cudaMalloc(&d, 4 * sizeof(unsigned long long)));
        cudaMemsetAsync(d, 0, 4 * sizeof(unsigned long long), s);
        const int g = std::max(1, std::min(num_sms() * 8, (n + 255) / 256));
        k_feat<<<g, 256, 0, s>>>(n, A->rowptr, A->col, d);
        if (!A->sym_upper && nnz > 0) k_feat_sym<<<g, 256, 0, s>>>(n, A->rowptr, A->col, A->val, d + 3);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h, d, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaFree(d);
        if (e != cudaSuccess) return cuda_error(e, "features");
    }
    const double dn = n, mean = n > 0 ? (double)nnz / n : 0.0;
    double var = n > 0 ? ((double)h[0] - (double)nnz * mean) / dn : 0.0;
    if (var < 0) var = 0;
    const double r[7] = {dn, (double)nnz, mean, var, (double)h[1], (double)h[2],
                         (A->sym_upper || h[3] == 0) ? 1.0 : 0.0};
    if (raw)
        for (int i = 0; i < 7; i++) raw[i] = r[i];
    if (feat) {
        feat[0] = (float)std::log1p(r[0]);
        feat[1] = (float)std::log1p(r[1]);
        feat[2] = (float)std::log1p(r[2]);
        feat[3] = (float)std::log1p(r[3]);
        feat[4] = (float)std::log1p(r[4]);
        feat[5] = (float)std::log1p(r[5]);
        feat[6] = (float)r[6];
        feat[7] = (float)(std::log1p(r[4]) - std::log1p(r[2]));
    }
    return XB_OK;
}

}  // extern "C"

extern "C" int xb_sell_layout(int32_t n, const int32_t *rowptr, int32_t sigma, int32_t *perm,
                              int32_t *slen, int64_t *off, int64_t *total) {
    if (n < 0 || !rowptr || sigma < 1 || !total)
        return xb::set_error(XB_EINVAL, "sell_layout: bad argument");
    std::vector<int> pv, lv;
    std::vector<int64_t> ov;
    *total = xb::sell_layout(n, rowptr, sigma, pv, lv, ov);
    if (perm) std::copy(pv.begin(), pv.end(), perm);
    if (slen) std::copy(lv.begin(), lv.end(), slen);
    if (off) std::copy(ov.begin(), ov.end(), off);
    return XB_OK;
}

extern "C" int xb_u2_layout(int32_t n, const int32_t *rowptr, int32_t ipt, int32_t *tiles,
                            int32_t cap_tiles, int32_t *ntiles, int32_t *longs, int32_t cap_long,
                            int32_t *nlong) {
    if (n < 0 || !rowptr || ipt < 1 || ipt > 16 || !ntiles || !nlong || cap_tiles < 0 ||
        cap_long < 0 || (cap_tiles > 0 && !tiles) || (cap_long > 0 && !longs))
        return xb::set_error(XB_EINVAL, "u2_layout: bad argument");
    std::vector<int4> tv;
    std::vector<int> lv;
    xb::u2_layout(n, rowptr, ipt, tv, lv);
    *ntiles = (int32_t)tv.size();
    *nlong = (int32_t)lv.size();
    for (int i = 0; i < (int)tv.size() && i < cap_tiles; i++) {
        tiles[4 * i] = tv[i].x;
        tiles[4 * i + 1] = tv[i].y;
        tiles[4 * i + 2] = tv[i].z;
        tiles[4 * i + 3] = tv[i].w;
    }
    for (int i = 0; i < (int)lv.size() && i < cap_long; i++) longs[i] = lv[i];
    return XB_OK;
}

extern "C" int xb_bcsr_layout(int32_t n, const int32_t *rowptr, const int32_t *col, int32_t r,
                              int32_t *bptr, int32_t *bcol, int64_t cap, int64_t *nblocks) {
    if (n < 0 || !rowptr || (n > 0 && rowptr[n] > 0 && !col) || r < 1 || !nblocks || cap < 0 ||
        (cap > 0 && !bcol))
        return xb::set_error(XB_EINVAL, "bcsr_layout: bad argument");
    std::vector<int> bp, bc;
    *nblocks = xb::bcsr_layout(n, rowptr, col, r, bp, bc);
    if (bptr) std::copy(bp.begin(), bp.end(), bptr);
    for (int64_t i = 0; i < *nblocks && i < cap; i++) bcol[i] = bc[i];
    return XB_OK;
}

namespace xb {

int split_rows64(int n, const int64_t *rp, int64_t max_nnz, std::vector<int> &starts) {
    starts.clear();
    if (max_nnz < 1) return set_error(XB_EINVAL, "split_rows64: max_nnz %lld", (long long)max_nnz);
    if (n > 0 && rp[0] != 0) return set_error(XB_EINVAL, "split_rows64: rowptr[0] = %lld", (long long)rp[0]);
    int r = 0;
    while (r < n) {
        if (rp[r + 1] < rp[r])
            return set_error(XB_EINVAL, "split_rows64: rowptr decreases at row %d", r);
        if (rp[r + 1] - rp[r] > max_nnz)
            return set_error(XB_EINVAL, "split_rows64: row %d holds %lld non-zeros (> %lld)", r,
                             (long long)(rp[r + 1] - rp[r]), (long long)max_nnz);
        starts.push_back(r);
        int rb = r + 1;
        while (rb < n && rp[rb + 1] >= rp[rb] && rp[rb + 1] - rp[r] <= max_nnz) rb++;
        r = rb;
    }
    starts.push_back(n);
    return XB_OK;
}

// rp32[i] = rp64[i] - base, i < count
__global__ void k_rp_narrow(int64_t count, const int64_t *__restrict__ rp64, int64_t base,
                            int *__restrict__ rp32) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < count) rp32[i] = (int)(rp64[i] - base);
}

}  // namespace xb

extern "C" int xb_split_rows64(int32_t n, const int64_t *rowptr, int64_t max_nnz, int32_t *starts,
                               int32_t cap, int32_t *nblocks) {
    if (n < 0 || !rowptr || !nblocks || cap < 0 || (cap > 0 && !starts))
        return xb::set_error(XB_EINVAL, "split_rows64: bad argument");
    std::vector<int> st;
    XB_TRY(xb::split_rows64(n, rowptr, max_nnz, st));
    *nblocks = (int32_t)st.size() - 1;
    for (int i = 0; i < (int)st.size() && i < cap; i++) starts[i] = st[i];
    return XB_OK;
}

extern "C" int xb_plan_create64(const xb_csr64 *A, const xb_options *opt, void *stream,
                                xb_plan **out) {
    (void)opt;
    if (!A || !out) return xb::set_error(XB_EINVAL, "plan_create64: NULL argument");
    *out = nullptr;
    const int n = A->n;
    const int64_t nnz = A->nnz;
    if (n < 0 || nnz < 0 || n > INT_MAX - 64)
        return xb::set_error(XB_EINVAL, "plan_create64: n=%d nnz=%lld", n, (long long)nnz);
    if (n > 0 && (!A->rowptr || (nnz > 0 && (!A->col || !A->val))))
        return xb::set_error(XB_EINVAL, "plan_create64: NULL CRS array");
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int64_t> rp((size_t)n + 1, 0);
    if (n > 0) {
        cudaError_t e = cudaMemcpyAsync(rp.data(), A->rowptr, ((size_t)n + 1) * sizeof(int64_t),
                                        cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return xb::cuda_error(e, "plan_create64: read rowptr");
    }
    if (rp[0] != 0 || rp[n] != nnz)
        return xb::set_error(XB_EINVAL, "plan_create64: rowptr[0]=%lld rowptr[n]=%lld nnz=%lld",
                             (long long)rp[0], (long long)rp[n], (long long)nnz);
    int64_t limit = INT_MAX - 64;
    if (const char *e = std::getenv("XB_PLAN_SPLIT_NNZ")) limit = std::max(1LL, std::atoll(e));
    std::vector<int> starts;
    XB_TRY(xb::split_rows64(n, rp.data(), std::min<int64_t>(limit, INT_MAX - 64), starts));
    // one row block (or none): an ordinary plan on an int32 copy of rowptr
    auto narrow = [&](int r0, int r1, int **d32) -> int {
        const int64_t cnt = (int64_t)(r1 - r0) + 1;
        cudaError_t e = cudaMalloc(d32, cnt * sizeof(int));
        if (e == cudaSuccess) {
            xb::k_rp_narrow<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(cnt, A->rowptr + r0, rp[r0],
                                                                         *d32);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            cudaFree(*d32);
            *d32 = nullptr;
            return xb::cuda_error(e, "plan_create64: narrow rowptr");
        }
        return XB_OK;
    };
    if (starts.size() <= 2) {
        int *d32 = nullptr;
        XB_TRY(narrow(0, n, &d32));
        xb_csr c{n, (int32_t)nnz, d32, A->col, A->val, A->sym_upper};
        const int r = xb::plan_create_impl(&c, n, s, out);
        if (r != XB_OK) {
            cudaFree(d32);
            return r;
        }
        (*out)->d_rp32_own = d32;
        return XB_OK;
    }
    if (A->sym_upper)
        return xb::set_error(XB_EINVAL, "plan_create64: symmetric storage beyond 2^31 - 64 non-zeros");
    xb_plan *p = new (std::nothrow) xb_plan();
    if (!p) return xb::set_error(XB_ENOMEM, "plan_create64: host allocation");
    auto fail = [&](int code) {
        xb_plan_destroy(p);
        return code;
    };
    p->n = n;
    p->ncols = n;
    p->nnz64 = nnz;
    p->nnz = INT_MAX - 64;  // saturated; nnz64 holds the count
    {
        const int r = xb::plan_scratch(p, s);
        if (r != XB_OK) return fail(r);
    }
    for (size_t b = 0; b + 1 < starts.size(); b++) {
        const int r0 = starts[b], r1 = starts[b + 1];
        int *d32 = nullptr;
        {
            const int r = narrow(r0, r1, &d32);
            if (r != XB_OK) return fail(r);
        }
        xb_csr c{r1 - r0, (int32_t)(rp[r1] - rp[r0]), d32, A->col + rp[r0], A->val + rp[r0], 0};
        xb_plan *q = nullptr;
        const int r = xb::plan_create_impl(&c, n, s, &q);
        if (r != XB_OK) {
            cudaFree(d32);
            return fail(r);
        }
        q->d_rp32_own = d32;
        p->subs.push_back({r0, q});
        p->max_row = std::max(p->max_row, q->max_row);
        p->n_empty += q->n_empty;
    }
    p->variant = p->subs[0].plan->variant;
    p->block = p->subs[0].plan->block;
    p->ipt = p->subs[0].plan->ipt;
    *out = p;
    return XB_OK;
}
