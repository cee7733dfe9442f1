// Krylov vector kernels: deterministic two-stage reductions (per-CTA partials,
// the last CTA to finish reduces them in a fixed order, so no extra launch and
// no run-to-run variation), the fused modified Gram-Schmidt step of Arnoldi
// (Sec. 3.2.2, MGS) with the Givens update folded into its final CTA, and the
// fused BiCGStab updates.  Scalars never leave the device inside a step.
#include <cstdlib>
#include "krylov.cuh"

#include <cmath>

namespace {

constexpr int kVB = 256;  // block size of all streaming vector kernels

// Reduce NV per-thread values over the grid.  Returns true in every thread of
// the last CTA to finish; tot[] is then valid in thread 0 of that CTA.
template <int NV>
__device__ __forceinline__ bool grid_reduce(double (&v)[NV], double *__restrict__ part,
                                            unsigned *__restrict__ ticket, double (&tot)[NV]) {
    __shared__ double sh[32];
    __shared__ bool last;
    const int G = gridDim.x;
#pragma unroll
    for (int k = 0; k < NV; k++) {
        const double b = xbd::block_sum(v[k], sh);
        if (threadIdx.x == 0) part[k * G + blockIdx.x] = b;
    }
    if (threadIdx.x == 0) {
        __threadfence();
        last = (atomicAdd(ticket, 1u) == (unsigned)G - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
#pragma unroll
    for (int k = 0; k < NV; k++) {
        double a = 0.0;
        for (int i = threadIdx.x; i < G; i += blockDim.x) a += __ldcg(part + k * G + i);
        tot[k] = xbd::block_sum(a, sh);
    }
    if (threadIdx.x == 0) *ticket = 0u;
    return true;
}

__device__ __forceinline__ int64_t gtid() { return blockIdx.x * (int64_t)blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gstride() { return (int64_t)gridDim.x * blockDim.x; }

// ---- plain vector ops --------------------------------------------------------

__global__ void k_dot(int64_t n, const double *__restrict__ x, const double *__restrict__ y,
                      double *__restrict__ part, unsigned *__restrict__ ticket,
                      double *__restrict__ out, int sq, int vec) {
    double a0 = 0.0, a1 = 0.0;
    int64_t done = 0;
    if (vec) {
        const double2 *x2 = reinterpret_cast<const double2 *>(x);
        const double2 *y2 = reinterpret_cast<const double2 *>(y);
        const int64_t nv = n / 2;
        for (int64_t e = gtid(); e < nv; e += gstride()) {
            const double2 a = x2[e], b = y2[e];
            a0 = fma(a.x, b.x, a0);
            a1 = fma(a.y, b.y, a1);
        }
        done = nv * 2;
    }
    for (int64_t i = done + gtid(); i < n; i += gstride()) a0 = fma(x[i], y[i], a0);
    double v[1] = {a0 + a1};
    double t[1];
    if (grid_reduce<1>(v, part, ticket, t) && threadIdx.x == 0) *out = sq ? sqrt(t[0]) : t[0];
}

__global__ void k_axpy(int64_t n, double a, const double *__restrict__ x, double *__restrict__ y) {
    for (int64_t i = gtid(); i < n; i += gstride()) y[i] = fma(a, x[i], y[i]);
}
__global__ void k_copy(int64_t n, const double *__restrict__ x, double *__restrict__ y) {
    for (int64_t i = gtid(); i < n; i += gstride()) y[i] = x[i];
}
__global__ void k_scale(int64_t n, double a, double *__restrict__ x) {
    for (int64_t i = gtid(); i < n; i += gstride()) x[i] *= a;
}
__global__ void k_fill(int64_t n, double a, double *__restrict__ x) {
    for (int64_t i = gtid(); i < n; i += gstride()) x[i] = a;
}

// Grid of a streaming/reduction launch of kernel k over n elements: exactly the
// CTAs that fit on the GPU at once (fewer for small n), so a grid-stride pass
// runs as one coherent wave.
template <typename K>
int rgrid(K k, int64_t n) {
    return xb::resident_grid((const void *)k, kVB, n, 4);
}

// ---- GMRES ----------------------------------------------------------------------

// ||r0|| -> start a cycle: g = (beta, 0, ...), sc[0] = 1/beta.
template <typename VB>
__global__ void k_gm_init(int64_t n, const VB *__restrict__ r0, xb::GmDev st, double tau,
                          double *__restrict__ part, unsigned *__restrict__ ticket) {
    double v[1] = {0.0};
    for (int64_t i = gtid(); i < n; i += gstride()) {
        const double a = (double)r0[i];
        v[0] = fma(a, a, v[0]);
    }
    double t[1];
    if (grid_reduce<1>(v, part, ticket, t)) {
        for (int i = threadIdx.x; i <= st.M; i += blockDim.x) st.g[i] = 0.0;
        __syncthreads();
        if (threadIdx.x == 0) {
            const double beta = sqrt(t[0]);
            st.g[0] = beta;
            st.sc[0] = beta > 0.0 ? 1.0 / beta : 0.0;
            st.scf[0] = (float)st.sc[0];
            st.misc[xb::GM_BETA] = beta;
            const double bn = st.misc[xb::GM_BNORM];
            st.misc[xb::GM_RES] = bn > 0.0 ? beta / bn : 0.0;
            st.misc[xb::GM_K] = 0.0;
            st.misc[xb::GM_STOP] = 0.0;
            st.misc[xb::GM_TAU] = tau;
            st.misc[xb::GM_LEN2] = 0.0;
            st.misc[xb::GM_RAW] = 0.0;
        }
    }
}

// Givens update of column j after h_{j+1,j} = hn (single thread).
__device__ void gm_givens(xb::GmDev st, int j, double hn) {
    double *col = st.H + (size_t)j * (st.M + 1);
    col[j + 1] = hn;
    const double len2 = st.misc[xb::GM_LEN2] + hn * hn;
    for (int i = 0; i < j; i++) {
        const double a = col[i], b = col[i + 1];
        col[i] = st.cs[i] * a + st.sn[i] * b;
        col[i + 1] = -st.sn[i] * a + st.cs[i] * b;
    }
    const double a = col[j];
    const double rr = hypot(a, hn);
    if (rr == 0.0) {  // A v_j lies in span(v_0..v_{j-1}) with a zero pivot: singular
        st.misc[xb::GM_STOP] = 2.0;
        return;
    }
    st.cs[j] = a / rr;
    st.sn[j] = hn / rr;
    col[j] = rr;
    col[j + 1] = 0.0;
    st.g[j + 1] = -st.sn[j] * st.g[j];
    st.g[j] = st.cs[j] * st.g[j];
    const double bn = st.misc[xb::GM_BNORM];
    const double res = fabs(st.g[j + 1]) / bn;
    st.misc[xb::GM_RES] = res;
    st.misc[xb::GM_K] = (double)(j + 1);
    if (hn <= 1e-14 * sqrt(len2)) {  // happy breakdown: the Krylov space is invariant
        st.misc[xb::GM_STOP] = 1.0;
        st.sc[j + 1] = 0.0;
        st.scf[j + 1] = 0.0f;
        return;
    }
    st.sc[j + 1] = 1.0 / hn;
    st.scf[j + 1] = (float)(1.0 / hn);
    if (res <= st.misc[xb::GM_TAU]) st.misc[xb::GM_STOP] = 1.0;
}

template <typename VB>
struct V16;
template <>
struct V16<double> {
    using T = double2;
    static constexpr int N = 2;
    __device__ static double get(const double2 &v, int k) { return k == 0 ? v.x : v.y; }
    __device__ static void set(double2 &v, int k, double a) {
        if (k == 0) v.x = a;
        else v.y = a;
    }
};
template <>
struct V16<float> {
    using T = float4;
    static constexpr int N = 4;
    __device__ static float get(const float4 &v, int k) {
        return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
    }
    __device__ static void set(float4 &v, int k, float a) {
        if (k == 0) v.x = a;
        else if (k == 1) v.y = a;
        else if (k == 2) v.z = a;
        else v.w = a;
    }
};

// One element of the MGS launch: OP 0 dot(w, vn); OP 1 w -= c vp, dot(w, vn);
// OP 2 w -= c vp, dot(w, w).
template <int OP, typename VB>
__device__ __forceinline__ VB mgs_elem(VB &w, VB vp, VB vn, VB c, VB acc) {
    if (OP != 0) w = fma(-c, vp, w);
    return OP == 2 ? fma(w, w, acc) : fma(w, vn, acc);
}

// 16-byte load with an L2 evict-first policy: v_{i-1} is read for the last time
// in the sweep, so its lines should make way for w and v_i.
__device__ __forceinline__ uint64_t l2_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ double2 ld_last_use(const double2 *a, uint64_t pol) {
    double2 v;
    asm volatile("ld.global.nc.L2::cache_hint.v2.f64 {%0,%1}, [%2], %3;"
                 : "=d"(v.x), "=d"(v.y) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ float4 ld_last_use(const float4 *a, uint64_t pol) {
    float4 v;
    asm volatile("ld.global.nc.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(a), "l"(pol));
    return v;
}

// One launch of the MGS sweep of Arnoldi step j:
//   i == 0      : h_0j = (w, v_0)
//   0 < i <= j  : w -= h_{i-1,j} v_{i-1};  h_ij = (w, v_i)
//   i == j+1    : w -= h_jj v_j;  h_{j+1,j} = ||w||, then Givens.
// Basis vectors are stored unnormalised with scales sc (v_i = sc[i]*V_i).
// Operands move as 16-byte vectors (two grid-wide chunks per thread per
// iteration) when the three arrays are 16-byte aligned.  flags bit 0: walk the
// chunks from the end of the vectors (consecutive launches of a sweep alternate
// direction, so each starts on the w and v_i lines that the previous one
// touched last and still finds them in L2); bit 1: load v_{i-1} with an L2
// evict-first policy.
template <int OP, typename VB>
__global__ void __launch_bounds__(kVB) k_mgs(int64_t n, VB *__restrict__ w,
                                             const VB *__restrict__ vprev,
                                             const VB *__restrict__ vnext, xb::GmDev st, int j,
                                             int i, double *__restrict__ part,
                                             unsigned *__restrict__ ticket, int vec, int flags) {
    if (st.misc[xb::GM_STOP] != 0.0) return;
    const VB c = (VB)(OP != 0 ? st.misc[xb::GM_COEF] : 0.0);
    VB acc0 = VB(0), acc1 = VB(0);
    int64_t done = 0;
    if (vec) {
        using T = typename V16<VB>::T;
        constexpr int N = V16<VB>::N;
        const int64_t nv = n / N;
        T *w2 = reinterpret_cast<T *>(w);
        const T *p2 = reinterpret_cast<const T *>(OP != 0 ? vprev : w);
        const T *q2 = reinterpret_cast<const T *>(OP != 2 ? vnext : w);
        const bool rev = flags & 1, hint = flags & 2;
        const uint64_t pol = l2_evict_first();
        const int64_t gs = gstride();
        const int64_t full = nv / gs;            // grid-wide chunks every thread owns
        const int64_t et = full * gs + gtid();   // this thread's slot in the partial chunk
        auto one = [&](int64_t e) {
            T a = w2[e];
            const T pa = OP != 0 ? (hint ? ld_last_use(p2 + e, pol) : p2[e]) : a;
            const T qa = OP != 2 ? q2[e] : a;
#pragma unroll
            for (int k = 0; k < N; k++) {
                VB x = V16<VB>::get(a, k);
                acc0 = mgs_elem<OP>(x, V16<VB>::get(pa, k), V16<VB>::get(qa, k), c, acc0);
                V16<VB>::set(a, k, x);
            }
            if (OP != 0) w2[e] = a;
        };
        if (rev && et < nv) one(et);
        int64_t k = 0;
        for (; k + 1 < full; k += 2) {
            const int64_t ka = rev ? full - 1 - k : k;
            const int64_t e = ka * gs + gtid();
            const int64_t f = rev ? e - gs : e + gs;
            T a = w2[e], b = w2[f];
            const T pa = OP != 0 ? (hint ? ld_last_use(p2 + e, pol) : p2[e]) : a;
            const T pb = OP != 0 ? (hint ? ld_last_use(p2 + f, pol) : p2[f]) : b;
            const T qa = OP != 2 ? q2[e] : a, qb = OP != 2 ? q2[f] : b;
#pragma unroll
            for (int q = 0; q < N; q++) {
                VB x = V16<VB>::get(a, q), y = V16<VB>::get(b, q);
                acc0 = mgs_elem<OP>(x, V16<VB>::get(pa, q), V16<VB>::get(qa, q), c, acc0);
                acc1 = mgs_elem<OP>(y, V16<VB>::get(pb, q), V16<VB>::get(qb, q), c, acc1);
                V16<VB>::set(a, q, x);
                V16<VB>::set(b, q, y);
            }
            if (OP != 0) {
                w2[e] = a;
                w2[f] = b;
            }
        }
        if (k < full) one((rev ? full - 1 - k : k) * gs + gtid());
        if (!rev && et < nv) one(et);
        done = nv * N;
    }
    for (int64_t e = done + gtid(); e < n; e += gstride()) {
        VB x = w[e];
        acc0 = mgs_elem<OP>(x, OP != 0 ? vprev[e] : x, OP != 2 ? vnext[e] : x, c, acc0);
        if (OP != 0) w[e] = x;
    }
    double v[1] = {(double)acc0 + (double)acc1};
    double t[1];
    if (grid_reduce<1>(v, part, ticket, t) && threadIdx.x == 0) {
        if (OP != 2) {
            const double h = st.sc[i] * t[0];
            st.H[(size_t)j * (st.M + 1) + i] = h;
            st.misc[xb::GM_COEF] = st.sc[i] * h;
            st.misc[xb::GM_LEN2] = (i == 0 ? 0.0 : st.misc[xb::GM_LEN2]) + h * h;
        } else if (st.misc[xb::GM_RAW] != 0.0) {
            st.H[(size_t)j * (st.M + 1) + j + 1] = sqrt(t[0]);
        } else {
            gm_givens(st, j, sqrt(t[0]));
        }
    }
}

// ---- block Gram-Schmidt family: CGS, DGKS, BCGS (Sec. 3.2.2) ----------------------

constexpr int kMaxCoef = 520;  // >= M + 1 for every basis capacity M <= 512
constexpr int kBgsAcc = 1, kBgsFin = 2, kBgsRev = 4;

// Sum cnt <= NV per-thread values over the grid.  Returns true in every thread
// of the last CTA to finish, with the totals in tot[0..cnt) (shared memory),
// summed in a fixed order (deterministic).
template <int NV>
__device__ bool grid_reduce_n(const double (&v)[NV], int cnt, double *__restrict__ part,
                              unsigned *__restrict__ ticket, double *tot) {
    __shared__ double sh[NV][kVB / 32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int G = gridDim.x;
#pragma unroll
    for (int q = 0; q < NV; q++) {
        if (q < cnt) {
            double a = v[q];
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            if (lane == 0) sh[q][wp] = a;
        }
    }
    __syncthreads();
    if ((int)threadIdx.x < cnt) {
        double a = 0.0;
        for (int k = 0; k < nw; k++) a += sh[threadIdx.x][k];
        part[(size_t)threadIdx.x * G + blockIdx.x] = a;
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == (unsigned)G - 1);
    __syncthreads();
    if (!last) return false;
    __threadfence();
    for (int q = wp; q < cnt; q += nw) {
        double a = 0.0;
        for (int i = lane; i < G; i += 32) a += __ldcg(part + (size_t)q * G + i);
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) tot[q] = a;
    }
    if (threadIdx.x == 0) *ticket = 0u;
    __syncthreads();
    return true;
}

// U elements (16-byte vectors at e[0..U)) of one block Gram-Schmidt pass:
// update by the nu pending vectors (at most KU when KU > 0), store w, then the
// nd dot products (or the squared norm when fin).  The U elements' loads are
// issued together.
template <typename VB, int KD, int KU, int U>
__device__ __forceinline__ void bgs_elems(int64_t ea, int64_t eb, typename V16<VB>::T *w2,
                                          const typename V16<VB>::T *V2, int64_t ldv, int u0,
                                          int nu, int d0, int nd, bool fin, const VB *cf,
                                          VB (&acc)[KD]) {
    using T = typename V16<VB>::T;
    constexpr int N = V16<VB>::N;
    const int64_t e[2] = {ea, eb};
    T x[U];
#pragma unroll
    for (int u = 0; u < U; u++) x[u] = w2[e[u]];
    if (nu > 0) {
        const int cnt = KU > 0 ? KU : nu;
#pragma unroll 4
        for (int i = 0; i < cnt; i++) {
            if (KU > 0 && i >= nu) break;
            const T *vi = V2 + (size_t)(u0 + i) * ldv;
            T v[U];
#pragma unroll
            for (int u = 0; u < U; u++) v[u] = vi[e[u]];
            const VB c = cf[i];
#pragma unroll
            for (int u = 0; u < U; u++)
#pragma unroll
                for (int q = 0; q < N; q++)
                    V16<VB>::set(x[u], q, fma(-c, V16<VB>::get(v[u], q), V16<VB>::get(x[u], q)));
        }
#pragma unroll
        for (int u = 0; u < U; u++) w2[e[u]] = x[u];
    }
    if (fin) {
#pragma unroll
        for (int u = 0; u < U; u++)
#pragma unroll
            for (int q = 0; q < N; q++)
                acc[0] = fma(V16<VB>::get(x[u], q), V16<VB>::get(x[u], q), acc[0]);
        return;
    }
#pragma unroll
    for (int d = 0; d < KD; d++) {
        if (d < nd) {
            const T *vd = V2 + (size_t)(d0 + d) * ldv;
            T v[U];
#pragma unroll
            for (int u = 0; u < U; u++) v[u] = vd[e[u]];
#pragma unroll
            for (int u = 0; u < U; u++)
#pragma unroll
                for (int q = 0; q < N; q++)
                    acc[d] = fma(V16<VB>::get(x[u], q), V16<VB>::get(v[u], q), acc[d]);
        }
    }
}

// One pass of the block Gram-Schmidt family for Arnoldi step j:
//   w -= sum_{u0 <= i < u1} coef_i V_i          (the pending update; none if u0 == u1;
//                                               at most KU vectors when KU > 0)
//   then either the dots (w, V_i) for d0 <= i < d0 + nd (nd <= KD), or, with
//   kBgsFin (nd == 0), (w, w).
// The last CTA turns dots into Hessenberg entries h_i = sc_i (w, V_i) (added to
// the column with kBgsAcc: the second pass of DGKS) and the coefficients the
// next pass subtracts, coef_i = sc_i h_i; with kBgsFin it stores
// h_{j+1,j} = ||w|| and applies the Givens update (or only stores it in raw
// mode).  kBgsRev walks the grid-wide chunks from the end (alternating passes
// start on the lines the previous pass touched last).  Operands move as
// 16-byte vectors, two grid-wide chunks per thread per iteration, when V, w
// and the row stride allow it.
template <typename VB, int KD, int KU, int MINB>
__global__ void __launch_bounds__(kVB, MINB) k_bgs(int64_t n, VB *__restrict__ w,
                                             const VB *__restrict__ V, int64_t ld, int u0, int u1,
                                             int d0, int nd, int flags, xb::GmDev st, int j,
                                             double *__restrict__ part,
                                             unsigned *__restrict__ ticket, int vec) {
    if (st.misc[xb::GM_STOP] != 0.0) return;
    __shared__ VB cf[kMaxCoef];
    __shared__ double tot[KD];
    const int nu = u1 - u0;
    for (int i = threadIdx.x; i < nu; i += blockDim.x) cf[i] = (VB)st.coef[u0 + i];
    __syncthreads();
    const bool fin = flags & kBgsFin, rev = flags & kBgsRev;
    VB acc[KD];
#pragma unroll
    for (int q = 0; q < KD; q++) acc[q] = VB(0);
    int64_t done = 0;
    if (vec) {
        using T = typename V16<VB>::T;
        constexpr int N = V16<VB>::N;
        const int64_t nv = n / N, ldv = ld / N;
        T *w2 = reinterpret_cast<T *>(w);
        const T *V2 = reinterpret_cast<const T *>(V);
        const int64_t gs = gstride();
        const int64_t full = nv / gs;           // grid-wide chunks every thread owns
        const int64_t et = full * gs + gtid();  // this thread's slot in the partial chunk
        if (rev && et < nv)
            bgs_elems<VB, KD, KU, 1>(et, et, w2, V2, ldv, u0, nu, d0, nd, fin, cf, acc);
        int64_t k = 0;
        for (; k + 1 < full; k += 2) {
            const int64_t e = (rev ? full - 1 - k : k) * gs + gtid();
            bgs_elems<VB, KD, KU, 2>(e, rev ? e - gs : e + gs, w2, V2, ldv, u0, nu, d0, nd, fin, cf,
                                     acc);
        }
        if (k < full) {
            const int64_t e = (rev ? full - 1 - k : k) * gs + gtid();
            bgs_elems<VB, KD, KU, 1>(e, e, w2, V2, ldv, u0, nu, d0, nd, fin, cf, acc);
        }
        if (!rev && et < nv)
            bgs_elems<VB, KD, KU, 1>(et, et, w2, V2, ldv, u0, nu, d0, nd, fin, cf, acc);
        done = nv * N;
    }
    for (int64_t e = done + gtid(); e < n; e += gstride()) {
        VB x = w[e];
        if (nu > 0) {
            for (int i = 0; i < nu; i++) x = fma(-cf[i], V[(size_t)(u0 + i) * ld + e], x);
            w[e] = x;
        }
        if (fin) {
            acc[0] = fma(x, x, acc[0]);
        } else {
#pragma unroll
            for (int q = 0; q < KD; q++)
                if (q < nd) acc[q] = fma(x, V[(size_t)(d0 + q) * ld + e], acc[q]);
        }
    }
    double v[KD];
#pragma unroll
    for (int q = 0; q < KD; q++) v[q] = (double)acc[q];
    if (!grid_reduce_n<KD>(v, fin ? 1 : nd, part, ticket, tot)) return;
    double *col = st.H + (size_t)j * (st.M + 1);
    if (!fin) {
        for (int q = threadIdx.x; q < nd; q += blockDim.x) {
            const int i = d0 + q;
            const double h = st.sc[i] * tot[q];
            col[i] = (flags & kBgsAcc) ? col[i] + h : h;
            st.coef[i] = st.sc[i] * h;
        }
    } else if (threadIdx.x == 0) {
        double len2 = 0.0;
        for (int i = 0; i <= j; i++) len2 += col[i] * col[i];
        st.misc[xb::GM_LEN2] = len2;
        if (st.misc[xb::GM_RAW] != 0.0) col[j + 1] = sqrt(tot[0]);
        else gm_givens(st, j, sqrt(tot[0]));
    }
}

// Least squares R y = g (upper triangular k x k), then y_i *= sc[i].
__global__ void k_gm_solve(xb::GmDev st) {
    if (threadIdx.x != 0) return;
    const int k = (int)st.misc[xb::GM_K];
    for (int i = k - 1; i >= 0; i--) {
        double s = st.g[i];
        for (int q = i + 1; q < k; q++) s -= st.H[(size_t)q * (st.M + 1) + i] * st.y[q];
        st.y[i] = s / st.H[(size_t)i * (st.M + 1) + i];
    }
    for (int i = 0; i < k; i++) st.y[i] *= st.sc[i];
}

// x += sum_i y_i V_i (each basis vector read once; 16-byte vectors when the
// basis and x are aligned).
template <typename VB, typename VX>
__global__ void __launch_bounds__(kVB) k_gm_xupd(int64_t n, const VB *__restrict__ V, int64_t ld,
                                                 xb::GmDev st, VX *__restrict__ x, int vec) {
    __shared__ double ys[512];
    const int k = (int)st.misc[xb::GM_K];
    for (int i = threadIdx.x; i < k && i < 512; i += blockDim.x) ys[i] = st.y[i];
    __syncthreads();
    int64_t done = 0;
    if (vec) {
        using T = typename V16<VB>::T;
        using TX = typename V16<VX>::T;
        constexpr int N = V16<VB>::N;
        static_assert(V16<VB>::N == V16<VX>::N, "same width");
        const int64_t nv = n / N;
        for (int64_t e = gtid(); e < nv; e += gstride()) {
            VX s[N];
#pragma unroll
            for (int q = 0; q < N; q++) s[q] = VX(0);
            for (int i = 0; i < k; i++) {
                const T v = reinterpret_cast<const T *>(V + (size_t)i * ld)[e];
                const VX yi = (VX)ys[i];
#pragma unroll
                for (int q = 0; q < N; q++) s[q] = fma(yi, (VX)V16<VB>::get(v, q), s[q]);
            }
            TX a = reinterpret_cast<TX *>(x)[e];
#pragma unroll
            for (int q = 0; q < N; q++) V16<VX>::set(a, q, V16<VX>::get(a, q) + s[q]);
            reinterpret_cast<TX *>(x)[e] = a;
        }
        done = nv * N;
    }
    for (int64_t e = done + gtid(); e < n; e += gstride()) {
        VX s = VX(0);
        for (int i = 0; i < k; i++) s = fma((VX)ys[i], (VX)V[(size_t)i * ld + e], s);
        x[e] += s;
    }
}

// ---- BiCGStab ------------------------------------------------------------------
// Every kernel walks its vectors as 16-byte pairs when all of them are 16-byte
// aligned (vec != 0), then finishes the odd tail element by element.

__device__ __forceinline__ double2 ld2(const double *a, int64_t i) {
    return reinterpret_cast<const double2 *>(a)[i];
}
__device__ __forceinline__ void st2(double *a, int64_t i, double2 v) {
    reinterpret_cast<double2 *>(a)[i] = v;
}

// rho = (rhat, r) with rhat = r at a (re)start; alpha = omega = rho_old = 1.
__global__ void k_bi_init(int64_t n, const double *__restrict__ r, double *__restrict__ sc,
                          double tau2, double *__restrict__ part, unsigned *__restrict__ ticket,
                          int vec) {
    double v[1] = {0.0};
    int64_t done = 0;
    if (vec) {
        for (int64_t i = gtid(); i < n / 2; i += gstride()) {
            const double2 a = ld2(r, i);
            v[0] = fma(a.y, a.y, fma(a.x, a.x, v[0]));
        }
        done = n / 2 * 2;
    }
    for (int64_t i = done + gtid(); i < n; i += gstride()) v[0] = fma(r[i], r[i], v[0]);
    double t[1];
    if (grid_reduce<1>(v, part, ticket, t) && threadIdx.x == 0) {
        sc[xb::BI_RHO] = t[0];
        sc[xb::BI_RHO_OLD] = 1.0;
        sc[xb::BI_ALPHA] = 1.0;
        sc[xb::BI_OMEGA] = 1.0;
        sc[xb::BI_RNORM2] = t[0];
        sc[xb::BI_SNORM2] = INFINITY;
        sc[xb::BI_FLAG] = 0.0;
        sc[xb::BI_TAU2] = tau2;
    }
}

// p = r + beta (p - omega v), beta = (rho/rho_old)(alpha/omega).
__global__ void k_bi_p(int64_t n, const double *__restrict__ sc, const double *__restrict__ r,
                       double *__restrict__ p, const double *__restrict__ v, int vec) {
    if (sc[xb::BI_FLAG] != 0.0) return;
    const double beta =
        (sc[xb::BI_RHO] / sc[xb::BI_RHO_OLD]) * (sc[xb::BI_ALPHA] / sc[xb::BI_OMEGA]);
    const double om = sc[xb::BI_OMEGA];
    auto f = [=](double ri, double pi, double vi) { return fma(beta, fma(-om, vi, pi), ri); };
    int64_t done = 0;
    if (vec) {
        for (int64_t i = gtid(); i < n / 2; i += gstride()) {
            const double2 a = ld2(r, i), c = ld2(v, i);
            double2 q = ld2(p, i);
            q.x = f(a.x, q.x, c.x);
            q.y = f(a.y, q.y, c.y);
            st2(p, i, q);
        }
        done = n / 2 * 2;
    }
    for (int64_t i = done + gtid(); i < n; i += gstride()) p[i] = f(r[i], p[i], v[i]);
}

// sigma = (rhat, v); alpha = rho / sigma.
__global__ void k_bi_sigma(int64_t n, double *__restrict__ sc, const double *__restrict__ rh,
                           const double *__restrict__ v, double *__restrict__ part,
                           unsigned *__restrict__ ticket, int vec) {
    if (sc[xb::BI_FLAG] != 0.0) return;
    double a[1] = {0.0};
    int64_t done = 0;
    if (vec) {
        for (int64_t i = gtid(); i < n / 2; i += gstride()) {
            const double2 h = ld2(rh, i), w = ld2(v, i);
            a[0] = fma(h.y, w.y, fma(h.x, w.x, a[0]));
        }
        done = n / 2 * 2;
    }
    for (int64_t i = done + gtid(); i < n; i += gstride()) a[0] = fma(rh[i], v[i], a[0]);
    double t[1];
    if (grid_reduce<1>(a, part, ticket, t) && threadIdx.x == 0) {
        if (t[0] == 0.0) sc[xb::BI_FLAG] = 3.0;
        else sc[xb::BI_ALPHA] = sc[xb::BI_RHO] / t[0];
    }
}

// s = r - alpha v, ||s||^2.
__global__ void k_bi_s(int64_t n, double *__restrict__ sc, const double *__restrict__ r,
                       const double *__restrict__ v, double *__restrict__ s,
                       double *__restrict__ part, unsigned *__restrict__ ticket, int vec) {
    if (sc[xb::BI_FLAG] != 0.0) return;
    const double al = sc[xb::BI_ALPHA];
    double a[1] = {0.0};
    int64_t done = 0;
    if (vec) {
        for (int64_t i = gtid(); i < n / 2; i += gstride()) {
            const double2 q = ld2(r, i), w = ld2(v, i);
            double2 si;
            si.x = fma(-al, w.x, q.x);
            si.y = fma(-al, w.y, q.y);
            st2(s, i, si);
            a[0] = fma(si.y, si.y, fma(si.x, si.x, a[0]));
        }
        done = n / 2 * 2;
    }
    for (int64_t i = done + gtid(); i < n; i += gstride()) {
        const double si = fma(-al, v[i], r[i]);
        s[i] = si;
        a[0] = fma(si, si, a[0]);
    }
    double t[1];
    if (grid_reduce<1>(a, part, ticket, t) && threadIdx.x == 0) sc[xb::BI_SNORM2] = t[0];
}

// omega = (t, s) / (t, t).
__global__ void k_bi_omega(int64_t n, double *__restrict__ sc, const double *__restrict__ t,
                           const double *__restrict__ s, double *__restrict__ part,
                           unsigned *__restrict__ ticket, int vec) {
    if (sc[xb::BI_FLAG] != 0.0) return;
    double a[2] = {0.0, 0.0};
    int64_t done = 0;
    if (vec) {
        for (int64_t i = gtid(); i < n / 2; i += gstride()) {
            const double2 u = ld2(t, i), w = ld2(s, i);
            a[0] = fma(u.y, w.y, fma(u.x, w.x, a[0]));
            a[1] = fma(u.y, u.y, fma(u.x, u.x, a[1]));
        }
        done = n / 2 * 2;
    }
    for (int64_t i = done + gtid(); i < n; i += gstride()) {
        a[0] = fma(t[i], s[i], a[0]);
        a[1] = fma(t[i], t[i], a[1]);
    }
    double tt[2];
    if (grid_reduce<2>(a, part, ticket, tt) && threadIdx.x == 0) {
        if (sc[xb::BI_SNORM2] <= sc[xb::BI_TAU2]) return;  // s already converged
        if (tt[1] == 0.0) sc[xb::BI_FLAG] = 4.0;
        else sc[xb::BI_OMEGA] = tt[0] / tt[1];
    }
}

// x += alpha p + omega sx;  r = s - omega t;  ||r||^2, rho_next = (rhat, r).
// sx is s itself, or M^{-1} s (and p is M^{-1} p) under right preconditioning.
// When ||s|| already met the threshold: x += alpha p only, flag = 1 (done).
__global__ void k_bi_xr(int64_t n, double *__restrict__ sc, double *__restrict__ x,
                        const double *__restrict__ p, const double *__restrict__ s,
                        const double *sx, const double *__restrict__ t,
                        double *__restrict__ r, const double *__restrict__ rh,
                        double *__restrict__ part, unsigned *__restrict__ ticket, int vec) {
    if (sc[xb::BI_FLAG] != 0.0) return;
    const double al = sc[xb::BI_ALPHA];
    if (sc[xb::BI_SNORM2] <= sc[xb::BI_TAU2]) {
        for (int64_t i = gtid(); i < n; i += gstride()) x[i] = fma(al, p[i], x[i]);
        double a[1] = {0.0}, tt[1];
        if (grid_reduce<1>(a, part, ticket, tt) && threadIdx.x == 0) {
            sc[xb::BI_RNORM2] = sc[xb::BI_SNORM2];
            sc[xb::BI_FLAG] = 1.0;
        }
        return;
    }
    const double om = sc[xb::BI_OMEGA];
    double a[2] = {0.0, 0.0};
    auto f = [&](double &xi, double pi, double si, double sxi, double ti, double hi) {
        xi = fma(om, sxi, fma(al, pi, xi));
        const double ri = fma(-om, ti, si);
        a[0] = fma(ri, ri, a[0]);
        a[1] = fma(hi, ri, a[1]);
        return ri;
    };
    int64_t done = 0;
    if (vec) {
        for (int64_t i = gtid(); i < n / 2; i += gstride()) {
            double2 xv = ld2(x, i), rv;
            const double2 pv = ld2(p, i), sv = ld2(s, i), tv = ld2(t, i), hv = ld2(rh, i);
            const double2 zv = ld2(sx, i);
            rv.x = f(xv.x, pv.x, sv.x, zv.x, tv.x, hv.x);
            rv.y = f(xv.y, pv.y, sv.y, zv.y, tv.y, hv.y);
            st2(x, i, xv);
            st2(r, i, rv);
        }
        done = n / 2 * 2;
    }
    for (int64_t i = done + gtid(); i < n; i += gstride()) {
        double xi = x[i];
        r[i] = f(xi, p[i], s[i], sx[i], t[i], rh[i]);
        x[i] = xi;
    }
    double tt[2];
    if (grid_reduce<2>(a, part, ticket, tt) && threadIdx.x == 0) {
        sc[xb::BI_RNORM2] = tt[0];
        sc[xb::BI_RHO_OLD] = sc[xb::BI_RHO];
        sc[xb::BI_RHO] = tt[1];
        if (tt[0] <= sc[xb::BI_TAU2]) sc[xb::BI_FLAG] = 1.0;
        else if (tt[1] == 0.0) sc[xb::BI_FLAG] = 2.0;
        else if (om == 0.0) sc[xb::BI_FLAG] = 5.0;
    }
}

// ---- mixed precision helpers ------------------------------------------------------

__global__ void k_cast_scaled(int64_t n, const double *__restrict__ a,
                              const double *__restrict__ scale, float *__restrict__ b) {
    const double s = *scale;
    const double inv = s > 0.0 ? 1.0 / s : 0.0;
    for (int64_t i = gtid(); i < n; i += gstride()) b[i] = (float)(a[i] * inv);
}

__global__ void k_add_scaled(int64_t n, double *__restrict__ x, const double *__restrict__ scale,
                             const float *__restrict__ d) {
    const double s = *scale;
    for (int64_t i = gtid(); i < n; i += gstride()) x[i] = fma(s, (double)d[i], x[i]);
}

}  // namespace

namespace xb {

GmDev gm_layout(double *base, int M) {
    GmDev st;
    st.M = M;
    double *q = base;
    st.H = q; q += (size_t)(M + 1) * M;
    st.cs = q; q += M;
    st.sn = q; q += M;
    st.g = q; q += M + 1;
    st.sc = q; q += M + 1;
    st.y = q; q += M;
    st.coef = q; q += M + 1;
    st.misc = q; q += GM_NMISC;
    st.scf = reinterpret_cast<float *>(q);
    return st;
}

int vdot(xb_plan *p, int64_t n, const double *x, const double *y, double *out, cudaStream_t s) {
    const int g = rgrid(k_dot, n);
    const int vec = (((uintptr_t)x | (uintptr_t)y) % 16) == 0 ? 1 : 0;
    k_dot<<<g, kVB, 0, s>>>(n, x, y, p->d_part, p->d_ticket, out, 0, vec);
    XB_LAUNCHED("k_dot");
    return XB_OK;
}
int vnrm2(xb_plan *p, int64_t n, const double *x, double *out, cudaStream_t s) {
    const int g = rgrid(k_dot, n);
    const int vec = ((uintptr_t)x % 16) == 0 ? 1 : 0;
    k_dot<<<g, kVB, 0, s>>>(n, x, x, p->d_part, p->d_ticket, out, 1, vec);
    XB_LAUNCHED("k_nrm2");
    return XB_OK;
}
int vaxpy(int64_t n, double a, const double *x, double *y, cudaStream_t s) {
    if (n <= 0) return XB_OK;
    k_axpy<<<rgrid(k_axpy, n), kVB, 0, s>>>(n, a, x, y);
    XB_LAUNCHED("k_axpy");
    return XB_OK;
}
int vcopy(int64_t n, const double *x, double *y, cudaStream_t s) {
    if (n <= 0) return XB_OK;
    k_copy<<<rgrid(k_copy, n), kVB, 0, s>>>(n, x, y);
    XB_LAUNCHED("k_copy");
    return XB_OK;
}
int vscale(int64_t n, double a, double *x, cudaStream_t s) {
    if (n <= 0) return XB_OK;
    k_scale<<<rgrid(k_scale, n), kVB, 0, s>>>(n, a, x);
    XB_LAUNCHED("k_scale");
    return XB_OK;
}
int vfill(int64_t n, double a, double *x, cudaStream_t s) {
    if (n <= 0) return XB_OK;
    k_fill<<<rgrid(k_fill, n), kVB, 0, s>>>(n, a, x);
    XB_LAUNCHED("k_fill");
    return XB_OK;
}

int gm_cycle_init(xb_plan *p, GmDev st, int64_t n, const double *r0, double tau, cudaStream_t s) {
    k_gm_init<double><<<rgrid(k_gm_init<double>, n), kVB, 0, s>>>(n, r0, st, tau, p->d_part,
                                                                 p->d_ticket);
    XB_LAUNCHED("k_gm_init");
    return XB_OK;
}
int gm_cycle_init_f32(xb_plan *p, GmDev st, int64_t n, const float *r0, double tau,
                      cudaStream_t s) {
    k_gm_init<float><<<rgrid(k_gm_init<float>, n), kVB, 0, s>>>(n, r0, st, tau, p->d_part,
                                                               p->d_ticket);
    XB_LAUNCHED("k_gm_init_f32");
    return XB_OK;
}

// MGS traversal mode (flags of k_mgs: bit 0 alternate direction, bit 1
// evict-first loads of v_{i-1}); XB_MGS_MODE=0..3 overrides the default.
int mgs_mode(size_t elem) {
    static const int env = [] {
        const char *e = std::getenv("XB_MGS_MODE");
        return e ? std::atoi(e) & 3 : -1;
    }();
    (void)elem;
    return env >= 0 ? env : 3;
}

template <typename VB>
int gm_mgs_step(xb_plan *p, GmDev st, int64_t n, const VB *V, int64_t ld, VB *w, int j,
                cudaStream_t s) {
    const int g = rgrid(k_mgs<1, VB>, n);
    const int vec = (((uintptr_t)V % 16) == 0 && ((uintptr_t)w % 16) == 0 &&
                     ((ld * sizeof(VB)) % 16) == 0) ? 1 : 0;
    // With alternation on, pass i walks backwards when i is even (pass 0 then
    // starts on the tail of w that the SpMV wrote last).
    const int mode = mgs_mode(sizeof(VB));
    auto fl = [mode](int i) { return ((mode & 1) && !(i & 1) ? 1 : 0) | (mode & 2); };
    k_mgs<0, VB><<<g, kVB, 0, s>>>(n, w, nullptr, V, st, j, 0, p->d_part, p->d_ticket, vec, fl(0));
    for (int i = 1; i <= j; i++)
        k_mgs<1, VB><<<g, kVB, 0, s>>>(n, w, V + (size_t)(i - 1) * ld, V + (size_t)i * ld, st, j, i,
                                       p->d_part, p->d_ticket, vec, fl(i));
    k_mgs<2, VB><<<g, kVB, 0, s>>>(n, w, V + (size_t)j * ld, nullptr, st, j, j + 1, p->d_part,
                                   p->d_ticket, vec, fl(j + 1));
    XB_LAUNCHED("k_mgs");
    return XB_OK;
}
template int gm_mgs_step<double>(xb_plan *, GmDev, int64_t, const double *, int64_t, double *,
                                  int, cudaStream_t);
template int gm_mgs_step<float>(xb_plan *, GmDev, int64_t, const float *, int64_t, float *, int,
                                 cudaStream_t);

double ortho_passes(int ortho, int j) {
    const int nb = (j + 1 + 3) / 4;
    switch (ortho) {
        case XB_ORTHO_CGS: return 2.0 * j + 5.0;
        case XB_ORTHO_DGKS: return 3.0 * j + 8.0;
        case XB_ORTHO_BCGS: return 2.0 * (j + 1) + 2.0 * nb + 1.0;
        default: return 4.0 * j + 5.0;
    }
}

int ortho_choice(int ortho, double tol, bool faulted) {
    if (ortho != XB_ORTHO_AUTO) return ortho;
    if (faulted) return XB_ORTHO_DGKS;
    return tol <= 1e-10 ? XB_ORTHO_MGS : XB_ORTHO_BCGS;
}

template <typename VB>
int gm_ortho_step(xb_plan *p, GmDev st, int64_t n, const VB *V, int64_t ld, VB *w, int j,
                  int ortho, cudaStream_t s) {
    if (ortho == XB_ORTHO_MGS) return gm_mgs_step<VB>(p, st, n, V, ld, w, j, s);
    constexpr int KD = 8;
    // grids of exactly the resident CTAs (measured 12 % faster than 8 CTAs per SM in waves)
    const int g4 = rgrid(k_bgs<VB, 4, 4, 4>, n);
    const int g8 = rgrid(k_bgs<VB, KD, 0, 4>, n);
    const int vec = (((uintptr_t)V % 16) == 0 && ((uintptr_t)w % 16) == 0 &&
                     ((ld * sizeof(VB)) % 16) == 0) ? 1 : 0;
    const bool zig = mgs_mode(sizeof(VB)) & 1;
    int pass = 0;
    // the first pass walks backwards (it starts on the tail of w the SpMV wrote last)
    auto L = [&](int u0, int u1, int d0, int nd, int flags) {
        if (zig && !(pass & 1)) flags |= kBgsRev;
        pass++;
        // 4 resident CTAs per SM (64 registers) measured faster than 2 with no spills
        if (nd <= 4 && u1 - u0 <= 4)  // BCGS passes, and short CGS/DGKS sweeps
            k_bgs<VB, 4, 4, 4><<<g4, kVB, 0, s>>>(n, w, V, ld, u0, u1, d0, nd, flags, st, j,
                                                  p->d_part, p->d_ticket, vec);
        else
            k_bgs<VB, KD, 0, 4><<<g8, kVB, 0, s>>>(n, w, V, ld, u0, u1, d0, nd, flags, st, j,
                                                   p->d_part, p->d_ticket, vec);
    };
    const int k = j + 1;  // basis vectors v_0..v_j
    if (ortho == XB_ORTHO_BCGS) {
        const int nb = (k + 3) / 4;
        L(0, 0, 0, std::min(4, k), 0);
        for (int b = 1; b < nb; b++) L(4 * (b - 1), 4 * b, 4 * b, std::min(4, k - 4 * b), 0);
        L(4 * (nb - 1), k, 0, 0, kBgsFin);
    } else {
        for (int c = 0; c < k; c += KD) L(0, 0, c, std::min(KD, k - c), 0);
        if (ortho == XB_ORTHO_DGKS)  // second CGS: update by the first, dots added to H
            for (int c = 0; c < k; c += KD) L(0, c == 0 ? k : 0, c, std::min(KD, k - c), kBgsAcc);
        L(0, k, 0, 0, kBgsFin);
    }
    XB_LAUNCHED("k_bgs");
    return XB_OK;
}
template int gm_ortho_step<double>(xb_plan *, GmDev, int64_t, const double *, int64_t, double *,
                                   int, int, cudaStream_t);
template int gm_ortho_step<float>(xb_plan *, GmDev, int64_t, const float *, int64_t, float *,
                                  int, int, cudaStream_t);

template <typename VB, typename VX>
int gm_update(xb_plan *p, GmDev st, int64_t n, const VB *V, int64_t ld, int k, VX *x,
              cudaStream_t s) {
    (void)p;
    (void)k;
    k_gm_solve<<<1, 32, 0, s>>>(st);
    XB_LAUNCHED("k_gm_solve");
    const int vec = (((uintptr_t)V % 16) == 0 && ((uintptr_t)x % 16) == 0 &&
                     ((ld * sizeof(VB)) % 16) == 0) ? 1 : 0;
    k_gm_xupd<VB, VX><<<rgrid(k_gm_xupd<VB, VX>, n), kVB, 0, s>>>(n, V, ld, st, x, vec);
    XB_LAUNCHED("k_gm_xupd");
    return XB_OK;
}
template int gm_update<double, double>(xb_plan *, GmDev, int64_t, const double *, int64_t, int,
                                       double *, cudaStream_t);
template int gm_update<float, float>(xb_plan *, GmDev, int64_t, const float *, int64_t, int,
                                     float *, cudaStream_t);

static int al16(const void *a) { return ((uintptr_t)a % 16) == 0; }

int bi_init(xb_plan *p, double *scal, int64_t n, const double *r, double tau2, cudaStream_t s) {
    k_bi_init<<<rgrid(k_bi_init, n), kVB, 0, s>>>(n, r, scal, tau2, p->d_part, p->d_ticket,
                                                  al16(r));
    XB_LAUNCHED("k_bi_init");
    return XB_OK;
}
int bi_p_update(double *scal, int64_t n, const double *r, double *pv, const double *v,
                cudaStream_t s) {
    k_bi_p<<<rgrid(k_bi_p, n), kVB, 0, s>>>(n, scal, r, pv, v, al16(r) & al16(pv) & al16(v));
    XB_LAUNCHED("k_bi_p");
    return XB_OK;
}
int bi_sigma(xb_plan *p, double *scal, int64_t n, const double *rh, const double *v,
             cudaStream_t s) {
    k_bi_sigma<<<rgrid(k_bi_sigma, n), kVB, 0, s>>>(n, scal, rh, v, p->d_part, p->d_ticket,
                                                   al16(rh) & al16(v));
    XB_LAUNCHED("k_bi_sigma");
    return XB_OK;
}
int bi_s_update(xb_plan *p, double *scal, int64_t n, const double *r, const double *v, double *sv,
                cudaStream_t s) {
    k_bi_s<<<rgrid(k_bi_s, n), kVB, 0, s>>>(n, scal, r, v, sv, p->d_part, p->d_ticket,
                                               al16(r) & al16(v) & al16(sv));
    XB_LAUNCHED("k_bi_s");
    return XB_OK;
}
int bi_omega(xb_plan *p, double *scal, int64_t n, const double *t, const double *sv,
             cudaStream_t s) {
    k_bi_omega<<<rgrid(k_bi_omega, n), kVB, 0, s>>>(n, scal, t, sv, p->d_part, p->d_ticket,
                                                   al16(t) & al16(sv));
    XB_LAUNCHED("k_bi_omega");
    return XB_OK;
}
int bi_xr_update(xb_plan *p, double *scal, int64_t n, double *x, const double *pv,
                 const double *sv, const double *sx, const double *t, double *r, const double *rh,
                 cudaStream_t s) {
    const int vec = al16(x) & al16(pv) & al16(sv) & al16(sx) & al16(t) & al16(r) & al16(rh);
    k_bi_xr<<<rgrid(k_bi_xr, n), kVB, 0, s>>>(n, scal, x, pv, sv, sx, t, r, rh, p->d_part,
                                                p->d_ticket, vec);
    XB_LAUNCHED("k_bi_xr");
    return XB_OK;
}

// r = b - A x
int residual(xb_plan *p, const double *b, const double *x, double *r, cudaStream_t s) {
    XB_TRY(vcopy(p->n, b, r, s));
    return spmv_launch(p, XB_VAR_AUTO, 0, 0, -1.0, x, 1.0, r, s);
}

int cast_f64_to_f32_scaled(int64_t n, const double *a, const double *scale_dev, float *b,
                           cudaStream_t s) {
    if (n <= 0) return XB_OK;
    k_cast_scaled<<<rgrid(k_cast_scaled, n), kVB, 0, s>>>(n, a, scale_dev, b);
    XB_LAUNCHED("k_cast_scaled");
    return XB_OK;
}

int add_scaled_f32(int64_t n, double *x, const double *scale_dev, const float *d, cudaStream_t s) {
    if (n <= 0) return XB_OK;
    k_add_scaled<<<rgrid(k_add_scaled, n), kVB, 0, s>>>(n, x, scale_dev, d);
    XB_LAUNCHED("k_add_scaled");
    return XB_OK;
}

}  // namespace xb
