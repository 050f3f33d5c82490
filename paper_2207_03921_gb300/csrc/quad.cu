// Pair quadrature (Sec. 2.3): Alg. 1 per ordered pair (E_k, E_l).
//
// k_trunc: the truncation quadrature (eq. discrete-inner) for every pair that does not
//   take the singular rule. For each outer point x_p of E_k the inner element E_l is cut
//   by the ball approximation around x_p (canonical FP64 geometry, see
//   nlfem_internal.cuh), the cut polygon is fan-triangulated and the inner rule is put
//   on every sub-triangle; basis values are interpolated from the sub-triangle vertices'
//   barycentric coordinates. One thread per pair. The integrand is accumulated in R
//   (FP32 in the bulk path, FP64 in the plain path) from vectors relative to x_p, so
//   the FP32 path never subtracts absolute coordinates.
// k_duffy: the singular rule (Tab. 1 "club") for intersecting pairs: regularising maps
//   of S x S to (0,1)^4 and a tensor Gauss rule, in FP64. One warp per pair.
//   Directions along which the integrand is constant are summed in closed form (the
//   same tensor sum, reordered). Of two exchanged orders (k, l), (l, k) that the rule maps
//   onto the same points only one is evaluated; k_duffy_mirror copies its block.
// k_load: F_i = sum over Omega elements of sum_p a_p f(x_p) phi_i(x_p), thread per node.
#include <algorithm>

#include <cstring>

#include "nlfem_internal.cuh"

namespace nlfem {

static inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

__device__ __constant__ int q_E1[6][6] = {
    {0, 1, 2, 3, 4, 5}, {1, 6, 7, 8, 9, 10}, {2, 7, 11, 12, 13, 14},
    {3, 8, 12, 15, 16, 17}, {4, 9, 13, 16, 18, 19}, {5, 10, 14, 17, 19, 20}};

struct QuadArgs {
    const int* pk;
    const int* pl;
    const int8_t* pcls;
    const int8_t* whole;   // census only: 1 if the pair is in the whole-pair list, 2 in the cut list
    int64_t npairs;        // number of pairs to process (of ids, if given)
    const int* ids;        // optional list of pair ids
    int compact;           // records at the list position instead of the pair id
    const double2* X;
    const int4* T;
    const double* det;
    Params prm;
};

template <typename R>
__device__ __forceinline__ R rsqrt_r(R x);
template <>
__device__ __forceinline__ float rsqrt_r<float>(float x) { return rsqrtf(x); }
template <>
__device__ __forceinline__ double rsqrt_r<double>(double x) { return rsqrt(x); }

// scalar kernel value (constant / fractional); d2 = |z|^2
template <typename R, int KER>
__device__ __forceinline__ R gamma_s(R d2, const Params& P) {
    if (KER == NLFEM_KERNEL_CONSTANT) return (R)P.c;
    if (KER == NLFEM_KERNEL_TABULATED) {
        if constexpr (sizeof(R) == 4) return (R)P.c * table_g<float>(P.tab32, P.ntab, (float)P.tinv, (float)d2);
        else return (R)P.c * table_g<double>(P.tab64, P.ntab, P.tinv, (double)d2);
    }
    if (P.s == 0.5) {
        R r = rsqrt_r<R>(d2);
        return (R)P.c * r * r * r;
    }
    if (sizeof(R) == 4) return (R)P.c * exp2f(log2f((float)d2) * (float)(-1.0 - P.s));
    return (R)P.c * (R)pow((double)d2, -1.0 - P.s);
}

// union of the vertex lists: E_k's vertices, then E_l's vertices not in E_k
__device__ __forceinline__ int union_pos(int4 tk, int4 tl, int posl[3], int u[6]) {
    u[0] = tk.x; u[1] = tk.y; u[2] = tk.z;
    int U = 3;
    int lv[3] = {tl.x, tl.y, tl.z};
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        int f = -1;
        if (lv[b] == tk.x) f = 0;
        if (lv[b] == tk.y) f = 1;
        if (lv[b] == tk.z) f = 2;
        if (f >= 0) posl[b] = f;
        else { u[U] = lv[b]; posl[b] = U; ++U; }
    }
    return U;
}

// Accumulators of one pair: kk (sym 3x3, 6), kl (3x3, 9), ll (sym, 6); NC components
// (1 scalar, 3 = xx, xy, yy for peridynamics).
template <typename R, int NC>
struct Acc {
    R kk[6][NC], kl[9][NC], ll[6][NC];
};

__device__ __forceinline__ int sym3(int a, int b) {  // index of (a, b) in a packed symmetric 3x3
    int lo = a < b ? a : b, hi = a < b ? b : a;
    return lo == 0 ? hi : (lo == 1 ? 2 + hi : 5);
}

// WHOLE: a list of pairs whose inner element lies in the ball of every point of the outer
// element (decided with a margin far above FP64 rounding when the lists are built), for which
// the canonical clip returns the whole element at every outer point: the clip is not called.
template <typename R, int KER, int NQI, bool WHOLE = false>
__global__ void __launch_bounds__(128) k_trunc(QuadArgs A, R* __restrict__ contrib) {
    constexpr int NC = (KER == NLFEM_KERNEL_PERIDYNAMIC) ? 3 : 1;
    constexpr int NS = (KER == NLFEM_KERNEL_PERIDYNAMIC) ? NLFEM_REC2 : NLFEM_REC1;  // record stride
    const Params& P = A.prm;
    for (int64_t pi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; pi < A.npairs;
         pi += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = A.ids ? (int64_t)A.ids[pi] : pi;
        const int cls = A.pcls[p];
        if (cls > 0 && P.singular) continue;  // k_duffy writes this pair
        const int k = A.pk[p], l = A.pl[p];
        const int4 tk = A.T[k], tl = A.T[l];
        const double2 Vk[3] = {A.X[tk.x], A.X[tk.y], A.X[tk.z]};
        const double2 Vl[3] = {A.X[tl.x], A.X[tl.y], A.X[tl.z]};
        const double dk = A.det[k], dl = A.det[l];
        const bool nzd = cls > 0 && P.nozerodiv;
        Acc<R, NC> acc;
#pragma unroll
        for (int i = 0; i < 6; ++i)
#pragma unroll
            for (int c = 0; c < NC; ++c) acc.kk[i][c] = acc.ll[i][c] = (R)0;
#pragma unroll
        for (int i = 0; i < 9; ++i)
#pragma unroll
            for (int c = 0; c < NC; ++c) acc.kl[i][c] = (R)0;

        for (int q0 = 0; q0 < P.ro.n; ++q0) {
            const double2 xp = nl_map(Vk, P.ro.l[q0][0], P.ro.l[q0][1], P.ro.l[q0][2]);
            CPt poly[NLFEM_MAXPOLY];
            bool full = true;
            const int np = WHOLE ? 3 : nl_clip_ball(P.ball, Vl, xp, P.delta, P.delta2, poly, full);
            if (np < 3) continue;
            // inner sums for this x_p: g = sum w, h_j = sum w Q_j, m_ij = sum w Q_i Q_j
            R g[NC], h[3][NC], mm[6][NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                g[c] = (R)0;
#pragma unroll
                for (int j = 0; j < 3; ++j) h[j][c] = (R)0;
#pragma unroll
                for (int j = 0; j < 6; ++j) mm[j][c] = (R)0;
            }
            const int ntri = full ? 1 : np - 2;
            for (int t = 0; t < ntri; ++t) {
                double2 tv[3];
                R bq[3][3];  // barycentric coordinates (w.r.t. E_l) of the sub-triangle vertices
                double dT;
                if (full) {
                    tv[0] = Vl[0]; tv[1] = Vl[1]; tv[2] = Vl[2];
#pragma unroll
                    for (int a = 0; a < 3; ++a)
#pragma unroll
                        for (int b = 0; b < 3; ++b) bq[a][b] = (R)(a == b ? 1.0 : 0.0);
                    dT = dl;
                } else {
                    const CPt* c3[3] = {&poly[0], &poly[t + 1], &poly[t + 2]};
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        tv[a] = make_double2(c3[a]->x, c3[a]->y);
                        bq[a][1] = (R)c3[a]->b1;
                        bq[a][2] = (R)c3[a]->b2;
                        bq[a][0] = (R)(1.0 - c3[a]->b1 - c3[a]->b2);
                    }
                    dT = fabs((tv[1].x - tv[0].x) * (tv[2].y - tv[0].y) -
                              (tv[1].y - tv[0].y) * (tv[2].x - tv[0].x));
                }
                // sub-triangle vertices relative to x_p (FP64 difference, rounded once)
                R rx[3], ry[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    rx[a] = (R)(tv[a].x - xp.x);
                    ry[a] = (R)(tv[a].y - xp.y);
                }
#pragma unroll
                for (int q = 0; q < NQI; ++q) {
                    const R l0 = (R)P.ri.l[q][0], l1 = (R)P.ri.l[q][1], l2 = (R)P.ri.l[q][2];
                    if (nzd) {
                        // Tab. 1 diamond: drop x_p = y_q, decided on the canonical FP64 point
                        double2 yq = nl_map(tv, P.ri.l[q][0], P.ri.l[q][1], P.ri.l[q][2]);
                        if (yq.x == xp.x && yq.y == xp.y) continue;
                    }
                    const R zx = l0 * rx[0] + l1 * rx[1] + l2 * rx[2];
                    const R zy = l0 * ry[0] + l1 * ry[1] + l2 * ry[2];
                    const R d2 = zx * zx + zy * zy;
                    const R wq = (R)(P.ri.w[q] * dT);
                    R Q[3];
#pragma unroll
                    for (int j = 0; j < 3; ++j) Q[j] = l0 * bq[0][j] + l1 * bq[1][j] + l2 * bq[2][j];
                    R wc[NC];
                    if (KER == NLFEM_KERNEL_PERIDYNAMIC) {
                        const R r = rsqrt_r<R>(d2);
                        const R s = wq * (R)P.c * r * r * r;
                        wc[0] = s * zx * zx;
                        if (NC > 1) {
                            wc[1 % NC] = s * zx * zy;
                            wc[2 % NC] = s * zy * zy;
                        }
                    } else {
                        wc[0] = wq * gamma_s<R, KER>(d2, P);
                    }
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        g[c] += wc[c];
#pragma unroll
                        for (int j = 0; j < 3; ++j) h[j][c] += wc[c] * Q[j];
                        mm[0][c] += wc[c] * Q[0] * Q[0];
                        mm[1][c] += wc[c] * Q[0] * Q[1];
                        mm[2][c] += wc[c] * Q[0] * Q[2];
                        mm[3][c] += wc[c] * Q[1] * Q[1];
                        mm[4][c] += wc[c] * Q[1] * Q[2];
                        mm[5][c] += wc[c] * Q[2] * Q[2];
                    }
                }
            }
            const R ap = (R)(P.ro.w[q0] * dk);
            const R Pa[3] = {(R)P.ro.l[q0][0], (R)P.ro.l[q0][1], (R)P.ro.l[q0][2]};
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const R ag = ap * g[c];
                acc.kk[0][c] += ag * Pa[0] * Pa[0];
                acc.kk[1][c] += ag * Pa[0] * Pa[1];
                acc.kk[2][c] += ag * Pa[0] * Pa[2];
                acc.kk[3][c] += ag * Pa[1] * Pa[1];
                acc.kk[4][c] += ag * Pa[1] * Pa[2];
                acc.kk[5][c] += ag * Pa[2] * Pa[2];
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int b = 0; b < 3; ++b) acc.kl[a * 3 + b][c] -= ap * Pa[a] * h[b][c];
#pragma unroll
                for (int j = 0; j < 6; ++j) acc.ll[j][c] += ap * mm[j][c];
            }
        }
        // fold the four blocks into the union block and write its upper triangle (times the
        // pair's factor of a label-dependent kernel)
        int posl[3], u[6];
        union_pos(tk, tl, posl, u);
        R* out = contrib + (A.compact ? pi : p) * NS;
        const R fm = (R)pair_factor64(P, k, l);
        R blk[6][6][NC];
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
            for (int b = 0; b < 6; ++b)
#pragma unroll
                for (int c = 0; c < NC; ++c) blk[a][b][c] = (R)0;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b)
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    blk[a][b][c] += acc.kk[sym3(a, b)][c];
                    blk[a][posl[b]][c] += acc.kl[a * 3 + b][c];
                    blk[posl[b]][a][c] += acc.kl[a * 3 + b][c];
                    blk[posl[a]][posl[b]][c] += acc.ll[sym3(a, b)][c];
                }
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
            for (int b = a; b < 6; ++b) {
                if (NC == 1) {
                    out[q_E1[a][b]] = fm * blk[a][b][0];
                } else {
                    // components (c1, c2) of Gamma: xx, xy, yx, yy
                    R* o = out + q_E1[a][b] * 4;
                    o[0] = fm * blk[a][b][0];
                    o[1] = fm * blk[a][b][1 % NC];
                    o[2] = fm * blk[a][b][1 % NC];
                    o[3] = fm * blk[a][b][2 % NC];
                }
            }
    }
}

// ------------------------------------------------------------------------------------------
// singular rule for intersecting pairs (FP64), warp per pair
// ------------------------------------------------------------------------------------------
struct DuffyArgs {
    const int* ids;
    int64_t n;
    int compact;  // records at the list position instead of the pair id
    const int* pk;
    const int* pl;
    const double2* X;
    const int4* T;
    const double* det;
    Params prm;
    const int4* Tp;  // vertex positions (original vertex ids of a discontinuous mesh)
    int dg;          // discontinuous mesh: touching pairs (k != l) take k_duffy_split
    const int64_t* pair_ptr;  // [K + 1] rows of the pair list (each sorted by its second element)
};

// Record index of the pair (l, k) whose singular-rule block the pair (k, l) takes, or -1 when
// (k, l) evaluates its own. With x and y exchanged, the rule's points for (l, k) are those of
// (k, l) (the two regions of a common vertex trade places, as do the four of a common edge) with
// the same weights and D -> -D, so D D^T is the same matrix over the union's nodes; that holds
// for a common vertex always, and for a common edge when both orders run along the edge in the
// same direction (the first shared vertex of each element's list is the same node: sl0 < sl1
// below). Reversing the edge changes the result by the rule's error, so such pairs evaluate
// both orders. Of each mirrored couple the order with k < l evaluates, the other copies.
__device__ __forceinline__ int64_t duffy_mirror(const DuffyArgs& A, int k, int l, int4 tk4, int4 tl4) {
    if (A.dg || k <= l) return -1;
    const int tk[3] = {tk4.x, tk4.y, tk4.z}, tl[3] = {tl4.x, tl4.y, tl4.z};
    int shared = 0, sl0 = -1, sl1 = -1;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            if (tk[a] == tl[b]) {
                if (shared == 0) sl0 = b; else sl1 = b;
                ++shared;
            }
    if (!(shared == 1 || (shared == 2 && sl0 < sl1))) return -1;
    // the pair id of (l, k) in row l
    const int64_t end = A.pair_ptr[l + 1];
    int64_t lo = A.pair_ptr[l], hi = end;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (A.pl[mid] < k) lo = mid + 1; else hi = mid;
    }
    if (lo == end || A.pl[lo] != k) return -1;
    if (!A.compact) return lo;
    // its position in the close list (pair ids in increasing order)
    int64_t a = 0, b = A.n;
    while (a < b) {
        const int64_t mid = (a + b) >> 1;
        if (A.ids[mid] < lo) a = mid + 1; else b = mid;
    }
    return a < A.n && A.ids[a] == lo ? a : -1;
}

// c |z|^(-2-2s) from d2 = |z|^2 by reciprocal square roots for s in {1/4, 1/2, 3/4}, with
// r = d2^(-1/2): r^3 (s = 1/2), r^3 rsqrt(r) (s = 1/4), r^4 rsqrt(r) (s = 3/4) (rsqrt is within
// 1 ulp, so a few ulps in all; no FP64 division or square root, which cost several times more
// on the FP64 pipe); exp2 / log2 otherwise (a relative error of a few 1e-15, far below the rule's)
__device__ __forceinline__ double gamma_d(double d2, const Params& P) {
    if (P.kernel == NLFEM_KERNEL_CONSTANT) return P.c;
    const double r = rsqrt(d2);
    if (P.s == 0.5) return P.c * (r * r * r);
    if (P.s == 0.25) return P.c * (r * r * r * rsqrt(r));
    if (P.s == 0.75) return P.c * (r * r * r * r * rsqrt(r));
    return P.c * exp2((-1.0 - P.s) * log2(d2));
}

// the same in FP32 for the FP32-bulk path (relative error of a few 1e-7): rsqrt powers for
// s in {1/4, 1/2, 3/4}, exp2 / log2 otherwise
__device__ __forceinline__ float gamma_f(float d2, const Params& P, float c) {
    if (P.kernel == NLFEM_KERNEL_CONSTANT) return c;
    const float r = rsqrtf(d2);  // |z|^-1
    if (P.s == 0.5) return c * r * r * r;
    if (P.s == 0.25) return c * r * r * sqrtf(r);
    if (P.s == 0.75) return c * r * r * r * sqrtf(r);
    return c * exp2f(log2f(d2) * (float)(-1.0 - P.s));
}

template <typename R>
__device__ __forceinline__ R gamma_r(R d2, const Params& P, R c);
template <>
__device__ __forceinline__ double gamma_r<double>(double d2, const Params& P, double) { return gamma_d(d2, P); }
template <>
__device__ __forceinline__ float gamma_r<float>(float d2, const Params& P, float c) { return gamma_f(d2, P, c); }

// add w * D D^T over the first M basis differences into the packed upper block (row-major)
template <typename R, int M>
__device__ __forceinline__ void duffy_add(R* acc, const R* D, R w) {
    int e = 0;
#pragma unroll
    for (int a = 0; a < M; ++a) {
        const R wa = w * D[a];
#pragma unroll
        for (int b = a; b < M; ++b) acc[e++] += wa * D[b];
    }
}

// R = double: the FP64 path; R = float: the FP32-bulk path (points and sums in FP32). The
// 1D Gauss rule sits in shared memory: lanes read it at different indices.
template <typename R>
__global__ void __launch_bounds__(128) k_duffy(DuffyArgs A, double* __restrict__ contrib64,
                                               float* __restrict__ contrib32) {
    // the 1D rule, 1 - x, and for the common vertex the weight products w_i1 w_i3 (with the
    // xi factor) and w_i2 x_i2 tabulated once per block
    __shared__ R s_x[32], s_w[32], s_1m[32], s_wx[32], s_w13[32 * 32];
    const Params& P = A.prm;
    const int nr = P.dr.n;
    for (int i = threadIdx.x; i < 32; i += blockDim.x) {
        s_x[i] = (R)(i < nr ? P.dr.x[i] : 0.0);
        s_w[i] = (R)(i < nr ? P.dr.w[i] : 0.0);
        s_1m[i] = (R)(i < nr ? 1.0 - P.dr.x[i] : 0.0);
        s_wx[i] = (R)(i < nr ? P.dr.w[i] * P.dr.x[i] : 0.0);
    }
    for (int i = threadIdx.x; i < nr * nr; i += blockDim.x)
        s_w13[i] = (R)(P.dr.w[i / nr] * P.dr.w[i % nr] * P.dr.sxi[2]);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t wi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (wi >= A.n) return;
    const int p = A.ids[wi];
    const int k = A.pk[p], l = A.pl[p];
    if (A.dg && k != l) return;  // the warp's pair is split (k_duffy_split)
    const int4 tk4 = A.T[k], tl4 = A.T[l];
    if (duffy_mirror(A, k, l, tk4, tl4) >= 0) return;  // k_duffy_mirror copies (l, k)'s block
    const int tk[3] = {tk4.x, tk4.y, tk4.z}, tl[3] = {tl4.x, tl4.y, tl4.z};
    int shared = 0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) shared += tk[a] == tl[b];
    int ak[3], bl[3] = {0, 1, 2};
    if (shared == 3) {
        ak[0] = 0; ak[1] = 1; ak[2] = 2;
    } else if (shared == 2) {
        int s0 = -1, s1 = -1, sl0 = -1, sl1 = -1;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                if (tk[a] == tl[b]) {
                    if (s0 < 0) { s0 = a; sl0 = b; } else { s1 = a; sl1 = b; }
                }
        ak[0] = s0; ak[1] = s1; ak[2] = 3 - s0 - s1;
        bl[0] = sl0; bl[1] = sl1; bl[2] = 3 - sl0 - sl1;
    } else {
        int s0 = 0, sl0 = 0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                if (tk[a] == tl[b]) { s0 = a; sl0 = b; }
        ak[0] = s0; ak[1] = (s0 + 1) % 3; ak[2] = (s0 + 2) % 3;
        bl[0] = sl0; bl[1] = (sl0 + 1) % 3; bl[2] = (sl0 + 2) % 3;
    }
    double2 Av[3], Bv[3];
    for (int a = 0; a < 3; ++a) {
        Av[a] = A.X[tk[ak[a]]];
        Bv[a] = A.X[tl[bl[a]]];
    }
    const int U = shared == 3 ? 3 : (shared == 2 ? 4 : 5);
    int uorder[5];
    for (int a = 0; a < 3; ++a) uorder[a] = tk[ak[a]];
    if (shared == 2) uorder[3] = tl[bl[2]];
    if (shared == 1) { uorder[3] = tl[bl[1]]; uorder[4] = tl[bl[2]]; }
    int posl[3], u[6];
    union_pos(tk4, tl4, posl, u);
    int upos[5];
    for (int a = 0; a < U; ++a) {
        upos[a] = 0;
        for (int v = 0; v < U; ++v)
            if (u[v] == uorder[a]) upos[a] = v;
    }
    const R scale = (R)(A.det[k] * A.det[l]);
    const R cR = (R)P.c;
    // element edge vectors: FP64 differences, rounded once to R
    const R e10x = (R)(Av[1].x - Av[0].x), e10y = (R)(Av[1].y - Av[0].y);
    const R e21x = (R)(Av[2].x - Av[1].x), e21y = (R)(Av[2].y - Av[1].y);
    const int n = P.dr.n;
    // The block is accumulated over the union's vertices in the order of the maps (uorder),
    // for the first U - 1 of them only: the basis differences of the union sum to zero (both
    // elements' basis functions sum to one), so every row of D D^T sums to zero and the last
    // row and column follow from the others once the points are summed.
    R acc[10];
    for (int e = 0; e < 10; ++e) acc[e] = (R)0;
    R D[4];
    // z, the basis differences D and the Jacobian are powers of xi times functions of the
    // other coordinates, and gamma is homogeneous (gamma(xi w) = xi^alpha gamma(w)), so the xi
    // sum of the tensor rule factors out: P.dr.sxi[case] = sum_i w_i xi_i^(e + alpha) (1 - xi_i)^m
    // (computed once per parameter set). The loops below run over the remaining coordinates
    // with z / xi and D / xi: the same tensor sum, reordered.
    if (shared == 3) {
        // identical: the integrand depends on (xi, e1) only; e2, e3 sum to sum_wx * sum_w
        const R fac = (R)(P.dr.sum_wx * P.dr.sum_w * P.dr.sxi[0]);
        const int npts = 6 * n;
        for (int t = lane; t < npts; t += 32) {
            const int r = t / n, i1 = t % n;
            const R e1 = s_x[i1];
            const R w = s_w[i1] * fac;
            // (P_r, Q_r): the six triangles tiling the hexagon S - S
            const R PQ[6][4] = {{0, 1, 1, 1}, {1, 0, 1, 1}, {1, 0, 0, -1},
                                {0, 1, -1, 0}, {-1, 0, -1, -1}, {0, -1, -1, -1}};
            const R h1 = ((R)1 - e1) * PQ[r][0] + e1 * PQ[r][2];
            const R h2 = ((R)1 - e1) * PQ[r][1] + e1 * PQ[r][3];
            const R zx = h1 * e10x + h2 * e21x, zy = h1 * e10y + h2 * e21y;
            D[0] = h1;
            D[1] = h2 - h1;  // the third difference is -h2
            const R g = gamma_r<R>(zx * zx + zy * zy, P, cR);
            duffy_add<R, 2>(acc, D, w * g);
        }
    } else if (shared == 2) {
        // common edge: constant along e3
        const R fx = (R)(Bv[2].x - Av[1].x), fy = (R)(Bv[2].y - Av[1].y);
        const R fac = (R)(P.dr.sum_w * P.dr.sxi[1]);
        const int npts = 4 * n * n;
        for (int t = lane; t < npts; t += 32) {
            const int r = t / (n * n), i1 = (t / n) % n, i2 = t % n;
            const R e1 = s_x[i1], e2 = s_x[i2];
            const R w = s_w[i1] * s_w[i2] * fac;
            R hu, hx2, hy2, wr;
            if (r == 0) { hu = (R)1 - e1; hx2 = e1; hy2 = e2; wr = (R)1; }
            else if (r == 1) { hu = e1 * ((R)1 - e2); hx2 = e1 * e2; hy2 = (R)1; wr = e1; }
            else if (r == 2) { hu = -e1 * ((R)1 - e2); hx2 = (R)1; hy2 = e1 * e2; wr = e1; }
            else { hu = e1 - (R)1; hx2 = e2; hy2 = e1; wr = (R)1; }
            const R zx = hu * e10x + hy2 * fx - hx2 * e21x;
            const R zy = hu * e10y + hy2 * fy - hx2 * e21y;
            D[0] = hu;
            D[1] = -hu - hx2 + hy2;
            D[2] = hx2;  // the fourth difference is -hy2
            const R g = gamma_r<R>(zx * zx + zy * zy, P, cR);
            duffy_add<R, 3>(acc, D, w * wr * g);
        }
    } else {
        // common vertex: all four directions matter
        const R g10x = (R)(Bv[1].x - Av[0].x), g10y = (R)(Bv[1].y - Av[0].y);
        const R g21x = (R)(Bv[2].x - Bv[1].x), g21y = (R)(Bv[2].y - Bv[1].y);
        const int npts = 2 * n * n * n;
        for (int t = lane; t < npts; t += 32) {
            const int r = t / (n * n * n);
            const int i1 = (t / (n * n)) % n, i2 = (t / n) % n, i3 = t % n;
            const R e1 = s_x[i1], e2 = s_x[i2], e3 = s_x[i3];
            const R w = s_w13[i1 * n + i3] * s_wx[i2];  // w_i1 w_i2 w_i3 sxi e2
            const R hx1 = r == 0 ? (R)1 : e2, hy1 = r == 0 ? e2 : (R)1;
            const R zx = hy1 * (g10x + e3 * g21x) - hx1 * (e10x + e1 * e21x);
            const R zy = hy1 * (g10y + e3 * g21y) - hx1 * (e10y + e1 * e21y);
            D[0] = hy1 - hx1;
            D[1] = hx1 * s_1m[i1];
            D[2] = hx1 * e1;
            D[3] = -hy1 * s_1m[i3];  // the fifth difference is -hy1 e3
            const R g = gamma_r<R>(zx * zx + zy * zy, P, cR);
            duffy_add<R, 4>(acc, D, w * g);
        }
    }
    // the pair's factor det_k det_l, once on the lane sums
    const int L = U - 1, na = L * (L + 1) / 2;  // accumulated rows and entries
    for (int e = 0; e < 10; ++e) acc[e] *= scale;
    // warp reduction in a fixed tree (deterministic), in R: five levels of additions add a
    // relative error of a few R ulps to the lane sums (the FP64 pipe's 1/64 rate would make
    // an FP64 tree the costliest part of the FP32 kernel)
    double accd[10];
    for (int e = 0; e < 10; ++e) {
        R v = acc[e];
        if (e < na)
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        accd[e] = (double)v;
    }
    if (lane == 0) {
        // the block over the maps' vertex order: the accumulated rows, then the last row and
        // column from the zero row sums
        double mu[5][5];
        int e = 0;
        for (int a = 0; a < L; ++a)
            for (int b = a; b < L; ++b, ++e) {
                mu[a][b] = accd[e];
                mu[b][a] = accd[e];
            }
        double last = 0.0;
        for (int a = 0; a < L; ++a) {
            double s = 0.0;
            for (int b = 0; b < L; ++b) s += mu[a][b];
            mu[a][L] = -s;
            mu[L][a] = -s;
            last += s;
        }
        mu[L][L] = last;
        // write all 21 entries of the union block (unused ones are zero)
        double blk[6][6];
        for (int a = 0; a < 6; ++a)
            for (int b = 0; b < 6; ++b) blk[a][b] = 0.0;
        for (int a = 0; a < U; ++a)
            for (int b = 0; b < U; ++b) blk[upos[a]][upos[b]] = mu[a][b];
        const int64_t r = A.compact ? wi : (int64_t)p;
        const double fm = pair_factor64(P, k, l);
        for (int a = 0; a < 6; ++a)
            for (int b = a; b < 6; ++b) {
                if (contrib64) contrib64[r * NLFEM_REC1 + q_E1[a][b]] = fm * blk[a][b];
                else contrib32[r * NLFEM_REC1 + q_E1[a][b]] = (float)(fm * blk[a][b]);
            }
    }
}

// Touching pairs of a discontinuous mesh (eq. case-one-factoredOut, admissible for s <= 1/2):
// the shared vertices carry one dof per element, so the integrand's vector over the six dofs
// of the pair is (phi^k(x), -phi^l(y)) and its outer product holds the local, nonlocal and
// primed terms of that equation. The maps and weights are k_duffy's (common edge: 4 regions,
// common vertex: 2), but the basis values do not vanish with xi, so xi is summed with the
// Gauss rule like the other directions: n^4 points per region. Warp per pair, lanes over the
// points, a fixed shuffle tree in R; the record is the 6 x 6 block over (E_k's dofs, E_l's).
template <typename R>
__global__ void __launch_bounds__(128) k_duffy_split(DuffyArgs A, double* __restrict__ contrib64,
                                                     float* __restrict__ contrib32) {
    __shared__ R s_x[32], s_w[32];
    const Params& P = A.prm;
    for (int i = threadIdx.x; i < 32; i += blockDim.x) {
        s_x[i] = (R)(i < P.dr.n ? P.dr.x[i] : 0.0);
        s_w[i] = (R)(i < P.dr.n ? P.dr.w[i] : 0.0);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t wi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (wi >= A.n) return;
    const int p = A.ids[wi];
    const int k = A.pk[p], l = A.pl[p];
    if (k == l) return;  // identical pairs: k_duffy
    const int4 tk4 = A.T[k], tl4 = A.T[l];
    const int4 pk4 = A.Tp[k], pl4 = A.Tp[l];
    const int tk[3] = {tk4.x, tk4.y, tk4.z}, tl[3] = {tl4.x, tl4.y, tl4.z};
    const int qk[3] = {pk4.x, pk4.y, pk4.z}, ql[3] = {pl4.x, pl4.y, pl4.z};
    // shared vertices by position, in the same order in both elements
    int shared = 0, s0 = -1, s1 = -1, sl0 = -1, sl1 = -1;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            if (qk[a] == ql[b]) {
                if (s0 < 0) { s0 = a; sl0 = b; } else { s1 = a; sl1 = b; }
                ++shared;
            }
    if (shared < 1 || shared > 2) {
        // two elements on the same three points (a mesh with a duplicated triangle): no
        // admissible factored form; the record is zero
        if (lane == 0 && shared == 3) {
            const int64_t rr = A.compact ? wi : (int64_t)p;
            for (int e = 0; e < 21; ++e) {
                if (contrib64) contrib64[rr * NLFEM_REC1 + e] = 0.0;
                else contrib32[rr * NLFEM_REC1 + e] = 0.f;
            }
        }
        return;
    }
    int ak[3], bl[3];
    if (shared == 2) {
        ak[0] = s0; ak[1] = s1; ak[2] = 3 - s0 - s1;
        bl[0] = sl0; bl[1] = sl1; bl[2] = 3 - sl0 - sl1;
    } else {
        ak[0] = s0; ak[1] = (s0 + 1) % 3; ak[2] = (s0 + 2) % 3;
        bl[0] = sl0; bl[1] = (sl0 + 1) % 3; bl[2] = (sl0 + 2) % 3;
    }
    double2 Av[3], Bv[3];
    for (int a = 0; a < 3; ++a) {
        Av[a] = A.X[tk[ak[a]]];
        Bv[a] = A.X[tl[bl[a]]];
    }
    const R scale = (R)(A.det[k] * A.det[l]);
    const R cR = (R)P.c;
    const R e10x = (R)(Av[1].x - Av[0].x), e10y = (R)(Av[1].y - Av[0].y);
    const R e21x = (R)(Av[2].x - Av[1].x), e21y = (R)(Av[2].y - Av[1].y);
    const int n = P.dr.n, n2 = n * n, n4 = n2 * n2;
    R acc[21];
    for (int e = 0; e < 21; ++e) acc[e] = (R)0;
    R D[6];  // (phi^k_A0, phi^k_A1, phi^k_A2)(x), -(phi^l_B0, phi^l_B1, phi^l_B2)(y)
    const int npts = (shared == 2 ? 4 : 2) * n4;
    for (int t = lane; t < npts; t += 32) {
        const int r = t / n4, i0 = (t / (n2 * n)) % n, i1 = (t / n2) % n, i2 = (t / n) % n, i3 = t % n;
        const R xi = s_x[i0], e1 = s_x[i1], e2 = s_x[i2], e3 = s_x[i3];
        const R wq = s_w[i0] * s_w[i1] * s_w[i2] * s_w[i3];
        R zx, zy, w;
        if (shared == 2) {
            const R fx = (R)(Bv[2].x - Av[1].x), fy = (R)(Bv[2].y - Av[1].y);
            const R L = (R)1 - xi;
            R hu, hx2, hy2, wr;
            if (r == 0) { hu = (R)1 - e1; hx2 = e1; hy2 = e2; wr = (R)1; }
            else if (r == 1) { hu = e1 * ((R)1 - e2); hx2 = e1 * e2; hy2 = (R)1; wr = e1; }
            else if (r == 2) { hu = -e1 * ((R)1 - e2); hx2 = (R)1; hy2 = e1 * e2; wr = e1; }
            else { hu = e1 - (R)1; hx2 = e2; hy2 = e1; wr = (R)1; }
            const R u = xi * hu, x2 = xi * hx2, y2 = xi * hy2;
            const R x1 = (x2 > y2 - u ? x2 : y2 - u) + L * e3;
            const R y1 = x1 + u;
            zx = xi * (hu * e10x + hy2 * fx - hx2 * e21x);
            zy = xi * (hu * e10y + hy2 * fy - hx2 * e21y);
            w = wq * scale * xi * xi * L * wr;
            D[0] = (R)1 - x1; D[1] = x1 - x2; D[2] = x2;
            D[3] = -((R)1 - y1); D[4] = -(y1 - y2); D[5] = -y2;
        } else {
            const R g10x = (R)(Bv[1].x - Av[0].x), g10y = (R)(Bv[1].y - Av[0].y);
            const R g21x = (R)(Bv[2].x - Bv[1].x), g21y = (R)(Bv[2].y - Bv[1].y);
            const R x1 = xi * (r == 0 ? (R)1 : e2), y1 = xi * (r == 0 ? e2 : (R)1);
            zx = y1 * (g10x + e3 * g21x) - x1 * (e10x + e1 * e21x);
            zy = y1 * (g10y + e3 * g21y) - x1 * (e10y + e1 * e21y);
            w = wq * scale * xi * xi * xi * e2;
            D[0] = (R)1 - x1; D[1] = x1 * ((R)1 - e1); D[2] = x1 * e1;
            D[3] = -((R)1 - y1); D[4] = -y1 * ((R)1 - e3); D[5] = -y1 * e3;
        }
        const R wg = w * gamma_r<R>(zx * zx + zy * zy, P, cR);
        int e = 0;
#pragma unroll
        for (int a = 0; a < 6; ++a) {
            const R wa = wg * D[a];
#pragma unroll
            for (int b = a; b < 6; ++b) acc[e++] += wa * D[b];
        }
    }
    double accd[21];
    for (int e = 0; e < 21; ++e) {
        R v = acc[e];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        accd[e] = (double)v;
    }
    if (lane == 0) {
        // acc runs over (a <= b) of D's order; the record's block is over (E_k's dofs as
        // given, then E_l's): vertex A_a sits at ak[a], vertex B_b at 3 + bl[b]
        const int bpos[6] = {ak[0], ak[1], ak[2], 3 + bl[0], 3 + bl[1], 3 + bl[2]};
        const int64_t rr = A.compact ? wi : (int64_t)p;
        const double fm = pair_factor64(P, k, l);
        int e = 0;
        for (int a = 0; a < 6; ++a)
            for (int b = a; b < 6; ++b, ++e) {
                const int lo = min(bpos[a], bpos[b]), hi = max(bpos[a], bpos[b]);
                if (contrib64) contrib64[rr * NLFEM_REC1 + q_E1[lo][hi]] = fm * accd[e];
                else contrib32[rr * NLFEM_REC1 + q_E1[lo][hi]] = (float)(fm * accd[e]);
            }
    }
}

// The blocks k_duffy left to the mirrored order (duffy_mirror): each entry (a, b) of the pair's
// union block is the mirror's entry for the same two nodes. Thread per close-list entry; the
// mirrors (k < l) are only read.
template <typename RT>
__global__ void k_duffy_mirror(DuffyArgs A, RT* __restrict__ rec) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    const int p = A.ids[i];
    const int k = A.pk[p], l = A.pl[p];
    const int4 tk4 = A.T[k], tl4 = A.T[l];
    const int64_t j = duffy_mirror(A, k, l, tk4, tl4);
    if (j < 0) return;
    int posl[3], u[6], v[6];
    const int U = union_pos(tk4, tl4, posl, u);
    union_pos(tl4, tk4, posl, v);
    int pm[6];  // position in the mirror's union of each node of this pair's union
    for (int a = 0; a < 6; ++a) {
        pm[a] = 0;
        for (int b = 0; b < U; ++b)
            if (a < U && v[b] == u[a]) pm[a] = b;
    }
    const RT* src = rec + j * NLFEM_REC1;
    RT* dst = rec + (A.compact ? i : (int64_t)p) * NLFEM_REC1;
    for (int a = 0; a < 6; ++a)
        for (int b = a; b < 6; ++b)
            dst[q_E1[a][b]] = a < U && b < U ? src[q_E1[min(pm[a], pm[b])][max(pm[a], pm[b])]] : (RT)0;
}

// the singular rule over the close list: k_duffy (and k_duffy_mirror for the orders it leaves
// to their mirrors), and k_duffy_split for the touching pairs of a discontinuous mesh
template <typename R>
static void launch_duffy(const Mesh& m, const PairCache& pc, const Params& prm, int compact, double* out64,
                         float* out32, cudaStream_t st) {
    DuffyArgs d{pc.duffy_ids.p, pc.nduffy, compact, pc.pk.p, pc.pl.p, m.X.p, m.T.p, m.det.p, prm,
                m.tpos(), m.dg ? 1 : 0, pc.pair_ptr.p};
    const unsigned g = nblk(pc.nduffy * 32, 128);
    k_duffy<R><<<g, 128, 0, st>>>(d, out64, out32);
    NLFEM_LAUNCH_CHECK();
    if (!m.dg) {
        if (out64) k_duffy_mirror<double><<<nblk(pc.nduffy, 128), 128, 0, st>>>(d, out64);
        else k_duffy_mirror<float><<<nblk(pc.nduffy, 128), 128, 0, st>>>(d, out32);
        NLFEM_LAUNCH_CHECK();
    }
    if (m.dg) {
        k_duffy_split<R><<<g, 128, 0, st>>>(d, out64, out32);
        NLFEM_LAUNCH_CHECK();
    }
}

// ------------------------------------------------------------------------------------------
// load vector: F_i = sum_{E_k in Omega, i in E_k} sum_p a_p f(x_p) phi_i(x_p), f in P1
// ------------------------------------------------------------------------------------------
__global__ void k_load(int64_t M, int ndof, const int* ne_ptr, const int* ne_idx, const int4* T,
                       const int8_t* lab, const double* det, const double* f, Rule ro, double* F) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    for (int c = 0; c < ndof; ++c) {
        double acc = 0.0;
        for (int t = ne_ptr[i]; t < ne_ptr[i + 1]; ++t) {
            int k = ne_idx[t];
            if (!lab[k]) continue;
            int4 tk = T[k];
            int a = tk.x == i ? 0 : (tk.y == i ? 1 : 2);
            double fv[3] = {f[(int64_t)tk.x * ndof + c], f[(int64_t)tk.y * ndof + c], f[(int64_t)tk.z * ndof + c]};
            for (int p = 0; p < ro.n; ++p) {
                double fx = ro.l[p][0] * fv[0] + ro.l[p][1] * fv[1] + ro.l[p][2] * fv[2];
                acc += ro.w[p] * det[k] * fx * ro.l[p][a];
            }
        }
        F[i * ndof + c] = acc;
    }
}

template <typename R, bool WHOLE = false>
static void launch_trunc(const QuadArgs& a, R* out, cudaStream_t st) {
    const int NQI = a.prm.ri.n;
    const int K = a.prm.kernel;
    unsigned grid = (unsigned)std::min<int64_t>(nblk(a.npairs, 128), 152 * 64);
    if (grid == 0) return;
#define NLFEM_TR(KK, NQ) k_trunc<R, KK, NQ, WHOLE><<<grid, 128, 0, st>>>(a, out)
    if (K == NLFEM_KERNEL_CONSTANT) {
        if (NQI == 7) NLFEM_TR(NLFEM_KERNEL_CONSTANT, 7); else NLFEM_TR(NLFEM_KERNEL_CONSTANT, 16);
    } else if (K == NLFEM_KERNEL_FRACTIONAL) {
        if (NQI == 7) NLFEM_TR(NLFEM_KERNEL_FRACTIONAL, 7); else NLFEM_TR(NLFEM_KERNEL_FRACTIONAL, 16);
    } else if (K == NLFEM_KERNEL_TABULATED) {
        if (NQI == 7) NLFEM_TR(NLFEM_KERNEL_TABULATED, 7); else NLFEM_TR(NLFEM_KERNEL_TABULATED, 16);
    } else {
        if (NQI == 7) NLFEM_TR(NLFEM_KERNEL_PERIDYNAMIC, 7); else NLFEM_TR(NLFEM_KERNEL_PERIDYNAMIC, 16);
    }
#undef NLFEM_TR
    NLFEM_LAUNCH_CHECK();
}

// Close-list records (singular or diamond rule, FP32 in list order) into the fixed-point
// accumulators: each upper entry E(a, b) of the folded union block goes to the upper CSR
// entry of the node pair (u_a, u_b). acc == nullptr: only the largest |value| is recorded.
template <int NDOF, typename RT>
__global__ void k_close_acc(const int* __restrict__ ids, int64_t n, const int* __restrict__ pk,
                            const int* __restrict__ pl, const int4* __restrict__ T, const RT* __restrict__ rec,
                            const int64_t* __restrict__ nptr, const int* __restrict__ ncol,
                            const int64_t* __restrict__ up_start, unsigned long long* acc,
                            const float* __restrict__ scale_p, unsigned int* maxabs) {
    constexpr int NS = NDOF == 1 ? NLFEM_REC1 : NLFEM_REC2;
    constexpr int NCOMP = NDOF == 1 ? 1 : 4;
    constexpr int NC = NDOF == 1 ? 1 : 3;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float vmax = 0.f;
    const float scale = acc ? *scale_p : 1.f;
    if (i < n) {
        const int p = ids[i];
        int posl[3], u[6];
        const int U = union_pos(T[pk[p]], T[pl[p]], posl, u);
        const RT* r = rec + i * NS;
        for (int a = 0; a < U; ++a)
            for (int b = a; b < U; ++b) {
                const int lo = min(u[a], u[b]), hi = max(u[a], u[b]);
                const int64_t up = acc ? up_start[lo] + max(upper_rank(nptr, ncol, lo, hi), 0) : 0;
                const RT* v = r + q_E1[a][b] * NCOMP;
                const RT comp[3] = {v[0], v[NCOMP > 1 ? 1 : 0], v[NCOMP > 1 ? 3 : 0]};
                for (int c = 0; c < NC; ++c) {
                    vmax = fmaxf(vmax, fabsf((float)comp[c]));
                    // FP64 records (the singular rule in FP64) are scaled and rounded in FP64:
                    // the fixed-point sum then keeps their digits beyond FP32
                    const long long q = sizeof(RT) == 8 ? __double2ll_rn((double)comp[c] * (double)scale)
                                                        : __float2ll_rn((float)comp[c] * scale);
                    if (acc && q) atomicAdd(acc + up * NC + c, (unsigned long long)q);
                }
            }
    }
    for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    if ((threadIdx.x & 31) == 0 && vmax > 0.f) atomicMax(maxabs, __float_as_uint(vmax));
}

// ll of every element summed over its pairs (., l) in the order of the transposed index: a warp
// per element, a fixed butterfly, then one fixed-point add per node pair of the element. Pairs
// of the close list (singular or diamond rule) have no record and are skipped.
template <int NC>
__global__ void k_ll_sums(int64_t K, const int64_t* __restrict__ ptr, const int* __restrict__ perm,
                          const int8_t* __restrict__ pcls, int skip_close, const float* __restrict__ llrec,
                          const int* __restrict__ epos, unsigned long long* __restrict__ acc,
                          const float* __restrict__ scale_p) {
    const int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (e >= K) return;  // whole warps leave together
    float s[6 * NC];
#pragma unroll
    for (int x = 0; x < 6 * NC; ++x) s[x] = 0.f;
    for (int64_t j = ptr[e] + lane; j < ptr[e + 1]; j += 32) {
        const int64_t p = perm[j];
        if (skip_close && pcls[p] > 0) continue;
        const float2* r = reinterpret_cast<const float2*>(llrec + p * (6 * NC));
#pragma unroll
        for (int x = 0; x < 3 * NC; ++x) {
            const float2 v = r[x];
            s[2 * x] += v.x;
            s[2 * x + 1] += v.y;
        }
    }
#pragma unroll
    for (int x = 0; x < 6 * NC; ++x)
        for (int o = 16; o > 0; o >>= 1) s[x] += __shfl_xor_sync(0xffffffffu, s[x], o);
    const float scale = *scale_p;
    if (lane == 0)
#pragma unroll
        for (int x = 0; x < 6; ++x) {
            const int64_t u = epos[e * 8 + x];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const long long q = __float2ll_rn(s[c * 6 + x] * scale);
                if (q) atomicAdd(acc + u * NC + c, (unsigned long long)q);
            }
        }
}

static void ll_sums(Mesh& m, PairCache& pc, const Params& prm, System& sys, const float* scale, cudaStream_t st) {
    const int skip = close_mode(prm) != 0;
    const unsigned g = nblk(m.K * 32, 256);
    if (m.K == 0) return;
    if (pc.ndof == 1)
        k_ll_sums<1><<<g, 256, 0, st>>>(m.K, pc.pT_ptr.p, pc.pT_id.p, pc.pcls.p, skip, sys.llrec.p, pc.epos.p,
                                        sys.acc.p, scale);
    else
        k_ll_sums<3><<<g, 256, 0, st>>>(m.K, pc.pT_ptr.p, pc.pT_id.p, pc.pcls.p, skip, sys.llrec.p, pc.epos.p,
                                        sys.acc.p, scale);
    NLFEM_LAUNCH_CHECK();
}

// the close list's records are FP64 when the singular rule ran in FP64 (bulk_close64)
static bool bulk_close64(const Params& prm) { return prm.singular && !prm.sing32; }

static void close_acc(Mesh& m, PairCache& pc, const System& sys, unsigned long long* acc, const float* scale,
                      unsigned int* maxabs, cudaStream_t st) {
    if (pc.nduffy == 0) return;
    const unsigned g = nblk(pc.nduffy, 128);
    const bool r64 = bulk_close64(sys.prm);
    if (pc.ndof == 1 && r64)
        k_close_acc<1, double><<<g, 128, 0, st>>>(pc.duffy_ids.p, pc.nduffy, pc.pk.p, pc.pl.p, m.T.p,
                                                  sys.contrib64.p, pc.nrow_ptr.p, pc.ncol.p, pc.up_start.p, acc,
                                                  scale, maxabs);
    else if (pc.ndof == 1)
        k_close_acc<1, float><<<g, 128, 0, st>>>(pc.duffy_ids.p, pc.nduffy, pc.pk.p, pc.pl.p, m.T.p,
                                                 sys.contrib32.p, pc.nrow_ptr.p, pc.ncol.p, pc.up_start.p, acc,
                                                 scale, maxabs);
    else  // peridynamics has no singular rule: FP32 records of the diamond or standard rule
        k_close_acc<2, float><<<g, 128, 0, st>>>(pc.duffy_ids.p, pc.nduffy, pc.pk.p, pc.pl.p, m.T.p,
                                                 sys.contrib32.p, pc.nrow_ptr.p, pc.ncol.p, pc.up_start.p, acc,
                                                 scale, maxabs);
    NLFEM_LAUNCH_CHECK();
}

// the close list of the FP32-bulk path: the singular rule (FP64 records by default, FP32 with
// sing32) or the truncation kernel in FP32 (diamond / standard rule) into compact records
static void bulk_close(Mesh& m, PairCache& pc, const Params& prm, System& sys, cudaStream_t st, bool ensure) {
    if (pc.nduffy == 0) return;
    const int64_t n = pc.nduffy * contrib_entries(pc.ndof);
    if (bulk_close64(prm)) {
        if (ensure) sys.contrib64.ensure(n, st);
        else sys.contrib64.alloc(n, st);
        launch_duffy<double>(m, pc, prm, 1, sys.contrib64.p, nullptr, st);
        return;
    }
    if (ensure) sys.contrib32.ensure(n, st);
    else sys.contrib32.alloc(n, st);
    if (prm.singular) {
        launch_duffy<float>(m, pc, prm, 1, nullptr, sys.contrib32.p, st);
    } else {
        QuadArgs c{pc.pk.p, pc.pl.p, pc.pcls.p, nullptr, pc.nduffy, pc.duffy_ids.p, 1, m.X.p, m.T.p, m.det.p, prm};
        launch_trunc<float>(c, sys.contrib32.p, st);
    }
}

// FNV-1a over the parameter bytes with the device pointers cleared (the struct is zeroed
// before it is filled, so its padding is zero too)
static uint64_t params_key(const Params& prm) {
    Params q = prm;
    q.mat = nullptr;
    q.msc64 = nullptr;
    q.msc32 = nullptr;
    q.tab64 = nullptr;
    q.tab32 = nullptr;
    const unsigned char* b = reinterpret_cast<const unsigned char*>(&q);
    uint64_t h = 1469598103934665603ull;
    for (size_t i = 0; i < sizeof q; ++i) h = (h ^ b[i]) * 1099511628211ull;
    return h ? h : 1;
}

// the scale from the pilot's largest |value|, with 2^8 of headroom
__global__ void k_fix_pick(FixState* f, int64_t terms) {
    const int S = fix_shift(__uint_as_float(f->max_pilot), terms, 8);
    f->shift = S;
    f->scale = ldexpf(1.f, S);
    f->max_exact = 0u;
    f->redo = 0;
}

void pick_scale(Mesh& m, PairCache& pc, const Params& prm, FixState* f, cudaStream_t st) {
    launch_trunc_fast(m, pc, prm, BulkAcc{nullptr, nullptr, nullptr, &f->max_pilot, 61}, st, nullptr);
    k_fix_pick<<<1, 1, 0, st>>>(f, pc.acc_terms);
    NLFEM_LAUNCH_CHECK();
}

// the main pass may keep its scale if no sum could overflow and at most 2^16 of range is unused
__global__ void k_fix_check(FixState* f, int64_t terms) {
    const int Se = fix_shift(__uint_as_float(f->max_exact), terms, 0);
    f->shift_exact = Se;
    f->redo = (f->shift <= Se && f->shift >= Se - 16) ? 0 : 1;
}

__global__ void k_fix_exact(FixState* f) {
    f->shift = f->shift_exact;
    f->scale = ldexpf(1.f, f->shift);
    f->max_exact = 0u;
    f->redo = 0;
}

static void bulk_main(Mesh& m, PairCache& pc, const Params& prm, System& sys, cudaStream_t st, cudaEvent_t* ev) {
    FixState* f = sys.fix.p;
    sys.acc.zero(st);
    launch_trunc_fast(m, pc, prm, BulkAcc{sys.acc.p, sys.llrec.p, &f->scale, &f->max_exact, 1}, st, ev + 2);
    ll_sums(m, pc, prm, sys, &f->scale, st);
    close_acc(m, pc, sys, sys.acc.p, &f->scale, &f->max_exact, st);
    NLFEM_CUDA_TRY(cudaEventRecord(ev[5], st));
    k_fix_check<<<1, 1, 0, st>>>(f, pc.acc_terms);
    NLFEM_LAUNCH_CHECK();
}

// FP32-bulk path, stream-ordered with no host round trip: (1) the close list (singular rule
// in FP64, or the canonical truncation kernel) writes compact records; (2) a pilot pass over
// every 61st pair of the whole and cut lists, plus the close records, records the largest
// |value| and k_fix_pick fixes the scale 2^S; (3) the bulk kernels add kl into the
// fixed-point accumulators (kl per pair, kk per outer element of a warp tile) and write ll
// records, which k_ll_sums sums per element, and the close records are added, recording the
// exact largest |value|; (4) k_fix_check
// flags the assembly if that value could overflow a sum or leaves more than 2^16 of unused
// range; the caller then runs bulk_redo (3 again with the scale from the exact value). S is
// a function of the inputs alone, so the result is the same in every run.
static void run_bulk(Mesh& m, PairCache& pc, const Params& prm, System& sys, cudaStream_t st, cudaEvent_t* ev) {
    const int NC = pc.ndof == 1 ? 1 : 3;
    NLFEM_CUDA_TRY(cudaEventRecord(ev[0], st));
    bulk_close(m, pc, prm, sys, st, false);
    NLFEM_CUDA_TRY(cudaEventRecord(ev[1], st));
    sys.fix.alloc(1, st);
    sys.fix.zero(st);
    FixState* f = sys.fix.p;
    // the pilot's pick depends on the pattern and the parameters only: for the same parameters
    // (no device tables) the scale of the last assembly on this pattern is reused
    const uint64_t key = (prm.nmat == 0 && prm.ntab == 0) ? params_key(prm) : 0;
    if (key && pc.scale_memo_valid && pc.scale_key == key) {
        NLFEM_CUDA_TRY(cudaMemcpyAsync(f, pc.scale_memo.p, sizeof(FixState), cudaMemcpyDeviceToDevice, st));
    } else {
        launch_trunc_fast(m, pc, prm, BulkAcc{nullptr, nullptr, nullptr, &f->max_pilot, 61}, st, nullptr);
        close_acc(m, pc, sys, nullptr, nullptr, &f->max_pilot, st);
        k_fix_pick<<<1, 1, 0, st>>>(f, pc.acc_terms);
        NLFEM_LAUNCH_CHECK();
        if (key) {
            pc.scale_memo.alloc(1, st);
            NLFEM_CUDA_TRY(cudaMemcpyAsync(pc.scale_memo.p, f, sizeof(FixState), cudaMemcpyDeviceToDevice, st));
            pc.scale_key = key;
            pc.scale_memo_valid = true;
        }
    }
    sys.acc.alloc(std::max<int64_t>(pc.n_upper * NC, 1), st);
    sys.llrec.alloc(std::max<int64_t>(pc.npairs * 6 * NC, 1), st);
    bulk_main(m, pc, prm, sys, st, ev);
}

void bulk_redo(Mesh& m, PairCache& pc, const Params& prm, System& sys, cudaStream_t st, cudaEvent_t* ev) {
    k_fix_exact<<<1, 1, 0, st>>>(sys.fix.p);
    NLFEM_LAUNCH_CHECK();
    bulk_main(m, pc, prm, sys, st, ev);
}

// FP32-bulk assembly of several systems: the same steps as run_bulk, with the whole- and
// cut-pair kernels of all requests of one kernel class fused into one launch each (pilot and
// main pass). Each system's scale is chosen from its own pilot values, so every system is
// the same bits as when it is assembled alone. Events (optional): [0, 1] close-list kernels,
// [2, 3] fused whole-pair launches, [3, 4] fused cut-pair launches, [4, 5] ll sums and
// close-list adds.
static int64_t class_key(const Params& p) {
    return ((int64_t)p.kernel * 64 + p.ro.n) * 64 * 8 + (int64_t)p.ri.n * 8 + p.ball;
}

void BatchExec::prepare(cudaStream_t st) {
    set_fast_attributes();
    for (BatchSys& it : items) {
        PairCache& pc = *it.pc;
        System& sys = *it.sys;
        const int NC = pc.ndof == 1 ? 1 : 3;
        if (pc.nduffy > 0) {
            if (bulk_close64(it.prm)) sys.contrib64.ensure(pc.nduffy * contrib_entries(pc.ndof), st);
            else sys.contrib32.ensure(pc.nduffy * contrib_entries(pc.ndof), st);
        }
        sys.fix.ensure(1, st);
        sys.acc.ensure(std::max<int64_t>(pc.n_upper * NC, 1), st);
        sys.llrec.ensure(std::max<int64_t>(pc.npairs * 6 * NC, 1), st);
    }
    std::vector<int64_t> keys;  // kernel classes, in the order of first appearance
    for (BatchSys& it : items) {
        const int64_t k = class_key(it.prm);
        if (std::find(keys.begin(), keys.end(), k) == keys.end()) keys.push_back(k);
    }
    pilot.clear();
    whole.clear();
    cut.clear();
    for (int64_t key : keys) {
        std::vector<BulkItem> gp, gm;
        for (BatchSys& it : items) {
            if (class_key(it.prm) != key) continue;
            FixState* f = it.sys->fix.p;
            gp.push_back(BulkItem{it.m, it.pc, it.prm, BulkAcc{nullptr, nullptr, nullptr, &f->max_pilot, 61}});
            gm.push_back(BulkItem{it.m, it.pc, it.prm, BulkAcc{it.sys->acc.p, it.sys->llrec.p, &f->scale, &f->max_exact,
                                                               1}});
        }
        pilot.push_back(make_fused(gp, 0, 61, st));
        pilot.push_back(make_fused(gp, 1, 61, st));
        whole.push_back(make_fused(gm, 0, 0, st));
        cut.push_back(make_fused(gm, 1, 0, st));
    }
}

void BatchExec::record(cudaStream_t st, cudaEvent_t* ev, bool finish, const std::vector<const double*>& f) {
    if (ev) NLFEM_CUDA_TRY(cudaEventRecord(ev[0], st));
    for (BatchSys& it : items) {
        Mesh& m = *it.m;
        PairCache& pc = *it.pc;
        System& sys = *it.sys;
        bulk_close(m, pc, it.prm, sys, st, true);
        sys.fix.zero(st);
    }
    if (ev) NLFEM_CUDA_TRY(cudaEventRecord(ev[1], st));
    for (const auto& fl : pilot) run_fused(*fl, st);
    for (BatchSys& it : items) {
        close_acc(*it.m, *it.pc, *it.sys, nullptr, nullptr, &it.sys->fix.p->max_pilot, st);
        k_fix_pick<<<1, 1, 0, st>>>(it.sys->fix.p, it.pc->acc_terms);
        NLFEM_LAUNCH_CHECK();
        it.sys->acc.zero(st);
    }
    if (ev) NLFEM_CUDA_TRY(cudaEventRecord(ev[2], st));
    for (const auto& fl : whole) run_fused(*fl, st);
    if (ev) NLFEM_CUDA_TRY(cudaEventRecord(ev[3], st));
    for (const auto& fl : cut) run_fused(*fl, st);
    if (ev) NLFEM_CUDA_TRY(cudaEventRecord(ev[4], st));
    for (BatchSys& it : items) {
        FixState* fx = it.sys->fix.p;
        ll_sums(*it.m, *it.pc, it.prm, *it.sys, &fx->scale, st);
        close_acc(*it.m, *it.pc, *it.sys, it.sys->acc.p, &fx->scale, &fx->max_exact, st);
        k_fix_check<<<1, 1, 0, st>>>(fx, it.pc->acc_terms);
        NLFEM_LAUNCH_CHECK();
    }
    if (ev) NLFEM_CUDA_TRY(cudaEventRecord(ev[5], st));
    if (!finish) return;
    for (size_t i = 0; i < items.size(); ++i) {
        BatchSys& it = items[i];
        run_reduction(*it.m, *it.pc, it.prm, *it.sys, st);
        run_load(*it.m, it.prm, f.empty() ? nullptr : f[i], *it.sys, st);
    }
}

void run_bulk_batch(std::vector<BatchSys>& items, cudaStream_t st, cudaEvent_t* ev) {
    BatchExec e;
    e.items = items;
    e.prepare(st);
    e.record(st, ev, false, {});
}

void run_quadrature(Mesh& m, PairCache& pc, const Params& prm, System& sys, cudaStream_t st, cudaEvent_t* ev) {
    if (prm.precision == NLFEM_PREC_FP32_BULK) {
        run_bulk(m, pc, prm, sys, st, ev);
        return;
    }
    // FP64 plain: the canonical kernel over the whole-pair list (no clip), the cut-pair list and,
    // under the diamond rule, the close list (reported together as the cut-pair time; every
    // list's warps then do the same kind of work), then the singular rule on the close list.
    // Records go to each pair's id, so the reduction does not depend on the split.
    NLFEM_CUDA_TRY(cudaEventRecord(ev[2], st));
    NLFEM_CUDA_TRY(cudaEventRecord(ev[3], st));
    {
        QuadArgs a{pc.pk.p, pc.pl.p, pc.pcls.p, nullptr, pc.nwhole, pc.whole_ids.p, 0, m.X.p, m.T.p, m.det.p, prm};
        launch_trunc<double, true>(a, sys.contrib64.p, st);
        a.npairs = pc.ncut;
        a.ids = pc.cut_ids.p;
        launch_trunc<double>(a, sys.contrib64.p, st);
        if (!prm.singular && pc.nduffy > 0) {
            a.npairs = pc.nduffy;
            a.ids = pc.duffy_ids.p;
            launch_trunc<double>(a, sys.contrib64.p, st);
        }
    }
    NLFEM_CUDA_TRY(cudaEventRecord(ev[4], st));
    NLFEM_CUDA_TRY(cudaEventRecord(ev[0], st));
    if (prm.singular && pc.nduffy > 0) launch_duffy<double>(m, pc, prm, 0, sys.contrib64.p, nullptr, st);
    NLFEM_CUDA_TRY(cudaEventRecord(ev[1], st));
    NLFEM_CUDA_TRY(cudaEventRecord(ev[5], st));
}

void run_load(Mesh& m, const Params& prm, const double* f_nodal, System& sys, cudaStream_t st) {
    if (!f_nodal) {
        NLFEM_CUDA_TRY(cudaMemsetAsync(sys.F.p, 0, sys.F.bytes(), st));
        return;
    }
    k_load<<<nblk(m.M, 128), 128, 0, st>>>(m.M, prm.ndof, m.ne_ptr.p, m.ne_idx.p, m.T.p, m.lab.p, m.det.p,
                                           f_nodal, prm.ro, sys.F.p);
    NLFEM_LAUNCH_CHECK();
}

}  // namespace nlfem

// ------------------------------------------------------------------------------------------
// census: the work of the last assembly, counted on the device with the same geometry
// ------------------------------------------------------------------------------------------
namespace nlfem {

__device__ __forceinline__ void warp_add(unsigned long long* c, unsigned long long v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(c, v);
}

__global__ void k_census(QuadArgs A, unsigned long long* cnt) {
    const Params& P = A.prm;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n_iter = (A.npairs + stride - 1) / stride;
    for (int64_t it = 0; it < n_iter; ++it) {
        int64_t p = it * stride + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        unsigned long long evals = 0, full = 0, cut = 0, sub = 0, empty = 0, tp = 0, sp = 0, outer = 0;
        int list = 0;  // 1: whole-pair kernel, 2: cut-pair kernel, 0: canonical kernels
        if (p < A.npairs) {
            const int cls = A.pcls[p];
            if (cls > 0 && P.singular) {
                sp = 1;
            } else {
                list = A.whole ? A.whole[p] : 0;
                tp = 1;
                const int4 tk = A.T[A.pk[p]], tl = A.T[A.pl[p]];
                const double2 Vk[3] = {A.X[tk.x], A.X[tk.y], A.X[tk.z]};
                const double2 Vl[3] = {A.X[tl.x], A.X[tl.y], A.X[tl.z]};
                for (int q0 = 0; q0 < P.ro.n; ++q0) {
                    const double2 xp = nl_map(Vk, P.ro.l[q0][0], P.ro.l[q0][1], P.ro.l[q0][2]);
                    bool f;
                    const int np = nl_clip_ball(P.ball, Vl, xp, P.delta, P.delta2, nullptr, f);
                    ++outer;
                    if (np < 3) { ++empty; continue; }
                    if (f) { ++full; evals += P.ri.n; }
                    else { ++cut; sub += np - 2; evals += (unsigned long long)(np - 2) * P.ri.n; }
                }
            }
        }
        warp_add(&cnt[0], evals);
        warp_add(&cnt[1], full);
        warp_add(&cnt[2], cut);
        warp_add(&cnt[3], sub);
        warp_add(&cnt[5], tp);
        warp_add(&cnt[6], sp);
        warp_add(&cnt[7], empty);
        warp_add(&cnt[8], outer);
        warp_add(&cnt[9], list == 1 ? evals : 0ull);
        warp_add(&cnt[10], list == 2 ? evals : 0ull);
        warp_add(&cnt[11], list == 2 ? outer : 0ull);
        warp_add(&cnt[12], list == 2 ? cut : 0ull);
        warp_add(&cnt[13], list == 2 ? full + cut : 0ull);
        warp_add(&cnt[14], list == 2 ? sub * P.ri.n : 0ull);
        warp_add(&cnt[15], list == 0 ? evals : 0ull);
    }
}

// close-list pairs that take their block from the mirrored order (duffy_mirror): [0] common
// edge, [1] common vertex
__global__ void k_mirror_count(DuffyArgs A, unsigned long long* cnt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long e = 0, v = 0;
    if (i < A.n) {
        const int p = A.ids[i];
        const int k = A.pk[p], l = A.pl[p];
        const int4 tk = A.T[k], tl = A.T[l];
        if (duffy_mirror(A, k, l, tk, tl) >= 0) {
            const int shared = (tk.x == tl.x) + (tk.x == tl.y) + (tk.x == tl.z) + (tk.y == tl.x) + (tk.y == tl.y) +
                               (tk.y == tl.z) + (tk.z == tl.x) + (tk.z == tl.y) + (tk.z == tl.z);
            e = shared == 2;
            v = shared == 1;
        }
    }
    warp_add(&cnt[0], e);
    warp_add(&cnt[1], v);
}

__global__ void k_mark(const int* ids, int64_t n, int8_t v, int8_t* flag) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[ids[i]] = v;
}

void run_census(Mesh& m, PairCache& pc, const Params& prm, int64_t* out, cudaStream_t st) {
    DBuf<unsigned long long> c;
    c.alloc(18, st);  // the census, then the mirrored common-edge and common-vertex pairs
    c.zero(st);
    DBuf<int8_t> wflag;
    wflag.alloc(pc.npairs, st);
    wflag.zero(st);
    if (pc.nwhole > 0) {
        k_mark<<<nblk(pc.nwhole, 256), 256, 0, st>>>(pc.whole_ids.p, pc.nwhole, 1, wflag.p);
        NLFEM_LAUNCH_CHECK();
    }
    if (pc.ncut > 0) {
        k_mark<<<nblk(pc.ncut, 256), 256, 0, st>>>(pc.cut_ids.p, pc.ncut, 2, wflag.p);
        NLFEM_LAUNCH_CHECK();
    }
    QuadArgs a{pc.pk.p, pc.pl.p, pc.pcls.p, wflag.p, pc.npairs, nullptr, 0, m.X.p, m.T.p, m.det.p, prm};
    unsigned grid = (unsigned)std::min<int64_t>(nblk(pc.npairs, 256), 152 * 32);
    if (grid) {
        k_census<<<grid, 256, 0, st>>>(a, c.p);
        NLFEM_LAUNCH_CHECK();
    }
    if (prm.singular && !m.dg && pc.nduffy > 0) {
        DuffyArgs d{pc.duffy_ids.p, pc.nduffy, 1, pc.pk.p, pc.pl.p, m.X.p, m.T.p, m.det.p, prm,
                    m.tpos(), 0, pc.pair_ptr.p};
        k_mirror_count<<<nblk(pc.nduffy, 256), 256, 0, st>>>(d, c.p + 16);
        NLFEM_LAUNCH_CHECK();
    }
    unsigned long long h[18];
    NLFEM_CUDA_TRY(cudaMemcpyAsync(h, c.p, sizeof h, cudaMemcpyDeviceToHost, st));
    NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
    // singular-rule kernel evaluations: 6 n (identical), 4 n^2 (edge), 2 n^3 (vertex), for the
    // pairs that evaluate (the mirrored orders copy); the xi direction (and the directions along
    // which the integrand is constant) are summed in closed form. Touching pairs of a
    // discontinuous mesh: 4 n^4 (edge), 2 n^4 (vertex).
    const int64_t n = prm.dr.n;
    int64_t duffy = 0;
    if (prm.singular && m.dg) duffy = pc.counts[3] * 6 * n + (pc.counts[2] * 4 + pc.counts[1] * 2) * n * n * n * n;
    else if (prm.singular)
        duffy = pc.counts[3] * 6 * n + (pc.counts[2] - (int64_t)h[16]) * 4 * n * n +
                (pc.counts[1] - (int64_t)h[17]) * 2 * n * n * n;
    h[4] = (unsigned long long)duffy;
    for (int i = 0; i < 16; ++i) out[i] = (int64_t)h[i];
}

}  // namespace nlfem
