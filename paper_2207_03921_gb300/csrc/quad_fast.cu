// FP32-bulk truncation quadrature for separated pairs (Sec. 2.3.1, eq. discrete-inner)
// with exact geometric decisions.
//
// GB300 runs FP64 at 1/58 of the FP32 rate, so the canonical FP64 clip of every
// (pair, x_p) would dominate the bulk path. Here the geometry runs in FP32 on vectors
// relative to x_p (the pair offset v0_l - v0_k is formed once in FP64 and rounded once;
// element edges are stored in FP32), and every decision the canonical FP64 geometry
// takes — vertex in ball, number of crossings on an edge, a cap on a chord — is taken in
// FP32 only when its margin exceeds a bound on the FP32 error (nl_decide32). Otherwise
// the outer point falls back to the canonical FP64 clip (nl_clip). The interaction
// pattern and the polygon topology therefore equal the FP64 ones; crossing points, cap
// centres and sub-triangle areas carry FP32 rounding (about 1e-7 relative).
//
// Work layout: one thread per ordered pair. Pairs whose inner element lies in the ball of
// every outer point (decided at pair-search time) take k_trunc_whole: no geometry, fully
// uniform. The others take k_trunc_cut: the geometry of a chunk of outer points runs in
// lockstep across the warp, then a drain loop integrates one fan triangle per lane and
// iteration, so the inner rule runs with (nearly) the whole warp and exists once in the
// code.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "nlfem_internal.cuh"

namespace nlfem {

static inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

static constexpr int FAST_THREADS = 128;

// Arguments shared by every pair of a launch: the quadrature rules (one kernel class).
struct FastRule {
    float ol[16][3], ow[16];  // outer rule in FP32
    float il[16][3], iw[16];  // inner rule in FP32
    double ro[16][3];         // outer barycentrics in FP64 (canonical fallback)
    int nqo;
};

// Arguments of one request (one mesh and parameter set), read from a device table so that
// one launch can serve the pairs of many requests.
struct FastReq {
    const int* pk;
    const int* pl;
    const int8_t* pcls;
    const int* ids;           // the work list (whole or cut pairs)
    const int2* lkl;          // whole-pair list: (k, l) of every entry (the kernel skips the pk / pl lookups)
    int64_t npairs;           // its length
    const double2* X;
    const int4* T;
    const float4* E32;
    const float* det32;
    const ElemRec* rec;
    float delta, d2, c, s;
    double delta64, delta2_64;
    int ball;     // NLFEM_BALL_*
    int geo64;    // every cut outer point takes the canonical FP64 cut (no FP32 positions)
    int nmat;     // label-dependent kernel: factor msc[mat[k] * nmat + mat[l]] (0: none)
    const int8_t* mat;
    const float* msc;
    int ntab;     // user-defined radial kernel: table of g at r_i = i / tinv
    float tinv;
    const float* tab;
    // fixed-point accumulation into the upper CSR entries (see accumulate_pair)
    unsigned long long* acc;  // [n_upper][NC] int64 two's complement sums
    float* llrec;             // [P][6 NC] ll of every pair, by pair id (summed per element later)
    const int64_t* up_start;  // [M + 1] first upper entry of each node row
    const int* epos;          // [K][8] upper entries of an element's six node pairs (kkI order), padded
    const uint16_t* klr;      // [9][npairs] rank of the kl node pair in its upper row, list order
    const float* scale_p;     // 2^S (device memory)
    unsigned int* maxabs;     // bits of the largest |value| seen (a positive float), atomicMax
};

// A launch processes tiles of 32 consecutive list positions of one request, one warp per
// tile (warps never wait for each other): tile t = (request, first position); without a
// table, tile t of request 0 starts at 32 t. pilot > 0: only every pilot-th pair of each
// list, largest |value| only.
struct FastLaunch {
    const FastReq* reqs;      // batched launches: the request table (device memory)
    const int64_t* tile_off;  //   and the first tile of each request [nreq + 1]
    int nreq;
    int64_t ntiles;
    int pilot;
    int chunk;                // cut-pair kernel: outer points per chunk (1 .. CHUNK; 0 = CHUNK)
    FastReq one;              // single-request launches: the request itself (constant bank)
};

template <int NC>
struct Inner {
    float g[NC], h[3][NC], m[6][NC];
};

// the inner rule on triangle (a, b, c) of area dT / 2: positions relative to x_p (read by kernels
// other than the constant one), barycentric (b1, b2) w.r.t. E_l
template <int KER, int NQI, int NC>
__device__ __forceinline__ void tri_quad(const FastRule& R, const FastReq& Q, Inner<NC>& I, float dT, float ax,
                                         float ay, float a1, float a2,
                                         float bx, float by, float b1, float b2, float cx, float cy, float c1,
                                         float c2) {
    // the basis functions sum to one (Q0 = 1 - Q1 - Q2), so per point only the sums of w,
    // w Q1, w Q2, w Q1^2, w Q1 Q2 and w Q2^2 are formed; h0 and the m entries with Q0 follow
    // from them per triangle (the same quadrature sums, rearranged)
    // the weights' common factor |det| c of the triangle is applied once to the six sums; the
    // basis values are interpolated from vertex a along the two edge differences
    float g[NC], h1[NC], h2[NC], m11[NC], m12[NC], m22[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) g[c] = h1[c] = h2[c] = m11[c] = m12[c] = m22[c] = 0.f;
    const float d1b = b1 - a1, d1c = c1 - a1, d2b = b2 - a2, d2c = c2 - a2;
#pragma unroll
    for (int q = 0; q < NQI; ++q) {
        const float l0 = R.il[q][0], l1 = R.il[q][1], l2 = R.il[q][2];
        const float Q1 = fmaf(l2, d1c, fmaf(l1, d1b, a1));
        const float Q2 = fmaf(l2, d2c, fmaf(l1, d2b, a2));
        const float wq = R.iw[q];
        float wc[NC];
        if (KER == NLFEM_KERNEL_CONSTANT) {
            wc[0] = wq;
        } else {
            const float zx = l0 * ax + l1 * bx + l2 * cx;
            const float zy = l0 * ay + l1 * by + l2 * cy;
            const float r2 = zx * zx + zy * zy;
            if (KER == NLFEM_KERNEL_FRACTIONAL) {
                if (Q.s == 0.5f) {
                    const float r = rsqrtf(r2);
                    wc[0] = wq * r * r * r;
                } else {
                    wc[0] = wq * exp2f(log2f(r2) * (-1.f - Q.s));
                }
            } else if (KER == NLFEM_KERNEL_TABULATED) {
                wc[0] = wq * table_g<float>(Q.tab, Q.ntab, Q.tinv, r2);
            } else {
                const float r = rsqrtf(r2);
                const float sc = wq * r * r * r;
                wc[0] = sc * zx * zx;
                wc[1 % NC] = sc * zx * zy;
                wc[2 % NC] = sc * zy * zy;
            }
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const float w = wc[c];
            const float w1 = w * Q1, w2 = w * Q2;
            g[c] += w;
            h1[c] += w1;
            h2[c] += w2;
            m11[c] += w1 * Q1;
            m12[c] += w1 * Q2;
            m22[c] += w2 * Q2;
        }
    }
    const float f = dT * Q.c;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        g[c] *= f;
        h1[c] *= f;
        h2[c] *= f;
        m11[c] *= f;
        m12[c] *= f;
        m22[c] *= f;
        const float h0 = g[c] - h1[c] - h2[c];
        const float m01 = h1[c] - m11[c] - m12[c];
        const float m02 = h2[c] - m12[c] - m22[c];
        I.g[c] += g[c];
        I.h[0][c] += h0;
        I.h[1][c] += h1[c];
        I.h[2][c] += h2[c];
        I.m[0][c] += h0 - m01 - m02;
        I.m[1][c] += m01;
        I.m[2][c] += m02;
        I.m[3][c] += m11[c];
        I.m[4][c] += m12[c];
        I.m[5][c] += m22[c];
    }
}

// kk += a_p g P P^T, kl -= a_p P h^T, ll += a_p m for outer point q0 (P = its barycentrics)
// o = (l0, l1, l2, w) of the outer point
template <int NC>
__device__ __forceinline__ void outer_update(float4 o, float dk, const Inner<NC>& I, float (&kk)[6][NC],
                                             float (&kl)[9][NC], float (&ll)[6][NC]) {
    const float ap = o.w * dk;
    const float Pa[3] = {o.x, o.y, o.z};
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const float ag = ap * I.g[c];
        kk[0][c] += ag * Pa[0] * Pa[0];
        kk[1][c] += ag * Pa[0] * Pa[1];
        kk[2][c] += ag * Pa[0] * Pa[2];
        kk[3][c] += ag * Pa[1] * Pa[1];
        kk[4][c] += ag * Pa[1] * Pa[2];
        kk[5][c] += ag * Pa[2] * Pa[2];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) kl[a * 3 + b][c] -= ap * Pa[a] * I.h[b][c];
#pragma unroll
        for (int j = 0; j < 6; ++j) ll[j][c] += ap * I.m[j][c];
    }
}

// Accumulation of a pair's block [[kk, kl], [kl^T, ll]] into the fixed-point upper CSR
// entries: each value v is rounded once to the signed 64-bit integer v * 2^S and added with an
// integer atomic. Integer addition is associative, so the sums are the same bits in every run
// whatever order the pairs (or the warps) are processed in. kl[a][b] belongs to the node pair
// (k_a, l_b) (counted twice when the two nodes coincide: both mirrored entries of the symmetric
// block are diagonal); kk belongs to the node pairs of E_k and is first summed over the warp's
// pairs with the same outer element (accumulate_kk); ll belongs to those of E_l, which differ
// from lane to lane: it is written to the pair's record and summed per element in a fixed order
// (k_ll_sums), since six more atomics per pair would make the whole-pair kernel bound by the L2
// atomic rate. Peridynamics: NC = 3 components xx, xy, yy (a node pair's block is symmetric).
__device__ __forceinline__ long long to_fixed(float sc, float v, float& vmax) {
    vmax = fmaxf(vmax, fabsf(v));
    return __float2ll_rn(v * sc);
}

template <int NC>
__device__ __forceinline__ void accumulate_pair(const FastReq& Q, bool pilot, float sc, int64_t pi, int64_t p, int4 tk,
                                                int4 tl, const int* upos, float (&kk)[6][NC], float (&kl)[9][NC],
                                                float (&ll)[6][NC], float& vmax, int k, int l) {
    const int kn[3] = {tk.x, tk.y, tk.z}, ln[3] = {tl.x, tl.y, tl.z};
    if (Q.nmat) {  // label-dependent kernel: the pair's factor
        const float fm = Q.msc[Q.mat[k] * Q.nmat + Q.mat[l]];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
#pragma unroll
            for (int e = 0; e < 6; ++e) {
                kk[e][c] *= fm;
                ll[e][c] *= fm;
            }
#pragma unroll
            for (int e = 0; e < 9; ++e) kl[e][c] *= fm;
        }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int e = 0; e < 6; ++e) vmax = fmaxf(vmax, fmaxf(fabsf(kk[e][c]), fabsf(ll[e][c])));
    if (pilot) {
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int e = 0; e < 9; ++e) vmax = fmaxf(vmax, fabsf(kl[e][c]) * (kn[e / 3] == ln[e % 3] ? 2.f : 1.f));
        return;
    }
    float2* rl = reinterpret_cast<float2*>(Q.llrec + p * (6 * NC));
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int x = 0; x < 3; ++x) rl[3 * c + x] = make_float2(ll[2 * x][c], ll[2 * x + 1][c]);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const int i = kn[a], j = ln[b];
            const float f = i == j ? 2.f : 1.f;
            const int64_t u = upos ? (int64_t)upos[a * 3 + b]
                                   : Q.up_start[min(i, j)] + Q.klr[(int64_t)(a * 3 + b) * Q.npairs + pi];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const long long q = to_fixed(sc, f * kl[a * 3 + b][c], vmax);
                if (q) atomicAdd(Q.acc + u * NC + c, (unsigned long long)q);
            }
        }
}

// kk summed over the warp's pairs of each outer element present in the tile (pairs of one tile
// mostly share E_k): a masked xor butterfly, which leaves the same bits in every lane, then one
// fixed-point add per node pair of E_k. All 32 lanes call it; valid = the lane holds a pair.
// The sum of at most 32 values of one E_k stays within the bound the scale S assumes (every value
// counts among the terms added into that entry).
template <int NC>
__device__ __forceinline__ void accumulate_kk(const FastReq& Q, bool pilot, float sc, bool valid, int k,
                                              const float (&kk)[6][NC]) {
    if (pilot) return;
    const int lane = threadIdx.x & 31;
    unsigned todo = __ballot_sync(0xffffffffu, valid);
    while (todo) {
        const int src = __ffs(todo) - 1;
        const int kx = __shfl_sync(0xffffffffu, k, src);
        const bool mine = valid && k == kx;
        todo &= ~__ballot_sync(0xffffffffu, mine);
        float v[6][NC];
#pragma unroll
        for (int e = 0; e < 6; ++e)
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                float x = mine ? kk[e][c] : 0.f;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                v[e][c] = x;
            }
        // every lane holds the sums: lane e NC + c converts and adds value (e, c), so the 6 NC
        // float-to-int64 conversions (a 1/64-rate pipe) take one warp instruction
        float mv = 0.f;
#pragma unroll
        for (int e = 0; e < 6; ++e)
#pragma unroll
            for (int c = 0; c < NC; ++c)
                if (lane == e * NC + c) mv = v[e][c];
        if (lane < 6 * NC) {
            const int e = lane / NC, c = lane - e * NC;
            const long long q = __float2ll_rn(mv * sc);
            if (q) atomicAdd(Q.acc + (int64_t)Q.epos[(int64_t)kx * 8 + e] * NC + c, (unsigned long long)q);
        }
    }
}

__device__ __forceinline__ void flush_max(unsigned int* maxabs, float vmax) {
    for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    if ((threadIdx.x & 31) == 0 && vmax > 0.f) atomicMax(maxabs, __float_as_uint(vmax));
}

static constexpr int FAST_WARPS = FAST_THREADS / 32;

// tile t of a launch: its request (binary search over the requests' first tiles) and first
// list position
__device__ __forceinline__ int2 tile_of(const FastLaunch& L, int64_t t) {
    if (!L.reqs) return make_int2(0, (int)(t * 32));
    int lo = 0, hi = L.nreq - 1;  // the last request whose first tile is <= t
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (L.tile_off[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    return make_int2(lo, (int)((t - L.tile_off[lo]) * 32));
}

// the request of a tile into the warp's shared-memory copy (all lanes of the warp call it;
// the copy is reloaded only when the request changes)
__device__ __forceinline__ void load_req(FastReq& sq, int& cur, const FastReq* reqs, int r) {
    __syncwarp();
    constexpr int W = (int)(sizeof(FastReq) / sizeof(int));
    static_assert(sizeof(FastReq) % sizeof(int) == 0, "FastReq is copied in 4-byte words");
    const int* src = reinterpret_cast<const int*>(reqs + r);
    int* dst = reinterpret_cast<int*>(&sq);
    for (int w = threadIdx.x & 31; w < W; w += 32) dst[w] = src[w];
    __syncwarp();
    cur = r;
}

// FP32 decisions of one outer point, all evaluated (no early exit, so a warp stays
// converged). Same margins and outcomes as nl_decide32; ok = false where a decision is too
// close to call. For two crossings on one edge, both ends outside, the vertex of the
// quadratic t_c = -B/A must lie in (0, 1): tested as 0 < -B < A (no division). Where disc is
// decided positive and both ends are decided outside, t_c is bounded away from 0 and 1 by
// sqrt(floor2 / A), so the test cannot flip under rounding.
struct GeoF {
    float ta[3], tb[3];
    int nc[3];
    bool in[3];
};

// Edge vectors of E_l (u_e = v_{e+1} - v_e, from the FP32 edge vectors E = (v1 - v0, v2 - v0))
// with their squared lengths and 1-norms: the same for every outer point of a pair.
struct EdgesF {
    float ux[3], uy[3], A[3], n1[3];
};

__device__ __forceinline__ EdgesF edges_of(float4 El) {
    EdgesF g;
    g.ux[0] = El.x;
    g.uy[0] = El.y;
    g.ux[1] = El.z - El.x;
    g.uy[1] = El.w - El.y;
    g.ux[2] = -El.z;
    g.uy[2] = -El.w;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        g.A[e] = g.ux[e] * g.ux[e] + g.uy[e] * g.uy[e];
        g.n1[e] = fabsf(g.ux[e]) + fabsf(g.uy[e]);
    }
    return g;
}

// WARP: all 32 lanes call it (skip = the lane's result is not needed); when every lane's
// inner element is inside the ball the edge work is skipped for the whole warp
template <bool WARP = false>
__device__ __forceinline__ bool decide_flat(const float Rx[3], const float Ry[3], const float C[3], const EdgesF& E,
                                            float eps, float floor2, float d2, GeoF& g, bool skip = false) {
    bool ok = true;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        ok &= fabsf(C[m]) > floor2 + 2.f * (fabsf(Rx[m]) + fabsf(Ry[m])) * eps;
        g.in[m] = C[m] < 0.f;
    }
    if (WARP && __all_sync(0xffffffffu, skip || (g.in[0] && g.in[1] && g.in[2]))) {
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            g.nc[e] = 0;
            g.ta[e] = g.tb[e] = 0.f;
        }
        return ok;
    }
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        const int b = (e + 1) % 3;
        const float ux = E.ux[e], uy = E.uy[e];
        const float Aq = E.A[e];
        const float Bq = Rx[e] * ux + Ry[e] * uy;
        const float Cq = C[e];
        const float disc = Bq * Bq - Aq * Cq;
        const bool one = g.in[e] != g.in[b];
        const bool out2 = !g.in[e] && !g.in[b];
        const float e1n = fabsf(Rx[e]) + fabsf(Ry[e]), u1n = E.n1[e];
        const float bound = 2.f * fabsf(Bq) * (u1n + 2.f * e1n) * eps + Aq * (2.f * e1n * eps + 1e-6f * d2) +
                            fabsf(Cq) * 4.f * u1n * eps + 1e-6f * (Bq * Bq + fabsf(Aq * Cq));
        ok &= !(out2 && fabsf(disc) <= bound);
        // roots (-B -+ sqrt(disc)) / A: near a root at 0 the cancellation leaves an absolute error
        // of about eps |R| in the crossing point, the size of the coordinates' own error
        const float sq = sqrtf(fmaxf(disc, 0.f));
        const float iA = __fdividef(1.f, Aq);
        const float lo = (-Bq - sq) * iA, hi = (-Bq + sq) * iA;
        const bool two = out2 && disc > 0.f && Bq < 0.f && -Bq < Aq;
        g.nc[e] = one ? 1 : (two ? 2 : 0);
        g.ta[e] = (one && g.in[e]) ? hi : lo;
        g.tb[e] = hi;
    }
    return ok;
}

// Polygon points are stored as barycentric coordinates (b1, b2) of E_l (b0 = 1 - b1 - b2): the
// drain needs them for the basis values, the sub-triangle's area is |det E_l| times their own
// area, and positions relative to x_p (kernels other than the constant one) follow with two
// FMAs per coordinate.

// canonical FP64 clip of one outer point (near ties); the canonical routine carries the
// barycentric coordinates of its points in FP64, rounded once here. Out of line, so that its
// registers do not weigh on the common path.
__device__ __noinline__ int clip_canonical(const double2* __restrict__ X, int4 tk, int4 tl, double o0, double o1,
                                           double o2, double delta, double delta2, bool caps, float2* dst,
                                           int maxp) {
    const double2 Vk[3] = {X[tk.x], X[tk.y], X[tk.z]};
    const double2 Vl[3] = {X[tl.x], X[tl.y], X[tl.z]};
    const double2 xp = nl_map(Vk, o0, o1, o2);
    CPt poly[NLFEM_MAXPOLY];
    bool full;
    int n = nl_clip(Vl, xp, delta, delta2, caps, poly, full);
    if (full) {
        dst[0] = make_float2(0.f, 0.f);
        dst[FAST_THREADS] = make_float2(1.f, 0.f);
        dst[2 * FAST_THREADS] = make_float2(0.f, 1.f);
        return 3;
    }
    n = min(n, maxp);
    for (int m = 0; m < n; ++m) dst[m * FAST_THREADS] = make_float2((float)poly[m].b1, (float)poly[m].b2);
    return n;
}

// Phase A3 for the Euclidean ball: an outer point whose FP32 decisions were not all beyond their
// error bounds. With caps, or when every cut outer point takes the FP64 cut (geo64), the whole
// canonical cut. Without caps the vertices relative to x_p are formed in FP64 and rounded once to
// FP32, and each predicate whose margin exceeds its error bound (the bounds of nl_decide32, taken
// one predicate at a time) keeps the FP32 outcome, which is the canonical one; the others are
// taken with the canonical clip's FP64 expressions (nl_d2 and the per-edge quadratic of nl_clip,
// the same operations in the same order, so the same outcomes): the vertex tests near the
// circle, and the edges at such a vertex or near tangency, whose roots are snapped to the
// vertices as the canonical clip snaps them. The other edges keep FP32 crossings. Points merge
// where the canonical clip merges them: one vertex pushed twice in a row, or last and first the
// same vertex (a crossing never coincides with a vertex: its parameter is at least 1e-12 away).
// On grids with delta a multiple of h most such outer points have one vertex on the circle, so
// one vertex test and two edges run in FP64 instead of the whole canonical cut. One call site in
// the kernel for both cases, and the same arguments as the canonical cut.
// mode: 0 canonical without caps, 1 canonical with caps, 2 mixed (without caps)
__device__ __noinline__ int clip_job(const double2* __restrict__ X, int4 tk, int4 tl, double o0, double o1,
                                     double o2, double delta, double delta2, int mode, float2* dst, int maxp) {
    if (mode != 2) return clip_canonical(X, tk, tl, o0, o1, o2, delta, delta2, mode == 1, dst, maxp);
    const double2 Vl[3] = {X[tl.x], X[tl.y], X[tl.z]};
    // x_p as nl_map forms it; at a vertex of E_k (barycentrics 1, 0, 0 in some order) that sum is
    // the vertex itself (up to the sign of a zero coordinate, which no product, square or
    // comparison below can see)
    // (tested on the bit patterns, so that the test costs no FP64 instructions)
    const long long b0 = __double_as_longlong(o0), b1 = __double_as_longlong(o1), b2 = __double_as_longlong(o2);
    const long long one = 0x3FF0000000000000ll;
    double2 xp;
    if (b0 == one && b1 == 0 && b2 == 0) xp = X[tk.x];
    else if (b1 == one && b0 == 0 && b2 == 0) xp = X[tk.y];
    else if (b2 == one && b0 == 0 && b1 == 0) xp = X[tk.z];
    else {
        const double2 Vk[3] = {X[tk.x], X[tk.y], X[tk.z]};
        xp = nl_map(Vk, o0, o1, o2);
    }
    float Rx[3], Ry[3], C[3];
    bool dec[3], ins[3];
    float rmax = 0.f;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        Rx[m] = (float)(Vl[m].x - xp.x);
        Ry[m] = (float)(Vl[m].y - xp.y);
        rmax = fmaxf(rmax, fmaxf(fabsf(Rx[m]), fabsf(Ry[m])));
    }
    // each component is the FP64 difference rounded once: within 2^-24 of its value, plus the
    // FP64 rounding of x_p and of the difference (far below); 2^-23 of the largest covers both
    const float eps = 1.2e-7f * rmax;
    const float d2 = (float)delta2, floor2 = 1e-5f * d2;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        C[m] = Rx[m] * Rx[m] + Ry[m] * Ry[m] - d2;
        dec[m] = fabsf(C[m]) > floor2 + 2.f * (fabsf(Rx[m]) + fabsf(Ry[m])) * eps;
        ins[m] = dec[m] ? C[m] < 0.f : nl_d2(Vl[m], xp) <= delta2;
    }
    if (ins[0] && ins[1] && ins[2]) {
        dst[0] = make_float2(0.f, 0.f);
        dst[FAST_THREADS] = make_float2(1.f, 0.f);
        dst[2 * FAST_THREADS] = make_float2(0.f, 1.f);
        return 3;
    }
    const float vb1[3] = {0.f, 1.f, 0.f}, vb2[3] = {0.f, 0.f, 1.f};
    int n = 0, last = -2, first = -2;  // kind of a point: its vertex index, or -1 for a crossing
    auto put = [&](int kind, float b1, float b2) {
        if (kind >= 0 && kind == last) return;
        if (n < maxp) dst[n * FAST_THREADS] = make_float2(b1, b2);
        if (n == 0) first = kind;
        last = kind;
        ++n;
    };
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        const int b = (e + 1) % 3;
        const float d1 = vb1[b] - vb1[e], d2e = vb2[b] - vb2[e];
        if (ins[e]) put(e, vb1[e], vb2[e]);
        const bool one = ins[e] != ins[b], out2 = !ins[e] && !ins[b];
        // the FP32 quadratic of the edge, as nl_decide32 forms it (u from the relative vertices)
        const float ux = Rx[b] - Rx[e], uy = Ry[b] - Ry[e];
        const float Aq = ux * ux + uy * uy;
        const float Bq = Rx[e] * ux + Ry[e] * uy;
        const float Cq = C[e];
        const float disc = Bq * Bq - Aq * Cq;
        bool f32 = dec[e] && dec[b];
        if (f32 && out2) {
            const float e1n = fabsf(Rx[e]) + fabsf(Ry[e]), u1n = fabsf(ux) + fabsf(uy);
            const float bound = 2.f * fabsf(Bq) * (u1n + 2.f * e1n) * eps + Aq * (2.f * e1n * eps + 1e-6f * d2) +
                                fabsf(Cq) * 4.f * u1n * eps + 1e-6f * (Bq * Bq + fabsf(Aq * Cq));
            f32 = fabsf(disc) > bound;
        }
        if (f32) {
            // the roots as decide_flat forms them (the vertex of the quadratic in (0, 1) tested as
            // 0 < -B < A)
            const float sq = sqrtf(fmaxf(disc, 0.f));
            const float iA = __fdividef(1.f, Aq);
            const float lo = (-Bq - sq) * iA, hi = (-Bq + sq) * iA;
            if (one) {
                const float t = ins[e] ? hi : lo;
                put(-1, fmaf(t, d1, vb1[e]), fmaf(t, d2e, vb2[e]));
            } else if (out2 && disc > 0.f && Bq < 0.f && -Bq < Aq) {
                put(-1, fmaf(lo, d1, vb1[e]), fmaf(lo, d2e, vb2[e]));
                put(-1, fmaf(hi, d1, vb1[e]), fmaf(hi, d2e, vb2[e]));
            }
        } else {
            const double2 A_ = Vl[e], B_ = Vl[b];
            const double uxd = __dsub_rn(B_.x, A_.x), uyd = __dsub_rn(B_.y, A_.y);
            const double ex = __dsub_rn(A_.x, xp.x), ey = __dsub_rn(A_.y, xp.y);
            const double A = __dadd_rn(__dmul_rn(uxd, uxd), __dmul_rn(uyd, uyd));
            const double B = __dadd_rn(__dmul_rn(ex, uxd), __dmul_rn(ey, uyd));
            const double Cd = __dsub_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), delta2);
            const double dd = __dsub_rn(__dmul_rn(B, B), __dmul_rn(A, Cd));
            if (dd > 0.0) {
                const double r = __dsqrt_rn(dd);
                const double ts[2] = {__ddiv_rn(__dsub_rn(-B, r), A), __ddiv_rn(__dadd_rn(-B, r), A)};
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const double t = ts[j];
                    if (!(t > 0.0 && t < 1.0)) continue;
                    if (t < NLFEM_TAU) {
                        put(e, vb1[e], vb2[e]);
                    } else if (t > 1.0 - NLFEM_TAU) {
                        put(b, vb1[b], vb2[b]);
                    } else {  // a crossing: its position rounded to FP32
                        const float tf = (float)t;
                        const float c1 = (e == 1 ? 1.f - tf : 0.f) + (b == 1 ? tf : 0.f);
                        const float c2 = (e == 2 ? 1.f - tf : 0.f) + (b == 2 ? tf : 0.f);
                        put(-1, c1, c2);
                    }
                }
            }
        }
    }
    if (n >= 2 && last >= 0 && last == first) --n;
    return n < 3 ? 0 : min(n, maxp);
}

// Infinity ball: the canonical FP64 cut of one outer point, its points mapped to barycentric
// coordinates of E_l in FP64 and rounded once
__device__ __noinline__ int clip_square_f32(const double2* __restrict__ X, int4 tk, int4 tl, double o0, double o1,
                                            double o2, double delta, float2* dst) {
    const double2 Vk[3] = {X[tk.x], X[tk.y], X[tk.z]};
    const double2 Vl[3] = {X[tl.x], X[tl.y], X[tl.z]};
    const double2 xp = nl_map(Vk, o0, o1, o2);
    double2 rel[NLFEM_MAXSQ];
    bool full;
    const int n = nl_clip_square_rel(Vl, xp, delta, rel, full);
    const double e1x = Vl[1].x - Vl[0].x, e1y = Vl[1].y - Vl[0].y, e2x = Vl[2].x - Vl[0].x, e2y = Vl[2].y - Vl[0].y;
    const double ij = 1.0 / (e1x * e2y - e1y * e2x);
    const double ox = xp.x - Vl[0].x, oy = xp.y - Vl[0].y;  // x_p - v0_l
    for (int m = 0; m < n && m < 7; ++m) {
        const double px = rel[m].x + ox, py = rel[m].y + oy;
        dst[m * FAST_THREADS] = make_float2((float)((px * e2y - py * e2x) * ij), (float)((e1x * py - e1y * px) * ij));
    }
    return n < 7 ? n : 7;
}

// Infinity ball in FP32 with exact decisions: the canonical Sutherland-Hodgman passes
// (x <= d, y <= d, x >= -d, y >= -d) on FP32 points that carry a bound e on the absolute
// difference of both coordinates from the canonical FP64 values. An inside test is taken only
// if its margin exceeds that bound (plus the rounding of delta and of the test itself), so
// every decision equals the canonical one; with all decisions strict no two points coincide,
// which is checked as well (two points closer than their bounds: undecided). Returns the
// number of polygon points written to dst (0 = empty), or -1 when some decision is too close
// to call (the caller then takes the canonical FP64 cut).
__device__ __forceinline__ int sh_pass32(const float* ix, const float* iy, const float* ie, int n, int a, float s,
                                         float d, float* ox, float* oy, float* oe, bool& ok, bool exact) {
    if (n == 0) return 0;
    int m = 0;
    float Sx = ix[n - 1], Sy = iy[n - 1], Se = ie[n - 1];
    float Sa = a ? Sy : Sx;
    float mS = s * Sa - d;  // > 0: outside
    if (exact) ok &= fabsf(mS) > Se + 2.4e-7f * (d + fabsf(Sa));
    bool s_in = mS <= 0.f;
    for (int i = 0; i < n; ++i) {
        const float Ex = ix[i], Ey = iy[i], Ee = ie[i];
        const float Ea = a ? Ey : Ex;
        const float mE = s * Ea - d;
        if (exact) ok &= fabsf(mE) > Ee + 2.4e-7f * (d + fabsf(Ea));
        const bool e_in = mE <= 0.f;
        if (e_in != s_in) {
            const float Sb = a ? Sx : Sy, Eb = a ? Ex : Ey;
            const float num = s * d - Sa, den = Ea - Sa;
            const float t = num / den;
            const float db = Eb - Sb;
            const float xb = fmaf(t, db, Sb);
            // error: the ends' bounds, the slope times the error of t, the roundings
            const float et = (Se + 1.2e-7f * (d + fabsf(Sa)) + t * (Se + Ee + 1.2e-7f * fabsf(den))) / fabsf(den) +
                             2.4e-7f * t;
            const float eb = Se + t * (Se + Ee) + et * fabsf(db) + 2.4e-7f * (fabsf(Sb) + fabsf(db));
            const float e = fmaxf(eb, 1.2e-7f * d) * 1.5f;
            if (m < 8) {
                ox[m] = a ? xb : s * d;
                oy[m] = a ? s * d : xb;
                oe[m] = e;
            }
            ++m;
        }
        if (e_in) {
            if (m < 8) {
                ox[m] = Ex;
                oy[m] = Ey;
                oe[m] = Ee;
            }
            ++m;
        }
        Sx = Ex; Sy = Ey; Se = Ee; Sa = Ea; s_in = e_in;
    }
    return m < 8 ? m : 8;
}

// exact = false: the FP32 passes alone (a decision within rounding of a side may differ from the
// FP64 one, which moves that polygon edge by a rounding-sized sliver); -1 only when more than 7
// points come out
// (the polygon is written as barycentric coordinates of E_l: El its edge vectors, idet the
// inverse of their determinant; Rx[0], Ry[0] is v0_l relative to x_p)
__device__ __noinline__ int clip_square_fast(const float Rx[3], const float Ry[3], float eps, float d, float2* dst,
                                             bool exact, float4 El, float idet) {
    float Ax[8], Ay[8], Ae[8], Bx[8], By[8], Be[8];
    for (int v = 0; v < 3; ++v) {
        Ax[v] = Rx[v];
        Ay[v] = Ry[v];
        Ae[v] = eps;
    }
    bool ok = true;
    int n = sh_pass32(Ax, Ay, Ae, 3, 0, 1.f, d, Bx, By, Be, ok, exact);
    n = sh_pass32(Bx, By, Be, n, 1, 1.f, d, Ax, Ay, Ae, ok, exact);
    n = sh_pass32(Ax, Ay, Ae, n, 0, -1.f, d, Bx, By, Be, ok, exact);
    n = sh_pass32(Bx, By, Be, n, 1, -1.f, d, Ax, Ay, Ae, ok, exact);
    if (!ok || n > 7) return -1;
    if (exact)
        for (int i = 0; i < n; ++i) {  // no two consecutive points may coincide (all decisions strict)
            const int j = i + 1 < n ? i + 1 : 0;
            if (n > 1 && fabsf(Ax[i] - Ax[j]) + fabsf(Ay[i] - Ay[j]) <= 2.f * (Ae[i] + Ae[j])) return -1;
        }
    if (n < 3) return 0;
    for (int i = 0; i < n; ++i) {
        const float rx = Ax[i] - Rx[0], ry = Ay[i] - Ry[0];
        dst[i * FAST_THREADS] = make_float2((rx * El.w - ry * El.z) * idet, (El.x * ry - El.y * rx) * idet);
    }
    return n;
}

// Cut pairs: the outer points are processed in chunks of at most CHUNK (8; 7 with caps, whose
// polygons need 9 slots per outer point). Phase A1 decides, in lockstep across the warp, every
// outer point of the chunk whose inner element is whole (every vertex inside the ball) or empty
// (every vertex outside and, for the Euclidean ball, the point of each edge closest to x_p
// outside that edge: then no edge reaches the ball), each test taken only beyond its FP32 error
// bound. The other outer points are cut, not all lanes have one, so they go to a per-warp job
// list: phase A2 cuts them one per lane and round, writing the polygon into the owner's slots,
// and jobs whose decisions are too close to call go to a second list for phase A3, which takes
// the undecided predicates with the canonical FP64 expressions (cut_mixed; the infinity ball and
// geo64, where every cut outer point goes there, take the whole canonical cut). Polygon points are
// barycentric coordinates of E_l; 4 bits per outer point record their number. Phase B drains
// the fan triangles: each iteration integrates one triangle per lane, walking through the lane's
// outer points in order, and applies that triangle's inner sums with its outer point's factors.
// The cut list is ordered by fan-triangle count (order_cut_pairs), so the lanes of a warp drain
// about the same number of triangles.
template <int BALL>
struct CutShape {
    static constexpr bool CAPS = BALL == NLFEM_BALL_APPROXCAPS;
    static constexpr bool SQUARE = BALL == NLFEM_BALL_INFINITY;
    // polygon points: 6 raw plus up to 3 cap centres; a triangle cut by a square: at most 7
    static constexpr int MAXP = CAPS ? 9 : (SQUARE ? 7 : 6);
    // With caps the polygons need 9 slots per outer point, and the job lists' shared memory would
    // cost the block its third slot per SM: caps cut every outer point in lockstep (chunks of 8),
    // the others use the job lists (chunks of 7, the 7-point rule in one chunk, four blocks per SM
    // without caps)
    static constexpr bool JOBS = !CAPS;
    static constexpr int CHUNK = CAPS ? 8 : 7;
};

// Phase A2 for the Euclidean ball: the cut of one outer point from its relative coordinates,
// written as barycentric coordinates to dst (stride FAST_THREADS). Returns the number of points,
// or -1 if a decision is too close to call (the canonical FP64 cut then takes it).
// whole: every vertex inside the ball (valid when the result is not -1)
template <bool CAPS>
__device__ __forceinline__ int cut_euclid(const float Rx[3], const float Ry[3], const EdgesF& Ed, float4 El,
                                          float idet, float eps, float floor2, float d2, float delta, float2* dst,
                                          bool& whole) {
    constexpr int MAXP = CAPS ? 9 : 6;
    float Cc[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) Cc[m] = Rx[m] * Rx[m] + Ry[m] * Ry[m] - d2;
    GeoF G;
    bool ok = decide_flat(Rx, Ry, Cc, Ed, eps, floor2, d2, G);
    whole = G.in[0] && G.in[1] && G.in[2];
    // barycentric coordinates of the vertices: v0 (0, 0), v1 (1, 0), v2 (0, 1); edge e runs from
    // vertex e to vertex e + 1
    const float vb1[3] = {0.f, 1.f, 0.f}, vb2[3] = {0.f, 0.f, 1.f};
    int n = 0;
    auto put = [&](int slot, float b1, float b2) { dst[min(slot, MAXP - 1) * FAST_THREADS] = make_float2(b1, b2); };
    if (!CAPS) {
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            const int b = (e + 1) % 3;
            const float d1 = vb1[b] - vb1[e], d2e = vb2[b] - vb2[e];
            if (G.in[e]) put(n, vb1[e], vb2[e]);
            n += G.in[e];
            if (G.nc[e] >= 1) put(n, fmaf(G.ta[e], d1, vb1[e]), fmaf(G.ta[e], d2e, vb2[e]));
            n += G.nc[e] >= 1;
            if (G.nc[e] >= 2) put(n, fmaf(G.tb[e], d1, vb1[e]), fmaf(G.tb[e], d2e, vb2[e]));
            n += G.nc[e] >= 2;
        }
    } else if (ok) {
        // with caps: a cap centre between consecutive points not joined along an edge; the cap
        // logic runs on positions relative to x_p, the cap centre's barycentric coordinates come
        // from E_l's inverse map
        int nraw = 0, fe = 0, fv = 0, le = 0;
        float fx = 0, fy = 0, lx = 0, ly = 0;
        auto cap = [&](float px, float py, float qx, float qy) {
            const float cx = qx - px, cy = qy - py;
            const float len = sqrtf(cx * cx + cy * cy);
            ok &= len > 1e-6f * delta;
            const float sc = __fdividef(delta, len);
            const float rx = sc * cy - Rx[0], ry = -sc * cx - Ry[0];  // cap centre - v0_l
            put(n, (rx * El.w - ry * El.z) * idet, (El.x * ry - El.y * rx) * idet);
            ++n;
        };
        auto raw = [&](float x, float y, float b1, float b2, int e, int v) {
            if (nraw >= 1 && !((e == le) || (v && e == (le + 1) % 3))) cap(lx, ly, x, y);
            put(n, b1, b2);
            ++n;
            if (nraw == 0) { fx = x; fy = y; fe = e; fv = v; }
            lx = x; ly = y; le = e;
            ++nraw;
        };
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            const int b = (e + 1) % 3;
            const float ux = Ed.ux[e], uy = Ed.uy[e];
            const float d1 = vb1[b] - vb1[e], d2e = vb2[b] - vb2[e];
            if (G.in[e]) raw(Rx[e], Ry[e], vb1[e], vb2[e], e, 1);
            if (G.nc[e] >= 1)
                raw(fmaf(G.ta[e], ux, Rx[e]), fmaf(G.ta[e], uy, Ry[e]), fmaf(G.ta[e], d1, vb1[e]),
                    fmaf(G.ta[e], d2e, vb2[e]), e, 0);
            if (G.nc[e] >= 2)
                raw(fmaf(G.tb[e], ux, Rx[e]), fmaf(G.tb[e], uy, Ry[e]), fmaf(G.tb[e], d1, vb1[e]),
                    fmaf(G.tb[e], d2e, vb2[e]), e, 0);
        }
        if (!(G.in[0] && G.in[1] && G.in[2]) && nraw >= 2 && !(fv && fe == (le + 1) % 3)) cap(lx, ly, fx, fy);
    }
    if (!ok) return -1;
    return n < 3 ? 0 : n;
}

template <int KER, int NQI, int BALL, bool BATCH>
__global__ void __launch_bounds__(FAST_THREADS, 4) k_trunc_cut(const __grid_constant__ FastRule R,
                                                           const __grid_constant__ FastLaunch L) {
    constexpr int NC = (KER == NLFEM_KERNEL_PERIDYNAMIC) ? 3 : 1;
    constexpr bool CAPS = CutShape<BALL>::CAPS;
    constexpr bool SQUARE = CutShape<BALL>::SQUARE;
    constexpr int MAXP = CutShape<BALL>::MAXP;
    constexpr int CHUNK = CutShape<BALL>::CHUNK;
    constexpr bool JOBS = CutShape<BALL>::JOBS;
    extern __shared__ float2 s_pts[];   // [CHUNK][MAXP][FAST_THREADS] barycentric coordinates
    float2* my = s_pts + threadIdx.x;
    __shared__ FastReq sq[BATCH ? FAST_WARPS : 1];
    // per lane: its pair's elements and v0_l - v0_k with the error bound of the relative
    // coordinates (for the jobs other lanes run on its behalf); per warp: the job lists of the
    // FP32 cuts and of the canonical cuts (owner lane << 3 | outer point), the jobs' point counts
    constexpr int NJ = JOBS ? FAST_THREADS : 1;
    __shared__ int s_k[NJ], s_l[NJ];
    __shared__ float4 s_pd[NJ], s_ek[NJ], s_el[NJ];
    __shared__ unsigned char s_job[JOBS ? FAST_WARPS * 32 * CHUNK : 1], s_job64[JOBS ? FAST_WARPS * 32 * CHUNK : 1];
    __shared__ unsigned char s_cnt[JOBS ? FAST_THREADS * CHUNK : 1];
    __shared__ float4 s_orule[16];  // outer rule (l0, l1, l2, w)
    for (int i = threadIdx.x; i < 16; i += blockDim.x)
        s_orule[i] = make_float4(R.ol[i][0], R.ol[i][1], R.ol[i][2], R.ow[i]);
    __syncthreads();
    const int nqo = R.nqo;
    const bool pilot = L.pilot > 0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wbase = warp * 32;
    const unsigned lanes_below = (1u << lane) - 1u;
    int cur = -1;
    float vmax = 0.f;            // largest |value| of this warp's pairs of request cur
    unsigned int* vdst = nullptr;
    for (int64_t t = (int64_t)blockIdx.x * FAST_WARPS + warp; t < L.ntiles; t += (int64_t)gridDim.x * FAST_WARPS) {
        const int2 tile = tile_of(L, t);
        if (BATCH && tile.x != cur) {  // warp-uniform
            if (vdst) flush_max(vdst, vmax);
            vmax = 0.f;
            load_req(sq[warp], cur, L.reqs, tile.x);
        }
        const FastReq& Q = BATCH ? sq[warp] : L.one;
        vdst = Q.maxabs;
        const float sc = pilot ? 1.f : *Q.scale_p;
        const int64_t pi = (int64_t)tile.y + lane;
        const int64_t nlist = pilot ? (Q.npairs + L.pilot - 1) / L.pilot : Q.npairs;
        const bool valid = pi < nlist;
        const int64_t p = valid ? (int64_t)Q.ids[pilot ? pi * L.pilot : pi] : 0;
        int4 tk = make_int4(0, 0, 0, 0), tl = make_int4(0, 0, 0, 0);
        float4 Ek = make_float4(0, 0, 0, 0), El = make_float4(1, 0, 0, 1);
        float dk = 0.f, dx = 0.f, dy = 0.f;
        int k = 0, l = 0;
        if (valid) {
            k = Q.pk[p];
            l = Q.pl[p];
            if (!pilot)  // the kl ranks are read after the quadrature: bring their lines into L2 now
#pragma unroll
                for (int e = 0; e < 9; ++e)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(Q.klr + (int64_t)e * Q.npairs + pi));
            const ElemRec rk = Q.rec[k], rl = Q.rec[l];
            tk = make_int4(rk.n0, rk.n1, rk.n2, 0);
            tl = make_int4(rl.n0, rl.n1, rl.n2, 0);
            dx = (float)(rl.v0.x - rk.v0.x);
            dy = (float)(rl.v0.y - rk.v0.y);
            Ek = rk.E;
            El = rl.E;
            dk = rk.det;
        }
        const float dl = fabsf(El.x * El.w - El.y * El.z);  // |det E_l|: sub-triangle area factor
        const float W0x = dx, W0y = dy;
        const float W1x = dx + El.x, W1y = dy + El.y, W2x = dx + El.z, W2y = dy + El.w;
        const float span = fabsf(dx) + fabsf(dy) + fabsf(Ek.x) + fabsf(Ek.y) + fabsf(Ek.z) + fabsf(Ek.w) +
                           fabsf(El.x) + fabsf(El.y) + fabsf(El.z) + fabsf(El.w);
        const float eps = 4.8e-7f * span;    // bound on the FP32 error of the relative coordinates
        const float floor2 = 1e-5f * Q.d2;   // floor of the vertex margin (see nl_decide32)
        if (JOBS) {
            s_k[threadIdx.x] = k;
            s_l[threadIdx.x] = l;
            s_pd[threadIdx.x] = make_float4(W0x, W0y, eps, 0.f);
            s_ek[threadIdx.x] = Ek;
            s_el[threadIdx.x] = El;
        }
        const EdgesF Ed = edges_of(El);  // caps: the lockstep cut's edge data
        // Euclidean ball: squared edge lengths of E_l (the closest-point test of phase A1)
        const float A0 = El.x * El.x + El.y * El.y;
        const float A1 = (El.z - El.x) * (El.z - El.x) + (El.w - El.y) * (El.w - El.y);
        const float A2 = El.z * El.z + El.w * El.w;

        float kk[6][NC], kl[9][NC], ll[6][NC];
#pragma unroll
        for (int i = 0; i < 6; ++i)
#pragma unroll
            for (int c = 0; c < NC; ++c) kk[i][c] = ll[i][c] = 0.f;
#pragma unroll
        for (int i = 0; i < 9; ++i)
#pragma unroll
            for (int c = 0; c < NC; ++c) kl[i][c] = 0.f;

        // outer points per chunk: the launch shape the autotuner picked (the drain walks a lane's
        // outer points in the same order whatever the chunk, so the sums are the same bits)
        const int ck = (L.chunk > 0 && L.chunk < CHUNK) ? L.chunk : CHUNK;
#pragma unroll 1
        for (int qb = 0; qb < nqo; qb += ck) {
            const int qn = min(ck, nqo - qb);
            // ---- phase A1: whole and empty outer points in lockstep, the others become jobs
            unsigned long long counts = 0;  // 4 bits per outer point: number of polygon points
            unsigned need = 0;              // outer points to cut (jobs)
#pragma unroll 1
            for (int q = 0; q < qn; ++q) {
                const int q0 = qb + q;
                const float Xx = R.ol[q0][1] * Ek.x + R.ol[q0][2] * Ek.z;  // x_p - v0_k
                const float Xy = R.ol[q0][1] * Ek.y + R.ol[q0][2] * Ek.w;
                const float Rx[3] = {W0x - Xx, W1x - Xx, W2x - Xx}, Ry[3] = {W0y - Xy, W1y - Xy, W2y - Xy};
                if (!JOBS) {
                    // caps: the cut of every outer point in lockstep, the canonical FP64 cut in place
                    // for an undecided one (and with geo64 for every cut one)
                    int n = 0;
                    if (valid) {
                        const float idet = 1.f / (El.x * El.w - El.y * El.z);
                        bool wh = false;
                        n = cut_euclid<CAPS>(Rx, Ry, Ed, El, idet, eps, floor2, Q.d2, Q.delta,
                                             my + q * MAXP * FAST_THREADS, wh);
                        if (n < 0 || (Q.geo64 && n >= 3 && !wh))
                            n = clip_canonical(Q.X, tk, tl, R.ro[q0][0], R.ro[q0][1], R.ro[q0][2], Q.delta64,
                                               Q.delta2_64, CAPS, my + q * MAXP * FAST_THREADS, MAXP);
                    }
                    counts |= (unsigned long long)(n < 3 ? 0 : n) << (4 * q);
                    continue;
                }
                bool whole, empty;
                if (SQUARE) {
                    // vertex tests against the square's sides; the constant kernel decides in FP32
                    // without margins (its result depends on the cut region only, which the
                    // square cut moves continuously), the others only beyond the error bound
                    const bool exact = KER != NLFEM_KERNEL_CONSTANT || Q.geo64;
                    const float mg = exact ? eps + 1e-6f * Q.delta : 0.f;
                    const float lo = Q.delta - mg, hi = Q.delta + mg;
                    bool allin = true;
                    int oxp = 0, oxm = 0, oyp = 0, oym = 0;
#pragma unroll
                    for (int m = 0; m < 3; ++m) {
                        allin &= fabsf(Rx[m]) <= lo && fabsf(Ry[m]) <= lo;
                        oxp += Rx[m] > hi;
                        oxm += Rx[m] < -hi;
                        oyp += Ry[m] > hi;
                        oym += Ry[m] < -hi;
                    }
                    whole = allin;
                    empty = oxp == 3 || oxm == 3 || oyp == 3 || oym == 3;
                } else {
                    // every vertex decided inside: the whole element; every vertex decided outside
                    // and, on every edge, the point closest to x_p (parameter -B/A) outside the
                    // edge: the distance along each edge grows from its outside ends, so no edge
                    // reaches the ball (a sign of B within rounding cannot matter: the vertex margin
                    // exceeds B^2 / A there)
                    bool okv = true, in0, in1, in2;
                    float Cc[3];
#pragma unroll
                    for (int m = 0; m < 3; ++m) {
                        Cc[m] = Rx[m] * Rx[m] + Ry[m] * Ry[m] - Q.d2;
                        okv &= fabsf(Cc[m]) > floor2 + 2.f * (fabsf(Rx[m]) + fabsf(Ry[m])) * eps;
                    }
                    in0 = Cc[0] < 0.f;
                    in1 = Cc[1] < 0.f;
                    in2 = Cc[2] < 0.f;
                    const float B0 = Rx[0] * El.x + Ry[0] * El.y;
                    const float B1 = Rx[1] * (El.z - El.x) + Ry[1] * (El.w - El.y);
                    const float B2 = -(Rx[2] * El.z + Ry[2] * El.w);
                    const bool apart = !(B0 < 0.f && -B0 < A0) && !(B1 < 0.f && -B1 < A1) && !(B2 < 0.f && -B2 < A2);
                    whole = okv && in0 && in1 && in2;
                    empty = okv && !in0 && !in1 && !in2 && apart;
                }
                int n = 0;
                if (valid && whole) {
                    my[(q * MAXP + 0) * FAST_THREADS] = make_float2(0.f, 0.f);
                    my[(q * MAXP + 1) * FAST_THREADS] = make_float2(1.f, 0.f);
                    my[(q * MAXP + 2) * FAST_THREADS] = make_float2(0.f, 1.f);
                    n = 3;
                } else if (valid && !empty) {
                    need |= 1u << q;
                }
                counts |= (unsigned long long)n << (4 * q);
            }
            if (JOBS && __any_sync(0xffffffffu, need != 0)) {
                // the jobs of the chunk, outer point by outer point and in lane order within one: job j
                // of the warp is (owner lane, outer point). A round of 32 jobs then mostly holds distinct
                // owners, whose polygon slots lie in distinct shared-memory banks.
                int total = 0;
#pragma unroll 1
                for (int q = 0; q < qn; ++q) {
                    const unsigned m = __ballot_sync(0xffffffffu, (need >> q) & 1u);
                    if ((need >> q) & 1u) s_job[wbase * CHUNK + total + __popc(m & lanes_below)] =
                        (unsigned char)((lane << 3) | q);
                    total += __popc(m);
                }
                __syncwarp();
                // ---- phase A2: one cut per lane and round in FP32; undecided ones to the FP64 list
                int n64 = 0;
#pragma unroll 1
                for (int jb = 0; jb < total; jb += 32) {
                    const int jj = jb + lane;
                    const bool act = jj < total;
                    const int code = act ? s_job[wbase * CHUNK + jj] : 0;
                    const int owner = code >> 3, q = code & 7, q0 = qb + q;
                    int n = 0;
                    bool und = false;
                    if (act) {
                        const float4 pd = s_pd[wbase + owner];
                        const float4 Ejk = s_ek[wbase + owner], Ejl = s_el[wbase + owner];
                        const float4 orule = s_orule[q0];
                        const float Xx = orule.y * Ejk.x + orule.z * Ejk.z;
                        const float Xy = orule.y * Ejk.y + orule.z * Ejk.w;
                        const float Rx[3] = {pd.x - Xx, pd.x + Ejl.x - Xx, pd.x + Ejl.z - Xx};
                        const float Ry[3] = {pd.y - Xy, pd.y + Ejl.y - Xy, pd.y + Ejl.w - Xy};
                        const float ijd = 1.f / (Ejl.x * Ejl.w - Ejl.y * Ejl.z);
                        float2* dst = s_pts + wbase + owner + q * MAXP * FAST_THREADS;
                        if (Q.geo64) {
                            und = true;
                        } else if (SQUARE) {
                            n = clip_square_fast(Rx, Ry, pd.z, Q.delta, dst, KER != NLFEM_KERNEL_CONSTANT, Ejl, ijd);
                            und = n < 0;
                        } else {
                            bool wh = false;
                            n = cut_euclid<CAPS>(Rx, Ry, edges_of(Ejl), Ejl, ijd, pd.z, floor2, Q.d2, Q.delta, dst, wh);
                            und = n < 0;
                        }
                    }
                    const unsigned um = __ballot_sync(0xffffffffu, und);
                    if (und) s_job64[wbase * CHUNK + n64 + __popc(um & lanes_below)] = (unsigned char)code;
                    n64 += __popc(um);
                    if (act) s_cnt[(wbase + owner) * CHUNK + q] = (unsigned char)(und || n < 3 ? 0 : n);
                }
                __syncwarp();
                // ---- phase A3: the undecided predicates in FP64 (or the canonical cut), one job per lane
                for (int jj = lane; jj < n64; jj += 32) {
                    const int code = s_job64[wbase * CHUNK + jj];
                    const int owner = code >> 3, q = code & 7, q0 = qb + q;
                    float2* dst = s_pts + wbase + owner + q * MAXP * FAST_THREADS;
                    const int4 tkj = Q.T[s_k[wbase + owner]], tlj = Q.T[s_l[wbase + owner]];
                    const int n = SQUARE ? clip_square_f32(Q.X, tkj, tlj, R.ro[q0][0], R.ro[q0][1], R.ro[q0][2],
                                                           Q.delta64, dst)
                                         : clip_job(Q.X, tkj, tlj, R.ro[q0][0], R.ro[q0][1], R.ro[q0][2],
                                                    Q.delta64, Q.delta2_64, CAPS ? 1 : (Q.geo64 ? 0 : 2), dst, MAXP);
                    s_cnt[(wbase + owner) * CHUNK + q] = (unsigned char)(n < 3 ? 0 : n);
                }
                __syncwarp();
                for (unsigned b = need; b; b &= b - 1) {
                    const int q = __ffs(b) - 1;
                    counts |= (unsigned long long)s_cnt[threadIdx.x * CHUNK + q] << (4 * q);
                }
                __syncwarp();
            }
            // ---- phase B: one fan triangle per lane and iteration
            int qc = 0, sc = 2;
            while (qc < qn && ((counts >> (4 * qc)) & 15) == 0) ++qc;
            while (__any_sync(0xffffffffu, qc < qn)) {
                if (qc < qn) {
                    const int q0 = qb + qc;
                    // lanes sit at different outer points here: the rule comes from shared memory
                    // (a parameter-space read at per-lane indices would serialise)
                    const float4 orule = s_orule[q0];
                    float b1[3], b2[3], px[3], py[3];
                    const int slot[3] = {0, sc - 1, sc};
#pragma unroll
                    for (int t = 0; t < 3; ++t) {
                        const float2 pt = my[(qc * MAXP + slot[t]) * FAST_THREADS];
                        b1[t] = pt.x;
                        b2[t] = pt.y;
                    }
                    // the triangle's area: |det E_l| times its area in barycentric coordinates
                    const float dT = dl * fabsf((b1[1] - b1[0]) * (b2[2] - b2[0]) - (b2[1] - b2[0]) * (b1[2] - b1[0]));
                    if (KER != NLFEM_KERNEL_CONSTANT) {
                        // positions relative to x_p: v0_l - x_p + b1 (v1_l - v0_l) + b2 (v2_l - v0_l)
                        const float R0x = W0x - (orule.y * Ek.x + orule.z * Ek.z);
                        const float R0y = W0y - (orule.y * Ek.y + orule.z * Ek.w);
#pragma unroll
                        for (int t = 0; t < 3; ++t) {
                            px[t] = fmaf(b2[t], El.z, fmaf(b1[t], El.x, R0x));
                            py[t] = fmaf(b2[t], El.w, fmaf(b1[t], El.y, R0y));
                        }
                    } else {
#pragma unroll
                        for (int t = 0; t < 3; ++t) px[t] = py[t] = 0.f;
                    }
                    Inner<NC> I;
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        I.g[c] = 0.f;
#pragma unroll
                        for (int j = 0; j < 3; ++j) I.h[j][c] = 0.f;
#pragma unroll
                        for (int j = 0; j < 6; ++j) I.m[j][c] = 0.f;
                    }
                    tri_quad<KER, NQI, NC>(R, Q, I, dT, px[0], py[0], b1[0], b2[0], px[1], py[1], b1[1], b2[1], px[2],
                                           py[2], b1[2], b2[2]);
                    outer_update<NC>(orule, dk, I, kk, kl, ll);
                    if (++sc >= (int)((counts >> (4 * qc)) & 15)) {
                        sc = 2;
                        ++qc;
                        while (qc < qn && ((counts >> (4 * qc)) & 15) == 0) ++qc;
                    }
                }
            }
        }
        if (valid) accumulate_pair<NC>(Q, pilot, sc, pi, p, tk, tl, nullptr, kk, kl, ll, vmax, k, l);
        accumulate_kk<NC>(Q, pilot, sc, valid, k, kk);
    }
    if (vdst) flush_max(vdst, vmax);
}

// Fan triangles of a cut pair summed over its outer points, from the same FP32 decisions
// (an undecided outer point counts its FP32 outcome; the count only orders the work).
__global__ void k_cut_tris(FastRule R, FastReq Q, int* __restrict__ key) {
    const int64_t pi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pi >= Q.npairs) return;
    const int64_t p = Q.ids[pi];
    const int k = Q.pk[p], l = Q.pl[p];
    const int4 tk = Q.T[k], tl = Q.T[l];
    const double2 v0k = Q.X[tk.x], v0l = Q.X[tl.x];
    const float dx = (float)(v0l.x - v0k.x), dy = (float)(v0l.y - v0k.y);
    const float4 Ek = Q.E32[k], El = Q.E32[l];
    const float Wx[3] = {dx, dx + El.x, dx + El.z}, Wy[3] = {dy, dy + El.y, dy + El.w};
    const int nqo = R.nqo;
    int tris = 0;
    if (Q.ball == NLFEM_BALL_INFINITY) {  // the square cut's triangle count (ordering only)
        const double2 Vk[3] = {v0k, Q.X[tk.y], Q.X[tk.z]}, Vl[3] = {v0l, Q.X[tl.y], Q.X[tl.z]};
        for (int q0 = 0; q0 < nqo; ++q0) {
            const double2 xp = nl_map(Vk, R.ro[q0][0], R.ro[q0][1], R.ro[q0][2]);
            bool full;
            const int n = nl_clip_square(Vl, xp, Q.delta64, nullptr, full);
            tris += n >= 3 ? n - 2 : 0;
        }
        key[pi] = tris;
        return;
    }
    // an outer point farther than delta + r_l from E_l's centroid (with a margin of 1e-4) sees no
    // point of E_l: no triangles, without deciding anything (r_l from the vertices in FP32)
    const float gx = (Wx[0] + Wx[1] + Wx[2]) * (1.f / 3.f), gy = (Wy[0] + Wy[1] + Wy[2]) * (1.f / 3.f);
    float rl2 = 0.f;
    for (int m = 0; m < 3; ++m) rl2 = fmaxf(rl2, (Wx[m] - gx) * (Wx[m] - gx) + (Wy[m] - gy) * (Wy[m] - gy));
    const float reach = (Q.delta + sqrtf(rl2)) * (1.f + 1e-4f);
    for (int q0 = 0; q0 < nqo; ++q0) {
        const float Xx = R.ol[q0][1] * Ek.x + R.ol[q0][2] * Ek.z;
        const float Xy = R.ol[q0][1] * Ek.y + R.ol[q0][2] * Ek.w;
        if ((gx - Xx) * (gx - Xx) + (gy - Xy) * (gy - Xy) > reach * reach) continue;
        float Rx[3], Ry[3], Cc[3];
        for (int m = 0; m < 3; ++m) {
            Rx[m] = Wx[m] - Xx;
            Ry[m] = Wy[m] - Xy;
            Cc[m] = Rx[m] * Rx[m] + Ry[m] * Ry[m] - Q.d2;
        }
        GeoF G;
        decide_flat(Rx, Ry, Cc, edges_of(El), 0.f, 0.f, Q.d2, G);
        int n = 0;
        for (int e = 0; e < 3; ++e) n += (int)G.in[e] + G.nc[e];
        if (Q.ball == NLFEM_BALL_APPROXCAPS && n >= 2 && !(G.in[0] && G.in[1] && G.in[2])) n += 1;  // a cap
        tris += n >= 3 ? n - 2 : 0;
    }
    key[pi] = tris;
}

// sort key within a window of the cut list: fan triangles, then the position in the window
__global__ void k_window_key(int* key, int64_t n, int wbits) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) key[i] = (key[i] << wbits) | (int)(i & ((1 << wbits) - 1));
}

__global__ void k_window_ptr(int64_t* ptr, int64_t nwin, int64_t n, int w) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= nwin) ptr[i] = i * w < n ? i * w : n;
}

// Pairs with E_l inside the ball of every point of E_k: the whole inner element at every
// outer point, no geometry at all.
// Scalar kernels with the 7-point inner rule run at 64 registers, 8 blocks per SM: the kernel
// waits on the dependent loads that start each pair, and 32 warps per SM hide them better than
// 24 at 80 registers without spills (a few spilled words; 720k: 5.14 -> 4.80 ms, A/B in one run).
template <int KER, int NQI, bool BATCH>
__global__ void __launch_bounds__(FAST_THREADS, (KER != NLFEM_KERNEL_PERIDYNAMIC && !BATCH && NQI == 7) ? 8 : 1)
    k_trunc_whole(const __grid_constant__ FastRule R, const __grid_constant__ FastLaunch L) {
    constexpr int NC = (KER == NLFEM_KERNEL_PERIDYNAMIC) ? 3 : 1;
    __shared__ FastReq sq[BATCH ? FAST_WARPS : 1];
    const int nqo = R.nqo;
    const bool pilot = L.pilot > 0;
    const int warp = threadIdx.x >> 5;
    int cur = -1;
    float vmax = 0.f;            // largest |value| of this warp's pairs of request cur
    unsigned int* vdst = nullptr;
    for (int64_t t = (int64_t)blockIdx.x * FAST_WARPS + warp; t < L.ntiles; t += (int64_t)gridDim.x * FAST_WARPS) {
        const int2 tile = tile_of(L, t);
        if (BATCH && tile.x != cur) {  // warp-uniform
            if (vdst) flush_max(vdst, vmax);
            vmax = 0.f;
            load_req(sq[warp], cur, L.reqs, tile.x);
        }
        const FastReq& Q = BATCH ? sq[warp] : L.one;
        vdst = Q.maxabs;
        const float sc = pilot ? 1.f : *Q.scale_p;
        const int64_t pi = (int64_t)tile.y + (threadIdx.x & 31);
        const int64_t nlist = pilot ? (Q.npairs + L.pilot - 1) / L.pilot : Q.npairs;
        const bool valid = pi < nlist;
        float kk[6][NC];
        int k = 0;
        if (valid) {
            const int64_t li = pilot ? pi * L.pilot : pi;
            const int64_t p = Q.ids[li];
            const int2 kl2 = Q.lkl[li];
            k = kl2.x;
            const int l = kl2.y;
            const ElemRec rk = Q.rec[k], rl = Q.rec[l];
            const int4 tk = make_int4(rk.n0, rk.n1, rk.n2, 0), tl = make_int4(rl.n0, rl.n1, rl.n2, 0);
            const float dx = (float)(rl.v0.x - rk.v0.x), dy = (float)(rl.v0.y - rk.v0.y);
            const float4 Ek = rk.E, El = rl.E;
            const float dk = rk.det;
            // the upper entries of the nine kl node pairs, loaded now so that their latency
            // hides behind the quadrature
            int upos[9];
            if (!pilot) {
                const int kn[3] = {rk.n0, rk.n1, rk.n2}, ln[3] = {rl.n0, rl.n1, rl.n2};
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int b = 0; b < 3; ++b)
                        upos[a * 3 + b] = (int)(Q.up_start[min(kn[a], ln[b])] +
                                                Q.klr[(int64_t)(a * 3 + b) * Q.npairs + pi]);
            }
            float kl[9][NC], ll[6][NC];
#pragma unroll
            for (int i = 0; i < 6; ++i)
#pragma unroll
                for (int c = 0; c < NC; ++c) kk[i][c] = ll[i][c] = 0.f;
#pragma unroll
            for (int i = 0; i < 9; ++i)
#pragma unroll
                for (int c = 0; c < NC; ++c) kl[i][c] = 0.f;
            for (int q0 = 0; q0 < nqo; ++q0) {
                const float Xx = R.ol[q0][1] * Ek.x + R.ol[q0][2] * Ek.z;
                const float Xy = R.ol[q0][1] * Ek.y + R.ol[q0][2] * Ek.w;
                Inner<NC> I;
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    I.g[c] = 0.f;
#pragma unroll
                    for (int j = 0; j < 3; ++j) I.h[j][c] = 0.f;
#pragma unroll
                    for (int j = 0; j < 6; ++j) I.m[j][c] = 0.f;
                }
                const float ax = dx - Xx, ay = dy - Xy, bx = dx + El.x - Xx, by = dy + El.y - Xy;
                const float cx = dx + El.z - Xx, cy = dy + El.w - Xy;
                const float dT = fabsf((bx - ax) * (cy - ay) - (by - ay) * (cx - ax));
                tri_quad<KER, NQI, NC>(R, Q, I, dT, ax, ay, 0.f, 0.f, bx, by, 1.f, 0.f, cx, cy, 0.f, 1.f);
                outer_update<NC>(make_float4(R.ol[q0][0], R.ol[q0][1], R.ol[q0][2], R.ow[q0]), dk, I, kk, kl, ll);
            }
            accumulate_pair<NC>(Q, pilot, sc, pi, p, tk, tl, upos, kk, kl, ll, vmax, k, l);
        }
        accumulate_kk<NC>(Q, pilot, sc, valid, k, kk);
    }
    if (vdst) flush_max(vdst, vmax);
}

static FastRule make_rule(const Params& prm) {
    FastRule r;
    for (int i = 0; i < 16; ++i) {
        for (int j = 0; j < 3; ++j) {
            r.ol[i][j] = i < prm.ro.n ? (float)prm.ro.l[i][j] : 0.f;
            r.il[i][j] = i < prm.ri.n ? (float)prm.ri.l[i][j] : 0.f;
            r.ro[i][j] = i < prm.ro.n ? prm.ro.l[i][j] : 0.0;
        }
        r.ow[i] = i < prm.ro.n ? (float)prm.ro.w[i] : 0.f;
        r.iw[i] = i < prm.ri.n ? (float)prm.ri.w[i] : 0.f;
    }
    r.nqo = prm.ro.n;
    return r;
}

// the request of one (mesh, parameters) for a work list (0: whole pairs, 1: cut pairs)
FastReq make_req(Mesh& m, PairCache& pc, const Params& prm, int list) {
    FastReq q;
    std::memset(&q, 0, sizeof q);
    q.pk = pc.pk.p; q.pl = pc.pl.p; q.pcls = pc.pcls.p;
    q.ids = list == 0 ? pc.whole_ids.p : pc.cut_ids.p;
    q.npairs = list == 0 ? pc.nwhole : pc.ncut;
    q.klr = list == 0 ? pc.klr_whole.p : pc.klr_cut.p;
    q.lkl = list == 0 ? pc.kl_whole.p : nullptr;
    q.X = m.X.p; q.T = m.T.p; q.E32 = m.E32.p; q.det32 = m.det32.p; q.rec = m.rec.p;
    q.delta = (float)prm.delta;
    q.d2 = (float)prm.delta * (float)prm.delta;
    q.c = (float)prm.c;
    q.s = (float)prm.s;
    q.delta64 = prm.delta;
    q.delta2_64 = prm.delta2;
    q.ball = prm.ball;
    q.geo64 = prm.geo64;
    q.nmat = prm.nmat;
    q.mat = prm.mat;
    q.msc = prm.msc32;
    q.ntab = prm.ntab;
    q.tinv = (float)prm.tinv;
    q.tab = prm.tab32;
    q.up_start = pc.up_start.p;
    q.epos = pc.epos.p;
    q.scale_p = nullptr;
    return q;
}

// Reorder of the cut list by fan-triangle count within windows of FAST_THREADS consecutive
// pairs, one block's share of a grid-stride step (pattern time): the lanes of a warp then
// drain similar work, and a warp's pairs still share their outer element, so their
// accumulator entries stay in L2.
void order_cut_pairs(Mesh& m, PairCache& pc, const Params& prm, cudaStream_t st) {
    const int64_t n = pc.ncut;
    if (n < 2) return;
    constexpr int WBITS = 7, W = 1 << WBITS;
    static_assert(W == FAST_THREADS, "sort windows are the blocks' pair ranges");
    const FastRule r = make_rule(prm);
    const FastReq q = make_req(m, pc, prm, 1);
    DBuf<int> key;
    key.alloc(n, st);
    k_cut_tris<<<nblk(n, 256), 256, 0, st>>>(r, q, key.p);
    NLFEM_LAUNCH_CHECK();
    k_window_key<<<nblk(n, 256), 256, 0, st>>>(key.p, n, WBITS);
    NLFEM_LAUNCH_CHECK();
    const int64_t nwin = (n + W - 1) / W;
    DBuf<int64_t> ptr;
    ptr.alloc(nwin + 1, st);
    k_window_ptr<<<nblk(nwin + 1, 256), 256, 0, st>>>(ptr.p, nwin, n, W);
    NLFEM_LAUNCH_CHECK();
    segmented_sort_i32(key.p, pc.cut_ids.p, ptr.p, nwin, (int)std::min<int64_t>(n, W), st);
}

template <int BALL>
static constexpr size_t cut_smem() {
    return sizeof(float2) * CutShape<BALL>::CHUNK * FAST_THREADS * CutShape<BALL>::MAXP;
}

template <int KER, int NQI, int BALL, bool BATCH>
static void launch_cut(const FastRule& r, const FastLaunch& L, unsigned grid, cudaStream_t st) {
    k_trunc_cut<KER, NQI, BALL, BATCH><<<grid, FAST_THREADS, cut_smem<BALL>(), st>>>(r, L);
}

template <int KER, int NQI, int BALL, bool BATCH>
static void cut_attr() {
    NLFEM_CUDA_TRY(cudaFuncSetAttribute(k_trunc_cut<KER, NQI, BALL, BATCH>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cut_smem<BALL>()));
}

template <int KER, int NQI>
static void cut_attrs() {
    cut_attr<KER, NQI, NLFEM_BALL_NOCAPS, false>();
    cut_attr<KER, NQI, NLFEM_BALL_APPROXCAPS, false>();
    cut_attr<KER, NQI, NLFEM_BALL_INFINITY, false>();
    cut_attr<KER, NQI, NLFEM_BALL_NOCAPS, true>();
    cut_attr<KER, NQI, NLFEM_BALL_APPROXCAPS, true>();
    cut_attr<KER, NQI, NLFEM_BALL_INFINITY, true>();
}

// cudaFuncSetAttribute is not a stream operation: done once per device, outside any capture
void set_fast_attributes() {
    static std::mutex mu;
    static std::vector<int> done;
    int dev = 0;
    NLFEM_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> g(mu);
    if (std::find(done.begin(), done.end(), dev) != done.end()) return;
    cut_attrs<NLFEM_KERNEL_CONSTANT, 7>();
    cut_attrs<NLFEM_KERNEL_CONSTANT, 16>();
    cut_attrs<NLFEM_KERNEL_FRACTIONAL, 7>();
    cut_attrs<NLFEM_KERNEL_FRACTIONAL, 16>();
    cut_attrs<NLFEM_KERNEL_PERIDYNAMIC, 7>();
    cut_attrs<NLFEM_KERNEL_PERIDYNAMIC, 16>();
    cut_attrs<NLFEM_KERNEL_TABULATED, 7>();
    cut_attrs<NLFEM_KERNEL_TABULATED, 16>();
    done.push_back(dev);
}

template <int KER, int NQI, bool BATCH>
static void launch_class(int list, int ball, const FastRule& r, const FastLaunch& L, unsigned grid,
                         cudaStream_t st) {
    if (list == 0) k_trunc_whole<KER, NQI, BATCH><<<grid, FAST_THREADS, 0, st>>>(r, L);
    else if (ball == NLFEM_BALL_APPROXCAPS) launch_cut<KER, NQI, NLFEM_BALL_APPROXCAPS, BATCH>(r, L, grid, st);
    else if (ball == NLFEM_BALL_INFINITY) launch_cut<KER, NQI, NLFEM_BALL_INFINITY, BATCH>(r, L, grid, st);
    else launch_cut<KER, NQI, NLFEM_BALL_NOCAPS, BATCH>(r, L, grid, st);
}

template <bool BATCH>
static void launch_kernel(const Params& prm, int list, const FastRule& r, const FastLaunch& L, unsigned grid,
                          cudaStream_t st) {
    const int ball = prm.ball;
    if (prm.kernel == NLFEM_KERNEL_CONSTANT) {
        if (prm.ri.n == 7) launch_class<NLFEM_KERNEL_CONSTANT, 7, BATCH>(list, ball, r, L, grid, st);
        else launch_class<NLFEM_KERNEL_CONSTANT, 16, BATCH>(list, ball, r, L, grid, st);
    } else if (prm.kernel == NLFEM_KERNEL_FRACTIONAL) {
        if (prm.ri.n == 7) launch_class<NLFEM_KERNEL_FRACTIONAL, 7, BATCH>(list, ball, r, L, grid, st);
        else launch_class<NLFEM_KERNEL_FRACTIONAL, 16, BATCH>(list, ball, r, L, grid, st);
    } else if (prm.kernel == NLFEM_KERNEL_TABULATED) {
        if (prm.ri.n == 7) launch_class<NLFEM_KERNEL_TABULATED, 7, BATCH>(list, ball, r, L, grid, st);
        else launch_class<NLFEM_KERNEL_TABULATED, 16, BATCH>(list, ball, r, L, grid, st);
    } else {
        if (prm.ri.n == 7) launch_class<NLFEM_KERNEL_PERIDYNAMIC, 7, BATCH>(list, ball, r, L, grid, st);
        else launch_class<NLFEM_KERNEL_PERIDYNAMIC, 16, BATCH>(list, ball, r, L, grid, st);
    }
    NLFEM_LAUNCH_CHECK();
}

// one launch of the whole-pair (list 0) or cut-pair (list 1) kernel over the tiles of L:
// a request table (L.reqs, L.tile_off) or the single request L.one
// ---- grid size of the bulk launches (the tile shape the autotuner picks) -------------------
static int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        NLFEM_CUDA_TRY(cudaGetDevice(&dev));
        NLFEM_CUDA_TRY(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
    }
    return n;
}

// Launch shape per kernel class and list: resident blocks per SM (grid size) and, for the
// cut-pair kernel, outer points per chunk
struct TuneEntry {
    int64_t key;
    int bps, chunk;
};
static std::mutex g_tune_mu;
static std::vector<TuneEntry> g_tune;

int64_t fast_tune_key(const Params& prm, int list) {
    return ((((int64_t)prm.kernel * 64 + prm.ro.n) * 64 + prm.ri.n) * 4 + prm.ball) * 2 + list;
}

int fast_blocks_per_sm(int64_t key) {
    std::lock_guard<std::mutex> g(g_tune_mu);
    for (auto& e : g_tune)
        if (e.key == key) return e.bps;
    return 64;  // untuned: oversubscribe; warps take 32-pair tiles in a grid-stride loop
}

int fast_chunk(int64_t key) {
    std::lock_guard<std::mutex> g(g_tune_mu);
    for (auto& e : g_tune)
        if (e.key == key) return e.chunk;
    return 0;  // untuned: the full chunk
}

void set_fast_shape(int64_t key, int bps, int chunk) {
    std::lock_guard<std::mutex> g(g_tune_mu);
    for (auto& e : g_tune)
        if (e.key == key) {
            e.bps = bps;
            e.chunk = chunk;
            return;
        }
    g_tune.push_back(TuneEntry{key, bps, chunk});
}

void set_fast_blocks_per_sm(int64_t key, int bps) { set_fast_shape(key, bps, fast_chunk(key)); }

int fast_max_chunk(const Params& prm) {
    return prm.ball == NLFEM_BALL_APPROXCAPS ? CutShape<NLFEM_BALL_APPROXCAPS>::CHUNK
                                             : CutShape<NLFEM_BALL_NOCAPS>::CHUNK;
}

void launch_fast_list(const Params& prm, int list, const FastLaunch& L0, cudaStream_t st) {
    set_fast_attributes();
    const int64_t key = fast_tune_key(prm, list);
    const int64_t cap = (int64_t)sm_count() * fast_blocks_per_sm(key);
    const unsigned grid = (unsigned)std::min<int64_t>((L0.ntiles + FAST_WARPS - 1) / FAST_WARPS, cap);
    if (!grid) return;
    FastLaunch L = L0;
    L.chunk = fast_chunk(key);
    const FastRule r = make_rule(prm);
    if (L.reqs) launch_kernel<true>(prm, list, r, L, grid, st);
    else launch_kernel<false>(prm, list, r, L, grid, st);
}

// One launch of list `list` (0 whole, 1 cut) over the pairs of several requests of one kernel
// class (the rules and kernel type of prm; per-request delta, constants and buffers in the
// table).
struct FusedLaunch {
    Params prm;
    int list = 0;
    FastLaunch L;
    DBuf<FastReq> reqs;
    DBuf<int64_t> off;
};

std::shared_ptr<FusedLaunch> make_fused(const std::vector<BulkItem>& items, int list, int pilot, cudaStream_t st) {
    auto f = std::make_shared<FusedLaunch>();
    const int n = (int)items.size();
    f->prm = items[0].prm;
    f->list = list;
    std::memset(&f->L, 0, sizeof f->L);
    std::vector<FastReq> reqs;
    std::vector<int64_t> off(n + 1, 0);
    for (int i = 0; i < n; ++i) {
        const BulkItem& it = items[i];
        FastReq q = make_req(*it.m, *it.pc, it.prm, list);
        q.acc = it.b.acc;
        q.llrec = it.b.llrec;
        q.scale_p = it.b.scale_p;
        q.maxabs = it.b.maxabs;
        reqs.push_back(q);
        const int64_t np = pilot ? (q.npairs + pilot - 1) / pilot : q.npairs;
        off[i + 1] = off[i] + (np + 31) / 32;
    }
    f->reqs.alloc(n, st);
    f->off.alloc(n + 1, st);
    // copies from pageable host memory are staged before cudaMemcpyAsync returns
    NLFEM_CUDA_TRY(cudaMemcpyAsync(f->reqs.p, reqs.data(), sizeof(FastReq) * n, cudaMemcpyHostToDevice, st));
    NLFEM_CUDA_TRY(cudaMemcpyAsync(f->off.p, off.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, st));
    f->L.reqs = f->reqs.p;
    f->L.tile_off = f->off.p;
    f->L.nreq = n;
    f->L.ntiles = off[n];
    f->L.pilot = pilot;
    return f;
}

void run_fused(const FusedLaunch& f, cudaStream_t st) {
    if (f.L.ntiles > 0) launch_fast_list(f.prm, f.list, f.L, st);
}

void launch_trunc_fast(Mesh& m, PairCache& pc, const Params& prm, const BulkAcc& b, cudaStream_t st,
                       cudaEvent_t* ev) {
    FastReq q[2];
    for (int list = 0; list < 2; ++list) {
        q[list] = make_req(m, pc, prm, list);
        q[list].acc = b.acc;
        q[list].llrec = b.llrec;
        q[list].scale_p = b.scale_p;
        q[list].maxabs = b.maxabs;
    }
    const int pilot = b.pstride > 1 ? (int)b.pstride : 0;
    for (int list = 0; list < 2; ++list) {
        if (ev) NLFEM_CUDA_TRY(cudaEventRecord(ev[list], st));  // ev[0..2] bracket the two launches
        const int64_t n = pilot ? (q[list].npairs + pilot - 1) / pilot : q[list].npairs;
        FastLaunch L;
        L.reqs = nullptr;
        L.tile_off = nullptr;
        L.nreq = 1;
        L.ntiles = (n + 31) / 32;
        L.pilot = pilot;
        L.one = q[list];
        launch_fast_list(prm, list, L, st);
    }
    if (ev) NLFEM_CUDA_TRY(cudaEventRecord(ev[2], st));
}

}  // namespace nlfem
