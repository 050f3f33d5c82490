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

#include "nlfem_internal.cuh"

namespace nlfem {

static inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

static constexpr int FAST_THREADS = 128;

struct FastArgs {
    const int* pk;
    const int* pl;
    const int8_t* pcls;
    const int* ids;   // the pairs to process
    int64_t npairs;   // number of ids
    const double2* X;
    const int4* T;
    const float4* E32;
    const float* det32;
    Params prm;
    float ol[16][3], ow[16];  // outer rule in FP32
    float il[16][3], iw[16];  // inner rule in FP32
    float delta, d2, c, s;
    int caps;
    // fixed-point accumulation into the upper CSR entries (see accumulate_pair)
    unsigned long long* acc;  // [n_upper][NC] int64 two's complement sums; nullptr: pilot (max only)
    float* kkll;              // [2][P][6 NC] kk, then ll, of every pair, by pair id
    int64_t npairs_all;       // P
    const int64_t* up_start;  // [M + 1] first upper entry of each node row
    const int* epos;          // [K][6] upper entries of an element's node pairs (kkI order)
    const uint16_t* klr;      // [9][npairs] rank of the kl node pair in its upper row, list order
    float scale;              // 2^S
    unsigned int* maxabs;     // bits of the largest |value| seen (a positive float), atomicMax
    int64_t pstride;          // pair i of this launch is ids[i * pstride] (pilot samples)
};

template <int NC>
struct Inner {
    float g[NC], h[3][NC], m[6][NC];
};

// the inner rule on triangle (a, b, c): positions relative to x_p, barycentric (b1, b2) w.r.t. E_l
template <int KER, int NQI, int NC>
__device__ __forceinline__ void tri_quad(const FastArgs& A, Inner<NC>& I, float ax, float ay, float a1, float a2,
                                         float bx, float by, float b1, float b2, float cx, float cy, float c1,
                                         float c2) {
    const float dT = fabsf((bx - ax) * (cy - ay) - (by - ay) * (cx - ax));
    const float a0 = 1.f - a1 - a2, b0 = 1.f - b1 - b2, c0 = 1.f - c1 - c2;
#pragma unroll
    for (int q = 0; q < NQI; ++q) {
        const float l0 = A.il[q][0], l1 = A.il[q][1], l2 = A.il[q][2];
        const float zx = l0 * ax + l1 * bx + l2 * cx;
        const float zy = l0 * ay + l1 * by + l2 * cy;
        const float Q0 = l0 * a0 + l1 * b0 + l2 * c0;
        const float Q1 = l0 * a1 + l1 * b1 + l2 * c1;
        const float Q2 = l0 * a2 + l1 * b2 + l2 * c2;
        const float wq = A.iw[q] * dT;
        float wc[NC];
        if (KER == NLFEM_KERNEL_CONSTANT) {
            wc[0] = wq * A.c;
        } else if (KER == NLFEM_KERNEL_FRACTIONAL) {
            const float r2 = zx * zx + zy * zy;
            if (A.s == 0.5f) {
                const float r = rsqrtf(r2);
                wc[0] = wq * A.c * r * r * r;
            } else {
                wc[0] = wq * A.c * exp2f(log2f(r2) * (-1.f - A.s));
            }
        } else {
            const float r2 = zx * zx + zy * zy;
            const float r = rsqrtf(r2);
            const float sc = wq * A.c * r * r * r;
            wc[0] = sc * zx * zx;
            wc[1 % NC] = sc * zx * zy;
            wc[2 % NC] = sc * zy * zy;
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const float w = wc[c];
            I.g[c] += w;
            const float w0 = w * Q0, w1 = w * Q1, w2 = w * Q2;
            I.h[0][c] += w0;
            I.h[1][c] += w1;
            I.h[2][c] += w2;
            I.m[0][c] += w0 * Q0;
            I.m[1][c] += w0 * Q1;
            I.m[2][c] += w0 * Q2;
            I.m[3][c] += w1 * Q1;
            I.m[4][c] += w1 * Q2;
            I.m[5][c] += w2 * Q2;
        }
    }
}

// kk += a_p g P P^T, kl -= a_p P h^T, ll += a_p m for outer point q0 (P = its barycentrics)
template <int NC>
__device__ __forceinline__ void outer_update(const FastArgs& A, int q0, float dk, const Inner<NC>& I,
                                             float (&kk)[6][NC], float (&kl)[9][NC], float (&ll)[6][NC]) {
    const float ap = A.ow[q0] * dk;
    const float Pa[3] = {A.ol[q0][0], A.ol[q0][1], A.ol[q0][2]};
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

// Accumulation of a pair's block [[kk, kl], [kl^T, ll]].
// kk and ll only involve the nodes of one element: they are written to the pair's record
// (kk of pair p at kkll[p], ll at kkll[P + p], 6 values per component) and summed per
// element later in a fixed order
// (k_elem_sums). kl[a][b] belongs to the node pair (k_a, l_b); it is rounded once to a signed
// 64-bit fixed-point number v * 2^S and added to that upper CSR entry with an integer atomic
// (counted twice when the two nodes coincide: both mirrored entries of the symmetric block
// are diagonal). Integer addition is associative, so the sums are the same bits in every
// run whatever order the pairs are processed in. Peridynamics: NC = 3 components xx, xy, yy
// (the block of a node pair is symmetric).
__device__ __forceinline__ long long to_fixed(const FastArgs& A, float v, float& vmax) {
    vmax = fmaxf(vmax, fabsf(v));
    return __float2ll_rn(v * A.scale);
}

template <int NC>
__device__ __forceinline__ void accumulate_pair(const FastArgs& A, int64_t pi, int64_t p, int4 tk, int4 tl,
                                                const float (&kk)[6][NC], const float (&kl)[9][NC],
                                                const float (&ll)[6][NC], float& vmax) {
    const int kn[3] = {tk.x, tk.y, tk.z}, ln[3] = {tl.x, tl.y, tl.z};
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int e = 0; e < 6; ++e) vmax = fmaxf(vmax, fmaxf(fabsf(kk[e][c]), fabsf(ll[e][c])));
    if (!A.acc) {  // pilot
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int e = 0; e < 9; ++e) vmax = fmaxf(vmax, fabsf(kl[e][c]) * (kn[e / 3] == ln[e % 3] ? 2.f : 1.f));
        return;
    }
    float2* rk = reinterpret_cast<float2*>(A.kkll + p * (6 * NC));
    float2* rl = reinterpret_cast<float2*>(A.kkll + (A.npairs_all + p) * (6 * NC));
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int x = 0; x < 3; ++x) {
            rk[3 * c + x] = make_float2(kk[2 * x][c], kk[2 * x + 1][c]);
            rl[3 * c + x] = make_float2(ll[2 * x][c], ll[2 * x + 1][c]);
        }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const int i = kn[a], j = ln[b];
            const float f = i == j ? 2.f : 1.f;
            const int64_t u = A.up_start[min(i, j)] + A.klr[(int64_t)(a * 3 + b) * A.npairs + pi];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const long long q = to_fixed(A, f * kl[a * 3 + b][c], vmax);
                if (q) atomicAdd(A.acc + u * NC + c, (unsigned long long)q);
            }
        }
}

__device__ __forceinline__ void flush_max(const FastArgs& A, float vmax) {
    for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    if ((threadIdx.x & 31) == 0 && vmax > 0.f) atomicMax(A.maxabs, __float_as_uint(vmax));
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

__device__ __forceinline__ bool decide_flat(const float Rx[3], const float Ry[3], const float C[3], float eps,
                                            float floor2, float d2, GeoF& g) {
    bool ok = true;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        ok &= fabsf(C[m]) > floor2 + 2.f * (fabsf(Rx[m]) + fabsf(Ry[m])) * eps;
        g.in[m] = C[m] < 0.f;
    }
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        const int b = (e + 1) % 3;
        const float ux = Rx[b] - Rx[e], uy = Ry[b] - Ry[e];
        const float Aq = ux * ux + uy * uy;
        const float Bq = Rx[e] * ux + Ry[e] * uy;
        const float Cq = C[e];
        const float disc = Bq * Bq - Aq * Cq;
        const bool one = g.in[e] != g.in[b];
        const bool out2 = !g.in[e] && !g.in[b];
        const float e1n = fabsf(Rx[e]) + fabsf(Ry[e]), u1n = fabsf(ux) + fabsf(uy);
        const float bound = 2.f * fabsf(Bq) * (u1n + 2.f * e1n) * eps + Aq * (2.f * e1n * eps + 1e-6f * d2) +
                            fabsf(Cq) * 4.f * u1n * eps + 1e-6f * (Bq * Bq + fabsf(Aq * Cq));
        ok &= !(out2 && fabsf(disc) <= bound);
        // stable roots; qq != 0 whenever a crossing exists (disc > 0)
        const float sq = sqrtf(fmaxf(disc, 0.f));
        const float qq = -(Bq + copysignf(sq, Bq));
        const float r1 = __fdividef(qq, Aq), r2 = __fdividef(Cq, qq);
        const float lo = fminf(r1, r2), hi = fmaxf(r1, r2);
        const bool two = out2 && disc > 0.f && Bq < 0.f && -Bq < Aq;
        g.nc[e] = one ? 1 : (two ? 2 : 0);
        g.ta[e] = (one && g.in[e]) ? hi : lo;
        g.tb[e] = hi;
    }
    return ok;
}

// canonical FP64 clip of one outer point (near ties), written relative to x_p; kept out of
// line so that its registers do not weigh on the common path
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
        for (int m = 0; m < 3; ++m)
            dst[m * FAST_THREADS] = make_float2((float)(Vl[m].x - xp.x), (float)(Vl[m].y - xp.y));
        return 3;
    }
    n = min(n, maxp);
    for (int m = 0; m < n; ++m)
        dst[m * FAST_THREADS] = make_float2((float)(poly[m].x - xp.x), (float)(poly[m].y - xp.y));
    return n;
}

// Cut pairs: the outer points are processed in chunks of CHUNK. Phase A sets up every
// outer point of the chunk in lockstep across the warp (decisions, polygon points relative
// to x_p into shared memory; 4 bits per outer point record the number of points). Phase B
// drains the fan triangles: each iteration integrates one triangle per lane, walking
// through the lane's outer points in order, and applies that triangle's inner sums with its
// outer point's factors. Barycentric coordinates are recomputed from positions with E_l's
// inverse map. The cut list is ordered by fan-triangle count (order_cut_pairs), so the
// lanes of a warp drain about the same number of triangles.
static constexpr int CHUNK = 8;

template <int KER, int NQI, bool CAPS>
__global__ void __launch_bounds__(FAST_THREADS) k_trunc_cut(FastArgs A) {
    constexpr int NC = (KER == NLFEM_KERNEL_PERIDYNAMIC) ? 3 : 1;
    constexpr int MAXP = CAPS ? 9 : 6;  // polygon points: 6 raw, plus up to 3 cap centres
    extern __shared__ float2 s_pts[];   // [CHUNK][MAXP][FAST_THREADS]
    float2* my = s_pts + threadIdx.x;
    auto put = [&](int q, int slot, float x, float y) { my[(q * MAXP + slot) * FAST_THREADS] = make_float2(x, y); };
    const Params& P = A.prm;
    const int nqo = P.ro.n;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    float vmax = 0.f;
    for (int64_t p0 = (int64_t)blockIdx.x * blockDim.x; p0 < A.npairs; p0 += stride) {
        const int64_t pi = p0 + threadIdx.x;
        const bool valid = pi < A.npairs;
        const int64_t p = valid ? (int64_t)A.ids[pi * A.pstride] : 0;
        int4 tk = make_int4(0, 0, 0, 0), tl = make_int4(0, 0, 0, 0);
        float4 Ek = make_float4(0, 0, 0, 0), El = make_float4(1, 0, 0, 1);
        float dk = 0.f, dx = 0.f, dy = 0.f;
        int k = 0, l = 0;
        if (valid) {
            k = A.pk[p];
            l = A.pl[p];
            tk = A.T[k];
            tl = A.T[l];
            const double2 v0k = A.X[tk.x], v0l = A.X[tl.x];
            dx = (float)(v0l.x - v0k.x);
            dy = (float)(v0l.y - v0k.y);
            Ek = A.E32[k];
            El = A.E32[l];
            dk = A.det32[k];
        }
        const float idet = 1.f / (El.x * El.w - El.y * El.z);
        const float W0x = dx, W0y = dy;
        const float W1x = dx + El.x, W1y = dy + El.y, W2x = dx + El.z, W2y = dy + El.w;
        const float span = fabsf(dx) + fabsf(dy) + fabsf(Ek.x) + fabsf(Ek.y) + fabsf(Ek.z) + fabsf(Ek.w) +
                           fabsf(El.x) + fabsf(El.y) + fabsf(El.z) + fabsf(El.w);
        const float eps = 4.8e-7f * span;    // bound on the FP32 error of the relative coordinates
        const float floor2 = 1e-5f * A.d2;   // floor of the vertex margin (see nl_decide32)

        float kk[6][NC], kl[9][NC], ll[6][NC];
#pragma unroll
        for (int i = 0; i < 6; ++i)
#pragma unroll
            for (int c = 0; c < NC; ++c) kk[i][c] = ll[i][c] = 0.f;
#pragma unroll
        for (int i = 0; i < 9; ++i)
#pragma unroll
            for (int c = 0; c < NC; ++c) kl[i][c] = 0.f;

#pragma unroll 1
        for (int qb = 0; qb < nqo; qb += CHUNK) {
            const int qn = min(CHUNK, nqo - qb);
            // ---- phase A: polygons of outer points qb .. qb + qn - 1, in lockstep
            unsigned long long counts = 0;  // 4 bits per outer point: number of polygon points
#pragma unroll 1
            for (int q = 0; q < qn; ++q) {
                const int q0 = qb + q;
                const float l1o = A.ol[q0][1], l2o = A.ol[q0][2];
                const float Xx = l1o * Ek.x + l2o * Ek.z;  // x_p - v0_k
                const float Xy = l1o * Ek.y + l2o * Ek.w;
                const float Rx[3] = {W0x - Xx, W1x - Xx, W2x - Xx}, Ry[3] = {W0y - Xy, W1y - Xy, W2y - Xy};
                float Cc[3];
#pragma unroll
                for (int m = 0; m < 3; ++m) Cc[m] = Rx[m] * Rx[m] + Ry[m] * Ry[m] - A.d2;
                GeoF G;
                bool ok = decide_flat(Rx, Ry, Cc, eps, floor2, A.d2, G);
                int n = 0;
                if (!CAPS) {
                    // vertices inside and crossings in boundary order; predicated stores
#pragma unroll
                    for (int e = 0; e < 3; ++e) {
                        const int b = (e + 1) % 3;
                        const float ux = Rx[b] - Rx[e], uy = Ry[b] - Ry[e];
                        if (G.in[e]) put(q, n, Rx[e], Ry[e]);
                        n += G.in[e];
                        if (G.nc[e] >= 1) put(q, n, fmaf(G.ta[e], ux, Rx[e]), fmaf(G.ta[e], uy, Ry[e]));
                        n += G.nc[e] >= 1;
                        if (G.nc[e] >= 2) put(q, n, fmaf(G.tb[e], ux, Rx[e]), fmaf(G.tb[e], uy, Ry[e]));
                        n += G.nc[e] >= 2;
                    }
                } else if (ok) {
                    // with caps: a cap centre between consecutive points not joined along an edge
                    int nraw = 0, fe = 0, fv = 0, le = 0;
                    float fx = 0, fy = 0, lx = 0, ly = 0;
                    auto cap = [&](float px, float py, float qx, float qy) {
                        const float cx = qx - px, cy = qy - py;
                        const float len = sqrtf(cx * cx + cy * cy);
                        ok &= len > 1e-6f * A.delta;
                        const float sc = __fdividef(A.delta, len);
                        put(q, min(n, MAXP - 1), sc * cy, -sc * cx);
                        ++n;
                    };
                    auto raw = [&](float x, float y, int e, int v) {
                        if (nraw >= 1 && !((e == le) || (v && e == (le + 1) % 3))) cap(lx, ly, x, y);
                        put(q, min(n, MAXP - 1), x, y);
                        ++n;
                        if (nraw == 0) { fx = x; fy = y; fe = e; fv = v; }
                        lx = x; ly = y; le = e;
                        ++nraw;
                    };
#pragma unroll
                    for (int e = 0; e < 3; ++e) {
                        const int b = (e + 1) % 3;
                        const float ux = Rx[b] - Rx[e], uy = Ry[b] - Ry[e];
                        if (G.in[e]) raw(Rx[e], Ry[e], e, 1);
                        if (G.nc[e] >= 1) raw(fmaf(G.ta[e], ux, Rx[e]), fmaf(G.ta[e], uy, Ry[e]), e, 0);
                        if (G.nc[e] >= 2) raw(fmaf(G.tb[e], ux, Rx[e]), fmaf(G.tb[e], uy, Ry[e]), e, 0);
                    }
                    if (!(G.in[0] && G.in[1] && G.in[2]) && nraw >= 2 && !(fv && fe == (le + 1) % 3))
                        cap(lx, ly, fx, fy);
                }
                if (!valid) n = 0;
                else if (!ok)
                    n = clip_canonical(A.X, tk, tl, P.ro.l[q0][0], P.ro.l[q0][1], P.ro.l[q0][2], P.delta, P.delta2,
                                       CAPS, my + q * MAXP * FAST_THREADS, MAXP);
                counts |= (unsigned long long)(n < 3 ? 0 : n) << (4 * q);
            }
            // ---- phase B: one fan triangle per lane and iteration
            int qc = 0, sc = 2;
            while (qc < qn && ((counts >> (4 * qc)) & 15) == 0) ++qc;
            while (__any_sync(0xffffffffu, qc < qn)) {
                if (qc < qn) {
                    const int q0 = qb + qc;
                    const float l1o = A.ol[q0][1], l2o = A.ol[q0][2];
                    // x_p - v0_l, for the barycentric coordinates of the points
                    const float Bx = l1o * Ek.x + l2o * Ek.z - W0x, By = l1o * Ek.y + l2o * Ek.w - W0y;
                    float px[3], py[3], b1[3], b2[3];
                    const int slot[3] = {0, sc - 1, sc};
#pragma unroll
                    for (int t = 0; t < 3; ++t) {
                        const float2 pt = my[(qc * MAXP + slot[t]) * FAST_THREADS];
                        px[t] = pt.x;
                        py[t] = pt.y;
                        const float rx = pt.x + Bx, ry = pt.y + By;
                        b1[t] = (rx * El.w - ry * El.z) * idet;
                        b2[t] = (El.x * ry - El.y * rx) * idet;
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
                    tri_quad<KER, NQI, NC>(A, I, px[0], py[0], b1[0], b2[0], px[1], py[1], b1[1], b2[1], px[2], py[2],
                                           b1[2], b2[2]);
                    outer_update<NC>(A, q0, dk, I, kk, kl, ll);
                    if (++sc >= (int)((counts >> (4 * qc)) & 15)) {
                        sc = 2;
                        ++qc;
                        while (qc < qn && ((counts >> (4 * qc)) & 15) == 0) ++qc;
                    }
                }
            }
        }
        if (valid) accumulate_pair<NC>(A, pi, p, tk, tl, kk, kl, ll, vmax);
    }
    flush_max(A, vmax);
}

// Fan triangles of a cut pair summed over its outer points, from the same FP32 decisions
// (an undecided outer point counts its FP32 outcome; the count only orders the work).
__global__ void k_cut_tris(FastArgs A, int* __restrict__ key) {
    const int64_t pi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pi >= A.npairs) return;
    const int64_t p = A.ids[pi];
    const int k = A.pk[p], l = A.pl[p];
    const int4 tk = A.T[k], tl = A.T[l];
    const double2 v0k = A.X[tk.x], v0l = A.X[tl.x];
    const float dx = (float)(v0l.x - v0k.x), dy = (float)(v0l.y - v0k.y);
    const float4 Ek = A.E32[k], El = A.E32[l];
    const float Wx[3] = {dx, dx + El.x, dx + El.z}, Wy[3] = {dy, dy + El.y, dy + El.w};
    const int nqo = A.prm.ro.n;
    int tris = 0;
    for (int q0 = 0; q0 < nqo; ++q0) {
        const float Xx = A.ol[q0][1] * Ek.x + A.ol[q0][2] * Ek.z;
        const float Xy = A.ol[q0][1] * Ek.y + A.ol[q0][2] * Ek.w;
        float Rx[3], Ry[3], Cc[3];
        for (int m = 0; m < 3; ++m) {
            Rx[m] = Wx[m] - Xx;
            Ry[m] = Wy[m] - Xy;
            Cc[m] = Rx[m] * Rx[m] + Ry[m] * Ry[m] - A.d2;
        }
        GeoF G;
        decide_flat(Rx, Ry, Cc, 0.f, 0.f, A.d2, G);
        int n = 0;
        for (int e = 0; e < 3; ++e) n += (int)G.in[e] + G.nc[e];
        if (A.caps && n >= 2 && !(G.in[0] && G.in[1] && G.in[2])) n += 1;  // at least one cap
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
template <int KER, int NQI>
__global__ void __launch_bounds__(FAST_THREADS) k_trunc_whole(FastArgs A) {
    constexpr int NC = (KER == NLFEM_KERNEL_PERIDYNAMIC) ? 3 : 1;
    const int nqo = A.prm.ro.n;
    float vmax = 0.f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p0 = (int64_t)blockIdx.x * blockDim.x; p0 < A.npairs; p0 += stride) {
        const int64_t pi = p0 + threadIdx.x;
        const bool valid = pi < A.npairs;
        const int64_t p = valid ? (int64_t)A.ids[pi * A.pstride] : 0;
        const int k = A.pk[p], l = A.pl[p];
        const int4 tk = A.T[k], tl = A.T[l];
        const double2 v0k = A.X[tk.x], v0l = A.X[tl.x];
        const float dx = (float)(v0l.x - v0k.x), dy = (float)(v0l.y - v0k.y);
        const float4 Ek = A.E32[k], El = A.E32[l];
        const float dk = A.det32[k];
        float kk[6][NC], kl[9][NC], ll[6][NC];
#pragma unroll
        for (int i = 0; i < 6; ++i)
#pragma unroll
            for (int c = 0; c < NC; ++c) kk[i][c] = ll[i][c] = 0.f;
#pragma unroll
        for (int i = 0; i < 9; ++i)
#pragma unroll
            for (int c = 0; c < NC; ++c) kl[i][c] = 0.f;
        for (int q0 = 0; q0 < nqo; ++q0) {
            const float Xx = A.ol[q0][1] * Ek.x + A.ol[q0][2] * Ek.z;
            const float Xy = A.ol[q0][1] * Ek.y + A.ol[q0][2] * Ek.w;
            Inner<NC> I;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                I.g[c] = 0.f;
#pragma unroll
                for (int j = 0; j < 3; ++j) I.h[j][c] = 0.f;
#pragma unroll
                for (int j = 0; j < 6; ++j) I.m[j][c] = 0.f;
            }
            tri_quad<KER, NQI, NC>(A, I, dx - Xx, dy - Xy, 0.f, 0.f, dx + El.x - Xx, dy + El.y - Xy, 1.f, 0.f,
                                   dx + El.z - Xx, dy + El.w - Xy, 0.f, 1.f);
            outer_update<NC>(A, q0, dk, I, kk, kl, ll);
        }
        if (valid) accumulate_pair<NC>(A, pi, p, tk, tl, kk, kl, ll, vmax);
    }
    flush_max(A, vmax);
}

static FastArgs fast_args(Mesh& m, PairCache& pc, const Params& prm) {
    FastArgs a;
    a.pk = pc.pk.p; a.pl = pc.pl.p; a.pcls = pc.pcls.p;
    a.X = m.X.p; a.T = m.T.p; a.E32 = m.E32.p; a.det32 = m.det32.p;
    a.prm = prm;
    for (int i = 0; i < 16; ++i) {
        for (int j = 0; j < 3; ++j) {
            a.ol[i][j] = i < prm.ro.n ? (float)prm.ro.l[i][j] : 0.f;
            a.il[i][j] = i < prm.ri.n ? (float)prm.ri.l[i][j] : 0.f;
        }
        a.ow[i] = i < prm.ro.n ? (float)prm.ro.w[i] : 0.f;
        a.iw[i] = i < prm.ri.n ? (float)prm.ri.w[i] : 0.f;
    }
    a.delta = (float)prm.delta;
    a.d2 = (float)prm.delta * (float)prm.delta;
    a.c = (float)prm.c;
    a.s = (float)prm.s;
    a.caps = prm.ball == NLFEM_BALL_APPROXCAPS;
    a.ids = nullptr;
    a.npairs = 0;
    a.acc = nullptr;
    a.kkll = nullptr;
    a.npairs_all = pc.npairs;
    a.up_start = nullptr;
    a.epos = nullptr;
    a.klr = nullptr;
    a.scale = 1.f;
    a.maxabs = nullptr;
    a.pstride = 1;
    return a;
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
    FastArgs a = fast_args(m, pc, prm);
    a.ids = pc.cut_ids.p;
    a.npairs = n;
    DBuf<int> key;
    key.alloc(n, st);
    k_cut_tris<<<nblk(n, 256), 256, 0, st>>>(a, key.p);
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

template <int KER, int NQI, bool CAPS>
static void launch_cut(const FastArgs& a, unsigned grid, cudaStream_t st) {
    constexpr int MAXP = CAPS ? 9 : 6;
    const size_t smem = sizeof(float2) * CHUNK * MAXP * FAST_THREADS;
    NLFEM_CUDA_TRY(cudaFuncSetAttribute(k_trunc_cut<KER, NQI, CAPS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
    k_trunc_cut<KER, NQI, CAPS><<<grid, FAST_THREADS, smem, st>>>(a);
}

template <int KER, int NQI>
static void launch_pair_kernels(int pass, const FastArgs& a, unsigned grid, cudaStream_t st) {
    if (pass == 0) k_trunc_whole<KER, NQI><<<grid, FAST_THREADS, 0, st>>>(a);
    else if (a.caps) launch_cut<KER, NQI, true>(a, grid, st);
    else launch_cut<KER, NQI, false>(a, grid, st);
}

void launch_trunc_fast(Mesh& m, PairCache& pc, const Params& prm, const BulkAcc& b, cudaStream_t st,
                       cudaEvent_t* ev) {
    FastArgs a = fast_args(m, pc, prm);
    a.acc = b.acc;
    a.kkll = b.kkll;
    a.up_start = pc.up_start.p;
    a.epos = pc.epos.p;
    a.scale = b.scale;
    a.maxabs = b.maxabs;
    a.pstride = b.pstride;
    for (int pass = 0; pass < 2; ++pass) {
        a.ids = pass == 0 ? pc.whole_ids.p : pc.cut_ids.p;
        const int64_t n = pass == 0 ? pc.nwhole : pc.ncut;
        a.klr = pass == 0 ? pc.klr_whole.p : pc.klr_cut.p;
        a.npairs = (n + b.pstride - 1) / b.pstride;
        if (ev) NLFEM_CUDA_TRY(cudaEventRecord(ev[pass], st));  // ev[0..2] bracket the two launches
        const unsigned grid = (unsigned)std::min<int64_t>(nblk(a.npairs, FAST_THREADS), 152 * 64);
        if (!grid) continue;
        if (prm.kernel == NLFEM_KERNEL_CONSTANT) {
            if (prm.ri.n == 7) launch_pair_kernels<NLFEM_KERNEL_CONSTANT, 7>(pass, a, grid, st);
            else launch_pair_kernels<NLFEM_KERNEL_CONSTANT, 16>(pass, a, grid, st);
        } else if (prm.kernel == NLFEM_KERNEL_FRACTIONAL) {
            if (prm.ri.n == 7) launch_pair_kernels<NLFEM_KERNEL_FRACTIONAL, 7>(pass, a, grid, st);
            else launch_pair_kernels<NLFEM_KERNEL_FRACTIONAL, 16>(pass, a, grid, st);
        } else {
            if (prm.ri.n == 7) launch_pair_kernels<NLFEM_KERNEL_PERIDYNAMIC, 7>(pass, a, grid, st);
            else launch_pair_kernels<NLFEM_KERNEL_PERIDYNAMIC, 16>(pass, a, grid, st);
        }
        NLFEM_LAUNCH_CHECK();
    }
    if (ev) NLFEM_CUDA_TRY(cudaEventRecord(ev[2], st));
}

}  // namespace nlfem
