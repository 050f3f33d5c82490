// FP32-bulk truncation quadrature for separated pairs (Sec. 2.3.1, eq. discrete-inner)
// with exact geometric decisions.
//
// GB300 runs FP64 at 1/58 of the FP32 rate, so the canonical FP64 clip of every
// (pair, x_p) would dominate the bulk path. Here the geometry runs in FP32 on vectors
// relative to x_p (the pair offset v0_l - v0_k is formed once in FP64 and rounded once;
// element edges are stored in FP32), and every decision the canonical FP64 geometry
// takes — vertex in ball, number of crossings on an edge — is taken in FP32 only when
// its margin exceeds a bound on the FP32 error. Otherwise the outer point falls back
// to the canonical FP64 clip (nl_clip). The interaction pattern and the polygon
// topology therefore equal the FP64 ones; crossing points, cap centres and sub-triangle
// areas carry FP32 rounding (about 1e-7 relative), well inside the 1e-5 bar.
// Without near ties no root snaps, no points merge and no cap is skipped, so the
// canonical tie rules never need to be reproduced in FP32.
//
// The cut polygon is never stored: its points are emitted in boundary order and fed to
// a fan triangulation that integrates triangle (P0, P_prev, P) as soon as P arrives.
// One thread per ordered pair; intersecting pairs go to the canonical kernels.
#include <algorithm>

#include "nlfem_internal.cuh"

namespace nlfem {

static inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

struct FastArgs {
    const int* pk;
    const int* pl;
    const int8_t* pcls;
    int64_t npairs;
    const double2* X;
    const int4* T;
    const float4* E32;
    const float* det32;
    Params prm;
    float ol[16][3], ow[16];  // outer rule in FP32
    float il[16][3], iw[16];  // inner rule in FP32
    float delta, d2, c, s;
    int caps;
};

// accumulators of the inner sums for one x_p
template <int NC>
struct Inner {
    float g[NC], h[3][NC], m[6][NC];
};

template <int KER, int NQI>
__device__ __forceinline__ void tri_quad(const FastArgs& A, Inner<(KER == NLFEM_KERNEL_PERIDYNAMIC) ? 3 : 1>& I,
                                         float ax, float ay, float a1, float a2, float bx, float by, float b1,
                                         float b2, float cx, float cy, float c1, float c2) {
    constexpr int NC = (KER == NLFEM_KERNEL_PERIDYNAMIC) ? 3 : 1;
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

// fan triangulation state: first point and previous point (position relative to x_p,
// barycentric coordinates b1, b2 w.r.t. E_l)
struct Fan {
    float x0, y0, p1, p2;
    float xp, yp, q1, q2;
    int n;
};

template <int KER, int NQI>
__device__ __forceinline__ void fan_emit(const FastArgs& A, Fan& F, Inner<(KER == NLFEM_KERNEL_PERIDYNAMIC) ? 3 : 1>& I,
                                         float x, float y, float b1, float b2) {
    if (F.n == 0) {
        F.x0 = x; F.y0 = y; F.p1 = b1; F.p2 = b2;
    } else {
        if (F.n >= 2) tri_quad<KER, NQI>(A, I, F.x0, F.y0, F.p1, F.p2, F.xp, F.yp, F.q1, F.q2, x, y, b1, b2);
    }
    F.xp = x; F.yp = y; F.q1 = b1; F.q2 = b2;
    ++F.n;
}

// raw boundary point with its position tags (edge, parameter, vertex flag)
struct Raw {
    float x, y, b1, b2, t;
    int e, vert;
};

__device__ __forceinline__ bool joined_r(const Raw& P, const Raw& Q) {
    if (Q.e == P.e && Q.t > P.t) return true;
    if (Q.vert && Q.e == (P.e + 1) % 3) return true;
    return false;
}

struct Walk {
    Raw first, last;
    int nraw;
};

// cap centre between raw points P -> Q: x + delta * (right-hand unit normal of the chord)
template <int KER, int NQI>
__device__ __forceinline__ void emit_cap(const FastArgs& A, Fan& F, Inner<(KER == NLFEM_KERNEL_PERIDYNAMIC) ? 3 : 1>& I,
                                         const Raw& P, const Raw& Q, float Xx, float Xy, float W0x, float W0y,
                                         float4 El, float detE) {
    const float qx = Q.x - P.x, qy = Q.y - P.y;
    const float len = sqrtf(qx * qx + qy * qy);
    if (!(len > 1e-9f * A.delta)) return;
    const float mx = A.delta * (qy / len), my = A.delta * (-qx / len);
    // barycentric coordinates of the cap centre: relative to v0_l, through E_l's inverse map
    const float rx = mx + Xx - W0x, ry = my + Xy - W0y;
    const float b1 = (rx * El.w - ry * El.z) / detE;
    const float b2 = (El.x * ry - El.y * rx) / detE;
    fan_emit<KER, NQI>(A, F, I, mx, my, b1, b2);
}

template <int KER, int NQI>
__device__ __forceinline__ void walk_raw(const FastArgs& A, Walk& Wk, Fan& F,
                                         Inner<(KER == NLFEM_KERNEL_PERIDYNAMIC) ? 3 : 1>& I, const Raw& B, float Xx,
                                         float Xy, float W0x, float W0y, float4 El, float detE) {
    if (A.caps && Wk.nraw >= 1 && !joined_r(Wk.last, B))
        emit_cap<KER, NQI>(A, F, I, Wk.last, B, Xx, Xy, W0x, W0y, El, detE);
    fan_emit<KER, NQI>(A, F, I, B.x, B.y, B.b1, B.b2);
    if (Wk.nraw == 0) Wk.first = B;
    Wk.last = B;
    ++Wk.nraw;
}

template <int KER, int NQI>
__global__ void __launch_bounds__(128) k_trunc_fast(FastArgs A, float* __restrict__ contrib) {
    constexpr int NC = (KER == NLFEM_KERNEL_PERIDYNAMIC) ? 3 : 1;
    constexpr int NE = (KER == NLFEM_KERNEL_PERIDYNAMIC) ? 84 : 21;
    const Params& P = A.prm;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < A.npairs;
         p += (int64_t)gridDim.x * blockDim.x) {
        if (A.pcls[p] != 0) continue;  // intersecting pairs: canonical kernels
        const int k = A.pk[p], l = A.pl[p];
        const int4 tk = A.T[k], tl = A.T[l];
        const double2 v0k = A.X[tk.x], v0l = A.X[tl.x];
        const float dx = (float)(v0l.x - v0k.x), dy = (float)(v0l.y - v0k.y);
        const float4 Ek = A.E32[k], El = A.E32[l];
        const float dk = A.det32[k];
        const float detE = El.x * El.w - El.y * El.z;
        // E_l's vertices relative to v0_k
        const float W0x = dx, W0y = dy;
        const float W1x = dx + El.x, W1y = dy + El.y, W2x = dx + El.z, W2y = dy + El.w;
        // eps bounds the absolute FP32 error of every vertex-relative coordinate R = W - X:
        // each is a short chain (one rounding of v0_l - v0_k, edge vectors rounded once, two
        // FMAs for x_p, one subtraction) of magnitudes <= span; 8 units of 2^-24 each, times 4
        const float span = fabsf(dx) + fabsf(dy) + fabsf(Ek.x) + fabsf(Ek.y) + fabsf(Ek.z) + fabsf(Ek.w) +
                           fabsf(El.x) + fabsf(El.y) + fabsf(El.z) + fabsf(El.w);
        const float eps = 4.8e-7f * span;
        const float floor2 = 1e-5f * A.d2;  // floor of the vertex margin (see nl_decide32)
        float kk[6][NC], kl[9][NC], ll[6][NC];
#pragma unroll
        for (int i = 0; i < 6; ++i)
#pragma unroll
            for (int c = 0; c < NC; ++c) kk[i][c] = ll[i][c] = 0.f;
#pragma unroll
        for (int i = 0; i < 9; ++i)
#pragma unroll
            for (int c = 0; c < NC; ++c) kl[i][c] = 0.f;

        for (int q0 = 0; q0 < P.ro.n; ++q0) {
            const float l1o = A.ol[q0][1], l2o = A.ol[q0][2];
            const float Xx = l1o * Ek.x + l2o * Ek.z, Xy = l1o * Ek.y + l2o * Ek.w;  // x_p - v0_k
            const float R0x = W0x - Xx, R0y = W0y - Xy, R1x = W1x - Xx, R1y = W1y - Xy;
            const float R2x = W2x - Xx, R2y = W2y - Xy;
            const float c0 = R0x * R0x + R0y * R0y - A.d2;
            const float c1 = R1x * R1x + R1y * R1y - A.d2;
            const float c2 = R2x * R2x + R2y * R2y - A.d2;
            Inner<NC> I;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                I.g[c] = 0.f;
#pragma unroll
                for (int j = 0; j < 3; ++j) I.h[j][c] = 0.f;
#pragma unroll
                for (int j = 0; j < 6; ++j) I.m[j][c] = 0.f;
            }
            bool any = false;
            const float Rx[3] = {R0x, R1x, R2x}, Ry[3] = {R0y, R1y, R2y}, Cc[3] = {c0, c1, c2};
            Geo32 G;
            bool tie = !nl_decide32(Rx, Ry, Cc, eps, floor2, A.d2, G);
            if (!tie && G.in[0] && G.in[1] && G.in[2]) {
                tri_quad<KER, NQI>(A, I, R0x, R0y, 0.f, 0.f, R1x, R1y, 1.f, 0.f, R2x, R2y, 0.f, 1.f);
                any = true;
            } else if (!tie) {
                const bool* in = G.in;
                const int* nc = G.nc;
                const float* ta = G.ta;
                const float* tb = G.tb;
                {
                    Fan F;
                    F.n = 0;
                    Walk Wk;
                    Wk.nraw = 0;
#pragma unroll
                    for (int e = 0; e < 3; ++e) {
                        const int b = (e + 1) % 3;
                        const float e1 = (e == 1) ? 1.f : 0.f, e2 = (e == 2) ? 1.f : 0.f;
                        const float f1 = (b == 1) ? 1.f : 0.f, f2 = (b == 2) ? 1.f : 0.f;
                        if (in[e]) {
                            Raw V{Rx[e], Ry[e], e1, e2, 0.f, e, 1};
                            walk_raw<KER, NQI>(A, Wk, F, I, V, Xx, Xy, W0x, W0y, El, detE);
                        }
                        for (int j = 0; j < nc[e]; ++j) {
                            const float t = j == 0 ? ta[e] : tb[e];
                            const float ux = Rx[b] - Rx[e], uy = Ry[b] - Ry[e];
                            Raw Cp{Rx[e] + t * ux, Ry[e] + t * uy, e1 + t * (f1 - e1), e2 + t * (f2 - e2), t, e, 0};
                            walk_raw<KER, NQI>(A, Wk, F, I, Cp, Xx, Xy, W0x, W0y, El, detE);
                        }
                    }
                    if (A.caps && Wk.nraw >= 2 && !joined_r(Wk.last, Wk.first))
                        emit_cap<KER, NQI>(A, F, I, Wk.last, Wk.first, Xx, Xy, W0x, W0y, El, detE);
                    any = F.n >= 3;
                }
            }
            if (tie) {
                // canonical FP64 geometry for this outer point
                const double2 Vk[3] = {v0k, A.X[tk.y], A.X[tk.z]};
                const double2 Vl[3] = {v0l, A.X[tl.y], A.X[tl.z]};
                const double2 xp = nl_map(Vk, P.ro.l[q0][0], P.ro.l[q0][1], P.ro.l[q0][2]);
                CPt poly[NLFEM_MAXPOLY];
                bool full;
                const int np = nl_clip(Vl, xp, P.delta, P.delta2, A.caps != 0, poly, full);
                if (np >= 3) {
                    any = true;
                    if (full) {
                        tri_quad<KER, NQI>(A, I, (float)(Vl[0].x - xp.x), (float)(Vl[0].y - xp.y), 0.f, 0.f,
                                           (float)(Vl[1].x - xp.x), (float)(Vl[1].y - xp.y), 1.f, 0.f,
                                           (float)(Vl[2].x - xp.x), (float)(Vl[2].y - xp.y), 0.f, 1.f);
                    } else {
                        Fan F;
                        F.n = 0;
                        for (int i = 0; i < np; ++i)
                            fan_emit<KER, NQI>(A, F, I, (float)(poly[i].x - xp.x), (float)(poly[i].y - xp.y),
                                               (float)poly[i].b1, (float)poly[i].b2);
                    }
                }
            }
            if (!any) continue;
            const float ap = A.ow[q0] * dk;
            const float Pa[3] = {A.ol[q0][0], l1o, l2o};
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
        // union block of a separated pair: [[kk, kl], [kl^T, ll]]; write its upper triangle
        float* out = contrib + p * NE;
        // entry order E(a,b), a <= b over the union (k0 k1 k2 l0 l1 l2)
        const int kkI[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
        int e = 0;
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
            for (int b = a; b < 6; ++b) {
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    float v;
                    if (b < 3) v = kk[kkI[a][b]][c];
                    else if (a < 3) v = kl[a * 3 + (b - 3)][c];
                    else v = ll[kkI[a - 3][b - 3]][c];
                    if (NC == 1) {
                        out[e] = v;
                    } else if (c == 0) {
                        out[e * 4 + 0] = v;
                    } else if (c == 1) {
                        out[e * 4 + 1] = v;
                        out[e * 4 + 2] = v;
                    } else {
                        out[e * 4 + 3] = v;
                    }
                }
                ++e;
            }
    }
}

void launch_trunc_fast(Mesh& m, PairCache& pc, const Params& prm, float* contrib, cudaStream_t st) {
    FastArgs a;
    a.pk = pc.pk.p; a.pl = pc.pl.p; a.pcls = pc.pcls.p; a.npairs = pc.npairs;
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
    unsigned grid = (unsigned)std::min<int64_t>(nblk(pc.npairs, 128), 152 * 64);
    if (!grid) return;
#define NLFEM_TF(KK, NQ) k_trunc_fast<KK, NQ><<<grid, 128, 0, st>>>(a, contrib)
    if (prm.kernel == NLFEM_KERNEL_CONSTANT) {
        if (prm.ri.n == 7) NLFEM_TF(NLFEM_KERNEL_CONSTANT, 7); else NLFEM_TF(NLFEM_KERNEL_CONSTANT, 16);
    } else if (prm.kernel == NLFEM_KERNEL_FRACTIONAL) {
        if (prm.ri.n == 7) NLFEM_TF(NLFEM_KERNEL_FRACTIONAL, 7); else NLFEM_TF(NLFEM_KERNEL_FRACTIONAL, 16);
    } else {
        if (prm.ri.n == 7) NLFEM_TF(NLFEM_KERNEL_PERIDYNAMIC, 7); else NLFEM_TF(NLFEM_KERNEL_PERIDYNAMIC, 16);
    }
#undef NLFEM_TF
    NLFEM_LAUNCH_CHECK();
}

}  // namespace nlfem
