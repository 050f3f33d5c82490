// Element-pair search within the horizon (the interaction graph T_S of Sec. 2.4).
//
// The paper finds the partners of E_k by a breadth-first traversal of the adjacency
// graph (Alg. 2). Here the same set is found data-parallel: elements are binned into a
// uniform grid of cell size >= delta + 2 r_max, every candidate in the 3 x 3 cell block
// is tested with the exact FP64 predicate, and the survivors are compacted with a
// prefix sum. The predicate: E_l interacts with E_k iff they share a vertex (intersecting
// pairs always interact; T_adj spans T_S) or some outer quadrature point x_p of E_k sees
// a polygon of >= 3 points when E_l is cut by the ball approximation around x_p.
#include <algorithm>
#include <cmath>

#include "nlfem_internal.cuh"

namespace nlfem {

static inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// Uniform grid over the element centroids. A partner's centroid lies within reach + r_k + r_l
// of the element's centroid, at most span cells away in each direction (cells of at least
// (reach + 2 r_max) / span).
struct Grid {
    double x0, y0, cs;
    int nx, ny;
    int span;
};

__global__ void k_bin_count(const double2* cen, int64_t K, Grid g, int64_t* cnt, int* cell_of) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    double2 c = cen[k];
    int cx = min(g.nx - 1, max(0, (int)floor((c.x - g.x0) / g.cs)));
    int cy = min(g.ny - 1, max(0, (int)floor((c.y - g.y0) / g.cs)));
    int cell = cy * g.nx + cx;
    cell_of[k] = cell;
    atomicAdd((unsigned long long*)&cnt[cell], 1ull);
}

__global__ void k_bin_fill(const int* cell_of, int64_t K, const int64_t* start, int* cursor, int* list) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    int cell = cell_of[k];
    int pos = atomicAdd(&cursor[cell], 1);
    list[start[cell] + pos] = (int)k;
}

__device__ __forceinline__ int shared_count(int4 a, int4 b) {
    int c = 0;
    c += (a.x == b.x) + (a.x == b.y) + (a.x == b.z);
    c += (a.y == b.x) + (a.y == b.y) + (a.y == b.z);
    c += (a.z == b.x) + (a.z == b.y) + (a.z == b.z);
    return c;
}

struct SearchArgs {
    const double2* X;
    const int4* T;
    const float4* E32;
    float ol[16][2];  // outer rule barycentrics (l1, l2) in FP32
    float delta32, d2f;
    const double2* cen;
    const double* rad;
    const int* cell_of;
    const int64_t* cell_start;
    const int* cell_list;
    Grid g;
    int64_t K;
    double reach, rmax;  // search radius (delta, or sqrt(2) delta for the infinity ball), largest element radius
    double delta, delta2;
    int caps;
    int ball;
    const int4* Tp;  // vertex positions of the elements (shared vertices decide intersecting pairs)
    Rule ro;
};

// Centroid tests of the candidate (k, l): 0 = not a partner, 1 = a partner, 2 = the cut of
// E_l by the balls of E_k's outer points decides (interacts_clip).
// Elements sharing a vertex have centroids at most rk + rl apart, so the far tests come first
// and the vertex triples are read only for the candidates that pass them.
__device__ int interacts_centroid(const SearchArgs& a, int k, int l, double2 ck, double rk, float rkf) {
    const double2 cl = a.cen[l];
    const double rl = a.rad[l];
    const double cdx = cl.x - ck.x, cdy = cl.y - ck.y;
    if (a.ball == NLFEM_BALL_INFINITY) {
        // infinity ball: the square's circumradius sqrt(2) delta and, for the whole element,
        // its half side
        const double dist = sqrt(cdx * cdx + cdy * cdy);
        if (dist - rk - rl > a.delta * 1.4142135623730951 * (1.0 + 1e-9)) return 0;
        if (shared_count(a.Tp[k], a.Tp[l]) > 0) return 1;
        if (fmax(fabs(cdx), fabs(cdy)) + rk + rl <= a.delta * (1.0 - 1e-9)) return 1;
        return 2;
    }
    // decided in FP32 on squared distances when the margin (1e-5 relative, far above the FP32
    // error of about 3e-7) allows, else by the FP64 expressions below. The FP32 bounds are
    // widened by 1e-6 of delta (far up, near down), above the rounding of their FP32 sums, so
    // that an FP32 decision is one the FP64 bounds also take; the band between goes to the
    // FP64 tests or to the cut, which agree with them.
    const float d2f = (float)cdx * (float)cdx + (float)cdy * (float)cdy;
    const float rlf = (float)rl;
    const float far = rkf + rlf + a.delta32 * (1.f + 1e-6f);
    const float innerf = a.delta32 * (1.f - 1e-6f) - rkf - rlf;
    const float nearf = innerf > 0.f ? innerf : -1.f;
    if (d2f > far * far * (1.f + 1e-5f)) return 0;
    if (shared_count(a.Tp[k], a.Tp[l]) > 0) return 1;
    if (nearf > 0.f && d2f < nearf * nearf * (1.f - 1e-5f)) return 1;  // E_l inside the ball of every x in E_k
    if (d2f >= far * far * (1.f - 1e-5f) || (nearf > 0.f && d2f <= nearf * nearf * (1.f + 1e-5f))) {
        const double dist = sqrt(cdx * cdx + cdy * cdy);
        if (dist - rk - rl > a.delta * (1.0 + 1e-9)) return 0;
        if (dist + rk + rl <= a.delta * (1.0 - 1e-9)) return 1;
    }
    return 2;
}

// The cut decides: some outer point x_p of E_k sees a polygon of >= 3 points.
__device__ bool interacts_clip(const SearchArgs& a, int k, int l, const double2 Vk[3]) {
    const int4 tl = a.T[l];
    const double2 v0l = a.X[tl.x];
    if (a.ball == NLFEM_BALL_INFINITY) {
        const double2 Vl[3] = {v0l, a.X[tl.y], a.X[tl.z]};
        for (int p = 0; p < a.ro.n; ++p) {
            const double2 xp = nl_map(Vk, a.ro.l[p][0], a.ro.l[p][1], a.ro.l[p][2]);
            bool full;
            if (nl_clip_square(Vl, xp, a.delta, nullptr, full) >= 3) return true;
        }
        return false;
    }
    // FP32 geometry with exact decisions; the canonical FP64 clip only for near ties
    const float dx = (float)(v0l.x - Vk[0].x), dy = (float)(v0l.y - Vk[0].y);
    const float4 Ek = a.E32[k], El = a.E32[l];
    const float span = fabsf(dx) + fabsf(dy) + fabsf(Ek.x) + fabsf(Ek.y) + fabsf(Ek.z) + fabsf(Ek.w) +
                       fabsf(El.x) + fabsf(El.y) + fabsf(El.z) + fabsf(El.w);
    const float eps = 4.8e-7f * span, floor2 = 1e-5f * a.d2f;
    const float Wx[3] = {dx, dx + El.x, dx + El.z}, Wy[3] = {dy, dy + El.y, dy + El.w};
    // a vertex of E_l strictly inside some ball: that polygon has the vertex and a point on
    // each of its two edges, so >= 3 points
    for (int p = 0; p < a.ro.n; ++p) {
        const float Xx = a.ol[p][0] * Ek.x + a.ol[p][1] * Ek.z, Xy = a.ol[p][0] * Ek.y + a.ol[p][1] * Ek.w;
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            const float rx = Wx[m] - Xx, ry = Wy[m] - Xy;
            if (rx * rx + ry * ry - a.d2f < -(floor2 + 2.f * (fabsf(rx) + fabsf(ry)) * eps)) return true;
        }
    }
    // E_l lies in the disc of radius r_l about its centroid: an outer point farther than
    // delta + r_l from it (beyond the FP32 error of the relative coordinates) sees no point of
    // E_l, so its cut is empty without deciding anything
    const float gx = (Wx[0] + Wx[1] + Wx[2]) * (1.f / 3.f), gy = (Wy[0] + Wy[1] + Wy[2]) * (1.f / 3.f);
    const float reach = a.delta32 + (float)a.rad[l] + 8.f * eps;
    const float reach2 = reach * reach * (1.f + 1e-5f);
    for (int p = 0; p < a.ro.n; ++p) {
        const float Xx = a.ol[p][0] * Ek.x + a.ol[p][1] * Ek.z, Xy = a.ol[p][0] * Ek.y + a.ol[p][1] * Ek.w;
        if ((gx - Xx) * (gx - Xx) + (gy - Xy) * (gy - Xy) > reach2) continue;
        float Rx[3], Ry[3], C[3];
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            Rx[m] = Wx[m] - Xx;
            Ry[m] = Wy[m] - Xy;
            C[m] = Rx[m] * Rx[m] + Ry[m] * Ry[m] - a.d2f;
        }
        Geo32 G;
        if (nl_decide32(Rx, Ry, C, eps, floor2, a.d2f, G)) {
            if (nl_count32(G, a.caps != 0) >= 3) return true;
        } else {
            const double2 Vl[3] = {v0l, a.X[tl.y], a.X[tl.z]};
            const double2 xp = nl_map(Vk, a.ro.l[p][0], a.ro.l[p][1], a.ro.l[p][2]);
            bool full;
            if (nl_clip(Vl, xp, a.delta, a.delta2, a.caps != 0, nullptr, full) >= 3) return true;
        }
    }
    return false;
}

// One warp per outer element k. FILL = false: count partners; true: write them at ptr[k].
// SLOTS: write them at k * cap (cap = the largest candidate count) and count them, in one
// pass; k_compact_slots then packs the slots.
template <bool FILL, bool SLOTS = false>
__global__ void __launch_bounds__(128) k_search(SearchArgs a, int64_t* count, const int64_t* ptr, int* out_l,
                                                int64_t cap = 0) {
    __shared__ int s_queue[4 * 64];  // launched with 128 threads: 4 warps, 64 queue slots each
    int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (k >= a.K) return;
    int4 tk = a.T[k];
    double2 Vk[3] = {a.X[tk.x], a.X[tk.y], a.X[tk.z]};
    double2 ck = a.cen[k];
    double rk = a.rad[k];
    const float rkf = (float)rk;
    int cell = a.cell_of[k];
    int cx = cell % a.g.nx, cy = cell / a.g.nx;
    int64_t n = 0;
    int64_t base = SLOTS ? k * cap : (FILL ? ptr[k] : 0);
    // candidates the centroid tests leave open wait in a per-warp queue and are cut 32 at a
    // time with every lane busy (the partners' order does not matter: the lists are sorted)
    int* q = s_queue + (threadIdx.x >> 5) * 64;
    int qn = 0;  // warp-uniform
    auto emit = [&](bool ok, int l) {
        const unsigned m = __ballot_sync(0xffffffffu, ok);
        if ((FILL || SLOTS) && ok) out_l[base + n + __popc(m & ((1u << lane) - 1u))] = l;
        n += __popc(m);
    };
    auto drain = [&](int cnt) {  // cut the first cnt (<= 32) queued candidates, keep the rest
        const int l = lane < cnt ? q[lane] : -1;
        const bool ok = lane < cnt && interacts_clip(a, (int)k, l, Vk);
        emit(ok, l);
        const int rest = qn - cnt;
        const int v = lane < rest ? q[cnt + lane] : 0;
        __syncwarp();
        if (lane < rest) q[lane] = v;
        __syncwarp();
        qn = rest;
    };
    // with span > 1, cells whose rectangle lies farther than reach + r_k + r_max from the centroid
    // are skipped: the distance is taken in cell units in FP32 on the centroid's position inside
    // its cell, with a margin of 1e-3 cells (far above the FP32 error of numbers below span + 1)
    const int S = a.g.span;
    const double ics = 1.0 / a.g.cs;
    const float fx = (float)((ck.x - a.g.x0) * ics - cx), fy = (float)((ck.y - a.g.y0) * ics - cy);
    const float lim = (float)((a.reach + rk + a.rmax) * (1.0 + 1e-6) * ics) + 1e-3f;
    for (int dyc = -S; dyc <= S; ++dyc) {
        int yy = cy + dyc;
        if (yy < 0 || yy >= a.g.ny) continue;
        const float gy = dyc > 0 ? dyc - fy : (dyc < 0 ? fy - (dyc + 1) : 0.f);
        for (int dxc = -S; dxc <= S; ++dxc) {
            int xx = cx + dxc;
            if (xx < 0 || xx >= a.g.nx) continue;
            const float gx = dxc > 0 ? dxc - fx : (dxc < 0 ? fx - (dxc + 1) : 0.f);
            if (S > 1 && gx * gx + gy * gy > lim * lim) continue;
            int c = yy * a.g.nx + xx;
            int64_t s = a.cell_start[c], e = a.cell_start[c + 1];
            for (int64_t j0 = s; j0 < e; j0 += 32) {
                int64_t j = j0 + lane;
                int r = 0;
                int l = -1;
                if (j < e) {
                    l = a.cell_list[j];
                    r = interacts_centroid(a, (int)k, l, ck, rk, rkf);
                }
                emit(r == 1, l);
                const unsigned mb = __ballot_sync(0xffffffffu, r == 2);
                if (r == 2) q[qn + __popc(mb & ((1u << lane) - 1u))] = l;
                qn += __popc(mb);
                __syncwarp();
                if (qn >= 32) drain(32);
            }
        }
    }
    while (qn > 0) drain(qn < 32 ? qn : 32);
    if ((!FILL || SLOTS) && lane == 0) count[k] = n;
}

// Ordered search. The candidates of every element of cell c are N(c): the elements of the
// cells of c's block of (2 span + 1)^2 cells, sorted by id, once per cell. Candidate j of element
// k owns slot k * cap + j, which receives l when the pair (k, l) interacts and -1 otherwise, at
// whatever time its decision is taken (the queued ones later); packing the slots in order then
// gives the partner list sorted by l, so no sort follows.
__global__ void k_block_count(Grid g, const int64_t* cell_start, int64_t* cnt) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= (int64_t)g.nx * g.ny) return;
    const int cx = (int)(c % g.nx), cy = (int)(c / g.nx);
    int64_t n = 0;
    for (int yy = max(cy - g.span, 0); yy <= min(cy + g.span, g.ny - 1); ++yy)
        for (int xx = max(cx - g.span, 0); xx <= min(cx + g.span, g.nx - 1); ++xx) {
            const int64_t cc = (int64_t)yy * g.nx + xx;
            n += cell_start[cc + 1] - cell_start[cc];
        }
    cnt[c] = n;
}

// warp per cell: the elements of its block's cells (sorted afterwards)
__global__ void k_block_fill(Grid g, const int64_t* cell_start, const int* cell_list, const int64_t* nptr,
                             int* nlist) {
    const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (c >= (int64_t)g.nx * g.ny) return;
    const int cx = (int)(c % g.nx), cy = (int)(c / g.nx);
    int64_t o = nptr[c];
    for (int yy = max(cy - g.span, 0); yy <= min(cy + g.span, g.ny - 1); ++yy)
        for (int xx = max(cx - g.span, 0); xx <= min(cx + g.span, g.nx - 1); ++xx) {
            const int64_t cc = (int64_t)yy * g.nx + xx;
            const int64_t s = cell_start[cc], e = cell_start[cc + 1];
            for (int64_t j = s + lane; j < e; j += 32) nlist[o + (j - s)] = cell_list[j];
            o += e - s;
        }
}

__global__ void __launch_bounds__(128) k_search_ordered(SearchArgs a, const int64_t* nptr, const int* nlist,
                                                        int64_t* count, int* slots, int8_t* scls, int64_t cap) {
    __shared__ int s_queue[4 * 64];  // launched with 128 threads: 4 warps, 64 queued candidate indices each
    const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (k >= a.K) return;
    const int4 tk = a.T[k];
    const double2 Vk[3] = {a.X[tk.x], a.X[tk.y], a.X[tk.z]};
    const double2 ck = a.cen[k];
    const double rk = a.rad[k];
    const float rkf = (float)rk;
    const int c = a.cell_of[k];
    const int64_t start = nptr[c];
    const int len = (int)(nptr[c + 1] - start);
    int* const row = slots + k * cap;
    int8_t* const crow = scls + k * cap;  // the partners' classes (shared vertices, Tab. 1)
    const int4 tpk = a.Tp[k];
    int* q = s_queue + (threadIdx.x >> 5) * 64;
    int qn = 0;  // warp-uniform
    int64_t n = 0;
    auto drain = [&](int cnt) {  // cut the first cnt (<= 32) queued candidates, keep the rest
        const int j = lane < cnt ? q[lane] : 0;
        const int l = lane < cnt ? nlist[start + j] : -1;
        const bool ok = lane < cnt && interacts_clip(a, (int)k, l, Vk);
        if (lane < cnt) row[j] = ok ? l : -1;
        if (ok) crow[j] = (int8_t)shared_count(tpk, a.Tp[l]);
        n += __popc(__ballot_sync(0xffffffffu, ok));
        const int rest = qn - cnt;
        const int v = lane < rest ? q[cnt + lane] : 0;
        __syncwarp();
        if (lane < rest) q[lane] = v;
        __syncwarp();
        qn = rest;
    };
    for (int j0 = 0; j0 < len; j0 += 32) {
        const int j = j0 + lane;
        int r = 0;
        if (j < len) {
            const int l = nlist[start + j];
            r = interacts_centroid(a, (int)k, l, ck, rk, rkf);
            if (r != 2) row[j] = r == 1 ? l : -1;
            if (r == 1) crow[j] = (int8_t)shared_count(tpk, a.Tp[l]);
        }
        n += __popc(__ballot_sync(0xffffffffu, r == 1));
        const unsigned mb = __ballot_sync(0xffffffffu, r == 2);
        if (r == 2) q[qn + __popc(mb & ((1u << lane) - 1u))] = j;
        qn += __popc(mb);
        __syncwarp();
        if (qn >= 32) drain(32);
    }
    while (qn > 0) drain(qn < 32 ? qn : 32);
    if (lane == 0) count[k] = n;
}

// Position of every element in the candidate lists that hold it: element e sits in N(c) for the
// cells c of its own cell's block; pos[e * bb + b] is its index in N(c) for the block cell b
// (row-major offsets (dy, dx) from -span to span; bb = (2 span + 1)^2).
__global__ void k_block_pos(Grid g, const int64_t* nptr, const int* nlist, const int* cell_of, int* pos) {
    const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (c >= (int64_t)g.nx * g.ny) return;
    const int cx = (int)(c % g.nx), cy = (int)(c / g.nx), w = 2 * g.span + 1;
    const int64_t s = nptr[c], e = nptr[c + 1];
    for (int64_t j = s + lane; j < e; j += 32) {
        const int el = nlist[j], ce = cell_of[el];
        const int dx = cx - ce % g.nx, dy = cy - ce / g.nx;
        pos[(int64_t)el * w * w + (dy + g.span) * w + (dx + g.span)] = (int)(j - s);
    }
}

// The transposed lists in order, the same way: pair (k, l) goes to slot l * cap + (index of k in
// N(cell(l))), and the slots of l packed in order list its pairs by increasing k, that is by
// increasing pair id.
__global__ void k_compact_transposed(const int* tslots, int64_t K, int64_t cap, const int* cell_of,
                                     const int64_t* nptr, const int64_t* tptr, int* out) {
    const int64_t l = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (l >= K) return;
    const int c = cell_of[l];
    const int len = (int)(nptr[c + 1] - nptr[c]);
    int64_t o = tptr[l];
    for (int j0 = 0; j0 < len; j0 += 32) {
        const int j = j0 + lane;
        const int v = j < len ? tslots[l * cap + j] : -1;
        const unsigned m = __ballot_sync(0xffffffffu, v >= 0);
        if (v >= 0) out[o + __popc(m & ((1u << lane) - 1u))] = v;
        o += __popc(m);
    }
}

// pack the candidate-indexed slots into the pair list and its classes (warp per element, order
// kept); count the pairs of every inner element (the transposed lists' lengths) and of every class
__global__ void k_compact_ordered(const int* slots, const int8_t* scls, int64_t K, int64_t cap, const int* cell_of,
                                  const int64_t* nptr, const int64_t* ptr, int* out, int8_t* cls,
                                  unsigned long long* counts, int64_t* tcount, Grid g, const int* pos,
                                  int* tslots) {
    const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (k >= K) return;
    const int c = cell_of[k];
    const int len = (int)(nptr[c + 1] - nptr[c]);
    const int cx = c % g.nx, cy = c / g.nx, w = 2 * g.span + 1;
    int64_t o = ptr[k];
    unsigned long long cc[4] = {0, 0, 0, 0};
    for (int j0 = 0; j0 < len; j0 += 32) {
        const int j = j0 + lane;
        const int v = j < len ? slots[k * cap + j] : -1;
        const unsigned m = __ballot_sync(0xffffffffu, v >= 0);
        if (v >= 0) {
            const int8_t cv = scls[k * cap + j];
            const int64_t at = o + __popc(m & ((1u << lane) - 1u));
            out[at] = v;
            cls[at] = cv;
            atomicAdd((unsigned long long*)&tcount[v], 1ull);
            // the transposed slot: k's index in N(cell(v)), from k's position table
            const int cv2 = cell_of[v];
            const int dx = cv2 % g.nx - cx, dy = cv2 / g.nx - cy;
            tslots[(int64_t)v * cap + pos[k * w * w + (dy + g.span) * w + (dx + g.span)]] = (int)at;
#pragma unroll
            for (int t = 0; t < 4; ++t) cc[t] += cv == t;
        }
        o += __popc(m);
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        unsigned long long x = cc[t];
        for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
        if (lane == 0 && x) atomicAdd(&counts[t], x);
    }
}

// the largest number of candidates of an element (its block of (2 span + 1)^2 cells)
__global__ void k_max_cand(const int* cell_of, int64_t K, Grid g, const int64_t* cell_start,
                           unsigned long long* out) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t n = 0;
    if (k < K) {
        const int cell = cell_of[k];
        const int cx = cell % g.nx, cy = cell / g.nx;
        for (int yy = max(cy - g.span, 0); yy <= min(cy + g.span, g.ny - 1); ++yy)
            for (int xx = max(cx - g.span, 0); xx <= min(cx + g.span, g.nx - 1); ++xx) {
                const int c = yy * g.nx + xx;
                n += cell_start[c + 1] - cell_start[c];
            }
    }
    warp_atomic_max(out, (unsigned long long)n);
}

// pack the per-element slots into the pair list (warp per element, order kept)
__global__ void k_compact_slots(const int* slots, int64_t K, int64_t cap, const int64_t* ptr, int* out) {
    const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (k >= K) return;
    const int64_t b = ptr[k], n = ptr[k + 1] - b;
    for (int64_t j = lane; j < n; j += 32) out[b + j] = slots[k * cap + j];
}

__global__ void k_fill_k(const int64_t* ptr, int64_t K, int* pk) {
    int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (k >= K) return;
    for (int64_t p = ptr[k] + lane; p < ptr[k + 1]; p += 32) pk[p] = (int)k;
}

__global__ void k_classify(const int* pk, const int* pl, int64_t P, const int4* T, int8_t* cls,
                           unsigned long long* counts, int64_t* tcount) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int c = -1;
    if (p < P) {
        int l = pl[p];
        c = shared_count(T[pk[p]], T[l]);
        cls[p] = (int8_t)c;
        atomicAdd((unsigned long long*)&tcount[l], 1ull);
    }
    // class counts, aggregated per warp
    for (int v = 0; v < 4; ++v) {
        unsigned m = __ballot_sync(0xffffffffu, c == v);
        if ((threadIdx.x & 31) == 0 && m) atomicAdd(&counts[v], (unsigned long long)__popc(m));
    }
}

__global__ void k_fill_T(const int* pl, int64_t P, const int64_t* tptr, int* cursor, int* tid) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    int l = pl[p];
    int pos = atomicAdd(&cursor[l], 1);
    tid[tptr[l] + pos] = (int)p;
}

// The work lists of the quadrature: every pair goes to exactly one of them. Close list (bit 2):
// intersecting pairs under the singular or the diamond rule. The other pairs take the standard
// rule, split by whether the inner element lies in the ball of every point of the outer
// element: whole (bit 0), when the largest vertex-to-vertex distance is below delta with a
// relative margin of 1e-6 (far above FP64 rounding, so the canonical clip finds all three
// vertices inside at every outer point), else cut (bit 1). For the infinity ball the same test
// runs on the largest coordinate difference against delta.
__device__ __forceinline__ int pair_list(int64_t p, const int* pk, const int* pl, const int8_t* cls, const double2* X,
                                         const int4* T, const ElemRec* rec, double delta2, int std_close, int inf,
                                         double delta) {
    if (cls[p] != 0 && !std_close) return 4;
    const int k = pk[p], l = pl[p];
    const ElemRec rk = rec[k], rl = rec[l];
    // vertices relative to vertex 0 of E_k in FP32 (the offset rounded once from FP64, the edge
    // vectors as stored): decided there unless within 1e-4 of the threshold, then from the FP64
    // vertices
    const float ox = (float)(rl.v0.x - rk.v0.x), oy = (float)(rl.v0.y - rk.v0.y);
    const float kx[3] = {0.f, rk.E.x, rk.E.z}, ky[3] = {0.f, rk.E.y, rk.E.w};
    const float lx[3] = {ox, ox + rl.E.x, ox + rl.E.z}, ly[3] = {oy, oy + rl.E.y, oy + rl.E.w};
    float mxf = 0.f;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            const float dx = lx[j] - kx[i], dy = ly[j] - ky[i];
            mxf = fmaxf(mxf, inf ? fmaxf(fabsf(dx), fabsf(dy)) : dx * dx + dy * dy);
        }
    const float thr = (float)((inf ? delta : delta2) * (1.0 - 1e-6));
    bool whole;
    if (mxf < thr * (1.f - 1e-4f)) whole = true;
    else if (mxf > thr * (1.f + 1e-4f)) whole = false;
    else {
        const int4 a = T[k], b = T[l];
        const double2 va[3] = {X[a.x], X[a.y], X[a.z]}, vb[3] = {X[b.x], X[b.y], X[b.z]};
        double mx = 0.0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                const double dx = vb[j].x - va[i].x, dy = vb[j].y - va[i].y;
                mx = fmax(mx, inf ? fmax(fabs(dx), fabs(dy)) : dx * dx + dy * dy);
            }
        whole = mx <= (inf ? delta : delta2) * (1.0 - 1e-6);
    }
    return whole ? 1 : 2;
}

// Ordered compaction of the three lists in two passes over blocks of LIST_BLOCK pairs: the
// first writes each pair's list (one byte) and every block's count per list, the counts are
// scanned, the second writes the pair ids at the block's offsets in pair order.
static constexpr int LIST_THREADS = 256;
static constexpr int LIST_BLOCK = 4 * LIST_THREADS;

__global__ void __launch_bounds__(LIST_THREADS) k_list_flags(const int* pk, const int* pl, const int8_t* cls,
                                                             int64_t P, const double2* X, const int4* T,
                                                             const ElemRec* rec, double delta2, int std_close,
                                                             int inf, double delta, int8_t* code, int64_t* bcount) {
    __shared__ int sc[3];
    if (threadIdx.x < 3) sc[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * LIST_BLOCK;
    int c0 = 0, c1 = 0, c2 = 0;
    for (int j = 0; j < 4; ++j) {
        const int64_t p = base + j * LIST_THREADS + threadIdx.x;
        if (p >= P) continue;
        const int c = pair_list(p, pk, pl, cls, X, T, rec, delta2, std_close, inf, delta);
        code[p] = (int8_t)c;
        c0 += c & 1;
        c1 += (c >> 1) & 1;
        c2 += (c >> 2) & 1;
    }
    c0 = __reduce_add_sync(0xffffffffu, c0);
    c1 = __reduce_add_sync(0xffffffffu, c1);
    c2 = __reduce_add_sync(0xffffffffu, c2);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&sc[0], c0);
        atomicAdd(&sc[1], c1);
        atomicAdd(&sc[2], c2);
    }
    __syncthreads();
    if (threadIdx.x < 3) bcount[(int64_t)threadIdx.x * gridDim.x + blockIdx.x] = sc[threadIdx.x];
}

// boff: [3][nb + 1] exclusive scans of the block counts; out[i]: list i (whole, cut, close)
__global__ void __launch_bounds__(LIST_THREADS) k_list_fill(const int8_t* code, int64_t P, const int64_t* boff,
                                                            int* out0, int* out1, int* out2) {
    __shared__ int wsum[3][LIST_THREADS / 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t nb1 = (int64_t)gridDim.x + 1;
    int64_t off[3] = {boff[blockIdx.x], boff[nb1 + blockIdx.x], boff[2 * nb1 + blockIdx.x]};
    int* out[3] = {out0, out1, out2};
    const int64_t base = (int64_t)blockIdx.x * LIST_BLOCK;
    for (int j = 0; j < 4; ++j) {
        // pairs base + j * LIST_THREADS + t, in order of t: a warp's ballot, then the warps' prefix
        const int64_t p = base + j * LIST_THREADS + threadIdx.x;
        const int c = p < P ? code[p] : 0;
        unsigned m[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            m[i] = __ballot_sync(0xffffffffu, (c >> i) & 1);
            if (lane == 0) wsum[i][warp] = __popc(m[i]);
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            int before = 0, total = 0;
            for (int w = 0; w < LIST_THREADS / 32; ++w) {
                before += w < warp ? wsum[i][w] : 0;
                total += wsum[i][w];
            }
            if ((c >> i) & 1) out[i][off[i] + before + __popc(m[i] & ((1u << lane) - 1u))] = (int)p;
            off[i] += total;
        }
        __syncthreads();
    }
}

__global__ void k_max_seg64(const int64_t* ptr, int64_t n, unsigned long long* out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    warp_atomic_max(out, i < n ? (unsigned long long)(ptr[i + 1] - ptr[i]) : 0ull);
}

int64_t max_segment_i64(const int64_t* ptr, int64_t n, cudaStream_t st) {
    DBuf<unsigned long long> mx;
    mx.alloc(1, st);
    mx.zero(st);
    if (n > 0) {
        k_max_seg64<<<nblk(n, 256), 256, 0, st>>>(ptr, n, mx.p);
        NLFEM_LAUNCH_CHECK();
    }
    unsigned long long h = 0;
    NLFEM_CUDA_TRY(cudaMemcpyAsync(&h, mx.p, sizeof h, cudaMemcpyDeviceToHost, st));
    NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
    return (int64_t)h;
}

void build_pairs(Mesh& m, const Params& prm, PairCache& pc, cudaStream_t st) {
    const int64_t K = m.K;
    Grid g;
    // candidates lie within delta (sqrt(2) delta for the infinity ball) + 2 r_max of the centroid
    const double reach = prm.ball == NLFEM_BALL_INFINITY ? prm.delta * 1.4142135623730951 : prm.delta;
    // cells of half the reach plus two radii, searched over 5 x 5 blocks less the cells out of
    // reach: about 40% fewer candidates than 3 x 3 blocks of full-size cells
    const double cs0 = (reach + 2.0 * m.rmax) * (1.0 + 1e-9) + 1e-300;
    g.cs = 0.5 * cs0;
    g.span = 2;
    double W = m.bbox[2] - m.bbox[0], H = m.bbox[3] - m.bbox[1];
    g.nx = std::max(1, (int)std::ceil(W / g.cs));
    g.ny = std::max(1, (int)std::ceil(H / g.cs));
    // cap the grid at 2^24 cells by enlarging the cells (coarser cells stay correct)
    while ((int64_t)g.nx * g.ny > (1 << 24)) {
        g.cs *= 2.0;
        if (g.cs >= cs0) g.span = 1;
        g.nx = std::max(1, (int)std::ceil(W / g.cs));
        g.ny = std::max(1, (int)std::ceil(H / g.cs));
    }
    g.x0 = m.bbox[0];
    g.y0 = m.bbox[1];
    const int64_t ncell = (int64_t)g.nx * g.ny;
    DBuf<int64_t> ccount, cstart;
    DBuf<int> cell_of, cursor, clist;
    ccount.alloc(ncell, st);
    ccount.zero(st);
    cstart.alloc(ncell + 1, st);
    cell_of.alloc(K, st);
    clist.alloc(K, st);
    cursor.alloc(ncell, st);
    cursor.zero(st);
    k_bin_count<<<nblk(K, 256), 256, 0, st>>>(m.cen.p, K, g, ccount.p, cell_of.p);
    NLFEM_LAUNCH_CHECK();
    exclusive_scan_i64(ccount.p, cstart.p, ncell, st);
    k_bin_fill<<<nblk(K, 256), 256, 0, st>>>(cell_of.p, K, cstart.p, cursor.p, clist.p);
    NLFEM_LAUNCH_CHECK();

    SearchArgs a;
    a.X = m.X.p; a.T = m.T.p; a.cen = m.cen.p; a.rad = m.rad.p; a.cell_of = cell_of.p;
    a.cell_start = cstart.p; a.cell_list = clist.p; a.g = g; a.K = K;
    a.delta = prm.delta; a.delta2 = prm.delta2; a.caps = prm.ball == NLFEM_BALL_APPROXCAPS; a.ro = prm.ro;
    a.ball = prm.ball;
    a.reach = reach;
    a.rmax = m.rmax;
    a.Tp = m.tpos();
    a.E32 = m.E32.p;
    for (int i = 0; i < 16; ++i) {
        a.ol[i][0] = i < prm.ro.n ? (float)prm.ro.l[i][1] : 0.f;
        a.ol[i][1] = i < prm.ro.n ? (float)prm.ro.l[i][2] : 0.f;
    }
    a.delta32 = (float)prm.delta;
    a.d2f = (float)prm.delta * (float)prm.delta;

    DBuf<int64_t> cnt;
    cnt.alloc(K, st);
    pc.pair_ptr.alloc(K + 1, st);
    // the sorted candidate list of every cell's block; when the candidate-indexed slots fit
    // (8 GB) the search writes each partner list in order (no sort)
    DBuf<int64_t> bcnt, nptr;
    DBuf<int> nlist;
    bcnt.alloc(ncell, st);
    nptr.alloc(ncell + 1, st);
    k_block_count<<<nblk(ncell, 256), 256, 0, st>>>(g, cstart.p, bcnt.p);
    NLFEM_LAUNCH_CHECK();
    exclusive_scan_i64(bcnt.p, nptr.p, ncell, st);
    bcnt.release();
    int64_t ntot = 0;
    NLFEM_CUDA_TRY(cudaMemcpyAsync(&ntot, nptr.p + ncell, sizeof ntot, cudaMemcpyDeviceToHost, st));
    NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
    const int64_t ncap = max_segment_i64(nptr.p, ncell, st);
    const bool ordered = ntot < ((int64_t)1 << 31) && ncap <= 32768 &&
                         K * ncap * (int64_t)sizeof(int) <= ((int64_t)8 << 30);
    int64_t P = 0;
    DBuf<int> bpos, tslots;  // ordered search: positions in the candidate lists, transposed slots
    DBuf<unsigned long long> counts;
    counts.alloc(4, st);
    DBuf<int64_t> tcount;
    tcount.alloc(K, st);
    if (ordered) {
        nlist.alloc(std::max<int64_t>(ntot, 1), st);
        k_block_fill<<<nblk(ncell * 32, 256), 256, 0, st>>>(g, cstart.p, clist.p, nptr.p, nlist.p);
        NLFEM_LAUNCH_CHECK();
        segmented_sort_i32(nlist.p, nullptr, nptr.p, ncell, (int)ncap, st);
        DBuf<int> slot_buf;
        DBuf<int8_t> scls;
        slot_buf.alloc(std::max<int64_t>(K * ncap, 1), st);
        scls.alloc(std::max<int64_t>(K * ncap, 1), st);
        const int bw = 2 * g.span + 1;
        bpos.alloc(K * bw * bw, st);
        k_block_pos<<<nblk(ncell * 32, 256), 256, 0, st>>>(g, nptr.p, nlist.p, cell_of.p, bpos.p);
        NLFEM_LAUNCH_CHECK();
        k_search_ordered<<<nblk(K * 32, 128), 128, 0, st>>>(a, nptr.p, nlist.p, cnt.p, slot_buf.p, scls.p, ncap);
        NLFEM_LAUNCH_CHECK();
        exclusive_scan_i64(cnt.p, pc.pair_ptr.p, K, st);
        NLFEM_CUDA_TRY(cudaMemcpyAsync(&P, pc.pair_ptr.p + K, sizeof P, cudaMemcpyDeviceToHost, st));
        NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
        NLFEM_CHECK(P < ((int64_t)1 << 31), NLFEM_ERR_UNSUPPORTED, "more than 2^31 element pairs");
        pc.npairs = P;
        pc.pl.alloc(P, st);
        pc.pk.alloc(P, st);
        pc.pcls.alloc(P, st);
        counts.zero(st);
        tcount.zero(st);
        tslots.alloc(std::max<int64_t>(K * ncap, 1), st);
        NLFEM_CUDA_TRY(cudaMemsetAsync(tslots.p, 0xff, tslots.bytes(), st));  // -1: no pair
        k_compact_ordered<<<nblk(K * 32, 128), 128, 0, st>>>(slot_buf.p, scls.p, K, ncap, cell_of.p, nptr.p,
                                                             pc.pair_ptr.p, pc.pl.p, pc.pcls.p, counts.p, tcount.p,
                                                             g, bpos.p, tslots.p);
        NLFEM_LAUNCH_CHECK();
        slot_buf.release();
        scls.release();
        bpos.release();
    } else {
        // one pass into per-element slots when they fit (8 GB), else a count pass and a fill pass
        int64_t cap = 0;
        {
            DBuf<unsigned long long> mc;
            mc.alloc(1, st);
            mc.zero(st);
            k_max_cand<<<nblk(K, 256), 256, 0, st>>>(cell_of.p, K, g, cstart.p, mc.p);
            NLFEM_LAUNCH_CHECK();
            unsigned long long h = 0;
            NLFEM_CUDA_TRY(cudaMemcpyAsync(&h, mc.p, sizeof h, cudaMemcpyDeviceToHost, st));
            NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
            cap = (int64_t)h;
        }
        const bool slots = K * cap * (int64_t)sizeof(int) <= ((int64_t)8 << 30);
        DBuf<int> slot_buf;
        if (slots) {
            slot_buf.alloc(std::max<int64_t>(K * cap, 1), st);
            k_search<false, true><<<nblk(K * 32, 128), 128, 0, st>>>(a, cnt.p, nullptr, slot_buf.p, cap);
        } else {
            k_search<false><<<nblk(K * 32, 128), 128, 0, st>>>(a, cnt.p, nullptr, nullptr);
        }
        NLFEM_LAUNCH_CHECK();
        exclusive_scan_i64(cnt.p, pc.pair_ptr.p, K, st);
        NLFEM_CUDA_TRY(cudaMemcpyAsync(&P, pc.pair_ptr.p + K, sizeof P, cudaMemcpyDeviceToHost, st));
        NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
        NLFEM_CHECK(P < ((int64_t)1 << 31), NLFEM_ERR_UNSUPPORTED, "more than 2^31 element pairs");
        pc.npairs = P;
        pc.pl.alloc(P, st);
        pc.pk.alloc(P, st);
        if (slots) {
            k_compact_slots<<<nblk(K * 32, 128), 128, 0, st>>>(slot_buf.p, K, cap, pc.pair_ptr.p, pc.pl.p);
            slot_buf.release();
        } else {
            k_search<true><<<nblk(K * 32, 128), 128, 0, st>>>(a, nullptr, pc.pair_ptr.p, pc.pl.p);
        }
        NLFEM_LAUNCH_CHECK();
        int64_t mx = max_segment_i64(pc.pair_ptr.p, K, st);
        segmented_sort_i32(pc.pl.p, nullptr, pc.pair_ptr.p, K, (int)std::min<int64_t>(mx, 1 << 30), st);
    }
    k_fill_k<<<nblk(K * 32, 256), 256, 0, st>>>(pc.pair_ptr.p, K, pc.pk.p);
    NLFEM_LAUNCH_CHECK();

    // classification (the ordered search has done it) and the transposed index
    if (!ordered) {
        pc.pcls.alloc(P, st);
        counts.zero(st);
        tcount.zero(st);
        if (P) {
            k_classify<<<nblk(P, 256), 256, 0, st>>>(pc.pk.p, pc.pl.p, P, m.tpos(), pc.pcls.p, counts.p, tcount.p);
            NLFEM_LAUNCH_CHECK();
        }
    }
    pc.pT_ptr.alloc(K + 1, st);
    exclusive_scan_i64(tcount.p, pc.pT_ptr.p, K, st);
    pc.pT_id.alloc(P, st);
    if (ordered) {  // the transposed slots packed in order: lists by increasing pair id
        k_compact_transposed<<<nblk(K * 32, 128), 128, 0, st>>>(tslots.p, K, ncap, cell_of.p, nptr.p, pc.pT_ptr.p,
                                                                pc.pT_id.p);
        NLFEM_LAUNCH_CHECK();
        tslots.release();
    } else {  // placed by atomics, then sorted
        DBuf<int> tcur;
        tcur.alloc(K, st);
        tcur.zero(st);
        if (P) {
            k_fill_T<<<nblk(P, 256), 256, 0, st>>>(pc.pl.p, P, pc.pT_ptr.p, tcur.p, pc.pT_id.p);
            NLFEM_LAUNCH_CHECK();
        }
        int64_t mxT = max_segment_i64(pc.pT_ptr.p, K, st);
        segmented_sort_i32(pc.pT_id.p, nullptr, pc.pT_ptr.p, K, (int)std::min<int64_t>(mxT, 1 << 30), st);
    }
    unsigned long long hc[4];
    NLFEM_CUDA_TRY(cudaMemcpyAsync(hc, counts.p, sizeof hc, cudaMemcpyDeviceToHost, st));
    NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
    for (int i = 0; i < 4; ++i) pc.counts[i] = (int64_t)hc[i];

    // the work lists: whole and cut standard-rule pairs (the bulk kernels), intersecting pairs
    // under the singular rule (k_duffy) or the diamond rule (canonical k_trunc)
    pc.nwhole = pc.ncut = pc.nduffy = 0;
    pc.whole_ids.release();
    pc.cut_ids.release();
    pc.duffy_ids.release();
    if (P) {
        const int64_t nb = (P + LIST_BLOCK - 1) / LIST_BLOCK;
        DBuf<int8_t> code;
        DBuf<int64_t> bcount, boff;
        code.alloc(P, st);
        bcount.alloc(3 * nb, st);
        boff.alloc(3 * (nb + 1), st);
        k_list_flags<<<(unsigned)nb, LIST_THREADS, 0, st>>>(pc.pk.p, pc.pl.p, pc.pcls.p, P, m.X.p, m.T.p, m.rec.p,
                                                            prm.delta2, close_mode(prm) == 0,
                                                            prm.ball == NLFEM_BALL_INFINITY, prm.delta, code.p,
                                                            bcount.p);
        NLFEM_LAUNCH_CHECK();
        for (int i = 0; i < 3; ++i) exclusive_scan_i64(bcount.p + i * nb, boff.p + i * (nb + 1), nb, st);
        int64_t tot[3];
        for (int i = 0; i < 3; ++i)
            NLFEM_CUDA_TRY(cudaMemcpyAsync(&tot[i], boff.p + i * (nb + 1) + nb, sizeof(int64_t),
                                           cudaMemcpyDeviceToHost, st));
        NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
        pc.nwhole = tot[0];
        pc.ncut = tot[1];
        pc.nduffy = tot[2];
        pc.whole_ids.alloc(pc.nwhole, st);
        pc.cut_ids.alloc(pc.ncut, st);
        pc.duffy_ids.alloc(pc.nduffy, st);
        k_list_fill<<<(unsigned)nb, LIST_THREADS, 0, st>>>(code.p, P, boff.p, pc.whole_ids.p, pc.cut_ids.p,
                                                           pc.duffy_ids.p);
        NLFEM_LAUNCH_CHECK();
    }
}

}  // namespace nlfem

// ==========================================================================================
// nlfem_pairs_noalloc: the interaction graph of a small mesh without any device allocation.
//
// Every buffer the search needs beyond its inputs and outputs (oriented triangles,
// centroids, radii, FP32 edges, a vertex copy, grid cells, per-element counts and offsets)
// lives in g_noalloc_scratch below, a file-scope device array of NOALLOC_BYTES bytes that
// every GPU loading this library holds until the process exits. Host code never uses the
// array's name as an address: its device address is looked up once per device with
// cudaGetSymbolAddress (on the first call on that device, which should therefore come
// before any stream capture) and passed to the kernels. All calls share the array and it
// keeps the last call's contents, so each call clears the counters it needs; calls that
// overlap on the GPU (other streams, other host threads) race on it.
// ==========================================================================================
#include <mutex>

#include "rules_table.h"

namespace nlfem {

static constexpr int64_t NOALLOC_MAX_ELEMS = 32768;
static constexpr int64_t NOALLOC_MAX_VERTS = 65536;
static constexpr int64_t NOALLOC_MAX_CELLS = 65536;

// byte offsets of the sub-buffers (each a multiple of 256)
static constexpr size_t NA_X = 0;                                              // double2[MAX_VERTS]
static constexpr size_t NA_T = NA_X + 16 * NOALLOC_MAX_VERTS;                  // int4[MAX_ELEMS]
static constexpr size_t NA_CEN = NA_T + 16 * NOALLOC_MAX_ELEMS;                // double2[MAX_ELEMS]
static constexpr size_t NA_RAD = NA_CEN + 16 * NOALLOC_MAX_ELEMS;              // double[MAX_ELEMS]
static constexpr size_t NA_E32 = NA_RAD + 8 * NOALLOC_MAX_ELEMS;               // float4[MAX_ELEMS]
static constexpr size_t NA_CELLOF = NA_E32 + 16 * NOALLOC_MAX_ELEMS;           // int[MAX_ELEMS]
static constexpr size_t NA_CLIST = NA_CELLOF + 4 * NOALLOC_MAX_ELEMS;          // int[MAX_ELEMS]
static constexpr size_t NA_CNT = NA_CLIST + 4 * NOALLOC_MAX_ELEMS;             // int64[MAX_ELEMS]
static constexpr size_t NA_PTR = NA_CNT + 8 * NOALLOC_MAX_ELEMS;               // int64[MAX_ELEMS + 1], padded
static constexpr size_t NA_CCNT = NA_PTR + 8 * NOALLOC_MAX_ELEMS + 256;        // int64[MAX_CELLS]
static constexpr size_t NA_CSTART = NA_CCNT + 8 * NOALLOC_MAX_CELLS;           // int64[MAX_CELLS + 1], padded
static constexpr size_t NA_CCUR = NA_CSTART + 8 * NOALLOC_MAX_CELLS + 256;     // int[MAX_CELLS]
static constexpr size_t NA_MISC = NA_CCUR + 4 * NOALLOC_MAX_CELLS;             // 256 bytes: flags, stats
static constexpr size_t NOALLOC_BYTES = NA_MISC + 256;
static_assert(NOALLOC_BYTES == 4981504, "the header states the scratch size: 4,981,504 bytes");

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

// per-device address of g_noalloc_scratch, looked up on the first call on that device
static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[256];

static unsigned char* noalloc_scratch() {
    int dev = 0;
    NLFEM_CUDA_TRY(cudaGetDevice(&dev));
    NLFEM_CHECK(dev >= 0 && dev < 256, NLFEM_ERR_UNSUPPORTED, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        NLFEM_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        NLFEM_CHECK(p != nullptr, NLFEM_ERR_CUDA, "cudaGetSymbolAddress returned NULL for the scratch array");
        g_noalloc_addr[dev] = p;
    }
    return (unsigned char*)g_noalloc_addr[dev];
}

// misc block: [0] int error flags, [1] int max count, then doubles at +16: rmax, xmin, ymin, xmax, ymax
__global__ void k_na_init(unsigned char* misc) {
    int* fl = (int*)misc;
    fl[0] = 0;
    fl[1] = 0;
    double* st = (double*)(misc + 16);
    st[0] = 0.0;
    st[1] = 1e300;
    st[2] = 1e300;
    st[3] = -1e300;
    st[4] = -1e300;
}

__device__ __forceinline__ void na_atomic_max_d(double* a, double v) {
    unsigned long long* p = (unsigned long long*)a;
    unsigned long long old = *p, assumed;
    while (__longlong_as_double(old) < v) {
        assumed = old;
        old = atomicCAS(p, assumed, __double_as_longlong(v));
        if (old == assumed) break;
    }
}
__device__ __forceinline__ void na_atomic_min_d(double* a, double v) {
    unsigned long long* p = (unsigned long long*)a;
    unsigned long long old = *p, assumed;
    while (__longlong_as_double(old) > v) {
        assumed = old;
        old = atomicCAS(p, assumed, __double_as_longlong(v));
        if (old == assumed) break;
    }
}

__global__ void k_na_verts(const double* verts, int64_t M, double2* X, unsigned char* misc) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    double2 v = make_double2(verts[2 * i], verts[2 * i + 1]);
    X[i] = v;
    double* st = (double*)(misc + 16);
    na_atomic_min_d(&st[1], v.x);
    na_atomic_min_d(&st[2], v.y);
    na_atomic_max_d(&st[3], v.x);
    na_atomic_max_d(&st[4], v.y);
}

// same orientation arithmetic as the mesh upload (CCW by the sign of the FP64 determinant)
__global__ void k_na_elems(const int* T3, int64_t K, int64_t M, const double2* X, int4* T, double2* cen,
                           double* rad, float4* E32, unsigned char* misc) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    int* fl = (int*)misc;
    double* st = (double*)(misc + 16);
    int t0 = T3[3 * k], t1 = T3[3 * k + 1], t2 = T3[3 * k + 2];
    if (t0 < 0 || t1 < 0 || t2 < 0 || t0 >= M || t1 >= M || t2 >= M) {
        atomicOr(&fl[0], 1);
        T[k] = make_int4(0, 0, 0, 0);
        cen[k] = make_double2(0.0, 0.0);
        rad[k] = 0.0;
        E32[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    double2 a = X[t0], b = X[t1], c = X[t2];
    double d = __dsub_rn(__dmul_rn(__dsub_rn(b.x, a.x), __dsub_rn(c.y, a.y)),
                         __dmul_rn(__dsub_rn(b.y, a.y), __dsub_rn(c.x, a.x)));
    if (d < 0) {
        int tt = t1; t1 = t2; t2 = tt;
        double2 cc = b; b = c; c = cc;
        d = -d;
    }
    if (!(d > 0)) atomicOr(&fl[0], 2);
    T[k] = make_int4(t0, t1, t2, 0);
    E32[k] = make_float4((float)(b.x - a.x), (float)(b.y - a.y), (float)(c.x - a.x), (float)(c.y - a.y));
    double2 ce = make_double2((a.x + b.x + c.x) / 3.0, (a.y + b.y + c.y) / 3.0);
    cen[k] = ce;
    double r = sqrt(fmax(fmax((a.x - ce.x) * (a.x - ce.x) + (a.y - ce.y) * (a.y - ce.y),
                              (b.x - ce.x) * (b.x - ce.x) + (b.y - ce.y) * (b.y - ce.y)),
                         (c.x - ce.x) * (c.x - ce.x) + (c.y - ce.y) * (c.y - ce.y)));
    rad[k] = r;
    na_atomic_max_d(&st[0], r);
}

// exclusive scan of n <= 65536 int64 values in one block (out[n] = total)
__global__ void k_na_scan(const int64_t* in, int64_t* out, int64_t n) {
    __shared__ int64_t part[1024];
    const int per = (int)((n + 1023) / 1024);
    const int64_t b = (int64_t)threadIdx.x * per;
    int64_t s = 0;
    for (int i = 0; i < per; ++i)
        if (b + i < n) s += in[b + i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        int64_t t = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += t;
        __syncthreads();
    }
    int64_t run = part[threadIdx.x] - s;
    for (int i = 0; i < per; ++i)
        if (b + i < n) {
            out[b + i] = run;
            run += in[b + i];
        }
    if (threadIdx.x == 1023) out[n] = part[1023];
}

__global__ void k_na_maxcnt(const int64_t* cnt, int64_t K, unsigned char* misc) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < K) atomicMax(&((int*)misc)[1], (int)cnt[k]);
}

}  // namespace nlfem

extern "C" int nlfem_pairs_noalloc(const double* verts, int64_t M, const int32_t* elems, int64_t K, double delta,
                                   int ball, int quad_outer, int32_t* out_k, int32_t* out_l, int64_t capacity,
                                   int64_t* npairs, void* stream) {
    using namespace nlfem;
    try {
        set_error("");
        NLFEM_CHECK(verts && elems && out_k && out_l && npairs, NLFEM_ERR_INVALID_ARG, "NULL argument");
        *npairs = 0;
        NLFEM_CHECK(M >= 3 && K >= 1 && capacity >= 0, NLFEM_ERR_INVALID_ARG, "need M >= 3, K >= 1, capacity >= 0");
        NLFEM_CHECK(K <= NOALLOC_MAX_ELEMS && M <= NOALLOC_MAX_VERTS, NLFEM_ERR_UNSUPPORTED,
                    "nlfem_pairs_noalloc handles at most 32768 triangles and 65536 vertices (got " +
                        std::to_string(K) + " triangles, " + std::to_string(M) +
                        " vertices); use nlfem_mesh_create and nlfem_assemble for larger meshes");
        NLFEM_CHECK(delta > 0 && std::isfinite(delta), NLFEM_ERR_INVALID_ARG, "delta must be > 0");
        NLFEM_CHECK(ball == NLFEM_BALL_NOCAPS || ball == NLFEM_BALL_APPROXCAPS || ball == NLFEM_BALL_INFINITY,
                    NLFEM_ERR_INVALID_ARG, "unknown ball");
        NLFEM_CHECK(quad_outer == 7 || quad_outer == 16, NLFEM_ERR_INVALID_ARG, "quad_outer must be 7 or 16");
        const void* devp[4] = {verts, elems, out_k, out_l};
        for (const void* q : devp) {
            cudaPointerAttributes at;
            cudaError_t e = cudaPointerGetAttributes(&at, q);
            if (e != cudaSuccess) (void)cudaGetLastError();
            NLFEM_CHECK(e == cudaSuccess && (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged),
                        NLFEM_ERR_INVALID_ARG, "verts, elems, out_k and out_l must be device memory");
        }
        cudaStream_t st = (cudaStream_t)stream;
        unsigned char* base = noalloc_scratch();
        double2* X = (double2*)(base + NA_X);
        int4* T = (int4*)(base + NA_T);
        double2* cen = (double2*)(base + NA_CEN);
        double* rad = (double*)(base + NA_RAD);
        float4* E32 = (float4*)(base + NA_E32);
        int* cell_of = (int*)(base + NA_CELLOF);
        int* clist = (int*)(base + NA_CLIST);
        int64_t* cnt = (int64_t*)(base + NA_CNT);
        int64_t* ptr = (int64_t*)(base + NA_PTR);
        int64_t* ccnt = (int64_t*)(base + NA_CCNT);
        int64_t* cstart = (int64_t*)(base + NA_CSTART);
        int* ccur = (int*)(base + NA_CCUR);
        unsigned char* misc = base + NA_MISC;

        k_na_init<<<1, 1, 0, st>>>(misc);
        NLFEM_LAUNCH_CHECK();
        k_na_verts<<<nblk(M, 256), 256, 0, st>>>(verts, M, X, misc);
        NLFEM_LAUNCH_CHECK();
        k_na_elems<<<nblk(K, 256), 256, 0, st>>>(elems, K, M, X, T, cen, rad, E32, misc);
        NLFEM_LAUNCH_CHECK();
        int hfl[2];
        double hs[5];
        NLFEM_CUDA_TRY(cudaMemcpyAsync(hfl, misc, sizeof hfl, cudaMemcpyDeviceToHost, st));
        NLFEM_CUDA_TRY(cudaMemcpyAsync(hs, misc + 16, sizeof hs, cudaMemcpyDeviceToHost, st));
        NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
        NLFEM_CHECK(!(hfl[0] & 1), NLFEM_ERR_BAD_MESH, "triangle vertex index out of range");
        NLFEM_CHECK(!(hfl[0] & 2), NLFEM_ERR_BAD_MESH, "triangle with zero area");

        // grid over the element centroids, at most NOALLOC_MAX_CELLS cells
        Grid g;
        const double reach = ball == NLFEM_BALL_INFINITY ? delta * 1.4142135623730951 : delta;
        g.cs = (reach + 2.0 * hs[0]) * (1.0 + 1e-9) + 1e-300;
        g.span = 1;
        const double W = hs[3] - hs[1], H = hs[4] - hs[2];
        g.nx = std::max(1, (int)std::ceil(W / g.cs));
        g.ny = std::max(1, (int)std::ceil(H / g.cs));
        while ((int64_t)g.nx * g.ny > NOALLOC_MAX_CELLS) {
            g.cs *= 2.0;
            g.nx = std::max(1, (int)std::ceil(W / g.cs));
            g.ny = std::max(1, (int)std::ceil(H / g.cs));
        }
        g.x0 = hs[1];
        g.y0 = hs[2];
        const int64_t ncell = (int64_t)g.nx * g.ny;
        NLFEM_CUDA_TRY(cudaMemsetAsync(ccnt, 0, 8 * ncell, st));
        NLFEM_CUDA_TRY(cudaMemsetAsync(ccur, 0, 4 * ncell, st));
        k_bin_count<<<nblk(K, 256), 256, 0, st>>>(cen, K, g, ccnt, cell_of);
        NLFEM_LAUNCH_CHECK();
        k_na_scan<<<1, 1024, 0, st>>>(ccnt, cstart, ncell);
        NLFEM_LAUNCH_CHECK();
        k_bin_fill<<<nblk(K, 256), 256, 0, st>>>(cell_of, K, cstart, ccur, clist);
        NLFEM_LAUNCH_CHECK();

        SearchArgs a;
        a.X = X; a.T = T; a.cen = cen; a.rad = rad; a.cell_of = cell_of; a.cell_start = cstart; a.cell_list = clist;
        a.g = g; a.K = K; a.delta = delta; a.delta2 = delta * delta; a.caps = ball == NLFEM_BALL_APPROXCAPS;
        a.reach = reach; a.rmax = hs[0];
        a.ball = ball;
        a.Tp = T;
        a.ro.n = quad_outer;
        const double(*tab)[4] = quad_outer == 7 ? NLFEM_RULE7 : NLFEM_RULE16;
        for (int i = 0; i < 16; ++i) {
            for (int j = 0; j < 3; ++j) a.ro.l[i][j] = i < quad_outer ? tab[i][j] : 0.0;
            a.ro.w[i] = i < quad_outer ? tab[i][3] : 0.0;
            a.ol[i][0] = i < quad_outer ? (float)tab[i][1] : 0.f;
            a.ol[i][1] = i < quad_outer ? (float)tab[i][2] : 0.f;
        }
        a.E32 = E32;
        a.delta32 = (float)delta;
        a.d2f = (float)delta * (float)delta;
        k_search<false><<<nblk(K * 32, 128), 128, 0, st>>>(a, cnt, nullptr, nullptr);
        NLFEM_LAUNCH_CHECK();
        k_na_scan<<<1, 1024, 0, st>>>(cnt, ptr, K);
        NLFEM_LAUNCH_CHECK();
        k_na_maxcnt<<<nblk(K, 256), 256, 0, st>>>(cnt, K, misc);
        NLFEM_LAUNCH_CHECK();
        int64_t total = 0;
        int mx = 0;
        NLFEM_CUDA_TRY(cudaMemcpyAsync(&total, ptr + K, sizeof total, cudaMemcpyDeviceToHost, st));
        NLFEM_CUDA_TRY(cudaMemcpyAsync(&mx, misc + 4, sizeof mx, cudaMemcpyDeviceToHost, st));
        NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
        *npairs = total;
        NLFEM_CHECK(total <= capacity, NLFEM_ERR_INVALID_ARG,
                    "out_k / out_l hold " + std::to_string(capacity) + " pairs, the mesh has " +
                        std::to_string(total) + " (returned in *npairs)");
        k_search<true><<<nblk(K * 32, 128), 128, 0, st>>>(a, nullptr, ptr, out_l);
        NLFEM_LAUNCH_CHECK();
        segmented_sort_i32(out_l, nullptr, ptr, K, mx, st);
        k_fill_k<<<nblk(K * 32, 256), 256, 0, st>>>(ptr, K, out_k);
        NLFEM_LAUNCH_CHECK();
        NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
        return NLFEM_OK;
    } catch (const Error& e) {
        set_error(e.msg);
        return e.code;
    } catch (...) {
        set_error("unexpected exception");
        return NLFEM_ERR_CUDA;
    }
}
