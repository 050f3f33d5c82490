/*
 * nlfem oracle: plain FP64 CPU assembler for the 2D nonlocal P1 stiffness
 * matrix and load vector of arXiv 2207.03921 (Klar, Vollmann, Schulz).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the independent reference the CUDA
 * path is checked against. Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load it. It shares no code,
 * header or table with the CUDA library, and it never calls it.
 *
 * What it computes, in the paper's order and notation:
 *   - mesh normalisation: CCW triangles, element labels, Dirichlet nodes (Sec. 2.2)
 *   - the interaction search by breadth-first traversal of the adjacency graph
 *     T_adj, enqueuing a neighbour iff its local contribution is nonzero (Alg. 2)
 *   - per ordered pair (E_k, E_l): Alg. 1. Singular kernel on intersecting pairs:
 *     regularising transforms to (0,1)^4 with a tensor Gauss rule (Sec. 2.3.2,
 *     Tab. 1 "club"). Otherwise the truncation quadrature (Sec. 2.3.1, eq.
 *     discrete-inner): per outer point x_p, E_l cut by the ball approximation
 *     (nocaps Def. 2.1 / approxcaps Def. 2.2) is retriangulated and the inner
 *     rule is put on every sub-triangle; basis values are evaluated at run time.
 *   - the approximate bilinear form A_h^# (eq. biFormApprox) in the symmetric
 *     weak form (eq. weakL) for a symmetric kernel: the integrand is
 *     (phi_i(x)-phi_i(y))^T Psi(x,y) (phi_j(x)-phi_j(y)).
 *   - kernels of Sec. 3: constant, truncated fractional (eq. fractional-scaling),
 *     bond-based peridynamics (eq. ker:peridynamics).
 *   - CSR accumulation of every ordered pair's block (Sec. 2.4 / 3.4), and the
 *     load vector F_i = int_Omega f phi_i with the outer rule.
 *
 * Arithmetic: FP64, compiled with -ffp-contract=off. The geometric decisions
 * (vertex in ball, edge crossings, cap centres) use the operation order written
 * out in the comments of clip_ball(); they decide the interaction pattern.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORC_K_CONST = 0, ORC_K_FRAC = 1, ORC_K_PERI = 2, ORC_K_TAB = 3 };
#define MAXTAB 1024
enum { ORC_BALL_NOCAPS = 0, ORC_BALL_APPROXCAPS = 1, ORC_BALL_INF = 2 };
enum { ORC_CLOSE_AUTO = 0, ORC_CLOSE_DUFFY = 1, ORC_CLOSE_NOZERODIV = 2, ORC_CLOSE_STANDARD = 3 };
enum { ORC_PAIRS_BFS = 0, ORC_PAIRS_BRUTE = 1 };

#define MAXQ 64
#define MAXPOLY 16
#define CLIP_TAU 1e-12
#define CLIP_CAP_MIN 1e-9

typedef struct {
    int n;
    double l[MAXQ][3]; /* barycentric coordinates of the points on the reference triangle */
    double w[MAXQ];    /* weights; they sum to 1/2, the reference area */
} rule_t;

typedef struct {
    int kernel, ball, close_rule, ndof;
    double delta, delta2, s, c;
    rule_t ro, ri;        /* outer (x) and inner (y) rules */
    int ng;               /* Gauss-Legendre points per direction on (0,1) for the transforms */
    double gx[64], gw[64];
    int ntab;             /* user kernel: values g(r_i) at r_i = i delta / (ntab - 1) */
    double tab[MAXTAB];
} params_t;

typedef struct {
    int M, K;
    const double *X;   /* M x 2 */
    int *T;            /* K x 3, counter-clockwise */
    double *det;       /* |det J_k| = 2 |E_k| */
    signed char *lab;  /* 1 = Omega */
    signed char *dir;  /* node is Dirichlet */
    int *ne_ptr, *ne_idx; /* position -> elements (nodes at the same point share one entry) */
    int *pos;          /* node -> its position: the smallest node id with the same coordinates */
} mesh_t;

typedef struct {
    long long evals;         /* kernel evaluations in the truncation quadrature */
    long long cut_points;    /* outer points whose inner element was retriangulated */
    long long full_points;   /* outer points whose inner element was fully inside */
    long long subtris;       /* sub-triangles integrated (cut case) */
    long long duffy_points;  /* points of the singular quadrature */
    long long pairs, pairs_identical, pairs_edge, pairs_vertex, pairs_separated;
} counts_t;

/* ---------------------------------------------------------------------------------------
 * Small helpers
 * ------------------------------------------------------------------------------------- */

static double det2(double ax, double ay, double bx, double by) { return ax * by - ay * bx; }

/* Physical point of barycentric coordinates l on triangle (v0, v1, v2):
 * x = (l0*v0 + l1*v1) + l2*v2, each product and sum rounded separately. */
static void map_point(const double V[3][2], const double *l, double *x, double *y)
{
    *x = (l[0] * V[0][0] + l[1] * V[1][0]) + l[2] * V[2][0];
    *y = (l[0] * V[0][1] + l[1] * V[1][1]) + l[2] * V[2][1];
}

static void elem_verts(const mesh_t *m, int k, double V[3][2])
{
    for (int a = 0; a < 3; ++a) {
        V[a][0] = m->X[2 * m->T[3 * k + a]];
        V[a][1] = m->X[2 * m->T[3 * k + a] + 1];
    }
}

/* Barycentric coordinates of (x, y) with respect to triangle V. */
static void barycentric(const double V[3][2], double x, double y, double *b)
{
    double d = det2(V[1][0] - V[0][0], V[1][1] - V[0][1], V[2][0] - V[0][0], V[2][1] - V[0][1]);
    double b1 = det2(x - V[0][0], y - V[0][1], V[2][0] - V[0][0], V[2][1] - V[0][1]) / d;
    double b2 = det2(V[1][0] - V[0][0], V[1][1] - V[0][1], x - V[0][0], y - V[0][1]) / d;
    b[0] = 1.0 - b1 - b2;
    b[1] = b1;
    b[2] = b2;
}

/* ---------------------------------------------------------------------------------------
 * Ball approximations (Sec. 2.2, Defs. 2.1 and 2.2)
 *
 * E_l cut by the ball around c. Walk the CCW boundary v0->v1->v2->v0. On edge a->b:
 *   - emit a if it lies in the closed ball:
 *       dx = ax - cx; dy = ay - cy; inside iff (dx*dx + dy*dy) <= delta2, delta2 = delta*delta
 *   - then the crossings with the circle at parameters t in (0,1), increasing:
 *       ux = bx - ax; uy = by - ay; ex = ax - cx; ey = ay - cy
 *       A = ux*ux + uy*uy; B = ex*ux + ey*uy; C = (ex*ex + ey*ey) - delta2
 *       disc = B*B - A*C; if disc > 0: r = sqrt(disc), t1 = (-B - r)/A, t2 = (-B + r)/A
 *       point = (ax + t*ux, ay + t*uy)
 *   - a root with t < TAU or t > 1 - TAU (TAU = 1e-12) is the circle passing through
 *     the edge's end vertex: that vertex is emitted instead of the crossing.
 * Consecutive points that coincide exactly are merged, keeping the vertex if one
 * of them is a vertex and otherwise the later one.
 * nocaps: the convex polygon of these points.
 * approxcaps: between consecutive points P -> Q that are not joined by a piece of
 * one edge (a vertex outside the ball lies between them on the boundary), insert
 * the cap centre m = c + delta * n, n the unit right-hand normal of the chord
 * P -> Q:  qx = Qx - Px; qy = Qy - Py; len = sqrt(qx*qx + qy*qy);
 *          m = (cx + delta*(qy/len), cy + delta*(-qx/len));
 * no cap is inserted on a chord with len <= 1e-9 * delta (its cap has no area).
 * Returns the number of polygon points; *full = 1 when all three vertices are
 * inside (the element is integrated whole with its own rule).
 * ------------------------------------------------------------------------------------- */
typedef struct { double x, y; int e; double t; int vert; } bpt_t;

static int joined(const bpt_t *P, const bpt_t *Q)
{
    if (Q->e == P->e && Q->t > P->t) return 1;
    if (Q->vert && Q->e == (P->e + 1) % 3) return 1;
    return 0;
}

int orc_clip_ball(const double V[3][2], double cx, double cy, double delta, double delta2,
                  int caps, double out[][2], int *full)
{
    bpt_t raw[12];
    int n = 0;
    int inside[3];
    for (int a = 0; a < 3; ++a) {
        double dx = V[a][0] - cx, dy = V[a][1] - cy;
        inside[a] = (dx * dx + dy * dy) <= delta2;
    }
    if (inside[0] && inside[1] && inside[2]) {
        *full = 1;
        for (int a = 0; a < 3; ++a) { out[a][0] = V[a][0]; out[a][1] = V[a][1]; }
        return 3;
    }
    *full = 0;
    for (int e = 0; e < 3; ++e) {
        const double *A_ = V[e], *B_ = V[(e + 1) % 3];
        bpt_t cand[4];
        int nc = 0;
        if (inside[e]) { cand[nc].x = A_[0]; cand[nc].y = A_[1]; cand[nc].e = e; cand[nc].t = 0.0; cand[nc].vert = 1; ++nc; }
        double ux = B_[0] - A_[0], uy = B_[1] - A_[1];
        double ex = A_[0] - cx, ey = A_[1] - cy;
        double A = ux * ux + uy * uy;
        double B = ex * ux + ey * uy;
        double C = (ex * ex + ey * ey) - delta2;
        double disc = B * B - A * C;
        if (disc > 0.0) {
            double r = sqrt(disc);
            double t1 = (-B - r) / A, t2 = (-B + r) / A;
            double ts[2] = {t1, t2};
            for (int r2 = 0; r2 < 2; ++r2) {
                double t = ts[r2];
                if (!(t > 0.0 && t < 1.0)) continue;
                if (t < CLIP_TAU) {                 /* the circle passes through a */
                    cand[nc].x = A_[0]; cand[nc].y = A_[1]; cand[nc].e = e; cand[nc].t = 0.0; cand[nc].vert = 1;
                } else if (t > 1.0 - CLIP_TAU) {    /* ... through b, the next edge's start */
                    cand[nc].x = B_[0]; cand[nc].y = B_[1]; cand[nc].e = (e + 1) % 3; cand[nc].t = 0.0; cand[nc].vert = 1;
                } else {
                    cand[nc].x = A_[0] + t * ux; cand[nc].y = A_[1] + t * uy; cand[nc].e = e; cand[nc].t = t; cand[nc].vert = 0;
                }
                ++nc;
            }
        }
        for (int i = 0; i < nc; ++i) {
            if (n > 0 && raw[n - 1].x == cand[i].x && raw[n - 1].y == cand[i].y) {
                if (raw[n - 1].vert && !cand[i].vert) continue; /* keep the vertex */
                raw[n - 1] = cand[i];                            /* keep the later one */
            } else {
                raw[n++] = cand[i];
            }
        }
    }
    if (n >= 2 && raw[n - 1].x == raw[0].x && raw[n - 1].y == raw[0].y) {
        if (raw[n - 1].vert && !raw[0].vert) raw[0] = raw[n - 1];
        --n;
    }
    int m = 0;
    for (int i = 0; i < n; ++i) {
        out[m][0] = raw[i].x; out[m][1] = raw[i].y; ++m;
        if (caps && n >= 2) {
            const bpt_t *P = &raw[i], *Q = &raw[(i + 1) % n];
            if (!joined(P, Q)) {
                double qx = Q->x - P->x, qy = Q->y - P->y;
                double len = sqrt(qx * qx + qy * qy);
                if (len > CLIP_CAP_MIN * delta) {
                    out[m][0] = cx + delta * (qy / len);
                    out[m][1] = cy + delta * (-qx / len);
                    ++m;
                }
            }
        }
    }
    return m;
}

/* ---------------------------------------------------------------------------------------
 * Infinity norm ball (Sec. 2.2, Def. of the infinity norm ball): E_l cut by the closed square
 * {y : |y - c|_inf <= delta} exactly. Sutherland-Hodgman clipping of the CCW triangle by the
 * four half-planes x <= delta, y <= delta, x >= -delta, y >= -delta, in this order, in
 * coordinates relative to c:
 *   p = (vx - cx, vy - cy) per vertex, each difference rounded once;
 *   half-plane (axis a, sign s): inside iff s * p[a] <= delta;
 *   one pass walks S -> E over consecutive points, starting with S = the last point and
 *   E = the first; where S and E lie on different sides it emits the crossing
 *     t = (s*delta - S[a]) / (E[a] - S[a]),  X[a] = s*delta,  X[b] = S[b] + t * (E[b] - S[b])
 *   (b the other axis), then E itself if E is inside.
 * Afterwards consecutive points that coincide exactly (also the last and the first) are
 * merged; fewer than 3 points mean an empty intersection. full = every vertex inside all four
 * half-planes (the element is integrated whole with its own rule). The points are returned
 * in absolute coordinates c + p.
 * ------------------------------------------------------------------------------------- */
static int sh_pass(double in[][2], int n, int a, double s, double delta, double out[][2])
{
    int m = 0;
    if (n == 0) return 0;
    const int b = 1 - a;
    const double *S = in[n - 1];
    int s_in = s * S[a] <= delta;
    for (int i = 0; i < n; ++i) {
        const double *E = in[i];
        int e_in = s * E[a] <= delta;
        if (e_in != s_in) {
            double t = (s * delta - S[a]) / (E[a] - S[a]);
            out[m][a] = s * delta;
            out[m][b] = S[b] + t * (E[b] - S[b]);
            ++m;
        }
        if (e_in) { out[m][0] = E[0]; out[m][1] = E[1]; ++m; }
        S = E;
        s_in = e_in;
    }
    return m;
}

int orc_clip_square(const double V[3][2], double cx, double cy, double delta, double out[][2], int *full)
{
    double A[MAXPOLY][2], B[MAXPOLY][2];
    int all_in = 1;
    for (int v = 0; v < 3; ++v) {
        A[v][0] = V[v][0] - cx;
        A[v][1] = V[v][1] - cy;
        all_in &= fabs(A[v][0]) <= delta && fabs(A[v][1]) <= delta;
    }
    if (all_in) {
        *full = 1;
        for (int v = 0; v < 3; ++v) { out[v][0] = V[v][0]; out[v][1] = V[v][1]; }
        return 3;
    }
    *full = 0;
    int n = 3;
    n = sh_pass(A, n, 0, 1.0, delta, B);
    n = sh_pass(B, n, 1, 1.0, delta, A);
    n = sh_pass(A, n, 0, -1.0, delta, B);
    n = sh_pass(B, n, 1, -1.0, delta, A);
    int m = 0;
    for (int i = 0; i < n; ++i) {
        if (m > 0 && A[i][0] == B[m - 1][0] && A[i][1] == B[m - 1][1]) continue;
        B[m][0] = A[i][0]; B[m][1] = A[i][1]; ++m;
    }
    while (m >= 2 && B[m - 1][0] == B[0][0] && B[m - 1][1] == B[0][1]) --m;
    if (m < 3) return 0;
    for (int i = 0; i < m; ++i) { out[i][0] = cx + B[i][0]; out[i][1] = cy + B[i][1]; }
    return m;
}

/* ---------------------------------------------------------------------------------------
 * Kernels (Sec. 3): value of gamma (scalar) or the 2x2 matrix Gamma (peridynamics)
 * at z = y - x.
 * ------------------------------------------------------------------------------------- */
/* User-defined radial kernel gamma = c g(|z|), g interpolated linearly between its values at
 * r_i = i delta / (n - 1) and held at g(delta) beyond delta (the Conclusion: kernels supplied
 * by the user; here as a table instead of compiled code). */
static double gamma_table(const params_t *P, double zx, double zy)
{
    double r = sqrt(zx * zx + zy * zy);
    double t = r * ((double)(P->ntab - 1) / P->delta);
    int i = (int)t;
    if (i >= P->ntab - 1) return P->c * P->tab[P->ntab - 1];
    double w = t - i;
    return P->c * ((1.0 - w) * P->tab[i] + w * P->tab[i + 1]);
}

static double gamma_scalar(const params_t *P, double zx, double zy)
{
    if (P->kernel == ORC_K_CONST) return P->c;
    if (P->kernel == ORC_K_TAB) return gamma_table(P, zx, zy);
    double r2 = zx * zx + zy * zy;
    return P->c * pow(r2, -1.0 - P->s); /* c |z|^(-2-2s) */
}

static void gamma_peri(const params_t *P, double zx, double zy, double G[3])
{
    double r2 = zx * zx + zy * zy;
    double r3 = r2 * sqrt(r2);
    G[0] = P->c * zx * zx / r3; /* c z z^T / |z|^3 */
    G[1] = P->c * zx * zy / r3;
    G[2] = P->c * zy * zy / r3;
}

/* ---------------------------------------------------------------------------------------
 * Local block of one ordered pair on its union vertices.
 * blk is U*ndof x U*ndof, row-major; union vertex u has dofs u*ndof + comp.
 * ------------------------------------------------------------------------------------- */
typedef struct {
    int U;
    int node[6];
    double blk[12 * 12];
} block_t;

/* union of the vertex lists: E_k's vertices, then E_l's vertices not in E_k */
static int union_nodes(const int *tk, const int *tl, int *node, int *posl)
{
    int U = 3;
    node[0] = tk[0]; node[1] = tk[1]; node[2] = tk[2];
    for (int b = 0; b < 3; ++b) {
        int f = -1;
        for (int a = 0; a < 3; ++a) if (tl[b] == tk[a]) f = a;
        if (f >= 0) posl[b] = f;
        else { node[U] = tl[b]; posl[b] = U; ++U; }
    }
    return U;
}

/* Add w * dk dk^T structure: for scalar problems
 *   block(u,v) += w * D[u] * D[v], with D = phi(x) - phi(y) on the union vertices.
 * For peridynamics the 2x2 Gamma replaces w. */
static void add_outer(block_t *B, int ndof, const double *D, double w, const double *G)
{
    int n = B->U * ndof;
    for (int u = 0; u < B->U; ++u) {
        if (D[u] == 0.0) continue;
        for (int v = 0; v < B->U; ++v) {
            if (D[v] == 0.0) continue;
            double dd = D[u] * D[v];
            if (ndof == 1) {
                B->blk[u * n + v] += w * dd;
            } else {
                B->blk[(2 * u) * n + 2 * v] += w * G[0] * dd;
                B->blk[(2 * u) * n + 2 * v + 1] += w * G[1] * dd;
                B->blk[(2 * u + 1) * n + 2 * v] += w * G[1] * dd;
                B->blk[(2 * u + 1) * n + 2 * v + 1] += w * G[2] * dd;
            }
        }
    }
}

/* Truncation quadrature (Sec. 2.3.1), the "heart" and "diamond" rules of Tab. 1.
 * Returns 1 if some outer point sees a nonempty polygon (the pair interacts). */
static int pair_truncation(const mesh_t *m, const params_t *P, int k, int l, int posl[3],
                           block_t *B, int accumulate, int nozerodiv, counts_t *cnt)
{
    double Vk[3][2], Vl[3][2];
    elem_verts(m, k, Vk);
    elem_verts(m, l, Vl);
    int interacts = 0;
    double poly[MAXPOLY][2];
    for (int p = 0; p < P->ro.n; ++p) {
        double xp, yp;
        map_point(Vk, P->ro.l[p], &xp, &yp);
        int full = 0;
        int np = P->ball == ORC_BALL_INF
                     ? orc_clip_square(Vl, xp, yp, P->delta, poly, &full)
                     : orc_clip_ball(Vl, xp, yp, P->delta, P->delta2, P->ball == ORC_BALL_APPROXCAPS, poly, &full);
        if (np < 3) continue;
        interacts = 1;
        if (!accumulate) return 1;
        double ap = P->ro.w[p] * m->det[k];
        const double *Pk = P->ro.l[p]; /* phi_a(x_p) for a in E_k */
        if (full) cnt->full_points++; else cnt->cut_points++;
        int ntri = full ? 1 : np - 2;
        for (int t = 0; t < ntri; ++t) {
            double T3[3][2];
            if (full) memcpy(T3, Vl, sizeof T3);
            else {
                T3[0][0] = poly[0][0]; T3[0][1] = poly[0][1];
                T3[1][0] = poly[t + 1][0]; T3[1][1] = poly[t + 1][1];
                T3[2][0] = poly[t + 2][0]; T3[2][1] = poly[t + 2][1];
                cnt->subtris++;
            }
            double dT = fabs(det2(T3[1][0] - T3[0][0], T3[1][1] - T3[0][1],
                                  T3[2][0] - T3[0][0], T3[2][1] - T3[0][1]));
            for (int q = 0; q < P->ri.n; ++q) {
                double yx, yy;
                map_point(T3, P->ri.l[q], &yx, &yy);
                double zx = yx - xp, zy = yy - yp;
                if (nozerodiv && zx == 0.0 && zy == 0.0) continue; /* Tab. 1 "diamond" */
                double Q[3];
                if (full) { Q[0] = P->ri.l[q][0]; Q[1] = P->ri.l[q][1]; Q[2] = P->ri.l[q][2]; }
                else barycentric(Vl, yx, yy, Q);
                double w = ap * (P->ri.w[q] * dT);
                double D[6] = {0, 0, 0, 0, 0, 0};
                for (int a = 0; a < 3; ++a) D[a] += Pk[a];
                for (int b = 0; b < 3; ++b) D[posl[b]] -= Q[b];
                cnt->evals++;
                if (P->ndof == 1) {
                    add_outer(B, 1, D, w * gamma_scalar(P, zx, zy), NULL);
                } else {
                    double G[3];
                    gamma_peri(P, zx, zy, G);
                    add_outer(B, 2, D, w, G);
                }
            }
        }
    }
    return interacts;
}

/* ---------------------------------------------------------------------------------------
 * Regularising transforms for intersecting pairs (Sec. 2.3.2, Tab. 1 "club").
 *
 * Reference triangle S = {0 <= s2 <= s1 <= 1}, chi(s) = A0 + s1 (A1 - A0) + s2 (A2 - A1),
 * basis (1 - s1, s1 - s2, s2), |det| = 2|E|. x in E_k at (x1, x2), y in E_l at (y1, y2).
 * Each sub-region of S x S is the image of (0,1)^4 in (xi, e1, e2, e3); the maps and
 * weights were derived for this code (the paper names the transforms only by reference):
 *
 *  identical (6 regions): zeta = y - x (reference) = xi((1-e1) P_r + e1 Q_r) over the six
 *    triangles (0, P_r, Q_r) tiling the hexagon S - S, L = 1 - xi; x = (a + c + L e2,
 *    a + L e2 e3) with a = max(0, -zeta2), c = max(0, zeta2 - zeta1); weight xi L^2 e2.
 *  common edge (4 regions), shared vertices A0 = B0, A1 = B1: u = y1 - x1,
 *    (a) (u, x2, y2) = xi(1-e1, e1, e2),            weight xi^2 L
 *    (b) (u, x2, y2) = xi(e1(1-e2), e1 e2, 1),      weight xi^2 e1 L
 *    (c) (u, x2, y2) = xi(-e1(1-e2), 1, e1 e2),     weight xi^2 e1 L
 *    (d) (u, x2, y2) = xi(e1 - 1, e2, e1),          weight xi^2 L
 *    x1 = max(x2, y2 - u) + L e3, L = 1 - xi.
 *  common vertex (2 regions), A0 = B0: x = x1 (1, e1), y = y1 (1, e3),
 *    (x1, y1) = (xi, xi e2) or (xi e2, xi); weight xi^3 e2.
 *
 * On a discontinuous ansatz (eq. case-one-factoredOut, admissible for s <= 1/2) the shared
 * vertices of a touching pair carry different dofs on the two elements: the integrand's
 * vector over the six dofs is (phi^k(x), -phi^l(y)), so its outer product holds the local,
 * nonlocal and primed terms of that equation. The maps and points are those above.
 * ------------------------------------------------------------------------------------- */
static void duffy_eval(const params_t *P, int U, const double *D, double zx, double zy,
                       double w, block_t *B)
{
    if (P->ndof == 1) {
        double g = gamma_scalar(P, zx, zy);
        add_outer(B, 1, D, w * g, NULL);
    } else {
        double G[3];
        gamma_peri(P, zx, zy, G);
        add_outer(B, 2, D, w, G);
    }
    (void)U;
}

static void pair_duffy(const mesh_t *m, const params_t *P, int k, int l, int shared,
                       block_t *B, counts_t *cnt)
{
    const int *tk = &m->T[3 * k], *tl = &m->T[3 * l];
    /* Reorder so that the shared vertices come first, in the same order in both. Vertices are
     * matched by position; on a discontinuous ansatz the matched dofs differ (split). */
    int ak[3], bl[3] = {0, 1, 2};
    if (shared == 3) {
        for (int a = 0; a < 3; ++a) { ak[a] = a; }
    } else if (shared == 2) {
        int s0 = -1, s1 = -1, sl0 = -1, sl1 = -1;
        for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) if (m->pos[tk[a]] == m->pos[tl[b]]) {
            if (s0 < 0) { s0 = a; sl0 = b; } else { s1 = a; sl1 = b; }
        }
        ak[0] = s0; ak[1] = s1; ak[2] = 3 - s0 - s1;
        bl[0] = sl0; bl[1] = sl1; bl[2] = 3 - sl0 - sl1;
    } else {
        int s0 = -1, sl0 = -1;
        for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) if (m->pos[tk[a]] == m->pos[tl[b]]) { s0 = a; sl0 = b; }
        ak[0] = s0; ak[1] = (s0 + 1) % 3; ak[2] = (s0 + 2) % 3;
        bl[0] = sl0; bl[1] = (sl0 + 1) % 3; bl[2] = (sl0 + 2) % 3;
    }
    const int split = shared < 3 && tk[ak[0]] != tl[bl[0]];
    double A[3][2], Bv[3][2];
    for (int a = 0; a < 3; ++a) {
        A[a][0] = m->X[2 * tk[ak[a]]]; A[a][1] = m->X[2 * tk[ak[a]] + 1];
    }
    if (shared < 3) for (int b = 0; b < 3; ++b) {
        Bv[b][0] = m->X[2 * tl[bl[b]]]; Bv[b][1] = m->X[2 * tl[bl[b]] + 1];
    }
    /* union vertices in the transform's order and their positions in B->node */
    int uorder[5], U;
    if (shared == 3) { U = 3; for (int a = 0; a < 3; ++a) uorder[a] = tk[ak[a]]; }
    else if (shared == 2) { U = 4; for (int a = 0; a < 3; ++a) uorder[a] = tk[ak[a]]; uorder[3] = tl[bl[2]]; }
    else { U = 5; for (int a = 0; a < 3; ++a) uorder[a] = tk[ak[a]]; uorder[3] = tl[bl[1]]; uorder[4] = tl[bl[2]]; }
    int upos[5];
    for (int u = 0; u < U; ++u) {
        upos[u] = -1;
        for (int v = 0; v < B->U; ++v) if (B->node[v] == uorder[u]) upos[u] = v;
    }
    /* split pairs: block positions of E_k's dofs (A0, A1, A2) and E_l's (B0, B1, B2) */
    int kpos[3] = {0, 0, 0}, lpos[3] = {0, 0, 0};
    if (split) for (int a = 0; a < 3; ++a) for (int v = 0; v < B->U; ++v) {
        if (B->node[v] == tk[ak[a]]) kpos[a] = v;
        if (B->node[v] == tl[bl[a]]) lpos[a] = v;
    }
    double scale = m->det[k] * m->det[l];
    double e10x = A[1][0] - A[0][0], e10y = A[1][1] - A[0][1];
    double e21x = A[2][0] - A[1][0], e21y = A[2][1] - A[1][1];
    int ng = P->ng;
    double Dz[6];
    for (int i0 = 0; i0 < ng; ++i0)
    for (int i1 = 0; i1 < ng; ++i1)
    for (int i2 = 0; i2 < ng; ++i2)
    for (int i3 = 0; i3 < ng; ++i3) {
        double xi = P->gx[i0], e1 = P->gx[i1], e2 = P->gx[i2], e3 = P->gx[i3];
        double wq = P->gw[i0] * P->gw[i1] * P->gw[i2] * P->gw[i3];
        double L = 1.0 - xi;
        if (shared == 3) {
            static const double PQ[6][4] = {
                {0, 1, 1, 1}, {1, 0, 1, 1}, {1, 0, 0, -1},
                {0, 1, -1, 0}, {-1, 0, -1, -1}, {0, -1, -1, -1}};
            for (int r = 0; r < 6; ++r) {
                double h1 = (1.0 - e1) * PQ[r][0] + e1 * PQ[r][2]; /* zeta / xi */
                double h2 = (1.0 - e1) * PQ[r][1] + e1 * PQ[r][3];
                double z1 = xi * h1, z2 = xi * h2;
                double a = z2 < 0.0 ? -z2 : 0.0;
                double c = (z2 - z1) > 0.0 ? (z2 - z1) : 0.0;
                double x1 = a + c + L * e2, x2 = a + L * e2 * e3;
                (void)x1; (void)x2; /* the integrand depends on zeta only */
                double zx = xi * (h1 * e10x + h2 * e21x);
                double zy = xi * (h1 * e10y + h2 * e21y);
                /* D_u = psi_u(x) - psi_u(y) */
                double D0 = xi * h1, D1 = xi * (h2 - h1), D2 = -xi * h2;
                double D[6] = {0, 0, 0, 0, 0, 0};
                D[upos[0]] = D0; D[upos[1]] = D1; D[upos[2]] = D2;
                (void)Dz;
                duffy_eval(P, U, D, zx, zy, wq * scale * xi * L * L * e2, B);
                cnt->duffy_points++;
            }
        } else if (shared == 2) {
            double fx = Bv[2][0] - A[1][0], fy = Bv[2][1] - A[1][1]; /* B2 - A1 */
            for (int r = 0; r < 4; ++r) {
                double hu, hx2, hy2, wr;
                switch (r) {
                case 0: hu = 1.0 - e1; hx2 = e1; hy2 = e2; wr = 1.0; break;
                case 1: hu = e1 * (1.0 - e2); hx2 = e1 * e2; hy2 = 1.0; wr = e1; break;
                case 2: hu = -e1 * (1.0 - e2); hx2 = 1.0; hy2 = e1 * e2; wr = e1; break;
                default: hu = e1 - 1.0; hx2 = e2; hy2 = e1; wr = 1.0; break;
                }
                double u = xi * hu, x2 = xi * hx2, y2 = xi * hy2;
                double lo = x2 > (y2 - u) ? x2 : (y2 - u);
                double x1 = lo + L * e3;
                double zx = xi * (hu * e10x + hy2 * fx - hx2 * e21x);
                double zy = xi * (hu * e10y + hy2 * fy - hx2 * e21y);
                double D[6] = {0, 0, 0, 0, 0, 0};
                if (split) {
                    double y1 = x1 + u;
                    D[kpos[0]] = 1.0 - x1; D[kpos[1]] = x1 - x2; D[kpos[2]] = x2;
                    D[lpos[0]] = -(1.0 - y1); D[lpos[1]] = -(y1 - y2); D[lpos[2]] = -y2;
                } else {
                    D[upos[0]] = u;                 /* y1 - x1 */
                    D[upos[1]] = -u - x2 + y2;      /* (x1 - x2) - (y1 - y2) */
                    D[upos[2]] = x2;
                    D[upos[3]] = -y2;
                }
                duffy_eval(P, U, D, zx, zy, wq * scale * xi * xi * L * wr, B);
                cnt->duffy_points++;
            }
        } else {
            double g10x = Bv[1][0] - A[0][0], g10y = Bv[1][1] - A[0][1]; /* B1 - A0 */
            double g21x = Bv[2][0] - Bv[1][0], g21y = Bv[2][1] - Bv[1][1];
            for (int r = 0; r < 2; ++r) {
                double hx1 = r == 0 ? 1.0 : e2, hy1 = r == 0 ? e2 : 1.0;
                double w1 = e1, w2 = e3;
                double x1 = xi * hx1, y1 = xi * hy1;
                double zx = y1 * (g10x + w2 * g21x) - x1 * (e10x + w1 * e21x);
                double zy = y1 * (g10y + w2 * g21y) - x1 * (e10y + w1 * e21y);
                double D[6] = {0, 0, 0, 0, 0, 0};
                if (split) {
                    D[kpos[0]] = 1.0 - x1; D[kpos[1]] = x1 * (1.0 - w1); D[kpos[2]] = x1 * w1;
                    D[lpos[0]] = -(1.0 - y1); D[lpos[1]] = -y1 * (1.0 - w2); D[lpos[2]] = -y1 * w2;
                } else {
                    D[upos[0]] = y1 - x1;
                    D[upos[1]] = x1 * (1.0 - w1);
                    D[upos[2]] = x1 * w1;
                    D[upos[3]] = -y1 * (1.0 - w2);
                    D[upos[4]] = -y1 * w2;
                }
                duffy_eval(P, U, D, zx, zy, wq * scale * xi * xi * xi * e2, B);
                cnt->duffy_points++;
            }
        }
    }
}

/* ---------------------------------------------------------------------------------------
 * Alg. 1 for one ordered pair. Returns 1 if the pair interacts.
 * ------------------------------------------------------------------------------------- */
/* Shared vertices of E_k and E_l as points (Sec. 2.3: intersecting pairs), so that a mesh whose
 * elements carry their own copies of the vertices (a discontinuous ansatz) classifies its pairs
 * like the continuous one. */
static int shared_count(const mesh_t *m, int k, int l)
{
    int c = 0;
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b)
        c += m->pos[m->T[3 * k + a]] == m->pos[m->T[3 * l + b]];
    return c;
}

static int singular_rule(const params_t *P)
{
    if (P->close_rule == ORC_CLOSE_DUFFY) return 1;
    if (P->close_rule == ORC_CLOSE_AUTO) return P->kernel == ORC_K_FRAC && P->s > 0.0;
    return 0;
}

static int nozerodiv_rule(const params_t *P)
{
    if (P->close_rule == ORC_CLOSE_NOZERODIV) return 1;
    if (P->close_rule == ORC_CLOSE_AUTO) return P->kernel == ORC_K_PERI ||
                                              (P->kernel == ORC_K_FRAC && P->s > -1.0 && P->s <= 0.0);
    return 0;
}

/* evaluate pair; if B != NULL accumulate into it */
static int eval_pair(const mesh_t *m, const params_t *P, int k, int l, block_t *B, counts_t *cnt)
{
    int sh = shared_count(m, k, l);
    if (B == NULL) {
        if (sh > 0) return 1; /* intersecting pairs always interact (T_adj spans T_S) */
        block_t dummy;
        int posl[3] = {3, 4, 5};
        return pair_truncation(m, P, k, l, posl, &dummy, 0, 0, cnt);
    }
    int posl[3];
    B->U = union_nodes(&m->T[3 * k], &m->T[3 * l], B->node, posl);
    int n = B->U * P->ndof;
    memset(B->blk, 0, sizeof(double) * n * n);
    if (sh > 0 && singular_rule(P)) {
        pair_duffy(m, P, k, l, sh, B, cnt);
        return 1;
    }
    int r = pair_truncation(m, P, k, l, posl, B, 1, sh > 0 && nozerodiv_rule(P), cnt);
    return r || sh > 0;
}

/* ---------------------------------------------------------------------------------------
 * Sparse accumulation: per row a sorted column list (pattern first, then values).
 * ------------------------------------------------------------------------------------- */
typedef struct { int n, cap; int *c; } ilist_t;

static void ilist_add(ilist_t *L, int v)
{
    int lo = 0, hi = L->n;
    while (lo < hi) { int mid = (lo + hi) / 2; if (L->c[mid] < v) lo = mid + 1; else hi = mid; }
    if (lo < L->n && L->c[lo] == v) return;
    if (L->n == L->cap) { L->cap = L->cap ? 2 * L->cap : 16; L->c = realloc(L->c, sizeof(int) * L->cap); }
    memmove(L->c + lo + 1, L->c + lo, sizeof(int) * (L->n - lo));
    L->c[lo] = v;
    L->n++;
}

typedef struct {
    int N, ndof, M, K;
    long long nnz;
    long long *row_ptr;
    int *col;
    double *val;
    double *F;
    long long npairs;
    int *pairs;          /* npairs x 2, (k, l) in BFS order per k */
    signed char *pclass; /* shared vertex count per pair */
    counts_t cnt;
    signed char *dirichlet;
    int *elems_ccw;
} orc_sys;

static long long find_slot(const orc_sys *S, int i, int j)
{
    long long lo = S->row_ptr[i], hi = S->row_ptr[i + 1];
    while (lo < hi) { long long mid = (lo + hi) / 2; if (S->col[mid] < j) lo = mid + 1; else hi = mid; }
    return lo;
}

/* ---------------------------------------------------------------------------------------
 * Interaction search: Alg. 2 (breadth-first traversal of T_adj) or brute force.
 * ------------------------------------------------------------------------------------- */
typedef struct { int n, cap; int *v; } ivec_t;
static void ivec_push(ivec_t *a, int x)
{
    if (a->n == a->cap) { a->cap = a->cap ? 2 * a->cap : 64; a->v = realloc(a->v, sizeof(int) * a->cap); }
    a->v[a->n++] = x;
}

static void neighbours_of(const mesh_t *m, int e, ivec_t *out, int *mark, int stamp)
{
    out->n = 0;
    for (int a = 0; a < 3; ++a) {
        int v = m->T[3 * e + a];
        v = m->pos[v];
        for (int t = m->ne_ptr[v]; t < m->ne_ptr[v + 1]; ++t) {
            int f = m->ne_idx[t];
            if (mark[f] != stamp) { mark[f] = stamp; ivec_push(out, f); }
        }
    }
}

/* partners of k in traversal order */
static void search_partners(const mesh_t *m, const params_t *P, int k, int mode, ivec_t *res,
                            int *visited, int *vstamp, int *nbmark, int *nbstamp, counts_t *cnt)
{
    res->n = 0;
    if (mode == ORC_PAIRS_BRUTE) {
        for (int l = 0; l < m->K; ++l) if (eval_pair(m, P, k, l, NULL, cnt)) ivec_push(res, l);
        return;
    }
    ivec_t queue = {0, 0, NULL}, nb = {0, 0, NULL};
    ++*vstamp;
    ivec_push(&queue, k);
    ivec_push(res, k);        /* (k, k) always interacts */
    visited[k] = *vstamp;
    for (int qi = 0; qi < queue.n; ++qi) {
        int e = queue.v[qi];
        ++*nbstamp;
        neighbours_of(m, e, &nb, nbmark, *nbstamp);
        for (int t = 0; t < nb.n; ++t) {
            int l = nb.v[t];
            if (visited[l] == *vstamp) continue;
            visited[l] = *vstamp;
            if (eval_pair(m, P, k, l, NULL, cnt)) { ivec_push(&queue, l); ivec_push(res, l); }
        }
    }
    free(queue.v);
    free(nb.v);
}

/* ---------------------------------------------------------------------------------------
 * Public entry points (ctypes)
 * ------------------------------------------------------------------------------------- */
typedef struct { double x, y; int id; } xyid_t;

static int cmp_xyid(const void *pa, const void *pb)
{
    const xyid_t *a = pa, *b = pb;
    if (a->x != b->x) return a->x < b->x ? -1 : 1;
    if (a->y != b->y) return a->y < b->y ? -1 : 1;
    return a->id - b->id;
}

static void build_mesh(mesh_t *m, int M, const double *X, int K, const int *T, const signed char *lab)
{
    m->M = M; m->K = K; m->X = X;
    m->T = malloc(sizeof(int) * 3 * (size_t)K + 4);
    m->det = malloc(sizeof(double) * (size_t)K + 8);
    m->lab = malloc((size_t)K + 1);
    m->dir = calloc((size_t)M + 1, 1);
    for (int k = 0; k < K; ++k) {
        int t0 = T[3 * k], t1 = T[3 * k + 1], t2 = T[3 * k + 2];
        double d = det2(X[2 * t1] - X[2 * t0], X[2 * t1 + 1] - X[2 * t0 + 1],
                        X[2 * t2] - X[2 * t0], X[2 * t2 + 1] - X[2 * t0 + 1]);
        if (d < 0) { int tmp = t1; t1 = t2; t2 = tmp; d = -d; }
        m->T[3 * k] = t0; m->T[3 * k + 1] = t1; m->T[3 * k + 2] = t2;
        m->det[k] = d;
        m->lab[k] = lab ? lab[k] : 1;
        if (!m->lab[k]) { m->dir[t0] = 1; m->dir[t1] = 1; m->dir[t2] = 1; }
    }
    /* positions: nodes with equal coordinates, found by sorting the nodes by (x, y) */
    m->pos = malloc(sizeof(int) * ((size_t)M + 1));
    {
        xyid_t *ord = malloc(sizeof(xyid_t) * ((size_t)M + 1));
        for (int v = 0; v < M; ++v) { ord[v].x = X[2 * v]; ord[v].y = X[2 * v + 1]; ord[v].id = v; }
        qsort(ord, (size_t)M, sizeof(xyid_t), cmp_xyid);
        for (int i = 0; i < M;) {
            int j = i, lo = ord[i].id;
            while (j < M && ord[j].x == ord[i].x && ord[j].y == ord[i].y) {
                if (ord[j].id < lo) lo = ord[j].id;
                ++j;
            }
            for (int t = i; t < j; ++t) m->pos[ord[t].id] = lo;
            i = j;
        }
        free(ord);
    }
    m->ne_ptr = calloc((size_t)M + 1, sizeof(int));
    for (int k = 0; k < K; ++k) for (int a = 0; a < 3; ++a) m->ne_ptr[m->pos[m->T[3 * k + a]] + 1]++;
    for (int v = 0; v < M; ++v) m->ne_ptr[v + 1] += m->ne_ptr[v];
    m->ne_idx = malloc(sizeof(int) * 3 * (size_t)K + 4);
    int *fill = calloc((size_t)M + 1, sizeof(int));
    for (int k = 0; k < K; ++k) for (int a = 0; a < 3; ++a) {
        int v = m->pos[m->T[3 * k + a]];
        m->ne_idx[m->ne_ptr[v] + fill[v]++] = k;
    }
    free(fill);
}

static void free_mesh(mesh_t *m)
{
    free(m->T); free(m->det); free(m->lab); free(m->dir); free(m->ne_ptr); free(m->ne_idx); free(m->pos);
}

static void set_rule(rule_t *r, int n, const double *q)
{
    r->n = n;
    for (int i = 0; i < n; ++i) {
        r->l[i][0] = q[4 * i]; r->l[i][1] = q[4 * i + 1]; r->l[i][2] = q[4 * i + 2];
        r->w[i] = q[4 * i + 3];
    }
}

static void set_params(params_t *P, int kernel, double delta, double s, double kconst, int ball,
                       int nqo, const double *qo, int nqi, const double *qi, int close_rule,
                       int ng, const double *gx, const double *gw, int ndof)
{
    memset(P, 0, sizeof *P);
    P->kernel = kernel; P->ball = ball; P->close_rule = close_rule; P->ndof = ndof;
    P->delta = delta; P->delta2 = delta * delta; P->s = s;
    if (!isnan(kconst)) P->c = kconst;
    else if (kernel == ORC_K_CONST && ball == ORC_BALL_INF)
        P->c = 3.0 / (4.0 * delta * delta * delta * delta);   /* c_delta^inf of Sec. 3.3 */
    else if (kernel == ORC_K_CONST) P->c = 4.0 / (M_PI * delta * delta * delta * delta);
    else if (kernel == ORC_K_TAB) P->c = 1.0;
    else if (kernel == ORC_K_FRAC) P->c = (2.0 - 2.0 * s) / (M_PI * pow(delta, 2.0 - 2.0 * s));
    else P->c = 3.0 / (delta * delta * delta);
    set_rule(&P->ro, nqo, qo);
    set_rule(&P->ri, nqi, qi);
    P->ng = ng;
    for (int i = 0; i < ng; ++i) { P->gx[i] = gx[i]; P->gw[i] = gw[i]; }
}

/* Interaction pattern only: pairs (k, l) for k in [0, K), in traversal order. */
void *orc_pairs(int M, const double *X, int K, const int *T, int kernel, double delta, double s,
                int ball, int nqo, const double *qo, int close_rule, int mode, int nthreads,
                long long *npairs_out)
{
    mesh_t m;
    build_mesh(&m, M, X, K, T, NULL);
    params_t P;
    double dummyq[4] = {1.0 / 3, 1.0 / 3, 1.0 / 3, 0.5}, g[1] = {0.5}, gw[1] = {1.0};
    set_params(&P, kernel, delta, s, NAN, ball, nqo, qo, 1, dummyq, close_rule, 1, g, gw, 1);
    ivec_t *lists = calloc((size_t)K, sizeof(ivec_t));
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        int *visited = calloc((size_t)K + 1, sizeof(int)), *nbmark = calloc((size_t)K + 1, sizeof(int));
        int vs = 0, ns = 0;
        counts_t cnt;
        memset(&cnt, 0, sizeof cnt);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
        for (int k = 0; k < K; ++k)
            search_partners(&m, &P, k, mode, &lists[k], visited, &vs, nbmark, &ns, &cnt);
        free(visited); free(nbmark);
    }
    long long tot = 0;
    for (int k = 0; k < K; ++k) tot += lists[k].n;
    int *out = malloc(sizeof(int) * 2 * (size_t)(tot + 1));
    long long o = 0;
    for (int k = 0; k < K; ++k) {
        for (int i = 0; i < lists[k].n; ++i) { out[2 * o] = k; out[2 * o + 1] = lists[k].v[i]; ++o; }
        free(lists[k].v);
    }
    free(lists);
    free_mesh(&m);
    *npairs_out = tot;
    return out;
}

void orc_free(void *p) { free(p); }

/* Full assembly: A_h^# over all nodes of the base domain (block per ordered pair,
 * summed into CSR in (k, l, p, q) order), F over Omega elements. If elem_subset is
 * given (n_subset outer elements), only pairs with k in the subset are assembled. If
 * node_keep is given (M flags), only pairs with a flagged node among the vertices of E_k
 * or E_l are kept: every pair that writes into the row of a flagged node is one of them, so
 * those rows are the full assembly's rows, summed in the same (k, l, p, q) order. */
orc_sys *orc_assemble(int M, const double *X, int K, const int *T, const signed char *lab,
                      int kernel, double delta, double s, double kconst, int ball,
                      int nqo, const double *qo, int nqi, const double *qi, int close_rule,
                      int ng, const double *gx, const double *gw, int ndof,
                      const double *f_nodal, int mode, int nthreads,
                      int n_subset, const int *elem_subset,
                      const signed char *mat, int nmat, const double *mscale,
                      int ntab, const double *tab, const signed char *node_keep)
{
    mesh_t m;
    build_mesh(&m, M, X, K, T, lab);
    params_t P;
    set_params(&P, kernel, delta, s, kconst, ball, nqo, qo, nqi, qi, close_rule, ng, gx, gw, ndof);
    P.ntab = ntab < MAXTAB ? ntab : MAXTAB;
    for (int i = 0; i < P.ntab; ++i) P.tab[i] = tab[i];
    orc_sys *S = calloc(1, sizeof(orc_sys));
    S->M = M; S->K = K; S->ndof = ndof; S->N = M * ndof;
    int nk = n_subset > 0 ? n_subset : K;
    /* 1. pairs */
    ivec_t *lists = calloc((size_t)nk, sizeof(ivec_t));
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        int *visited = calloc((size_t)K + 1, sizeof(int)), *nbmark = calloc((size_t)K + 1, sizeof(int));
        int vs = 0, ns = 0;
        counts_t cnt;
        memset(&cnt, 0, sizeof cnt);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
        for (int i = 0; i < nk; ++i) {
            int k = n_subset > 0 ? elem_subset[i] : i;
            search_partners(&m, &P, k, mode, &lists[i], visited, &vs, nbmark, &ns, &cnt);
            if (node_keep) {
                int kk = 0;
                for (int t = 0; t < lists[i].n; ++t) {
                    const int l = lists[i].v[t];
                    int hit = 0;
                    for (int a = 0; a < 3; ++a) hit |= node_keep[m.T[3 * k + a]] | node_keep[m.T[3 * l + a]];
                    if (hit) lists[i].v[kk++] = l;
                }
                lists[i].n = kk;
            }
        }
        free(visited); free(nbmark);
    }
    long long tot = 0;
    for (int i = 0; i < nk; ++i) tot += lists[i].n;
    S->npairs = tot;
    S->pairs = malloc(sizeof(int) * 2 * (size_t)(tot + 1));
    S->pclass = malloc((size_t)tot + 1);
    long long *pstart = malloc(sizeof(long long) * ((size_t)nk + 1));
    long long o = 0;
    for (int i = 0; i < nk; ++i) {
        int k = n_subset > 0 ? elem_subset[i] : i;
        pstart[i] = o;
        for (int t = 0; t < lists[i].n; ++t) {
            S->pairs[2 * o] = k; S->pairs[2 * o + 1] = lists[i].v[t];
            S->pclass[o] = (signed char)shared_count(&m, k, lists[i].v[t]);
            ++o;
        }
        free(lists[i].v);
    }
    pstart[nk] = o;
    free(lists);
    /* 2. pattern: union vertices of every pair, all dof couplings */
    int N = S->N;
    ilist_t *rows = calloc((size_t)N + 1, sizeof(ilist_t));
    for (long long pq = 0; pq < tot; ++pq) {
        int node[6], posl[3];
        int U = union_nodes(&m.T[3 * S->pairs[2 * pq]], &m.T[3 * S->pairs[2 * pq + 1]], node, posl);
        for (int u = 0; u < U; ++u) for (int v = 0; v < U; ++v)
            for (int a = 0; a < ndof; ++a) for (int b = 0; b < ndof; ++b)
                ilist_add(&rows[node[u] * ndof + a], node[v] * ndof + b);
    }
    S->row_ptr = malloc(sizeof(long long) * ((size_t)N + 1));
    S->row_ptr[0] = 0;
    for (int i = 0; i < N; ++i) S->row_ptr[i + 1] = S->row_ptr[i] + rows[i].n;
    S->nnz = S->row_ptr[N];
    S->col = malloc(sizeof(int) * (size_t)(S->nnz + 1));
    S->val = calloc((size_t)S->nnz + 1, sizeof(double));
    for (int i = 0; i < N; ++i) {
        memcpy(S->col + S->row_ptr[i], rows[i].c, sizeof(int) * rows[i].n);
        free(rows[i].c);
    }
    free(rows);
    /* 3. values: blocks computed in parallel in chunks of pairs, summed in (k, l) order */
    const long long CH = 16384;
    block_t *blocks = malloc(sizeof(block_t) * (size_t)CH);
    memset(&S->cnt, 0, sizeof S->cnt);
    for (long long p0 = 0; p0 < tot; p0 += CH) {
        long long p1 = p0 + CH < tot ? p0 + CH : tot;
        counts_t cacc;
        memset(&cacc, 0, sizeof cacc);
#ifdef _OPENMP
#pragma omp parallel
#endif
        {
            counts_t c;
            memset(&c, 0, sizeof c);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
            for (long long pq = p0; pq < p1; ++pq)
                eval_pair(&m, &P, S->pairs[2 * pq], S->pairs[2 * pq + 1], &blocks[pq - p0], &c);
#ifdef _OPENMP
#pragma omp critical
#endif
            {
                cacc.evals += c.evals; cacc.cut_points += c.cut_points; cacc.full_points += c.full_points;
                cacc.subtris += c.subtris; cacc.duffy_points += c.duffy_points;
            }
        }
        S->cnt.evals += cacc.evals; S->cnt.cut_points += cacc.cut_points;
        S->cnt.full_points += cacc.full_points; S->cnt.subtris += cacc.subtris;
        S->cnt.duffy_points += cacc.duffy_points;
        for (long long pq = p0; pq < p1; ++pq) {
            block_t *B = &blocks[pq - p0];
            int n = B->U * ndof;
            /* label-dependent kernel (Sec. 1): Psi on E_k x E_l scaled by s[mat_k][mat_l] */
            double fm = 1.0;
            if (mat && mscale) fm = mscale[mat[S->pairs[2 * pq]] * nmat + mat[S->pairs[2 * pq + 1]]];
            for (int u = 0; u < n; ++u) {
                int gi = B->node[u / ndof] * ndof + u % ndof;
                for (int v = u; v < n; ++v) {
                    int gj = B->node[v / ndof] * ndof + v % ndof;
                    /* (i,j) and (j,i) receive the same value at the same moment */
                    double x = v == u ? B->blk[u * n + v] : 0.5 * (B->blk[u * n + v] + B->blk[v * n + u]);
                    x *= fm;
                    if (v == u) { S->val[find_slot(S, gi, gi)] += x; }
                    else { S->val[find_slot(S, gi, gj)] += x; S->val[find_slot(S, gj, gi)] += x; }
                }
            }
        }
    }
    free(blocks);
    S->cnt.pairs = tot;
    for (long long pq = 0; pq < tot; ++pq) {
        switch (S->pclass[pq]) {
        case 3: S->cnt.pairs_identical++; break;
        case 2: S->cnt.pairs_edge++; break;
        case 1: S->cnt.pairs_vertex++; break;
        default: S->cnt.pairs_separated++; break;
        }
    }
    free(pstart);
    /* 4. load vector F_i = sum_{E_k in Omega} sum_p a_p f(x_p) phi_i(x_p), f interpolated in P1 */
    S->F = calloc((size_t)N + 1, sizeof(double));
    if (f_nodal) {
        for (int k = 0; k < K; ++k) {
            if (!m.lab[k]) continue;
            for (int p = 0; p < P.ro.n; ++p) {
                double ap = P.ro.w[p] * m.det[k];
                for (int c = 0; c < ndof; ++c) {
                    double fx = 0.0;
                    for (int a = 0; a < 3; ++a) fx += P.ro.l[p][a] * f_nodal[m.T[3 * k + a] * ndof + c];
                    for (int a = 0; a < 3; ++a) S->F[m.T[3 * k + a] * ndof + c] += ap * fx * P.ro.l[p][a];
                }
            }
        }
    }
    S->dirichlet = malloc((size_t)M + 1);
    memcpy(S->dirichlet, m.dir, (size_t)M);
    S->elems_ccw = malloc(sizeof(int) * 3 * (size_t)K + 4);
    memcpy(S->elems_ccw, m.T, sizeof(int) * 3 * (size_t)K);
    free_mesh(&m);
    return S;
}

void orc_sys_sizes(const orc_sys *S, long long *out /* N, nnz, npairs */)
{
    out[0] = S->N; out[1] = S->nnz; out[2] = S->npairs;
}

void orc_sys_copy(const orc_sys *S, long long *row_ptr, int *col, double *val, double *F,
                  int *pairs, signed char *pclass, signed char *dirichlet, long long *counts)
{
    if (row_ptr) memcpy(row_ptr, S->row_ptr, sizeof(long long) * ((size_t)S->N + 1));
    if (col) memcpy(col, S->col, sizeof(int) * (size_t)S->nnz);
    if (val) memcpy(val, S->val, sizeof(double) * (size_t)S->nnz);
    if (F) memcpy(F, S->F, sizeof(double) * (size_t)S->N);
    if (pairs) memcpy(pairs, S->pairs, sizeof(int) * 2 * (size_t)S->npairs);
    if (pclass) memcpy(pclass, S->pclass, (size_t)S->npairs);
    if (dirichlet) memcpy(dirichlet, S->dirichlet, (size_t)S->M);
    if (counts) {
        const counts_t *c = &S->cnt;
        long long v[10] = {c->evals, c->cut_points, c->full_points, c->subtris, c->duffy_points,
                           c->pairs, c->pairs_identical, c->pairs_edge, c->pairs_vertex, c->pairs_separated};
        memcpy(counts, v, sizeof v);
    }
}

void orc_sys_free(orc_sys *S)
{
    if (!S) return;
    free(S->row_ptr); free(S->col); free(S->val); free(S->F); free(S->pairs); free(S->pclass);
    free(S->dirichlet); free(S->elems_ccw);
    free(S);
}

/* Local block of one ordered pair (test hook). blk receives (U*ndof)^2 values, node U ids. */
int orc_pair_block(int M, const double *X, int K, const int *T, int kernel, double delta, double s,
                   double kconst, int ball, int nqo, const double *qo, int nqi, const double *qi,
                   int close_rule, int ng, const double *gx, const double *gw, int ndof,
                   int k, int l, int *node_out, double *blk_out)
{
    mesh_t m;
    build_mesh(&m, M, X, K, T, NULL);
    params_t P;
    set_params(&P, kernel, delta, s, kconst, ball, nqo, qo, nqi, qi, close_rule, ng, gx, gw, ndof);
    block_t B;
    counts_t c;
    memset(&c, 0, sizeof c);
    int r = eval_pair(&m, &P, k, l, &B, &c);
    int n = B.U * ndof;
    for (int u = 0; u < B.U; ++u) node_out[u] = B.node[u];
    memcpy(blk_out, B.blk, sizeof(double) * n * n);
    free_mesh(&m);
    return r ? B.U : -B.U;
}

/* Clip test hook: V is 3x2, out receives up to 16 points. Returns count, *full flag. */
/* ball: 0 nocaps, 1 approxcaps, 2 infinity norm ball */
int orc_clip(const double *V6, double cx, double cy, double delta, int ball, double *out, int *full)
{
    double V[3][2] = {{V6[0], V6[1]}, {V6[2], V6[3]}, {V6[4], V6[5]}};
    double P[MAXPOLY][2];
    int n = ball == ORC_BALL_INF ? orc_clip_square(V, cx, cy, delta, P, full)
                                 : orc_clip_ball(V, cx, cy, delta, delta * delta, ball == ORC_BALL_APPROXCAPS, P, full);
    for (int i = 0; i < n; ++i) { out[2 * i] = P[i][0]; out[2 * i + 1] = P[i][1]; }
    return n;
}
