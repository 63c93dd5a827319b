/*
 * CPU oracle for best-improvement VRP local search -- TEST INFRASTRUCTURE.
 * Loaded only by tests, the package smoke check and the benchmark's CPU
 * baseline; never by the GPU product path.  Plain, single-threaded C.
 *
 * Problem and objective: Section 2 of the paper (routes R_i = (v0, ..., v0),
 * distance objective, capacity and time windows), with the penalised
 * objective  cost(R) = dist(R) + w_load * max(0, load(R) - Q) + w_tw * warp(R)
 * where load(R) is the largest load on board (the total delivery when the
 * instance has no pickups; with pickups, Section 2's VRPSPDTW)
 * that a feasible/infeasible search uses (Appendix, Algorithm "Feasible and
 * infeasible search").  The fleet is fixed, so the vehicle term of the
 * Section 2 objective is a constant and is left out.
 *
 * Time warp (Section 4.3.3, after Nagata et al.): arriving after l_x costs
 * (arrival - l_x) of warp and the clock is set back to l_x; arriving before
 * e_x waits.  Travel time equals distance (the paper keeps one matrix T; the
 * instances here have T = C).
 *
 * Neighbourhood (Section 4.1 operators, Figure "operators"; or-opt is the
 * extension named at the end of Section 4.1):
 *   op 0 relocate  a = customer u, b = anchor v, v != u, v != pred(u):
 *                  move u to just after v (same or other route).
 *   op 1 swap      customers a < b: exchange their positions.
 *   op 2 2-opt     customers a, b of one route, pos(a) < pos(b):
 *                  reverse the run a..b.
 *   op 3 2-opt*    anchors a, b with route(a) < route(b): the new routes
 *                  are head(a)+tail-after(b) and head(b)+tail-after(a).
 *   op 4/5 or-opt  a = first of k = 2/3 consecutive customers of one route,
 *                  b = anchor outside the run, b != pred(a): move the run,
 *                  same orientation, to just after b.
 *   op 6 swap(1,2) a = customer, b = first of two consecutive customers of
 *                  one route, a not in that run: a takes the run's place and
 *                  the run (same orientation) takes a's (Section 5.3.1 Swap
 *                  with N1 = 1, N2 = 2; same or other route).
 *   op 7 swap(2,2) a < b, each the first of two consecutive customers, the
 *                  runs disjoint: the runs exchange places (N1 = N2 = 2).
 * The best move is the lexicographically smallest (delta, idx).
 */
#include "tga_oracle.h"

#include <stdlib.h>
#include <string.h>

#define DIST(in, i, j) ((int64_t)(in)->dist[(int64_t)(i) * ((in)->n + 1) + (j)])

static int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }
static int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }

/* ------------------------------------------------------------------------ */
/* Route cost by forward simulation: the plain definition.                  */

int64_t orc_route_warp(const orc_inst *in, const int32_t *nodes, int32_t len)
{
    if (!in->has_tw || len == 0) return 0;
    int64_t t = in->early[0], warp = 0;
    int32_t prev = 0;
    for (int32_t k = 0; k <= len; ++k) {
        int32_t x = (k < len) ? nodes[k] : 0;       /* k == len: back at depot */
        t += in->service[prev] + DIST(in, prev, x);
        if (t < in->early[x]) t = in->early[x];
        if (t > in->late[x]) { warp += t - in->late[x]; t = in->late[x]; }
        prev = x;
    }
    return warp;
}

/* Largest load on board (Section 2: the vehicle leaves the depot carrying
 * the deliveries of all its customers, then drops d_x and collects p_x at
 * each customer in turn); without pickups the load only falls, so the
 * largest load is the total delivery at departure. */
int64_t orc_route_peak_load(const orc_inst *in, const int32_t *nodes, int32_t len)
{
    int64_t load = 0;
    for (int32_t k = 0; k < len; ++k) load += in->demand[nodes[k]];
    if (!in->pickup) return load;
    int64_t peak = load;
    for (int32_t k = 0; k < len; ++k) {
        load += in->pickup[nodes[k]] - in->demand[nodes[k]];
        if (load > peak) peak = load;
    }
    return peak;
}

int64_t orc_route_cost(const orc_inst *in, const int32_t *nodes, int32_t len)
{
    if (len == 0) return 0;
    int64_t d = DIST(in, 0, nodes[0]) + DIST(in, nodes[len - 1], 0);
    for (int32_t k = 0; k + 1 < len; ++k) d += DIST(in, nodes[k], nodes[k + 1]);
    const int64_t load = orc_route_peak_load(in, nodes, len);
    int64_t cost = d + (int64_t)in->w_load * max64(0, load - in->capacity);
    if (in->has_tw) cost += (int64_t)in->w_tw * orc_route_warp(in, nodes, len);
    return cost;
}

int64_t orc_solution_cost(const orc_inst *in, const int32_t *tour, const int32_t *rs)
{
    int64_t c = 0;
    for (int32_t r = 0; r < in->m; ++r) c += orc_route_cost(in, tour + rs[r], rs[r + 1] - rs[r]);
    return c;
}

int orc_check_solution(const orc_inst *in, const int32_t *tour, const int32_t *rs)
{
    if (in->m < 1 || rs[0] != 0 || rs[in->m] != in->n) return 1;
    for (int32_t r = 0; r < in->m; ++r) if (rs[r + 1] < rs[r]) return 2;
    char *seen = (char *)calloc((size_t)in->n + 1, 1);
    int bad = 0;
    for (int32_t k = 0; k < in->n && !bad; ++k) {
        int32_t x = tour[k];
        if (x < 1 || x > in->n || seen[x]) bad = 3; else seen[x] = 1;
    }
    free(seen);
    return bad;
}

/* ------------------------------------------------------------------------ */
/* Solution view: per anchor its route and index.                            */

typedef struct {
    int32_t n, m, W;
    const int32_t *tour, *rs;
    int32_t *route_of;      /* [W] anchor -> route */
    int32_t *idx_of;        /* [W] customer -> index in route (0-based); depot -> -1 */
    int64_t *rcost;         /* [m] */
} view_t;

static void view_init(view_t *v, const orc_inst *in, const int32_t *tour, const int32_t *rs)
{
    v->n = in->n; v->m = in->m; v->W = in->n + 1 + in->m;
    v->tour = tour; v->rs = rs;
    v->route_of = (int32_t *)calloc((size_t)v->W, sizeof(int32_t));
    v->idx_of = (int32_t *)calloc((size_t)v->W, sizeof(int32_t));
    v->rcost = (int64_t *)calloc((size_t)v->m, sizeof(int64_t));
    for (int32_t r = 0; r < v->m; ++r) {
        v->route_of[v->n + 1 + r] = r;
        v->idx_of[v->n + 1 + r] = -1;
        for (int32_t k = rs[r]; k < rs[r + 1]; ++k) {
            v->route_of[tour[k]] = r;
            v->idx_of[tour[k]] = k - rs[r];
        }
        v->rcost[r] = orc_route_cost(in, tour + rs[r], rs[r + 1] - rs[r]);
    }
}

static void view_free(view_t *v) { free(v->route_of); free(v->idx_of); free(v->rcost); }

static int is_customer(const view_t *v, int32_t a) { return a >= 1 && a <= v->n; }
static int is_anchor(const view_t *v, int32_t a) { return a >= 1 && a < v->W; }
static int32_t rlen(const view_t *v, int32_t r) { return v->rs[r + 1] - v->rs[r]; }
static const int32_t *rnodes(const view_t *v, int32_t r) { return v->tour + v->rs[r]; }

static int32_t pred_anchor(const view_t *v, int32_t u)
{
    int32_t r = v->route_of[u], i = v->idx_of[u];
    return i == 0 ? v->n + 1 + r : rnodes(v, r)[i - 1];
}

/* ------------------------------------------------------------------------ */
/* Route surgery: the new node lists of the touched routes.                  */

typedef struct { int32_t nr; int32_t r[2]; int32_t len[2]; int32_t *buf[2]; } moved_t;

static void cat(int32_t *dst, int32_t *len, const int32_t *src, int32_t cnt)
{
    if (cnt > 0) memcpy(dst + *len, src, (size_t)cnt * sizeof(int32_t));
    *len += cnt;
}

/* Returns 1 and fills mv if (op, a, b) is a candidate of the neighbourhood,
 * 0 otherwise.  mv->buf[0..1] must hold n+3 entries each. */
static int build_move(const view_t *v, int32_t op, int32_t a, int32_t b, moved_t *mv)
{
    if (op == 0 || op == 4 || op == 5) {
        int32_t k = (op == 0) ? 1 : op - 2;
        if (!is_customer(v, a) || !is_anchor(v, b)) return 0;
        int32_t A = v->route_of[a], i = v->idx_of[a], LA = rlen(v, A);
        if (i + k > LA) return 0;
        const int32_t *ra = rnodes(v, A);
        for (int32_t t = 0; t < k; ++t) if (ra[i + t] == b) return 0;
        if (b == pred_anchor(v, a)) return 0;
        int32_t B = v->route_of[b], j = v->idx_of[b];   /* j = -1: after the depot */
        int32_t *na = mv->buf[0];
        int32_t la = 0;
        cat(na, &la, ra, i);
        cat(na, &la, ra + i + k, LA - i - k);
        if (B != A) {
            const int32_t *rb = rnodes(v, B);
            int32_t *nb = mv->buf[1], lb = 0, LB = rlen(v, B);
            cat(nb, &lb, rb, j + 1);
            cat(nb, &lb, ra + i, k);
            cat(nb, &lb, rb + j + 1, LB - j - 1);
            mv->nr = 2; mv->r[0] = A; mv->r[1] = B; mv->len[0] = la; mv->len[1] = lb;
        } else {
            /* insert the run after b inside the reduced route */
            int32_t *nb = mv->buf[1], lb = 0;
            int32_t at = -1;
            if (j >= 0) { for (int32_t t = 0; t < la; ++t) if (na[t] == b) at = t; }
            cat(nb, &lb, na, at + 1);
            cat(nb, &lb, ra + i, k);
            cat(nb, &lb, na + at + 1, la - at - 1);
            memcpy(na, nb, (size_t)lb * sizeof(int32_t));
            mv->nr = 1; mv->r[0] = A; mv->len[0] = lb;
        }
        return 1;
    }
    if (op == 1) {
        if (!is_customer(v, a) || !is_customer(v, b) || !(a < b)) return 0;
        int32_t A = v->route_of[a], B = v->route_of[b];
        int32_t i = v->idx_of[a], j = v->idx_of[b];
        int32_t *na = mv->buf[0], la = 0;
        cat(na, &la, rnodes(v, A), rlen(v, A));
        if (A == B) {
            na[i] = b; na[j] = a;
            mv->nr = 1; mv->r[0] = A; mv->len[0] = la;
        } else {
            int32_t *nb = mv->buf[1], lb = 0;
            cat(nb, &lb, rnodes(v, B), rlen(v, B));
            na[i] = b; nb[j] = a;
            mv->nr = 2; mv->r[0] = A; mv->r[1] = B; mv->len[0] = la; mv->len[1] = lb;
        }
        return 1;
    }
    if (op == 2) {
        if (!is_customer(v, a) || !is_customer(v, b)) return 0;
        int32_t A = v->route_of[a];
        if (v->route_of[b] != A) return 0;
        int32_t i = v->idx_of[a], j = v->idx_of[b];
        if (!(i < j)) return 0;
        int32_t *na = mv->buf[0], la = 0;
        cat(na, &la, rnodes(v, A), rlen(v, A));
        for (int32_t lo = i, hi = j; lo < hi; ++lo, --hi) { int32_t t = na[lo]; na[lo] = na[hi]; na[hi] = t; }
        mv->nr = 1; mv->r[0] = A; mv->len[0] = la;
        return 1;
    }
    if (op == 3) {
        if (!is_anchor(v, a) || !is_anchor(v, b)) return 0;
        int32_t A = v->route_of[a], B = v->route_of[b];
        if (!(A < B)) return 0;
        int32_t i = v->idx_of[a], j = v->idx_of[b];     /* -1 for a depot anchor */
        const int32_t *ra = rnodes(v, A), *rb = rnodes(v, B);
        int32_t LA = rlen(v, A), LB = rlen(v, B);
        int32_t *na = mv->buf[0], la = 0, *nb = mv->buf[1], lb = 0;
        cat(na, &la, ra, i + 1);
        cat(na, &la, rb + j + 1, LB - j - 1);
        cat(nb, &lb, rb, j + 1);
        cat(nb, &lb, ra + i + 1, LA - i - 1);
        mv->nr = 2; mv->r[0] = A; mv->r[1] = B; mv->len[0] = la; mv->len[1] = lb;
        return 1;
    }
    if (op == 6 || op == 7) {
        /* run of k1 customers at a (k1 = 1 for op 6), run of 2 at b */
        const int32_t k1 = (op == 6) ? 1 : 2;
        if (!is_customer(v, a) || !is_customer(v, b)) return 0;
        if (op == 7 && !(a < b)) return 0;
        int32_t A = v->route_of[a], i = v->idx_of[a], LA = rlen(v, A);
        int32_t B = v->route_of[b], j = v->idx_of[b], LB = rlen(v, B);
        if (i + k1 > LA || j + 2 > LB) return 0;
        const int32_t *ra = rnodes(v, A), *rb = rnodes(v, B);
        if (A == B && !(i + k1 <= j || j + 2 <= i)) return 0;   /* the runs overlap */
        int32_t *na = mv->buf[0], la = 0;
        if (A != B) {
            int32_t *nb = mv->buf[1], lb = 0;
            cat(na, &la, ra, i);
            cat(na, &la, rb + j, 2);
            cat(na, &la, ra + i + k1, LA - i - k1);
            cat(nb, &lb, rb, j);
            cat(nb, &lb, ra + i, k1);
            cat(nb, &lb, rb + j + 2, LB - j - 2);
            mv->nr = 2; mv->r[0] = A; mv->r[1] = B; mv->len[0] = la; mv->len[1] = lb;
            return 1;
        }
        /* one route: first run (x, length kx) before second run (y, length ky) */
        int32_t x = i, kx = k1, y = j, ky = 2;
        if (j < i) { x = j; kx = 2; y = i; ky = k1; }
        cat(na, &la, ra, x);
        cat(na, &la, ra + y, ky);
        cat(na, &la, ra + x + kx, y - x - kx);
        cat(na, &la, ra + x, kx);
        cat(na, &la, ra + y + ky, LA - y - ky);
        mv->nr = 1; mv->r[0] = A; mv->len[0] = la;
        return 1;
    }
    return 0;
}

static int64_t delta_def(const orc_inst *in, const view_t *v, const moved_t *mv)
{
    int64_t d = 0;
    for (int32_t t = 0; t < mv->nr; ++t)
        d += orc_route_cost(in, mv->buf[t], mv->len[t]) - v->rcost[mv->r[t]];
    return d;
}

/* ------------------------------------------------------------------------ */
/* Sequence concatenation (Sections 4.2-4.3).                                */

typedef struct { int64_t D, LI, LO, LM, TD, TE, TL, TV; } seg_t;

static seg_t seg_of_node(const orc_inst *in, int32_t x)
{
    seg_t s;
    const int64_t p = in->pickup ? in->pickup[x] : 0;
    s.D = 0;
    s.LI = in->demand[x]; s.LO = p; s.LM = max64(s.LI, p);
    s.TD = in->service[x];
    s.TE = in->early[x]; s.TL = in->late[x]; s.TV = 0;
    return s;
}

/* sigma1 (+) sigma2 with travel t between last(sigma1) and first(sigma2).
 * Distance and load rules as printed (Section 4.3.1-4.3.2): with pickups the
 * incoming, outgoing and largest loads L_I, L_O, L_M; without them the
 * simplified rule in which L_M is additive.  For the time fields the offset
 * Delta_t = T_D(s1) - T_V(s1) + t: the printed extra "T_W(s1)" term names
 * no attribute (waiting is already inside T_D), so it is read as absent. */
static seg_t concat(const orc_inst *in, seg_t a, seg_t b, int64_t t)
{
    seg_t s;
    int64_t dt = a.TD - a.TV + t;
    int64_t dw = max64(b.TE - dt - a.TL, 0);
    int64_t dv = max64(a.TE + dt - b.TL, 0);
    s.D = a.D + t + b.D;
    s.LI = a.LI + b.LI;
    s.LO = a.LO + b.LO;
    s.LM = in->pickup ? max64(a.LM + b.LI, a.LO + b.LM) : a.LM + b.LM;
    s.TD = a.TD + t + dw + b.TD;
    s.TE = max64(b.TE - dt, a.TE) - dw;
    s.TL = min64(b.TL - dt, a.TL) + dv;
    s.TV = a.TV + dv + b.TV;
    return s;
}

static void seg_out(const seg_t *s, int64_t first, int64_t last, int64_t *o)
{
    o[0] = s->D; o[1] = s->LI; o[2] = s->LO; o[3] = s->LM;
    o[4] = s->TD; o[5] = s->TE; o[6] = s->TL; o[7] = s->TV; o[8] = first; o[9] = last;
}

void orc_seg_node(const orc_inst *in, int32_t v, int64_t *o)
{
    seg_t s = seg_of_node(in, v);
    seg_out(&s, v, v, o);
}

void orc_seg_concat(const orc_inst *in, const int64_t *p, const int64_t *q, int64_t *o)
{
    seg_t a = {p[0], p[1], p[2], p[3], p[4], p[5], p[6], p[7]};
    seg_t b = {q[0], q[1], q[2], q[3], q[4], q[5], q[6], q[7]};
    seg_t s = concat(in, a, b, DIST(in, p[9], q[8]));
    seg_out(&s, p[8], q[9], o);
}

/* Attribute matrix of one route: entry (i, j), 0 <= i <= j <= L+1, is the
 * subsequence of route positions i..j (position 0 = start depot, L+1 = end
 * depot); rev(i, j) is the same nodes visited from j back to i. */
typedef struct { int32_t L; int32_t *nd; seg_t *fw; seg_t *rv; } amat_t;

static seg_t *AM(const amat_t *m, int32_t i, int32_t j) { return &m->fw[(int64_t)i * (m->L + 2) + j]; }
static seg_t *AR(const amat_t *m, int32_t i, int32_t j) { return &m->rv[(int64_t)i * (m->L + 2) + j]; }

static void amat_build(const orc_inst *in, amat_t *m, const int32_t *nodes, int32_t L, int need_rev)
{
    int32_t P = L + 2;
    m->L = L;
    m->nd = (int32_t *)malloc((size_t)P * sizeof(int32_t));
    m->nd[0] = 0; m->nd[L + 1] = 0;
    for (int32_t k = 0; k < L; ++k) m->nd[k + 1] = nodes[k];
    m->fw = (seg_t *)malloc((size_t)P * P * sizeof(seg_t));
    m->rv = need_rev ? (seg_t *)malloc((size_t)P * P * sizeof(seg_t)) : NULL;
    for (int32_t i = 0; i < P; ++i) {
        *AM(m, i, i) = seg_of_node(in, m->nd[i]);
        for (int32_t j = i + 1; j < P; ++j)
            *AM(m, i, j) = concat(in, *AM(m, i, j - 1), seg_of_node(in, m->nd[j]), DIST(in, m->nd[j - 1], m->nd[j]));
        if (need_rev) {
            *AR(m, i, i) = seg_of_node(in, m->nd[i]);
            for (int32_t j = i + 1; j < P; ++j)
                *AR(m, i, j) = concat(in, seg_of_node(in, m->nd[j]), *AR(m, i, j - 1), DIST(in, m->nd[j], m->nd[j - 1]));
        }
    }
}

static void amat_free(amat_t *m) { free(m->nd); free(m->fw); free(m->rv); }

/* A neighbour route as a chain of pieces, folded left to right. */
typedef struct { seg_t s; int32_t first, last; } piece_t;

static piece_t pc_fw(const amat_t *m, int32_t i, int32_t j) { piece_t p = {*AM(m, i, j), m->nd[i], m->nd[j]}; return p; }
static piece_t pc_rv(const amat_t *m, int32_t i, int32_t j) { piece_t p = {*AR(m, i, j), m->nd[j], m->nd[i]}; return p; }

static int64_t chain_cost(const orc_inst *in, const piece_t *p, int32_t np_)
{
    seg_t s = p[0].s;
    for (int32_t k = 1; k < np_; ++k) s = concat(in, s, p[k].s, DIST(in, p[k - 1].last, p[k].first));
    int64_t c = s.D + (int64_t)in->w_load * max64(0, s.LM - in->capacity);
    if (in->has_tw) c += (int64_t)in->w_tw * s.TV;
    return c;
}

/* Delta of (op, a, b) by concatenation; the candidate must be valid. */
static int64_t delta_concat(const orc_inst *in, const view_t *v, const amat_t *am,
                            int32_t op, int32_t a, int32_t b)
{
    piece_t p[6], q[6];
    if (op == 0 || op == 4 || op == 5) {
        int32_t k = (op == 0) ? 1 : op - 2;
        int32_t A = v->route_of[a], i = v->idx_of[a] + 1;       /* 1-based positions */
        int32_t B = v->route_of[b], j = v->idx_of[b] + 1;       /* depot anchor: 0 */
        const amat_t *ma = &am[A], *mb = &am[B];
        int32_t LA = ma->L, LB = mb->L;
        piece_t run = pc_fw(ma, i, i + k - 1);
        if (A != B) {
            p[0] = pc_fw(ma, 0, i - 1); p[1] = pc_fw(ma, i + k, LA + 1);
            q[0] = pc_fw(mb, 0, j); q[1] = run; q[2] = pc_fw(mb, j + 1, LB + 1);
            return chain_cost(in, p, 2) + chain_cost(in, q, 3) - v->rcost[A] - v->rcost[B];
        }
        if (j >= i + k) {
            p[0] = pc_fw(ma, 0, i - 1); p[1] = pc_fw(ma, i + k, j); p[2] = run; p[3] = pc_fw(ma, j + 1, LA + 1);
        } else {   /* j < i - 1 */
            p[0] = pc_fw(ma, 0, j); p[1] = run; p[2] = pc_fw(ma, j + 1, i - 1); p[3] = pc_fw(ma, i + k, LA + 1);
        }
        return chain_cost(in, p, 4) - v->rcost[A];
    }
    if (op == 1) {
        int32_t A = v->route_of[a], B = v->route_of[b];
        int32_t i = v->idx_of[a] + 1, j = v->idx_of[b] + 1;
        if (A != B) {
            const amat_t *ma = &am[A], *mb = &am[B];
            p[0] = pc_fw(ma, 0, i - 1); p[1] = pc_fw(mb, j, j); p[2] = pc_fw(ma, i + 1, ma->L + 1);
            q[0] = pc_fw(mb, 0, j - 1); q[1] = pc_fw(ma, i, i); q[2] = pc_fw(mb, j + 1, mb->L + 1);
            return chain_cost(in, p, 3) + chain_cost(in, q, 3) - v->rcost[A] - v->rcost[B];
        }
        const amat_t *ma = &am[A];
        if (i > j) { int32_t t = i; i = j; j = t; }
        int32_t np_ = 0;
        p[np_++] = pc_fw(ma, 0, i - 1);
        p[np_++] = pc_fw(ma, j, j);
        if (j > i + 1) p[np_++] = pc_fw(ma, i + 1, j - 1);
        p[np_++] = pc_fw(ma, i, i);
        p[np_++] = pc_fw(ma, j + 1, ma->L + 1);
        return chain_cost(in, p, np_) - v->rcost[A];
    }
    if (op == 2) {
        int32_t A = v->route_of[a];
        int32_t i = v->idx_of[a] + 1, j = v->idx_of[b] + 1;
        const amat_t *ma = &am[A];
        p[0] = pc_fw(ma, 0, i - 1); p[1] = pc_rv(ma, i, j); p[2] = pc_fw(ma, j + 1, ma->L + 1);
        return chain_cost(in, p, 3) - v->rcost[A];
    }
    if (op == 6 || op == 7) {
        const int32_t k1 = (op == 6) ? 1 : 2;
        int32_t A = v->route_of[a], B = v->route_of[b];
        int32_t i = v->idx_of[a] + 1, j = v->idx_of[b] + 1;     /* 1-based */
        const amat_t *ma = &am[A], *mb = &am[B];
        if (A != B) {
            p[0] = pc_fw(ma, 0, i - 1); p[1] = pc_fw(mb, j, j + 1); p[2] = pc_fw(ma, i + k1, ma->L + 1);
            q[0] = pc_fw(mb, 0, j - 1); q[1] = pc_fw(ma, i, i + k1 - 1); q[2] = pc_fw(mb, j + 2, mb->L + 1);
            return chain_cost(in, p, 3) + chain_cost(in, q, 3) - v->rcost[A] - v->rcost[B];
        }
        int32_t x = i, kx = k1, y = j, ky = 2;
        if (j < i) { x = j; kx = 2; y = i; ky = k1; }
        int32_t np_ = 0;
        p[np_++] = pc_fw(ma, 0, x - 1);
        p[np_++] = pc_fw(ma, y, y + ky - 1);
        if (y > x + kx) p[np_++] = pc_fw(ma, x + kx, y - 1);
        p[np_++] = pc_fw(ma, x, x + kx - 1);
        p[np_++] = pc_fw(ma, y + ky, ma->L + 1);
        return chain_cost(in, p, np_) - v->rcost[A];
    }
    /* op 3: 2-opt* */
    int32_t A = v->route_of[a], B = v->route_of[b];
    int32_t i = v->idx_of[a] + 1, j = v->idx_of[b] + 1;
    const amat_t *ma = &am[A], *mb = &am[B];
    p[0] = pc_fw(ma, 0, i); p[1] = pc_fw(mb, j + 1, mb->L + 1);
    q[0] = pc_fw(mb, 0, j); q[1] = pc_fw(ma, i + 1, ma->L + 1);
    return chain_cost(in, p, 2) + chain_cost(in, q, 2) - v->rcost[A] - v->rcost[B];
}

/* ------------------------------------------------------------------------ */
/* Enumeration of the candidate set.                                         */

typedef struct {
    const orc_inst *in;
    const view_t *v;
    int method;
    amat_t *am;
    moved_t mv;
    /* best */
    int64_t best_delta; uint64_t best_idx; int32_t bop, ba, bb; int found;
    int64_t count;
    /* listing */
    uint64_t *idx_out; int64_t *delta_out; int64_t cap;
    int count_only;
    /* slice: visit only the candidates whose outermost enumeration index
     * (u, a, b, route r or route A, per operator) is phase mod stride */
    int32_t stride, phase;
} scan_t;

static int in_slice(const scan_t *s, int32_t outer)
{
    return s->stride <= 1 || outer % s->stride == s->phase;
}

/* Granular mask of the edge-based extraction (see tga_oracle.h). */
static int in_mask(const orc_inst *in, int32_t x, int32_t y)
{
    for (int32_t k = 0; k < in->theta; ++k)
        if (in->nbr[(int64_t)x * in->theta + k] == y) return 1;
    return 0;
}

static int granular_kept(const orc_inst *in, const view_t *v, int32_t op, int32_t a, int32_t b)
{
    const int32_t n = v->n;
    if (op == 2 || v->route_of[a] == v->route_of[b]) return 1;     /* intra-route */
    if (op == 0 || op == 4 || op == 5) return b > n || in_mask(in, a, b);
    if (op == 1 || op == 6 || op == 7) return in_mask(in, a, b) || in_mask(in, b, a);
    if (a > n && b > n) return 0;                                    /* 2-opt* */
    if (a > n || b > n) return 1;
    return in_mask(in, a, b) || in_mask(in, b, a);
}

static void visit(scan_t *s, int32_t op, int32_t a, int32_t b)
{
    const view_t *v = s->v;
    if (s->in->theta > 0 && !granular_kept(s->in, v, op, a, b)) return;
    s->count++;
    if (s->count_only) return;
    int64_t d;
    if (s->method == ORC_DEF) {
        if (!build_move(v, op, a, b, &s->mv)) { s->count--; return; }
        d = delta_def(s->in, v, &s->mv);
    } else {
        d = delta_concat(s->in, v, s->am, op, a, b);
    }
    uint64_t W = (uint64_t)v->W;
    uint64_t idx = (uint64_t)op * W * W + (uint64_t)a * W + (uint64_t)b;
    if (s->idx_out && s->count - 1 < s->cap) { s->idx_out[s->count - 1] = idx; s->delta_out[s->count - 1] = d; }
    if (!s->found || d < s->best_delta || (d == s->best_delta && idx < s->best_idx)) {
        s->found = 1; s->best_delta = d; s->best_idx = idx; s->bop = op; s->ba = a; s->bb = b;
    }
}

static void scan_all(scan_t *s, uint32_t mask)
{
    const view_t *v = s->v;
    int32_t n = v->n, m = v->m;
    /* op 0 and or-opt: run starting at customer u, destination anchor b */
    for (int32_t op = 0; op <= 7; ++op) {
        if (!(mask & (1u << op))) continue;
        if (op == 0 || op == 4 || op == 5) {
            int32_t k = (op == 0) ? 1 : op - 2;
            for (int32_t u = 1; u <= n; ++u) {
                if (!in_slice(s, u)) continue;
                int32_t A = v->route_of[u], i = v->idx_of[u];
                if (i + k > rlen(v, A)) continue;
                const int32_t *ra = rnodes(v, A);
                int32_t pu = pred_anchor(v, u);
                for (int32_t b = 1; b <= n + m; ++b) {
                    if (b == pu) continue;
                    int inrun = 0;
                    for (int32_t t = 0; t < k; ++t) if (ra[i + t] == b) inrun = 1;
                    if (inrun) continue;
                    visit(s, op, u, b);
                }
            }
        } else if (op == 1) {
            for (int32_t a = 1; a <= n; ++a) {
                if (!in_slice(s, a)) continue;
                for (int32_t b = a + 1; b <= n; ++b) visit(s, 1, a, b);
            }
        } else if (op == 6 || op == 7) {
            /* b starts a run of 2; a is a single customer (op 6) or starts a
             * run of 2 with a < b (op 7); the runs must not overlap */
            const int32_t k1 = (op == 6) ? 1 : 2;
            for (int32_t b = 1; b <= n; ++b) {
                if (!in_slice(s, b)) continue;
                int32_t B = v->route_of[b], j = v->idx_of[b];
                if (j + 2 > rlen(v, B)) continue;
                for (int32_t a = 1; a <= n; ++a) {
                    if (op == 7 && !(a < b)) continue;
                    int32_t A = v->route_of[a], i = v->idx_of[a];
                    if (i + k1 > rlen(v, A)) continue;
                    if (A == B && !(i + k1 <= j || j + 2 <= i)) continue;
                    visit(s, op, a, b);
                }
            }
        } else if (op == 2) {
            for (int32_t r = 0; r < m; ++r) {
                if (!in_slice(s, r)) continue;
                const int32_t *rr = rnodes(v, r);
                int32_t L = rlen(v, r);
                for (int32_t i = 0; i < L; ++i)
                    for (int32_t j = i + 1; j < L; ++j) visit(s, 2, rr[i], rr[j]);
            }
        } else {   /* op 3 */
            for (int32_t A = 0; A < m; ++A)
                for (int32_t B = A + 1; B < m && in_slice(s, A); ++B) {
                    const int32_t *ra = rnodes(v, A), *rb = rnodes(v, B);
                    for (int32_t i = -1; i < rlen(v, A); ++i) {
                        int32_t a = (i < 0) ? n + 1 + A : ra[i];
                        for (int32_t j = -1; j < rlen(v, B); ++j) {
                            int32_t b = (j < 0) ? n + 1 + B : rb[j];
                            visit(s, 3, a, b);
                        }
                    }
                }
        }
    }
}

int64_t orc_count_candidates(const orc_inst *in, const int32_t *tour, const int32_t *rs, uint32_t mask)
{
    scan_t s;
    view_t v;
    view_init(&v, in, tour, rs);
    memset(&s, 0, sizeof(s));
    s.in = in; s.v = &v; s.count_only = 1;
    scan_all(&s, mask);
    view_free(&v);
    return s.count;
}

int orc_best_move(const orc_inst *in, const int32_t *tour, const int32_t *rs, uint32_t mask,
                  int method, orc_move *out, int64_t *n_cands)
{
    scan_t s;
    view_t v;
    view_init(&v, in, tour, rs);
    memset(&s, 0, sizeof(s));
    s.in = in; s.v = &v; s.method = method;
    s.mv.buf[0] = (int32_t *)malloc((size_t)(in->n + 3) * sizeof(int32_t));
    s.mv.buf[1] = (int32_t *)malloc((size_t)(in->n + 3) * sizeof(int32_t));
    if (method == ORC_CONCAT) {
        s.am = (amat_t *)calloc((size_t)in->m, sizeof(amat_t));
        for (int32_t r = 0; r < in->m; ++r)
            amat_build(in, &s.am[r], tour + rs[r], rs[r + 1] - rs[r], (mask >> 2) & 1);
    }
    scan_all(&s, mask);
    out->found = s.found;
    out->delta = s.best_delta; out->idx = s.best_idx;
    out->op = s.bop; out->a = s.ba; out->b = s.bb;
    if (n_cands) *n_cands = s.count;
    if (s.am) { for (int32_t r = 0; r < in->m; ++r) amat_free(&s.am[r]); free(s.am); }
    free(s.mv.buf[0]); free(s.mv.buf[1]);
    view_free(&v);
    return 0;
}

int orc_best_move_slice(const orc_inst *in, const int32_t *tour, const int32_t *rs, uint32_t mask,
                        int method, int32_t phase, int32_t stride, orc_move *out, int64_t *n_cands)
{
    if (stride < 1 || phase < 0 || phase >= stride) return -1;
    scan_t s;
    view_t v;
    view_init(&v, in, tour, rs);
    memset(&s, 0, sizeof(s));
    s.in = in; s.v = &v; s.method = method;
    s.stride = stride; s.phase = phase;
    s.mv.buf[0] = (int32_t *)malloc((size_t)(in->n + 3) * sizeof(int32_t));
    s.mv.buf[1] = (int32_t *)malloc((size_t)(in->n + 3) * sizeof(int32_t));
    if (method == ORC_CONCAT) {
        s.am = (amat_t *)calloc((size_t)in->m, sizeof(amat_t));
        for (int32_t r = 0; r < in->m; ++r)
            amat_build(in, &s.am[r], tour + rs[r], rs[r + 1] - rs[r], (mask >> 2) & 1);
    }
    scan_all(&s, mask);
    out->found = s.found;
    out->delta = s.best_delta; out->idx = s.best_idx;
    out->op = s.bop; out->a = s.ba; out->b = s.bb;
    if (n_cands) *n_cands = s.count;
    if (s.am) { for (int32_t r = 0; r < in->m; ++r) amat_free(&s.am[r]); free(s.am); }
    free(s.mv.buf[0]); free(s.mv.buf[1]);
    view_free(&v);
    return 0;
}

int64_t orc_list_moves(const orc_inst *in, const int32_t *tour, const int32_t *rs, uint32_t mask,
                       int method, uint64_t *idx_out, int64_t *delta_out, int64_t cap)
{
    scan_t s;
    view_t v;
    view_init(&v, in, tour, rs);
    memset(&s, 0, sizeof(s));
    s.in = in; s.v = &v; s.method = method;
    s.idx_out = idx_out; s.delta_out = delta_out; s.cap = cap;
    s.mv.buf[0] = (int32_t *)malloc((size_t)(in->n + 3) * sizeof(int32_t));
    s.mv.buf[1] = (int32_t *)malloc((size_t)(in->n + 3) * sizeof(int32_t));
    if (method == ORC_CONCAT) {
        s.am = (amat_t *)calloc((size_t)in->m, sizeof(amat_t));
        for (int32_t r = 0; r < in->m; ++r)
            amat_build(in, &s.am[r], tour + rs[r], rs[r + 1] - rs[r], (mask >> 2) & 1);
    }
    scan_all(&s, mask);
    if (s.am) { for (int32_t r = 0; r < in->m; ++r) amat_free(&s.am[r]); free(s.am); }
    free(s.mv.buf[0]); free(s.mv.buf[1]);
    view_free(&v);
    return s.count;
}

/* Apply a candidate by route surgery and rewrite the giant tour. */
int orc_apply_move(const orc_inst *in, int32_t *tour, int32_t *rs, int32_t op, int32_t a, int32_t b)
{
    view_t v;
    view_init(&v, in, tour, rs);
    moved_t mv;
    mv.buf[0] = (int32_t *)malloc((size_t)(in->n + 3) * sizeof(int32_t));
    mv.buf[1] = (int32_t *)malloc((size_t)(in->n + 3) * sizeof(int32_t));
    int ok = build_move(&v, op, a, b, &mv);
    if (ok) {
        int32_t *nt = (int32_t *)malloc((size_t)(in->n + 1) * sizeof(int32_t));
        int32_t *nrs = (int32_t *)malloc((size_t)(in->m + 1) * sizeof(int32_t));
        int32_t w = 0;
        for (int32_t r = 0; r < in->m; ++r) {
            nrs[r] = w;
            int32_t t = -1;
            for (int32_t q = 0; q < mv.nr; ++q) if (mv.r[q] == r) t = q;
            if (t >= 0) { memcpy(nt + w, mv.buf[t], (size_t)mv.len[t] * sizeof(int32_t)); w += mv.len[t]; }
            else { memcpy(nt + w, tour + rs[r], (size_t)(rs[r + 1] - rs[r]) * sizeof(int32_t)); w += rs[r + 1] - rs[r]; }
        }
        nrs[in->m] = w;
        memcpy(tour, nt, (size_t)in->n * sizeof(int32_t));
        memcpy(rs, nrs, (size_t)(in->m + 1) * sizeof(int32_t));
        free(nt); free(nrs);
    }
    free(mv.buf[0]); free(mv.buf[1]);
    view_free(&v);
    return ok ? 0 : 1;
}

/* Best-improvement descent: evaluate, accept iff delta < 0, repeat, at most
 * max_steps applied moves.  The key log gets one entry per evaluation, so a
 * run that reaches a local optimum logs steps+1 keys (the last one is the
 * non-improving evaluation); an empty neighbourhood logs ~0.
 * key = ((uint32)(delta + 2^31) << 32) | idx. */
int64_t orc_descend(const orc_inst *in, int32_t *tour, int32_t *rs, uint32_t mask, int method,
                    int64_t max_steps, uint64_t *key_log, int64_t log_cap,
                    int64_t *cands_total, int64_t *n_evals)
{
    int64_t steps = 0, cands = 0, evals = 0;
    while (steps < max_steps) {
        orc_move mvb;
        int64_t nc = 0;
        orc_best_move(in, tour, rs, mask, method, &mvb, &nc);
        cands += nc;
        uint64_t key = ~(uint64_t)0;
        if (mvb.found)
            key = ((uint64_t)(uint32_t)(mvb.delta + 2147483648LL) << 32) | mvb.idx;
        if (key_log && evals < log_cap) key_log[evals] = key;
        ++evals;
        if (!mvb.found || mvb.delta >= 0) break;
        orc_apply_move(in, tour, rs, mvb.op, mvb.a, mvb.b);
        ++steps;
    }
    if (cands_total) *cands_total = cands;
    if (n_evals) *n_evals = evals;
    return steps;
}
