/*
 * CPU oracle for best-improvement VRP local search -- TEST INFRASTRUCTURE.
 *
 * Only the tests, the package's smoke check and the benchmark's CPU-baseline
 * leg may load this library.  The GPU product path never calls it and shares
 * no code, header, table or helper with it.
 *
 * Two independent evaluators of the same neighbourhood:
 *   ORC_DEF    -- the plain definition: build every modified route explicitly
 *                 and cost it by forward simulation (Section 2 objective with
 *                 the time-warp relaxation of Section 4.3.3).
 *   ORC_CONCAT -- the paper's sequence concatenation (Section 4.1-4.3): per
 *                 route attribute matrices (Section 4.2) holding D, L_I, L_O,
 *                 L_M, T_D, T_E, T_L, T_V for every subsequence, and each neighbour's
 *                 route attributes obtained by the concatenation operator.
 * Both return the lexicographically smallest (delta, move index).
 *
 * Solution format: giant tour tour[n] (customers in route order) and
 * route_start[m+1]; route r is tour[route_start[r] .. route_start[r+1]-1]
 * between two visits of depot 0.  Anchors: customers 1..n, and the start
 * depot of route r is anchor n+1+r; W = n+1+m.  Move index
 * idx = op*W*W + a*W + b with op ranks 0 relocate, 1 swap, 2 2-opt,
 * 3 2-opt*, 4 or-opt(2), 5 or-opt(3), 6 swap of a customer with a run of
 * two (a the customer, b the run's first), 7 swap of two runs of two (a < b).
 */
#ifndef TGA_ORACLE_H
#define TGA_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* theta > 0 restricts the neighbourhood to the edge-based extraction of
 * Section 5.3.1 with a granular mask: nbr[x*theta + k] (k < theta) are the
 * customers y with M[x][y] = 1 for customer x (row 0 unused).  Intra-route
 * candidates are always evaluated (route-based extraction); an inter-route
 * candidate (op, a, b) is kept when
 *   relocate / or-opt (the run starting at a moves after b): b is a start
 *     depot, or M[a][b];
 *   swap (ranks 1, 6, 7): M[a][b] or M[b][a];
 *   2-opt*: exactly one of a, b is a start depot, or M[a][b] or M[b][a].
 * theta = 0: the full neighbourhood (node-based extraction). */
/* pickup: NULL for the CVRP and VRPTW; for the VRPSPDTW the pickup
 * quantity p_x of every node (n+1 entries, p_0 = 0).  A vehicle leaves the
 * depot with every delivery of its route on board, drops d_x and collects
 * p_x at each customer; the capacity term uses the largest load on board
 * (Section 4.3.2, attributes L_I, L_O, L_M). */
typedef struct {
    int32_t n, m, capacity, has_tw, w_load, w_tw;
    const int32_t *dist;                 /* (n+1)*(n+1), row-major */
    const int32_t *demand, *service, *early, *late;   /* n+1 each */
    int32_t theta;
    const int32_t *nbr;                  /* (n+1)*theta, or NULL when theta = 0 */
    const int32_t *pickup;               /* n+1, or NULL */
} orc_inst;

typedef struct {
    int64_t delta;      /* cost(new) - cost(old) over the touched routes */
    uint64_t idx;       /* op*W*W + a*W + b */
    int32_t op, a, b;
    int32_t found;      /* 0: the neighbourhood is empty */
} orc_move;

enum { ORC_DEF = 0, ORC_CONCAT = 1 };

int64_t orc_route_cost(const orc_inst *in, const int32_t *nodes, int32_t len);
/* Largest load on board along the route (the total delivery without pickups). */
int64_t orc_route_peak_load(const orc_inst *in, const int32_t *nodes, int32_t len);
int64_t orc_route_warp(const orc_inst *in, const int32_t *nodes, int32_t len);
int64_t orc_solution_cost(const orc_inst *in, const int32_t *tour, const int32_t *route_start);
int     orc_check_solution(const orc_inst *in, const int32_t *tour, const int32_t *route_start);
int64_t orc_count_candidates(const orc_inst *in, const int32_t *tour,
                             const int32_t *route_start, uint32_t op_mask);
int     orc_best_move(const orc_inst *in, const int32_t *tour, const int32_t *route_start,
                      uint32_t op_mask, int method, orc_move *out, int64_t *n_cands);
/* The same over one slice of the candidate set: only the candidates whose
 * outermost enumeration index -- the moved customer (relocate, or-opt), the
 * first customer a (swap), the run's first b (ranks 6, 7), the route
 * (2-opt) or the first route A (2-opt*) -- is phase modulo stride
 * (0 <= phase < stride; else -1).  The stride slices partition the set, so
 * the smallest (delta, idx) over all of them is orc_best_move's and their
 * counts add up to its count.  Used to spread one evaluation over several
 * processes (the CPU baseline on all host cores). */
int     orc_best_move_slice(const orc_inst *in, const int32_t *tour, const int32_t *route_start,
                            uint32_t op_mask, int method, int32_t phase, int32_t stride,
                            orc_move *out, int64_t *n_cands);
int64_t orc_list_moves(const orc_inst *in, const int32_t *tour, const int32_t *route_start,
                       uint32_t op_mask, int method, uint64_t *idx_out, int64_t *delta_out,
                       int64_t cap);
int     orc_apply_move(const orc_inst *in, int32_t *tour, int32_t *route_start,
                       int32_t op, int32_t a, int32_t b);
int64_t orc_descend(const orc_inst *in, int32_t *tour, int32_t *route_start, uint32_t op_mask,
                    int method, int64_t max_steps, uint64_t *key_log, int64_t log_cap,
                    int64_t *cands_total, int64_t *n_evals);
/* Concatenation of two segments (Section 4.3), exposed for property tests.
 * seg = {D, LI, LO, LM, TD, TE, TL, TV, first, last}. */
void    orc_seg_node(const orc_inst *in, int32_t v, int64_t *seg8);
void    orc_seg_concat(const orc_inst *in, const int64_t *s1, const int64_t *s2, int64_t *out8);

#ifdef __cplusplus
}
#endif
#endif
