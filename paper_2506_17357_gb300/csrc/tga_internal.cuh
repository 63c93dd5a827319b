// Internal device-side layout of libtga (not part of the public ABI).
//
// Representation (Section 5.2 "attribute-based solution tensor", redesigned
// for one GPU): instead of a dense I x J x K x K tensor the context keeps
//   * the position sequence seq[p] of the giant tour with the start depot of
//     every route interleaved (route r occupies positions
//     route_start[r]+r .. route_start[r+1]+r, depot first), plus a sentinel
//     depot at position n+m -- the positional index P_r / P_pi of the
//     node-based extraction (Section 5.3.1, Eqs. "node_based1/2");
//   * per anchor the attributes of its prefix (start depot .. x) and of the
//     suffix after it (x+ .. end depot): distance, load and the time-window
//     attributes of Section 4.3.3 (T_D, T_E, T_L, T_V); with pickups also
//     the outgoing and largest loads L_O, L_M of Section 4.3.2;
//   * hoisted per-anchor constants that make every candidate an O(1)
//     integer expression (ERec);
//   * a copy of the distance matrix whose columns are in position order
//     (pcol[node][position]), so a tile of candidate pairs reads its distances
//     as contiguous row segments.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "tga.h"

namespace tga {

constexpr int kBig = 1 << 29;                 // offset that marks an invalid candidate
constexpr int kBestInit = (1 << 28) - 1;      // every valid |delta| is below 2^28
constexpr long long kRouteCostLim = 1LL << 27;
constexpr unsigned long long kNoKey = ~0ull;
constexpr int kColOff = 4;                    // pcol storage column of position q is q + 4
constexpr int kMaxTileCols = 256;             // widest tile (8 warps x 32 columns)
constexpr int kMaxW = 26754;                  // 6 * W^2 < 2^32
constexpr int kMaxWExt = 23170;               // 8 * W^2 < 2^32 (swaps of runs enabled)
constexpr unsigned kExtOps = 0xC0u;           // op ranks 6, 7: swaps of runs
constexpr int kXswapRows = 16, kXswapThreads = 128;   // swaps of runs: rows per block, columns per block
constexpr int kIntraVec = 10;                 // per-element int arrays of an intra-route view
constexpr int kIntraVecPD = 15;               // ... with the five load arrays of pickups

// Per-anchor base attributes (prefix through x, suffix after x).  Loads:
// loadf / loadg are the incoming loads L_I (total delivery) of the prefix
// and the suffix; lof, lmf are the prefix's outgoing and largest loads and
// lmg the suffix's largest load (Section 4.3.2; written only with pickups).
struct __align__(16) BRec {
    int node, route, idx, rlen;               // idx: 0 for the start depot, 1..L customers; rlen = L
    int tau, twf, distf, loadf;               // prefix: departure time after x, warp, distance, load
    int Lg, twg, distg, loadg;                // suffix after x: latest arrival (T_L), warp, distance, load
    int rcost, lof, lmf, lmg;                 // cost of the route; pickup loads
};

// Per-anchor hoisted constants of the inter-route candidate expressions.
// Groups g0..g3 are all a CVRP evaluation reads; g4..g6 add the time fields.
// succ / succ2 are the nodes of the next two elements of x's route (0 past
// its last customer, i.e. the end depot).
struct __align__(16) ERec {
    int route, d, rem1, K1;                   // g0
    int LQ, K2, LQd, Fc;                      // g1
    int Gc, loadf, loadgQ, anchor;            // g2
    int C2, ld2, C3, ld3;                     // g3
    int e, l, s, tau;                         // g4
    int Lg, tauP, E2, L2;                     // g5
    int Dm2, E3, L3, Dm3;                     // g6
    int node, idx, succ, succ2;               // g7: x's node and index; the nodes after it and after those
};

// Per-anchor hoisted constants of the inter-route candidates with pickups
// (P = prefix through x, S = suffix after x, P- = prefix through the
// predecessor; every load excess is that of the largest load L_M of the
// new route, Section 4.3.2).  A segment s inserted between x and x+ gives
// the excess max(IA + L_I(s), IB + L_M(s), IC + L_O(s)); a customer y in
// place of x gives max(SA + d_y, SB + max(d_y, p_y), SC + p_y); the 2-opt*
// route head(x) + tail after z gives max(HM(x) + TI(z), HO(x) + TM(z)).
struct __align__(16) PRec {
    int IA, IB, IC, pk;                       // LM_P + LI_S - Q, LO_P + LI_S - Q, LO_P + LM_S - Q; p_x
    int SA, SB, SC, mx;                       // the same with P-; max(d_x, p_x)
    int HM, HO, TI, TM;                       // LM_P - Q, LO_P - Q, LI_S, LM_S
    int LO2, LM2, LO3, LM3;                   // L_O, L_M of the runs of 2 and 3 starting at x
};

// Per-anchor constants of the swaps of runs (op ranks 6, 7: a customer with
// a run of two, two runs of two; Section 5.3.1 Swap with N1, N2 in {1, 2}).
// For customer x: the gap left by x alone (S1) or by the run x, x+ (S2) --
// prefix distance and warp through the predecessor plus suffix after the
// gap, minus the route cost (2^29 when the run does not exist) -- with the
// departure time after the predecessor and the latest arrival and load
// slack of the suffix; the run x, x+ as a time-window segment {E, L,
// D - T_V} with RC2 = its distance + w_tw * its warp and its load; and the
// node data of x.
struct __align__(16) XRec {
    int S1, tauP, Lg1, LQd1;                  // gap of x: removal constant, tau(x-), T_L after x, load - d_x - Q
    int S2, Lg2, LQd2, ld2;                   // gap of the run: removal constant, T_L after x+, load - run - Q, run load
    int E2, L2, Dm2, RC2;                     // the run as a segment; RC2 = dist + w_tw * warp
    int e, l, s, d;                           // x's window, service and demand
};

// load = total delivery (L_I); with pickups lo = total pickup (L_O) and lm
// = the largest load on board (L_M), which the cost penalises
struct RouteRec {
    int start, len, load, dist, tw, cost, lo, lm;
};

// A decoded move.  Routes, indices, lengths and depot positions are the
// ones before the move.
struct MovePlan {
    int op, a, b, delta;
    int A, B, i, j, k;        // routes, 1-based indices (0 = depot), run length
    int LA, LB, pA, pB;       // old lengths and depot positions
    int nLA, nLB;             // new lengths
};

// What one step rewrites, decoded once by the applying CTA and published to
// the CTAs that permute the columns of the position-ordered distance copy.
// Positions [b1, b1+n1) and [b2, b2+n2) change; with two routes lo < hi
// whose combined length is kept, every position strictly between them
// (including the depot of hi) moves by dl = new length - old length of lo.
struct StepPlan {
    MovePlan mp;
    int act;                  // 1: a move is applied this step
    int lo, hi, dl;
    int b1, n1, b2, n2;
    int oldLA, oldLB;
    long long oldcost;        // cost of routes A and B before the move
};

struct Control {
    unsigned long long best_key;              // min packed key of the running evaluation
    long long steps, evals, cand_total, cost, initial_cost, step_limit, cand_per_eval;
    long long sumL2, sumLm1, sumLm2;          // sum L^2, sum max(0,L-1), sum max(0,L-2)
    int done, status, pad1, local_opt;
    int maxL, maxLoad;                        // longest route and heaviest load (range check)
    int maxc, maxl, maxs, maxd, maxe, built;
    int last_op, last_a, last_b, last_delta;
    // batched descent: chunk scheduling of this job (evaluation phase, then
    // the column-permutation phase of the applied move)
    int next_chunk, done_chunks, finished, band_next;
    int band_done, pad2[3];
    // single-instance apply: the plan of the running step, its publication
    // flag, and the count of CTAs that finished the step's apply launch
    StepPlan plan;
    int plan_ready, plan_done, pad3[2];
    // persistent descent: grid-barrier arrivals (only grows within a launch)
    // and the step whose plan was last published; CTAs of the running
    // evaluation that have finished (the last one decodes the step's plan)
    unsigned long long bar_count;
    int plan_seq, eval_done;
    int plan_cta, pad5[3];                    // persistent descent: the CTA applying the step
    long long cand_op[8];                     // candidates evaluated per operator rank, all evaluations
    // edge-based extraction: sum max(0,L-1)^2, sum max(0,L-2)^2 (intra-route
    // or-opt counts) and the inter-route candidates the running evaluation
    // kept, per operator rank
    long long sumLm1sq, sumLm2sq;
    unsigned long long gcount[6];
    // debug build with index checks (TGA_BOUNDS_CHECK): the first failed
    // check -- site = file id * 100000 + source line, the index and the limit
    int bad_site, pad6;
    long long bad_index, bad_limit;
};

// The device workspace of one instance: every array a context (or the
// allocation-free entry point) carves out of one block of device memory,
// each piece 256-byte aligned.  Sized for n1 = n+1 nodes, m routes,
// w1 = W+1 anchor records and p = n+m+1 positions; pd adds the pickup
// records, xs the swaps-of-runs records.  Every offset and the total grow
// monotonically with each argument, so the layout at upper bounds of the
// four sizes bounds the layout of every instance below them.
struct WsLayout {
    size_t ctl, seq, pos, brec, erec, prec, xrec, rrec, seen, intra, saved, pcol, bytes;
};

constexpr size_t ws_align(size_t x) { return (x + 255) / 256 * 256; }

// Row pitch (ints) of the position-ordered distance copy for p positions.
constexpr size_t pcol_pitch(size_t p) { return (p + kMaxTileCols - 1) / kMaxTileCols * kMaxTileCols + 16; }

constexpr WsLayout workspace_pieces(size_t n1, size_t m, size_t w1, size_t p, bool pd, bool xs) {
    WsLayout L{};
    size_t off = 0;
    L.ctl = off;   off = ws_align(off + sizeof(Control));
    L.seq = off;   off = ws_align(off + sizeof(int) * p);
    L.pos = off;   off = ws_align(off + sizeof(int) * w1);
    L.brec = off;  off = ws_align(off + sizeof(BRec) * w1);
    L.erec = off;  off = ws_align(off + sizeof(ERec) * w1);
    L.prec = off;  off = ws_align(off + (pd ? sizeof(PRec) * w1 : 0));
    L.xrec = off;  off = ws_align(off + (xs ? sizeof(XRec) * w1 : 0));
    L.rrec = off;  off = ws_align(off + sizeof(RouteRec) * m);
    L.seen = off;  off = ws_align(off + sizeof(int) * n1);
    L.intra = off; off = ws_align(off + sizeof(int) * kIntraVecPD * (p + m));
    L.saved = off; off = ws_align(off + sizeof(int) * p);
    L.pcol = off;  off = ws_align(off + sizeof(int) * n1 * pcol_pitch(p));
    L.bytes = off;
    return L;
}

constexpr WsLayout workspace_layout(size_t n, size_t m, bool pd, bool xs) {
    return workspace_pieces(n + 1, m, n + m + 2, n + m + 1, pd, xs);
}

// Everything a kernel needs, passed by value.
// Default limits of the bounded device waits (nanoseconds).
constexpr long long kWaitPersistNs = 5LL * 1000 * 1000 * 1000;    // persistent descent: plan, grid barrier
constexpr long long kWaitApplyNs = 1LL * 1000 * 1000 * 1000;      // apply launch: plan publication
constexpr long long kWaitBatchNs = 20LL * 1000 * 1000 * 1000;     // batched descent: idle chunk polling
__host__ __device__ inline long long wait_limit(long long override_ns, long long dflt) {
    return override_ns < 0 ? dflt : override_ns;
}

struct Dev {
    int n, m, W, Wp, ldp;
    int nsm;                  // SMs of the device (grid caps of the helper launches)
    long long wait_ns;        // limit of every bounded device wait; < 0: each wait's default
    int Q, wL, wT, has_tw;
    int has_pd;               // pickups (VRPSPDTW; requires has_tw)
    int cvrp_by_route;        // CVRP intra-route moves: one warp per route (short routes) instead of one per customer
    unsigned op_mask;
    const int *dist, *demand, *service, *early, *late;
    const int *pickup;        // [n+1] or null
    int *tour, *route_start;
    int *seq;                 // [Wp]  anchor at each position (sentinel: W)
    int *pos_of;              // [W+1]
    BRec *brec;               // [W+1] (index W is the dummy record)
    ERec *erec;               // [W+1]
    PRec *prec;               // [W+1] (pickups only)
    XRec *xrec;               // [W+1] (swaps of runs only)
    RouteRec *rrec;           // [m]
    int *pcol;                // [(n+1) * ldp]
    Control *ctl;
    unsigned long long *log;  // optional key log
    long long log_cap;
    int *seen;                // [n+1] permutation check scratch
    int *scr_intra;           // [kIntraVecPD * (Wp+m)] per-element arrays of routes too long for shared memory
    // edge-based extraction (theta > 0): granular mask rows nbr[x*theta + k]
    // and, per entry, whether the reverse entry exists (x in the row of nbr[x*theta+k])
    int theta;
    const int *nbr;
    const unsigned char *nbr_rev;
};

__host__ __device__ inline int node_of(int anchor, int n) { return anchor <= n ? anchor : 0; }

// CVRP intra-route evaluation by route (a warp per route, the route's
// distance block in shared memory) when routes are short on average (at most
// 16 customers per route): long routes would serialise a whole route on one
// warp, so instances with long routes keep a warp per moved customer.  The
// swaps of runs always take the per-customer kernel.
__host__ __device__ inline int cvrp_intra_by_route(int n, int m, int has_tw, unsigned op_mask) {
    return (!has_tw && !(op_mask & kExtOps) && n <= 16 * m) ? 1 : 0;
}

// Debug build (compiled with -DTGA_BOUNDS_CHECK): every indexed access of
// the search state and the instance goes through TGA_IX(index, limit).  An
// index outside [0, limit) records the first failure in the control block
// (site = TGA_FILE_ID * 100000 + source line, the index, the limit), sets
// the status TGA_ERR_BOUNDS, and the access uses index 0 instead, so nothing
// outside the arrays is touched.  The release build compiles TGA_IX(i, lim)
// to (i).  File ids: 1 this header, 2 tga_device.cuh, 3 tga_kernels.cu,
// 4 tga_persist.cu, 5 tga_batch.cu, 6 tga_noalloc.cu.
#ifdef TGA_BOUNDS_CHECK
static __device__ __noinline__ long long tga_ix_fail(const Dev &d, long long i, long long lim, int site) {
    Control *C = d.ctl;
    if (atomicCAS(&C->bad_site, 0, site) == 0) {
        C->bad_index = i;
        C->bad_limit = lim;
    }
    atomicCAS(&C->status, 0, TGA_ERR_BOUNDS);
    return 0;
}
__device__ __forceinline__ long long tga_ix(const Dev &d, long long i, long long lim, int site) {
    return ((unsigned long long)i < (unsigned long long)lim) ? i : tga_ix_fail(d, i, lim, site);
}
#define TGA_IX(i, lim) tga_ix(d, (long long)(i), (long long)(lim), TGA_FILE_ID * 100000 + __LINE__)
#else
#define TGA_IX(i, lim) (i)
#endif
#undef TGA_FILE_ID
#define TGA_FILE_ID 1

__device__ __forceinline__ int dmat(const Dev &d, int i, int j) {
    return __ldg(d.dist + (size_t)TGA_IX(i, d.n + 1) * (d.n + 1) + TGA_IX(j, d.n + 1));
}

// Time-window segment in the form of Section 4.3.3: earliest start E,
// latest start L, duration D (service + travel + waiting), warp TW; plus
// distance and load.  "out" carries the length of the edge leaving the
// segment's last node, so a chain of consecutive route elements can be
// concatenated by a scan without looking the edge up again.
struct Seg {
    int E, L, D, TW, dist, load, out;
};

// a (+) b, the concatenation of Section 4.3 with travel time a.out between
// them.  Delta_t = T_D(a) - T_V(a) + t (the printed extra "T_W(a)" names no
// attribute; waiting is already inside T_D, so it is read as absent).
__device__ __forceinline__ Seg seg_cat(const Seg &a, const Seg &b) {
    const int t = a.out;
    const int dt = a.D - a.TW + t;
    const int dw = max(b.E - dt - a.L, 0);
    const int dv = max(a.E + dt - b.L, 0);
    Seg s;
    s.D = a.D + t + dw + b.D;
    s.E = max(b.E - dt, a.E) - dw;
    s.L = min(b.L - dt, a.L) + dv;
    s.TW = a.TW + dv + b.TW;
    s.dist = a.dist + t + b.dist;
    s.load = a.load + b.load;
    s.out = b.out;
    return s;
}

__device__ __forceinline__ Seg seg_node(const Dev &d, int node, int out) {
    Seg s;
    if (d.has_tw) {
        s.E = __ldg(d.early + node); s.L = __ldg(d.late + node); s.D = __ldg(d.service + node);
    } else {
        s.E = 0; s.L = 0; s.D = 0;
    }
    s.TW = 0; s.dist = 0; s.load = __ldg(d.demand + node); s.out = out;
    return s;
}

// Loads of a segment with pickups (Section 4.3.2): incoming L_I (deliveries
// on board when it starts), outgoing L_O (pickups on board when it ends) and
// the largest load L_M.  {0, 0, 0} (a depot) is neutral on both sides
// because L_M >= L_I and L_M >= L_O for every segment.
struct Ld {
    int i, o, m;
};

__device__ __forceinline__ Ld ld_cat(const Ld &a, const Ld &b) {
    Ld s;
    s.i = a.i + b.i;
    s.o = a.o + b.o;
    s.m = max(a.m + b.i, a.o + b.m);
    return s;
}

__device__ __forceinline__ Ld ld_node(const Dev &d, int node) {
    Ld s;
    s.i = __ldg(d.demand + node);
    s.o = __ldg(d.pickup + node);
    s.m = max(s.i, s.o);
    return s;
}

// Largest load of prefix (o, m) + segment g + suffix (si, sm): the new
// route's L_M when the suffix's L_I and L_M are si and sm.
__device__ __forceinline__ int ld_close(int o, int m, const Ld &g, int si, int sm) {
    const int m1 = max(m + g.i, o + g.m);
    return max(m1 + si, o + g.o + sm);
}

__device__ __forceinline__ unsigned long long pack_key(int delta, unsigned idx) {
    return ((unsigned long long)((unsigned)delta + 0x80000000u) << 32) | idx;
}

__device__ __forceinline__ int key_delta(unsigned long long k) {
    return (int)((unsigned)(k >> 32) - 0x80000000u);
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        unsigned long long o = __shfl_xor_sync(0xffffffffu, v, off);
        v = o < v ? o : v;
    }
    return v;
}

// Block-wide min of a packed key, one atomicMin per block into *dst.
__device__ inline void block_min_to(unsigned long long key, unsigned long long *dst) {
    __shared__ unsigned long long s_red[32];
    key = warp_min_u64(key);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_red[warp] = key;
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        unsigned long long v = lane < nw ? s_red[lane] : kNoKey;
        v = warp_min_u64(v);
        if (lane == 0 && v != kNoKey) atomicMin(dst, v);
    }
}

// Strip-major order of the inter-route tiles (TR rows x TC columns with
// g = TC / TR an integer, nrt row tiles): column strip J holds the row tiles
// I that contain a pair p < q, i.e. I < n_J = min((J+1) g, nrt) -- the same
// tiles as the row-major tile list.  strip_before(J) counts the tiles of
// strips 0 .. J-1 (strips below nrt / g are not capped).
__host__ __device__ inline long long strip_before(int J, int nrt, int g) {
    const long long K = J < nrt / g ? J : nrt / g;
    return (long long)g * K * (K + 1) / 2 + (long long)(J - K) * nrt;
}

// Candidates of one evaluation per operator rank from the route-length sums
// (closed form; 0 for disabled operators).
__host__ __device__ inline long long op_candidates(int op, long long n, long long m, unsigned mask,
                                                   long long sumL2, long long sumLm1, long long sumLm2) {
    if (!(mask & (1u << op))) return 0;
    const long long A = n + m;
    switch (op) {
        case 0: return n * (A - 2);
        case 1: return n * (n - 1) / 2;
        case 2: return (sumL2 - n) / 2;
        case 3: return (A * A - (sumL2 + 2 * n + m)) / 2;
        case 4: return sumLm1 * (A - 3);
        case 5: return sumLm2 * (A - 4);
        // runs of two: sumLm1 of them; a customer outside the run (n - 2 each),
        // and pairs of runs minus the overlapping pairs (sumLm2: one per
        // three consecutive customers)
        case 6: return sumLm1 * (n - 2);
        default: return sumLm1 * (sumLm1 - 1) / 2 - sumLm2;
    }
}

__host__ __device__ inline long long candidate_count(long long n, long long m, unsigned mask,
                                                     long long sumL2, long long sumLm1,
                                                     long long sumLm2) {
    long long c = 0;
    for (int op = 0; op < 8; ++op) c += op_candidates(op, n, m, mask, sumL2, sumLm1, sumLm2);
    return c;
}

// Intra-route candidates of one evaluation per operator rank (closed form):
// a route of L customers has L(L-1) relocate and L(L-1)/2 swap and 2-opt
// candidates, (L-1)(L-2) or-opt-2 and (L-2)(L-3) or-opt-3 candidates.
__host__ __device__ inline long long intra_candidates(int op, long long n, unsigned mask, long long sumL2,
                                                      long long sumLm1, long long sumLm2, long long sumLm1sq,
                                                      long long sumLm2sq) {
    if (!(mask & (1u << op))) return 0;
    switch (op) {
        case 0: return sumL2 - n;
        case 1: case 2: return (sumL2 - n) / 2;
        case 3: return 0;
        case 4: return sumLm1sq - sumLm1;
        default: return sumLm2sq - sumLm2;
    }
}

// Count one evaluation of the current state (evaluation counter, candidate
// totals, per operator).  Edge-based extraction: the closed-form intra-route
// candidates plus the inter-route ones the evaluation kernel counted.
__device__ inline void count_evaluation(const Dev &d, Control *C) {
    C->evals += 1;
    if (d.theta > 0) {
        long long tot = 0;
        for (int op = 0; op < 6; ++op) {
            const long long c = intra_candidates(op, d.n, d.op_mask, C->sumL2, C->sumLm1, C->sumLm2,
                                                 C->sumLm1sq, C->sumLm2sq) + (long long)C->gcount[op];
            C->cand_op[op] += c;
            tot += c;
            C->gcount[op] = 0;
        }
        C->cand_total += tot;
        return;
    }
    C->cand_total += C->cand_per_eval;
    for (int op = 0; op < 8; ++op)
        C->cand_op[op] += op_candidates(op, d.n, d.m, d.op_mask, C->sumL2, C->sumLm1, C->sumLm2);
}

// Batched descent (tga_batch.cu): one persistent launch over many contexts.
constexpr int kBatchThreads = 256;            // 8 warps: 256-column inter tiles
constexpr int kBandRowsPerChunk = 32;
constexpr long long kChunkPairs = 1LL << 17;  // target candidate pairs per evaluation chunk
struct BatchJob {
    Dev d;
    int tr, nrt, nct, nchunks;                // tile rows; row/column tiles; evaluation chunks per step
    int nband, ninter;                        // column-permutation chunks; inter-route chunks
    const int *chunk_t0;                      // [ninter+1] first row tile of each inter-route chunk
};
struct BatchState {
    int build_next, jobs_done, status, pad;
};
// mode 0: build + descend; 1: build + one evaluation; 2: one evaluation of
// already-built jobs (autotuner timing)
int launch_batch(const BatchJob *jobs_dev, int njobs, BatchState *state_dev, long long max_steps, int mode,
                 int max_tr, int max_wp, long long idle_limit_ns, cudaStream_t s);

// Kernel entry points (tga_kernels.cu).
void launch_check_instance(const Dev &d, cudaStream_t s);
void launch_build(const Dev &d, cudaStream_t s);
// tail > 0: the evaluation of a descent step whose inter- and intra-route
// launches have `tail` CTAs in total (eval_blocks); the last CTA to finish
// decodes the step's plan for the apply launch that follows.
// strip > 0: the strip-major inter-route kernel (k_eval_strip) with `strip`
// CTAs (strip_grid); else one CTA per tile (k_eval_inter).
void launch_eval(const Dev &d, const int2 *tiles, int ntiles, int rows, int warps,
                 cudaStream_t s, int rs = 1, int tail = 0, int strip = 0);
void launch_inter(const Dev &d, const int2 *tiles, int ntiles, int rows, int warps,
                  cudaStream_t s, int rs = 1, int tail = 0, int strip = 0);
// Grid of the strip-major kernel for a tile shape: every CTA the device can
// hold at once, at most one per tile; 0 if the shape is not a strip shape
// (rows 16 or 32, 4 or 8 warps).
int strip_grid(const Dev &d, int rows, int warps, long long ntiles);
size_t strip_smem_bytes(int rows, int warps, bool pd);
void launch_intra(const Dev &d, cudaStream_t s, int tail = 0);
// swaps of runs between routes (op ranks 6, 7; no-op unless enabled)
void launch_xswap(const Dev &d, cudaStream_t s, int tail = 0);
int eval_blocks(const Dev &d, int ntiles, int strip = 0);
// Edge-based extraction (theta > 0): threads per CTA, mask-entry CTAs, and
// depot CTAs (row tiles of `rows` positions x `chunks` chunks of `dc` start
// depots).
struct EdgeGrid {
    int threads, nmask, ndepot, rows, chunks, dc;
};
EdgeGrid edge_grid(const Dev &d);
// pre = 1: apply the plan decoded by the evaluation's last CTA (descent
// steps); else decode *ext (or the best key) in the launch itself.
void launch_apply(const Dev &d, const tga_move *ext, unsigned long long cond, int use_cond,
                  cudaStream_t s, int pre = 0);
void launch_sync_solution(const Dev &d, cudaStream_t s);
void launch_finalize(const Dev &d, tga_move *out, cudaStream_t s);
void launch_begin(const Dev &d, long long max_steps, cudaStream_t s);
// Persistent single-instance descent (tga_persist.cu): one cooperative
// launch; returns TGA_OK or an error code (nothing launched on error).
int launch_persist(const Dev &d, const int2 *tiles, int ntiles, int rows, int warps, int rs, cudaStream_t s,
                   int *grid_out);
// Edge-based extraction: validate the mask rows and mark reverse entries;
// *bad_dev (device int) is set when an entry is not another customer.
void launch_granular_setup(const Dev &d, unsigned char *rev, int *bad_dev, cudaStream_t s);
size_t inter_smem_bytes(int rows, int warps, bool pd = false);
int setup_kernel_attrs(int max_band);

}  // namespace tga
