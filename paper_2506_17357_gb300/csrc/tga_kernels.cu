// libtga kernels for sm_103a.
//
// Step map (Section 5.1 workflow, five steps of Section 5.3):
//   k_build_*      tensor initialisation: positions + per-anchor attributes
//                  (warp-parallel prefix/suffix scans with the concatenation
//                  operator of Section 4.3), route totals, hoisted constants.
//   k_eval_inter   Extraction + Concatenation + Differencing + Evaluation for
//                  every inter-route pair in one fused pass (node-based
//                  3-Seq, Section 5.3.1, Eqs. "node_based1/2"): each thread
//                  owns one column anchor v, its warp walks the rows u of a
//                  tile whose distances sit in shared memory, every candidate
//                  delta is an O(1) integer expression in registers, and the
//                  argmin (Eq. "min_obj") is a per-thread running minimum
//                  reduced by warp shuffles and one 64-bit atomicMin per
//                  block over packed (delta, move index) keys.
//   k_eval_intra   the same for intra-route candidates with time windows
//                  (route-based extraction of Section 5.3.1): one CTA per
//                  route builds the route's subsequence tables (Section 4.2)
//                  in shared memory and takes the (i, j) pairs in parallel;
//                  k_eval_intra_cvrp: one warp per CVRP route.
//   k_apply        Tensor update (Section 5.3.5) on the device: CTA 0 decodes
//                  the best key, rewrites the positions and rebuilds the
//                  attributes of the <= 2 touched routes; the other CTAs keep
//                  the position-ordered distance copy in step (a permutation
//                  of the changed columns of every row).
//   k_sync_solution  write the caller's giant tour and route offsets back
//                  once a descent (or an applied move) is done.
#include <cstdio>

#define TGA_LDG(p) __ldg(p)
#include "tga_device.cuh"
#undef TGA_FILE_ID
#define TGA_FILE_ID 3

namespace tga {

// ---------------------------------------------------------------------------
// single-instance kernels (one launch per phase; state changes only between
// launches)

__global__ void __launch_bounds__(256) k_check_instance(Dev d) { check_instance_tiles(d, blockIdx.x, gridDim.x); }

__global__ void k_build_positions(Dev d) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    build_positions_route(d, r);
}

__global__ void k_check_perm(Dev d) { check_perm_one(d, blockIdx.x * blockDim.x + threadIdx.x + 1); }

__global__ void k_build_routes(Dev d) {
    if (d.ctl->status != 0) return;
    const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (r >= d.m) return;
    if (d.has_pd) rebuild_route<true>(d, r, threadIdx.x & 31);
    else if (d.op_mask & kExtOps) rebuild_route<false, true>(d, r, threadIdx.x & 31);
    else rebuild_route<false>(d, r, threadIdx.x & 31);
}

__global__ void __launch_bounds__(1024) k_build_finish(Dev d) { finish_block(d); }

__global__ void k_pcol_init(Dev d) {
    pcol_init_range(d, blockIdx.x * (long long)blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x);
}

// tail > 0: a descent step's evaluation (see eval_tail); every launch of
// the step's evaluation returns at once on a finished descent.
// The finished-descent flag is loaded first but tested only before the key
// is folded in, so its round trip overlaps the staging loads (a launch on a
// finished descent does its work and discards it).
template <bool TW, bool OR, bool PD = false, bool GATE = false>
__global__ void __launch_bounds__(256) k_eval_inter(Dev d, int TR, int RS, int tail) {
    const int done = *(volatile int *)&d.ctl->done;
    extern __shared__ __align__(16) int smem[];
    const int TC = (int)blockDim.x / RS;
    const int2 tl = tile_of(blockIdx.x, d.Wp, TR, TC);
    int best = kBestInit;
    unsigned bidx = 0xffffffffu;
    inter_tile<TW, OR, PD, GATE>(d, tl.x * TR, tl.y * TC, TR, RS, smem, best, bidx);
    if (done) return;
    const unsigned long long key = (bidx != 0xffffffffu) ? pack_key(best, bidx) : kNoKey;
    block_min_to(key, &d.ctl->best_key);
    if (tail && threadIdx.x == 0) eval_tail(d, tail);
}

// ---------------------------------------------------------------------------
// Strip-major inter-route evaluation (the per-step paths).  The tiles of the
// pair triangle are ordered column strip by column strip (strip J: the row
// tiles I = 0 .. n_J - 1 that hold a pair p < q, see strip_before) and every
// CTA of a grid sized to the resident capacity walks one contiguous range of
// that order.  So a CTA keeps its column anchors' constants in registers for
// a whole strip instead of gathering them for every tile, and it stages the
// next tile's distance rows and row records with asynchronous copies
// (cp.async, global -> shared, 16 B each) into the second of two buffers
// while it computes the current tile.  The candidates and their order are
// those of k_eval_inter (the same row loop, inter_rows).


template <bool TW, bool OR, bool PD = false, bool GATE = false>
__global__ void __launch_bounds__(256, TW ? 3 : 4) k_eval_strip(Dev d, int TR, long long T, int tail) {
    const int done = *(volatile int *)&d.ctl->done;
    extern __shared__ __align__(16) int smem[];
    const long long t0 = (long long)blockIdx.x * T / gridDim.x;
    const long long t1 = (long long)(blockIdx.x + 1) * T / gridDim.x;
    int best = kBestInit;
    unsigned bidx = 0xffffffffu;
    strip_walk<TW, OR, PD, GATE>(d, TR, T, t0, t1, smem, best, bidx);
    if (done) return;
    const unsigned long long key = (bidx != 0xffffffffu) ? pack_key(best, bidx) : kNoKey;
    block_min_to(key, &d.ctl->best_key);
    if (tail && threadIdx.x == 0) eval_tail(d, tail);
}

// Edge-based extraction (ETGA, Section 5.3.1): the kept inter-route pairs
// of a customer u are u's theta mask entries and the start depots of the
// other routes.  One launch, two kinds of CTA (blockDim threads each):
//
//   mask CTAs (the first ceil(n*theta / blockDim)): one thread per directed
//     mask entry (u, v).  The first loads fetch the entry, u's records and
//     u's position; the second v's records and position and the distances that
//     need only v (c(u,v), c(u+,v), c(u-,v) from the position-ordered copy's
//     row v at u's predecessor position); the third the distances to v's
//     successor (named in v's record) and c(u, v-) from row u of the copy at
//     v's predecessor position.
//   depot CTAs: the (customer, start depot) pairs are dense -- every
//     customer with every other route -- so they are tiled like the
//     node-based kernel.  A CTA takes R consecutive positions (rows) and a
//     chunk of start depots, one per thread.  The rows' records sit in
//     shared memory with the depot's distances to them (row 0 of the
//     position-ordered copy); each thread holds its depot's record and the
//     copy's row of the depot's successor node f across the R+4 positions,
//     because c(u, f), c(u+, f), c(u++, f) of the row at position p are that
//     row's columns p, p+1, p+2 (the matrix is symmetric).  No distance is
//     gathered.
//
// The per-operator counts of the kept candidates are folded into the
// control block before the key, so the evaluation's last CTA sees them.
constexpr int kEdgeMaxThreads = 128;

template <bool TW, bool OR>
__device__ __forceinline__ void edge_mask_item(const Dev &d, long long item, int &best, unsigned &bidx,
                                               unsigned &evaluated) {
    const int th = d.theta;
    const int u = (int)(item / th) + 1, k = (int)(item - (long long)(u - 1) * th);
    const size_t e = (size_t)u * th + k;
    const int v = __ldg(d.nbr + TGA_IX(e, (long long)(d.n + 1) * d.theta));
    const bool rev = __ldg(d.nbr_rev + TGA_IX(e, (long long)(d.n + 1) * d.theta)) != 0;
    const int4 *ur = reinterpret_cast<const int4 *>(d.erec + TGA_IX(u, d.W + 1));
    const int4 u0 = __ldg(ur + 0), u1 = __ldg(ur + 1), u2 = __ldg(ur + 2), u7 = __ldg(ur + 7);
    const int4 z = make_int4(0, 0, 0, 0);
    const int4 u3 = OR ? __ldg(ur + 3) : z;
    const int4 u4 = TW ? __ldg(ur + 4) : z, u5 = TW ? __ldg(ur + 5) : z;
    const int4 u6 = (TW && OR) ? __ldg(ur + 6) : z;
    const int pu = __ldg(d.pos_of + TGA_IX(u, d.W + 1));
    // second loads: v's records, its position, and the distances that need only v
    const int4 *vr = reinterpret_cast<const int4 *>(d.erec + TGA_IX(v, d.W + 1));
    const int4 v0 = __ldg(vr + 0), v1 = __ldg(vr + 1), v2 = __ldg(vr + 2), v7 = __ldg(vr + 7);
    const int4 v4 = TW ? __ldg(vr + 4) : z, v5 = TW ? __ldg(vr + 5) : z;
    const int pv = __ldg(d.pos_of + TGA_IX(v, d.W + 1));
    const int up = u7.z, upp = u7.w;
    EdgeStencil t;
    t.t00 = dmat(d, u, v);
    t.t10 = dmat(d, up, v);
    t.tm10 = __ldg(d.pcol + (size_t)TGA_IX(v, d.n + 1) * d.ldp + TGA_IX(pu - 1 + kColOff, d.ldp));
    // third loads: the distances to v's successor, and c(u, v-)
    const int vp = v7.z;
    t.t01 = dmat(d, u, vp);
    t.t11 = dmat(d, up, vp);
    t.t21 = OR ? dmat(d, upp, vp) : 0;
    t.t0m1 = __ldg(d.pcol + (size_t)TGA_IX(u, d.n + 1) * d.ldp + TGA_IX(pv - 1 + kColOff, d.ldp));
    if (u0.x != v0.x) {
        const bool pair_once = !rev || u < v;
        evaluated |= edge_pair<TW, OR>(d, u, v, true, pair_once, u0, u1, u2, u3, u4, u5, u6, v0, v1, v2, v4, v5, t,
                                       best, bidx);
    }
}

template <bool TW, bool OR, int R>
__device__ __forceinline__ void edge_depot_tile(const Dev &d, int p0, int r, bool active, int &best, unsigned &bidx,
                                                unsigned *cnt) {
    __shared__ int4 sU[R * 7];          // ERec g0..g6 of the anchors at positions p0 .. p0+R-1
    __shared__ int sA[R];               // those anchors (W past the sequence)
    __shared__ __align__(16) int sC0[R + 4];   // c(0, node at p0 + i)
    const int tid = threadIdx.x, nt = blockDim.x;
    // columns p0 .. p0+R+3 of a copy row, in int4 pieces; a piece is read
    // only while it starts at or before position Wp (every row that holds a
    // customer reads columns up to its position + 2 <= Wp)
    const int pieces = (R + 4) / 4;
    for (int i = tid; i < R * 7; i += nt) {
        const int row = i / 7, g = i - row * 7;
        const int p = p0 + row;
        const int a = p < d.Wp ? d.seq[TGA_IX(p, d.Wp)] : d.W;
        if (g == 0) sA[row] = a;
        sU[i] = __ldg(reinterpret_cast<const int4 *>(d.erec + TGA_IX(a, d.W + 1)) + g);
    }
    for (int j = tid; j < pieces; j += nt) {
        const int4 x = (4 * j <= d.Wp - p0) ? __ldg(reinterpret_cast<const int4 *>(d.pcol + TGA_IX(p0 + kColOff + 4 * j, d.ldp - 3)))
                                            : make_int4(0, 0, 0, 0);
        reinterpret_cast<int4 *>(sC0)[j] = x;
    }
    const int4 z = make_int4(0, 0, 0, 0);
    int4 v0 = z, v1 = z, v2 = z, v4 = z, v5 = z;
    int T[R + 4];
    const int v = d.n + 1 + r;
    if (active) {
        const int4 *vr = reinterpret_cast<const int4 *>(d.erec + TGA_IX(v, d.W + 1));
        v0 = __ldg(vr + 0); v1 = __ldg(vr + 1); v2 = __ldg(vr + 2);
        if (TW) { v4 = __ldg(vr + 4); v5 = __ldg(vr + 5); }
        const int f = __ldg(vr + 7).z;                       // first customer of route r (0: empty)
        const int *row = d.pcol + (size_t)TGA_IX(f, d.n + 1) * d.ldp;
#pragma unroll
        for (int j = 0; j < (R + 4) / 4; ++j) {
            const int4 x = (4 * j <= d.Wp - p0)
                               ? __ldg(reinterpret_cast<const int4 *>(row + TGA_IX(p0 + kColOff + 4 * j, d.ldp - 3)))
                               : z;
            T[4 * j] = x.x; T[4 * j + 1] = x.y; T[4 * j + 2] = x.z; T[4 * j + 3] = x.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < R + 4; ++j) T[j] = 0;
    }
    __syncthreads();
    if (!active) return;
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int a = sA[i];
        if (a < 1 || a > d.n) continue;                      // a start depot or past the sequence
        const int4 u0 = sU[i * 7];
        if (u0.x == r) continue;                             // v's own route
        const int4 u1 = sU[i * 7 + 1], u2 = sU[i * 7 + 2];
        const int4 u3 = OR ? sU[i * 7 + 3] : z;
        const int4 u4 = TW ? sU[i * 7 + 4] : z, u5 = TW ? sU[i * 7 + 5] : z;
        const int4 u6 = (TW && OR) ? sU[i * 7 + 6] : z;
        EdgeStencil t;
        t.t00 = sC0[i];                                      // c(u, 0)
        t.t10 = sC0[i + 1];                                  // c(u+, 0)
        t.t01 = T[i];                                        // c(u, f)
        t.t11 = T[i + 1];                                    // c(u+, f)
        t.t21 = T[i + 2];                                    // c(u++, f)
        t.tm10 = 0;
        t.t0m1 = 0;
        const unsigned ev = edge_pair<TW, OR>(d, a, v, false, false, u0, u1, u2, u3, u4, u5, u6, v0, v1, v2, v4,
                                              v5, t, best, bidx);
#pragma unroll
        for (int op = 0; op < 6; ++op) cnt[op] += (ev >> op) & 1u;
    }
}

// nmask: CTAs of mask entries; chunks: start-depot chunks of dc depots per
// row tile of R positions.
template <bool TW, bool OR, int R>
__global__ void __launch_bounds__(kEdgeMaxThreads) k_eval_edges(Dev d, int nmask, int chunks, int dc, int tail) {
    const int done = *(volatile int *)&d.ctl->done;
    int best = kBestInit;
    unsigned bidx = 0xffffffffu;
    unsigned cnt[6] = {0, 0, 0, 0, 0, 0};
    if ((int)blockIdx.x < nmask) {
        const long long item = (long long)blockIdx.x * blockDim.x + threadIdx.x;
        unsigned ev = 0;
        if (item < (long long)d.n * d.theta) edge_mask_item<TW, OR>(d, item, best, bidx, ev);
#pragma unroll
        for (int op = 0; op < 6; ++op) cnt[op] = (ev >> op) & 1u;
    } else {
        const int b = (int)blockIdx.x - nmask;
        const int tile = b / chunks, ch = b - tile * chunks;
        const int r = ch * dc + (int)threadIdx.x;
        edge_depot_tile<TW, OR, R>(d, tile * R, r, (int)threadIdx.x < dc && r < d.m, best, bidx, cnt);
    }
    if (done) return;
#pragma unroll
    for (int op = 0; op < 6; ++op) {
        const unsigned c = __reduce_add_sync(0xffffffffu, cnt[op]);
        if ((threadIdx.x & 31) == 0 && c) atomicAdd(&d.ctl->gcount[op], (unsigned long long)c);
    }
    const unsigned long long key = (bidx != 0xffffffffu) ? pack_key(best, bidx) : kNoKey;
    block_min_to(key, &d.ctl->best_key);
    if (tail && threadIdx.x == 0) eval_tail(d, tail);
}

// Mask rows of the edge-based extraction: every entry must be another
// customer; rev marks entries whose reverse entry exists.
__global__ void k_granular_setup(Dev d, unsigned char *rev, int *bad) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)d.n * d.theta) return;
    const int u = (int)(t / d.theta) + 1;
    const int v = d.nbr[TGA_IX((size_t)u * d.theta + (t - (long long)(u - 1) * d.theta), (long long)(d.n + 1) * d.theta)];
    unsigned char r = 0;
    if (v < 1 || v > d.n || v == u) {
        atomicExch(bad, 1);
    } else {
        for (int k = 0; k < d.theta; ++k)
            if (d.nbr[TGA_IX((size_t)v * d.theta + k, (long long)(d.n + 1) * d.theta)] == u) r = 1;
    }
    rev[(size_t)u * d.theta + (t - (long long)(u - 1) * d.theta)] = r;
}

// VRPTW intra-route moves: one block of kIntraWarps warps per route
// (subsequence tables in kIntraTabSmemInts ints of dynamic shared memory;
// kIntraTabSmemIntsPD with pickups).
template <bool PD, bool XS>
__global__ void __launch_bounds__(kIntraWarps * 32) k_eval_intra(Dev d, int tail) {
    const int done = *(volatile int *)&d.ctl->done;
    extern __shared__ __align__(16) int smem[];
    int best = kBestInit;
    unsigned bidx = 0xffffffffu;
    intra_route_table<PD, XS>(d, blockIdx.x, smem, best, bidx);
    if (done) return;
    const unsigned long long key = (bidx != 0xffffffffu) ? pack_key(best, bidx) : kNoKey;
    block_min_to(key, &d.ctl->best_key);
    if (tail && threadIdx.x == 0) eval_tail(d, tail);
}

// CVRP intra-route moves: one warp per route (the route's distance block in
// shared memory, intra_cvrp_route) when routes are short on average (Dev
// cvrp_by_route); otherwise, and with the swaps of runs, one warp per moved
// customer (intra_cvrp_position).
template <bool XS>
__global__ void __launch_bounds__(256) k_eval_intra_cvrp(Dev d, int tail) {
    const int done = *(volatile int *)&d.ctl->done;
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int best = kBestInit;
    unsigned bidx = 0xffffffffu;
    if constexpr (XS) {
        intra_cvrp_position<XS>(d, wid, threadIdx.x & 31, best, bidx);
    } else {
        __shared__ int sD[8][32 * 33];
        __shared__ int sA[8][32];
        const int w = threadIdx.x >> 5;
        if (d.cvrp_by_route) intra_cvrp_route(d, wid, threadIdx.x & 31, sD[w], sA[w], best, bidx);
        else intra_cvrp_position<false>(d, wid, threadIdx.x & 31, best, bidx);
    }
    if (done) return;
    const unsigned long long key = (bidx != 0xffffffffu) ? pack_key(best, bidx) : kNoKey;
    block_min_to(key, &d.ctl->best_key);
    if (tail && threadIdx.x == 0) eval_tail(d, tail);
}

// Apply.  pre = 1 (descent steps): every CTA loads the plan the evaluation's
// last CTA decoded (no plan: the descent is over, nothing to do); CTA 0
// applies it and CTAs 1.. permute the columns of the position-ordered copy.
// pre = 0: CTA 0 decodes *ext (or the best key) and publishes the plan while
// the other CTAs wait for it.  The last CTA to finish re-arms the plan flag
// for the next step.
template <bool PD, bool XS>
__global__ void __launch_bounds__(512) k_apply(Dev d, const tga_move *ext, cudaGraphConditionalHandle cond,
                                               int use_cond, int pre) {
    extern __shared__ __align__(16) int smem[];
    __shared__ StepPlan sP;
    __shared__ int s_ok;
    Control *C = d.ctl;
    const int tid = threadIdx.x;
    if (pre) {
        if (tid == 0) s_ok = *(volatile int *)&C->plan_ready;
        load_plan(C, &sP);                       // same round trip as the flag
        __syncthreads();
        if (!s_ok && tid == 0) sP.act = 0;
        __syncthreads();
        if (blockIdx.x == 0) apply_plan_block<PD, XS>(d, sP, smem, false, cond, use_cond);
        else band_plan_rows(d, sP, smem, 0, d.n + 1, blockIdx.x - 1, gridDim.x - 1);
    } else if (blockIdx.x == 0) {
        if (tid == 0) {
            decode_plan(d, ext, sP);
            C->plan = sP;
            __threadfence();
            atomicExch(&C->plan_ready, 1);
        }
        __syncthreads();
        apply_plan_block<PD, XS>(d, sP, smem, ext != nullptr, cond, use_cond);
    } else {
        if (tid == 0) {
            s_ok = wait_flag(&C->plan_ready, wait_limit(d.wait_ns, kWaitApplyNs));
            if (!s_ok) set_status(C, TGA_ERR_TIMEOUT);
        }
        __syncthreads();
        if (s_ok) load_plan(C, &sP);
        else if (tid == 0) sP.act = 0;
        __syncthreads();
        band_plan_rows(d, sP, smem, 0, d.n + 1, blockIdx.x - 1, gridDim.x - 1);
    }
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(&C->plan_done, 1) == (int)gridDim.x - 1) {
            C->plan_done = 0;
            C->plan_ready = 0;
        }
    }
}

__global__ void k_sync_solution(Dev d) {
    sync_solution_range(d, blockIdx.x * (long long)blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x);
}

__global__ void k_finalize(Dev d, tga_move *out) {
    Control *C = d.ctl;
    const unsigned long long key = C->best_key;
    C->best_key = kNoKey;
    if (d.log && C->evals < d.log_cap) d.log[C->evals] = key;
    count_evaluation(d, C);
    tga_move m;
    if (key == kNoKey) {
        m.delta = 0; m.move_index = 0; m.op = -1; m.a = 0; m.b = 0; m.valid = 0;
    } else {
        const unsigned idx = (unsigned)(key & 0xffffffffu);
        const unsigned W = (unsigned)d.W, W2 = W * W;
        m.delta = key_delta(key); m.move_index = idx;
        m.op = (int)(idx / W2); m.a = (int)((idx % W2) / W); m.b = (int)(idx % W); m.valid = 1;
    }
    *out = m;
}

__global__ void k_begin(Dev d, long long max_steps) {
    Control *C = d.ctl;
    C->bar_count = 0;
    C->plan_seq = 0;
    C->eval_done = 0;
    C->plan_ready = 0;
    C->plan_done = 0;
    for (int op = 0; op < 6; ++op) C->gcount[op] = 0;
    if (C->status != 0 || !C->built) { C->done = 1; return; }
    C->done = 0;
    C->local_opt = 0;
    C->best_key = kNoKey;
    const long long lim = C->steps + max_steps;
    C->step_limit = lim < C->steps ? 0x7fffffffffffffffLL : lim;
}

// Swaps of runs between routes (op ranks 6, 7; Section 5.3.1 Swap with
// N1 in {1, 2}, N2 = 2).  The block stages kXswapRows rows (customer a at
// position p: its XRec, route and the nodes at p-1 .. p+2); thread q holds
// the column anchor b at position q.  For each row with a in another route
// than b, with t(r, c) = c(node at p+r, node at q+c) read from the
// position-ordered distance copy (contiguous over the threads):
//   rank 6, a alone <-> the run b b+:
//     route of a: prefix(a-) + (b b+) + suffix after a   links t(-1,0), t(1,1)
//     route of b: prefix(b-) + a + suffix after b+        links t(0,-1), t(0,2)
//   rank 7 (p < q), the runs a a+ <-> b b+:
//     route of a: prefix(a-) + (b b+) + suffix after a+  links t(-1,0), t(2,1)
//     route of b: prefix(b-) + (a a+) + suffix after b+  links t(0,-1), t(1,2)
// Intra-route exchanges are evaluated by the route kernels.
template <bool TW>
__global__ void __launch_bounds__(kXswapThreads) k_eval_xswap(Dev d, int tail) {
    const int done = *(volatile int *)&d.ctl->done;
    __shared__ int s_node[kXswapRows + 3], s_anc[kXswapRows], s_rt[kXswapRows];
    __shared__ XRec s_xr[kXswapRows];
    const int ncb = (d.Wp + kXswapThreads - 1) / kXswapThreads;
    const int rb = blockIdx.x / ncb, cb = blockIdx.x - rb * ncb;
    const int p0 = rb * kXswapRows, tid = threadIdx.x;
    if (tid < kXswapRows + 3) {
        const int pp = p0 - 1 + tid;
        s_node[tid] = (pp >= 0 && pp < d.Wp) ? node_of(d.seq[TGA_IX(pp, d.Wp)], d.n) : 0;
    }
    if (tid < kXswapRows) {
        const int p = p0 + tid;
        const int a = p < d.Wp ? d.seq[TGA_IX(p, d.Wp)] : d.W;
        const bool cust = a >= 1 && a <= d.n;
        s_anc[tid] = cust ? a : 0;
        s_rt[tid] = cust ? d.brec[TGA_IX(a, d.W + 1)].route : -1;
        s_xr[tid] = cust ? d.xrec[TGA_IX(a, d.W + 1)] : xrec_none();
    }
    const int q = cb * kXswapThreads + tid;
    const int b = q < d.Wp ? d.seq[TGA_IX(q, d.Wp)] : d.W;
    const bool bcust = b >= 1 && b <= d.n;
    const XRec xb = bcust ? d.xrec[TGA_IX(b, d.W + 1)] : xrec_none();
    const int Br = bcust ? d.brec[TGA_IX(b, d.W + 1)].route : -2;
    __syncthreads();
    int best = kBestInit;
    unsigned bidx = 0xffffffffu;
    if (bcust && xb.S2 < (kBig >> 1)) {       // both ranks need the run b b+
        const unsigned mask = d.op_mask;
        const unsigned W = (unsigned)d.W, W2 = W * W;
        const int wL = d.wL, wT = d.wT;
        const int *pc = d.pcol + kColOff + TGA_IX(q, d.Wp + 4);
        const size_t ldp = (size_t)d.ldp;
#pragma unroll 2
        for (int i = 0; i < kXswapRows; ++i) {
            const int a = s_anc[i];
            if (a == 0 || s_rt[i] == Br) continue;
            const XRec xa = s_xr[i];
            const int am = s_node[i], ap = s_node[i + 2], app = s_node[i + 3];
            const int c_amb = TGA_LDG(pc + (size_t)am * ldp);            // c(a-, b)
            const int c_abm = TGA_LDG(pc + (size_t)a * ldp - 1);         // c(a, b-)
            if (mask & 64u) {
                const int c_apb1 = TGA_LDG(pc + (size_t)ap * ldp + 1);   // c(a+, b+1)
                const int c_ab2 = TGA_LDG(pc + (size_t)a * ldp + 2);     // c(a, b+2)
                int dl = xa.S1 + c_amb + xb.RC2 + c_apb1 + xb.S2 + c_abm + c_ab2 +
                         wL * (max(xa.LQd1 + xb.ld2, 0) + max(xb.LQd2 + xa.d, 0));
                if (TW) {
                    const int x1 = xa.tauP + c_amb, w1 = max(x1 - xb.L2, 0);
                    const int x2 = max(x1, xb.E2) - w1 + xb.Dm2 + c_apb1, w2 = max(x2 - xa.Lg1, 0);
                    const int y1 = xb.tauP + c_abm, v1 = max(y1 - xa.l, 0);
                    const int y2 = max(y1, xa.e) - v1 + xa.s + c_ab2, v2 = max(y2 - xb.Lg2, 0);
                    dl += wT * (w1 + w2 + v1 + v2);
                }
                TGA_TRY(dl, 6u * W2 + (unsigned)a * W + (unsigned)b);
            }
            if ((mask & 128u) && p0 + i < q && xa.S2 < (kBig >> 1)) {
                const int c_appb1 = TGA_LDG(pc + (size_t)app * ldp + 1); // c(a+2, b+1)
                const int c_apb2 = TGA_LDG(pc + (size_t)ap * ldp + 2);   // c(a+1, b+2)
                int dl = xa.S2 + c_amb + xb.RC2 + c_appb1 + xb.S2 + c_abm + xa.RC2 + c_apb2 +
                         wL * (max(xa.LQd2 + xb.ld2, 0) + max(xb.LQd2 + xa.ld2, 0));
                if (TW) {
                    const int x1 = xa.tauP + c_amb, w1 = max(x1 - xb.L2, 0);
                    const int x2 = max(x1, xb.E2) - w1 + xb.Dm2 + c_appb1, w2 = max(x2 - xa.Lg2, 0);
                    const int y1 = xb.tauP + c_abm, v1 = max(y1 - xa.L2, 0);
                    const int y2 = max(y1, xa.E2) - v1 + xa.Dm2 + c_apb2, v2 = max(y2 - xb.Lg2, 0);
                    dl += wT * (w1 + w2 + v1 + v2);
                }
                TGA_TRY(dl, 7u * W2 + (unsigned)min(a, b) * W + (unsigned)max(a, b));
            }
        }
    }
    if (done) return;
    const unsigned long long key = (bidx != 0xffffffffu) ? pack_key(best, bidx) : kNoKey;
    block_min_to(key, &d.ctl->best_key);
    if (tail && threadIdx.x == 0) eval_tail(d, tail);
}

// ---------------------------------------------------------------------------
// host-side launchers

size_t inter_smem_bytes(int rows, int warps, bool pd) {
    const int LDT = warps * 32 + 8;
    return (size_t)(rows + 4) * LDT * sizeof(int) + (size_t)rows * (sizeof(ERec) + (pd ? sizeof(PRec) : 0));
}

namespace {
using InterFn = void (*)(Dev, int, int, int);
using StripFn = void (*)(Dev, int, long long, int);

template <bool G>
InterFn inter_fn_g(bool tw, bool orr, bool pd) {
    if (pd) return orr ? k_eval_inter<true, true, true, G> : k_eval_inter<true, false, true, G>;
    if (tw) return orr ? k_eval_inter<true, true, false, G> : k_eval_inter<true, false, false, G>;
    return orr ? k_eval_inter<false, true, false, G> : k_eval_inter<false, false, false, G>;
}
template <bool G>
StripFn strip_fn_g(bool tw, bool orr, bool pd) {
    if (pd) return orr ? k_eval_strip<true, true, true, G> : k_eval_strip<true, false, true, G>;
    if (tw) return orr ? k_eval_strip<true, true, false, G> : k_eval_strip<true, false, false, G>;
    return orr ? k_eval_strip<false, true, false, G> : k_eval_strip<false, false, false, G>;
}

// Whether the operator mask leaves out an inter-route operator that the
// kernel variant evaluates (relocate, swap, 2-opt*, and the or-opts in the
// or-opt variants): those launches take the gated kernels, which skip the
// disabled operators' arithmetic.
bool inter_gated(const Dev &d) {
    const unsigned ops = 0x0Bu | ((d.op_mask & 48u) ? 0x30u : 0u);
    return (d.op_mask & ops) != ops;
}

InterFn inter_fn(const Dev &d) {
    const bool tw = d.has_tw != 0, orr = (d.op_mask & 48u) != 0, pd = d.has_pd != 0;
    return inter_gated(d) ? inter_fn_g<true>(tw, orr, pd) : inter_fn_g<false>(tw, orr, pd);
}
StripFn strip_fn(const Dev &d) {
    const bool tw = d.has_tw != 0, orr = (d.op_mask & 48u) != 0, pd = d.has_pd != 0;
    return inter_gated(d) ? strip_fn_g<true>(tw, orr, pd) : strip_fn_g<false>(tw, orr, pd);
}
}  // namespace

// Any inter-route operator enabled (relocate, swap, 2-opt*, or-opt)?  Without
// one the inter-route launch is left out of the evaluation.
bool has_inter_ops(const Dev &d) { return (d.op_mask & 0x3Bu) != 0; }

int setup_kernel_attrs(int max_band) {
    const int big = 200 * 1024;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 16 && e == cudaSuccess; ++k) {
        const bool tw = (k & 1) != 0, orr = (k & 2) != 0, pd = (k & 4) != 0, g = (k & 8) != 0;
        if (pd && !tw) continue;                               // pickups come with time windows
        const void *fi = g ? (const void *)inter_fn_g<true>(tw, orr, pd) : (const void *)inter_fn_g<false>(tw, orr, pd);
        const void *fs = g ? (const void *)strip_fn_g<true>(tw, orr, pd) : (const void *)strip_fn_g<false>(tw, orr, pd);
        e = cudaFuncSetAttribute(fi, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(fs, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    }
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_apply<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_apply<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_apply<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    (void)max_band;
    return e == cudaSuccess ? 0 : 1;
}

void launch_check_instance(const Dev &d, cudaStream_t s) {
    const long long nt = (d.n + 1 + 31) / 32;
    long long blocks = nt * nt;
    if (blocks > (long long)d.nsm * 16) blocks = (long long)d.nsm * 16;
    k_check_instance<<<(int)blocks, 256, 0, s>>>(d);
}

void launch_build(const Dev &d, cudaStream_t s) {
    cudaMemsetAsync(d.seen, 0, sizeof(int) * (d.n + 1), s);
    k_build_positions<<<(d.m + 127) / 128, 128, 0, s>>>(d);
    k_check_perm<<<(d.n + 255) / 256, 256, 0, s>>>(d);
    k_build_routes<<<(d.m * 32 + 127) / 128, 128, 0, s>>>(d);
    k_build_finish<<<1, 1024, 0, s>>>(d);
    long long tot = (long long)(d.n + 1) * d.ldp;
    long long blocks = (tot + 255) / 256;
    if (blocks > (long long)d.nsm * 32) blocks = (long long)d.nsm * 32;
    k_pcol_init<<<(int)blocks, 256, 0, s>>>(d);
}

// Launch shape of the edge-based extraction: threads per CTA (a multiple of
// 32, at most kEdgeMaxThreads), the mask CTAs (one thread per entry), and the
// depot CTAs: row tiles of R positions (R the largest of 32, 16, 8 that still
// gives about eight CTAs per SM, else 8) times chunks of dc start depots.
EdgeGrid edge_grid(const Dev &d) {
    EdgeGrid g{};
    const int chunks = (d.m + kEdgeMaxThreads - 1) / kEdgeMaxThreads;
    g.chunks = chunks < 1 ? 1 : chunks;
    g.dc = (d.m + g.chunks - 1) / g.chunks;
    if (g.dc < 1) g.dc = 1;
    g.threads = (g.dc + 31) / 32 * 32;
    const long long entries = (long long)d.n * d.theta;
    g.nmask = (int)((entries + g.threads - 1) / g.threads);
    const int rows_pos = d.Wp - 1;                    // positions 0 .. Wp-2 (the sentinel holds no customer)
    g.rows = 8;
    for (int R = 32; R >= 16; R >>= 1)
        if ((long long)((rows_pos + R - 1) / R) * g.chunks >= 8LL * d.nsm) { g.rows = R; break; }
    g.ndepot = ((rows_pos + g.rows - 1) / g.rows) * g.chunks;
    return g;
}

size_t strip_smem_bytes(int rows, int warps, bool pd) {
    const int LDT = warps * 32 + 8;
    const size_t buf = (size_t)(rows + 4) * LDT * sizeof(int) + (size_t)rows * (pd ? 12 : 8) * 16;
    return 2 * buf + 2 * (size_t)(rows + 4) * sizeof(int);
}


int strip_grid(const Dev &d, int rows, int warps, long long ntiles) {
    if (!(rows == 16 || rows == 32) || !(warps == 4 || warps == 8) || ntiles <= 0) return 0;
    const size_t sm = strip_smem_bytes(rows, warps, d.has_pd != 0);
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, (const void *)strip_fn(d), warps * 32, sm) != cudaSuccess || per < 1) {
        cudaGetLastError();
        return 0;
    }
    const long long g = (long long)per * d.nsm;
    return (int)(g < ntiles ? g : ntiles);
}

void launch_inter(const Dev &d, const int2 *tiles, int ntiles, int rows, int warps, cudaStream_t s, int rs,
                  int tail, int strip) {
    if (!has_inter_ops(d)) return;
    if (d.theta > 0) {          // edge-based extraction
        const EdgeGrid g = edge_grid(d);
        const bool orr = (d.op_mask & 48u) != 0;
        const int blocks = g.nmask + g.ndepot;
#define TGA_EDGES(R)                                                                                        \
    do {                                                                                                    \
        if (d.has_tw) {                                                                                     \
            if (orr) k_eval_edges<true, true, R><<<blocks, g.threads, 0, s>>>(d, g.nmask, g.chunks, g.dc, tail); \
            else k_eval_edges<true, false, R><<<blocks, g.threads, 0, s>>>(d, g.nmask, g.chunks, g.dc, tail); \
        } else {                                                                                            \
            if (orr) k_eval_edges<false, true, R><<<blocks, g.threads, 0, s>>>(d, g.nmask, g.chunks, g.dc, tail); \
            else k_eval_edges<false, false, R><<<blocks, g.threads, 0, s>>>(d, g.nmask, g.chunks, g.dc, tail); \
        }                                                                                                   \
    } while (0)
        if (g.rows == 8) TGA_EDGES(8);
        else if (g.rows == 16) TGA_EDGES(16);
        else TGA_EDGES(32);
#undef TGA_EDGES
        return;
    }
    if (ntiles <= 0) return;
    if (strip > 0) {            // strip-major kernel: TC = 32 * warps columns, one row group
        const size_t sm = strip_smem_bytes(rows, warps, d.has_pd != 0);
        strip_fn(d)<<<strip, warps * 32, sm, s>>>(d, rows, ntiles, tail);
        return;
    }
    const size_t sm = inter_smem_bytes(rows, warps, d.has_pd != 0);
    inter_fn(d)<<<ntiles, warps * 32 * rs, sm, s>>>(d, rows, rs, tail);
}

// VRPTW: one block per route; CVRP: one warp per route (8 per block), or one
// warp per moved position (long routes, or the swaps of runs).
int intra_blocks(const Dev &d) {
    if (d.has_tw) return d.m;
    return d.cvrp_by_route ? (d.m + 7) / 8 : (d.Wp - 1 + 7) / 8;
}

int xswap_blocks(const Dev &d);

int eval_blocks(const Dev &d, int ntiles, int strip) {
    if (d.theta > 0) {
        const EdgeGrid g = edge_grid(d);
        return (has_inter_ops(d) ? g.nmask + g.ndepot : 0) + intra_blocks(d);
    }
    const int inter = (ntiles <= 0 || !has_inter_ops(d)) ? 0 : (strip > 0 ? strip : ntiles);
    return inter + intra_blocks(d) + xswap_blocks(d);
}

void launch_granular_setup(const Dev &d, unsigned char *rev, int *bad_dev, cudaStream_t s) {
    const long long t = (long long)d.n * d.theta;
    if (t <= 0) return;
    k_granular_setup<<<(int)((t + 255) / 256), 256, 0, s>>>(d, rev, bad_dev);
}

void launch_intra(const Dev &d, cudaStream_t s, int tail) {
    const bool xs = (d.op_mask & kExtOps) != 0;
    const size_t tab = kIntraTabSmemInts * sizeof(int);
    if (d.has_pd)
        k_eval_intra<true, false><<<intra_blocks(d), kIntraWarps * 32, kIntraTabSmemIntsPD * sizeof(int), s>>>(d, tail);
    else if (d.has_tw && xs) k_eval_intra<false, true><<<intra_blocks(d), kIntraWarps * 32, tab, s>>>(d, tail);
    else if (d.has_tw) k_eval_intra<false, false><<<intra_blocks(d), kIntraWarps * 32, tab, s>>>(d, tail);
    else if (xs) k_eval_intra_cvrp<true><<<intra_blocks(d), 256, 0, s>>>(d, tail);
    else k_eval_intra_cvrp<false><<<intra_blocks(d), 256, 0, s>>>(d, tail);
}

// Swaps of runs between routes: the block walks kXswapRows row positions,
// one thread per column position.
int xswap_blocks(const Dev &d) {
    if (!(d.op_mask & kExtOps)) return 0;
    return ((d.Wp + kXswapRows - 1) / kXswapRows) * ((d.Wp + kXswapThreads - 1) / kXswapThreads);
}

void launch_xswap(const Dev &d, cudaStream_t s, int tail) {
    const int blocks = xswap_blocks(d);
    if (blocks <= 0) return;
    if (d.has_tw) k_eval_xswap<true><<<blocks, kXswapThreads, 0, s>>>(d, tail);
    else k_eval_xswap<false><<<blocks, kXswapThreads, 0, s>>>(d, tail);
}

void launch_eval(const Dev &d, const int2 *tiles, int ntiles, int rows, int warps, cudaStream_t s, int rs,
                 int tail, int strip) {
    launch_inter(d, tiles, ntiles, rows, warps, s, rs, tail, strip);
    launch_intra(d, s, tail);
    launch_xswap(d, s, tail);
}

int apply_grid(const Dev &d) {
    const int rows = (d.n + 1 + 15) / 16;           // a warp per row, 16 warps per CTA
    return 1 + (rows < 3 * d.nsm ? rows : 3 * d.nsm);
}

void launch_apply(const Dev &d, const tga_move *ext, unsigned long long cond, int use_cond, cudaStream_t s,
                  int pre) {
    const size_t sm = (size_t)band_smem_ints(d.Wp, 16) * sizeof(int);
    const auto h = (cudaGraphConditionalHandle)cond;
    if (d.has_pd) k_apply<true, false><<<apply_grid(d), 512, sm, s>>>(d, ext, h, use_cond, pre);
    else if (d.op_mask & kExtOps) k_apply<false, true><<<apply_grid(d), 512, sm, s>>>(d, ext, h, use_cond, pre);
    else k_apply<false, false><<<apply_grid(d), 512, sm, s>>>(d, ext, h, use_cond, pre);
}

void launch_sync_solution(const Dev &d, cudaStream_t s) {
    int blocks = (d.Wp + 255) / 256;
    if (blocks > d.nsm * 4) blocks = d.nsm * 4;
    k_sync_solution<<<blocks, 256, 0, s>>>(d);
}

void launch_finalize(const Dev &d, tga_move *out, cudaStream_t s) { k_finalize<<<1, 1, 0, s>>>(d, out); }

void launch_begin(const Dev &d, long long max_steps, cudaStream_t s) { k_begin<<<1, 1, 0, s>>>(d, max_steps); }

}  // namespace tga
